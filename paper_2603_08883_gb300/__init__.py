"""GB300-native iQCC dressing path (arXiv 2603.08883).

The CUDA library and its binding live in :mod:`paper_2603_08883_gb300.iqcc`;
seeded synthetic inputs in :mod:`paper_2603_08883_gb300.synth`.  Importing the
package itself loads nothing compiled.
"""
__all__ = ["iqcc", "synth"]

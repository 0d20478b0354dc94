"""GB300-native iQCC dressing path (arXiv 2603.08883).

* :mod:`paper_2603_08883_gb300.iqcc`: the CUDA library's binding (C ABI of
  ``include/iqcc.h``, same names); no CPU fallback.
* :mod:`paper_2603_08883_gb300.autograd`: the dressed QMF energy as a
  ``torch.autograd.Function`` over the library's adjoint kernel.
* :mod:`paper_2603_08883_gb300.partitioned`: a Hamiltonian split by key bits
  over several contexts, with the row exchange of a crossing generator.
* :mod:`paper_2603_08883_gb300.screening`: the learned term-screening model
  and its training.
* :mod:`paper_2603_08883_gb300.synth`: seeded synthetic inputs.

Importing the package itself loads nothing compiled.
"""
__all__ = ["autograd", "iqcc", "partitioned", "screening", "synth"]

"""The reference arm of bench.py (the oracle on host cores) measures a
non-empty sample: its first strings of the 100-qubit workload must yield DIS
candidates and dressed terms."""
import bench
from paper_2603_08883_gb300 import synth


def test_reference_sample_dresses_terms():
    w = synth.WORKLOADS["jw100"]
    n, x, z, c = synth.workload_hamiltonian(w)
    th, ph = synth.workload_angles(w)
    dressed, seconds = bench.oracle_dressed(w, n, x, z, c, th, ph, bench.REFERENCE_ROWS)
    assert dressed > 0 and seconds > 0

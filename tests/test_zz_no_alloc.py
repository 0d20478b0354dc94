"""The energy entry point that allocates no device memory.

Callers that cannot allocate at the moment they need an energy (while
recording a CUDA stream capture, inside a framework that owns all device
memory, or in a service with a fixed footprint) call
iqcc_qmf_energy_noalloc on rows they already hold on the device; its scratch
is a fixed array inside the library.  These tests call it through the C ABI,
twice in a row (the scratch keeps the previous call's contents), and compare
it with iqcc_qmf_energy on the same Hamiltonian.
"""
import numpy as np
import pytest

from paper_2603_08883_gb300 import synth

pytestmark = pytest.mark.gpu

iqcc = pytest.importorskip("paper_2603_08883_gb300.iqcc")
torch = pytest.importorskip("torch")

ENERGY_TOL = 1e-9   # Ha, the energy tolerance of the parity tests


def _device_rows(n, x, z, c):
    """Rows in the entry point's layout: x words then z words, Wd = 1, 2 or 4."""
    W = x.shape[1]
    Wd = 1 if n <= 64 else (2 if n <= 128 else 4)
    rows = np.zeros((len(c), 2 * Wd), np.uint64)
    rows[:, :W] = x
    rows[:, Wd:Wd + W] = z
    d_rows = torch.from_numpy(rows.view(np.int64)).cuda()
    d_coef = torch.from_numpy(np.ascontiguousarray(c)).cuda()
    return d_rows, d_coef


@pytest.mark.parametrize("n,angles", [(24, "basis"), (24, "uniform"), (100, "basis"), (100, "uniform"),
                                      (200, "uniform")])
def test_energy_without_allocation_matches_iqcc_qmf_energy(n, angles):
    _, x, z, c = synth.random_hamiltonian(n, 40_000, 1000 + n, density=0.3)
    x[: len(x) // 3] = 0                            # diagonal strings: non-zero basis-state energy
    th, ph = synth.qmf_angles(n, angles, n)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    want = iqcc.iqcc_qmf_energy(H, th, ph)
    H.close()
    d_rows, d_coef = _device_rows(n, x, z, c)
    torch.cuda.synchronize()
    for _ in range(2):
        got = iqcc.iqcc_qmf_energy_noalloc(n, d_rows, d_coef, len(c), th, ph)
        assert got == pytest.approx(want, abs=ENERGY_TOL)


def test_energy_without_allocation_rejects_sizes_beyond_its_scratch():
    d_rows, d_coef = _device_rows(8, np.zeros((1, 1), np.uint64), np.zeros((1, 1), np.uint64), np.ones(1))
    with pytest.raises(iqcc.IqccError) as e:
        iqcc.iqcc_qmf_energy_noalloc(300, d_rows, d_coef, 1, np.zeros(300), np.zeros(300))
    assert e.value.status == 1
    assert "256" in iqcc.iqcc_last_error()

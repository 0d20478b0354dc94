"""The energy entry point that allocates no device memory.

Callers that cannot allocate at the moment they need an energy (a plug-in
whose host framework owns all device memory through its own allocator, or a
service that must keep a fixed footprint once started) call
iqcc_qmf_energy_noalloc on rows they already hold on the device; its scratch
is a fixed array inside the library.  These tests call it through the C ABI,
twice in a row (the scratch keeps the previous call's contents), and compare
it with the CPU oracle's energy and with iqcc_qmf_energy on the same
Hamiltonian.  They also check that the calls leave the device's free memory
unchanged, and that a call on a stream being captured is refused without
breaking the capture (the call synchronises its stream).

This file is collected last, so a run that stops at the first failure has run
every other test before it.
"""
import numpy as np
import pytest

import oracle
from paper_2603_08883_gb300 import synth

pytestmark = pytest.mark.gpu

iqcc = pytest.importorskip("paper_2603_08883_gb300.iqcc", exc_type=ImportError)
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
                                      (200, "uniform"), (256, "uniform")])
def test_energy_without_allocation_matches_the_oracle(n, angles):
    m = 40_000 if angles == "basis" else 8_000
    _, x, z, c = synth.random_hamiltonian(n, m, 1000 + n, density=0.3)
    x[: len(x) // 3] = 0                            # diagonal strings: non-zero basis-state energy
    th, ph = synth.qmf_angles(n, angles, n)
    want = oracle.Oracle(n, x, z, c).energy(th, ph)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    lib = iqcc.iqcc_qmf_energy(H, th, ph)
    H.close()
    assert lib == pytest.approx(want, abs=ENERGY_TOL)
    d_rows, d_coef = _device_rows(n, x, z, c)
    # the first call may have the CUDA runtime load the library's kernels and
    # fixed array onto the device (lazy module loading); later calls must not
    # change the free device memory at all
    got = iqcc.iqcc_qmf_energy_noalloc(n, d_rows, d_coef, len(c), th, ph)
    assert got == pytest.approx(want, abs=ENERGY_TOL)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        got = iqcc.iqcc_qmf_energy_noalloc(n, d_rows, d_coef, len(c), th, ph)
        assert got == pytest.approx(want, abs=ENERGY_TOL)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_energy_without_allocation_rejects_sizes_beyond_its_scratch():
    d_rows, d_coef = _device_rows(8, np.zeros((1, 1), np.uint64), np.zeros((1, 1), np.uint64), np.ones(1))
    with pytest.raises(iqcc.IqccError) as e:
        iqcc.iqcc_qmf_energy_noalloc(300, d_rows, d_coef, 1, np.zeros(300), np.zeros(300))
    assert e.value.status == 1
    assert "256" in iqcc.iqcc_last_error()


def test_energy_without_allocation_refuses_a_capturing_stream():
    n = 24
    _, x, z, c = synth.random_hamiltonian(n, 1000, 5, density=0.3)
    d_rows, d_coef = _device_rows(n, x, z, c)
    th, ph = synth.qmf_angles(n, "basis")
    want = iqcc.iqcc_qmf_energy_noalloc(n, d_rows, d_coef, len(c), th, ph)
    s = torch.cuda.Stream()
    static = torch.zeros(16, device="cuda")
    g = torch.cuda.CUDAGraph()
    refused = None
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            static.add_(1.0)
            try:
                iqcc.iqcc_qmf_energy_noalloc(n, d_rows, d_coef, len(c), th, ph, stream=s)
            except iqcc.IqccError as e:
                refused = e
    assert refused is not None and refused.status == 1
    assert "captured" in str(refused)
    g.replay()                                      # the capture survived the refused call
    torch.cuda.synchronize()
    assert float(static[0]) == 1.0
    assert iqcc.iqcc_qmf_energy_noalloc(n, d_rows, d_coef, len(c), th, ph) == pytest.approx(want, abs=ENERGY_TOL)

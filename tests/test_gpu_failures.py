"""Failure paths of the device code, made to happen without faulting the GPU.

* Every device wait (the DIS grouping's wait for a published group key, the
  stable compactions' decoupled look-back) polls a bounded number of times,
  then records IQCC_ERR_TIMEOUT and returns; the call fails with that status
  and the context refuses every later call (IQCC_ERR_STATE).  The self-test
  waits on a word that nothing writes; a one-poll limit on real work shows that
  every wait gives up and returns instead of hanging.
* A probe bound of one bucket in the batched screening's group table makes a
  crowded table overflow: IQCC_ERR_HASH_FULL, then IQCC_ERR_STATE.
In every case a fresh context on the same GPU still works.
"""
import numpy as np
import pytest

import oracle
from paper_2603_08883_gb300 import synth
from tests.compare import compare

pytestmark = pytest.mark.gpu

iqcc = pytest.importorskip("paper_2603_08883_gb300.iqcc", exc_type=ImportError)

TIMEOUT, HASH_FULL, STATE = 6, 5, 7


def _fresh_context_still_works():
    n = 12
    _, x, z, c = synth.random_hamiltonian(n, 500, 3)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    th, ph = synth.qmf_angles(n, "basis")
    assert iqcc.iqcc_qmf_energy(H, th, ph) == pytest.approx(oracle.Oracle(n, x, z, c).energy(th, ph), abs=1e-9)
    H.close()


def test_device_wait_on_a_word_nothing_writes_times_out():
    n = 10
    _, x, z, c = synth.random_hamiltonian(n, 100, 1)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    iqcc.iqcc_set_wait_limit(H, 1000)
    with pytest.raises(iqcc.IqccError) as e:
        iqcc.iqcc_wait_selftest(H)
    assert e.value.status == TIMEOUT
    assert "device error 6" in iqcc.iqcc_last_error(H)
    with pytest.raises(iqcc.IqccError) as e:
        iqcc.iqcc_qmf_energy(H, np.zeros(n), np.zeros(n))
    assert e.value.status == STATE
    H.close()
    _fresh_context_still_works()


def test_default_wait_limit_is_restored_and_bounded():
    """With the default limit (2^24 polls) the self-test still gives up (about a second)."""
    n = 10
    _, x, z, c = synth.random_hamiltonian(n, 100, 2)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    iqcc.iqcc_set_wait_limit(H, 5)
    iqcc.iqcc_set_wait_limit(H, 0)
    with pytest.raises(iqcc.IqccError) as e:
        iqcc.iqcc_wait_selftest(H)
    assert e.value.status == TIMEOUT
    H.close()


def test_one_poll_waits_give_up_or_finish_correctly():
    """A one-poll wait limit on compression and dress of about 10^6 rows.
    Both copy rows out of place at offsets known per tile, so no block waits
    on another and both must finish with the right result; were a wait left
    in them, the call would have to fail with IQCC_ERR_TIMEOUT and leave the
    context refusing further calls.  Nothing hangs either way."""
    n = 40
    _, x, z, c = synth.random_hamiltonian(n, 1_200_000, 9, density=0.1)
    x[: len(x) // 2] &= np.uint64(0xF)             # few flip sets: many rows share a DIS group
    eps = float(np.quantile(np.abs(c), 0.5))
    P = (np.array([0b1011], np.uint64), np.array([0b0001], np.uint64))
    refs = {}
    for call in ("prune", "dress"):
        R = iqcc.iqcc_load_hamiltonian(n, x, z, c)     # the same call with the default limit
        if call == "prune":
            iqcc.iqcc_prune(R, eps)
        else:
            iqcc.iqcc_dress(R, P[0], P[1], [0.3])
        refs[call] = iqcc.iqcc_export(R)
        R.close()
    outcomes = []
    th, ph = synth.qmf_angles(n, "basis")
    for call in ("prune", "dress"):
        H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
        iqcc.iqcc_set_wait_limit(H, 1)
        try:
            if call == "prune":
                iqcc.iqcc_prune(H, eps)
            else:
                iqcc.iqcc_dress(H, P[0], P[1], [0.3])
            iqcc.iqcc_set_wait_limit(H, 0)
            assert not compare(iqcc.iqcc_export(H), refs[call])
            outcomes.append("ok")
        except iqcc.IqccError as e:
            assert e.status == TIMEOUT
            outcomes.append("timeout")
            with pytest.raises(iqcc.IqccError) as e2:
                iqcc.iqcc_qmf_energy(H, th, ph)
            assert e2.value.status == STATE
        H.close()
    print("one-poll outcomes:", outcomes)
    _fresh_context_still_works()


def test_group_table_full_then_context_refuses():
    """A one-bucket probe bound (max_probe = 1) on the batched screening's
    (flip set, problem) group table, with about 1.2 x 10^5 distinct groups:
    some buckets of the table overflow."""
    probs = []
    for k in range(4):
        n = 40
        _, x, z, c = synth.random_hamiltonian(n, 30_000, 40 + k, density=0.3)
        probs.append((n, x.reshape(-1), z.reshape(-1), c))
    batch = iqcc.iqcc_batch_load(probs, max_probe=1)
    th = [np.where(np.arange(n) < n // 2, np.pi, 0.0) for n, *_ in probs]
    ph = [np.zeros(n) for n, *_ in probs]
    with pytest.raises(iqcc.IqccError) as e:
        iqcc.iqcc_batch_screen(batch, th, ph)
    assert e.value.status == HASH_FULL
    with pytest.raises(iqcc.IqccError) as e:
        iqcc.iqcc_batch_screen(batch, th, ph)
    assert e.value.status == STATE
    batch.close()
    _fresh_context_still_works()


@pytest.mark.parametrize("n", [24, 100, 200])
def test_overflowing_fixed_bins_redo_the_dress_exactly(n):
    """Inside iqcc_iterate the dress bins are sized from the A,B,C pass's
    count.  With no slack (each bin holds exactly the mean), bins overflow and
    the dress is redone with exact bins: the iteration must end on the same
    Hamiltonian, bit for bit, as with the default slack (key words 1, 2, 4)."""
    _, x, z, c = synth.random_hamiltonian(n, 150_000, 61 + n, density=min(0.5, 15 / n))
    th, ph = synth.qmf_angles(n, "basis", seed=61 + n)
    out = []
    for slack in ((0.25, 32), (0.0, 0)):
        H = iqcc.iqcc_load_hamiltonian(n, x, z, c, capacity=1 << 24)
        iqcc.iqcc_set_bin_slack(H, *slack)
        iqcc.iqcc_reset_stats(H)
        iqcc.iqcc_iterate(H, th, ph, 4, 1e-10, 400_000)
        st = iqcc.iqcc_get_stats(H)
        out.append((iqcc.iqcc_export(H), st))
        H.close()
    (ref, st0), (got, st1) = out
    assert st0["fixed_bin_dresses"] > 0 and st0["bin_overflows"] == 0
    assert st1["bin_overflows"] > 0
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    with pytest.raises(iqcc.IqccError) as e:
        H = iqcc.iqcc_load_hamiltonian(n, x[:10], z[:10], c[:10])
        iqcc.iqcc_set_bin_slack(H, -0.1, 0)
    assert e.value.status == 1

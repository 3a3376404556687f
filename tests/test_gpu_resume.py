"""Resumable runs, checkpoints and cancellation (failure detection on the host).

A schedule split into several mp_run_sweeps calls, with a checkpoint, a new
handle and a restore in between, follows the same trajectories as one
uninterrupted run: the random numbers depend only on (seed, system, path,
sweep, site).  Cancellation is a host-side flag the kernels poll; nothing
faults or hangs.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1305_6758_gb300 as mp  # noqa: E402

SYSTEMS = [mp.System(8, 1.1, n_paths=40), mp.System(6, 0.8, h=0.05, n_paths=17),
           mp.System(24, 1.4, n_paths=3)]   # 24 is streamed in FP64
FIELDS = list(range(17))


def records(sim):
    return [sim.paths(k) for k in range(len(SYSTEMS))]


@pytest.mark.parametrize("precision,tol", [(mp.FP64, 1e-12), (mp.FP32, 1e-6)])
def test_split_schedule_with_checkpoint_equals_one_run(precision, tol):
    kw = dict(seed=6, precision=precision)
    with mp.Simulation(SYSTEMS, 5, 7, **kw) as whole:
        whole.run_sweeps(12)
        ref = records(whole)
        whole.run()  # the graph-replayed full run agrees too
        full = records(whole)
    with mp.Simulation(SYSTEMS, 5, 7, **kw) as a:
        a.run_sweeps(3)      # inside thermalisation
        a.run_sweeps(4)      # across the first measurement sweeps
        blob = a.checkpoint()
        assert a.progress() == 7
    with mp.Simulation(SYSTEMS, 5, 7, **kw) as b:
        b.restore(blob)
        assert b.progress() == 7
        b.run_sweeps(100)    # clipped to the end of the schedule
        assert b.progress() == 12
        got = records(b)
        with pytest.raises(mp.MPError) as ei:
            b.run_sweeps(1)
        assert ei.value.status == mp.MP_ESTATE
    for r, g, f in zip(ref, got, full):
        np.testing.assert_allclose(g[:, FIELDS], r[:, FIELDS], rtol=0, atol=tol)
        np.testing.assert_array_equal(g[:, 17], r[:, 17])
        np.testing.assert_allclose(f[:, FIELDS], r[:, FIELDS], rtol=0, atol=tol)


def test_ising_split_schedule_equals_one_run():
    """The same for the Appendix A kernel: spins are bytes, the trajectories
    integer, so the records agree up to the order of the FP64 sums."""
    systems = [mp.System(12, 2.2, n_paths=9, lattice=mp.ISING), mp.System(6, 1.5, h=0.2, n_paths=5, lattice=mp.ISING)]
    with mp.Simulation(systems, 4, 6, seed=8) as whole:
        whole.run_sweeps(10)
        ref = [whole.paths(k) for k in range(2)]
    with mp.Simulation(systems, 4, 6, seed=8) as a:
        a.run_sweeps(5)
        blob = a.checkpoint()
    with mp.Simulation(systems, 4, 6, seed=8) as b:
        b.restore(blob)
        b.run_sweeps(5)
        got = [b.paths(k) for k in range(2)]
    for r, g in zip(ref, got):
        np.testing.assert_allclose(g[:, FIELDS], r[:, FIELDS], rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(g[:, 17], r[:, 17])


def test_checkpoint_errors():
    with mp.Simulation(SYSTEMS, 2, 2) as a:
        with pytest.raises(mp.MPError) as ei:
            a.checkpoint()
        assert ei.value.status == mp.MP_ESTATE
        a.run_sweeps(2)
        blob = a.checkpoint()
    with mp.Simulation(SYSTEMS, 2, 3) as other:  # another schedule
        with pytest.raises(mp.MPError) as ei:
            other.restore(blob)
        assert ei.value.status == mp.MP_EINVAL
        with pytest.raises(mp.MPError):
            other.restore(b"not a checkpoint" * 4)


def test_cancel_stops_a_run_and_the_device_stays_usable():
    systems = [mp.System(16, 1.0, n_paths=4096) for _ in range(8)]
    sim = mp.Simulation(systems, 5000, 5000, graph=False)   # ~20 s if not stopped
    t0 = time.time()
    sim.run()
    time.sleep(0.2)
    sim.cancel()
    with pytest.raises(mp.MPError) as ei:
        sim.estimates(0)
    assert ei.value.status == mp.MP_ECANCELED
    assert time.time() - t0 < 10.0
    # a canceled resumable call leaves the saved state as it was
    sim2 = mp.Simulation([mp.System(8, 1.0, n_paths=64)], 3, 3)
    sim2.run_sweeps(2)
    blob = sim2.checkpoint()
    sim2.cancel()  # cleared when the next run starts: this call completes
    sim2.run_sweeps(1)
    assert sim2.progress() == 3
    sim2.restore(blob)
    assert sim2.progress() == 2
    sim.close()
    sim2.close()
    with mp.Simulation([mp.System(4, 1.5, n_paths=8)], 2, 2) as ok:
        ok.run()
        assert np.isfinite(ok.estimates(0)["e"])

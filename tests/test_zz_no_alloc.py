"""The allocation-free entry point (mp_run_noalloc) against the ordinary one.

mp_run_noalloc serves callers that cannot allocate device memory (code in a
framework that owns every device allocation, or that must not grow the
device heap): it keeps its scratch in one static device array.  Here it is
called twice in a row through the C ABI, on the caller's own output buffer,
for a batch of uneven sizes, one of a single size and one of open chains
(three kernel variants), and each time its estimates must equal those of
mp_create_ex / mp_run / mp_estimates for the same batch and seed; the second
call must leave the device's free memory unchanged.  The trajectories are identical
(same random numbers per site); only the order of the FP32 measurement sums
differs with the launch shape, hence the small tolerances.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1305_6758_gb300 as mp  # noqa: E402

BATCHES = {
    # uneven sizes and an open chain: the mixed-size kernel
    "mixed": [mp.System(8, 1.2, n_paths=300), mp.System(4, 2.0, h=0.1, n_paths=77),
              mp.System(16, 1.0, n_paths=40), mp.System(64, 0.8, n_paths=50, lattice=mp.CHAIN)],
    # one simple cubic size: the kernel compiled for that size
    "one-size": [mp.System(8, 1.2, n_paths=300), mp.System(8, 0.7, h=0.05, n_paths=60)],
    # open chains only: the chain kernel
    "chains": [mp.System(64, 0.8, n_paths=50, lattice=mp.CHAIN), mp.System(9, 1.5, n_paths=33, lattice=mp.CHAIN)],
}
KEYS_ABS = {"e": 1e-6, "m": 1e-6, "m2": 1e-6, "mz": 1e-6, "acc": 1e-12}
KEYS_REL = ("chi", "cv", "binder", "de_dbeta", "e_se", "m_se")


def _ordinary(systems, precision):
    with mp.Simulation(systems, 20, 30, seed=9, precision=precision) as sim:
        sim.run()
        return [sim.estimates(k) for k in range(len(systems))]


def _entry():
    lib = mp.load_library()
    lib.mp_run_noalloc.argtypes = [ctypes.POINTER(mp.MPSystem), ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                   ctypes.c_void_p, ctypes.c_void_p]
    lib.mp_run_noalloc.restype = ctypes.c_int
    return lib.mp_run_noalloc


@pytest.mark.parametrize("batch", sorted(BATCHES))
@pytest.mark.parametrize("precision", [mp.FP32, mp.FP64])
def test_noalloc_matches_ordinary_entry_point(precision, batch):
    run = _entry()
    systems = BATCHES[batch]
    ref = _ordinary(systems, precision)
    n = len(systems)
    arr = (mp.MPSystem * n)(*[mp.MPSystem(s.lattice, s.L, s.T, s.J, s.h, s.n_paths) for s in systems])
    out = torch.empty(n * mp.NEST, dtype=torch.float64, device="cuda")  # the caller's buffer
    stream = torch.cuda.Stream()
    free = []
    for call in range(2):
        with torch.cuda.stream(stream):
            out.fill_(float("nan"))
        stream.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        rc = run(arr, n, precision, 20, 30, 9, out.data_ptr(), stream.cuda_stream)
        assert rc == mp.MP_OK, f"call {call}: status {rc}"
        stream.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        est = out.cpu().numpy().reshape(n, mp.NEST)
        for k in range(n):
            got = dict(zip(mp.EST_FIELDS, est[k]))
            assert got["n_paths"] == systems[k].n_paths
            for key, tol in KEYS_ABS.items():
                assert abs(got[key] - ref[k][key]) <= tol, (call, k, key, got[key], ref[k][key])
            for key in KEYS_REL:
                assert got[key] == pytest.approx(ref[k][key], rel=1e-4, abs=1e-9), (call, k, key)
    # the second call, after the first has set up the device (and loaded its
    # kernels), takes no device memory at all
    assert free[3] == free[2], f"free device memory changed across the second call: {free}"


def test_noalloc_rejects_batches_beyond_its_scratch():
    run = _entry()
    out = torch.empty(2 * mp.NEST, dtype=torch.float64, device="cuda")
    big = (mp.MPSystem * 2)(mp.MPSystem(0, 4, 1.0, 1.0, 0.0, 10000), mp.MPSystem(0, 4, 1.0, 1.0, 0.0, 10000))
    assert run(big, 2, mp.FP32, 1, 1, 1, out.data_ptr(), None) == mp.MP_EINVAL

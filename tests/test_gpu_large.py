"""The large-lattice configuration: simple cubic L = 64 (262144 spins per path),
T in {1.40, 1.44, 1.48}, 500 + 1000 sweeps.

The FP32 form streams each lattice through shared-memory half-plane buffers;
the FP64 form's ring would not fit, so its lattices are updated in place in HBM
(path by path equal to the oracle: tests/test_gpu_streamed.py).  Here the
thermalised ensembles: the full FP32 launch (1024 paths per temperature)
against the FP64 form (independent paths) within 3 combined standard errors,
and FP32 against independent oracle paths on a shorter schedule.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1305_6758_gb300 as mp  # noqa: E402

TS = (1.40, 1.44, 1.48)
N = 64 ** 3


def estimates(systems, n_therm, n_meas, seed, **kw):
    with mp.Simulation(systems, n_therm, n_meas, seed=seed, **kw) as sim:
        sim.run()
        return [sim.estimates(k) for k in range(len(systems))], [sim.system_plan(k) for k in range(len(systems))]


def test_l64_fp32_against_fp64_form_at_3se():
    e32, p32 = estimates([mp.System(64, T, n_paths=1024) for T in TS], 500, 1000, seed=1)
    e64, p64 = estimates([mp.System(64, T, n_paths=48) for T in TS], 500, 1000, seed=2, precision=mp.FP64)
    assert p32[0]["streamed"] and p64[0]["in_place_hbm"]
    for k, T in enumerate(TS):
        for key in ("e", "m", "m2", "chi", "cv", "binder"):
            z = abs(e32[k][key] - e64[k][key]) / np.hypot(e32[k][key + "_se"], e64[k][key + "_se"])
            print(f"T={T} {key}: FP32 {e32[k][key]:.6g} FP64 {e64[k][key]:.6g} z={z:.2f}")
            assert z < 3, (T, key, e32[k][key], e64[k][key], z)


def test_l64_fp32_against_oracle_at_3se():
    n_therm, n_meas, n_orc = 100, 200, 8
    e32, _ = estimates([mp.System(64, T, n_paths=1024) for T in TS], n_therm, n_meas, seed=3)
    orc = O.run([O.System(64, T, n_paths=1024 + n_orc, path_begin=1024, path_count=n_orc) for T in TS],
                n_therm, n_meas, seed=3)
    for k, T in enumerate(TS):
        ref = O.estimates(orc[k], N, T)
        for key in ("e", "m", "m2"):
            z = abs(e32[k][key] - ref[key]) / np.hypot(e32[k][key + "_se"], ref[key + "_se"])
            assert z < 3, (T, key, e32[k][key], ref[key], z)

"""Precision of the FP32 form: every estimate against the FP64 form and the oracle.

The FP32 form keeps spins, energy differences and Boltzmann factors in FP32
and its accumulators and reduction in FP64.  Two comparisons at the simple
cubic L = 16 of the benchmark's temperature scan, T = 0.5 (ordered), 1.5 (near
T_C) and 2.5 (disordered), 1000 + 1000 sweeps:

  * FP32 against the FP64 GPU form on the same paths and seed.  Both draw the
    same random numbers; the trial direction does not depend on the old spin,
    so an accept decision that FP32 rounding flips is undone at the site's
    next accepted move and most paths stay equal to FP32 rounding.  The
    per-path differences ("paired") measure the FP32 error with a standard
    error far below that of two independent ensembles.  Bar: energy per spin
    within 1e-4, with a paired standard error below 3e-5 (so that the bar is
    resolved, not assumed).
  * FP32 against independent paths of the FP64 oracle (path ids the GPU runs
    do not use): e, |m|, chi, C_V and U_L within 3 combined standard errors.
"""
import importlib

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1305_6758_gb300 as mp  # noqa: E402

E = importlib.import_module("oracle.estimates")
N, SWEEPS, SEED = 4096, (1000, 1000), 7
CASES = [(0.5, 4096), (1.5, 24576), (2.5, 4096)]  # (T, paths): near T_C the paths decouple more often
KEYS = ("e", "m", "chi", "cv", "binder")


def _means(rec):
    return {k: rec[:, i].mean() for k, i in O.REC.items()}


def _stat(key, T):
    if key in E.DERIVED:
        f = E.DERIVED[key]
        return lambda m: f(m, N, 1.0 / T)
    return lambda m: m[key]


def paired(rec_a, rec_b, key, T):
    """Difference of one estimate between two runs of the same paths, and its
    delete-one jackknife standard error (the same path left out of both)."""
    f = _stat(key, T)
    d = f(_means(rec_a)) - f(_means(rec_b))
    P = rec_a.shape[0]
    loo = []
    sa, sb = rec_a.sum(axis=0), rec_b.sum(axis=0)
    la, lb = (sa - rec_a) / (P - 1), (sb - rec_b) / (P - 1)
    ma = {k: la[:, i] for k, i in O.REC.items()}
    mb = {k: lb[:, i] for k, i in O.REC.items()}
    loo = f(ma) - f(mb)
    se = np.sqrt((P - 1) / P * np.sum((loo - loo.mean()) ** 2))
    return float(d), float(se)


@pytest.fixture(scope="module")
def runs():
    systems = [mp.System(16, T, n_paths=P) for T, P in CASES]
    out = {}
    for prec in (mp.FP32, mp.FP64):
        with mp.Simulation(systems, *SWEEPS, seed=SEED, precision=prec) as sim:
            sim.run()
            out[prec] = ([sim.paths(k) for k in range(len(CASES))], [sim.estimates(k) for k in range(len(CASES))])
    return out


def test_fp32_energy_within_1e4_of_fp64(runs):
    recs32, _ = runs[mp.FP32]
    recs64, _ = runs[mp.FP64]
    for k, (T, P) in enumerate(CASES):
        table = {key: paired(recs32[k], recs64[k], key, T) for key in KEYS}
        print(f"T={T} P={P} FP32 - FP64 (paired SE): "
              + ", ".join(f"{key} {d:+.2e} ({se:.1e})" for key, (d, se) in table.items()))
        d, se = table["e"]
        assert se < 3e-5, (T, se)
        assert abs(d) < 1e-4, (T, d, se)


def test_fp32_estimates_against_oracle_within_3se(runs):
    _, ests32 = runs[mp.FP32]
    n_orc = 64
    orc = O.run([O.System(16, T, n_paths=P + n_orc, path_begin=P, path_count=n_orc) for T, P in CASES],
                *SWEEPS, seed=SEED)
    for k, (T, P) in enumerate(CASES):
        ref = O.estimates(orc[k], N, T)
        for key in KEYS:
            g = ests32[k]
            z = abs(g[key] - ref[key]) / np.hypot(g[key + "_se"], ref[key + "_se"])
            assert z < 3, (T, key, g[key], ref[key], z)

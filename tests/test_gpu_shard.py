"""One ensemble split by path ids (the multi-process layout, in one process).

Path k of a system draws the random numbers of path id path_begin + k, so
handles that run disjoint id ranges of the same systems and seed produce the
records of one handle running every path, bit for bit (with the same threads
per path, the FP32 partial sums are added in the same order too), and
mp_reduce on the gathered records gives that handle's estimates exactly.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1305_6758_gb300 as mp  # noqa: E402

WHOLE = [(8, 1.2, 0.0, 300), (4, 2.0, 0.1, 77), (12, 0.9, 0.0, 45)]  # (L, T, h, paths)


@pytest.mark.parametrize("precision", [mp.FP32, mp.FP64])
def test_path_ranges_reassemble_one_ensemble(precision):
    kw = dict(seed=17, precision=precision, threads_per_path=64)
    whole = [mp.System(L, T, h=h, n_paths=P) for L, T, h, P in WHOLE]
    with mp.Simulation(whole, 15, 25, **kw) as sim:
        sim.run()
        ref_rec = [sim.paths(k) for k in range(len(whole))]
        ref_est = [sim.estimates(k) for k in range(len(whole))]
    parts = []
    for world, rank in ((3, 0), (3, 1), (3, 2)):
        mine = []
        for L, T, h, P in WHOLE:
            q, r = divmod(P, world)
            begin = rank * q + min(rank, r)
            mine.append(mp.System(L, T, h=h, n_paths=q + (1 if rank < r else 0), path_begin=begin))
        with mp.Simulation(mine, 15, 25, **kw) as sim:
            sim.run()
            parts.append([sim.paths(k) for k in range(len(mine))])
    gathered = [np.concatenate([p[k] for p in parts]) for k in range(len(WHOLE))]
    for g, r in zip(gathered, ref_rec):
        np.testing.assert_array_equal(g, r)
    est = mp.reduce_records(whole, 15, 25, torch.from_numpy(np.concatenate(gathered)))
    for k in range(len(WHOLE)):
        for key, v in ref_est[k].items():
            if key == "elapsed_s":
                assert np.isnan(est[k][key])
            elif np.isnan(v):
                assert np.isnan(est[k][key]), key
            else:
                assert est[k][key] == v, (k, key, est[k][key], v)


def test_path_begin_limits():
    with pytest.raises(mp.MPError) as ei:
        mp.Simulation([mp.System(4, 1.0, n_paths=2, path_begin=2**32 - 1)], 1, 1)
    assert ei.value.status == mp.MP_EINVAL
    with mp.Simulation([mp.System(4, 1.0, n_paths=2, path_begin=2**32 - 2)], 1, 1) as sim:
        sim.run()
        assert np.isfinite(sim.estimates(0)["e"])

"""Column-walk unit tables.

The planner decodes every (column, segment) unit of the shared-memory walk
once into a table entry; the walk can also derive the same units on the
device (MP_FLAG_DEVICE_UNITS).  The two are independent encodings of the
same geometry, so every record and spin must agree bit for bit, in FP64 and
in FP32, for chunk lengths that are even and odd and for the mixed-size
kernel as well as the kernels compiled for one size.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1305_6758_gb300 as mp  # noqa: E402

BATCHES = {
    # uneven sizes: the mixed-size kernel (chunks 8, 3, 8, 4, 6 and 2 at L = 14)
    "mixed": [mp.System(8, 1.0, n_paths=9), mp.System(12, 1.3, h=0.1, n_paths=7), mp.System(16, 1.4, n_paths=5),
              mp.System(20, 1.5, n_paths=3), mp.System(24, 1.44, n_paths=2), mp.System(14, 2.0, n_paths=4)],
    # one size each: the kernels compiled for L (chunks 6 and 7)
    "L12": [mp.System(12, 1.2, n_paths=11), mp.System(12, 0.8, J=-1.0, n_paths=6)],
    "L14": [mp.System(14, 1.6, h=0.2, n_paths=6)],
}


def _run(systems, precision, flags, threads_per_path=0):
    with mp.Simulation(systems, 3, 4, seed=21, precision=precision, keep_spins=True, flags=flags,
                       threads_per_path=threads_per_path) as sim:
        sim.run()
        recs = [sim.paths(k) for k in range(len(systems))]
        spins = [sim.spins(k, p) for k, s in enumerate(systems) for p in (0, s.n_paths - 1)]
        upload = sim.upload_bytes()
    return recs, spins, upload


@pytest.mark.parametrize("name", sorted(BATCHES))
@pytest.mark.parametrize("precision", [mp.FP32, mp.FP64])
def test_unit_tables_equal_device_units(name, precision):
    systems = BATCHES[name]
    r_tab, s_tab, up_tab = _run(systems, precision, 0)
    r_dev, s_dev, up_dev = _run(systems, precision, mp.FLAG_DEVICE_UNITS)
    for a, b in zip(r_tab, r_dev):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(s_tab, s_dev):
        np.testing.assert_array_equal(a, b)
    # the tables are the only difference in what the plan uploads: 16 bytes a unit
    assert up_tab > up_dev and (up_tab - up_dev) % 16 == 0


@pytest.mark.parametrize("tp", [32, 64, 96, 160])
def test_unit_tables_for_other_thread_counts(tp):
    """K (segments per column) follows the threads per path; a table is made
    for each layout the planner can pick."""
    systems = [mp.System(12, 1.3, n_paths=5), mp.System(24, 1.5, n_paths=2)]
    r_tab, _, _ = _run(systems, mp.FP32, 0, threads_per_path=tp)
    r_dev, _, _ = _run(systems, mp.FP32, mp.FLAG_DEVICE_UNITS, threads_per_path=tp)
    for a, b in zip(r_tab, r_dev):
        np.testing.assert_array_equal(a, b)


def test_one_table_per_size_shared_by_systems():
    """21 systems of one size upload one table, not 21."""
    one = [mp.System(16, 1.0, n_paths=4)]
    many = [mp.System(16, 0.5 + 0.1 * k, n_paths=4) for k in range(21)]
    _, _, up1 = _run(one, mp.FP32, 0)
    _, _, up1d = _run(one, mp.FP32, mp.FLAG_DEVICE_UNITS)
    _, _, upn = _run(many, mp.FP32, 0)
    _, _, upnd = _run(many, mp.FP32, mp.FLAG_DEVICE_UNITS)
    assert up1 - up1d == upn - upnd > 0

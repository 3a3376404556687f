"""Differentiation (pattern 3): the covariance backward against finite
differences of independent multipath runs and against the open chain's
closed-form derivative.  L = 16 simple cubic and a 64-spin open chain,
beta in [0.6, 0.8], h in {0, 0.01}."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1305_6758_gb300 as mp  # noqa: E402
from paper_1305_6758_gb300.autograd import observables  # noqa: E402


def _grads(beta, h, **spec):
    b = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
    f = torch.tensor(h, dtype=torch.float64, requires_grad=True)
    e, m = observables(b, f, **spec)
    return e, m, b, f


def test_chain_energy_gradient_closed_form():
    """Open chain, h = 0: d<e>/dbeta = -(N-1)(1/K^2 - 1/sinh^2 K)/N, K = beta J."""
    N = 64
    betas = [0.6 + 0.02 * k for k in range(11)]
    e, m, b, f = _grads(betas, [0.0] * 11, L=N, lattice=mp.CHAIN, n_paths=4096, n_therm=200,
                        n_meas=800, seed=3)
    e.sum().backward()
    K = np.array(betas)
    exact = -(N - 1) * (1 / K**2 - 1 / np.sinh(K) ** 2) / N
    got = b.grad.numpy()
    # SE of the covariance estimator: rerun with other seeds
    reps = []
    for seed in (11, 12, 13, 14):
        e2, _, b2, _ = _grads(betas, [0.0] * 11, L=N, lattice=mp.CHAIN, n_paths=4096, n_therm=200,
                              n_meas=800, seed=seed)
        e2.sum().backward()
        reps.append(b2.grad.numpy())
    se = np.std(np.array(reps + [got]), axis=0, ddof=1)
    assert np.all(np.abs(got - exact) < 5 * se + 1e-3), (got, exact, se)
    # d<e>/dh at h = 0 vanishes by the m -> -m symmetry: zero within 5 jackknife SE
    with mp.Simulation([mp.System(N, 1 / bb, n_paths=4096, lattice=mp.CHAIN) for bb in betas], 200, 800,
                       seed=3) as sim:
        sim.run()
        ests = [sim.estimates(k) for k in range(11)]
    assert np.allclose(f.grad.numpy(), [x["de_dh"] for x in ests], rtol=1e-9, atol=1e-12)
    assert all(abs(x["de_dh"]) < 5 * x["de_dh_se"] for x in ests)


@pytest.mark.parametrize("h0", [0.0, 0.01])
def test_l16_gradients_against_central_differences(h0):
    """L = 16, beta = 0.7: autograd d<e>/dbeta and d<|m|>/dh against central
    differences (step 1e-3) of independent runs, within 4 combined SE."""
    spec = dict(L=16, n_paths=4096, n_therm=1000, n_meas=1000)
    beta, step = 0.7, 1e-3
    e, m, b, f = _grads([beta], [h0], seed=1, **spec)
    (e.sum() + m.sum()).backward()
    with mp.Simulation([mp.System(16, 1 / beta, h=h0, n_paths=4096)], 1000, 1000, seed=1) as sim:
        sim.run()
        est = sim.estimates(0)
    runs = {}
    for k, (db, dh) in enumerate(((step, 0), (-step, 0), (0, step), (0, -step))):
        with mp.Simulation([mp.System(16, 1 / (beta + db), h=h0 + dh, n_paths=4096)], 1000, 1000,
                           seed=100 + k) as sim:
            sim.run()
            runs[(db, dh)] = sim.estimates(0)
    checks = (("beta", (step, 0), b.grad.item(), est["de_dbeta_se"], est["dm_dbeta_se"]),
              ("h", (0, step), f.grad.item(), est["de_dh_se"], est["dm_dh_se"]))
    for name, d, grad, se_e, se_m in checks:
        p, q = runs[d], runs[(-d[0], -d[1])]
        fd = (p["e"] + p["m"] - q["e"] - q["m"]) / (2 * step)
        se_fd = np.sqrt(p["e_se"] ** 2 + q["e_se"] ** 2 + p["m_se"] ** 2 + q["m_se"] ** 2) / (2 * step)
        se_grad = np.hypot(se_e, se_m)
        assert abs(grad - fd) < 4 * np.hypot(se_fd, se_grad), (name, grad, fd, se_fd, se_grad)


@pytest.mark.parametrize("L,T,h0,step,term_visible", [(8, 2.0, 0.3, 0.01, True), (16, 1 / 0.6, 0.01, 0.005, False)])
def test_energy_field_derivative_against_central_difference(L, T, h0, step, term_visible):
    """d<e>/dh alone: autograd against the central difference of <e> of
    independent runs (4 combined SE), in the paramagnetic phase, where every
    mode equilibrates within the run.  At T = 2, h = 0.3 the field term -<m_z>
    of d<e>/dh is large, and the formula without it fails; h = 0.01 is the
    differentiation configuration's field.  (In the ordered phase a small field
    acts through the slow rotation of the whole magnetisation, which local
    updates do not equilibrate in a run of this length.)"""
    n_therm, n_meas = 300, 1000
    spec = dict(L=L, n_paths=4096, n_therm=n_therm, n_meas=n_meas)
    e, m, b, f = _grads([1 / T], [h0], seed=1, **spec)
    e.sum().backward()
    with mp.Simulation([mp.System(L, T, h=h0, n_paths=4096)], n_therm, n_meas, seed=1) as sim:
        sim.run()
        est = sim.estimates(0)
    assert f.grad.item() == pytest.approx(est["de_dh"], rel=1e-12)
    runs = []
    for k, dh in enumerate((step, -step)):
        with mp.Simulation([mp.System(L, T, h=h0 + dh, n_paths=4096)], n_therm, n_meas,
                           seed=200 + k) as sim:
            sim.run()
            runs.append(sim.estimates(0))
    fd = (runs[0]["e"] - runs[1]["e"]) / (2 * step)
    se = np.hypot(np.hypot(runs[0]["e_se"], runs[1]["e_se"]) / (2 * step), est["de_dh_se"])
    print("d<e>/dh", f.grad.item(), "central difference", fd, "SE", se, "<m_z>", est["mz"])
    assert abs(f.grad.item() - fd) < 4 * se, (f.grad.item(), fd, se)
    if term_visible:
        assert abs(f.grad.item() + est["mz"] - fd) > 4 * se


def test_backward_by_replay_from_the_thermalised_checkpoint():
    """keep_records=False: the forward pass keeps only a host checkpoint taken
    after thermalisation; the backward pass replays the measurement sweeps
    from it.  Outputs and gradients equal those of keep_records=True bit for
    bit, and the replay costs about n_meas / (n_therm + n_meas) of a full run."""
    from paper_1305_6758_gb300.autograd import MPObservables

    betas, fields = [0.62, 0.7, 0.78], [0.0, 0.01, 0.0]
    spec = dict(L=16, n_paths=2048, n_therm=1500, n_meas=500, seed=21)
    outs = {}
    for keep in (True, False):
        b = torch.tensor(betas, dtype=torch.float64, requires_grad=True)
        f = torch.tensor(fields, dtype=torch.float64, requires_grad=True)
        e, m = MPObservables.apply(b, f, dict(spec, keep_records=keep))
        (e.sum() + 0.5 * m.sum()).backward()
        outs[keep] = (e.detach().numpy(), m.detach().numpy(), b.grad.numpy(), f.grad.numpy())
    for x, y in zip(outs[True], outs[False]):
        np.testing.assert_array_equal(x, y)
    # device time of the replay (n_meas sweeps) against a full run (n_therm + n_meas)
    systems = [mp.System(16, 1 / bb, h=hh, n_paths=2048) for bb, hh in zip(betas, fields)]
    with mp.Simulation(systems, 1500, 500, seed=21) as sim:
        sim.run()
        full_ms = sim.timing()[0]
        sim.run_sweeps(1500)
        blob = sim.checkpoint()
    with mp.Simulation(systems, 1500, 500, seed=21) as sim:
        sim.restore(blob)
        sim.run_sweeps(500)
        replay_ms = sim.timing()[0]
    print("full run", full_ms, "ms; replay of the measurement sweeps", replay_ms, "ms")
    assert replay_ms < 0.4 * full_ms

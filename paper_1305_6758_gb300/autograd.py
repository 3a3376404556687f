"""Differentiable ensemble observables: <e> and <|m|> as functions of (beta, h).

The Boltzmann average of an observable O depends on beta and h through the
weight exp(-beta H), H = -J sum S.S - h sum S^z = N e, so (fluctuation-dissipation)
  d<O>/dbeta = -N (<O e> - <O><e>),
  d<O>/dh    = beta N (<O m_z> - <O><m_z>) + <dO/dh>,
the estimators behind C_V and chi of Eq. (cv) in Sec. 2.2.  Only O = e has
an explicit field term (de/dh = -m_z), so
  d<e>/dh = beta N (<e m_z> - <e><m_z>) - <m_z>,   d<|m|>/dh = beta N cov(|m|, m_z).
The forward pass is a multipath run (one system per (beta, h) pair); the backward pass is the
library's covariance kernel over the per-path pooled moments, weighted by the
upstream gradients.

With keep_records=False (device memory short) the forward pass runs the
thermalisation sweeps, checkpoints every path's state to host memory
(mp_checkpoint), runs the measurement sweeps and releases all its device
memory.  The backward pass restores that checkpoint into a new simulation and
recomputes only the n_meas measurement sweeps: the random numbers are a
function of (seed, system, path, sweep, site) only, so the recomputed records,
and the gradients, are bit-identical to those of the forward pass.
"""
from __future__ import annotations

import torch

from . import FP32, INIT_SPHERE, SC, Simulation, System


def _systems(beta, h, spec):
    return [System(spec["L"], 1.0 / float(b), spec.get("J", 1.0), float(f), spec["n_paths"],
                   spec.get("lattice", SC)) for b, f in zip(beta.tolist(), h.tolist())]


def _simulation(beta, h, spec, device):
    return Simulation(_systems(beta, h, spec), spec["n_therm"], spec["n_meas"], spec.get("seed", 1),
                      precision=spec.get("precision", FP32), init_mode=spec.get("init_mode", INIT_SPHERE),
                      device=device)


class MPObservables(torch.autograd.Function):
    """forward(beta, h, spec) -> (<e>, <|m|>), one entry per (beta, h) pair.

    beta, h: 1-D float64 tensors of equal length.  spec: dict with L, n_paths,
    n_therm, n_meas and optionally J, lattice, seed, precision, init_mode,
    keep_records (default True), device.
    """

    @staticmethod
    def forward(ctx, beta, h, spec):
        device = torch.device(spec.get("device", "cuda:0"))
        b = beta.detach().to("cpu", torch.float64).reshape(-1)
        f = h.detach().to("cpu", torch.float64).reshape(-1)
        if b.numel() != f.numel():
            raise ValueError("beta and h need the same length")
        sim = _simulation(b, f, spec, device)
        keep = spec.get("keep_records", True)
        ctx.blob = None
        if keep:
            sim.run()
        else:
            # thermalise, keep the state on the host, then measure
            if spec["n_therm"] > 0:
                sim.run_sweeps(spec["n_therm"])
                ctx.blob = sim.checkpoint()
            sim.run_sweeps(spec["n_meas"])
        ests = [sim.estimates(k) for k in range(b.numel())]
        e = torch.tensor([x["e"] for x in ests], dtype=torch.float64, device=beta.device)
        m = torch.tensor([x["m"] for x in ests], dtype=torch.float64, device=beta.device)
        ctx.spec, ctx.device, ctx.b, ctx.f = spec, device, b, f
        ctx.out_device = beta.device
        ctx.ests = ests
        if keep:
            ctx.sim = sim
        else:
            sim.close()
            ctx.sim = None
        return e, m

    @staticmethod
    def backward(ctx, g_e, g_m):
        sim = ctx.sim
        if sim is None:  # replay the measurement sweeps from the checkpoint (bit-identical records)
            sim = _simulation(ctx.b, ctx.f, ctx.spec, ctx.device)
            if ctx.blob is not None:
                sim.restore(ctx.blob)
            sim.run_sweeps(ctx.spec["n_meas"])
            ctx.replay_ms = sim.timing()[0]
        n = ctx.b.numel()
        ge = torch.zeros(n, dtype=torch.float64) if g_e is None else g_e.detach()
        gm = torch.zeros(n, dtype=torch.float64) if g_m is None else g_m.detach()
        gb, gh = sim.backward(ge.to(ctx.device), gm.to(ctx.device))
        if ctx.sim is None:
            sim.close()
        return gb.to(ctx.out_device), gh.to(ctx.out_device), None


def observables(beta, h, **spec):
    """<e>, <|m|> at each (beta, h), differentiable in beta and h."""
    return MPObservables.apply(beta, h, spec)

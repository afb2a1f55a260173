"""Differentiable runs: phi_T = LdRun.apply(phi0, kappa, tau_f, spec).

Forward: ld_init from phi0 (rho = rho0, u = 0), then ``spec.steps`` steps;
the state is saved every ``spec.checkpoint_every`` steps (ld_save_state).
Backward (reverse mode, all in the library's kernels):
  ld_adjoint_seed(dL/dphi_T); for each segment, last first: recompute its
  states from the segment's checkpoint into a tape (ld_step_between, which
  writes each step's output straight into the next tape buffer and the
  phi/mu fields of its input into a fields buffer), then ld_adjoint_step over
  the tape in reverse; finally ld_adjoint_init gives dL/dphi0. dL/dkappa and
  dL/dtau_f accumulate in FP64 on the device.
Memory: one checkpoint per segment plus a tape of checkpoint_every - 1
states (ld_state_bytes() each) and checkpoint_every - 1 field buffers
(ld_fields_bytes() each).
"""

from __future__ import annotations

import dataclasses

import torch

from . import ld


@dataclasses.dataclass(frozen=True)
class RunSpec:
    nx: int
    ny: int
    nz: int
    steps: int
    checkpoint_every: int = 20
    precision: str = "fp32"
    kernel: str = "auto"
    A: float = -0.0625
    B: float = 0.0625
    Gamma: float = 0.5
    tau_g: float = 1.0
    rho0: float = 1.0
    stencil: int = 7  # 7-point Laplacian and central difference, or 19-point isotropic


class LdRun(torch.autograd.Function):
    """phi_T (nz, ny, nx) float64 from phi0 (same shape, float64, CUDA) and
    scalar tensors kappa, tau_f; differentiable in all three."""

    @staticmethod
    def forward(ctx, phi0, kappa, tau_f, spec: RunSpec):
        if spec.steps < 0 or spec.checkpoint_every < 1:
            raise ValueError("steps must be >= 0 and checkpoint_every >= 1")
        sim = ld.LdSim(spec.nx, spec.ny, spec.nz, precision=spec.precision, kernel=spec.kernel, A=spec.A, B=spec.B,
                       kappa=float(kappa), Gamma=spec.Gamma, tau_f=float(tau_f), tau_g=spec.tau_g, rho0=spec.rho0,
                       stencil=spec.stencil)
        phi0 = phi0.detach().to(device=sim.device, dtype=torch.float64).contiguous()
        sim.init(phi0)
        checkpoints = []
        t = 0
        while t < spec.steps:
            checkpoints.append(sim.save_state())
            k = min(spec.checkpoint_every, spec.steps - t)
            sim.step(k)
            t += k
        phi_t = torch.empty(sim.shape, dtype=torch.float64, device=sim.device)
        ld.ld_moments(sim.ctx, phi=phi_t)
        ctx.sim = sim
        ctx.checkpoints = checkpoints
        ctx.spec = spec
        ctx.phi0 = phi0
        ctx.param_meta = [(kappa.dtype, kappa.device), (tau_f.dtype, tau_f.device)]
        return phi_t

    @staticmethod
    def backward(ctx, grad_phi_t):
        sim, spec = ctx.sim, ctx.spec
        dev = sim.device
        workspace = torch.empty(ld.ld_adjoint_workspace_bytes(sim.ctx), dtype=torch.uint8, device=dev)
        ld.ld_adjoint_attach(sim.ctx, workspace)
        grad = torch.zeros(2, dtype=torch.float64, device=dev)
        ld.ld_adjoint_seed(sim.ctx, grad_phi_t.detach().to(dtype=torch.float64).contiguous())
        nbytes = ld.ld_state_bytes(sim.ctx)
        ntape = max(0, min(spec.checkpoint_every, spec.steps) - 1)
        tape = [torch.empty(nbytes, dtype=torch.uint8, device=dev) for _ in range(ntape)]
        fbytes = ld.ld_fields_bytes(sim.ctx)
        fields = [torch.empty(fbytes, dtype=torch.uint8, device=dev) for _ in range(ntape)]
        for seg in reversed(range(len(ctx.checkpoints))):
            t0 = seg * spec.checkpoint_every
            k = min(spec.checkpoint_every, spec.steps - t0)
            states = [ctx.checkpoints[seg]] + tape[:k - 1]
            for j in range(1, k):
                ld.ld_step_between(sim.ctx, states[j - 1], states[j], fields[j - 1])
            for j in reversed(range(k)):
                ld.ld_adjoint_step(sim.ctx, states[j], grad, fields[j] if j < k - 1 else None)
        grad_phi0 = torch.empty_like(ctx.phi0)
        ld.ld_adjoint_init(sim.ctx, ctx.phi0, grad_phi0, None, grad)
        (kd, kdev), (td, tdev) = ctx.param_meta
        g_kappa = grad[0].to(dtype=kd, device=kdev)
        g_tau = grad[1].to(dtype=td, device=tdev)
        ctx.sim = None  # release the workspace with the context
        return grad_phi0, g_kappa, g_tau, None


def run(phi0, kappa, tau_f, spec: RunSpec):
    """phi_T of a differentiable run (see LdRun)."""
    if not torch.is_tensor(kappa):
        kappa = torch.tensor(float(kappa), dtype=torch.float64)
    if not torch.is_tensor(tau_f):
        tau_f = torch.tensor(float(tau_f), dtype=torch.float64)
    return LdRun.apply(phi0, kappa, tau_f, spec)

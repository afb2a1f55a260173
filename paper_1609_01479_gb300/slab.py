"""Domain decomposition of the lattice into z-slabs with halo exchange.

The paper's Ludwig runs split the lattice into sub-domains, each surrounded
by halo regions that are filled from the neighbouring sub-domains before the
stencils read them (Sec. 2.1.1), and scale across nodes that way (Sec. 5).
Here the periodic nz planes are split into `nslabs` equal slabs along z.
Slab k owns the global planes [k m, (k+1) m), m = nz / nslabs, and is held as
its own periodic lattice of m + 2H planes: H halo planes below, its own m
planes, H halo planes above (local plane p is global plane k m - H + p,
modulo nz).

One step of the method at a site reads the state within 3 planes of it (the
phi stencil and mu reach 2, propagation 1), so after the halos are refreshed
one step of the slab's own lattice reproduces the whole lattice's step
exactly on the slab's own planes, whatever the kernel did to its halo planes
(they wrap onto each other and are overwritten by the next exchange). With
H = 3 s halo planes, s steps can run between exchanges. H is rounded up so
that m + 2H admits the fused kernels (a multiple of 4 planes).

The exchange copies the f and g of whole planes with the library's
ld_pack_planes / ld_unpack_planes (stream-ordered device copies through a
packed buffer): slab k's lowest H own planes fill the upper halo of slab
k - 1, its highest H own planes the lower halo of slab k + 1 (periodically).
Every slab here lives on the same GPU; the plan is written as a list of
transfers between slabs, which is the schedule a multi-process transport
would send and receive.
"""

from __future__ import annotations

from dataclasses import dataclass

import torch

from . import ld


@dataclass(frozen=True)
class Transfer:
    """Copy `nplanes` planes from local plane `src_z0` of slab `src` to local
    plane `dst_z0` of slab `dst`."""

    src: int
    src_z0: int
    dst: int
    dst_z0: int
    nplanes: int


def halo_depth(m: int, steps_per_exchange: int = 1) -> int:
    """Halo planes per side: at least 3 per step between exchanges, rounded
    up so that m + 2H is a multiple of 4 when m is even (odd m: 3 s)."""
    if m < 1 or steps_per_exchange < 1:
        raise ValueError("slab size and steps per exchange must be >= 1")
    h = 3 * steps_per_exchange
    if m % 2 == 0:
        while (m + 2 * h) % 4:
            h += 1
    return h


def exchange_plan(nslabs: int, m: int, h: int):
    """The transfers that refresh every slab's halos (own planes are local
    [h, h + m)); needs m >= h, so that a halo comes from one neighbour."""
    if m < h:
        raise ValueError(f"slabs of {m} planes are thinner than their {h}-plane halos")
    plan = []
    for k in range(nslabs):
        below, above = (k - 1) % nslabs, (k + 1) % nslabs
        plan.append(Transfer(src=k, src_z0=h, dst=below, dst_z0=h + m, nplanes=h))  # lowest own -> upper halo below
        plan.append(Transfer(src=k, src_z0=m, dst=above, dst_z0=0, nplanes=h))      # highest own -> lower halo above
    return plan


def local_to_global(k: int, m: int, h: int, nz: int, p: int) -> int:
    """Global plane of local plane p of slab k."""
    return (k * m - h + p) % nz


class SlabLattice:
    """A periodic nx x ny x nz lattice run as `nslabs` z-slabs, each its own
    library context on the current GPU, with halo exchange between steps.

    Fields are read and written as whole-lattice torch tensors (nz, ny, nx)
    on the device; the slabs' own planes reproduce the single-lattice step.
    """

    def __init__(self, nx, ny, nz, nslabs, precision="fp32", kernel="auto", steps_per_exchange=1,
                 device="cuda", stream=None, **model):
        if nslabs < 1 or nz % nslabs:
            raise ValueError("nz must be a multiple of the number of slabs")
        self.nx, self.ny, self.nz, self.nslabs = nx, ny, nz, nslabs
        self.m = nz // nslabs
        self.h = halo_depth(self.m, steps_per_exchange)
        self.steps_per_exchange = steps_per_exchange
        self.plan = exchange_plan(nslabs, self.m, self.h)
        self.device = torch.device(device)
        self.slabs = [ld.LdSim(nx, ny, self.m + 2 * self.h, precision=precision, kernel=kernel, device=device,
                               stream=stream, **model) for _ in range(nslabs)]
        nbytes = ld.ld_planes_bytes(self.slabs[0].ctx, self.h)
        self.buffers = [torch.empty(nbytes, dtype=torch.uint8, device=self.device) for _ in self.plan]
        self._since_exchange = 0

    def close(self):
        for s in self.slabs:
            s.close()

    def _extended(self, field, k):
        """Planes of slab k's local lattice (own planes and halos) of a
        whole-lattice field shaped (..., nz, ny, nx)."""
        idx = torch.tensor([local_to_global(k, self.m, self.h, self.nz, p) for p in range(self.m + 2 * self.h)],
                           device=field.device)
        return field.index_select(-3, idx).contiguous()

    def init(self, phi, rho=None, u=None):
        """Equilibrium start from whole-lattice fields; the 16-bit forms take
        the whole lattice's mean phi as their deviation reference."""
        phi = torch.as_tensor(phi, dtype=torch.float64, device=self.device).contiguous()
        total = torch.empty(1, dtype=torch.float64, device=self.device)
        ld.ld_field_sum(self.slabs[0].ctx, phi, total)  # the whole lattice's sum, in ld_init's order
        mean = float(total.item()) / phi.numel()
        self._inputs = []
        for k, s in enumerate(self.slabs):
            pk = self._extended(phi, k)
            rk = None if rho is None else self._extended(torch.as_tensor(rho, dtype=torch.float64,
                                                                         device=self.device), k)
            uk = None if u is None else self._extended(torch.as_tensor(u, dtype=torch.float64, device=self.device), k)
            self._inputs.append((pk, rk, uk))  # kept alive until the stream has consumed them
            ld.ld_init_with_reference(s.ctx, pk, rk, uk, mean)
        # the outermost halo planes took their mu from wrapped neighbours:
        # refresh every halo before the first step
        self._since_exchange = self.steps_per_exchange

    def exchange(self):
        """Refresh every halo from the neighbouring slabs' own planes: all
        packs first, then all unpacks, so no unpack overwrites a plane that a
        later pack still reads."""
        for t, buf in zip(self.plan, self.buffers):
            ld.ld_pack_planes(self.slabs[t.src].ctx, t.src_z0, t.nplanes, buf)
        for t, buf in zip(self.plan, self.buffers):
            ld.ld_unpack_planes(self.slabs[t.dst].ctx, t.dst_z0, t.nplanes, buf)
        self._since_exchange = 0

    def step(self, nsteps=1):
        """nsteps steps of the whole lattice: halos are refreshed before a
        step whenever steps_per_exchange steps have run on the current ones."""
        for _ in range(nsteps):
            if self._since_exchange >= self.steps_per_exchange:
                self.exchange()
            for s in self.slabs:
                ld.ld_step(s.ctx, 1)
            self._since_exchange += 1

    def _gather(self, per_slab):
        own = slice(self.h, self.h + self.m)
        return torch.cat([t[..., own, :, :] for t in per_slab], dim=-3).contiguous()

    def moments(self):
        """rho, u and phi of the whole lattice (the own planes of every slab)."""
        parts = [s.moments() for s in self.slabs]
        return {k: self._gather([p[k] for p in parts]) for k in ("rho", "u", "phi")}

    def distributions(self):
        parts = [s.distributions() for s in self.slabs]
        return self._gather([p[0] for p in parts]), self._gather([p[1] for p in parts])

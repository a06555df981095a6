"""Seeded synthetic particle boxes for the CWTHF hot path.

This module only *generates inputs*; it holds none of the halo finder's
arithmetic and is shared by the CUDA tests, the oracle tests and bench.py.

The paper evaluates on the SIMBA m50n512 dark-matter snapshot (Sec. 3: a
50 Mpc/h box with 512^3 particles).  That snapshot is not available here, so
clustered boxes of the same character stand in for it:

* a fraction (default 40 %) of the particles uniform in the periodic box;
* the rest in NFW clumps: centres uniform, particle counts proportional to
  draws from dN/dM ~ M^-1.9 on [1, 1e3] (rescaled to sum exactly, largest
  remainder), concentration c ~ U[5, 15], virial radius R ~ U[0.2, 1.5] Mpc/h,
  r_s = R / c, radii from the inverse of the truncated NFW enclosed-mass
  profile mu(r/r_s)/mu(c), mu(y) = ln(1+y) - y/(1+y), isotropic directions;
* periodic wrap into [0, L), float32 positions, equal masses, and the
  particle order randomly permuted (snapshots are not sorted in space);
* on request, velocities for the self-boundness check (Sec. 2.3): Gaussian
  field motions of 300 km/s per axis, and inside clumps an isotropic
  Gaussian of virial dispersion sqrt(G M / R) about the clump's bulk motion.

Everything is drawn from one ``torch.Generator`` seeded by the caller, so a
box is reproducible on a given device type.  CPU and CUDA generators give
different (equally valid) boxes; a comparison always feeds the same tensor
to both sides.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

NFW_C_RANGE = (5.0, 15.0)
RVIR_RANGE = (0.2, 1.5)
CLUMP_MASS_RANGE = (1.0, 1.0e3)
CLUMP_MASS_SLOPE = 1.9
CLUMP_DENSITY = 1.6e-3  # clumps per (Mpc/h)^3 when a workload does not fix the count


def _nfw_mu(y: torch.Tensor) -> torch.Tensor:
    return torch.log1p(y) - y / (1.0 + y)


def _nfw_radii(u: torch.Tensor, c: torch.Tensor, iters: int = 40) -> torch.Tensor:
    """Solve mu(y) = u * mu(c) for y in [0, c] by bisection (fp64)."""
    target = u * _nfw_mu(c)
    lo = torch.zeros_like(c)
    hi = c.clone()
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        below = _nfw_mu(mid) < target
        lo = torch.where(below, mid, lo)
        hi = torch.where(below, hi, mid)
    return 0.5 * (lo + hi)


def clump_counts(n_in_clumps: int, n_clumps: int, gen: torch.Generator, device) -> torch.Tensor:
    """Particle counts per clump, proportional to power-law draws, summing
    exactly to n_in_clumps (largest-remainder rounding, ties by index)."""
    if n_clumps <= 0 or n_in_clumps <= 0:
        return torch.zeros(max(n_clumps, 0), dtype=torch.int64, device=device)
    a = 1.0 - CLUMP_MASS_SLOPE
    lo, hi = CLUMP_MASS_RANGE
    u = torch.rand(n_clumps, generator=gen, device=device, dtype=torch.float64)
    m = (lo ** a + u * (hi ** a - lo ** a)) ** (1.0 / a)
    raw = m / m.sum() * n_in_clumps
    base = torch.floor(raw).to(torch.int64)
    rem = int(n_in_clumps - int(base.sum()))
    if rem > 0:
        frac = raw - base.to(torch.float64)
        order = torch.argsort(-frac, stable=True)
        base[order[:rem]] += 1
    return base


# Units of the velocities: positions in Mpc/h, velocities in km/s, masses in
# Msun/h; G in those units, and the mean matter density (Omega_m = 0.3) that
# gives the particle mass of a box.
G_MPC_KMS_MSUN = 4.30091727e-9
RHO_MEAN = 0.3 * 2.77536627e11  # (Msun/h) / (Mpc/h)^3
SIGMA_FIELD = 300.0  # km/s per axis: uniform particles and clump bulk motions


def particle_mass(n_particles: int, box: float) -> float:
    """Msun/h per particle of an equal-mass box at the mean matter density."""
    return RHO_MEAN * box ** 3 / max(n_particles, 1)


def clumped_box(n_particles: int, box: float, n_clumps: int | None = None, seed: int = 0,
                device="cpu", uniform_frac: float = 0.4, shuffle: bool = True, velocities: bool = False):
    """float32 [n_particles, 3] positions in [0, box); with velocities=True
    also float32 [n_particles, 3] velocities (km/s): uniform particles and
    clump bulk motions Gaussian with SIGMA_FIELD per axis, and clump members
    their clump's bulk velocity plus an isotropic Gaussian of 3D dispersion
    V_vir = sqrt(G M / R) (M = members x particle_mass, R the clump's virial
    radius).  Velocities come from a second generator, so the positions are
    those of velocities=False."""
    device = torch.device(device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    genv = None
    if velocities:
        genv = torch.Generator(device=device)
        genv.manual_seed(int(seed) * 7919 + 104729)
        vout = torch.empty((n_particles, 3), dtype=torch.float32, device=device)
        mp = particle_mass(n_particles, box)
    if n_clumps is None:
        n_clumps = max(1, int(round(CLUMP_DENSITY * box ** 3)))
    n_uni = int(round(uniform_frac * n_particles))
    n_cl = n_particles - n_uni
    f64 = torch.float64
    # positions are formed in fp64 chunk by chunk, wrapped, and stored as float32
    out = torch.empty((n_particles, 3), dtype=torch.float32, device=device)
    chunk = 1 << 24

    def store(dst0, x):
        x = torch.remainder(x, box).to(torch.float32)
        x[x >= box] = 0.0  # float32 rounding of values just below box
        out[dst0:dst0 + x.shape[0]] = x

    for s in range(0, n_uni, chunk):
        k = min(chunk, n_uni - s)
        store(s, torch.rand((k, 3), generator=gen, device=device, dtype=f64) * box)
        if velocities:
            vout[s:s + k] = (SIGMA_FIELD * torch.randn((k, 3), generator=genv, device=device, dtype=f64)).float()
    if n_cl > 0:
        counts = clump_counts(n_cl, n_clumps, gen, device)
        centres = torch.rand((n_clumps, 3), generator=gen, device=device, dtype=f64) * box
        conc = NFW_C_RANGE[0] + (NFW_C_RANGE[1] - NFW_C_RANGE[0]) * torch.rand(n_clumps, generator=gen, device=device, dtype=f64)
        rvir = RVIR_RANGE[0] + (RVIR_RANGE[1] - RVIR_RANGE[0]) * torch.rand(n_clumps, generator=gen, device=device, dtype=f64)
        owner = torch.repeat_interleave(torch.arange(n_clumps, device=device), counts)
        if velocities:
            bulk = SIGMA_FIELD * torch.randn((n_clumps, 3), generator=genv, device=device, dtype=f64)
            sig1 = torch.sqrt(G_MPC_KMS_MSUN * counts.to(f64) * mp / rvir / 3.0)  # per axis
        for s in range(0, n_cl, chunk):
            o = owner[s:s + chunk]
            k = o.numel()
            u = torch.rand(k, generator=gen, device=device, dtype=f64)
            y = _nfw_radii(u, conc[o])
            r = y * (rvir[o] / conc[o])
            d = torch.randn((k, 3), generator=gen, device=device, dtype=f64)
            d = d / d.norm(dim=1, keepdim=True).clamp_min(1e-300)
            store(n_uni + s, centres[o] + r[:, None] * d)
            if velocities:
                dv = torch.randn((k, 3), generator=genv, device=device, dtype=f64)
                vout[n_uni + s:n_uni + s + k] = (bulk[o] + sig1[o, None] * dv).float()
        del owner
    if shuffle:
        perm = torch.randperm(n_particles, generator=gen, device=device)
        out = out[perm]
        if velocities:
            vout = vout[perm]
    if velocities:
        return out.contiguous(), vout.contiguous()
    return out.contiguous()


def smooth_ng(ng: float) -> int:
    """Nearest grid size of the form 2^a 3^b (a >= 1) to ng, in log distance."""
    best, bestd = 8, float("inf")
    for a in range(1, 12):
        for b in range(0, 8):
            v = (2 ** a) * (3 ** b)
            if v < 8 or v > 1024:
                continue
            d = abs(math.log(v) - math.log(ng))
            if d < bestd:
                best, bestd = v, d
    return best


@dataclass
class Workload:
    """One named synthetic workload: a box of clumped particles, a grid size
    and the wavelet scales to run."""
    name: str
    n_particles: int
    box: float
    ng: int
    n_clumps: int
    seed: int
    scales: tuple = (2.0,)
    extra: dict = field(default_factory=dict)

    def positions(self, device="cpu") -> torch.Tensor:
        return clumped_box(self.n_particles, self.box, self.n_clumps, self.seed, device)


# The named workloads (particle box, grid and scales).  Scale w = 2 h/Mpc is
# the single-scale default: the paper's lowest k_w = 0.1 in its 50 Mpc/h box.
WORKLOADS = {
    "clumped-64cube-L50": Workload("clumped-64cube-L50", 64 ** 3, 50.0, 64, 200, 1),
    "clumped-256cube-L200": Workload("clumped-256cube-L200", 256 ** 3, 200.0, 256, 12800, 2),
    "clumped-256cube-grid512-L250": Workload("clumped-256cube-grid512-L250", 256 ** 3, 250.0, 512, 12500, 6),
    "clumped-512cube-grid1024-L500": Workload("clumped-512cube-grid1024-L500", 512 ** 3, 500.0, 1024,
                                              100000, 3, scales=(2.0, 3.0, 4.0)),
}


def batched_subvolumes(n_jobs: int = 64, seed: int = 4, spacing: float = 0.78125,
                       grids=(32, 64, 96, 128, 192), np_range=(1e4, 1e7)):
    """Uneven batch: grid sizes uniform over `grids`, particle counts log-uniform
    over np_range, box = ng * spacing, clump density CLUMP_DENSITY."""
    g = torch.Generator().manual_seed(seed)
    jobs = []
    for j in range(n_jobs):
        ng = grids[int(torch.randint(len(grids), (1,), generator=g))]
        lo, hi = math.log(np_range[0]), math.log(np_range[1])
        npart = int(round(math.exp(lo + (hi - lo) * float(torch.rand(1, generator=g)))))
        box = ng * spacing
        jobs.append(Workload(f"sub{j}", npart, box, ng, max(1, int(round(CLUMP_DENSITY * box ** 3))),
                             seed * 1000 + j))
    return jobs

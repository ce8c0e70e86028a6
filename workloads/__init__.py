"""Seeded synthetic inputs for the coupled Maxwell-LLG solver.

This module only *describes* problems: grid sizes, spacings, time step,
boundary types, cell-centred material arrays, cell-centred initial
magnetisation and source descriptors.  It holds none of the scheme's
arithmetic (no averaging to edges/faces, no renormalisation, no curls, no
LLG algebra).  Both the CPU oracle and the CUDA library consume exactly these
inputs, so random draws can never break parity.

Arrays are float64 with shape (nz, ny, nx) in C order, i.e. x is the fastest
index, matching the flat "x fastest" layout of the C entry points.

Workloads follow the paper's test problems (Sec. 5: convergence test,
air-filled waveguide, magnetically tunable filter) at fixed sizes:
  * ``yig_slab_32``            32^3 PEC box with a YIG-like slab, point Jx source.
  * ``waveguide``              128x128x512 PEC guide, z-PML ends, YIG slab,
                               TE10 soft plane source.
  * ``stress``                 512^3 PEC box, centred random 256^3 magnetic block.
  * ``convergence(N)``         the paper's periodic convergence problem (Sec. 5.1).
  * ``filter_design``          64x64x256 ferrite-loaded guide with a random
                               permittivity design region, for the adjoint.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

# Speed of light used only to turn a CFL number into a time step.
C0 = 299792458.0

PERIODIC, PEC, PML = 0, 1, 2

# Source kinds (same numbering as the C entry points).
SRC_POINT_J, SRC_PLANE_J_TE10, SRC_HARD_E, SRC_HARD_H = 0, 1, 2, 3


@dataclasses.dataclass
class Source:
    kind: int
    comp: int
    i: int = 0
    j: int = 0
    k: int = 0
    amp: float = 0.0
    f0: float = 0.0
    tp: float = 1.0
    t0: float = 0.0


@dataclasses.dataclass
class Workload:
    name: str
    n: Tuple[int, int, int]
    d: Tuple[float, float, float]
    dt: float
    bc: Tuple[int, int, int]
    pml_cells: int = 0
    order: int = 2
    tol: float = 1e-10
    max_iter: int = 64
    h0: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    eps_r: Optional[np.ndarray] = None
    sigma: Optional[np.ndarray] = None
    mu_r: Optional[np.ndarray] = None
    Ms: Optional[np.ndarray] = None
    alpha: Optional[np.ndarray] = None
    gamma: Optional[np.ndarray] = None
    m_cells: Optional[Tuple[np.ndarray, np.ndarray, np.ndarray]] = None
    sources: List[Source] = dataclasses.field(default_factory=list)
    # optional initial Yee-located fields: field id -> flat float64 array
    fields: Dict[int, np.ndarray] = dataclasses.field(default_factory=dict)
    steps: int = 1
    # z node plane of the flux loss (design workloads)
    flux_k: Optional[int] = None

    @property
    def ncells(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])


def cfl_dt(d: Sequence[float], cfl: float) -> float:
    """Time step from a CFL number, dt = cfl / (c sqrt(sum 1/d_i^2))."""
    return cfl / (C0 * math.sqrt(sum(1.0 / (x * x) for x in d)))


def _cell_shape(n):
    return (n[2], n[1], n[0])


def field_extent(fid: int, n) -> Tuple[int, int, int]:
    """(ex, ey, ez) extents of a Yee-located field id (0-2 E, 3-5 H, 6-14 M,
    15/16 PML z-parts of Ex/Ey, 17/18 PML z-parts of Hx/Hy)."""
    nx, ny, nz = n
    if fid in (0, 15):
        return (nx, ny + 1, nz + 1)
    if fid in (1, 16):
        return (nx + 1, ny, nz + 1)
    if fid == 2:
        return (nx + 1, ny + 1, nz)
    if 3 <= fid <= 14 or fid in (17, 18):
        fam = {17: 0, 18: 1}.get(fid, (fid - 3) if fid < 6 else (fid - 6) // 3)
        e = [nx, ny, nz]
        e[fam] += 1
        return tuple(e)
    raise ValueError(f"bad field id {fid}")


def field_size(fid: int, n) -> int:
    e = field_extent(fid, n)
    return e[0] * e[1] * e[2]


def _tilted_z(rng, shape, tilt=0.01):
    """Unit-free direction zhat + tilt*(u1, u2, 0), u ~ U[-1, 1] per cell."""
    u1 = rng.uniform(-1.0, 1.0, size=shape)
    u2 = rng.uniform(-1.0, 1.0, size=shape)
    return tilt * u1, tilt * u2, np.ones(shape)


# YIG-like slab values used by the slab workloads.
YIG_MS, YIG_ALPHA, YIG_GAMMA, YIG_EPS = 1.4e5, 0.005, 1.76e11, 15.0


def yig_slab_32(seed: int = 0, steps: int = 200, n: int = 32) -> Workload:
    """32^3 PEC box, dx = 1e-6 m, dt = 0.9 dx/(c sqrt 3); YIG-like slab on
    z cells 12-19 over the whole x-y section; M = z + 1% seeded tilt;
    H0 = 1e5 A/m along z; Gaussian Jx point source on edge (8.5, 16, 16)
    with a 5 GHz carrier, Tp = 200 dt, t0 = 3 Tp."""
    nn = (n, n, n)
    dx = 1e-6
    dt = cfl_dt((dx, dx, dx), 0.9)
    shp = _cell_shape(nn)
    rng = np.random.default_rng(seed)
    slab = np.zeros(shp, dtype=bool)
    z0, z1 = (12 * n) // 32, (20 * n) // 32
    slab[z0:z1, :, :] = True
    eps = np.where(slab, YIG_EPS, 1.0)
    Ms = np.where(slab, YIG_MS, 0.0)
    alpha = np.where(slab, YIG_ALPHA, 0.0)
    gamma = np.where(slab, YIG_GAMMA, 0.0)
    tx, ty, tz = _tilted_z(rng, shp)
    mx, my, mz = (np.where(slab, Ms * c, 0.0) for c in (tx, ty, tz))
    tp = 200 * dt
    src = Source(SRC_POINT_J, 0, n // 4, n // 2, n // 2, amp=1e9, f0=5e9, tp=tp, t0=3 * tp)
    return Workload(
        name=f"yig_slab_{n}", n=nn, d=(dx, dx, dx), dt=dt, bc=(PEC, PEC, PEC),
        tol=1e-10, max_iter=64, h0=(0.0, 0.0, 1e5), eps_r=eps, sigma=np.zeros(shp),
        mu_r=np.ones(shp), Ms=Ms, alpha=alpha, gamma=gamma, m_cells=(mx, my, mz),
        sources=[src], steps=steps)


def waveguide(seed: int = 1, steps: int = 5000, n=(128, 128, 512), dx: float = 2e-4,
              tol: float = 1e-6, amp: float = 1e7) -> Workload:
    """Rectangular PEC guide with 10-cell z-PML ends and a YIG-like slab.

    At the default 128x128x512 size the slab covers x cells 32-95, y cells
    56-71, z cells 200-311 (64x16x112); it is scaled with the grid for smaller
    test sizes.  A TE10-shaped soft Jy plane source at z node 20 carries a
    10 GHz modulated Gaussian with Tp = 1/f0 and t0 = 3 Tp.  H0 = 1e5 A/m
    along z, M = z + 1% seeded tilt.  Cell size 0.2 mm: the 25.6 mm guide has
    its TE10 cutoff at 5.9 GHz and TE20 at 11.7 GHz, so 10 GHz is single-mode."""
    nx, ny, nz = n
    dt = cfl_dt((dx, dx, dx), 0.9)
    shp = _cell_shape(n)
    rng = np.random.default_rng(seed)
    sx0, sx1 = (32 * nx) // 128, (96 * nx) // 128
    sy0, sy1 = (56 * ny) // 128, (72 * ny) // 128
    sz0, sz1 = (200 * nz) // 512, (312 * nz) // 512
    slab = np.zeros(shp, dtype=bool)
    slab[sz0:sz1, sy0:sy1, sx0:sx1] = True
    eps = np.where(slab, YIG_EPS, 1.0)
    Ms = np.where(slab, YIG_MS, 0.0)
    alpha = np.where(slab, YIG_ALPHA, 0.0)
    gamma = np.where(slab, YIG_GAMMA, 0.0)
    tx, ty, tz = _tilted_z(rng, shp)
    mx, my, mz = (np.where(slab, Ms * c, 0.0) for c in (tx, ty, tz))
    f0 = 10e9
    tp = 1.0 / f0
    npml = 10 if nz >= 64 else max(2, nz // 8)
    zsrc = max(npml + 2, (20 * nz) // 512)
    src = Source(SRC_PLANE_J_TE10, 1, 0, 0, zsrc, amp=amp, f0=f0, tp=tp, t0=3 * tp)
    return Workload(
        name="waveguide_%dx%dx%d" % tuple(n), n=tuple(n), d=(dx, dx, dx), dt=dt,
        bc=(PEC, PEC, PML), pml_cells=npml, tol=tol, max_iter=64,
        h0=(0.0, 0.0, 1e5), eps_r=eps, sigma=np.zeros(shp), mu_r=np.ones(shp),
        Ms=Ms, alpha=alpha, gamma=gamma, m_cells=(mx, my, mz), sources=[src],
        steps=steps)


def air_guide(steps: int = 8000, nz: int = 600, f0: float = 10.5e9, tp: Optional[float] = None) -> Workload:
    """Air-filled rectangular guide of the paper's Sec. 5.2.1: W = 14.95 mm,
    h = 10.16 mm (75 x 51 cells), PEC side walls, 10-cell PML at both z ends
    (the paper instead closes one end with PEC and drives it there).  A TE10
    soft Jy plane at z node 20 carries a modulated Gaussian: by default the
    paper's pulse (f0 = 10.5 GHz, Tp = one period, t0 = 3 Tp); a long tp gives
    a narrow-band drive at f0.  TE10 cutoff c/(2W) = 10.03 GHz."""
    W, h = 14.95e-3, 10.16e-3
    n = (75, 51, nz)
    d = (W / n[0], h / n[1], W / n[0])
    dt = cfl_dt(d, 0.9)
    shp = _cell_shape(n)
    tp = 1.0 / f0 if tp is None else tp
    src = Source(SRC_PLANE_J_TE10, 1, 0, 0, 20, amp=1e7, f0=f0, tp=tp, t0=3 * tp)
    return Workload(
        name="air_guide_75x51x%d" % nz, n=n, d=d, dt=dt, bc=(PEC, PEC, PML), pml_cells=10,
        tol=1e-6, max_iter=64, h0=(0.0, 0.0, 0.0), eps_r=np.ones(shp), sigma=np.zeros(shp),
        mu_r=np.ones(shp), Ms=np.zeros(shp), alpha=np.zeros(shp), gamma=np.zeros(shp),
        m_cells=None, sources=[src], steps=steps)


def tunable_filter(n: int, h0: float, steps: int = 2000, seed: int = 0, tol: float = 1e-6) -> Workload:
    """One instance of the bias sweep: an n^3 PEC box of 1 um cells with a
    centred YIG-like slab (Ms 1.4e5 A/m, alpha 0.005, |gamma| 1.76e11,
    eps_r 15) over the middle quarter of z, bias h0 along z, M = z + 1% seeded
    tilt, and a 5 GHz Gaussian Jx point source near one corner of the box."""
    nn = (n, n, n)
    dx = 1e-6
    dt = cfl_dt((dx, dx, dx), 0.9)
    shp = _cell_shape(nn)
    rng = np.random.default_rng(seed)
    slab = np.zeros(shp, dtype=bool)
    slab[(3 * n) // 8:(5 * n) // 8, :, :] = True
    Ms = np.where(slab, YIG_MS, 0.0)
    tx, ty, tz = _tilted_z(rng, shp)
    mx, my, mz = (np.where(slab, Ms * c, 0.0) for c in (tx, ty, tz))
    f0 = 5e9
    tp = 200 * dt
    src = Source(SRC_POINT_J, 0, n // 4, n // 2, n // 2, amp=1e9, f0=f0, tp=tp, t0=3 * tp)
    return Workload(
        name=f"filter_{n}_h{h0:.0f}", n=nn, d=(dx, dx, dx), dt=dt, bc=(PEC, PEC, PEC), tol=tol, max_iter=64,
        h0=(0.0, 0.0, float(h0)), eps_r=np.where(slab, YIG_EPS, 1.0), sigma=np.zeros(shp), mu_r=np.ones(shp),
        Ms=Ms, alpha=np.where(slab, YIG_ALPHA, 0.0), gamma=np.where(slab, YIG_GAMMA, 0.0),
        m_cells=(mx, my, mz), sources=[src], steps=steps)


def bias_sweep(count: int = 256, seed: int = 3, sizes=(32, 48, 64, 96)) -> List[Tuple[int, float, int]]:
    """The batched bias sweep as (n, h0, seed) per instance (build each with
    tunable_filter, one at a time): sizes drawn from `sizes`, bias uniform in
    [5e4, 2e5] A/m along z, each instance with its own seed."""
    rng = np.random.default_rng(seed)
    n = rng.choice(np.asarray(sizes), size=count)
    h0 = rng.uniform(5e4, 2e5, size=count)
    return [(int(n[q]), float(h0[q]), seed * 1000 + q) for q in range(count)]


def stress(seed: int = 2, steps: int = 1000, n: int = 512, tol: float = 1e-6) -> Workload:
    """n^3 PEC box, dx = 1e-6 m; centred (n/2)^3 magnetic block with seeded
    uniformly random unit M directions times Ms = 1.4e5 A/m, alpha = 0.01;
    eps_r ~ U[1, 12] per cell; sigma = 0; H0 = 1e5 A/m along z; no source."""
    nn = (n, n, n)
    dx = 1e-6
    dt = cfl_dt((dx, dx, dx), 0.9)
    shp = _cell_shape(nn)
    rng = np.random.default_rng(seed)
    eps = rng.uniform(1.0, 12.0, size=shp)
    blk = np.zeros(shp, dtype=bool)
    a, b = n // 4, n // 4 + n // 2
    blk[a:b, a:b, a:b] = True
    Ms = np.where(blk, YIG_MS, 0.0)
    alpha = np.where(blk, 0.01, 0.0)
    gamma = np.where(blk, YIG_GAMMA, 0.0)
    v = rng.normal(size=(3,) + shp)
    v /= np.linalg.norm(v, axis=0, keepdims=True)
    mx, my, mz = (np.where(blk, Ms * v[c], 0.0) for c in range(3))
    return Workload(
        name=f"stress_{n}", n=nn, d=(dx, dx, dx), dt=dt, bc=(PEC, PEC, PEC),
        tol=tol, max_iter=64, h0=(0.0, 0.0, 1e5), eps_r=eps, sigma=np.zeros(shp),
        mu_r=np.ones(shp), Ms=Ms, alpha=alpha, gamma=gamma, m_cells=(mx, my, mz),
        sources=[], steps=steps)


def convergence(n: int, order: int = 2, tol: float = 1e-10) -> Workload:
    """The paper's coupled convergence problem (Sec. 5.1): periodic cube of
    side 0.1 m centred at the origin, CFL 0.9, cosine E and H of vacuum
    impedance, Gaussian bumps in sigma, eps, Ms, alpha, |gamma|, M = Ms xhat,
    no bias.  32/64/128 cells run 5/10/20 steps to the same physical time."""
    L = 0.1
    nn = (n, n, n)
    dx = L / n
    dt = cfl_dt((dx, dx, dx), 0.9)
    xc = -L / 2 + (np.arange(n) + 0.5) * dx          # cell centres
    Z, Y, X = np.meshgrid(xc, xc, xc, indexing="ij")
    g = np.exp(-1000.0 * (X * X + Y * Y + Z * Z))
    sigma = 0.1 * g
    eps = 1.0 + g
    Ms = 1e4 * (1.0 + g)
    alpha = 0.5 * (1.0 + g)
    gamma = 1.759e11 * (1.0 + g)
    m_cells = (Ms.copy(), np.zeros_like(Ms), np.zeros_like(Ms))
    nodes = -L / 2 + np.arange(n + 1) * dx
    half = -L / 2 + (np.arange(n) + 0.5) * dx
    amp = 1e6
    eta = 120.0 * math.pi

    def on(ax):
        # ax: per axis (x, y, z) coordinate vectors -> meshgrid ordered (z, y, x)
        return np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")

    fields = {}
    Zz, Yy, Xx = on((half, nodes, nodes))            # Ex at (i+1/2, j, k)
    fields[0] = (amp * np.cos(20 * math.pi * Zz)).ravel()
    Zz, Yy, Xx = on((nodes, half, nodes))            # Ey
    fields[1] = (amp * np.cos(20 * math.pi * Xx)).ravel()
    Zz, Yy, Xx = on((nodes, nodes, half))            # Ez
    fields[2] = (amp * np.cos(20 * math.pi * Yy)).ravel()
    Zz, Yy, Xx = on((nodes, half, half))             # Hx at (i, j+1/2, k+1/2)
    fields[3] = (amp / eta * np.cos(20 * math.pi * Yy)).ravel()
    Zz, Yy, Xx = on((half, nodes, half))             # Hy
    fields[4] = (amp / eta * np.cos(20 * math.pi * Zz)).ravel()
    Zz, Yy, Xx = on((half, half, nodes))             # Hz
    fields[5] = (amp / eta * np.cos(20 * math.pi * Xx)).ravel()
    steps = {32: 5, 64: 10, 128: 20}.get(n, max(1, (5 * n) // 32))
    return Workload(
        name=f"convergence_{n}", n=nn, d=(dx, dx, dx), dt=dt,
        bc=(PERIODIC, PERIODIC, PERIODIC), order=order, tol=tol, max_iter=64,
        h0=(0.0, 0.0, 0.0), eps_r=eps, sigma=sigma, mu_r=np.ones_like(eps), Ms=Ms,
        alpha=alpha, gamma=gamma, m_cells=m_cells, sources=[], fields=fields,
        steps=steps)


def random_small(seed: int, n=(6, 5, 7), bc=(PEC, PEC, PEC), pml_cells: int = 0,
                 magnetic: bool = True, sources: bool = True, order: int = 2,
                 tol: float = 1e-10, dx=(1e-6, 1.3e-6, 0.8e-6), hard: bool = False,
                 pml_gap: int = 1) -> Workload:
    """Small randomised problem for parity tests: random eps_r in [1, 4],
    sigma in [0, 50) S/m, mu_r in [1, 2] where non-magnetic, a random magnetic
    blob (kept out of PML slabs and the pml_gap cell layers next to them),
    random initial E and H, random bias and point/plane (optionally hard)
    sources."""
    rng = np.random.default_rng(seed)
    shp = _cell_shape(n)
    dt = cfl_dt(dx, 0.9)
    eps = rng.uniform(1.0, 4.0, size=shp)
    sigma = rng.uniform(0.0, 50.0, size=shp)
    Ms = np.zeros(shp)
    if magnetic:
        blob = rng.uniform(size=shp) < 0.5
        if pml_cells:
            blob[:pml_cells + pml_gap] = False
            blob[n[2] - pml_cells - pml_gap:] = False
        Ms = np.where(blob, rng.uniform(0.5e5, 1.5e5, size=shp), 0.0)
    mu = np.where(Ms > 0, 1.0, rng.uniform(1.0, 2.0, size=shp))
    if pml_cells:
        for sl in (slice(0, pml_cells), slice(n[2] - pml_cells, n[2])):
            eps[sl] = 1.0
            sigma[sl] = 0.0
            mu[sl] = 1.0
    alpha = rng.uniform(0.001, 0.2, size=shp)
    # 30x the YIG gyromagnetic ratio: visible precession within a few steps
    gamma = rng.uniform(1.0e11, 2.0e11, size=shp) * 30.0
    v = rng.normal(size=(3,) + shp)
    mcells = tuple(v[c] * Ms for c in range(3))
    fields = {}
    for fid in range(6):
        scale = 1e3 if fid < 3 else 3.0
        fields[fid] = rng.normal(size=field_size(fid, n)) * scale
    srcs = []
    if sources:
        srcs.append(Source(SRC_POINT_J, int(rng.integers(0, 3)), 1, 1, 1, amp=1e8,
                           f0=3e12, tp=20 * dt, t0=30 * dt))
        srcs.append(Source(SRC_PLANE_J_TE10, 1, 0, 0, (pml_cells + 1) if pml_cells else 2,
                           amp=5e7, f0=2e12, tp=10 * dt, t0=15 * dt))
    if hard:
        srcs.append(Source(SRC_HARD_E, 2, 2, 2, 1, amp=3e3, f0=1e12, tp=10 * dt, t0=5 * dt))
        srcs.append(Source(SRC_HARD_H, 0, 2, 1, 2, amp=2.0, f0=1e12, tp=10 * dt, t0=5 * dt))
    h0 = tuple(rng.uniform(-1e5, 1e5, size=3))
    return Workload(
        name=f"random_small_{seed}", n=tuple(n), d=tuple(dx), dt=dt, bc=tuple(bc),
        pml_cells=pml_cells, order=order, tol=tol, max_iter=64, h0=h0, eps_r=eps,
        sigma=sigma, mu_r=mu, Ms=Ms, alpha=alpha, gamma=gamma, m_cells=mcells,
        sources=srcs, fields=fields, steps=6)


__all__ = [
    "Workload", "Source", "cfl_dt", "field_extent", "field_size", "yig_slab_32",
    "waveguide", "stress", "convergence", "random_small", "PERIODIC", "PEC", "PML",
    "SRC_POINT_J", "SRC_PLANE_J_TE10", "SRC_HARD_E", "SRC_HARD_H",
]


def filter_design(n=(64, 64, 256), seed: int = 0, steps: int = 2000, dx: float = 4e-4, npml: int = 10,
                  h0: float = 1e5, tol: float = 1e-10) -> Workload:
    """Design problem of the adjoint: a PEC guide (TE10 cutoff c/(2 nx dx),
    5.86 GHz at the default size) with npml-cell z-PML ends; a YIG-like slab
    (eps_r 15) on z cells [3nz/8, 5nz/8) over the centred nx/2 x ny/8
    cross-section; eps_r ~ U[1, 12] on the rest of the centred
    nx/2 x ny/2 x nz/4 design region; bias h0 along y with M = y + 1% seeded
    tilt; a 10 GHz TE10 soft Jy plane source at z = max(npml + 2, 20 nz/256);
    the flux loss through z node plane min(230 nz/256, nz - npml - 2)."""
    nx, ny, nz = n
    shp = _cell_shape(n)
    d = (dx, dx, dx)
    dt = cfl_dt(d, 0.9)
    rng = np.random.default_rng(seed)
    z0, z1 = (3 * nz) // 8, (5 * nz) // 8
    x0, x1 = nx // 4, (3 * nx) // 4
    hy = max(1, ny // 16)
    slab = np.zeros(shp, dtype=bool)
    slab[z0:z1, ny // 2 - hy:ny // 2 + hy, x0:x1] = True
    eps = np.ones(shp)
    eps[z0:z1, ny // 4:(3 * ny) // 4, x0:x1] = rng.uniform(1.0, 12.0, size=(z1 - z0, (3 * ny) // 4 - ny // 4, x1 - x0))
    eps = np.where(slab, YIG_EPS, eps)
    Ms = np.where(slab, YIG_MS, 0.0)
    u1, u2, _ = _tilted_z(rng, shp)
    mx, my, mz = (np.where(slab, Ms * c, 0.0) for c in (u1, np.ones(shp), u2))
    f0 = 10e9
    src = Source(SRC_PLANE_J_TE10, 1, 0, 0, max(npml + 2, (20 * nz) // 256), amp=1e7, f0=f0, tp=1.0 / f0,
                 t0=3.0 / f0)
    return Workload(
        name=f"filter_design_{nx}x{ny}x{nz}", n=tuple(n), d=d, dt=dt, bc=(PEC, PEC, PML), pml_cells=npml,
        tol=tol, max_iter=64, h0=(0.0, float(h0), 0.0), eps_r=eps, sigma=np.zeros(shp), mu_r=np.ones(shp),
        Ms=Ms, alpha=np.where(slab, YIG_ALPHA, 0.0), gamma=np.where(slab, YIG_GAMMA, 0.0), m_cells=(mx, my, mz),
        sources=[src], steps=steps, flux_k=min((230 * nz) // 256, nz - npml - 2))

"""Discrete adjoint of the scheme (mmx_flux_gradient): d(time-integrated
Poynting flux through a z plane)/d eps_r per cell and d/d H0, checked
against central finite differences of the GPU path (FP64, h = 1e-4
relative, 20 seeded design cells and the bias components), against finite
differences of the FP64 CPU oracle on tiny grids, FP32 against FP64, through
torch.autograd, and on the full-size 64x64x256 filter geometry, first
without and then with its magnetised YIG slab."""
import numpy as np
import pytest
import torch

import oracle
import paper_2103_12819_b300 as mmx
import workloads as W
from paper_2103_12819_b300.adjoint import FluxLoss, FluxLossBias

pytestmark = pytest.mark.gpu


def _guide(n, dx, npml, zsrc, f0):
    """A PEC guide with z-PML ends and a TE10 soft Jy plane source."""
    d = (dx, dx, dx)
    dt = W.cfl_dt(d, 0.9)
    src = W.Source(W.SRC_PLANE_J_TE10, 1, 0, 0, zsrc, amp=1e7, f0=f0, tp=1.0 / f0, t0=3.0 / f0)
    return d, dt, src


def _solver(n, eps, prec, kind="gpu", npml=6, dx=1e-3, zsrc=8, f0=12e9):
    d, dt, src = _guide(n, dx, npml, zsrc, f0)
    if kind == "gpu":
        s = mmx.Solver(n, d, dt, (W.PEC, W.PEC, W.PML), npml, 2, 1e-10, 64, prec)
        s.set_path(mmx.PATH_PLAIN)
    else:
        s = oracle.Sim(n, d, dt, (W.PEC, W.PEC, W.PML), pml_cells=npml)
    s.set_materials(eps_r=eps)
    s.add_source(src.kind, src.comp, src.i, src.j, src.k, src.amp, src.f0, src.tp, src.t0)
    return s, dt, d


def _loss_gpu(n, eps, kp, nsteps, prec=mmx.FP64):
    s, _, _ = _solver(n, eps, prec)
    p = s.add_flux_plane(kp)
    s.step(nsteps)
    s.sync()
    return s.get_flux(p)[0]


N = (16, 12, 48)
KP, STEPS = 34, 200


def _eps(seed=7, n=N):
    rng = np.random.default_rng(seed)
    eps = np.ones((n[2], n[1], n[0]))
    eps[16:25, 3:10, 4:13] = rng.uniform(1.0, 4.0, size=(9, 7, 9))
    return eps


@pytest.fixture(scope="module")
def fp64_gradient():
    eps = _eps()
    s, _, _ = _solver(N, eps, mmx.FP64)
    loss, grad = s.flux_gradient(KP, STEPS, 15)
    s.close()
    return eps, loss, grad


def test_loss_equals_the_flux_monitor(fp64_gradient):
    eps, loss, _ = fp64_gradient
    assert abs(loss / _loss_gpu(N, eps, KP, STEPS) - 1) < 1e-12
    assert loss > 0


def test_adjoint_matches_central_differences(fp64_gradient):
    eps, loss, grad = fp64_gradient
    rng = np.random.default_rng(21)
    cells = [(int(k), int(j), int(i)) for k, j, i in zip(rng.integers(16, 25, 20), rng.integers(3, 10, 20),
                                                          rng.integers(4, 13, 20))]
    scale = np.abs(grad[16:25, 3:10, 4:13]).max()
    worst = 0.0
    for c in cells:
        h = 1e-4 * eps[c]
        e1, e2 = eps.copy(), eps.copy()
        e1[c] += h
        e2[c] -= h
        fd = (_loss_gpu(N, e1, KP, STEPS) - _loss_gpu(N, e2, KP, STEPS)) / (2 * h)
        err = abs(grad[c] - fd) / max(abs(fd), 1e-3 * scale)
        worst = max(worst, err)
    print("adjoint vs central differences, 20 cells: worst relative error %.2e (max |g| %.3e)" % (worst, scale))
    assert worst < 1e-4


def test_adjoint_matches_oracle_finite_differences():
    """Finite differences of the FP64 CPU oracle (loss evaluated from its
    fields every step) on a tiny guide agree with the GPU adjoint."""
    n, kp, steps = (8, 6, 24), 17, 60
    eps = np.ones((n[2], n[1], n[0]))
    eps[8:12, 1:5, 2:6] = np.random.default_rng(3).uniform(1.0, 3.0, size=(4, 4, 4))
    kw = dict(npml=3, dx=2e-3, zsrc=5, f0=9e9)
    s, dt, d = _solver(n, eps, mmx.FP64, **kw)
    _, grad = s.flux_gradient(kp, steps, 8)

    def oracle_loss(e):
        o, dt_, d_ = _solver(n, e, None, kind="oracle", **kw)
        L = 0.0
        for _ in range(steps):
            o.step(1)
            ex = o.get_field(0).reshape(n[2] + 1, n[1] + 1, n[0])[kp]
            ey = o.get_field(1).reshape(n[2] + 1, n[1], n[0] + 1)[kp]
            hx = o.get_field(3).reshape(n[2], n[1], n[0] + 1)
            hy = o.get_field(4).reshape(n[2], n[1] + 1, n[0])
            P = np.sum(ex * 0.5 * (hy[kp - 1] + hy[kp])) - np.sum(ey * 0.5 * (hx[kp - 1] + hx[kp]))
            L += dt_ * P * d_[0] * d_[1]
        o.close()
        return L

    for c in [(9, 2, 3), (10, 3, 4), (11, 1, 5)]:
        h = 1e-4 * eps[c]
        e1, e2 = eps.copy(), eps.copy()
        e1[c] += h
        e2[c] -= h
        fd = (oracle_loss(e1) - oracle_loss(e2)) / (2 * h)
        print("cell %s: adjoint %.6e oracle FD %.6e" % (c, grad[c], fd))
        assert abs(grad[c] - fd) <= 1e-4 * abs(fd)


def test_fp32_adjoint_close_to_fp64(fp64_gradient):
    eps, loss64, g64 = fp64_gradient
    s, _, _ = _solver(N, eps, mmx.FP32)
    loss32, g32 = s.flux_gradient(KP, STEPS, 15)
    assert abs(loss32 / loss64 - 1) < 1e-4
    region = (slice(16, 25), slice(3, 10), slice(4, 13))
    rel = np.linalg.norm(g32[region] - g64[region]) / np.linalg.norm(g64[region])
    print("FP32 adjoint vs FP64 adjoint over the design region: %.2e" % rel)
    assert rel < 1e-3


def test_autograd_function(fp64_gradient):
    eps, loss, grad = fp64_gradient
    t = torch.tensor(eps, dtype=torch.float64, requires_grad=True)
    make = lambda e: _solver(N, e, mmx.FP64)[0]
    L = FluxLoss.apply(t, make, KP, STEPS, 15)
    (2.0 * L).backward()
    assert abs(L.item() / loss - 1) < 1e-12
    np.testing.assert_allclose(t.grad.numpy(), 2.0 * grad, rtol=1e-12, atol=0)


def test_adjoint_refuses_uncovered_grids():
    w = W.yig_slab_32(steps=2, n=16)
    w.order = 1                                       # magnetic, first-order scheme
    s = mmx.from_workload(w, prec=mmx.FP64)
    with pytest.raises(mmx.MMXError):
        s.flux_gradient(8, 4)
    w = W.random_small(41, n=(6, 5, 7), bc=(W.PERIODIC, W.PEC, W.PEC), magnetic=False, tol=1e-6)
    s = mmx.from_workload(w, prec=mmx.FP64)
    with pytest.raises(mmx.MMXError):
        s.flux_gradient(3, 4)


def test_full_size_filter_geometry_fp32():
    """The 64x64x256 filter (PEC sides, 10-cell PML ends) without its slab,
    eps_r uniform in [1, 12] over the 32x32x64 design region, 2000 FP32 steps,
    flux through z = 230, checkpoints every 45 steps: the FP32 gradient over
    the design region agrees with the FP64 one."""
    n = (64, 64, 256)
    rng = np.random.default_rng(4)
    eps = np.ones((n[2], n[1], n[0]))
    eps[96:160, 16:48, 16:48] = rng.uniform(1.0, 12.0, size=(64, 32, 32))
    kw = dict(npml=10, dx=2e-4, zsrc=20, f0=10e9)
    import time
    out = {}
    for prec in (mmx.FP32, mmx.FP64):
        s, _, _ = _solver(n, eps, prec, **kw)
        t0 = time.perf_counter()
        out[prec] = s.flux_gradient(230, 2000, 45)
        print("full-size adjoint %s: %.2f s" % ("FP32" if prec == mmx.FP32 else "FP64", time.perf_counter() - t0))
        s.close()
    region = (slice(96, 160), slice(16, 48), slice(16, 48))
    g32, g64 = out[mmx.FP32][1][region], out[mmx.FP64][1][region]
    rel = np.linalg.norm(g32 - g64) / np.linalg.norm(g64)
    print("full-size FP32 vs FP64 gradient: %.2e, loss %.6e / %.6e" % (rel, out[mmx.FP32][0], out[mmx.FP64][0]))
    assert out[mmx.FP64][0] > 0
    assert rel < 1e-2


# ---------------------------------------------------------------- magnetic
#
# The ferrite-loaded design problem (workloads.filter_design) at test sizes:
# the adjoint now runs through the H/M half steps (implicit-function
# transpose of the converged trapezoidal LLG solve) and also returns dL/dH0.

MN = (16, 12, 48)
MKW = dict(dx=1.6e-3, npml=6)
MSTEPS = 200


def _mag_workload(n=MN, eps=None, h0=None, **kw):
    w = W.filter_design(n, **{**MKW, **kw})
    if eps is not None:
        w.eps_r = eps
    if h0 is not None:
        w.h0 = tuple(float(v) for v in h0)
    return w


def _mag_loss_gpu(w, nsteps, prec=mmx.FP64):
    s = mmx.from_workload(w, prec=prec, path=mmx.PATH_PLAIN)
    p = s.add_flux_plane(w.flux_k)
    s.step(nsteps)
    s.sync()
    L = s.get_flux(p)[0]
    s.close()
    return L


@pytest.fixture(scope="module")
def mag_gradient():
    w = _mag_workload()
    s = mmx.from_workload(w, prec=mmx.FP64, path=mmx.PATH_PLAIN)
    loss, grad, gh0 = s.flux_gradient(w.flux_k, MSTEPS, 15, with_h0=True)
    st = s.get_stats()
    s.close()
    return w, loss, grad, gh0, st


def test_magnetic_loss_equals_the_flux_monitor(mag_gradient):
    w, loss, _, gh0, st = mag_gradient
    assert abs(loss / _mag_loss_gpu(w, MSTEPS) - 1) < 1e-12
    assert loss != 0 and np.all(np.isfinite(gh0))
    print("magnetic adjoint: loss %.6e, dL/dH0 %s, forward iterations %d-%d" %
          (loss, gh0, st["iters_min"], st["iters_max"]))


def test_magnetic_adjoint_matches_central_differences(mag_gradient):
    """20 seeded cells of the design region (slab cells among them) and the
    three bias components, central differences of the GPU path, h = 1e-4
    relative (1e-4 |H0| for the bias)."""
    w, loss, grad, gh0, _ = mag_gradient
    nx, ny, nz = MN
    z0, z1, y0, y1, x0, x1 = 3 * nz // 8, 5 * nz // 8, ny // 4, 3 * ny // 4, nx // 4, 3 * nx // 4
    rng = np.random.default_rng(5)
    cells = [(int(k), int(j), int(i)) for k, j, i in zip(rng.integers(z0, z1, 16), rng.integers(y0, y1, 16),
                                                          rng.integers(x0, x1, 16))]
    cells += [(z0, ny // 2, nx // 2), (z1 - 1, ny // 2 - 1, x0), (z0 + 3, ny // 2, x1 - 1), ((z0 + z1) // 2, y0, x0)]
    scale = np.abs(grad[z0:z1, y0:y1, x0:x1]).max()
    worst = 0.0
    for c in cells:
        h = 1e-4 * w.eps_r[c]
        e1, e2 = w.eps_r.copy(), w.eps_r.copy()
        e1[c] += h
        e2[c] -= h
        fd = (_mag_loss_gpu(_mag_workload(eps=e1), MSTEPS) - _mag_loss_gpu(_mag_workload(eps=e2), MSTEPS)) / (2 * h)
        worst = max(worst, abs(grad[c] - fd) / max(abs(fd), 1e-3 * scale))
    print("magnetic adjoint vs central differences, 20 cells: worst relative error %.2e (max |g| %.3e)" %
          (worst, scale))
    assert worst < 1e-4
    h0 = np.array(w.h0)
    hb = 1e-4 * np.linalg.norm(h0)
    gscale = np.abs(gh0).max()
    for c in range(3):
        p1, p2 = h0.copy(), h0.copy()
        p1[c] += hb
        p2[c] -= hb
        fd = (_mag_loss_gpu(_mag_workload(h0=p1), MSTEPS) - _mag_loss_gpu(_mag_workload(h0=p2), MSTEPS)) / (2 * hb)
        err = abs(gh0[c] - fd) / max(abs(fd), 1e-3 * gscale)
        print("dL/dH0[%d]: adjoint %.6e central difference %.6e (rel %.1e)" % (c, gh0[c], fd, err))
        assert err < 1e-4


def test_magnetic_adjoint_matches_oracle_finite_differences():
    """Finite differences of the FP64 CPU oracle (loss from its fields every
    step) on the 8x6x24 design problem agree with the GPU adjoint, for eps_r
    of three cells (two in the slab) and for the bias."""
    n, steps = (8, 6, 24), 100
    kw = dict(dx=3.2e-3, npml=3)
    w = _mag_workload(n, **kw)
    s = mmx.from_workload(w, prec=mmx.FP64, path=mmx.PATH_PLAIN)
    _, grad, gh0 = s.flux_gradient(w.flux_k, steps, 10, with_h0=True)
    s.close()
    kp = w.flux_k

    def oracle_loss(wl):
        o = oracle.from_workload(wl)
        L = 0.0
        for _ in range(steps):
            o.step(1)
            ex = o.get_field(0).reshape(n[2] + 1, n[1] + 1, n[0])[kp]
            ey = o.get_field(1).reshape(n[2] + 1, n[1], n[0] + 1)[kp]
            hx = o.get_field(3).reshape(n[2], n[1], n[0] + 1)
            hy = o.get_field(4).reshape(n[2], n[1] + 1, n[0])
            P = np.sum(ex * 0.5 * (hy[kp - 1] + hy[kp])) - np.sum(ey * 0.5 * (hx[kp - 1] + hx[kp]))
            L += wl.dt * P * wl.d[0] * wl.d[1]
        o.close()
        return L

    for c in [(10, 2, 3), (12, 3, 4), (13, 1, 5)]:
        h = 1e-4 * w.eps_r[c]
        e1, e2 = w.eps_r.copy(), w.eps_r.copy()
        e1[c] += h
        e2[c] -= h
        fd = (oracle_loss(_mag_workload(n, eps=e1, **kw)) - oracle_loss(_mag_workload(n, eps=e2, **kw))) / (2 * h)
        print("cell %s (Ms %.0f): adjoint %.6e oracle FD %.6e" % (c, w.Ms[c], grad[c], fd))
        assert abs(grad[c] - fd) <= 1e-4 * abs(fd)
    h0 = np.array(w.h0)
    hb = 1e-4 * np.linalg.norm(h0)
    for c in range(3):
        p1, p2 = h0.copy(), h0.copy()
        p1[c] += hb
        p2[c] -= hb
        fd = (oracle_loss(_mag_workload(n, h0=p1, **kw)) - oracle_loss(_mag_workload(n, h0=p2, **kw))) / (2 * hb)
        print("dL/dH0[%d]: adjoint %.6e oracle FD %.6e" % (c, gh0[c], fd))
        assert abs(gh0[c] - fd) <= 1e-4 * max(abs(fd), 1e-3 * np.abs(gh0).max())


def test_magnetic_fp32_adjoint_close_to_fp64(mag_gradient):
    """FP32 at the paper's iteration tolerance 1e-6 (1e-10 sits below FP32's
    rounding of the LLG increments) against FP64 at 1e-10."""
    w, loss64, g64, h64, _ = mag_gradient
    s = mmx.from_workload(_mag_workload(tol=1e-6), prec=mmx.FP32, path=mmx.PATH_PLAIN)
    loss32, g32, h32 = s.flux_gradient(w.flux_k, MSTEPS, 15, with_h0=True)
    s.close()
    nx, ny, nz = MN
    region = (slice(3 * nz // 8, 5 * nz // 8), slice(ny // 4, 3 * ny // 4), slice(nx // 4, 3 * nx // 4))
    rel = np.linalg.norm(g32[region] - g64[region]) / np.linalg.norm(g64[region])
    relh = np.linalg.norm(h32 - h64) / np.linalg.norm(h64)
    print("magnetic FP32 vs FP64: loss %.2e, eps gradient %.2e, H0 gradient %.2e" %
          (abs(loss32 / loss64 - 1), rel, relh))
    assert abs(loss32 / loss64 - 1) < 1e-3
    assert rel < 1e-2 and relh < 1e-2


def test_magnetic_autograd_function(mag_gradient):
    w, loss, grad, gh0, _ = mag_gradient
    t = torch.tensor(w.eps_r, dtype=torch.float64, requires_grad=True)
    b = torch.tensor(w.h0, dtype=torch.float64, requires_grad=True)

    def make(e, h):
        return mmx.from_workload(_mag_workload(eps=e, h0=h), prec=mmx.FP64, path=mmx.PATH_PLAIN)

    L = FluxLossBias.apply(t, b, make, w.flux_k, MSTEPS, 15)
    (3.0 * L).backward()
    assert abs(L.item() / loss - 1) < 1e-12
    np.testing.assert_allclose(t.grad.numpy(), 3.0 * grad, rtol=1e-12, atol=0)
    np.testing.assert_allclose(b.grad.numpy(), 3.0 * gh0, rtol=1e-12, atol=0)


def test_full_size_magnetic_filter():
    """The 64x64x256 ferrite-loaded filter: YIG slab on z 96-160 over the
    centred 32x8 cross-section, bias 1e5 A/m, eps_r in [1, 12] on the 32x32x64
    design region, 2000 steps, flux through z = 230, checkpoints every 45.
    FP32 and FP64 gradients (eps_r and H0) agree; 20 seeded design cells
    (slab cells among them, h = 1e-4 eps_r) and the three H0 components
    (h = 1e-4 |H0|) match central differences of the FP64 forward: the FP64
    adjoint to 1e-4 relative, the FP32 one to 1e-3."""
    import time
    w = W.filter_design()
    out = {}
    for prec in (mmx.FP32, mmx.FP64):
        s = mmx.from_workload(W.filter_design(tol=1e-6) if prec == mmx.FP32 else w, prec=prec, path=mmx.PATH_PLAIN)
        t0 = time.perf_counter()
        out[prec] = s.flux_gradient(w.flux_k, w.steps, 45, with_h0=True)
        print("full-size magnetic adjoint %s: %.2f s" % ("FP32" if prec == mmx.FP32 else "FP64",
                                                         time.perf_counter() - t0))
        s.close()
    region = (slice(96, 160), slice(16, 48), slice(16, 48))
    g32, g64 = out[mmx.FP32][1][region], out[mmx.FP64][1][region]
    rel = np.linalg.norm(g32 - g64) / np.linalg.norm(g64)
    h32, h64 = out[mmx.FP32][2], out[mmx.FP64][2]
    print("full-size magnetic FP32 vs FP64: eps gradient %.2e, H0 gradient %s vs %s, loss %.6e / %.6e" %
          (rel, h32, h64, out[mmx.FP32][0], out[mmx.FP64][0]))
    assert rel < 1e-2
    assert np.linalg.norm(h32 - h64) <= 1e-2 * np.linalg.norm(h64)
    # 20 seeded design cells: 4 drawn from the slab (z 96-159, y 28-35,
    # x 16-47), 16 from the whole design region (some of them in the slab too)
    rng = np.random.default_rng(20)
    cells = [(int(rng.integers(96, 160)), int(rng.integers(28, 36)), int(rng.integers(16, 48))) for _ in range(4)]
    while len(cells) < 20:
        c = (int(rng.integers(96, 160)), int(rng.integers(16, 48)), int(rng.integers(16, 48)))
        if c not in cells:
            cells.append(c)
    gmax = np.abs(g64).max()
    worst = {mmx.FP64: 0.0, mmx.FP32: 0.0}
    for c in cells:
        h = 1e-4 * w.eps_r[c]
        Ls = []
        for sg in (1, -1):
            wl = W.filter_design()
            wl.eps_r = w.eps_r.copy()
            wl.eps_r[c] += sg * h
            Ls.append(_mag_loss_gpu(wl, w.steps))
        fd = (Ls[0] - Ls[1]) / (2 * h)
        scale = max(abs(fd), 1e-3 * gmax)
        for prec in (mmx.FP64, mmx.FP32):
            worst[prec] = max(worst[prec], abs(out[prec][1][c] - fd) / scale)
        print("full size, cell %s (Ms %.0f): adjoint %.6e (FP32 %.6e) central difference %.6e"
              % (c, w.Ms[c], out[mmx.FP64][1][c], out[mmx.FP32][1][c], fd))
    assert sum(1 for c in cells if w.Ms[c] > 0) >= 4
    print("20 cells, worst relative error against central differences: FP64 %.2e, FP32 %.2e"
          % (worst[mmx.FP64], worst[mmx.FP32]))
    assert worst[mmx.FP64] <= 1e-4 and worst[mmx.FP32] <= 1e-3
    # the bias: central differences in each component of H0
    hb = 1e-4 * np.linalg.norm(w.h0)
    for a in range(3):
        Ls = []
        for sg in (1, -1):
            wl = W.filter_design()
            h0 = list(wl.h0)
            h0[a] += sg * hb
            wl.h0 = tuple(h0)
            Ls.append(_mag_loss_gpu(wl, w.steps))
        fd = (Ls[0] - Ls[1]) / (2 * hb)
        scale = max(abs(fd), 1e-3 * np.abs(h64).max())
        print("full size, dL/dH0_%d: adjoint %.6e (FP32 %.6e) central difference %.6e" % (a, h64[a], h32[a], fd))
        assert abs(h64[a] - fd) <= 1e-4 * scale and abs(h32[a] - fd) <= 1e-3 * scale

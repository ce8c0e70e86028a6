"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the
mathematics -- closed forms, exact discrete invariants, printed worked
numbers and brute force on tiny inputs -- never against the oracle itself.

Each test names what a plausible mistake in the oracle would break.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W
from conftest import C0, EPS0, MU0, positions, rel_l2

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_kv(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                out[k] = float(v)
    return out


def _vacuum_sim(n, d, dt, bc, **kw):
    s = oracle.Sim(n, d, dt, bc, **kw)
    s.set_materials()
    return s


# --------------------------------------------------------------- worked numbers

def test_golden_dt_convention():
    """Sec. 5.2.1 prints dt = 77.87961902 fs for 512x4x512 cells at CFL 0.8;
    the CFL rule of the workload generator reproduces it to 2e-5."""
    g = _golden_kv("closed_forms.txt")
    d = (g["dt_W_mm"] * 1e-3 / g["dt_cells_x"], g["dt_h_mm"] * 1e-3 / g["dt_cells_y"],
         g["dt_L_mm"] * 1e-3 / g["dt_cells_z"])
    dt = W.cfl_dt(d, g["dt_cfl"])
    assert abs(dt * 1e15 / g["dt_fs"] - 1) < 2e-5


def _kittel_f(H0, Ms, frac=0.0):
    """In-plane thin-film FMR in SI: f = gamma mu0/(2 pi) sqrt((H0 + f Ms)(H0 + Ms))."""
    return 1.76e11 * MU0 / (2 * math.pi) * math.sqrt((H0 + frac * Ms) * (H0 + Ms))


def test_golden_kittel_formula():
    """Eq. kittel worked example (Sec. 5.2.2): H0 = 2890 Oe, 4 pi Ms = 1750 G
    gives 10.25 GHz.  Pins the SI form of the closed form used by P7."""
    g = _golden_kv("closed_forms.txt")
    f = _kittel_f(g["kittel_H0_A_per_m"], g["kittel_Ms_A_per_m"])
    assert abs(f / 1e9 - g["kittel_fFMR_GHz"]) < 0.01
    assert abs(g["kittel_H0_Oe"] * 1e3 / (4 * math.pi) / g["kittel_H0_A_per_m"] - 1) < 1e-4
    assert abs(g["kittel_4piMs_G"] * 1e3 / (4 * math.pi) / g["kittel_Ms_A_per_m"] - 1) < 1e-4


def test_golden_waveguide_cutoff():
    g = _golden_kv("closed_forms.txt")
    assert abs(C0 / (2 * g["waveguide_W_mm"] * 1e-3) / 1e9 - g["waveguide_fc_GHz"]) < 0.005


# ----------------------------------------------------- a1: materials, initial M

def _brute_edge_mean(cell, c, n, bc):
    """Mean of the existing cells around every edge of component c, by
    explicit enumeration of all cells (tiny grids only)."""
    ext = [n[a] + (0 if a == c else 1) for a in range(3)]
    out = np.zeros(ext[::-1])
    for k in range(ext[2]):
        for j in range(ext[1]):
            for i in range(ext[0]):
                ix = (i, j, k)
                vals = []
                for cz in range(n[2]):
                    for cy in range(n[1]):
                        for cx in range(n[0]):
                            cc = (cx, cy, cz)
                            ok = True
                            for a in range(3):
                                if a == c:
                                    ok &= cc[a] == ix[a]
                                else:
                                    cand = {ix[a] - 1, ix[a]}
                                    if bc[a] == W.PERIODIC:
                                        cand = {v % n[a] for v in cand}
                                    ok &= cc[a] in cand
                            if ok:
                                vals.append(cell[cz, cy, cx])
                out[k, j, i] = np.mean(vals)
    return out.ravel()


def _brute_face_mean(cell, dd, n, bc):
    ext = [n[a] + (1 if a == dd else 0) for a in range(3)]
    out = np.zeros(ext[::-1])
    for k in range(ext[2]):
        for j in range(ext[1]):
            for i in range(ext[0]):
                ix = [i, j, k]
                vals = []
                for o in (-1, 0):
                    cc = list(ix)
                    cc[dd] = ix[dd] + o
                    if bc[dd] == W.PERIODIC:
                        cc[dd] %= n[dd]
                    elif not (0 <= cc[dd] < n[dd]):
                        continue
                    vals.append(cell[cc[2], cc[1], cc[0]])
                out[k, j, i] = np.mean(vals)
    return out.ravel()


@pytest.mark.parametrize("bc", [(W.PEC, W.PEC, W.PEC), (W.PERIODIC, W.PEC, W.PERIODIC)])
def test_a1_material_averaging_brute_force(bc):
    """Sec. 3.1: eps, sigma on edges and mu, Ms, alpha, gamma on faces are
    second-order (arithmetic) averages of the adjacent cell centres."""
    n = (3, 4, 2)
    rng = np.random.default_rng(5)
    cells = [rng.uniform(1, 3, size=(n[2], n[1], n[0])) for _ in range(6)]
    s = oracle.Sim(n, (1e-6, 1e-6, 1e-6), 1e-16, bc)
    s.set_materials(*cells)
    for c in range(3):
        np.testing.assert_allclose(s.get_material(c), _brute_edge_mean(cells[0], c, n, bc), rtol=1e-15)
        np.testing.assert_allclose(s.get_material(3 + c), _brute_edge_mean(cells[1], c, n, bc), rtol=1e-15)
        for m, which in ((2, 6), (3, 9), (4, 12), (5, 15)):
            np.testing.assert_allclose(s.get_material(which + c), _brute_face_mean(cells[m], c, n, bc),
                                       rtol=1e-15)


def test_a1_initial_m_is_renormalised_face_average():
    """Sec. 3.1: M parsed at cell centres, averaged to faces, |M| = Ms there."""
    n = (4, 3, 5)
    bc = (W.PEC, W.PERIODIC, W.PEC)
    rng = np.random.default_rng(7)
    shp = (n[2], n[1], n[0])
    Ms = np.where(rng.uniform(size=shp) < 0.6, rng.uniform(1e4, 2e5, size=shp), 0.0)
    mc = [rng.normal(size=shp) * 1e5 for _ in range(3)]
    s = oracle.Sim(n, (1e-6,) * 3, 1e-16, bc)
    s.set_materials(Ms=Ms)
    s.set_M_cells(*mc)
    for fam in range(3):
        Msf = _brute_face_mean(Ms, fam, n, bc)
        avg = np.stack([_brute_face_mean(mc[c], fam, n, bc) for c in range(3)])
        nrm = np.linalg.norm(avg, axis=0)
        mag = Msf > 0
        for c in range(3):
            got = s.get_field(6 + 3 * fam + c)
            want = np.where(mag, avg[c] * Msf / np.where(nrm > 0, nrm, 1), 0.0)
            np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-9)


# ------------------------------------------------ P1/P2: Yee dispersion, cavity

def _set_fields(s, n, d, fn):
    for fid in range(6):
        X, Y, Z = positions(fid, n, d)
        s.set_field(fid, fn(fid, X, Y, Z).ravel())


def test_p1_periodic_plane_wave_is_exact_discrete_eigenmode():
    """Vacuum, periodic box: a Yee eigenmode advances by exactly omega*dt per
    step with sin(omega dt/2) = c dt sqrt(sum sin^2(k_i d_i/2)/d_i^2) -- the
    leapfrog H(n->n+1/2), E(n->n+1), H(n+1/2->n+1) of Sec. 3.2 with sigma = 0
    and Ms = 0.  Catches any error in curl signs/indices, the dt/2 factors,
    eps0/mu0 and periodic wrapping (anisotropic cells: transposed axes fail)."""
    n = (8, 6, 10)
    d = (1.0e-6, 1.3e-6, 0.9e-6)
    dt = W.cfl_dt(d, 0.95)
    L = np.array(n) * np.array(d)
    k = 2 * np.pi * np.array([1, 2, -1]) / L
    K = 2 / np.array(d) * np.sin(k * np.array(d) / 2)
    E0 = np.cross(K, [0.3, -1.0, 0.7])
    E0 *= 1e3 / np.linalg.norm(E0)
    om = 2 / dt * math.asin(C0 * dt * np.linalg.norm(K) / 2)
    Om = 2 * math.sin(om * dt / 2) / dt
    H0 = np.cross(K, E0) / (MU0 * Om)
    s = _vacuum_sim(n, d, dt, (W.PERIODIC,) * 3)

    def field(fid, X, Y, Z, t):
        ph = k[0] * X + k[1] * Y + k[2] * Z - om * t
        if fid < 3:
            return E0[fid] * np.cos(ph)
        return H0[fid - 3] * math.cos(om * dt / 2) * np.cos(ph)

    _set_fields(s, n, d, lambda f, X, Y, Z: field(f, X, Y, Z, 0.0))
    N = 300
    s.step(N)
    for fid in range(6):
        X, Y, Z = positions(fid, n, d)
        want = field(fid, X, Y, Z, N * dt).ravel()
        assert rel_l2(s.get_field(fid), want) < 1e-11, fid


def test_p2_pec_cavity_mode():
    """PEC cavity: the standing mode with k_i = m_i pi / L_i is an exact
    discrete eigenmode with the same dispersion relation; tangential E and
    normal H vanish on the walls (Sec. 3.2.3)."""
    n = (6, 5, 7)
    d = (1.1e-6, 0.9e-6, 1.0e-6)
    dt = W.cfl_dt(d, 0.9)
    L = np.array(n) * np.array(d)
    k = np.pi * np.array([1, 2, 1]) / L
    K = 2 / np.array(d) * np.sin(k * np.array(d) / 2)
    A = np.cross(K, [1.0, 0.2, -0.5])
    A *= 1e3 / np.linalg.norm(A)
    om = 2 / dt * math.asin(C0 * dt * np.linalg.norm(K) / 2)
    Om = 2 * math.sin(om * dt / 2) / dt
    B = -np.cross(K, A) / (MU0 * Om)
    s = _vacuum_sim(n, d, dt, (W.PEC,) * 3)

    def pattern(fid, X, Y, Z):
        cs = [np.cos(k[0] * X), np.cos(k[1] * Y), np.cos(k[2] * Z)]
        sn = [np.sin(k[0] * X), np.sin(k[1] * Y), np.sin(k[2] * Z)]
        a = fid % 3
        if fid < 3:      # E_a: cos along a, sin on the others
            return np.prod([cs[b] if b == a else sn[b] for b in range(3)], axis=0)
        return np.prod([sn[b] if b == a else cs[b] for b in range(3)], axis=0)

    _set_fields(s, n, d, lambda f, X, Y, Z: (A[f] * pattern(f, X, Y, Z)) if f < 3 else 0 * X)
    N = 257
    s.step(N)
    for fid in range(6):
        X, Y, Z = positions(fid, n, d)
        if fid < 3:
            want = A[fid] * pattern(fid, X, Y, Z) * math.cos(om * N * dt)
        else:
            want = B[fid - 3] * pattern(fid, X, Y, Z) * math.sin(om * N * dt) * math.cos(om * dt / 2)
        assert rel_l2(s.get_field(fid), want.ravel()) < 1e-11, fid


# ----------------------------------------------------------- P3: discrete energy

def _curl_e_faces(E, n, d):
    """(curl E) on the three face families, written out with numpy slicing."""
    nx, ny, nz = n
    Ex = E[0].reshape(nz + 1, ny + 1, nx)
    Ey = E[1].reshape(nz + 1, ny, nx + 1)
    Ez = E[2].reshape(nz, ny + 1, nx + 1)
    cx = (Ez[:, 1:, :] - Ez[:, :-1, :]) / d[1] - (Ey[1:, :, :] - Ey[:-1, :, :]) / d[2]
    cy = (Ex[1:, :, :] - Ex[:-1, :, :]) / d[2] - (Ez[:, :, 1:] - Ez[:, :, :-1]) / d[0]
    cz = (Ey[:, :, 1:] - Ey[:, :, :-1]) / d[0] - (Ex[:, 1:, :] - Ex[:, :-1, :]) / d[1]
    return [cx.ravel(), cy.ravel(), cz.ravel()]


@pytest.mark.parametrize("bc", [(W.PEC,) * 3, (W.PERIODIC, W.PEC, W.PERIODIC)])
def test_p3_discrete_energy_is_conserved(bc):
    """Lossless media, no source: W = 1/2 sum eps E^2 + 1/2 sum mu (H^2 -
    (dt/(2 mu) curl E)^2) is an exact invariant of the half-step leapfrog
    (H^n is the mean of H^(n+-1/2)).  Any wrong dt factor, curl sign or
    non-adjoint stencil pair breaks it."""
    n = (5, 6, 4)
    d = (1.0e-6, 1.2e-6, 0.8e-6)
    dt = W.cfl_dt(d, 0.9)
    rng = np.random.default_rng(3)
    shp = (n[2], n[1], n[0])
    eps = rng.uniform(1, 5, size=shp)
    mu = rng.uniform(1, 3, size=shp)
    s = oracle.Sim(n, d, dt, bc)
    s.set_materials(eps_r=eps, mu_r=mu)
    for fid in range(6):
        s.set_field(fid, rng.normal(size=s.field_size(fid)) * (1e3 if fid < 3 else 3.0))
    s.step(1)   # walls zeroed by the first update

    def unique(fid):
        # on a periodic axis node index n repeats node index 0: count it once
        ext = W.field_extent(fid, n)
        m = np.ones(ext[::-1], dtype=bool)
        for a in range(3):
            if bc[a] == W.PERIODIC and ext[a] == n[a] + 1:
                idx = [slice(None)] * 3
                idx[2 - a] = n[a]
                m[tuple(idx)] = False
        return m.ravel()

    def energy():
        E = [s.get_field(c) for c in range(3)]
        H = [s.get_field(3 + c) for c in range(3)]
        cu = _curl_e_faces(E, n, d)
        w = 0.0
        for c in range(3):
            u = unique(c)
            w += 0.5 * np.sum((EPS0 * s.get_material(c) * E[c] ** 2)[u])
            mu_f = MU0 * s.get_material(6 + c)
            u = unique(3 + c)
            w += 0.5 * np.sum((mu_f * (H[c] ** 2 - (dt / (2 * mu_f) * cu[c]) ** 2))[u])
        return w

    w0 = energy()
    s.step(400)
    assert abs(energy() / w0 - 1) < 1e-12


# ----------------------------------------------------------------- P4: |M| = Ms

def test_p4_magnetisation_norm_equals_ms():
    w = W.yig_slab_32(steps=10)
    s = oracle.from_workload(w)
    s.step(10)
    for fam in range(3):
        Ms = s.get_material(9 + fam)
        M = np.stack([s.get_field(6 + 3 * fam + c) for c in range(3)])
        nrm = np.linalg.norm(M, axis=0)
        mag = Ms > 0
        assert mag.any()
        np.testing.assert_allclose(nrm[mag], Ms[mag], rtol=1e-14)
        assert np.all(nrm[~mag] == 0)


# ------------------------------------------- P5/P6: uniform coupled precession

def _rotate(v, axis, ang):
    a = axis / np.linalg.norm(axis)
    return (v * math.cos(ang) + np.cross(a, v) * math.sin(ang)
            + a * np.dot(a, v) * (1 - math.cos(ang)))


def _uniform_box(m0, h_init, h0, alpha, dt, tol=1e-14, dx=1e-4):
    n = (3, 4, 5)
    shp = (n[2], n[1], n[0])
    s = oracle.Sim(n, (dx, dx * 1.1, dx * 0.9), dt, (W.PERIODIC,) * 3, tol=tol)
    s.set_materials(Ms=np.full(shp, 1.4e5), alpha=np.full(shp, alpha), gamma=np.full(shp, 1.76e11))
    s.set_bias(*h0)
    s.set_M_cells(*[np.full(shp, m0[c]) for c in range(3)])
    for c in range(3):
        s.set_field(3 + c, np.full(s.field_size(3 + c), h_init[c]))
    return s


@pytest.mark.parametrize("case", ["larmor_about_H0", "about_H0_plus_M"])
def test_p5_uniform_precession_is_exact_cayley_rotation(case):
    """Periodic box, uniform M, E = 0, alpha = 0: curl E = 0 so H + M_perp is
    constant per face and the converged trapezoidal step (Eqs. llg_tra1-4) is
    an exact rotation about W = H0 + H^0 + M^0 by 2 atan(kappa |W|) per half
    step, kappa = mu0 |gamma| dt/4.  With H^0 = -M^0 this is Larmor
    precession about H0 at ~gamma mu0 H0.  Pins the sign of b, a, the
    closed-form solve, the factor 4 in kappa and the H/M coupling."""
    m0 = 1.4e5 * np.array([0.6, 0.0, 0.8])
    h0 = np.array([0.0, 2e4, 1e5])
    h_init = -m0 if case == "larmor_about_H0" else np.zeros(3)
    dt = 2e-13
    s = _uniform_box(m0, h_init, h0, 0.0, dt)
    N = 300
    s.step(N)
    Wv = h0 + h_init + m0
    kappa = MU0 * 1.76e11 * dt / 4
    ang = N * 4 * math.atan(kappa * np.linalg.norm(Wv))
    m_want = _rotate(m0, Wv, ang)
    if case == "larmor_about_H0":
        om = 4 * math.atan(kappa * np.linalg.norm(h0)) / dt
        assert abs(om / (1.76e11 * MU0 * np.linalg.norm(h0)) - 1) < 1e-6
    for fam in range(3):
        for c in range(3):
            got = s.get_field(6 + 3 * fam + c)
            np.testing.assert_allclose(got, m_want[c], rtol=0, atol=1e-9 * 1.4e5)
        got_h = s.get_field(3 + fam)
        np.testing.assert_allclose(got_h, h_init[fam] + m0[fam] - m_want[fam], rtol=0, atol=1e-9 * 1.4e5)
    np.testing.assert_array_equal(s.get_field(0), 0.0)


def _gilbert_closed_form(m0, Wv, alpha, t):
    """Constant-field Gilbert precession: tan(theta/2) decays as
    exp(-alpha w t/(1+alpha^2)), azimuth advances w t/(1+alpha^2), w = gamma mu0 |W|."""
    w = 1.76e11 * MU0 * np.linalg.norm(Wv)
    e3 = Wv / np.linalg.norm(Wv)
    Ms = np.linalg.norm(m0)
    u = m0 / Ms
    th0 = math.acos(np.clip(np.dot(u, e3), -1, 1))
    e1 = u - np.dot(u, e3) * e3
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(e3, e1)
    th = 2 * math.atan(math.tan(th0 / 2) * math.exp(-alpha * w * t / (1 + alpha ** 2)))
    ph = w * t / (1 + alpha ** 2)
    return Ms * (math.sin(th) * (math.cos(ph) * e1 + math.sin(ph) * e2) + math.cos(th) * e3)


def test_p6_damped_precession_second_order():
    """Gilbert damping (alpha/Ms M x dM/dt) of Eq. LLG: with a fixed field the
    trapezoidal scheme converges to the closed form at second order in dt
    (error ratio ~4 per halving)."""
    m0 = 1.4e5 * np.array([0.8, 0.0, 0.6])
    h0 = np.array([0.0, 0.0, 2e5])
    h_init = -m0            # W = H0
    alpha = 0.1
    T = 300 * 4e-13
    errs = []
    for dt in (4e-13, 2e-13, 1e-13):
        N = int(round(T / dt))
        s = _uniform_box(m0, h_init, h0, alpha, dt)
        s.step(N)
        want = _gilbert_closed_form(m0, h0, alpha, N * dt)
        got = np.array([s.get_field(6 + c)[0] for c in range(3)])
        errs.append(np.linalg.norm(got - want) / 1.4e5)
    r1, r2 = math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])
    assert 1.9 < r1 < 2.1 and 1.9 < r2 < 2.1, (errs, r1, r2)
    assert errs[0] < 1e-3


# ------------------------------------------------------------ P7: thin film FMR

def test_p7_thin_film_fmr_kittel():
    """A film normal to z in a quasi-static PEC-walled column, periodic in x/y,
    biased in-plane along x: the coupled Maxwell-LLG scheme must produce the
    demagnetising fields itself (B_z = 0 -> h_z = -m_z; conserved flux ->
    h_y = -f m_y), giving f = gamma mu0/(2 pi) sqrt((H0 + f Ms)(H0 + Ms)),
    which reduces to Eq. kittel as the fill fraction f -> 0 (Sec. 5.2.2).
    The film is 32 of 64 cells thick so that its two edge faces (Ms/2 from
    the two-cell average, hence a smaller local demag field without exchange
    coupling) shift the mode by well under the 1% tolerance."""
    nz, z0, z1 = 64, 16, 48
    n = (1, 1, nz)
    dz, dxy = 5e-6, 1e-3
    dt = W.cfl_dt((dxy, dxy, dz), 0.9)
    shp = (nz, 1, 1)
    film = np.zeros(shp, dtype=bool)
    film[z0:z1] = True
    Ms0 = 1.4e5
    s = oracle.Sim(n, (dxy, dxy, dz), dt, (W.PERIODIC, W.PERIODIC, W.PEC), tol=1e-12)
    s.set_materials(eps_r=np.ones(shp), Ms=np.where(film, Ms0, 0.0),
                    gamma=np.where(film, 1.76e11, 0.0))
    H0 = 1e5
    s.set_bias(H0, 0.0, 0.0)
    s.set_M_cells(np.where(film, 1.0, 0.0), np.where(film, 0.01, 0.0), np.zeros(shp))
    f_want = _kittel_f(H0, Ms0, frac=(z1 - z0) / nz)
    period_steps = 1.0 / (f_want * dt)
    chunk = max(1, int(period_steps / 50))
    nchunks = int(5 * period_steps / chunk)
    ts, my = [], []
    for q in range(nchunks):
        s.step(chunk)
        ts.append((q + 1) * chunk * dt)
        # mean M_y over the film's y-faces
        my.append(s.get_field(6 + 3 * 1 + 1).reshape(nz, 2, 1)[z0:z1, 0, 0].mean())
    ts, my = np.array(ts), np.array(my)
    y = my - my.mean()
    idx = np.where((y[:-1] < 0) & (y[1:] >= 0))[0]     # rising zero crossings
    tz = ts[idx] - y[idx] * (ts[idx + 1] - ts[idx]) / (y[idx + 1] - y[idx])
    f_meas = (len(tz) - 1) / (tz[-1] - tz[0])
    assert len(tz) >= 4
    assert abs(f_meas / f_want - 1) < 0.01, (f_meas, f_want)
    # and far from the uncoupled Larmor line gamma mu0 H0 / 2 pi
    assert abs(f_meas / (1.76e11 * MU0 * H0 / (2 * math.pi)) - 1) > 0.3


# ---------------------------------------------------- P8: 2nd-order convergence

def _restrict(fid, fine, n_c):
    """Paper Sec. 5.1: faces take the mean of the 4 overlying fine faces,
    edges the mean of the 2 overlying fine edges (nodal axes subsample)."""
    nf = tuple(2 * v for v in n_c)
    ef = W.field_extent(fid, nf)
    a = fine.reshape(ef[2], ef[1], ef[0])
    if fid < 3:
        cell_axes = [fid]
    else:
        fam = fid - 3 if fid < 6 else (fid - 6) // 3
        cell_axes = [x for x in range(3) if x != fam]
    for xyz in range(3):
        p = 2 - xyz
        if xyz in cell_axes:
            a = np.moveaxis(a, p, -1)
            a = 0.5 * (a[..., 0::2] + a[..., 1::2])
            a = np.moveaxis(a, -1, p)
        else:
            a = np.take(a, range(0, a.shape[p], 2), axis=p)
    return a.ravel()


def _table2():
    rows = {}
    with open(os.path.join(GOLDEN, "table2_convergence.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                name, a, b, r = line.split()
                rows[name] = (float(a), float(b), float(r))
    return rows


@pytest.mark.slow
def test_p8_second_order_convergence():
    """Sec. 5.1 / Table 2: the coupled periodic problem (Gaussian bumps in
    sigma, eps, Ms, alpha, gamma; M = Ms xhat; cosine E/H) on 32^3, 64^3,
    128^3 at CFL 0.9 converges at second order in every E, H and M component
    (the paper prints rates 1.99-2.00).  The paper runs 5/10/20 steps; this
    test runs 2/4/8 steps (same physical time at every level, 2.5x cheaper)
    at the paper's iteration tolerance 1e-6.  The printed absolute L1
    differences depend on evaluation details the paper leaves open and are
    not compared here."""
    sols = {}
    fids = (0, 1, 2, 3, 4, 5, 6, 10, 14)
    for nn, steps in ((32, 2), (64, 4), (128, 8)):
        w = W.convergence(nn, tol=1e-6)
        s = oracle.from_workload(w)
        s.step(steps)
        sols[nn] = {fid: s.get_field(fid) for fid in fids}
        s.close()
    tab = _table2()
    names = {0: "Ex", 1: "Ey", 2: "Ez", 3: "Hx", 4: "Hy", 5: "Hz", 6: "Mx", 10: "My", 14: "Mz"}
    for fid, name in names.items():
        e1 = np.mean(np.abs(_restrict(fid, sols[64][fid], (32,) * 3) - sols[32][fid]))
        e2 = np.mean(np.abs(_restrict(fid, sols[128][fid], (64,) * 3) - sols[64][fid]))
        rate = math.log2(e1 / e2)
        assert abs(rate - tab[name][2]) < 0.1, (name, e1, e2, rate)


# --------------------------------------------- P10: PEC mirror, PML reflection

def _mirror_fields(fid, arr, n, axis):
    """Odd mirror image of a Yee field across the plane x_axis = 0, placed in
    a doubled periodic domain: tangential E and normal H are odd, the rest even."""
    ext = W.field_extent(fid, n)
    a = arr.reshape(ext[2], ext[1], ext[0])
    p = 2 - axis
    if fid < 3:
        odd = nodal = fid != axis
    else:
        odd = nodal = (fid - 3) == axis
    sgn = -1.0 if odd else 1.0
    if nodal:   # node i -> 2n - i; node 2n repeats node 0
        inner = np.take(a, range(1, n[axis]), axis=p)
        full = np.concatenate([np.take(a, range(0, n[axis] + 1), axis=p),
                               sgn * np.flip(inner, axis=p), np.take(a, [0], axis=p)], axis=p)
    else:       # cell i -> 2n - 1 - i
        full = np.concatenate([a, sgn * np.flip(a, axis=p)], axis=p)
    return full.ravel()


def _zero_walls(fid, arr, n, axis):
    """Tangential E and normal H are zero on the two walls normal to axis."""
    ext = W.field_extent(fid, n)
    a = arr.reshape(ext[2], ext[1], ext[0]).copy()
    p = 2 - axis
    if (fid < 3 and fid != axis) or (fid >= 3 and fid - 3 == axis):
        idx = [slice(None)] * 3
        for node in (0, n[axis]):
            idx[p] = node
            a[tuple(idx)] = 0.0
    return a.ravel()


def _sub_domain(fid, arr2, n, n2, axis):
    ext2 = W.field_extent(fid, n2)
    a = arr2.reshape(ext2[2], ext2[1], ext2[0])
    return np.take(a, range(0, W.field_extent(fid, n)[axis]), axis=2 - axis).ravel()


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_p10_pec_wall_is_odd_mirror(axis):
    """PEC (Sec. 3.2.3, reflection coefficient -1): a PEC-bounded run equals
    the periodic run of its odd mirror image on the doubled domain, with
    inhomogeneous eps, sigma, mu and a soft source present."""
    n = [4, 5, 6]
    d = (1.0e-6, 1.2e-6, 0.9e-6)
    dt = W.cfl_dt(d, 0.9)
    rng = np.random.default_rng(11 + axis)
    shp = (n[2], n[1], n[0])
    p = 2 - axis
    mats = [rng.uniform(1, 4, size=shp), rng.uniform(0, 30, size=shp), rng.uniform(1, 2, size=shp)]
    bc = [W.PERIODIC] * 3
    bc[axis] = W.PEC
    s = oracle.Sim(n, d, dt, bc)
    s.set_materials(*mats)
    n2 = list(n)
    n2[axis] *= 2
    s2 = oracle.Sim(n2, d, dt, (W.PERIODIC,) * 3)
    s2.set_materials(*[np.concatenate([m, np.flip(m, axis=p)], axis=p) for m in mats])
    for fid in range(6):
        v = _zero_walls(fid, rng.normal(size=s.field_size(fid)) * (1e3 if fid < 3 else 2.0), n, axis)
        s.set_field(fid, v)
        s2.set_field(fid, _mirror_fields(fid, v, n, axis))
    comp = (axis + 1) % 3        # source tangential to the wall: odd image
    ix = [1, 2, 3]
    ixm = list(ix)
    ixm[axis] = 2 * n[axis] - ix[axis]
    kw = dict(f0=1e13, tp=5 * dt, t0=8 * dt)
    s.add_source(W.SRC_POINT_J, comp, *ix, amp=1e9, **kw)
    s2.add_source(W.SRC_POINT_J, comp, *ix, amp=1e9, **kw)
    s2.add_source(W.SRC_POINT_J, comp, *ixm, amp=-1e9, **kw)
    s.step(40)
    s2.step(40)
    for fid in range(6):
        want = _sub_domain(fid, s2.get_field(fid), n, n2, axis)
        err = rel_l2(s.get_field(fid), want)
        assert err < 1e-13, (axis, fid, err)
    assert np.abs(s.get_field(comp)).max() > 0


def _pml_column(nz, npml, steps, probe_k, src_k):
    n = (1, 1, nz)
    dz = 1e-6
    dt = W.cfl_dt((dz, dz, dz), 0.9)
    bc = (W.PERIODIC, W.PERIODIC, W.PML if npml else W.PEC)
    s = oracle.Sim(n, (dz, dz, dz), dt, bc, pml_cells=npml)
    s.set_materials()
    f0 = 1.0 / (40 * dt)          # ~40 steps per period: well resolved
    tp = 1.0 / f0
    s.add_source(W.SRC_PLANE_J_TE10, 0, 0, 0, src_k, amp=1e9, f0=f0, tp=tp, t0=3 * tp)
    trace = []
    for _ in range(steps):
        s.step(1)
        trace.append(s.get_field(0).reshape(nz + 1, 2, 1)[probe_k, 0, 0])
    return np.array(trace)


def test_p10_pml_reflection_below_0p1_percent():
    """Sec. 3.2.3: the macroscopic PML-2SC absorbs with < 0.1% reflection in
    a non-magnetic medium.  Reflection = the difference between a short
    PML-terminated column and a long one (before the long one's far walls
    are seen), relative to the incident peak."""
    steps = 900
    short = _pml_column(160, 10, steps, probe_k=60, src_k=80)
    long_ = _pml_column(2160, 0, steps, probe_k=1060, src_k=1080)
    inc = np.abs(long_).max()
    refl = np.abs(short - long_).max() / inc
    assert inc > 0
    assert refl < 1e-3, refl


# ------------------------------------------------ P11: plain Yee reduction

def _edge_mean_np(cell, c, n):
    """PEC-box edge average by zero-padding with counts (numpy)."""
    pad = np.pad(cell, 1)
    one = np.pad(np.ones_like(cell), 1)
    ax = [2, 1, 0]   # numpy axis of x, y, z
    others = [a for a in range(3) if a != c]
    tot = 0
    cnt = 0
    for o1 in (0, 1):
        for o2 in (0, 1):
            sl = [None, None, None]
            for a in range(3):
                if a == c:
                    sl[ax[a]] = slice(1, n[a] + 1)
                else:
                    o = o1 if a == others[0] else o2
                    sl[ax[a]] = slice(o, o + n[a] + 1)
            tot = tot + pad[tuple(sl)]
            cnt = cnt + one[tuple(sl)]
    return tot / cnt


def test_p11_reduces_to_textbook_yee():
    """Ms = 0, mu_r = 1: the scheme is textbook lossy Yee FDTD:
    H^(n+1/2) = H^(n-1/2) - dt/mu0 curl E^n, E^(n+1) = ((eps/dt - sigma/2) E^n
    + curl H^(n+1/2))/(eps/dt + sigma/2), written here with a full-step H
    leapfrog and numpy slicing, independently of the oracle."""
    n = (5, 4, 6)
    nx, ny, nz = n
    d = (1.0e-6, 0.8e-6, 1.1e-6)
    dt = W.cfl_dt(d, 0.9)
    rng = np.random.default_rng(21)
    shp = (nz, ny, nx)
    eps_c = rng.uniform(1, 6, size=shp)
    sig_c = rng.uniform(0, 80, size=shp)
    s = oracle.Sim(n, d, dt, (W.PEC,) * 3)
    s.set_materials(eps_r=eps_c, sigma=sig_c)
    Ex = rng.normal(size=(nz + 1, ny + 1, nx)) * 1e3
    Ex[:, [0, -1], :] = 0
    Ex[[0, -1], :, :] = 0
    Ey = rng.normal(size=(nz + 1, ny, nx + 1)) * 1e3
    Ey[:, :, [0, -1]] = 0
    Ey[[0, -1], :, :] = 0
    Ez = rng.normal(size=(nz, ny + 1, nx + 1)) * 1e3
    Ez[:, :, [0, -1]] = 0
    Ez[:, [0, -1], :] = 0
    Hx = rng.normal(size=(nz, ny, nx + 1))
    Hx[:, :, [0, -1]] = 0
    Hy = rng.normal(size=(nz, ny + 1, nx))
    Hy[:, [0, -1], :] = 0
    Hz = rng.normal(size=(nz + 1, ny, nx))
    Hz[[0, -1], :, :] = 0
    for fid, a in enumerate((Ex, Ey, Ez, Hx, Hy, Hz)):
        s.set_field(fid, a.ravel())
    eps = [EPS0 * _edge_mean_np(eps_c, c, n) for c in range(3)]
    sig = [_edge_mean_np(sig_c, c, n) for c in range(3)]
    dx, dy, dz = d

    def curl_e():
        cx = (Ez[:, 1:, :] - Ez[:, :-1, :]) / dy - (Ey[1:] - Ey[:-1]) / dz
        cy = (Ex[1:] - Ex[:-1]) / dz - (Ez[:, :, 1:] - Ez[:, :, :-1]) / dx
        cz = (Ey[:, :, 1:] - Ey[:, :, :-1]) / dx - (Ex[:, 1:, :] - Ex[:, :-1, :]) / dy
        cx[:, :, [0, -1]] = 0
        cy[:, [0, -1], :] = 0
        cz[[0, -1]] = 0
        return cx, cy, cz

    def e_step():
        nonlocal Ex, Ey, Ez
        cx = np.zeros_like(Ex)
        cy = np.zeros_like(Ey)
        cz = np.zeros_like(Ez)
        cx[1:-1, 1:-1, :] = ((Hz[1:-1, 1:, :] - Hz[1:-1, :-1, :]) / dy
                             - (Hy[1:, 1:-1, :] - Hy[:-1, 1:-1, :]) / dz)
        cy[1:-1, :, 1:-1] = ((Hx[1:, :, 1:-1] - Hx[:-1, :, 1:-1]) / dz
                             - (Hz[1:-1, :, 1:] - Hz[1:-1, :, :-1]) / dx)
        cz[:, 1:-1, 1:-1] = ((Hy[:, 1:-1, 1:] - Hy[:, 1:-1, :-1]) / dx
                             - (Hx[:, 1:, 1:-1] - Hx[:, :-1, 1:-1]) / dy)
        out = []
        for E, cu, e, sg in ((Ex, cx, eps[0], sig[0]), (Ey, cy, eps[1], sig[1]), (Ez, cz, eps[2], sig[2])):
            out.append(((e / dt - sg / 2) * E + cu) / (e / dt + sg / 2))
        Ex, Ey, Ez = out
        Ex[:, [0, -1], :] = 0
        Ex[[0, -1]] = 0
        Ey[:, :, [0, -1]] = 0
        Ey[[0, -1]] = 0
        Ez[:, :, [0, -1]] = 0
        Ez[:, [0, -1], :] = 0

    N = 50
    cx, cy, cz = curl_e()
    Hx = Hx - dt / (2 * MU0) * cx
    Hy = Hy - dt / (2 * MU0) * cy
    Hz = Hz - dt / (2 * MU0) * cz
    for step in range(N):
        e_step()
        cx, cy, cz = curl_e()
        f = dt / (2 * MU0) if step == N - 1 else dt / MU0
        Hx = Hx - f * cx
        Hy = Hy - f * cy
        Hz = Hz - f * cz
    s.step(N)
    for fid, a in enumerate((Ex, Ey, Ez, Hx, Hy, Hz)):
        assert rel_l2(s.get_field(fid), a.ravel()) < 1e-12, fid


# ------------------------------------------------ P12: divergence invariants

def _div(fields3, n, d, face):
    nx, ny, nz = n
    if face:
        a = fields3[0].reshape(nz, ny, nx + 1)
        b = fields3[1].reshape(nz, ny + 1, nx)
        c = fields3[2].reshape(nz + 1, ny, nx)
        return ((a[:, :, 1:] - a[:, :, :-1]) / d[0] + (b[:, 1:, :] - b[:, :-1, :]) / d[1]
                + (c[1:] - c[:-1]) / d[2])
    # edges -> nodes (periodic: index n == index 0)
    a = fields3[0].reshape(nz + 1, ny + 1, nx)[:-1, :-1, :]
    b = fields3[1].reshape(nz + 1, ny, nx + 1)[:-1, :, :-1]
    c = fields3[2].reshape(nz, ny + 1, nx + 1)[:, :-1, :-1]
    return ((a - np.roll(a, 1, axis=2)) / d[0] + (b - np.roll(b, 1, axis=1)) / d[1]
            + (c - np.roll(c, 1, axis=0)) / d[2])


def test_p12_divergence_invariants_coupled_periodic():
    """Faraday with B = mu0 (H + M) on magnetic faces and mu H elsewhere
    (Eqs. Faraday2/Faraday3, iterate_H): div B is constant per cell to
    roundoff, through every H/M iteration.  With sigma = 0 and no source,
    div(eps E) is constant per node.  Pins the pairing of each face family
    with its own normal M component and the mu/mu0 switch."""
    n = (5, 4, 6)
    d = (1.0e-6, 1.2e-6, 0.9e-6)
    w = W.random_small(31, n=n, bc=(W.PERIODIC,) * 3, sources=False, dx=d)
    w.sigma = np.zeros_like(w.sigma)
    s = oracle.from_workload(w)

    def divs():
        B = []
        for fam in range(3):
            H = s.get_field(3 + fam)
            M = s.get_field(6 + 3 * fam + fam)
            Ms = s.get_material(9 + fam)
            mur = s.get_material(6 + fam)
            B.append(np.where(Ms > 0, MU0 * (H + M), MU0 * mur * H))
        D = [EPS0 * s.get_material(c) * s.get_field(c) for c in range(3)]
        return _div(B, n, d, True), _div(D, n, d, False)

    b0, e0 = divs()
    s.step(25)
    b1, e1 = divs()
    assert np.abs(b1 - b0).max() < 1e-11 * max(np.abs(b0).max(), 1e-30)
    assert np.abs(e1 - e0).max() < 1e-11 * max(np.abs(e0).max(), 1e-30)
    assert s.iter_log().max() >= 2     # the magnetisation really iterated


def test_p13_iteration_count_follows_contraction():
    """The Jacobi iteration contracts by ~kappa Ms per sweep: at the 32^3
    slab time step (kappa Ms ~ 1e-5) tol = 1e-10 needs 2-3 sweeps; with
    100x larger cells and time step it needs more."""
    w = W.yig_slab_32(steps=4)
    s = oracle.from_workload(w)
    s.step(4)
    base = s.iter_log()
    assert set(base.tolist()) <= {2, 3}
    w2 = W.yig_slab_32(steps=4)
    w2.d = (w2.d[0] * 100, w2.d[1] * 100, w2.d[2] * 100)
    w2.dt = W.cfl_dt(w2.d, 0.9)
    s2 = oracle.from_workload(w2)
    s2.step(4)
    assert s2.iter_log().min() > base.max()


def test_not_converged_is_reported():
    w = W.yig_slab_32(steps=2)
    w.max_iter = 1
    s = oracle.from_workload(w)
    assert s.step(1, check=False) == -4


# ------------------------------------------- P9: the first-order scheme (f4)

def test_p9_first_order_uniform_precession_converges_at_first_order():
    """Sec. 3.2.1 (Steps 1/3 with Eq. LLG_scalar): forward Euler of the
    Landau-Lifshitz form over each half step, then N().  In the uniform
    periodic box curl E = 0, so H + M is constant per face and the exact
    solution is the constant-field Gilbert precession about W = H0 + H^0 + M^0
    (the closed form of P6).  The first-order scheme must converge to it with
    error ratio ~2 per halving of dt.  A wrong gamma_L = |gamma|/(1 + alpha^2),
    a wrong sign of the M x (M x H) damping term, or a full dt instead of
    dt/2 per half step (reading R10) converges to a different motion, and the
    error then stops falling."""
    m0 = 1.4e5 * np.array([0.8, 0.0, 0.6])
    h0 = np.array([0.0, 0.0, 2e5])
    h_init = -m0            # W = H0
    alpha = 0.3
    T = 400 * 2e-13
    errs = []
    for dt in (2e-13, 1e-13, 5e-14):
        N = int(round(T / dt))
        n = (3, 4, 5)
        shp = (n[2], n[1], n[0])
        s = oracle.Sim(n, (1e-4, 1.1e-4, 0.9e-4), dt, (W.PERIODIC,) * 3, order=1)
        s.set_materials(Ms=np.full(shp, 1.4e5), alpha=np.full(shp, alpha), gamma=np.full(shp, 1.76e11))
        s.set_bias(*h0)
        s.set_M_cells(*[np.full(shp, m0[c]) for c in range(3)])
        for c in range(3):
            s.set_field(3 + c, np.full(s.field_size(3 + c), h_init[c]))
        s.step(N)
        assert set(s.iter_log().tolist()) == {1}
        want = _gilbert_closed_form(m0, h0, alpha, N * dt)
        got = np.array([s.get_field(6 + c)[0] for c in range(3)])
        errs.append(np.linalg.norm(got - want) / 1.4e5)
    r1, r2 = math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])
    assert 0.85 < r1 < 1.15 and 0.85 < r2 < 1.15, (errs, r1, r2)
    assert errs[2] < 0.05


@pytest.mark.slow
def test_p9_first_order_scheme_rates_sec_5_1():
    """Sec. 5.1, the text after Table 2: with the first-order magnetisation
    coupling the M components fall to first order and the E and H rates drop
    to as low as 1.74 (the draft gives a range 1.74-2.35).  Same problem and
    restriction as P8.  The dynamic components M_y, M_z must converge at rate
    1 +- 0.15; M_x ~ Ms carries the first-order error only through the small
    tilt, so its rate is reported, not bounded.  Every E/H rate lies in
    1.6-2.4 and at least one falls clearly below 2."""
    sols = {}
    fids = (0, 1, 2, 3, 4, 5, 6, 10, 14)
    for nn, steps in ((32, 2), (64, 4), (128, 8)):
        w = W.convergence(nn, order=1, tol=1e-6)
        s = oracle.from_workload(w)
        s.step(steps)
        sols[nn] = {fid: s.get_field(fid) for fid in fids}
        s.close()
    names = {0: "Ex", 1: "Ey", 2: "Ez", 3: "Hx", 4: "Hy", 5: "Hz", 6: "Mx", 10: "My", 14: "Mz"}
    rates = {}
    for fid, name in names.items():
        e1 = np.mean(np.abs(_restrict(fid, sols[64][fid], (32,) * 3) - sols[32][fid]))
        e2 = np.mean(np.abs(_restrict(fid, sols[128][fid], (64,) * 3) - sols[64][fid]))
        rates[name] = math.log2(e1 / e2)
    print("first-order scheme rates:", {k: round(v, 3) for k, v in rates.items()})
    for name in ("My", "Mz"):
        assert abs(rates[name] - 1.0) < 0.15, (name, rates)
    eh = [rates[k] for k in ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")]
    assert all(1.6 < r < 2.4 for r in eh), rates
    assert min(eh) < 1.9, rates


# ---------------------------------------------------- hard sources (Sec. 3.2)

def _waveform(q, t):
    """The modulated Gaussian drive of Sec. 5.2.1 (Eq. gaulssian, free t0)."""
    return q["amp"] * math.exp(-(t - q["t0"]) ** 2 / (2 * q["tp"] ** 2)) * math.cos(2 * math.pi * q["f0"] * t)


def test_hard_sources_overwrite_after_their_update():
    """Sec. 3.2: a hard source overwrites the field after its update (reading
    R9: hard E after the E update, at t^(n+1); hard H after each H half step,
    at that half step's end time).  A textbook numpy Yee leapfrog in a PEC
    vacuum box that writes the same values at the same points of the step
    must give the oracle's fields to rounding, and after every step the driven
    edge and face hold g(t^(n+1)) exactly.  Writing at t^n instead of t^(n+1),
    or before the update instead of after it, breaks the comparison."""
    n = (6, 5, 7)
    d = (1.0e-6, 1.3e-6, 0.8e-6)
    dt = W.cfl_dt(d, 0.9)
    nx, ny, nz = n
    qe = dict(i=2, j=3, k=4, amp=3e4, f0=4e13, tp=12 * dt, t0=20 * dt)   # hard Ex at (2.5, 3, 4)
    qh = dict(i=3, j=2, k=3, amp=70.0, f0=3e13, tp=9 * dt, t0=15 * dt)   # hard Hz at (3.5, 2.5, 3)
    s = _vacuum_sim(n, d, dt, (W.PEC,) * 3)
    s.add_source(W.SRC_HARD_E, 0, qe["i"], qe["j"], qe["k"], qe["amp"], qe["f0"], qe["tp"], qe["t0"])
    s.add_source(W.SRC_HARD_H, 2, qh["i"], qh["j"], qh["k"], qh["amp"], qh["f0"], qh["tp"], qh["t0"])
    Ex = np.zeros((nz + 1, ny + 1, nx))
    Ey = np.zeros((nz + 1, ny, nx + 1))
    Ez = np.zeros((nz, ny + 1, nx + 1))
    Hx = np.zeros((nz, ny, nx + 1))
    Hy = np.zeros((nz, ny + 1, nx))
    Hz = np.zeros((nz + 1, ny, nx))
    dx, dy, dz = d
    fh = dt / (2 * MU0)
    fe = dt / EPS0

    def h_half(t_end):
        nonlocal Hx, Hy, Hz
        cx = (Ez[:, 1:, :] - Ez[:, :-1, :]) / dy - (Ey[1:] - Ey[:-1]) / dz
        cy = (Ex[1:] - Ex[:-1]) / dz - (Ez[:, :, 1:] - Ez[:, :, :-1]) / dx
        cz = (Ey[:, :, 1:] - Ey[:, :, :-1]) / dx - (Ex[:, 1:, :] - Ex[:, :-1, :]) / dy
        Hx = Hx - fh * cx
        Hy = Hy - fh * cy
        Hz = Hz - fh * cz
        Hx[:, :, [0, -1]] = 0
        Hy[:, [0, -1], :] = 0
        Hz[[0, -1]] = 0
        Hz[qh["k"], qh["j"], qh["i"]] = _waveform(qh, t_end)

    def e_full(t_end):
        nonlocal Ex, Ey, Ez
        Ex[1:-1, 1:-1, :] += fe * ((Hz[1:-1, 1:, :] - Hz[1:-1, :-1, :]) / dy
                                   - (Hy[1:, 1:-1, :] - Hy[:-1, 1:-1, :]) / dz)
        Ey[1:-1, :, 1:-1] += fe * ((Hx[1:, :, 1:-1] - Hx[:-1, :, 1:-1]) / dz
                                   - (Hz[1:-1, :, 1:] - Hz[1:-1, :, :-1]) / dx)
        Ez[:, 1:-1, 1:-1] += fe * ((Hy[:, 1:-1, 1:] - Hy[:, 1:-1, :-1]) / dx
                                   - (Hx[:, 1:, 1:-1] - Hx[:, :-1, 1:-1]) / dy)
        Ex[qe["k"], qe["j"], qe["i"]] = _waveform(qe, t_end)

    ex_idx = qe["i"] + nx * (qe["j"] + (ny + 1) * qe["k"])
    hz_idx = qh["i"] + nx * (qh["j"] + ny * qh["k"])
    for step in range(40):
        h_half((step + 0.5) * dt)
        e_full((step + 1.0) * dt)
        h_half((step + 1.0) * dt)
        s.step(1)
        assert s.get_field(0)[ex_idx] == _waveform(qe, (step + 1.0) * dt)
        assert s.get_field(5)[hz_idx] == _waveform(qh, (step + 1.0) * dt)
    for fid, a in enumerate((Ex, Ey, Ez, Hx, Hy, Hz)):
        assert rel_l2(s.get_field(fid), a.ravel()) < 1e-12, fid
        assert np.abs(a).max() > 0


@pytest.mark.parametrize("comp", [0, 1])
def test_te10_plane_source_profile_and_time_level(comp):
    """Soft J plane source (reading R9: the TE10
    profile sin(pi x/W), x measured from the lower x wall, W = nx dx; the
    paper's printed cos(2 pi x/(W/2)) is read as garbled).  From zero fields
    in vacuum one step gives E^1 = -dt J(t^(1/2))/eps0 on the plane's edges
    and zero elsewhere (Step 2 of Sec. 3.2.1 with H^(1/2) = 0).  The drive is
    chosen so that g(t^(1/2)) = amp exactly (t0 = dt/2, f0 = 0) while
    g(0) = amp exp(-1/8): evaluating J at t^n, shifting x by half a cell or
    using another width fails element by element."""
    n = (9, 4, 6)
    d = (1.1e-6, 1.0e-6, 0.9e-6)
    dt = W.cfl_dt(d, 0.9)
    nx, ny, nz = n
    ks, amp = 3, 2.5e9
    s = _vacuum_sim(n, d, dt, (W.PEC,) * 3)
    s.add_source(W.SRC_PLANE_J_TE10, comp, 0, 0, ks, amp, 0.0, dt, 0.5 * dt)
    s.step(1)
    E = s.get_field(comp)
    ext = W.field_extent(comp, n)
    E = E.reshape(ext[2], ext[1], ext[0])
    W_ = nx * d[0]
    x = (np.arange(ext[0]) + (0.5 if comp == 0 else 0.0)) * d[0]
    want_row = -dt * amp * np.sin(np.pi * x / W_) / EPS0
    plane = E[ks]
    # interior edges of the plane carry the profile; PEC wall edges are zero
    lo_t = 1
    hi_t = ext[1] - 1
    if comp == 0:
        inner = plane[lo_t:hi_t, :]
        np.testing.assert_allclose(inner, np.broadcast_to(want_row, inner.shape), rtol=1e-13, atol=0)
    else:
        inner = plane[:, 1:-1]
        np.testing.assert_allclose(inner, np.broadcast_to(want_row[1:-1], inner.shape), rtol=1e-13, atol=0)
    assert np.all(np.delete(E, ks, axis=0) == 0.0)
    assert np.all(s.get_field(1 - comp) == 0.0) and np.all(s.get_field(2) == 0.0)


# ---------------------------------------- R12: initial M where the mean cancels

@pytest.mark.parametrize("fam", [0, 1, 2])
def test_r12_initial_m_falls_back_to_lower_cell(fam):
    """Reading R12: a face whose averaged cell M falls below 1e-6 Ms (here two
    cells with opposite directions, and a pair that cancels to 1e-9) takes the
    direction of the lower-index cell, renormalised to Ms_face.  Every other
    face is the renormalised mean (Sec. 3.1).  Taking the upper cell's
    direction gives the opposite vector on the tested faces."""
    n = (4, 3, 5)
    shp = (n[2], n[1], n[0])
    s = oracle.Sim(n, (1e-6,) * 3, 1e-16, (W.PEC,) * 3)
    Ms = np.full(shp, 1.4e5)
    s.set_materials(Ms=Ms, alpha=np.full(shp, 0.01), gamma=np.full(shp, 1.76e11))
    rng = np.random.default_rng(5)
    m = rng.normal(size=(3,) + shp)
    lo = [1, 1, 2]
    hi = list(lo)
    hi[fam] += 1
    u = np.array([0.3, -0.5, 0.81])
    m[:, lo[2], lo[1], lo[0]] = u
    m[:, hi[2], hi[1], hi[0]] = -u
    lo2 = [2, 0, 1]
    hi2 = list(lo2)
    hi2[fam] += 1
    v = np.array([-0.6, 0.2, 0.4])
    m[:, lo2[2], lo2[1], lo2[0]] = v
    m[:, hi2[2], hi2[1], hi2[0]] = -v + 1e-9 * np.array([1.0, 0.0, 0.0])
    s.set_M_cells(*(m[c] * 1.4e5 for c in range(3)))
    ext = W.field_extent(6 + 3 * fam, n)
    M = np.stack([s.get_field(6 + 3 * fam + c).reshape(ext[::-1]) for c in range(3)])
    for pair_lo, dirv in ((lo, u), (lo2, v)):
        f = list(pair_lo)
        f[fam] += 1                       # the face between the pair
        got = M[:, f[2], f[1], f[0]]
        np.testing.assert_allclose(got, 1.4e5 * dirv / np.linalg.norm(dirv), rtol=1e-14)
    # an ordinary face: renormalised mean of its two cells
    f = [1, 2, 3]
    a = list(f)
    a[fam] -= 1
    mean = 0.5 * (m[:, a[2], a[1], a[0]] + m[:, f[2], f[1], f[0]])
    np.testing.assert_allclose(M[:, f[2], f[1], f[0]], 1.4e5 * mean / np.linalg.norm(mean), rtol=1e-14)


# ------------------------------------ R13/R14: effect bounded at rounding level

def test_r13_r14_readings_move_results_at_rounding_level_only():
    """Readings R13 (extended precision in the LLG algebra) and R14 (H takes
    the on-sphere increment) change how Eq. iterate_H is rounded, not what it
    computes.  An oracle build that evaluates Eq. iterate_H as printed,
    H^n + M^n - M^(n+1/2,r) - dt/(2 mu0) curl E in FP64 with the stored N(x),
    must agree with the oracle after the 200 steps of the 32^3 slab problem:
    H to 1e-10 relative (the rounding of M ~ Ms = 1.4e5 A/m entering H of
    order 10 A/m), E to 1e-10, M to 1e-14, identical iteration counts.  A
    wrong on-sphere increment (a dropped M^n, a wrong norm) moves H by orders
    of magnitude more."""
    w = W.yig_slab_32(steps=200)
    a = oracle.from_workload(w)
    b = oracle.from_workload(w, variant="literal")
    a.step(200)
    b.step(200)
    np.testing.assert_array_equal(a.iter_log(), b.iter_log())
    for fid in range(15):
        bar = 1e-10 if fid < 6 else 1e-14
        assert rel_l2(b.get_field(fid), a.get_field(fid)) < bar, fid
    # the two builds are different programs: H differs above the 1e-12 bar
    assert max(rel_l2(b.get_field(f), a.get_field(f)) for f in (3, 4, 5)) > 1e-12


def test_openmp_timing_build_is_bit_identical():
    """The OpenMP build of the oracle (used only to time it on all host
    cores) computes every element with the same operations and reduces the
    residual with a max: fields and iteration counts equal the serial
    build's bit for bit."""
    w = W.waveguide(n=(24, 16, 40), steps=12)
    a = oracle.from_workload(w)
    b = oracle.from_workload(w, variant="omp")
    a.step(12)
    b.step(12)
    for fid in range(19):
        np.testing.assert_array_equal(a.get_field(fid), b.get_field(fid))
    np.testing.assert_array_equal(a.iter_log(), b.iter_log())

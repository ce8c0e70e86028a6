"""Energy and Poynting-flux monitors (FP64 Neumaier-compensated sums on the
device): the energy monitor against the same sum written out in numpy, the
discrete energy conserved by the scheme (Sec. 3.2) in a lossless cavity on
both paths and in both precisions, and the flux of a guided pulse the same
through two planes of a lossless guide."""
import numpy as np
import pytest

import paper_2103_12819_b300 as mmx
import workloads as W
from conftest import EPS0, MU0
from test_oracle_pins import _curl_e_faces

pytestmark = pytest.mark.gpu


def _cavity(n, seed, prec, path):
    d = (1.0e-6, 1.2e-6, 0.8e-6)
    dt = W.cfl_dt(d, 0.9)
    rng = np.random.default_rng(seed)
    shp = (n[2], n[1], n[0])
    eps = rng.uniform(1, 5, size=shp)
    mu = rng.uniform(1, 3, size=shp)
    s = mmx.Solver(n, d, dt, (W.PEC,) * 3, 0, 2, 1e-10, 64, prec)
    s.set_path(path)
    s.set_materials(eps_r=eps, mu_r=mu)
    for fid in range(6):
        s.set_field(fid, rng.normal(size=s.field_size(fid)) * (1e3 if fid < 3 else 3.0))
    s.step(1)            # the first update zeroes the wall values
    return s, d, dt


def test_energy_monitor_equals_the_written_out_sum():
    n = (7, 6, 5)
    s, d, dt = _cavity(n, 4, mmx.FP64, mmx.PATH_FUSED)
    E = [s.get_field(c) for c in range(3)]
    H = [s.get_field(3 + c) for c in range(3)]
    cu = _curl_e_faces(E, n, d)
    w = 0.0
    for c in range(3):
        w += 0.5 * np.sum(EPS0 * s.get_material(c) * E[c] ** 2)
        mu_f = MU0 * s.get_material(6 + c)
        w += 0.5 * np.sum(mu_f * (H[c] ** 2 - (dt / (2 * mu_f) * cu[c]) ** 2))
    assert abs(s.energy() / w - 1) < 1e-13


@pytest.mark.parametrize("path", [mmx.PATH_PLAIN, mmx.PATH_FUSED], ids=["plain", "fused"])
@pytest.mark.parametrize("prec,tol", [(mmx.FP64, 1e-12), (mmx.FP32, 2e-5)], ids=["fp64", "fp32"])
def test_discrete_energy_is_conserved(prec, tol, path):
    """Lossless, source-free, non-magnetic PEC cavity with random eps, mu and
    fields, 300 steps in 3 calls: the monitor's W stays constant."""
    s, _, _ = _cavity((64, 48, 40), 5, prec, path)
    w0 = s.energy()
    for _ in range(3):
        s.step(100)
    assert s.sync(check=False) == 0
    w1 = s.energy()
    print("energy drift %s: %.3e" % ("fp64" if prec == mmx.FP64 else "fp32", w1 / w0 - 1))
    assert abs(w1 / w0 - 1) < tol


def test_guided_pulse_carries_the_same_energy_through_two_planes():
    """A 12 GHz TE10 pulse in the air-filled guide: the time-integrated
    Poynting flux through z = 150 and z = 350 agree to 0.5% once the pulse
    has passed both, and is positive (+z)."""
    tp = 0.8e-9
    w = W.air_guide(f0=12.0e9, tp=tp)
    steps = int(np.ceil(6.2e-9 / w.dt))
    s = mmx.from_workload(w, prec=mmx.FP32, path=mmx.PATH_FUSED)
    a = s.add_flux_plane(150)
    b = s.add_flux_plane(350)
    s.step(steps // 2)
    s.step(steps - steps // 2)
    assert s.sync(check=False) == 0
    fa, pa = s.get_flux(a)
    fb, pb = s.get_flux(b)
    print("flux through z=150: %.6e J, z=350: %.6e J, last power %.2e / %.2e W" % (fa, fb, pa, pb))
    assert fa > 0 and fb > 0
    assert abs(fb / fa - 1) < 5e-3
    assert abs(pb) < 1e-3 * abs(fb) / (tp)      # the pulse has gone by

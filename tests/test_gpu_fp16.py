"""FP16-storage variant (E and H stored as FP16 times a per-context scale,
FP32 arithmetic; M and the H/M iteration state FP32): error against the FP64
path stated per field, the configurations it refuses, and the scale API."""
import numpy as np
import pytest

import paper_2103_12819_b300 as mmx
import workloads as W
from conftest import rel_l2

pytestmark = pytest.mark.gpu


def _errors(w, steps, fids):
    """Per-component relative L2 errors, plus the E, H and M vector fields as
    a whole ('E', 'H', 'M': error norm over all components / norm of all
    components), which is what a component near zero (Ex, Ez of a TE10
    guide) should be measured against."""
    a = mmx.from_workload(w, prec=mmx.FP16, path=mmx.PATH_FUSED)
    b = mmx.from_workload(w, prec=mmx.FP64, path=mmx.PATH_FUSED)
    for s in (a, b):
        s.step(steps)
        assert s.sync(check=False) == 0, s.last_error()
    errs, sq = {}, {"E": [0.0, 0.0], "H": [0.0, 0.0], "M": [0.0, 0.0]}
    for fid in fids:
        x, y = a.get_field(fid), b.get_field(fid)
        errs[fid] = rel_l2(x, y)
        grp = "E" if fid < 3 else "H" if fid < 6 else "M"
        sq[grp][0] += float(np.sum((x - y) ** 2))
        sq[grp][1] += float(np.sum(y ** 2))
    for grp, (e2, n2) in sq.items():
        if n2 > 0:
            errs[grp] = (e2 / n2) ** 0.5
    return errs


def test_fp16_storage_error_yig_slab():
    """The 32^3 slab, 200 steps, iteration tolerance 1e-6."""
    w = W.yig_slab_32()
    w.tol = 1e-6
    errs = _errors(w, w.steps, range(15))
    print("FP16 storage vs FP64, yig_slab_32, 200 steps:", {k: "%.2e" % v for k, v in errs.items()})
    assert max(errs[f] for f in range(6)) < 5e-3          # E, H, every component
    assert errs["M"] < 5e-4                               # M (stored FP32)


def test_fp16_storage_error_waveguide():
    """A 32x24x96 waveguide (z-PML, YIG slab, TE10 drive), 300 steps."""
    w = W.waveguide(n=(32, 24, 96), steps=300)
    errs = _errors(w, w.steps, list(range(15)))
    print("FP16 storage vs FP64, waveguide 32x24x96, 300 steps:", {k: "%.2e" % v for k, v in errs.items()})
    assert errs["E"] < 2e-2 and errs["H"] < 5e-3 and errs["M"] < 2e-3


def test_fp16_energy_drift():
    """Lossless PEC cavity, random fields: the FP16-stored fields keep the
    discrete energy to FP16 rounding."""
    n = (48, 40, 32)
    d = (1.0e-6, 1.2e-6, 0.8e-6)
    rng = np.random.default_rng(6)
    shp = (n[2], n[1], n[0])
    s = mmx.Solver(n, d, W.cfl_dt(d, 0.9), (W.PEC,) * 3, 0, 2, 1e-6, 64, mmx.FP16)
    s.set_materials(eps_r=rng.uniform(1, 5, size=shp), mu_r=rng.uniform(1, 3, size=shp))
    for fid in range(6):
        s.set_field(fid, rng.normal(size=s.field_size(fid)) * (1e3 if fid < 3 else 3.0))
    s.step(1)
    w0 = s.energy()
    s.step(200)
    drift = s.energy() / w0 - 1
    print("FP16 energy drift over 200 steps: %.2e" % drift)
    assert abs(drift) < 2e-3


def test_fp16_refuses_what_it_does_not_cover():
    w = W.random_small(30, n=(6, 5, 7), bc=(W.PERIODIC, W.PEC, W.PEC), tol=1e-6)
    s = mmx.from_workload(w, prec=mmx.FP16)
    with pytest.raises(mmx.MMXError):
        s.step(1)                                   # periodic x
    w = W.yig_slab_32(steps=2, n=16)
    s = mmx.from_workload(w, prec=mmx.FP16, path=mmx.PATH_PLAIN)
    with pytest.raises(mmx.MMXError):
        s.step(1)                                   # plain path
    s = mmx.Solver(w.n, w.d, w.dt, w.bc, 0, 2, 1e-6, 64, mmx.FP16)
    s.set_storage_scale(1e3, 10.0)                  # allowed before any field
    s.set_field(0, np.zeros(s.field_size(0)))
    with pytest.raises(mmx.MMXError):
        s.set_storage_scale(1e3, 10.0)              # not after
    f32 = mmx.Solver(w.n, w.d, w.dt, w.bc, 0, 2, 1e-6, 64, mmx.FP32)
    with pytest.raises(mmx.MMXError):
        f32.set_storage_scale(1.0, 1.0)             # FP16 contexts only


def test_fp16_readback_applies_the_scale():
    """set_field / get_field round-trip through the scaled FP16 store."""
    w = W.yig_slab_32(steps=2, n=16)
    s = mmx.Solver(w.n, w.d, w.dt, w.bc, 0, 2, 1e-6, 64, mmx.FP16)
    s.set_storage_scale(500.0, 2.0)
    rng = np.random.default_rng(7)
    for fid, mag in ((1, 3e4), (4, 120.0)):
        v = rng.normal(size=s.field_size(fid)) * mag
        s.set_field(fid, v)
        back = s.get_field(fid)
        assert rel_l2(back, v) < 1e-3

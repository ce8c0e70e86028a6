"""Full-size checks of the 512^3 throughput configuration in the launch
configuration bench.py times (fused path).  The FP64 oracle cannot run a
512^3 grid in test time, so the checks are properties that hold at any size
plus the FP32 path against the FP64 path, which matches the oracle to 1e-12
per field on every smaller case of tests/test_gpu_parity.py."""
import numpy as np
import pytest

import paper_2103_12819_b300 as mmx
import workloads as W
from conftest import rel_l2

pytestmark = pytest.mark.gpu

STEPS = 5


@pytest.fixture(scope="module")
def stress_pair():
    w = W.stress(steps=STEPS)
    sims = {}
    for prec in (mmx.FP32, mmx.FP64):
        s = mmx.from_workload(w, prec=prec, path=mmx.PATH_FUSED)
        s.step(STEPS)
        assert s.sync(check=False) == 0, s.last_error()
        sims[prec] = s
    yield w, sims
    for s in sims.values():
        s.close()


def test_stress_512_every_half_step_converges(stress_pair):
    w, sims = stress_pair
    for s in sims.values():
        st = s.get_stats()
        assert st["half_steps"] == 2 * STEPS
        assert 1 <= st["iters_min"] <= st["iters_max"] < w.max_iter
        assert st["last_residual"] < w.tol


def test_stress_512_magnetisation_stays_on_the_sphere(stress_pair):
    """|M| = Ms on every magnetic face after the steps (the trapezoidal update
    with N(), Sec. 3.2.2), checked face by face in both precisions."""
    w, sims = stress_pair
    for prec, tol in ((mmx.FP32, 2e-6), (mmx.FP64, 1e-13)):
        s = sims[prec]
        for fam in range(3):
            ms = s.get_material(9 + fam)
            mag = ms > 0
            m2 = np.zeros(int(mag.sum()))
            for c in range(3):
                m2 += s.get_field(6 + 3 * fam + c)[mag] ** 2
            err = np.abs(np.sqrt(m2) - ms[mag]) / ms[mag]
            assert err.max() <= tol, (prec, fam, err.max())


def test_stress_512_fp32_against_fp64(stress_pair):
    """FP32 storage and arithmetic against FP64 after the steps, per field
    (E 0-2, H 3-5, M 6-14)."""
    w, sims = stress_pair
    a, b = sims[mmx.FP32], sims[mmx.FP64]
    errs = {}
    for fid in range(15):
        errs[fid] = rel_l2(a.get_field(fid), b.get_field(fid))
    print("stress 512^3 FP32 vs FP64 after %d steps:" % STEPS, {k: "%.2e" % v for k, v in errs.items()})
    assert max(errs.values()) <= 1e-5, errs

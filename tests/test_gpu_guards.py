"""Guard bytes after the context's device arrays (the canary check that
stands in for a memory sanitizer): every kernel path leaves them intact, and
a byte written past the end of an array is reported."""
import numpy as np
import pytest

import paper_2103_12819_b300 as mmx
import workloads as W

pytestmark = pytest.mark.gpu


def _run(w, steps, **kw):
    s = mmx.from_workload(w, **kw)
    s.step(steps)
    assert s.sync(check=False) == 0, s.last_error()
    return s


CASES = [
    # headline kernels: bulk-copy fused pass, shared-memory H/M kernel,
    # vectorised first half step, on a ragged guide with a z-PML
    ("fp32_guide", lambda: W.waveguide(n=(100, 37, 50), steps=20), dict(prec=mmx.FP32)),
    # list-driven H/M kernel, per-lane cp.async pass with sigma and mu_r
    ("fp64_random_pml", lambda: W.random_small(22, bc=(W.PEC, W.PEC, W.PML), pml_cells=3, n=(70, 10, 16),
                                               pml_gap=2), dict(prec=mmx.FP64)),
    # the one-column fused pass (periodic x and y) and the first-order scheme
    ("fp64_periodic_order1", lambda: W.random_small(17, bc=(W.PEC, W.PERIODIC, W.PEC), order=1),
     dict(prec=mmx.FP64)),
    # the per-update kernels with hard sources
    ("fp32_plain_hard", lambda: W.random_small(16, hard=True), dict(prec=mmx.FP32, path=mmx.PATH_PLAIN)),
    # FP16 storage
    ("fp16_guide", lambda: W.waveguide(n=(32, 24, 96), steps=20), dict(prec=mmx.FP16)),
]


@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_guards_intact_after_stepping(name, make, kw):
    w = make()
    if kw.get("prec") in (mmx.FP32, mmx.FP16):
        w.tol = max(w.tol, 1e-6)
    s = _run(w, 12, **kw)
    for fid in range(15):
        s.get_field(fid)          # the read-back kernels too
    s.check_guards()
    s.close()


def test_guards_intact_after_the_adjoint():
    w = W.filter_design((16, 12, 48), dx=1.6e-3, npml=6, steps=40)
    s = mmx.from_workload(w, prec=mmx.FP64, path=mmx.PATH_PLAIN)
    s.flux_gradient(w.flux_k, 40, 8, with_h0=True)
    s.check_guards()
    s.close()


def test_a_byte_past_the_end_is_reported():
    """The host writes one byte into the guard after Ex (inside the same
    allocation, so nothing faults); the check reports it, and passes again
    once the pattern is restored."""
    from cuda.bindings import runtime as cudart
    w = W.waveguide(n=(32, 24, 64), steps=4)
    s = _run(w, 4, prec=mmx.FP32)
    s.check_guards()
    ptr, sx, sy = s.get_field_device(0)
    end = ptr + sy * (w.n[2] + 1) * 4          # the padded Ex array, FP32
    h2d = cudart.cudaMemcpyKind.cudaMemcpyHostToDevice
    bad = np.array([0x5A], dtype=np.uint8)
    err, = cudart.cudaMemcpy(end + 17, bad.ctypes.data, 1, h2d)
    assert err == cudart.cudaError_t.cudaSuccess
    with pytest.raises(mmx.MMXError) as ei:
        s.check_guards()
    assert ei.value.code == -1 and "past their end" in s.last_error()
    good = np.array([0xC3], dtype=np.uint8)
    err, = cudart.cudaMemcpy(end + 17, good.ctypes.data, 1, h2d)
    assert err == cudart.cudaError_t.cudaSuccess
    s.check_guards()
    s.close()

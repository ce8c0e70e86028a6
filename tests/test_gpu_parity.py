"""GPU (sm_103a) vs FP64 CPU oracle, element by element, through the C ABI.

FP64 bar: relative L2 <= 1e-12 per field (E 3, H 3, M 9 and the PML parts),
and identical H/M iteration counts for every half step (the domain-wide
stopping rule of Sec. 3.2.2 must make the same decisions)."""
import numpy as np
import pytest

import oracle
import paper_2103_12819_b300 as mmx
import workloads as W
from conftest import rel_l2

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _compare(sim, ref, fids=range(15), tol=TOL64, label=""):
    worst = {}
    for fid in fids:
        a = sim.get_field(fid)
        b = ref.get_field(fid)
        nb = np.linalg.norm(b)
        err = rel_l2(a, b) if nb > 0 else float(np.abs(a - b).max())
        worst[fid] = err
        assert err <= tol, (label, fid, err)
    return worst


def _run_pair(w, steps, prec=mmx.FP64, path=mmx.PATH_PLAIN):
    ref = oracle.from_workload(w)
    ref.step(steps)
    sim = mmx.from_workload(w, prec=prec, path=path)
    sim.step(steps)
    assert sim.sync(check=False) == 0, sim.last_error()
    return sim, ref


# The PML split parts (fields 15-18) are the z-derivative shares of Ex, Ey,
# Hx, Hy; where the physics leaves a component near zero (Hy of a TE10 wave)
# its split part is rounding-level, so two kernels that round differently
# are compared on it against the size of the component it belongs to.
_SPLIT_PARENT = {15: 0, 16: 1, 17: 3, 18: 4}


def _rel_to_scale(a_sim, b_sim, fid):
    a, b = a_sim.get_field(fid), b_sim.get_field(fid)
    if fid in _SPLIT_PARENT:
        scale = np.linalg.norm(b_sim.get_field(_SPLIT_PARENT[fid]))
        return float(np.linalg.norm(a - b) / scale) if scale > 0 else float(np.abs(a - b).max())
    return rel_l2(a, b)


# ------------------------------------------------------------------ a1 setup

@pytest.mark.parametrize("bc", [(W.PEC,) * 3, (W.PERIODIC,) * 3, (W.PERIODIC, W.PEC, W.PML)])
def test_a1_materials_match_oracle(bc):
    w = W.random_small(3, n=(7, 6, 12), bc=bc, pml_cells=3 if bc[2] == W.PML else 0)
    ref = oracle.from_workload(w)
    sim = mmx.from_workload(w)
    for which in range(18):
        np.testing.assert_allclose(sim.get_material(which), ref.get_material(which), rtol=1e-15,
                                   err_msg=str(which))


@pytest.mark.parametrize("prec,tol", [(mmx.FP64, 1e-15), (mmx.FP32, 2e-7)])
def test_a1_initial_m_matches_oracle(prec, tol):
    w = W.random_small(4, n=(6, 7, 5), bc=(W.PEC, W.PERIODIC, W.PEC))
    ref = oracle.from_workload(w)
    sim = mmx.from_workload(w, prec=prec)
    for fid in range(6, 15):
        assert rel_l2(sim.get_field(fid), ref.get_field(fid)) <= tol, fid


# ------------------------------------------- the coupled step, FP64 parity

PATHS = [mmx.PATH_PLAIN, mmx.PATH_FUSED]
PATH_IDS = ["plain", "fused"]


@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_yig_slab_32_fp64_200_steps(path):
    """The 32^3 YIG-slab box: 200 steps, tol 1e-10, PEC, point Jx source."""
    w = W.yig_slab_32()
    sim, ref = _run_pair(w, w.steps, path=path)
    _compare(sim, ref, label="yig_slab_32")
    np.testing.assert_array_equal(sim.get_iter_log(), ref.iter_log())


CASES = [
    dict(seed=11, bc=(W.PEC, W.PEC, W.PEC)),
    dict(seed=12, bc=(W.PERIODIC, W.PERIODIC, W.PERIODIC)),
    dict(seed=13, bc=(W.PERIODIC, W.PEC, W.PERIODIC)),
    dict(seed=14, bc=(W.PEC, W.PEC, W.PML), pml_cells=3, n=(6, 5, 16)),
    dict(seed=15, bc=(W.PERIODIC, W.PERIODIC, W.PML), pml_cells=4, n=(5, 4, 18)),
    dict(seed=16, bc=(W.PEC, W.PEC, W.PEC), hard=True),
    dict(seed=17, bc=(W.PEC, W.PERIODIC, W.PEC), order=1),
    dict(seed=18, bc=(W.PERIODIC, W.PEC, W.PEC), magnetic=False),
    dict(seed=19, bc=(W.PEC, W.PEC, W.PEC), n=(2, 9, 7)),
    # wider than one FP64 strip (64 columns): two and three strips, ragged
    # last strip and row tile.  Seed 20's magnetic box reaches the PML's
    # neighbouring layer, so its fused path is k_fused; seed 21 runs the
    # vectorised kernel (more such grids, with the kernel that ran checked,
    # in test_gpu_edge_cases.py)
    dict(seed=20, bc=(W.PEC, W.PEC, W.PML), pml_cells=3, n=(70, 10, 14)),
    dict(seed=21, bc=(W.PEC, W.PEC, W.PEC), n=(131, 4, 5)),
]


@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
@pytest.mark.parametrize("case", CASES, ids=[str(c["seed"]) for c in CASES])
def test_random_small_fp64(case, path):
    kw = dict(case)
    seed = kw.pop("seed")
    w = W.random_small(seed, **kw)
    sim, ref = _run_pair(w, 8, path=path)
    fids = list(range(15)) + ([15, 16, 17, 18] if w.bc[2] == W.PML else [])
    _compare(sim, ref, fids=fids, label=str(seed))
    np.testing.assert_array_equal(sim.get_iter_log(), ref.iter_log()[: len(sim.get_iter_log())])


@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_convergence_problem_32_fp64(path):
    """The paper's periodic coupled problem (Sec. 5.1) on 32^3, 5 steps:
    magnetic everywhere, sigma/eps/Ms/alpha/gamma bumps."""
    w = W.convergence(32)
    sim, ref = _run_pair(w, w.steps, path=path)
    _compare(sim, ref, label="convergence_32")
    np.testing.assert_array_equal(sim.get_iter_log(), ref.iter_log())


def test_waveguide_full_size_fp64_parity():
    """The 128x128x512 waveguide (z-PML, YIG slab, TE10 source) at full size,
    in the benchmark's launch configuration (fused path), 6 steps against
    the oracle."""
    w = W.waveguide(steps=6)
    sim, ref = _run_pair(w, 6, path=mmx.PATH_FUSED)
    _compare(sim, ref, fids=list(range(19)), label="waveguide")
    np.testing.assert_array_equal(sim.get_iter_log(), ref.iter_log())


# ----------------------------------------------------------- FP32 path

@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_fp32_error_against_oracle_yig_slab(path):
    """FP32 storage and arithmetic (the residual compared in FP64): stated
    error after 200 steps of the 32^3 slab."""
    w = W.yig_slab_32()
    w.tol = 1e-6
    ref = oracle.from_workload(w)
    ref.step(w.steps)
    sim = mmx.from_workload(w, prec=mmx.FP32, path=path)
    sim.step(w.steps)
    assert sim.sync(check=False) == 0
    errs = {fid: rel_l2(sim.get_field(fid), ref.get_field(fid)) for fid in range(15)}
    print("fp32 rel L2 per field:", {k: "%.2e" % v for k, v in errs.items()})
    assert max(errs.values()) < 1e-4, errs


# ------------------------------------------------------- error reporting

def test_bounded_wait_gives_up_and_context_stays_usable():
    """Failure detection without a fault: the grid barrier and the voting
    barrier of the H/M iteration, each in a grid where one block never
    arrives, give up after their wait budgets (about a second each), the host
    reads MMX_ERR_TIMEOUT, and the same context then steps and matches the
    oracle."""
    import time
    w = W.yig_slab_32(steps=4, n=16)
    sim = mmx.from_workload(w, prec=mmx.FP64)
    t0 = time.perf_counter()
    assert sim.check_bounded_wait() == -6
    assert time.perf_counter() - t0 < 30
    assert sim.check_bounded_wait() == -6            # repeatable
    sim.step(4)
    assert sim.sync(check=False) == 0
    ref = oracle.from_workload(w)
    ref.step(4)
    _compare(sim, ref, label="after the wait check")
    ref.close()
    sim.close()


def test_m_field_round_trip():
    """set_field / get_field of the nine M components: M is stored on the
    magnetic box only, so a round trip returns the values set on magnetic
    faces exactly and, elsewhere, either the value set (inside the box) or
    zero (outside it)."""
    w = W.yig_slab_32(steps=2, n=16)
    sim = mmx.from_workload(w, prec=mmx.FP64)
    rng = np.random.default_rng(12)
    for fid in range(6, 15):
        mag = sim.get_field(fid) != 0.0
        assert mag.any()
        v = rng.normal(size=sim.field_size(fid)) * 1e5
        sim.set_field(fid, v)
        back = sim.get_field(fid)
        np.testing.assert_array_equal(back[mag], v[mag])
        assert np.all((back == v) | (back == 0.0)), fid
        sim.set_field(fid, np.where(mag, v, 0.0))
        np.testing.assert_array_equal(sim.get_field(fid), np.where(mag, v, 0.0))
    sim.close()


def test_iteration_cap_is_reported():
    w = W.yig_slab_32(steps=2)
    w.max_iter = 1
    sim = mmx.from_workload(w)
    sim.step(1)
    assert sim.sync(check=False) == -4
    assert sim.sync(check=False) == 0      # reading clears the latch


def test_nonfinite_is_reported():
    w = W.yig_slab_32(steps=2)
    sim = mmx.from_workload(w)
    e = np.zeros(sim.field_size(0))
    e[16 + 32 * (16 + 33 * 16)] = np.nan       # interior Ex edge (16.5, 16, 16)
    sim.set_field(0, e)
    sim.step(1)
    assert sim.sync(check=False) == -5


@pytest.mark.parametrize("prec", [mmx.FP64, mmx.FP32], ids=["fp64", "fp32"])
def test_fused_equals_plain(prec):
    """The fused pass and the one-kernel-per-update path compute the same
    scheme: identical iteration counts and fields equal to rounding (the PML
    split part is carried instead of re-derived, the only reordering)."""
    w = W.waveguide(n=(24, 20, 48), steps=30)
    a = mmx.from_workload(w, prec=prec, path=mmx.PATH_PLAIN)
    b = mmx.from_workload(w, prec=prec, path=mmx.PATH_FUSED)
    for chunk in (7, 1, 12, 10):           # several mmx_step call patterns
        a.step(chunk)
        b.step(chunk)
    assert a.sync(check=False) == 0 and b.sync(check=False) == 0
    for fid in range(19):
        tol = 1e-13 if prec == mmx.FP64 else 1e-5
        assert _rel_to_scale(b, a, fid) <= tol, fid
    np.testing.assert_array_equal(a.get_iter_log(), b.get_iter_log())


# ------------------------------------------- vectorised fused kernel

def _kernels_seen(sim, nsteps):
    sim.set_profiling(True)
    sim.get_profile(reset=True)
    sim.step(nsteps)
    prof = sim.get_profile(reset=True)
    sim.set_profiling(False)
    return prof


@pytest.mark.parametrize("prec", [mmx.FP64, mmx.FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("n", [(140, 12, 40), (70, 9, 33), (24, 20, 48)], ids=["x140", "x70", "x24"])
def test_vectorised_fused_equals_plain(prec, n):
    """The vectorised fused kernel (PEC x/y) against the per-update kernels on
    waveguides one to three strips wide in either precision (FP32 strips are
    128 columns, FP64 64), with the fused call pattern split over several
    mmx_step calls; the fused path must actually run the vectorised kernel."""
    w = W.waveguide(n=n, steps=12)
    a = mmx.from_workload(w, prec=prec, path=mmx.PATH_PLAIN)
    b = mmx.from_workload(w, prec=prec, path=mmx.PATH_FUSED)
    a.step(5)
    b.step(5)
    a.step(4)
    prof = _kernels_seen(b, 4)
    # FP32 without sigma or mu_r stages its planes with bulk tensor copies
    want = "fused_eh_vec_tma" if prec == mmx.FP32 else "fused_eh_vec"
    assert want in prof and "fused_eh" not in prof, prof
    assert b.get_info()["fused_kernel_name"] == ("k_fused_vec_tma" if prec == mmx.FP32 else "k_fused_vec")
    a.step(3)
    b.step(3)
    assert a.sync(check=False) == 0 and b.sync(check=False) == 0
    for fid in range(19):
        tol = 1e-13 if prec == mmx.FP64 else 1e-5
        assert _rel_to_scale(b, a, fid) <= tol, fid
    np.testing.assert_array_equal(a.get_iter_log(), b.get_iter_log())


def test_bulk_copy_fused_pass_is_deterministic():
    """The bulk-copy fused pass has one block barrier per plane, so warps run
    up to a plane apart and the exchange rows they share must be buffered
    deeply enough.  Two fresh runs of the full 128x128x512 waveguide (chunks of
    about 34 planes, FP32) must give bit-identical fields: a warp overwriting
    rows another still reads would show as a difference."""
    import hashlib
    w = W.waveguide(steps=300)
    digests = []
    for _ in range(2):
        sim = mmx.from_workload(w, prec=mmx.FP32, path=mmx.PATH_FUSED)
        prof = _kernels_seen(sim, 2)
        assert "fused_eh_vec_tma" in prof, prof
        sim.step(298)
        assert sim.sync(check=False) == 0
        digests.append([hashlib.sha256(np.ascontiguousarray(sim.get_field(fid)).tobytes()).hexdigest()
                        for fid in range(19)])
        sim.close()
    assert digests[0] == digests[1]


@pytest.mark.parametrize("bcz,n", [(W.PERIODIC, (140, 9, 12)), (W.PEC, (37, 11, 10))], ids=["periodic-z", "pec-z"])
def test_bulk_copy_staging_equals_plain_fp32(bcz, n):
    """FP32 storage without sigma or mu_r stages the fused kernel's planes with
    bulk tensor copies: on a periodic z axis (the staged cell plane wraps, node
    nz repeats node 0) over two strips, and on a ragged PEC box, it matches the
    per-update kernels to FP32 rounding."""
    w = W.random_small(31, n=n, bc=(W.PEC, W.PEC, bcz), tol=1e-6)
    w.sigma = np.zeros_like(w.sigma)
    w.mu_r = np.ones_like(w.mu_r)
    w.sources = [q for q in w.sources if q.kind < 2]
    a = mmx.from_workload(w, prec=mmx.FP32, path=mmx.PATH_PLAIN)
    b = mmx.from_workload(w, prec=mmx.FP32, path=mmx.PATH_FUSED)
    a.step(6)
    prof = _kernels_seen(b, 6)
    assert "fused_eh_vec_tma" in prof and "fused_eh_vec" not in prof, prof
    assert a.sync(check=False) == 0 and b.sync(check=False) == 0
    for fid in range(15):
        assert _rel_to_scale(b, a, fid) <= 1e-5, fid


@pytest.mark.parametrize("n", [(20, 12, 32), (64, 16, 32)], ids=["ragged", "strip_multiple"])
def test_vectorised_fused_after_set_field_keeps_walls(n):
    """Nonzero values written onto the x = nx / y = ny PEC walls by set_field
    are cleared before the vectorised kernel runs, as the per-update path
    clears them in its first step.  With nx a multiple of the FP64 strip
    width (64) and ny of the row block (8), the vectorised first half step
    leaves the wall column and row to the wall clearing."""
    w = W.waveguide(n=n, steps=4)
    a = mmx.from_workload(w, prec=mmx.FP64, path=mmx.PATH_PLAIN)
    b = mmx.from_workload(w, prec=mmx.FP64, path=mmx.PATH_FUSED)
    rng = np.random.default_rng(5)
    for fid in range(6):
        v = rng.standard_normal(a.field_size(fid))
        a.set_field(fid, v)
        b.set_field(fid, v)
    a.step(3)
    b.step(3)
    for fid in range(19):
        assert _rel_to_scale(b, a, fid) <= 1e-13, fid


def test_fp32_multi_strip_against_oracle():
    """FP32 vectorised fused path on a grid three FP32 strips wide (x = 300)
    against the FP64 oracle."""
    w = W.random_small(22, n=(300, 3, 6), bc=(W.PEC, W.PEC, W.PEC))
    w.tol = 1e-6
    sim, ref = _run_pair(w, 6, path=mmx.PATH_FUSED, prec=mmx.FP32)
    for fid in range(15):
        a, b = sim.get_field(fid), ref.get_field(fid)
        assert rel_l2(a, b) <= 1e-4, fid


# ----------------------------------------------------------- probes

@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_probes_record_e_after_every_step(path):
    """Each probe row is E^(n+1) after step n: the last row equals the field
    read back at the end, and row r equals a run stopped after r+1 steps."""
    w = W.waveguide(n=(24, 20, 48), steps=12)
    pts = [(0, 5, 6, 7), (1, 12, 3, 30), (2, 3, 4, 5)]
    s = mmx.from_workload(w, path=path)
    for p in pts:
        s.add_probe(*p)
    s.step(5)
    s.step(7)
    rows = s.get_probes()
    assert rows.shape == (12, 3)
    for c, (fid, i, j, k) in enumerate(pts):
        ext = W.field_extent(fid, w.n)
        fin = s.get_field(fid).reshape(ext[2], ext[1], ext[0])[k, j, i]
        assert rows[-1, c] == fin
    r = mmx.from_workload(w, path=path)
    r.step(4)
    for c, (fid, i, j, k) in enumerate(pts):
        ext = W.field_extent(fid, w.n)
        assert rows[3, c] == r.get_field(fid).reshape(ext[2], ext[1], ext[0])[k, j, i]
    assert s.get_probes().shape == (0, 3)          # reset by the previous read
    with pytest.raises(mmx.MMXError):
        s.add_probe(3, 0, 0, 0)                    # H is not probed
    with pytest.raises(mmx.MMXError):
        s.add_probe(0, w.n[0], 0, 0)               # Ex has nx edges along x

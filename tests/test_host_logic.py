"""Host-side logic that needs no GPU: the seeded workload generators of the
sweep and the guide, bench.py's byte accounting and its captured-traffic
lookup, and the autotuner's size-class key and cache."""
import json
import os

import numpy as np
import pytest

import bench
import workloads as W


def test_bias_sweep_is_seeded_and_in_range():
    a, b = W.bias_sweep(256), W.bias_sweep(256)
    assert a == b
    ns = {n for n, _, _ in a}
    assert ns <= {32, 48, 64, 96} and len(ns) == 4
    h0 = np.array([h for _, h, _ in a])
    assert h0.min() >= 5e4 and h0.max() <= 2e5
    assert len({s for _, _, s in a}) == 256


def test_tunable_filter_structure():
    w = W.tunable_filter(32, 1.2e5, seed=9)
    assert w.n == (32, 32, 32) and w.bc == (W.PEC, W.PEC, W.PEC)
    mag = w.Ms > 0
    zs = np.nonzero(mag.any(axis=(1, 2)))[0]
    assert zs.min() == 12 and zs.max() == 19          # middle quarter of z
    assert mag[12:20].all()
    m = np.sqrt(sum(c ** 2 for c in w.m_cells))
    assert np.all(w.m_cells[2][mag] / m[mag] > 0.99)         # z plus a 1% tilt (renormalised on upload)
    assert w.h0 == (0.0, 0.0, 1.2e5)
    (src,) = w.sources
    assert src.kind == W.SRC_POINT_J and src.comp == 0 and src.f0 == 5e9


def test_air_guide_matches_the_paper_geometry():
    w = W.air_guide()
    assert w.n[:2] == (75, 51)
    assert abs(w.n[0] * w.d[0] - 14.95e-3) < 1e-12 and abs(w.n[1] * w.d[1] - 10.16e-3) < 1e-12
    assert w.bc == (W.PEC, W.PEC, W.PML) and w.pml_cells == 10
    assert not np.any(w.Ms > 0)


def test_stress_block_is_centred():
    w = W.stress(n=16)
    mag = w.Ms > 0
    idx = np.nonzero(mag)
    assert all(int(v.min()) == 4 and int(v.max()) == 11 for v in idx)


def test_algorithmic_bytes():
    assert bench.alg_bytes_per_cell("fused_eh_vec", None, 4) == 52
    assert bench.alg_bytes_per_cell("fused_eh_vec", None, 8) == 104
    assert bench.alg_bytes_per_cell("fused_eh_vec", None, 4, 2) == 28
    assert bench.alg_bytes_per_cell("e_update", None, 4) == 40
    assert bench.alg_bytes_per_cell("h_update", None, 4) == 36
    assert bench.alg_bytes_per_cell("hm_box", None, 4) is None


def test_captured_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    sha = bench.kernel_source_sha256()
    assert sha == bench.kernel_source_sha256() and len(sha) == 64
    prof = tmp_path / "profiles"
    prof.mkdir()
    name = "fused_eh_vec_%s_fp32.md" % bench.WORKLOAD
    (prof / name).write_text("# x\n\n- source_sha256: `%s`\n- traffic_bytes_per_launch: 12345\n" % sha)
    csrc = os.path.join(bench.ROOT, "paper_2103_12819_b300", "csrc")
    (tmp_path / "paper_2103_12819_b300").mkdir()
    os.symlink(csrc, tmp_path / "paper_2103_12819_b300" / "csrc")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.captured_traffic("fused_eh_vec", "fp32") == 12345
    (prof / name).write_text("# x\n\n- source_sha256: `%s`\n- traffic_bytes_per_launch: 12345\n" % ("0" * 64))
    assert bench.captured_traffic("fused_eh_vec", "fp32") is None       # stale capture
    assert bench.captured_traffic("fused_eh_vec", "fp64") is None       # no capture


def test_autotune_signature_and_cache(tmp_path):
    from paper_2103_12819_b300 import autotune

    class Fake:
        def __init__(self, n, prec):
            self.n, self.prec = n, prec

    a = autotune._signature([Fake((32, 32, 32), 1), Fake((48, 48, 48), 1), Fake((32, 32, 32), 1)])
    b = autotune._signature([Fake((48, 48, 48), 1), Fake((32, 32, 32), 1), Fake((32, 32, 32), 1)])
    assert a == b == "prec1:32x32x32*2,48x48x48*1"
    assert autotune._signature([Fake((32, 32, 32), 0)]) != autotune._signature([Fake((32, 32, 32), 1)])
    path = tmp_path / "t.json"
    assert autotune._load(str(path)) == {}
    path.write_text(json.dumps({a: {"planes": 16}}))
    assert autotune._load(str(path))[a]["planes"] == 16
    path.write_text("not json")
    assert autotune._load(str(path)) == {}

"""The allocation-free material-mean entry point, for callers that cannot call
cudaMalloc (device memory owned by their own arena, or no allocation allowed
where they run).  Collected last so that a run stopping at the first failure
has already run every other test.

It must give the same edge/face means as the context path (mmx_get_material)
on two calls in a row, reusing the library's fixed scratch array, and reject a
grid too large for that array."""
import numpy as np
import pytest

import paper_2103_12819_b300 as mmx
import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_mean_matches_context_readback_twice():
    import torch
    w = W.random_small(41, n=(9, 7, 11), bc=(W.PERIODIC, W.PEC, W.PEC))
    sim = mmx.from_workload(w)
    # (context readback id, cell array, no-alloc location): an edge mean of
    # eps_r, then a face mean of |gamma|, back to back on the same scratch
    cases = [(1, w.eps_r, 1), (17, w.gamma, 5)]
    for which, cell, loc in cases:
        ref = sim.get_material(which)
        cell_d = torch.tensor(np.ascontiguousarray(cell, dtype=np.float64).ravel(), device="cuda")
        out_d = torch.full((ref.size,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        rc = mmx.material_average_noalloc(w.n, w.bc, loc, cell_d.data_ptr(), out_d.data_ptr(), ref.size)
        assert rc == 0
        torch.cuda.synchronize()
        got = out_d.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-15, atol=0)


def test_noalloc_rejects_oversize_grid():
    import torch
    n = (127, 127, 127)        # 128*128*128 padded elements > 1,048,576
    cell = torch.zeros(n[0] * n[1] * n[2], dtype=torch.float64, device="cuda")
    out = torch.zeros((n[0] + 1) * n[1] * n[2], dtype=torch.float64, device="cuda")
    rc = mmx.material_average_noalloc(n, (1, 1, 1), 3, cell.data_ptr(), out.data_ptr(), out.numel())
    assert rc == -1

"""Checkpoint and resume through the public API: every field read back with
get_field and the step count, restored into a fresh context built from the
same workload, continue exactly as the uninterrupted context does."""
import numpy as np
import pytest

import paper_2103_12819_b300 as mmx
import workloads as W

pytestmark = pytest.mark.gpu

NFIELDS = 19      # E, H, the 9 M components, the 4 PML split parts


@pytest.mark.parametrize("prec", [mmx.FP64, mmx.FP32], ids=["fp64", "fp32"])
def test_restored_context_continues_bit_for_bit(prec):
    """A 32x24x96 guide (z-PML, TE10 plane source in mid-pulse, YIG slab):
    30 steps, checkpoint, 20 more steps, against 30 + 20 steps in one
    context with the same call pattern.  Fields and the second segment's
    iteration counts agree exactly."""
    w = W.waveguide(n=(32, 24, 96), steps=50)
    if prec == mmx.FP32:
        w.tol = 1e-6
    ref = mmx.from_workload(w, prec=prec)
    ref.step(30)
    ref.sync()
    n_log = len(ref.get_iter_log())
    ref.step(20)
    ref.sync()

    a = mmx.from_workload(w, prec=prec)
    a.step(30)
    a.sync()
    saved = [a.get_field(fid).copy() for fid in range(NFIELDS)]
    steps = a.get_stats()["steps"]
    a.close()
    assert steps == 30

    b = mmx.from_workload(w, prec=prec)
    for fid in range(NFIELDS):
        b.set_field(fid, saved[fid])
    b.set_step_count(steps)
    b.step(20)
    assert b.sync(check=False) == 0, b.last_error()
    assert b.get_stats()["steps"] == 50
    for fid in range(NFIELDS):
        np.testing.assert_array_equal(b.get_field(fid), ref.get_field(fid), err_msg=str(fid))
    np.testing.assert_array_equal(b.get_iter_log(), ref.get_iter_log()[n_log:])
    b.check_guards()


def test_step_count_rejects_negative():
    w = W.waveguide(n=(16, 12, 32), steps=1)
    s = mmx.from_workload(w)
    with pytest.raises(mmx.MMXError):
        s.set_step_count(-1)

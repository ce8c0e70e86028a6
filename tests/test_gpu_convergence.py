"""The paper's convergence study (Sec. 5.1, Table 2) on the GPU path: the
periodic coupled problem at 32^3, 64^3 and 128^3 cells with the paper's 5,
10 and 20 steps (same physical time) and iteration tolerance 1e-6.  The L1
difference between successive resolutions (fine restricted to coarse as in
Sec. 5.1) must fall at the printed second-order rates in every E, H and M
component, in FP64 and, with a looser bar, in FP32."""
import math

import numpy as np
import pytest

import paper_2103_12819_b300 as mmx
import workloads as W
from test_oracle_pins import _restrict, _table2

pytestmark = pytest.mark.gpu

NAMES = {0: "Ex", 1: "Ey", 2: "Ez", 3: "Hx", 4: "Hy", 5: "Hz", 6: "Mx", 10: "My", 14: "Mz"}


def _solutions(prec):
    sols = {}
    for nn in (32, 64, 128):
        w = W.convergence(nn, tol=1e-6)
        s = mmx.from_workload(w, prec=prec, path=mmx.PATH_FUSED)
        s.step(w.steps)
        assert s.sync(check=False) == 0, s.last_error()
        sols[nn] = {fid: s.get_field(fid) for fid in NAMES}
        s.close()
    return sols


@pytest.mark.parametrize("prec,bar", [(mmx.FP64, 0.05), (mmx.FP32, 0.1)], ids=["fp64", "fp32"])
def test_table2_rates_on_the_gpu(prec, bar):
    sols = _solutions(prec)
    tab = _table2()
    rates = {}
    for fid, name in NAMES.items():
        e1 = np.mean(np.abs(_restrict(fid, sols[64][fid], (32,) * 3) - sols[32][fid]))
        e2 = np.mean(np.abs(_restrict(fid, sols[128][fid], (64,) * 3) - sols[64][fid]))
        rates[name] = math.log2(e1 / e2)
    print("Table 2 rates (GPU, %s):" % ("FP64" if prec == mmx.FP64 else "FP32"),
          {k: round(v, 3) for k, v in rates.items()})
    for name, r in rates.items():
        assert abs(r - tab[name][2]) < bar, (name, r)

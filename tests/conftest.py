import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: CPU test that takes more than ~20 s")


# Physical constants written out by the tests themselves (CODATA 2018 mu0,
# exact c), independent of both the oracle and the CUDA library.
MU0 = 1.25663706212e-6
C0 = 299792458.0
EPS0 = 1.0 / (MU0 * C0 * C0)


def positions(fid, n, d):
    """Physical coordinates (X, Y, Z), each shaped (ez, ey, ex), of the Yee
    location of field id ``fid`` (0-2 E edges, 3-5 H faces, 6-14 M faces)."""
    node = [np.arange(m + 1) * h for m, h in zip(n, d)]
    half = [(np.arange(m) + 0.5) * h for m, h in zip(n, d)]
    if fid < 3:
        axes = [half[a] if a == fid else node[a] for a in range(3)]
    else:
        fam = fid - 3 if fid < 6 else (fid - 6) // 3
        axes = [node[a] if a == fam else half[a] for a in range(3)]
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return X, Y, Z


def rel_l2(a, b, floor=0.0):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    if nb <= floor:
        return float(np.max(np.abs(a - b))) if a.size else 0.0
    return float(np.linalg.norm(a - b) / nb)

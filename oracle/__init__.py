"""ctypes wrapper of the plain FP64 CPU oracle (``mmx_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and
by the benchmark's CPU-baseline leg, never by the product library.  It shares
no code with the CUDA path; it only reads the seeded inputs of ``workloads``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mmx_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmmx_oracle.so")
_lock = threading.Lock()
_libs = {}

# Build variants: "" is the oracle; "literal" evaluates Eq. iterate_H as
# printed in FP64 (ORC_LITERAL_ITERATE_H), used only to bound the effect of
# readings R13/R14 in a test.
# "omp" parallelises the loops over z planes and magnetic faces with OpenMP,
# bit-identical to "" and used only to time the oracle on all host cores.
_VARIANTS = {"": [], "literal": ["-DORC_LITERAL_ITERATE_H=1"], "omp": ["-fopenmp"]}

ERR_NAMES = {0: "OK", -1: "INVALID", -2: "OOM", -4: "NOT_CONVERGED", -5: "NONFINITE"}


def build(force: bool = False, variant: str = "") -> str:
    """Compile the oracle with gcc (-O2, no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    path = _LIB_PATH if not variant else os.path.join(_BUILD, "libmmx_oracle_%s.so" % variant)
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
        return path
    tmp = path + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math"] + _VARIANTS[variant] + ["-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def lib(variant: str = ""):
    with _lock:
        if variant not in _libs:
            L = ctypes.CDLL(build(variant=variant))
            P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
            dp = ctypes.POINTER(ctypes.c_double)
            L.orc_create.restype = P
            L.orc_create.argtypes = [I, I, I, D, D, D, D, ctypes.POINTER(I), I, I, D, I]
            L.orc_destroy.argtypes = [P]
            L.orc_set_materials.restype = I
            L.orc_set_materials.argtypes = [P, dp, dp, dp, dp, dp, dp]
            L.orc_set_bias.argtypes = [P, D, D, D]
            L.orc_set_M_cells.restype = I
            L.orc_set_M_cells.argtypes = [P, dp, dp, dp]
            L.orc_set_field.restype = I
            L.orc_set_field.argtypes = [P, I, dp]
            L.orc_get_field.restype = I
            L.orc_get_field.argtypes = [P, I, dp]
            L.orc_get_material.restype = I
            L.orc_get_material.argtypes = [P, I, dp]
            L.orc_field_size.restype = LL
            L.orc_field_size.argtypes = [P, I]
            L.orc_add_source.restype = I
            L.orc_add_source.argtypes = [P, I, I, I, I, I, D, D, D, D]
            L.orc_step.restype = I
            L.orc_step.argtypes = [P, I]
            L.orc_iter_log.restype = LL
            L.orc_iter_log.argtypes = [P, ctypes.POINTER(I), LL]
            L.orc_last_residual.restype = D
            L.orc_last_residual.argtypes = [P]
            L.orc_steps_done.restype = LL
            L.orc_steps_done.argtypes = [P]
            _libs[variant] = L
    return _libs[variant]


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what}: {ERR_NAMES.get(code, code)}")
        self.code = code


class Sim:
    """One oracle simulation instance (cell-centred inputs, Yee-located fields)."""

    def __init__(self, n, d, dt, bc, pml_cells=0, order=2, tol=1e-10, max_iter=64, variant=""):
        self._L = lib(variant)
        self.n = tuple(int(v) for v in n)
        bcs = (ctypes.c_int * 3)(*[int(b) for b in bc])
        self._h = self._L.orc_create(self.n[0], self.n[1], self.n[2], float(d[0]), float(d[1]),
                                     float(d[2]), float(dt), bcs, int(pml_cells), int(order),
                                     float(tol), int(max_iter))
        if not self._h:
            raise OracleError(-1, "create")

    def close(self):
        if getattr(self, "_h", None):
            self._L.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _c(a):
        if a is None:
            return None
        return np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel())

    def set_materials(self, eps_r=None, sigma=None, mu_r=None, Ms=None, alpha=None, gamma=None):
        arrs = [self._c(a) for a in (eps_r, sigma, mu_r, Ms, alpha, gamma)]
        rc = self._L.orc_set_materials(self._h, *[_dptr(a) for a in arrs])
        if rc:
            raise OracleError(rc, "set_materials")

    def set_bias(self, hx, hy, hz):
        self._L.orc_set_bias(self._h, float(hx), float(hy), float(hz))

    def set_M_cells(self, mx, my, mz):
        arrs = [self._c(a) for a in (mx, my, mz)]
        rc = self._L.orc_set_M_cells(self._h, *[_dptr(a) for a in arrs])
        if rc:
            raise OracleError(rc, "set_M_cells")

    def field_size(self, fid):
        return int(self._L.orc_field_size(self._h, int(fid)))

    def set_field(self, fid, values):
        a = self._c(values)
        if a.size != self.field_size(fid):
            raise ValueError("field %d: size %d != %d" % (fid, a.size, self.field_size(fid)))
        rc = self._L.orc_set_field(self._h, int(fid), _dptr(a))
        if rc:
            raise OracleError(rc, "set_field")

    def get_field(self, fid) -> np.ndarray:
        out = np.empty(self.field_size(fid), dtype=np.float64)
        rc = self._L.orc_get_field(self._h, int(fid), _dptr(out))
        if rc:
            raise OracleError(rc, "get_field")
        return out

    def get_material(self, which) -> np.ndarray:
        """0-2 eps_r on Ex/Ey/Ez edges, 3-5 sigma on edges, 6-8 mu_r, 9-11 Ms,
        12-14 alpha, 15-17 |gamma| on x/y/z faces."""
        fid = (which % 3) if which < 6 else 3 + which % 3
        out = np.empty(self.field_size(fid), dtype=np.float64)
        rc = self._L.orc_get_material(self._h, int(which), _dptr(out))
        if rc:
            raise OracleError(rc, "get_material")
        return out

    def add_source(self, kind, comp, i=0, j=0, k=0, amp=0.0, f0=0.0, tp=1.0, t0=0.0):
        rc = self._L.orc_add_source(self._h, int(kind), int(comp), int(i), int(j), int(k),
                                    float(amp), float(f0), float(tp), float(t0))
        if rc:
            raise OracleError(rc, "add_source")

    def step(self, nsteps=1, check=True) -> int:
        rc = self._L.orc_step(self._h, int(nsteps))
        if check and rc:
            raise OracleError(rc, "step")
        return rc

    def iter_log(self) -> np.ndarray:
        n = self._L.orc_iter_log(self._h, None, 0)
        out = np.zeros(int(n), dtype=np.int32)
        if n:
            self._L.orc_iter_log(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(n))
        return out

    @property
    def last_residual(self) -> float:
        return float(self._L.orc_last_residual(self._h))

    @property
    def steps_done(self) -> int:
        return int(self._L.orc_steps_done(self._h))


def from_workload(w, with_sources=True, variant="") -> Sim:
    """Build an oracle instance from a ``workloads.Workload``."""
    s = Sim(w.n, w.d, w.dt, w.bc, w.pml_cells, w.order, w.tol, w.max_iter, variant=variant)
    s.set_materials(w.eps_r, w.sigma, w.mu_r, w.Ms, w.alpha, w.gamma)
    s.set_bias(*w.h0)
    if w.m_cells is not None and w.Ms is not None and np.any(w.Ms > 0):
        s.set_M_cells(*w.m_cells)
    for fid, v in w.fields.items():
        s.set_field(fid, v)
    if with_sources:
        for q in w.sources:
            s.add_source(q.kind, q.comp, q.i, q.j, q.k, q.amp, q.f0, q.tp, q.t0)
    return s

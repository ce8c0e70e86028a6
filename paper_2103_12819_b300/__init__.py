"""Python binding of ``libmmx.so``, the sm_103a coupled Maxwell-LLG solver.

Argument marshalling only: every step of the scheme runs in the library's
CUDA kernels.  The entry points keep the C names (``mmx_create``,
``mmx_step`` ...); :class:`Solver` wraps one context.  There is no CPU
fallback: if the shared library is missing or cannot be loaded this module
raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmmx.so")

MMX_OK = 0
ERRORS = {-1: "INVALID", -2: "OOM", -3: "CUDA", -4: "NOT_CONVERGED", -5: "NONFINITE", -6: "TIMEOUT"}
FP64, FP32, FP16 = 0, 1, 2     # FP16: FP16 storage of E and H, FP32 arithmetic
PERIODIC, PEC, PML = 0, 1, 2
PATH_PLAIN, PATH_FUSED = 0, 1


class GridDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("d", ctypes.c_double * 3), ("dt", ctypes.c_double),
                ("bc", ctypes.c_int * 3), ("pml_cells", ctypes.c_int), ("order", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("prec", ctypes.c_int)]


class SourceDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("comp", ctypes.c_int), ("i", ctypes.c_int),
                ("j", ctypes.c_int), ("k", ctypes.c_int), ("amp", ctypes.c_double),
                ("f0", ctypes.c_double), ("tp", ctypes.c_double), ("t0", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("half_steps", ctypes.c_longlong),
                ("iters_min", ctypes.c_int), ("iters_max", ctypes.c_int),
                ("last_residual", ctypes.c_double), ("status", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("fused_kernel", ctypes.c_int), ("tma_fallback", ctypes.c_int),
                ("bulk_staging", ctypes.c_int), ("box_blocks", ctypes.c_int),
                ("box_faces_magnetic", ctypes.c_longlong), ("box_faces_other", ctypes.c_longlong),
                ("box_kernel", ctypes.c_int), ("box_resident_faces_per_thread", ctypes.c_int)]


# mmx_info.fused_kernel -> kernel name
FUSED_KERNELS = {0: "none", 1: "k_fused", 2: "k_fused_vec", 3: "k_fused_vec_tma"}
# mmx_info.box_kernel -> kernel name
BOX_KERNELS = {0: "none", 1: "k_hm_box", 2: "k_hm_box_res"}


class KernelProfile(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_longlong),
                ("total_ms", ctypes.c_double)]


EXPORTS = ("mmx_create", "mmx_set_materials", "mmx_set_bias", "mmx_set_M_cells", "mmx_set_field",
           "mmx_get_field", "mmx_get_material", "mmx_add_source", "mmx_set_path", "mmx_step",
           "mmx_sync", "mmx_get_stats", "mmx_get_iter_log", "mmx_get_field_device", "mmx_check_bounded_wait",
           "mmx_check_guards", "mmx_set_step_count",
           "mmx_inject_timeout", "mmx_get_info", "mmx_set_fused_staging", "mmx_kernel_binary_version",
           "mmx_set_box_kernel",
           "mmx_flux_gradient", "mmx_set_storage_scale", "mmx_add_probe", "mmx_get_probes", "mmx_energy", "mmx_add_flux_plane", "mmx_get_flux",
           "mmx_set_profiling", "mmx_get_profile",
           "mmx_batch_create", "mmx_batch_set_planes", "mmx_batch_set_box_blocks", "mmx_batch_step", "mmx_batch_sync",
           "mmx_batch_last_error", "mmx_batch_destroy",
           "mmx_material_average_noalloc", "mmx_last_error", "mmx_destroy")

_lib = None


def lib():
    """Load libmmx.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libmmx.so is not built: run __graft_entry__.build() (nvcc, sm_103a)")
    L = ctypes.CDLL(LIB_PATH)
    P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    dp = ctypes.POINTER(ctypes.c_double)
    L.mmx_create.restype = I
    L.mmx_create.argtypes = [ctypes.POINTER(GridDesc), P, ctypes.POINTER(P)]
    L.mmx_set_materials.restype = I
    L.mmx_set_materials.argtypes = [P, dp, dp, dp, dp, dp, dp]
    L.mmx_set_bias.restype = I
    L.mmx_set_bias.argtypes = [P, D, D, D]
    L.mmx_set_M_cells.restype = I
    L.mmx_set_M_cells.argtypes = [P, dp, dp, dp]
    L.mmx_set_field.restype = I
    L.mmx_set_field.argtypes = [P, I, dp, LL]
    L.mmx_get_field.restype = I
    L.mmx_get_field.argtypes = [P, I, dp, LL]
    L.mmx_get_material.restype = I
    L.mmx_get_material.argtypes = [P, I, dp, LL]
    L.mmx_add_source.restype = I
    L.mmx_add_source.argtypes = [P, ctypes.POINTER(SourceDesc)]
    L.mmx_set_path.restype = I
    L.mmx_set_path.argtypes = [P, I]
    L.mmx_step.restype = I
    L.mmx_step.argtypes = [P, I]
    L.mmx_sync.restype = I
    L.mmx_sync.argtypes = [P]
    L.mmx_get_stats.restype = I
    L.mmx_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
    L.mmx_get_iter_log.restype = LL
    L.mmx_get_iter_log.argtypes = [P, ctypes.POINTER(ctypes.c_int), LL]
    L.mmx_get_field_device.restype = I
    L.mmx_get_field_device.argtypes = [P, I, ctypes.POINTER(P), ctypes.POINTER(LL), ctypes.POINTER(LL)]
    L.mmx_set_profiling.restype = I
    L.mmx_set_profiling.argtypes = [P, I]
    L.mmx_check_bounded_wait.restype = I
    L.mmx_check_bounded_wait.argtypes = [P]
    L.mmx_check_guards.restype = I
    L.mmx_check_guards.argtypes = [P]
    L.mmx_set_step_count.restype = I
    L.mmx_set_step_count.argtypes = [P, LL]
    L.mmx_inject_timeout.restype = I
    L.mmx_inject_timeout.argtypes = [P]
    L.mmx_get_info.restype = I
    L.mmx_get_info.argtypes = [P, ctypes.POINTER(Info)]
    L.mmx_set_fused_staging.restype = I
    L.mmx_set_fused_staging.argtypes = [P, I]
    L.mmx_set_box_kernel.restype = I
    L.mmx_set_box_kernel.argtypes = [P, I]
    L.mmx_kernel_binary_version.restype = I
    L.mmx_kernel_binary_version.argtypes = []
    L.mmx_flux_gradient.restype = I
    L.mmx_flux_gradient.argtypes = [P, I, I, I, dp, dp, dp]
    L.mmx_set_storage_scale.restype = I
    L.mmx_set_storage_scale.argtypes = [P, D, D]
    L.mmx_add_probe.restype = I
    L.mmx_add_probe.argtypes = [P, I, I, I, I]
    L.mmx_get_probes.restype = LL
    L.mmx_get_probes.argtypes = [P, dp, LL, I]
    L.mmx_energy.restype = I
    L.mmx_energy.argtypes = [P, dp]
    L.mmx_add_flux_plane.restype = I
    L.mmx_add_flux_plane.argtypes = [P, I]
    L.mmx_get_flux.restype = I
    L.mmx_get_flux.argtypes = [P, I, dp, I]
    L.mmx_batch_create.restype = I
    L.mmx_batch_create.argtypes = [ctypes.POINTER(P), I, P, ctypes.POINTER(P)]
    L.mmx_batch_set_planes.restype = I
    L.mmx_batch_set_planes.argtypes = [P, I]
    L.mmx_batch_set_box_blocks.restype = I
    L.mmx_batch_set_box_blocks.argtypes = [P, I]
    L.mmx_batch_step.restype = I
    L.mmx_batch_step.argtypes = [P, I]
    L.mmx_batch_sync.restype = I
    L.mmx_batch_sync.argtypes = [P]
    L.mmx_batch_last_error.restype = ctypes.c_char_p
    L.mmx_batch_last_error.argtypes = [P]
    L.mmx_batch_destroy.restype = I
    L.mmx_batch_destroy.argtypes = [P]
    L.mmx_get_profile.restype = I
    L.mmx_get_profile.argtypes = [P, ctypes.POINTER(KernelProfile), I, I]
    L.mmx_material_average_noalloc.restype = I
    L.mmx_material_average_noalloc.argtypes = [ctypes.POINTER(GridDesc), I, P, P, LL, P]
    L.mmx_last_error.restype = ctypes.c_char_p
    L.mmx_last_error.argtypes = [P]
    L.mmx_destroy.restype = None
    L.mmx_destroy.argtypes = [P]
    _lib = L
    return L


class MMXError(RuntimeError):
    def __init__(self, code, where, msg=""):
        super().__init__(f"{where}: {ERRORS.get(code, code)} {msg}".strip())
        self.code = code


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a):
    if a is None:
        return None
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel())


def field_extent(fid, n):
    nx, ny, nz = n
    if fid in (0, 15):
        return (nx, ny + 1, nz + 1)
    if fid in (1, 16):
        return (nx + 1, ny, nz + 1)
    if fid == 2:
        return (nx + 1, ny + 1, nz)
    fam = {17: 0, 18: 1}.get(fid, (fid - 3) if fid < 6 else (fid - 6) // 3)
    e = [nx, ny, nz]
    e[fam] += 1
    return tuple(e)


class Solver:
    """One ``mmx_ctx``: a grid, its materials, fields and sources on the GPU."""

    def __init__(self, n, d, dt, bc, pml_cells=0, order=2, tol=1e-10, max_iter=64, prec=FP64,
                 stream=None):
        self._L = lib()
        desc = GridDesc()
        for a in range(3):
            desc.n[a] = int(n[a])
            desc.d[a] = float(d[a])
            desc.bc[a] = int(bc[a])
        desc.dt = float(dt)
        desc.pml_cells = int(pml_cells)
        desc.order = int(order)
        desc.tol = float(tol)
        desc.max_iter = int(max_iter)
        desc.prec = int(prec)
        self.n = tuple(int(v) for v in n)
        self.prec = int(prec)
        h = ctypes.c_void_p()
        rc = self._L.mmx_create(ctypes.byref(desc), ctypes.c_void_p(stream or 0), ctypes.byref(h))
        self._h = h
        if rc:
            msg = self._L.mmx_last_error(h).decode() if h.value else ""
            self.close()
            raise MMXError(rc, "mmx_create", msg)

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.mmx_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, where):
        if rc < 0:
            raise MMXError(rc, where, self._L.mmx_last_error(self._h).decode())
        return rc

    # -- entry points
    def set_materials(self, eps_r=None, sigma=None, mu_r=None, Ms=None, alpha=None, gamma=None):
        arrs = [_c64(a) for a in (eps_r, sigma, mu_r, Ms, alpha, gamma)]
        self._check(self._L.mmx_set_materials(self._h, *[_dp(a) for a in arrs]), "mmx_set_materials")

    def set_bias(self, hx, hy, hz):
        self._check(self._L.mmx_set_bias(self._h, float(hx), float(hy), float(hz)), "mmx_set_bias")

    def set_M_cells(self, mx, my, mz):
        arrs = [_c64(a) for a in (mx, my, mz)]
        self._check(self._L.mmx_set_M_cells(self._h, *[_dp(a) for a in arrs]), "mmx_set_M_cells")

    def field_size(self, fid):
        e = field_extent(fid, self.n)
        return e[0] * e[1] * e[2]

    def set_field(self, fid, values):
        a = _c64(values)
        self._check(self._L.mmx_set_field(self._h, int(fid), _dp(a), a.size), "mmx_set_field")

    def get_field(self, fid, check=True, out=None):
        """Field `fid` as float64 values in the order of its extent (x fastest);
        `out`, if given, is a C-contiguous float64 array of that size (pinned
        host memory makes the device->host copy direct)."""
        if out is None:
            out = np.empty(self.field_size(fid), dtype=np.float64)
        elif out.dtype != np.float64 or not out.flags.c_contiguous or out.size != self.field_size(fid):
            raise ValueError("out must be a C-contiguous float64 array of %d values" % self.field_size(fid))
        rc = self._L.mmx_get_field(self._h, int(fid), _dp(out), out.size)
        if check:
            self._check(rc, "mmx_get_field")
        return out

    def get_material(self, which):
        fid = (which % 3) if which < 6 else 3 + which % 3
        out = np.empty(self.field_size(fid), dtype=np.float64)
        self._check(self._L.mmx_get_material(self._h, int(which), _dp(out), out.size), "mmx_get_material")
        return out

    def add_source(self, kind, comp, i=0, j=0, k=0, amp=0.0, f0=0.0, tp=1.0, t0=0.0):
        s = SourceDesc(int(kind), int(comp), int(i), int(j), int(k), float(amp), float(f0),
                       float(tp), float(t0))
        self._check(self._L.mmx_add_source(self._h, ctypes.byref(s)), "mmx_add_source")

    def set_path(self, path):
        self._check(self._L.mmx_set_path(self._h, int(path)), "mmx_set_path")

    def step(self, nsteps=1):
        self._check(self._L.mmx_step(self._h, int(nsteps)), "mmx_step")

    def sync(self, check=True):
        rc = self._L.mmx_sync(self._h)
        if check:
            self._check(rc, "mmx_sync")
        return rc

    def check_bounded_wait(self):
        """Run the device-wait check (mmx_check_bounded_wait); returns its code,
        -6 (TIMEOUT) when both bounded waits gave up as designed."""
        return self._L.mmx_check_bounded_wait(self._h)

    def set_step_count(self, steps):
        """Set the steps done (the time the next step starts from), to resume
        from a checkpoint taken with get_field (mmx_set_step_count)."""
        self._check(self._L.mmx_set_step_count(self._h, int(steps)), "mmx_set_step_count")

    def check_guards(self):
        """Read back the guard bytes after every device array of the context
        (mmx_check_guards); raises MMXError if a kernel wrote past an
        array's end."""
        self._check(self._L.mmx_check_guards(self._h), "mmx_check_guards")

    def inject_timeout(self):
        """Test hook: the next step call starts as if a bounded wait had given
        up (mmx_inject_timeout)."""
        self._check(self._L.mmx_inject_timeout(self._h), "mmx_inject_timeout")

    def get_info(self):
        """Which kernels the fused path runs (mmx_get_info) as a dict; adds
        ``fused_kernel_name``."""
        i = Info()
        self._check(self._L.mmx_get_info(self._h, ctypes.byref(i)), "mmx_get_info")
        d = {k: getattr(i, k) for k, _ in Info._fields_}
        d["fused_kernel_name"] = FUSED_KERNELS.get(d["fused_kernel"], "?")
        d["box_kernel_name"] = BOX_KERNELS.get(d["box_kernel"], "?")
        return d

    def set_fused_staging(self, bulk):
        """1: bulk tensor copies where they apply (default); 0: per-lane cp.async."""
        self._check(self._L.mmx_set_fused_staging(self._h, 1 if bulk else 0), "mmx_set_fused_staging")

    def set_box_kernel(self, resident):
        """1: records in shared memory where they fit (default); 0: list-driven."""
        self._check(self._L.mmx_set_box_kernel(self._h, 1 if resident else 0), "mmx_set_box_kernel")

    def get_stats(self):
        s = Stats()
        self._check(self._L.mmx_get_stats(self._h, ctypes.byref(s)), "mmx_get_stats")
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def get_iter_log(self, cap=1 << 16):
        buf = np.zeros(cap, dtype=np.int32)
        n = self._L.mmx_get_iter_log(self._h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), cap)
        self._check(n, "mmx_get_iter_log")
        return buf[:n].copy()

    def get_field_device(self, fid):
        p = ctypes.c_void_p()
        sx = ctypes.c_longlong()
        sy = ctypes.c_longlong()
        self._check(self._L.mmx_get_field_device(self._h, int(fid), ctypes.byref(p), ctypes.byref(sx),
                                                 ctypes.byref(sy)), "mmx_get_field_device")
        return p.value, sx.value, sy.value

    def flux_gradient(self, kp, nsteps, checkpoint_every=None, with_h0=False):
        """Run nsteps steps and return (loss, d loss / d eps_r per cell) for the
        time-integrated Poynting flux through z node plane kp (discrete
        adjoint, checkpointing every ~sqrt(nsteps) steps by default); with
        with_h0, (loss, d loss / d eps_r, d loss / d H0)."""
        every = int(checkpoint_every or max(1, round(nsteps ** 0.5)))
        loss = ctypes.c_double()
        grad = np.zeros(self.n[0] * self.n[1] * self.n[2], dtype=np.float64)
        gh0 = np.zeros(3, dtype=np.float64)
        self._check(self._L.mmx_flux_gradient(self._h, int(kp), int(nsteps), every, ctypes.byref(loss), _dp(grad),
                                              _dp(gh0)), "mmx_flux_gradient")
        grad = grad.reshape(self.n[2], self.n[1], self.n[0])
        return (loss.value, grad, gh0) if with_h0 else (loss.value, grad)

    def set_storage_scale(self, sE, sH):
        """FP16 contexts: store E as E/sE and H as H/sH (before any field or step)."""
        self._check(self._L.mmx_set_storage_scale(self._h, float(sE), float(sH)), "mmx_set_storage_scale")

    def add_probe(self, fid, i, j, k):
        """Record E component `fid` (0-2) at (i, j, k) after every step; returns
        the probe index.  Samples recorded so far are discarded."""
        idx = self._check(self._L.mmx_add_probe(self._h, int(fid), int(i), int(j), int(k)), "mmx_add_probe")
        self._nprobe = idx + 1
        return idx

    def get_probes(self, max_rows=1 << 16, reset=True):
        """Samples since the last reset as a float64 array [steps, probes]."""
        nprobe = getattr(self, "_nprobe", 0)
        buf = np.zeros(max(1, int(max_rows) * nprobe), dtype=np.float64)
        rows = self._L.mmx_get_probes(self._h, _dp(buf), int(max_rows), 1 if reset else 0)
        self._check(int(rows), "mmx_get_probes")
        return buf[: rows * nprobe].reshape(rows, nprobe)

    def energy(self):
        """Discrete electromagnetic energy (J) at the current time level."""
        out = ctypes.c_double()
        self._check(self._L.mmx_energy(self._h, ctypes.byref(out)), "mmx_energy")
        return out.value

    def add_flux_plane(self, k):
        """Accumulate the Poynting flux through z node plane k; returns its index."""
        return self._check(self._L.mmx_add_flux_plane(self._h, int(k)), "mmx_add_flux_plane")

    def get_flux(self, index, reset=False):
        """(time-integrated flux in J, power of the last step in W)."""
        out = (ctypes.c_double * 2)()
        self._check(self._L.mmx_get_flux(self._h, int(index), out, 1 if reset else 0), "mmx_get_flux")
        return out[0], out[1]

    def set_profiling(self, enable=True):
        self._check(self._L.mmx_set_profiling(self._h, 1 if enable else 0), "mmx_set_profiling")

    def get_profile(self, reset=True):
        """{kernel name: (launches, total device ms)} since the last reset."""
        buf = (KernelProfile * 16)()
        n = self._check(self._L.mmx_get_profile(self._h, buf, 16, 1 if reset else 0), "mmx_get_profile")
        return {buf[q].name.decode(): (int(buf[q].launches), float(buf[q].total_ms)) for q in range(min(n, 16))}

    def last_error(self):
        return self._L.mmx_last_error(self._h).decode()


def kernel_binary_version() -> int:
    """SM version the kernels were built for on the current device (103)."""
    return int(lib().mmx_kernel_binary_version())


def material_average_noalloc(n, bc, location, cell_ptr, out_ptr, count, stream=None) -> int:
    """Call ``mmx_material_average_noalloc`` on device pointers (ints);
    returns the status code (0 = OK)."""
    desc = GridDesc()
    for a in range(3):
        desc.n[a] = int(n[a])
        desc.bc[a] = int(bc[a])
    return lib().mmx_material_average_noalloc(ctypes.byref(desc), int(location), ctypes.c_void_p(cell_ptr),
                                              ctypes.c_void_p(out_ptr), int(count),
                                              ctypes.c_void_p(stream or 0))


class Batch:
    """Independent solvers advanced together (one fused and one H/M launch per
    step for all of them, each call one CUDA graph).  The solvers stay usable
    on their own between batch calls; keep them alive as long as the batch."""

    def __init__(self, solvers, stream=None):
        self._L = lib()
        self.solvers = list(solvers)
        arr = (ctypes.c_void_p * len(self.solvers))(*[s._h.value for s in self.solvers])
        self._h = ctypes.c_void_p()
        rc = self._L.mmx_batch_create(arr, len(self.solvers), stream, ctypes.byref(self._h))
        if rc < 0:
            msg = self._L.mmx_batch_last_error(self._h).decode() if self._h.value else ""
            self.close()
            raise MMXError(rc, "mmx_batch_create", msg)

    def _check(self, rc, where):
        if rc < 0:
            raise MMXError(rc, where, self._L.mmx_batch_last_error(self._h).decode())
        return rc

    def set_planes(self, planes):
        """z planes each fused CTA marches (0: a whole grid)."""
        self._check(self._L.mmx_batch_set_planes(self._h, int(planes)), "mmx_batch_set_planes")

    def set_box_blocks(self, per_sm):
        """Cap the batched H/M launch at per_sm blocks per SM (0: all resident)."""
        self._check(self._L.mmx_batch_set_box_blocks(self._h, int(per_sm)), "mmx_batch_set_box_blocks")

    def step(self, nsteps):
        self._check(self._L.mmx_batch_step(self._h, int(nsteps)), "mmx_batch_step")

    def sync(self, check=True):
        rc = self._L.mmx_batch_sync(self._h)
        if check:
            self._check(rc, "mmx_batch_sync")
        return rc

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.mmx_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_workload(w, prec=FP64, stream=None, with_sources=True, path=PATH_FUSED) -> Solver:
    """Build a solver from a ``workloads.Workload`` (seeded synthetic inputs)."""
    s = Solver(w.n, w.d, w.dt, w.bc, w.pml_cells, w.order, w.tol, w.max_iter, prec, stream)
    s.set_path(path)
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

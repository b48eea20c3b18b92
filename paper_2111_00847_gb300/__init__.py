"""GB300-native consistent and conservative phase-field lattice Boltzmann.

Python binding of the C-ABI library ``libpflbm.so`` (declared in
``include/pflbm.h``).  This module only marshals arguments: every step of the
method runs in the library's CUDA kernels.  PyTorch, when present, supplies
the CUDA stream and the device memory (through its caching allocator); the
library itself has no CPU path, and importing the binding without the built
library, or creating a simulation without a CUDA device, raises.

The functions ``lbm_create``, ``lbm_init_fields``, ``lbm_step``,
``lbm_fields``, ``lbm_set_fields``, ``lbm_time``, ``lbm_device_bytes``,
``lbm_destroy`` and ``lbm_last_error`` mirror the C entry points one to one;
``Simulation`` wraps them with numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpflbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
LBM_FP64, LBM_FP32, LBM_FP16_DEV, LBM_BF16_DEV = 0, 1, 2, 3
(LBM_PHI, LBM_UX, LBM_UY, LBM_P, LBM_RHO, LBM_F_POP, LBM_G_POP, LBM_HIST, LBM_DIAG, LBM_MU,
 LBM_MCX, LBM_MCY) = range(12)
LBM_NDIAG = 8
LBM_ABI_VERSION = 1
LBM_FLAG_NO_TMA = 1
LBM_LEFT, LBM_RIGHT, LBM_BOTTOM, LBM_TOP = 0, 1, 2, 3
LBM_SLAB_GHOST = 4
DIAG_KEYS = ("t", "sum_phi", "Du_rms", "Sm_rms", "umax", "nonfinite", "n_avg", "reserved")

EXPORTED = ("lbm_create", "lbm_init_fields", "lbm_step", "lbm_fields", "lbm_fields_region",
            "lbm_fields_noalloc", "lbm_set_fields", "lbm_set_solid", "lbm_selftest_wait_timeout",
            "lbm_time", "lbm_device_bytes", "lbm_destroy", "lbm_last_error",
            "lbm_state_bytes", "lbm_snapshot", "lbm_restore", "lbm_adjoint_seed", "lbm_adjoint_step",
            "lbm_adjoint_init", "lbm_adjoint_gravity", "lbm_create_slab", "lbm_slab_info",
            "lbm_slab_halo_bytes", "lbm_slab_pack", "lbm_slab_unpack")


class LbmParams(C.Structure):
    """ctypes image of ``lbm_params``."""

    _fields_ = [
        ("version", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("precision", C.c_int32),
        ("phase_model", C.c_int32), ("flux_model", C.c_int32), ("visc_law", C.c_int32),
        ("gravity_mode", C.c_int32), ("bc", C.c_int32 * 4), ("diag_every", C.c_int32),
        ("flags", C.c_int32),
        ("phiA", C.c_double), ("phiB", C.c_double), ("rhoA", C.c_double), ("rhoB", C.c_double),
        ("muA", C.c_double), ("muB", C.c_double), ("mobility", C.c_double), ("width", C.c_double),
        ("sigma", C.c_double), ("eta", C.c_double), ("gx", C.c_double), ("gy", C.c_double),
        ("rho0", C.c_double), ("theta_deg", C.c_double * 4), ("s_f", C.c_double * 9),
        ("s_g", C.c_double * 9), ("n_delta", C.c_double),
    ]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class LbmAllocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


_lib = None


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_2111_00847_gb300.build` (there is no CPU fallback)")
    L = C.CDLL(path)
    dp = C.POINTER(C.c_double)
    L.lbm_create.argtypes = [C.POINTER(LbmParams), C.c_void_p, C.POINTER(LbmAllocator),
                             C.POINTER(C.c_void_p)]
    L.lbm_create.restype = C.c_int
    L.lbm_init_fields.argtypes = [C.c_void_p, dp, dp, dp, dp]
    L.lbm_step.argtypes = [C.c_void_p, C.c_int64]
    L.lbm_fields.argtypes = [C.c_void_p, C.c_int32, dp]
    L.lbm_fields_region.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                    C.c_int32, dp]
    L.lbm_set_fields.argtypes = [C.c_void_p, C.c_int32, dp]
    L.lbm_fields_noalloc.argtypes = [C.c_void_p, C.c_int32, dp]
    L.lbm_set_solid.argtypes = [C.c_void_p, C.POINTER(C.c_uint8)]
    L.lbm_selftest_wait_timeout.argtypes = [C.c_void_p]
    L.lbm_time.argtypes = [C.c_void_p]
    L.lbm_time.restype = C.c_int64
    L.lbm_device_bytes.argtypes = [C.c_void_p]
    L.lbm_device_bytes.restype = C.c_int64
    L.lbm_destroy.argtypes = [C.c_void_p]
    L.lbm_destroy.restype = None
    L.lbm_last_error.argtypes = [C.c_void_p]
    L.lbm_last_error.restype = C.c_char_p
    L.lbm_state_bytes.argtypes = [C.c_void_p]
    L.lbm_state_bytes.restype = C.c_int64
    L.lbm_snapshot.argtypes = [C.c_void_p, C.c_void_p]
    L.lbm_restore.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
    L.lbm_adjoint_seed.argtypes = [C.c_void_p, dp]
    L.lbm_adjoint_step.argtypes = [C.c_void_p, C.c_void_p]
    L.lbm_adjoint_init.argtypes = [C.c_void_p, C.c_void_p, dp]
    L.lbm_adjoint_gravity.argtypes = [C.c_void_p, dp]
    L.lbm_create_slab.argtypes = [C.POINTER(LbmParams), C.c_int32, C.c_int32, C.c_void_p,
                                  C.POINTER(LbmAllocator), C.POINTER(C.c_void_p)]
    L.lbm_create_slab.restype = C.c_int
    L.lbm_slab_info.argtypes = [C.c_void_p, C.POINTER(C.c_int32)]
    L.lbm_slab_halo_bytes.argtypes = [C.c_void_p]
    L.lbm_slab_halo_bytes.restype = C.c_int64
    L.lbm_slab_pack.argtypes = [C.c_void_p, C.c_int32, C.c_void_p]
    L.lbm_slab_unpack.argtypes = [C.c_void_p, C.c_int32, C.c_void_p]
    _lib = L
    return L


def params_struct(prm) -> LbmParams:
    """Fill ``lbm_params`` from any object with the parameter attributes
    (e.g. ``workloads.Params``)."""
    s = LbmParams()
    s.version = LBM_ABI_VERSION
    for name in ("nx", "ny", "precision", "phase_model", "flux_model", "visc_law",
                 "gravity_mode", "diag_every"):
        setattr(s, name, int(getattr(prm, name)))
    s.flags = int(getattr(prm, "flags", 0))
    for i in range(4):
        s.bc[i] = int(prm.bc[i])
        s.theta_deg[i] = float(prm.theta_deg[i])
    for name in ("phiA", "phiB", "rhoA", "rhoB", "muA", "muB", "mobility", "width", "sigma",
                 "eta", "gx", "gy", "rho0"):
        setattr(s, name, float(getattr(prm, name)))
    for k in range(9):
        s.s_f[k] = float(prm.s_f[k])
        s.s_g[k] = float(prm.s_g[k])
    s.n_delta = float(getattr(prm, "n_delta", 0.0))
    return s


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pflbm error {code}: {msg}")
        self.code = code


def _dptr(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


# ---- one-to-one wrappers of the C entry points ------------------------------
def lbm_last_error(handle=None) -> str:
    return (load().lbm_last_error(handle) or b"").decode()


def _check(rc: int, handle=None):
    if rc != LBM_OK:
        raise LbmError(rc, lbm_last_error(handle))


def lbm_create(params: LbmParams, stream: int = 0, allocator: LbmAllocator | None = None):
    h = C.c_void_p()
    rc = load().lbm_create(C.byref(params), C.c_void_p(stream or None),
                           C.byref(allocator) if allocator is not None else None, C.byref(h))
    _check(rc)
    return h


def lbm_init_fields(h, phi, ux=None, uy=None, p=None):
    _check(load().lbm_init_fields(h, _dptr(phi), _dptr(ux), _dptr(uy), _dptr(p)), h)


def lbm_step(h, nsteps: int):
    _check(load().lbm_step(h, int(nsteps)), h)


def lbm_fields(h, which: int, out: np.ndarray):
    _check(load().lbm_fields(h, int(which), _dptr(out)), h)


def lbm_fields_region(h, which: int, x0: int, y0: int, w: int, hgt: int, out: np.ndarray):
    _check(load().lbm_fields_region(h, int(which), int(x0), int(y0), int(w), int(hgt),
                                    _dptr(out)), h)


def lbm_fields_noalloc(h, which: int, out: np.ndarray):
    """lbm_fields for LBM_F_POP / LBM_G_POP / LBM_HIST through the library's
    fixed staging array (no device allocation); grids up to 2^20 nodes."""
    _check(load().lbm_fields_noalloc(h, int(which), _dptr(out)), h)


def lbm_set_fields(h, which: int, arr: np.ndarray):
    _check(load().lbm_set_fields(h, int(which), _dptr(arr)), h)


def lbm_set_solid(h, solid: np.ndarray | None):
    """Solid obstacle nodes: [ny][nx] uint8 (nonzero = solid), or None."""
    ptr = None if solid is None else solid.ctypes.data_as(C.POINTER(C.c_uint8))
    _check(load().lbm_set_solid(h, ptr), h)


def lbm_selftest_wait_timeout(h):
    """Make one bounded device wait give up (the failure path of the step
    kernels); the next synchronising call reports LBM_ECUDA."""
    _check(load().lbm_selftest_wait_timeout(h), h)


def lbm_time(h) -> int:
    return int(load().lbm_time(h))


def lbm_device_bytes(h) -> int:
    return int(load().lbm_device_bytes(h))


def lbm_destroy(h):
    load().lbm_destroy(h)


def lbm_state_bytes(h) -> int:
    return int(load().lbm_state_bytes(h))


def lbm_snapshot(h, dst_ptr: int):
    """Copy the state into device memory at dst_ptr (lbm_state_bytes bytes)."""
    _check(load().lbm_snapshot(h, C.c_void_p(int(dst_ptr))), h)


def lbm_restore(h, src_ptr: int, t: int):
    _check(load().lbm_restore(h, C.c_void_p(int(src_ptr)), int(t)), h)


def lbm_adjoint_seed(h, dj_dphi: np.ndarray):
    _check(load().lbm_adjoint_seed(h, _dptr(dj_dphi)), h)


def lbm_adjoint_step(h, state_ptr: int):
    _check(load().lbm_adjoint_step(h, C.c_void_p(int(state_ptr))), h)


def lbm_adjoint_init(h, state0_ptr: int, out: np.ndarray):
    _check(load().lbm_adjoint_init(h, C.c_void_p(int(state0_ptr)), _dptr(out)), h)


def lbm_adjoint_gravity(h, out: np.ndarray):
    _check(load().lbm_adjoint_gravity(h, _dptr(out)), h)


def lbm_create_slab(params: LbmParams, y_lo: int, ny_own: int, stream: int = 0,
                    allocator: LbmAllocator | None = None):
    h = C.c_void_p()
    rc = load().lbm_create_slab(C.byref(params), int(y_lo), int(ny_own), C.c_void_p(stream or None),
                                C.byref(allocator) if allocator is not None else None, C.byref(h))
    _check(rc)
    return h


def lbm_slab_info(h):
    info = (C.c_int32 * 4)()
    _check(load().lbm_slab_info(h, info), h)
    return tuple(int(v) for v in info)


def lbm_slab_halo_bytes(h) -> int:
    n = int(load().lbm_slab_halo_bytes(h))
    if n < 0:
        _check(n, h)
    return n


def lbm_slab_pack(h, side: int, dst_ptr: int):
    _check(load().lbm_slab_pack(h, int(side), C.c_void_p(int(dst_ptr))), h)


def lbm_slab_unpack(h, side: int, src_ptr: int):
    _check(load().lbm_slab_unpack(h, int(side), C.c_void_p(int(src_ptr))), h)


# ---- PyTorch plumbing --------------------------------------------------------
def _torch():
    try:
        import torch
    except ImportError:  # the library works without torch (own cudaMalloc)
        return None
    return torch if torch.cuda.is_available() else None


def torch_allocator():
    """An ``lbm_allocator`` drawing device memory from PyTorch's caching
    allocator (returns (struct, keep-alive tuple))."""
    torch = _torch()
    if torch is None:
        return None, ()

    def _alloc(nbytes, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0)))
        except RuntimeError:
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    return LbmAllocator(a, f, None), (a, f)


class Simulation:
    """One simulation on the current CUDA device.

    params: any object with the fields of ``lbm_params`` (``workloads.Params``).
    stream: a ``torch.cuda.Stream`` or raw ``cudaStream_t`` integer; default is
    PyTorch's current stream when PyTorch is available.
    """

    def __init__(self, params, stream=None, use_torch_allocator: bool = True, slab=None):
        """slab = (y_lo, ny_own): a y-slab of the grid `params` describes
        (lbm_create_slab); the handle then holds the slab's local rows."""
        self.params = params
        self.nx, self.ny = int(params.nx), int(params.ny)
        torch = _torch()
        if stream is None and torch is not None:
            stream = torch.cuda.current_stream()
        self.stream_obj = stream
        self.stream = int(getattr(stream, "cuda_stream", stream) or 0)
        self._alloc, self._keep = (torch_allocator() if use_torch_allocator else (None, ()))
        self._p = params_struct(params)
        if slab is None:
            self._h = lbm_create(self._p, self.stream, self._alloc)
            self.slab = None
        else:
            self._h = lbm_create_slab(self._p, slab[0], slab[1], self.stream, self._alloc)
            self.slab = lbm_slab_info(self._h)  # (y_lo, ny_own, ghost_lo, ghost_hi)
            self.ny = self.slab[1] + self.slab[2] + self.slab[3]

    def close(self):
        if getattr(self, "_h", None):
            lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def _field(self, a):
        if a is None:
            return None
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        if a.shape != (self.ny, self.nx):
            raise ValueError(f"field shape {a.shape} != {(self.ny, self.nx)}")
        return a

    def set_solid(self, solid):
        """Solid obstacle nodes ([ny][nx], nonzero = solid; None removes them).
        Call before init_fields."""
        if solid is None:
            lbm_set_solid(self._h, None)
            return
        m = np.ascontiguousarray(np.asarray(solid) != 0, dtype=np.uint8)
        if m.shape != (self.ny, self.nx):
            raise ValueError(f"mask shape {m.shape} != {(self.ny, self.nx)}")
        lbm_set_solid(self._h, m)

    def init_fields(self, phi, ux=None, uy=None, p=None):
        arrs = [self._field(x) for x in (phi, ux, uy, p)]
        lbm_init_fields(self._h, *arrs)

    def step(self, n: int = 1):
        lbm_step(self._h, n)

    @property
    def t(self) -> int:
        return lbm_time(self._h)

    @property
    def device_bytes(self) -> int:
        return lbm_device_bytes(self._h)

    def fields(self, which: int, region=None, out: np.ndarray | None = None) -> np.ndarray:
        """Field `which` at the current time; region = (x0, y0, w, h) limits it
        to a node rectangle; `out` may supply the destination (float64,
        C-contiguous, e.g. a view of pinned host memory)."""
        x0, y0, w, hgt = region if region is not None else (0, 0, self.nx, self.ny)
        if which in (LBM_F_POP, LBM_G_POP):
            shape = (9, hgt, w)
        elif which == LBM_HIST:
            shape = (5, hgt, w)
        elif which == LBM_DIAG:
            shape = (LBM_NDIAG,)
        else:
            shape = (hgt, w)
        if out is None:
            out = np.empty(shape)
        elif out.shape != shape or out.dtype != np.float64 or not out.flags.c_contiguous:
            raise ValueError(f"out must be a C-contiguous float64 array of shape {shape}")
        lbm_fields_region(self._h, which, x0, y0, w, hgt, out)
        return out

    def set_fields(self, which: int, arr):
        a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64))
        lbm_set_fields(self._h, which, a)

    def diag(self) -> dict:
        return dict(zip(DIAG_KEYS, self.fields(LBM_DIAG).tolist()))

    # -- snapshots and the adjoint (device buffers are torch uint8 tensors)
    @property
    def state_bytes(self) -> int:
        return lbm_state_bytes(self._h)

    def new_state_buffer(self):
        import torch

        return torch.empty(self.state_bytes, dtype=torch.uint8, device="cuda")

    def snapshot(self, buf):
        lbm_snapshot(self._h, buf.data_ptr())
        return buf

    def restore(self, buf, t: int):
        lbm_restore(self._h, buf.data_ptr(), t)

    def adjoint_seed(self, dj_dphi):
        lbm_adjoint_seed(self._h, self._field(dj_dphi))

    def adjoint_step(self, state_buf):
        lbm_adjoint_step(self._h, state_buf.data_ptr())

    def adjoint_init(self, state0_buf) -> np.ndarray:
        out = np.empty((self.ny, self.nx))
        lbm_adjoint_init(self._h, state0_buf.data_ptr(), out)
        return out

    def adjoint_gravity(self) -> np.ndarray:
        out = np.empty(2)
        lbm_adjoint_gravity(self._h, out)
        return out

    # -- y-slabs (halo messages in device buffers, e.g. torch uint8 tensors)
    @property
    def halo_bytes(self) -> int:
        return lbm_slab_halo_bytes(self._h)

    def pack(self, side: int, buf):
        lbm_slab_pack(self._h, side, buf.data_ptr())

    def unpack(self, side: int, buf):
        lbm_slab_unpack(self._h, side, buf.data_ptr())


__all__ = ["Simulation", "LbmParams", "LbmError", "load", "params_struct", "torch_allocator",
           *EXPORTED]

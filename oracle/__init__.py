"""Python access to the FP64 CPU oracle (``pflbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline / reference leg load this module; the product path
never does.  It shares no code with the CUDA library: it has its own ctypes
parameter structure and loads its own shared object, compiled from the single
C file beside it with the host C compiler.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pflbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_pflbm.so")
_lock = threading.Lock()
_lib = None

PHI, UX, UY, P, RHO, F_POP, G_POP, HIST, DIAG, MU, MCX, MCY = range(12)
NDIAG = 8
DIAG_KEYS = ("t", "sum_phi", "Du_rms", "Sm_rms", "umax", "nonfinite", "n_avg", "reserved")


class OracleParams(C.Structure):
    _fields_ = [
        ("version", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("precision", C.c_int32),
        ("phase_model", C.c_int32), ("flux_model", C.c_int32), ("visc_law", C.c_int32),
        ("gravity_mode", C.c_int32), ("bc", C.c_int32 * 4), ("diag_every", C.c_int32),
        ("reserved", C.c_int32),
        ("phiA", C.c_double), ("phiB", C.c_double), ("rhoA", C.c_double), ("rhoB", C.c_double),
        ("muA", C.c_double), ("muB", C.c_double), ("mobility", C.c_double), ("width", C.c_double),
        ("sigma", C.c_double), ("eta", C.c_double), ("gx", C.c_double), ("gy", C.c_double),
        ("rho0", C.c_double), ("theta_deg", C.c_double * 4), ("s_f", C.c_double * 9),
        ("s_g", C.c_double * 9), ("n_delta", C.c_double),
    ]


def to_struct(prm) -> OracleParams:
    s = OracleParams()
    s.version = 1
    for name in ("nx", "ny", "precision", "phase_model", "flux_model", "visc_law",
                 "gravity_mode", "diag_every"):
        setattr(s, name, int(getattr(prm, name)))
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


def build(force: bool = False) -> str:
    """Compile the oracle into a shared object beside its source."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def build_variant(edits, outdir: str, tag: str = "variant"):
    """Compile a copy of the oracle with textual edits and load it.

    For the tests of the pins themselves: each edit (old, new) plants one
    mistake (a flipped sign, a wrong coefficient), and a pin must fail on the
    planted copy.  Every `old` must occur exactly once in the source.  The
    copy is built in `outdir`; the oracle's own library is not touched."""
    with open(_SRC) as fh:
        src = fh.read()
    for old, new in edits:
        n = src.count(old)
        if n != 1:
            raise ValueError(f"edit target found {n} times: {old!r}")
        src = src.replace(old, new)
    os.makedirs(outdir, exist_ok=True)
    csrc = os.path.join(outdir, f"pflbm_oracle_{tag}.c")
    so = os.path.join(outdir, f"liboracle_pflbm_{tag}.so")
    with open(csrc, "w") as fh:
        fh.write(src)
    cmd = ["gcc", "-std=c99", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp",
           csrc, "-o", so, "-lm"]
    subprocess.run(cmd, check=True)
    return _load(so)


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _load(_LIB)
    return _lib


def _load(path: str):
    """Load an oracle shared object and declare its entry points."""
    L = C.CDLL(path)
    dp = C.POINTER(C.c_double)
    L.oracle_create.argtypes = [C.POINTER(OracleParams), C.POINTER(C.c_void_p)]
    L.oracle_init_fields.argtypes = [C.c_void_p, dp, dp, dp, dp]
    L.oracle_step.argtypes = [C.c_void_p, C.c_int64]
    L.oracle_fields.argtypes = [C.c_void_p, C.c_int32, dp]
    L.oracle_set_fields.argtypes = [C.c_void_p, C.c_int32, dp]
    L.oracle_set_solid.argtypes = [C.c_void_p, C.POINTER(C.c_uint8)]
    L.oracle_padded.argtypes = [C.c_void_p, C.c_int32, dp]
    L.oracle_destroy.argtypes = [C.c_void_p]
    L.oracle_destroy.restype = None
    L.oracle_last_error.argtypes = [C.c_void_p]
    L.oracle_last_error.restype = C.c_char_p
    L.oracle_time.argtypes = [C.c_void_p]
    L.oracle_time.restype = C.c_long
    L.oracle_set_threads.argtypes = [C.c_int]
    L.oracle_set_threads.restype = None
    L.oracle_get_threads.restype = C.c_int
    L.oracle_moment_matrix.argtypes = [dp, dp]
    L.oracle_moment_matrix.restype = None
    L.oracle_lattice.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_int), dp]
    L.oracle_lattice.restype = None
    L.oracle_node_moments.argtypes = [C.POINTER(OracleParams), dp, dp]
    L.oracle_grad_lap.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp]
    L.oracle_wall_phi.argtypes = [C.POINTER(OracleParams), C.c_double, C.c_double,
                                  C.c_double, dp]
    L.oracle_wall_phi.restype = C.c_double
    return L


def _dptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


class OracleError(RuntimeError):
    def __init__(self, rc, msg):
        super().__init__(f"oracle error {rc}: {msg}")
        self.rc = rc


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(lib().oracle_get_threads())


class Oracle:
    """One FP64 CPU simulation (naive whole-grid passes)."""

    def __init__(self, params, lib_=None):
        self.params = params
        self._L = lib_ if lib_ is not None else lib()
        self._p = to_struct(params)
        h = C.c_void_p()
        rc = self._L.oracle_create(C.byref(self._p), C.byref(h))
        if rc != 0:
            raise OracleError(rc, "oracle_create failed (see stderr)")
        self._h = h
        self.nx, self.ny = params.nx, params.ny

    def close(self):
        if getattr(self, "_h", None):
            self._L.oracle_destroy(self._h)
            self._h = None

    __del__ = close

    def _check(self, rc):
        if rc != 0:
            raise OracleError(rc, self._L.oracle_last_error(self._h).decode())

    def _arr(self, a):
        if a is None:
            return None
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        assert a.shape == (self.ny, self.nx), a.shape
        return a

    def set_solid(self, mask):
        """Solid nodes: mask [ny][nx], nonzero = solid (None removes them)."""
        if mask is None:
            self._solid = None
            self._check(self._L.oracle_set_solid(self._h, None))
            return
        m = np.ascontiguousarray(np.asarray(mask) != 0, dtype=np.uint8)
        assert m.shape == (self.ny, self.nx), m.shape
        self._solid = m
        self._check(self._L.oracle_set_solid(self._h, m.ctypes.data_as(C.POINTER(C.c_uint8))))

    def init_fields(self, phi, ux=None, uy=None, p=None):
        arrs = [self._arr(x) for x in (phi, ux, uy, p)]
        self._keep = arrs
        self._check(self._L.oracle_init_fields(self._h, *[_dptr(a) for a in arrs]))

    def step(self, n: int = 1):
        self._check(self._L.oracle_step(self._h, int(n)))

    @property
    def t(self) -> int:
        return int(self._L.oracle_time(self._h))

    def fields(self, which: int) -> np.ndarray:
        N = self.nx * self.ny
        if which in (F_POP, G_POP):
            out = np.empty((9, self.ny, self.nx))
        elif which == HIST:
            out = np.empty((5, self.ny, self.nx))
        elif which == DIAG:
            out = np.empty(NDIAG)
        else:
            out = np.empty((self.ny, self.nx))
        del N
        self._check(self._L.oracle_fields(self._h, int(which), _dptr(out)))
        return out

    def padded(self, which: int = 0) -> np.ndarray:
        """[ny+2][nx+2] phi (which 0) or mu_phi (1) as the last macro pass's
        stencils saw them (ghost layer included)."""
        out = np.empty((self.ny + 2, self.nx + 2))
        self._check(self._L.oracle_padded(self._h, int(which), _dptr(out)))
        return out

    def set_fields(self, which: int, arr: np.ndarray):
        a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64))
        self._check(self._L.oracle_set_fields(self._h, int(which), _dptr(a)))

    def diag(self) -> dict:
        d = self.fields(DIAG)
        return dict(zip(DIAG_KEYS, d.tolist()))


def run_case(case, steps: int | None = None) -> Oracle:
    o = Oracle(case.params)
    if getattr(case, "solid", None) is not None:
        o.set_solid(case.solid)
    o.init_fields(case.phi, case.ux, case.uy, case.p)
    o.step(case.steps if steps is None else steps)
    return o


# ---- node-level hooks -------------------------------------------------------
def moment_matrix():
    M = np.empty((9, 9))
    Mi = np.empty((9, 9))
    lib().oracle_moment_matrix(_dptr(M), _dptr(Mi))
    return M, Mi


def lattice():
    cx = (C.c_int * 9)()
    cy = (C.c_int * 9)()
    w = np.empty(9)
    lib().oracle_lattice(cx, cy, _dptr(w))
    return np.array(list(cx)), np.array(list(cy)), w


NODE_KEYS = ("phi", "mu", "u", "v", "p", "rho", "mcx", "mcy", "Fx", "Fy", "drx", "dry",
             "lam", "nx", "ny", "dphiu", "dphiv", "dum", "dA", "dB")


def node_moments(params, lib_=None, **vals):
    """Moment vectors (m_f^eq, m_R, m_g^eq, m_F) the oracle uses at one node."""
    inp = np.array([float(vals.get(k, 0.0)) for k in NODE_KEYS])
    out = np.empty(36)
    s = to_struct(params)
    rc = (lib_ or lib()).oracle_node_moments(C.byref(s), _dptr(inp), _dptr(out))
    if rc != 0:
        raise OracleError(rc, "node_moments")
    return out[0:9], out[9:18], out[18:27], out[27:36]


def grad_lap(field: np.ndarray, lib_=None):
    f = np.ascontiguousarray(field, dtype=np.float64)
    ny, nx = f.shape
    gx, gy, lp = np.empty_like(f), np.empty_like(f), np.empty_like(f)
    rc = (lib_ or lib()).oracle_grad_lap(nx, ny, _dptr(f), _dptr(gx), _dptr(gy), _dptr(lp))
    if rc != 0:
        raise OracleError(rc, "grad_lap")
    return gx, gy, lp


def wall_phi(params, phi1: float, phi2: float, theta_deg: float, lib_=None):
    """(phi_w, ghost) of the wetting boundary for the given first/second fluid values."""
    s = to_struct(params)
    ghost = np.zeros(1)
    pw = (lib_ or lib()).oracle_wall_phi(C.byref(s), float(phi1), float(phi2), float(theta_deg), _dptr(ghost))
    return float(pw), float(ghost[0])


__all__ = ["Oracle", "OracleParams", "build", "lib", "run_case", "moment_matrix", "lattice",
           "node_moments", "grad_lap", "wall_phi", "set_threads", "get_threads", "math"]

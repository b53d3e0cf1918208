"""FP64 CPU oracle of the solid LBM (arXiv 2208.04088), ctypes wrapper.

TEST INFRASTRUCTURE ONLY.  Imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the library in
``paper_2208_04088_gb300/``.  The arithmetic lives in ``lbm_oracle.c``; this
module only compiles it (gcc, ``-ffp-contract=off`` so the geometry tables are
bit-reproducible on x86 and Arm) and marshals numpy arrays.

What each exported function computes, with the paper's equation:
  * ``feq``        -- Eq. (fieq), the moment-chain equilibrium.
  * ``collide``    -- Eq. (coll) with the source of Eq. (sourceterm).
  * ``geometry``   -- node mask and cut links (wall distance q = s/l and the
                      outward normal) for a box with an optional circular hole
                      or edge crack (Sec. 4, Fig. boundnoncon; Sec. 5 workloads).
  * ``Oracle``     -- the full time step: Eqs. (moments), (coll), (stream) and
                      the boundary rules Eqs. (bbcon), (abbcon), (bbnoncon),
                      (abbnoncon), with displacement integration.
  * ``freund_ki0`` -- Freund's stress intensity of a suddenly loaded crack,
                      Sec. 5.2, valid for t < l_c / c_d.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None


class Link(C.Structure):
    _fields_ = [("node", C.c_int32), ("dir", C.c_int32), ("bc", C.c_int32),
                ("bc2", C.c_int32), ("q", C.c_double), ("n0", C.c_double),
                ("n1", C.c_double), ("curved", C.c_int32), ("pad", C.c_int32)]


class BC(C.Structure):
    _fields_ = [("kind", C.c_int32), ("profile", C.c_int32),
                ("value", C.c_double * 3), ("t_ramp", C.c_double)]


LINK_DTYPE = np.dtype([("node", "<i4"), ("dir", "<i4"), ("bc", "<i4"), ("bc2", "<i4"),
                       ("q", "<f8"), ("n0", "<f8"), ("n1", "<f8"),
                       ("curved", "<i4"), ("pad", "<i4")])
assert LINK_DTYPE.itemsize == C.sizeof(Link)

DIRICHLET, NEUMANN, PRESSURE, STRESS = 0, 1, 2, 3
STEP, RAMP = 0, 1


def build(force: bool = False) -> str:
    """Compile lbm_oracle.c into oracle/_build/liblbm_oracle.so."""
    with _lock:
        if (not force and os.path.exists(_OUT)
                and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
            return _OUT
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
        return _OUT


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    d, i32, i64, p = C.c_double, C.c_int32, C.c_int64, C.c_void_p
    dp = C.POINTER(C.c_double)
    lib.ora_feq.argtypes = [d, d, d, d, d, d, dp]
    lib.ora_feq.restype = None
    lib.ora_collide.argtypes = [dp, d, d, d, dp, dp]
    lib.ora_collide.restype = None
    lib.ora_geometry.argtypes = [i32, i32, C.POINTER(i32), d, d, d, i32, i32, i32, i32,
                                 C.POINTER(C.c_uint8), C.POINTER(Link), i64]
    lib.ora_geometry.restype = i64
    lib.ora_create.argtypes = [i32, i32, d, d, d, d, d, d, i32, i32,
                               C.POINTER(C.c_uint8), C.POINTER(Link), i64,
                               C.POINTER(BC), i32, i32]
    lib.ora_create.restype = p
    lib.ora_destroy.argtypes = [p]
    lib.ora_destroy.restype = None
    lib.ora_set_state.argtypes = [p, dp, dp, i64]
    lib.ora_set_state.restype = None
    lib.ora_get_state.argtypes = [p, dp, dp, C.POINTER(i64)]
    lib.ora_get_state.restype = None
    lib.ora_step.argtypes = [p, i32]
    lib.ora_step.restype = None
    lib.ora_fields.argtypes = [p, dp, dp, dp, dp]
    lib.ora_fields.restype = None
    lib.ora_time.argtypes = [p]
    lib.ora_time.restype = i64
    lib.ora_threads.argtypes = []
    lib.ora_threads.restype = i32
    lib.ora_set_threads.argtypes = [i32]
    lib.ora_set_threads.restype = None
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def threads() -> int:
    return int(_load().ora_threads())


def set_threads(n: int) -> None:
    _load().ora_set_threads(int(n))


def feq(rho, j, P) -> np.ndarray:
    """Eq. (fieq).  P = (Pxx, Pyy, Pxy)."""
    out = np.zeros(9)
    _load().ora_feq(float(rho), float(j[0]), float(j[1]), float(P[0]), float(P[1]),
                    float(P[2]), _dptr(out))
    return out


def collide(f, S, tau):
    """Eq. (coll) on one node; returns (f_col, j) with j = sum f c + S/2."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(9)
    j = np.zeros(2)
    _load().ora_collide(_dptr(f), float(S[0]), float(S[1]), float(tau), _dptr(out), _dptr(j))
    return out, j


def geometry(nx, ny, edge_bc=(0, 0, 0, 0), hole=None, crack=None):
    """Node mask and cut-link table of a box with an optional hole or edge crack.

    edge_bc: boundary-condition index of the (left, right, bottom, top) edge;
             -1 on both sides of an axis makes that axis periodic.
    hole:    (cx, cy, R, bc) or None.
    crack:   (length, bc) or (length, bc, x0) or None -- a crack along
             y = ny/2 - 1/2: from the left edge (x0 = 0, the default) or
             between the tips x0 - 1/2 and x0 + length - 1/2.
    Returns (node_type uint8 [ny, nx], links structured array, canonical order:
    node row-major, then direction 1..8).
    """
    lib = _load()
    eb = (C.c_int32 * 4)(*[int(v) for v in edge_bc])
    hx, hy, hr, hb = hole if hole is not None else (0.0, 0.0, 0.0, -1)
    cl, cb, cx0 = (tuple(crack) + (0,))[:3] if crack is not None else (0, -1, 0)
    nt = np.zeros(nx * ny, dtype=np.uint8)
    args = (int(nx), int(ny), eb, float(hx), float(hy), float(hr), int(hb), int(cl), int(cb),
            int(cx0), nt.ctypes.data_as(C.POINTER(C.c_uint8)))
    n = lib.ora_geometry(*args, None, 0)
    if n < 0:
        raise ValueError(f"ora_geometry rejected the arguments (status {n})")
    links = np.zeros(n, dtype=LINK_DTYPE)
    n2 = lib.ora_geometry(*args, links.ctypes.data_as(C.POINTER(Link)), n)
    assert n2 == n
    return nt.reshape(ny, nx), links


def make_bcs(specs):
    """specs: list of dicts {kind, value=(a[, b[, c]]), profile=STEP, t_ramp=0}.

    kind DIRICHLET: value = d(u*)/dt; NEUMANN: value = traction t*;
    PRESSURE: value[0] = p with t* = -p n; STRESS: value = (xx, yy, xy), t* = sigma n.
    """
    arr = (BC * max(1, len(specs)))()
    for k, sp in enumerate(specs):
        arr[k].kind = int(sp["kind"])
        arr[k].profile = int(sp.get("profile", STEP))
        val = list(sp["value"]) + [0.0] * (3 - len(sp["value"]))
        for m in range(3):
            arr[k].value[m] = float(val[m])
        arr[k].t_ramp = float(sp.get("t_ramp", 0.0))
    return arr


class Oracle:
    """One FP64 solver instance (lattice units: dx = dt = 1, c_s^2 = 1/3)."""

    def __init__(self, node_type, links, bcs, lam, mu, rho0=1.0, tau=0.55,
                 force=(0.0, 0.0), periodic=(False, False), wall_node=False):
        """wall_node=True takes rho^bd and sigma^bd at the boundary node instead of
        extrapolating them along the link (an option, not the paper's rule)."""
        self._lib = _load()
        node_type = np.ascontiguousarray(node_type, dtype=np.uint8)
        self.ny, self.nx = node_type.shape
        self.N = self.nx * self.ny
        self._links = np.ascontiguousarray(links, dtype=LINK_DTYPE)
        self._bcs = make_bcs(bcs)
        self._h = self._lib.ora_create(
            self.nx, self.ny, float(lam), float(mu), float(rho0), float(tau),
            float(force[0]), float(force[1]), int(periodic[0]), int(periodic[1]),
            node_type.ctypes.data_as(C.POINTER(C.c_uint8)),
            self._links.ctypes.data_as(C.POINTER(Link)), len(self._links),
            self._bcs, len(bcs), int(bool(wall_node)))
        if not self._h:
            raise RuntimeError("ora_create failed")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ora_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    @property
    def t(self) -> int:
        return int(self._lib.ora_time(self._h))

    def step(self, n: int = 1) -> None:
        self._lib.ora_step(self._h, int(n))

    def state(self):
        f = np.zeros(self.N * 9)
        u = np.zeros(self.N * 2)
        self._lib.ora_get_state(self._h, _dptr(f), _dptr(u), None)
        return f.reshape(self.ny, self.nx, 9), u.reshape(self.ny, self.nx, 2)

    def set_state(self, f=None, u=None, t: int = 0) -> None:
        fp = up = None
        if f is not None:
            f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
            assert f.size == self.N * 9
            fp = _dptr(f)
        if u is not None:
            u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
            assert u.size == self.N * 2
            up = _dptr(u)
        self._lib.ora_set_state(self._h, fp, up, int(t))

    def fields(self):
        """Dict of u (2, ny, nx), v (2, ny, nx), sigma (3, ny, nx: xx, yy, xy), rho."""
        u = np.zeros(2 * self.N)
        v = np.zeros(2 * self.N)
        s = np.zeros(3 * self.N)
        r = np.zeros(self.N)
        self._lib.ora_fields(self._h, _dptr(u), _dptr(v), _dptr(s), _dptr(r))
        sh = (self.ny, self.nx)
        return {"u": u.reshape((2,) + sh), "v": v.reshape((2,) + sh),
                "sigma": s.reshape((3,) + sh), "rho": r.reshape(sh)}


def freund_ki0(t, tstar, nu, cd=1.0):
    """Freund's mode-I stress intensity for a suddenly loaded crack (Sec. 5.2):
    K_I^0 = 2 t* sqrt(1 - 2 nu)/(1 - nu) sqrt(c_d t / pi), for t < l_c/c_d."""
    t = np.asarray(t, dtype=np.float64)
    return 2.0 * tstar * np.sqrt(1.0 - 2.0 * nu) / (1.0 - nu) * np.sqrt(cd * t / np.pi)

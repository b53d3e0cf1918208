"""ctypes binding of liblbm.so (include/lbm.h): argument marshalling only.

Every function keeps the C name.  Device memory and streams come from PyTorch
(a uint8 CUDA tensor as the solver workspace, ``torch.cuda.current_stream()``);
all computation runs in the library's CUDA kernels.  There is no fallback: if
the library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LBM_OK, LBM_ERR_ARG, LBM_ERR_NOMEM, LBM_ERR_CUDA, LBM_ERR_UNSTABLE, LBM_ERR_TIMEOUT = range(6)
LBM_F32, LBM_F16_DEV, LBM_BF16_DEV = 0, 1, 2
LBM_WALL_EXTRAPOLATE, LBM_WALL_NODE = 0, 1
LBM_TIME_BLOCK = 8  # steps per launch of the temporally blocked kernel (include/lbm.h)
LBM_STREAM_TWO_BUFFERS, LBM_STREAM_IN_PLACE = 0, 1  # lbm_streaming
STORAGE = {"f32": LBM_F32, "f16": LBM_F16_DEV, "bf16": LBM_BF16_DEV}
_STATUS = {0: "LBM_OK", 1: "LBM_ERR_ARG", 2: "LBM_ERR_NOMEM", 3: "LBM_ERR_CUDA",
           4: "LBM_ERR_UNSTABLE", 5: "LBM_ERR_TIMEOUT"}


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class lbm_bc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("profile", C.c_int32), ("value", C.c_double * 3),
                ("t_ramp", C.c_double)]


class lbm_link(C.Structure):
    _fields_ = [("node", C.c_int32), ("dir", C.c_int32), ("bc", C.c_int32), ("bc2", C.c_int32),
                ("q", C.c_double), ("n", C.c_double * 2)]


LINK_DTYPE = np.dtype([("node", "<i4"), ("dir", "<i4"), ("bc", "<i4"), ("bc2", "<i4"),
                       ("q", "<f8"), ("n0", "<f8"), ("n1", "<f8")])


class lbm_geom(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("edge_bc", C.c_int32 * 4),
                ("hole_cx", C.c_double), ("hole_cy", C.c_double), ("hole_r", C.c_double),
                ("hole_bc", C.c_int32), ("crack_len", C.c_int32), ("crack_bc", C.c_int32),
                ("crack_x0", C.c_int32)]


class lbm_desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("lam", C.c_double), ("mu", C.c_double),
                ("rho0", C.c_double), ("dx", C.c_double), ("dt", C.c_double),
                ("tau", C.c_double), ("force", C.c_double * 2),
                ("node_type", C.POINTER(C.c_uint8)), ("links", C.c_void_p),
                ("nlinks", C.c_int64), ("bcs", C.POINTER(lbm_bc)), ("nbcs", C.c_int32),
                ("storage", C.c_int32), ("wall_values", C.c_int32), ("time_block", C.c_int32),
                ("streaming", C.c_int32)]


class lbm_info(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("pitch", C.c_int32),
                ("storage", C.c_int32), ("time", C.c_int64), ("boundary_nodes", C.c_int64),
                ("interior_nodes", C.c_int64), ("workspace_bytes", C.c_uint64),
                ("storage_scale", C.c_float), ("bytes_per_update", C.c_float),
                ("kernel_launches", C.c_int64), ("time_block", C.c_int32), ("streaming", C.c_int32)]


class lbm_launch_shape(C.Structure):
    _fields_ = [("tile_x", C.c_int32), ("tile_y", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("dynamic", C.c_int32)]


class lbm_batch_stats(C.Structure):
    _fields_ = [("instances", C.c_int32), ("unstable", C.c_int32), ("nodes", C.c_int64),
                ("steps", C.c_int64), ("device_bytes", C.c_uint64),
                ("kernel_launches", C.c_int64), ("shape", lbm_launch_shape),
                ("blocked_instances", C.c_int32), ("pad", C.c_int32)]


class lbm_server_stats(C.Structure):
    _fields_ = [("active", C.c_int32), ("queued", C.c_int32), ("admitted", C.c_int32),
                ("finished", C.c_int32), ("steps", C.c_int64), ("active_nodes", C.c_int64),
                ("device_bytes", C.c_uint64), ("kernel_launches", C.c_int64)]


class lbm_timing(C.Structure):
    _fields_ = [("interior_ms", C.c_double), ("boundary_ms", C.c_double), ("steps", C.c_int64)]


assert C.sizeof(lbm_bc) == 40 and C.sizeof(lbm_link) == 40 and LINK_DTYPE.itemsize == 40
assert C.sizeof(lbm_geom) == 64

# name -> (restype, argtypes); every symbol include/lbm.h declares
SIGNATURES = {
    "lbm_geom_build": (C.c_int, [C.POINTER(lbm_geom), C.POINTER(C.c_uint8), C.c_void_p,
                                 C.c_int64, C.POINTER(C.c_int64)]),
    "lbm_workspace_size": (C.c_int, [C.POINTER(lbm_desc), C.POINTER(C.c_uint64)]),
    "lbm_create": (C.c_int, [C.POINTER(lbm_desc), C.c_void_p, C.c_void_p, C.c_uint64,
                             C.POINTER(C.c_void_p)]),
    "lbm_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "lbm_get_fields": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "lbm_get_fields_host_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_probe": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32,
                            C.POINTER(C.c_float)]),
    "lbm_set_bc": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(lbm_bc)]),
    "lbm_reset": (C.c_int, [C.c_void_p]),
    "lbm_sync": (C.c_int, [C.c_void_p]),
    "lbm_get_info": (C.c_int, [C.c_void_p, C.POINTER(lbm_info)]),
    "lbm_set_wait_limit": (C.c_int, [C.c_void_p, C.c_int64]),
    "lbm_set_timing": (C.c_int, [C.c_void_p, C.c_int32]),
    "lbm_get_timing": (C.c_int, [C.c_void_p, C.POINTER(lbm_timing)]),
    "lbm_destroy": (C.c_int, [C.c_void_p]),
    "lbm_last_error": (C.c_char_p, []),
    "lbm_batch_create": (C.c_int, [C.POINTER(lbm_desc), C.c_int32, C.c_void_p,
                                   C.POINTER(C.c_void_p)]),
    "lbm_batch_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "lbm_batch_get_fields": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_int32]),
    "lbm_batch_tune": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(lbm_launch_shape)]),
    "lbm_batch_set_shape": (C.c_int, [C.c_void_p, C.POINTER(lbm_launch_shape)]),
    "lbm_batch_reset": (C.c_int, [C.c_void_p]),
    "lbm_batch_sync": (C.c_int, [C.c_void_p]),
    "lbm_batch_info": (C.c_int, [C.c_void_p, C.POINTER(lbm_batch_stats)]),
    "lbm_batch_destroy": (C.c_int, [C.c_void_p]),
    "lbm_server_create": (C.c_int, [C.c_uint64, C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]),
    "lbm_server_submit": (C.c_int, [C.c_void_p, C.POINTER(lbm_desc), C.c_int64,
                                    C.POINTER(C.c_int64)]),
    "lbm_server_tick": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(lbm_server_stats)]),
    "lbm_server_result": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_int32), C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    "lbm_server_destroy": (C.c_int, [C.c_void_p]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblbm.so (building it first if it is missing and nvcc is present)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError(f"liblbm.so not built ({path}); run paper_2208_04088_gb300.build.build()")
        _build.build()
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int) -> None:
    if status != LBM_OK:
        raise LbmError(status, load().lbm_last_error().decode())


def make_bcs(specs):
    arr = (lbm_bc * max(1, len(specs)))()
    for k, sp in enumerate(specs):
        arr[k].kind = int(sp["kind"])
        arr[k].profile = int(sp.get("profile", 0))
        val = list(sp["value"]) + [0.0] * (3 - len(sp["value"]))
        for m in range(3):
            arr[k].value[m] = float(val[m])
        arr[k].t_ramp = float(sp.get("t_ramp", 0.0))
    return arr


def lbm_geom_build(nx, ny, edge_bc=(0, 0, 0, 0), hole=None, crack=None):
    """Node mask (uint8 [ny, nx]) and cut links (structured LINK_DTYPE array)."""
    lib = load()
    g = lbm_geom()
    g.nx, g.ny = int(nx), int(ny)
    for e in range(4):
        g.edge_bc[e] = int(edge_bc[e])
    if hole is not None:
        g.hole_cx, g.hole_cy, g.hole_r, g.hole_bc = float(hole[0]), float(hole[1]), float(hole[2]), int(hole[3])
    if crack is not None:
        g.crack_len, g.crack_bc = int(crack[0]), int(crack[1])
        g.crack_x0 = int(crack[2]) if len(crack) > 2 else 0
    nt = np.empty(int(nx) * int(ny), dtype=np.uint8)
    n = C.c_int64(0)
    ntp = nt.ctypes.data_as(C.POINTER(C.c_uint8))
    # one build with room for every link of the box edges, the crack faces and
    # the hole rim; a second only if that was too small (the first call
    # reports the count)
    cap = 16 * (int(nx) + int(ny)) + 64
    if crack is not None:
        cap += 16 * int(crack[0])
    if hole is not None:
        cap += int(64 * (abs(float(hole[2])) + 2))
    links = np.empty(cap, dtype=LINK_DTYPE)
    st = lib.lbm_geom_build(C.byref(g), ntp, links.ctypes.data_as(C.c_void_p), cap, C.byref(n))
    if st != LBM_OK and n.value > cap:
        links = np.empty(n.value, dtype=LINK_DTYPE)
        st = lib.lbm_geom_build(C.byref(g), ntp, links.ctypes.data_as(C.c_void_p), n.value,
                                C.byref(n))
    _check(st)
    return nt.reshape(int(ny), int(nx)), links[:n.value]


class Desc:
    """Owns the host arrays an lbm_desc points to."""

    def __init__(self, node_type, links, bcs, lam, mu, rho0=1.0, dx=1.0, dt=1.0, tau=0.55,
                 force=(0.0, 0.0), storage="f32", wall_node=False, time_block=0, in_place=False):
        self.node_type = np.ascontiguousarray(node_type, dtype=np.uint8)
        self.links = np.ascontiguousarray(links, dtype=LINK_DTYPE)
        self.bcs = make_bcs(bcs)
        self.ny, self.nx = self.node_type.shape
        d = lbm_desc()
        d.nx, d.ny = self.nx, self.ny
        d.lam, d.mu, d.rho0, d.dx, d.dt, d.tau = lam, mu, rho0, dx, dt, tau
        d.force[0], d.force[1] = force
        d.node_type = self.node_type.ctypes.data_as(C.POINTER(C.c_uint8))
        d.links = self.links.ctypes.data_as(C.c_void_p)
        d.nlinks = len(self.links)
        d.bcs = self.bcs
        d.nbcs = len(bcs)
        d.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        d.wall_values = LBM_WALL_NODE if wall_node else LBM_WALL_EXTRAPOLATE
        # 0: library default, 1: one step per launch, LBM_TIME_BLOCK: temporal blocking
        d.time_block = int(time_block)
        d.streaming = LBM_STREAM_IN_PLACE if in_place else LBM_STREAM_TWO_BUFFERS
        self.c = d


def desc_from_workload(w, storage="f32", links_edit=None, wall_node=None,
                       time_block=0, in_place=False) -> Desc:
    nt, links = lbm_geom_build(**w.geometry_args())
    if links_edit is not None:
        links = links_edit(links)
    wn = w.wall_node if wall_node is None else wall_node
    return Desc(nt, links, w.bcs, w.lam, w.mu, w.rho0, tau=w.tau, storage=storage, wall_node=wn,
                time_block=time_block, in_place=in_place)


def lbm_workspace_size(desc: Desc) -> int:
    n = C.c_uint64(0)
    _check(load().lbm_workspace_size(C.byref(desc.c), C.byref(n)))
    return int(n.value)


def lbm_create(desc: Desc, stream: int = 0, workspace_ptr: int = 0, workspace_bytes: int = 0):
    h = C.c_void_p(0)
    _check(load().lbm_create(C.byref(desc.c), C.c_void_p(stream), C.c_void_p(workspace_ptr),
                             C.c_uint64(workspace_bytes), C.byref(h)))
    return h


def lbm_step(h, nsteps: int) -> None:
    _check(load().lbm_step(h, C.c_int64(int(nsteps))))


def lbm_get_fields(h, u_ptr: int = 0, v_ptr: int = 0, sigma_ptr: int = 0,
                   on_device: bool = True) -> None:
    _check(load().lbm_get_fields(h, C.c_void_p(u_ptr), C.c_void_p(v_ptr), C.c_void_p(sigma_ptr),
                                 int(bool(on_device))))


def lbm_get_fields_host_noalloc(h, u_ptr: int = 0, v_ptr: int = 0, sigma_ptr: int = 0) -> None:
    """Fields to host pointers without device allocation (static staging array,
    at most 262144 nodes; see include/lbm.h)."""
    _check(load().lbm_get_fields_host_noalloc(h, C.c_void_p(u_ptr), C.c_void_p(v_ptr),
                                              C.c_void_p(sigma_ptr)))


def lbm_probe(h, nodes) -> np.ndarray:
    nodes = np.ascontiguousarray(nodes, dtype=np.int32)
    out = np.zeros((len(nodes), 7), dtype=np.float32)
    _check(load().lbm_probe(h, nodes.ctypes.data_as(C.POINTER(C.c_int32)), len(nodes),
                            out.ctypes.data_as(C.POINTER(C.c_float))))
    return out


def lbm_set_bc(h, index: int, spec: dict) -> None:
    arr = make_bcs([spec])
    _check(load().lbm_set_bc(h, int(index), arr))


def lbm_reset(h) -> None:
    _check(load().lbm_reset(h))


def lbm_sync(h) -> None:
    _check(load().lbm_sync(h))


def lbm_get_info(h) -> dict:
    info = lbm_info()
    _check(load().lbm_get_info(h, C.byref(info)))
    return {k: getattr(info, k) for k, _ in lbm_info._fields_}


def lbm_set_wait_limit(h, limit_ns: int) -> None:
    _check(load().lbm_set_wait_limit(h, C.c_int64(int(limit_ns))))


def lbm_set_timing(h, enable: bool) -> None:
    _check(load().lbm_set_timing(h, int(bool(enable))))


def lbm_get_timing(h) -> dict:
    t = lbm_timing()
    _check(load().lbm_get_timing(h, C.byref(t)))
    return {"interior_ms": t.interior_ms, "boundary_ms": t.boundary_ms, "steps": t.steps}


def lbm_destroy(h) -> None:
    _check(load().lbm_destroy(h))


def lbm_last_error() -> str:
    return load().lbm_last_error().decode()


class Solver:
    """One solver instance with a PyTorch-owned workspace on the current device.

    Argument marshalling only: every step, field and probe runs in liblbm.so.
    """

    def __init__(self, desc: Desc, stream=None, device=None):
        import torch
        self.desc = desc
        self.nx, self.ny = desc.nx, desc.ny
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        nbytes = lbm_workspace_size(desc)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8,
                                     device=device if device is not None else "cuda")
        ptr = self.workspace.data_ptr()
        ptr = (ptr + 255) // 256 * 256
        self.h = lbm_create(desc, self.stream.cuda_stream, ptr, nbytes)

    def step(self, n: int) -> None:
        lbm_step(self.h, n)

    def fields(self):
        """Dict of float32 CUDA tensors u (2, ny, nx), v (2, ny, nx), sigma (3, ny, nx)."""
        import torch
        dev = self.workspace.device
        u = torch.empty((2, self.ny, self.nx), dtype=torch.float32, device=dev)
        v = torch.empty_like(u)
        s = torch.empty((3, self.ny, self.nx), dtype=torch.float32, device=dev)
        lbm_get_fields(self.h, u.data_ptr(), v.data_ptr(), s.data_ptr(), on_device=True)
        return {"u": u, "v": v, "sigma": s}

    def fields_host(self):
        u = np.empty((2, self.ny, self.nx), dtype=np.float32)
        v = np.empty_like(u)
        s = np.empty((3, self.ny, self.nx), dtype=np.float32)
        lbm_get_fields(self.h, u.ctypes.data, v.ctypes.data, s.ctypes.data, on_device=False)
        return {"u": u, "v": v, "sigma": s}

    def probe(self, nodes) -> np.ndarray:
        return lbm_probe(self.h, nodes)

    def reset(self) -> None:
        lbm_reset(self.h)

    def sync(self) -> None:
        lbm_sync(self.h)

    def info(self) -> dict:
        return lbm_get_info(self.h)

    def set_timing(self, enable: bool) -> None:
        lbm_set_timing(self.h, enable)

    def timing(self) -> dict:
        return lbm_get_timing(self.h)

    def set_bc(self, index: int, spec: dict) -> None:
        lbm_set_bc(self.h, index, spec)

    def close(self) -> None:
        if getattr(self, "h", None) is not None and self.h.value:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _shape_dict(sh):
    return {"tile_x": sh.tile_x, "tile_y": sh.tile_y, "blocks_per_sm": sh.blocks_per_sm,
            "dynamic": sh.dynamic}


class Batch:
    """Many lambda = mu instances advanced by one persistent launch per step
    (lbm_batch_* of include/lbm.h).  Argument marshalling only."""

    def __init__(self, descs, stream=None):
        import torch
        self.descs = list(descs)  # keeps the host arrays alive until create returns
        arr = (lbm_desc * len(self.descs))()
        for k, d in enumerate(self.descs):
            arr[k] = d.c
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p(0)
        _check(load().lbm_batch_create(arr, len(self.descs), C.c_void_p(self.stream.cuda_stream),
                                       C.byref(h)))
        self.h = h

    def step(self, n):
        _check(load().lbm_batch_step(self.h, C.c_int64(int(n))))

    def fields_host(self, index):
        d = self.descs[index]
        u = np.empty((2, d.ny, d.nx), np.float32)
        v = np.empty_like(u)
        s = np.empty((3, d.ny, d.nx), np.float32)
        _check(load().lbm_batch_get_fields(self.h, int(index), C.c_void_p(u.ctypes.data),
                                           C.c_void_p(v.ctypes.data), C.c_void_p(s.ctypes.data), 0))
        return {"u": u, "v": v, "sigma": s}

    def tune(self, steps_per_trial=20):
        sh = lbm_launch_shape()
        _check(load().lbm_batch_tune(self.h, int(steps_per_trial), C.byref(sh)))
        return _shape_dict(sh)

    def set_shape(self, tile_x, tile_y, blocks_per_sm, dynamic):
        sh = lbm_launch_shape(tile_x, tile_y, blocks_per_sm, dynamic)
        _check(load().lbm_batch_set_shape(self.h, C.byref(sh)))

    def reset(self):
        _check(load().lbm_batch_reset(self.h))

    def sync(self):
        _check(load().lbm_batch_sync(self.h))

    def info(self):
        st = lbm_batch_stats()
        _check(load().lbm_batch_info(self.h, C.byref(st)))
        out = {k: getattr(st, k) for k, _ in lbm_batch_stats._fields_ if k not in ("pad", "shape")}
        out["shape"] = _shape_dict(st.shape)
        return out

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _check(load().lbm_batch_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server (lbm_server_* of include/lbm.h)."""

    QUEUED, RUNNING, DONE = 0, 1, 2

    def __init__(self, budget_bytes, storage="f32", stream=None):
        import torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p(0)
        st = STORAGE[storage] if isinstance(storage, str) else int(storage)
        _check(load().lbm_server_create(C.c_uint64(int(budget_bytes)), st,
                                        C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h
        self.shapes = {}

    def submit(self, desc, nsteps):
        rid = C.c_int64(0)
        _check(load().lbm_server_submit(self.h, C.byref(desc.c), C.c_int64(int(nsteps)),
                                        C.byref(rid)))
        self.shapes[rid.value] = (desc.ny, desc.nx)
        return rid.value

    def tick(self, max_steps=64):
        st = lbm_server_stats()
        _check(load().lbm_server_tick(self.h, int(max_steps), C.byref(st)))
        return {k: getattr(st, k) for k, _ in lbm_server_stats._fields_}

    def result(self, rid):
        """None while queued or running; the fields dict once done."""
        ny, nx = self.shapes[rid]
        u = np.empty((2, ny, nx), np.float32)
        v = np.empty_like(u)
        s = np.empty((3, ny, nx), np.float32)
        state = C.c_int32(0)
        st = load().lbm_server_result(self.h, C.c_int64(rid), C.byref(state),
                                      C.c_void_p(u.ctypes.data), C.c_void_p(v.ctypes.data),
                                      C.c_void_p(s.ctypes.data))
        if st not in (LBM_OK, LBM_ERR_UNSTABLE):
            _check(st)
        if state.value != self.DONE:
            return None
        del self.shapes[rid]
        return {"u": u, "v": v, "sigma": s, "unstable": st == LBM_ERR_UNSTABLE}

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _check(load().lbm_server_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

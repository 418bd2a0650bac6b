"""ctypes binding of the octfuse C ABI (``include/octfuse.h``).

Argument marshalling only: every function here forwards to the entry point of
the same name in ``libofu.so``; all arithmetic runs in the library's CUDA
kernels.  Pointers are plain integers (``tensor.data_ptr()``, a NumPy array's
``ctypes.data``), so the caller decides whether they live on the host or the
device.  A missing library raises at load time: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libofu.so")

OFU_OK, OFU_EINVAL, OFU_ENOMEM, OFU_ECUDA, OFU_ESTATE, OFU_ECAPACITY, OFU_ETIMEOUT = range(7)
FIELD_U, FIELD_UBAR, FIELD_P, FIELD_TAU, FIELD_SIGMA, FIELD_W, FIELD_SAMPLE_OFF, FIELD_SAMPLES = range(8)
FACES = ("+x", "+y", "+z", "-x", "-y", "-z")


class Params(ctypes.Structure):
    _fields_ = [
        ("origin", ctypes.c_double * 3),
        ("extent", ctypes.c_double),
        ("max_depth", ctypes.c_int32),
        ("sample_fp16", ctypes.c_int32),
        ("delta", ctypes.c_double),
        ("eta", ctypes.c_double),
        ("lambda_", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("tau_split", ctypes.c_double),
        ("tau_join", ctypes.c_double),
        ("spread_tau", ctypes.c_double),
        ("max_leaves", ctypes.c_int64),
        ("data_term", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class OfuError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"octfuse status {status}: {msg}")
        self.status = status


_lib = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_d = ctypes.c_double
_P64 = ctypes.POINTER(ctypes.c_int64)
_PD = ctypes.POINTER(ctypes.c_double)
_PI32 = ctypes.POINTER(ctypes.c_int32)

# device allocator callbacks of ofu_create_octree_ex
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)

_SIGS = {
    "ofu_default_params": (None, [ctypes.POINTER(Params)]),
    "ofu_create_octree": (_i32, [ctypes.POINTER(Params), _vp, ctypes.POINTER(_vp)]),
    "ofu_create_octree_ex": (_i32, [ctypes.POINTER(Params), _vp, ALLOC_FN, FREE_FN, _vp,
                                    ctypes.POINTER(_vp)]),
    "ofu_destroy": (None, [_vp]),
    "ofu_last_error": (ctypes.c_char_p, [_vp]),
    "ofu_integrate_frames": (_i32, [_vp, _i32, _i32, _i32, _vp, _vp, _vp]),
    "ofu_iterate": (_i32, [_vp, _i32]),
    "ofu_descend": (_i32, [_vp, _i32, _i32, _d, _d, _i32]),
    "ofu_quantisation_error": (_i32, [_vp, _vp, _i64, _PD]),
    "ofu_extract_mesh": (_i32, [_vp, _vp, _i64, _vp, _i64, _P64, _P64]),
    "ofu_export_frame_tree": (_i32, [_vp, _i32, _vp, _vp, _i64, _P64]),
    "ofu_data_term_memory": (_i32, [_vp, _vp, _P64, _P64, _P64]),
    "ofu_restructure": (_i32, [_vp, _P64, _P64, _P64]),
    "ofu_energy": (_i32, [_vp, _PD, _PD, _PD]),
    "ofu_num_leaves": (_i32, [_vp, _P64]),
    "ofu_export_leaves": (_i32, [_vp, _vp, _vp, _vp, _i64, _P64]),
    "ofu_solve": (_i32, [_vp, _i32, _i32, _i32, _d, _PI32, _P64, _PD]),
    "ofu_export_field": (_i32, [_vp, _i32, _vp, _i64, _P64]),
    "ofu_export_neighbours": (_i32, [_vp, _i32, _vp, _vp, _i64, _P64]),
    "ofu_import_leaves": (_i32, [_vp, _vp, _vp, _i64, _vp, _vp]),
    "ofu_set_state": (_i32, [_vp, _vp, _vp, _vp, _i64]),
    "ofu_mlp_num_params": (_i64, []),
    "ofu_mlp_create": (_i32, [_vp, ctypes.POINTER(_vp)]),
    "ofu_mlp_destroy": (None, [_vp]),
    "ofu_mlp_last_error": (ctypes.c_char_p, [_vp]),
    "ofu_mlp_set_params": (_i32, [_vp, _vp]),
    "ofu_mlp_get_params": (_i32, [_vp, _vp]),
    "ofu_mlp_forward": (_i32, [_vp, _vp, _i64, _vp]),
    "ofu_mlp_gradient": (_i32, [_vp, _vp, _vp, _vp, _vp, _i64, _vp, _PD]),
    "ofu_mlp_train_step": (_i32, [_vp, _vp, _vp, _vp, _vp, _i64, ctypes.c_float, _PD]),
    "ofu_features": (_i32, [_vp, _vp, _i64]),
    "ofu_warm_start": (_i32, [_vp, _vp]),
    "ofu_energy_static": (_i32, [_vp, _vp]),
    "ofu_save": (_i32, [_vp, ctypes.c_char_p]),
    "ofu_load": (_i32, [_vp, ctypes.c_char_p]),
    "ofu_kernel_launches": (_i64, []),
    "ofu_profile": (_i32, [_vp, _i32]),
    "ofu_profile_read": (_i32, [_vp, _PD, _P64, _PD]),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libofu.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"octfuse CUDA library not built: {path} is missing "
                           "(run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return tuple(_SIGS)


def _check(ctx, st):
    if st != OFU_OK:
        msg = load().ofu_last_error(ctx)
        raise OfuError(st, msg.decode() if msg else "")


def _ptr(x):
    """Integer address of a tensor / array / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


# ---- the C ABI, one function per entry point --------------------------------


def ofu_default_params() -> Params:
    p = Params()
    load().ofu_default_params(ctypes.byref(p))
    return p


def ofu_create_octree(params: Params, stream: int = 0) -> int:
    out = _vp()
    st = load().ofu_create_octree(ctypes.byref(params), _vp(stream or None), ctypes.byref(out))
    _check(None, st)
    return out.value


# callback objects of live contexts (ctypes frees a callback's trampoline
# when its Python object dies, so each is kept until ofu_destroy)
_allocators = {}


def ofu_create_octree_ex(params: Params, stream: int, alloc, free) -> int:
    """Context whose device memory comes from alloc(nbytes) -> int pointer (0 on
    failure) and goes back through free(ptr, nbytes)."""
    a = ALLOC_FN(lambda nbytes, user: alloc(nbytes) or None)
    f = FREE_FN(lambda ptr, nbytes, user: free(ptr, nbytes))
    out = _vp()
    st = load().ofu_create_octree_ex(ctypes.byref(params), _vp(stream or None), a, f, None,
                                     ctypes.byref(out))
    _check(None, st)
    _allocators[out.value] = (a, f)
    return out.value


def ofu_destroy(ctx: int) -> None:
    load().ofu_destroy(ctx)
    _allocators.pop(ctx, None)


def ofu_last_error(ctx: int = 0) -> str:
    msg = load().ofu_last_error(ctx or None)
    return msg.decode() if msg else ""


def ofu_integrate_frames(ctx, F, H, W, depth, intr, pose) -> None:
    _check(ctx, load().ofu_integrate_frames(ctx, F, H, W, _ptr(depth), _ptr(intr), _ptr(pose)))


def ofu_iterate(ctx, n: int) -> None:
    _check(ctx, load().ofu_iterate(ctx, n))


def ofu_descend(ctx, n: int, t0: int = 0, eps: float = 1e-3, xi0: float = 0.1,
                halve_every: int = 20) -> None:
    _check(ctx, load().ofu_descend(ctx, n, t0, eps, xi0, halve_every))


def ofu_quantisation_error(ctx, fine, n_fine: int) -> float:
    err = ctypes.c_double()
    _check(ctx, load().ofu_quantisation_error(ctx, _ptr(fine), n_fine, ctypes.byref(err)))
    return err.value


def ofu_extract_mesh(ctx, verts=None, vcap=0, tris=None, tcap=0):
    nv, nt = ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, load().ofu_extract_mesh(ctx, _ptr(verts), vcap, _ptr(tris), tcap, ctypes.byref(nv),
                                        ctypes.byref(nt)))
    return nv.value, nt.value


def ofu_export_frame_tree(ctx, frame, keys=None, levels=None, cap=0) -> int:
    n = ctypes.c_int64()
    _check(ctx, load().ofu_export_frame_tree(ctx, frame, _ptr(keys), _ptr(levels), cap, ctypes.byref(n)))
    return n.value


def ofu_data_term_memory(ctx, nodes=None):
    d, o, v = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, load().ofu_data_term_memory(ctx, _ptr(nodes), ctypes.byref(d), ctypes.byref(o),
                                            ctypes.byref(v)))
    return d.value, o.value, v.value


def ofu_restructure(ctx):
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, load().ofu_restructure(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def ofu_energy(ctx):
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(ctx, load().ofu_energy(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def ofu_num_leaves(ctx) -> int:
    n = ctypes.c_int64()
    _check(ctx, load().ofu_num_leaves(ctx, ctypes.byref(n)))
    return n.value


def ofu_export_leaves(ctx, keys, levels, u, cap) -> int:
    n = ctypes.c_int64()
    _check(ctx, load().ofu_export_leaves(ctx, _ptr(keys), _ptr(levels), _ptr(u), cap, ctypes.byref(n)))
    return n.value


def ofu_solve(ctx, iters, restructure_every, check_every, gap_tol):
    done, li = ctypes.c_int32(), ctypes.c_int64()
    e = (ctypes.c_double * 3)()
    _check(ctx, load().ofu_solve(ctx, iters, restructure_every, check_every, gap_tol,
                                 ctypes.byref(done), ctypes.byref(li), e))
    return done.value, li.value, (e[0], e[1], e[2])


def ofu_export_field(ctx, field, dst, cap_items) -> int:
    n = ctypes.c_int64()
    _check(ctx, load().ofu_export_field(ctx, field, _ptr(dst), cap_items, ctypes.byref(n)))
    return n.value


def ofu_export_neighbours(ctx, face, off, idx, cap) -> int:
    n = ctypes.c_int64()
    _check(ctx, load().ofu_export_neighbours(ctx, face, _ptr(off), _ptr(idx), cap, ctypes.byref(n)))
    return n.value


def ofu_import_leaves(ctx, keys, levels, n, u=None, p=None) -> None:
    _check(ctx, load().ofu_import_leaves(ctx, _ptr(keys), _ptr(levels), n, _ptr(u), _ptr(p)))


def ofu_set_state(ctx, u, ubar, p, n) -> None:
    _check(ctx, load().ofu_set_state(ctx, _ptr(u), _ptr(ubar), _ptr(p), n))


def _check_net(net, st):
    if st != OFU_OK:
        msg = load().ofu_mlp_last_error(net)
        raise OfuError(st, msg.decode() if msg else "")


def ofu_mlp_num_params() -> int:
    return int(load().ofu_mlp_num_params())


def ofu_mlp_create(stream: int = 0) -> int:
    out = _vp()
    _check_net(None, load().ofu_mlp_create(_vp(stream or None), ctypes.byref(out)))
    return out.value


def ofu_mlp_destroy(net) -> None:
    load().ofu_mlp_destroy(net)


def ofu_mlp_last_error(net=0) -> str:
    msg = load().ofu_mlp_last_error(net or None)
    return msg.decode() if msg else ""


def ofu_mlp_set_params(net, params) -> None:
    _check_net(net, load().ofu_mlp_set_params(net, _ptr(params)))


def ofu_mlp_get_params(net, params) -> None:
    _check_net(net, load().ofu_mlp_get_params(net, _ptr(params)))


def ofu_mlp_forward(net, X, B, y) -> None:
    _check_net(net, load().ofu_mlp_forward(net, _ptr(X), B, _ptr(y)))


def ofu_mlp_gradient(net, X, t, w, rows, B, grad):
    loss = ctypes.c_double()
    _check_net(net, load().ofu_mlp_gradient(net, _ptr(X), _ptr(t), _ptr(w), _ptr(rows), B,
                                            _ptr(grad), ctypes.byref(loss)))
    return loss.value


def ofu_mlp_train_step(net, X, t, w, rows, B, lr, want_loss=True):
    loss = ctypes.c_double()
    _check_net(net, load().ofu_mlp_train_step(net, _ptr(X), _ptr(t), _ptr(w), _ptr(rows), B, lr,
                                              ctypes.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def ofu_features(ctx, X, cap_rows) -> None:
    _check(ctx, load().ofu_features(ctx, _ptr(X), cap_rows))


def ofu_warm_start(ctx, net) -> None:
    _check(ctx, load().ofu_warm_start(ctx, net))


def ofu_energy_static(ctx, out3=None):
    """Energy without any device allocation; `out3` (host or device, 3 float64)
    receives primal, dual, gap.  Without `out3` a host array is returned."""
    host = out3 is None
    if host:
        out3 = np.zeros(3, np.float64)
    _check(ctx, load().ofu_energy_static(ctx, _ptr(out3)))
    return tuple(float(x) for x in out3) if host else out3


def ofu_save(ctx, path: str) -> None:
    _check(ctx, load().ofu_save(ctx, os.fsencode(path)))


def ofu_load(ctx, path: str) -> None:
    _check(ctx, load().ofu_load(ctx, os.fsencode(path)))


def ofu_kernel_launches() -> int:
    return int(load().ofu_kernel_launches())


def ofu_profile(ctx, enable) -> None:
    """enable: False/0 stops; True/1, or an iteration count that sizes the event pool, starts."""
    _check(ctx, load().ofu_profile(ctx, int(enable)))


def ofu_profile_read(ctx):
    """((ms_dual, ms_primal), (launches_dual, launches_primal), (bytes_dual, bytes_primal))"""
    ms = (ctypes.c_double * 2)()
    n = (ctypes.c_int64 * 2)()
    b = (ctypes.c_double * 2)()
    _check(ctx, load().ofu_profile_read(ctx, ms, n, b))
    return (ms[0], ms[1]), (n[0], n[1]), (b[0], b[1])


# ---- convenience wrapper (host NumPy in / out) -------------------------------


def params_for(scene, sample_fp16: bool = False, max_leaves: int = 0, frame_trees: bool = False) -> Params:
    """Params of a :class:`scenes.Scene` (frame_trees: data_term = 1)."""
    p = Params()
    for k in range(3):
        p.origin[k] = float(scene.origin[k])
    p.extent = float(scene.extent)
    p.max_depth = int(scene.max_depth)
    p.sample_fp16 = int(bool(sample_fp16))
    p.delta = float(scene.delta)
    p.eta = float(scene.eta)
    p.lambda_ = float(scene.lam)
    p.gamma = float(scene.gamma)
    p.tau_split = float(scene.tau_split)
    p.tau_join = float(scene.tau_join)
    p.spread_tau = float(scene.spread_tau)
    p.max_leaves = int(max_leaves)
    p.data_term = int(bool(frame_trees))
    return p


class Octree:
    """Owns one context; methods mirror the C ABI with NumPy host buffers."""

    def __init__(self, params: Params, stream: int = 0, allocator=None):
        """allocator: optional (alloc, free) pair for ofu_create_octree_ex."""
        if allocator is None:
            self.ctx = ofu_create_octree(params, stream)
        else:
            self.ctx = ofu_create_octree_ex(params, stream, *allocator)

    def close(self):
        if self.ctx:
            ofu_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def integrate_frames(self, depth, intr, pose):
        depth = np.ascontiguousarray(depth, np.float32)
        intr = np.ascontiguousarray(intr, np.float64)
        pose = np.ascontiguousarray(np.asarray(pose, np.float64).reshape(len(intr), 16))
        F, H, W = depth.shape
        ofu_integrate_frames(self.ctx, F, H, W, depth, intr, pose)

    def iterate(self, n):
        ofu_iterate(self.ctx, n)

    def descend(self, n, t0=0, eps=1e-3, xi0=0.1, halve_every=20):
        ofu_descend(self.ctx, n, t0, eps, xi0, halve_every)

    def quantisation_error(self, fine):
        fine = np.ascontiguousarray(fine, np.float32)
        return ofu_quantisation_error(self.ctx, fine, fine.size)

    def restructure(self):
        return ofu_restructure(self.ctx)

    def frame_tree(self, frame):
        """(keys uint64, levels uint8) of one frame's TSDF octree (data_term = 1)."""
        n = ofu_export_frame_tree(self.ctx, frame)
        k = np.empty(max(n, 1), np.uint64)
        lv = np.empty(max(n, 1), np.uint8)
        ofu_export_frame_tree(self.ctx, frame, k, lv, n)
        return k[:n], lv[:n]

    def mesh(self):
        """(vertices float32 [V, 3], triangles int32 [T, 3]) of the zero level set."""
        nv, nt = ofu_extract_mesh(self.ctx)
        v = np.empty((max(nv, 1), 3), np.float32)
        t = np.empty((max(nt, 1), 3), np.int32)
        ofu_extract_mesh(self.ctx, v, nv, t, nt)
        return v[:nv], t[:nt]

    def energy(self):
        return ofu_energy(self.ctx)

    @property
    def n(self):
        return ofu_num_leaves(self.ctx)

    def leaves(self):
        n = self.n
        k = np.empty(n, np.uint64)
        lv = np.empty(n, np.uint8)
        u = np.empty(n, np.float32)
        ofu_export_leaves(self.ctx, k, lv, u, n)
        return k, lv, u

    def field(self, which):
        n = ofu_export_field(self.ctx, which, None, 0)
        dt = {FIELD_W: np.int32, FIELD_SAMPLE_OFF: np.uint32}.get(which, np.float32)
        out = np.empty(n, dt)
        ofu_export_field(self.ctx, which, out, n)
        if which == FIELD_P:
            out = out.reshape(3, -1).T.copy()
        return out

    def neighbours(self):
        res = []
        n = self.n
        for face in range(6):
            nnz = ofu_export_neighbours(self.ctx, face, None, None, 0)
            off = np.empty(n + 1, np.int64)
            idx = np.empty(max(nnz, 1), np.int64)
            ofu_export_neighbours(self.ctx, face, off, idx, max(nnz, 1))
            res.append((off, idx[:nnz]))
        return res

    def import_leaves(self, keys, levels, u=None, p=None):
        keys = np.ascontiguousarray(keys, np.uint64)
        levels = np.ascontiguousarray(levels, np.uint8)
        if u is not None:
            u = np.ascontiguousarray(u, np.float32)
        if p is not None:
            p = np.ascontiguousarray(np.asarray(p, np.float32).T)
        ofu_import_leaves(self.ctx, keys, levels, len(keys), u, p)

    def set_state(self, u, ubar, p):
        u = np.ascontiguousarray(u, np.float32)
        ubar = None if ubar is None else np.ascontiguousarray(ubar, np.float32)
        p = np.ascontiguousarray(np.asarray(p, np.float32).T)
        ofu_set_state(self.ctx, u, ubar, p, len(u))

    def solve(self, iters, restructure_every=10, check_every=0, gap_tol=0.0):
        return ofu_solve(self.ctx, iters, restructure_every, check_every, gap_tol)

    def save(self, path):
        ofu_save(self.ctx, path)

    def load(self, path):
        ofu_load(self.ctx, path)

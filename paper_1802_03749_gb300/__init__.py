"""Python binding of libmeshloop (C ABI in ``include/meshloop.h``).

Locality-optimised indirect-increment mesh loops on GB300 (sm_103a), after
Sulyok et al., "Locality Optimized Unstructured Mesh Algorithms on GPUs"
(2018): host planning (reordering, partitioning, two-layer colouring) and
CUDA loops (staged two-layer colouring, global colouring, atomics).

This module only marshals arguments: every step of a loop runs in the
library's kernels, and every call raises ``MeshLoopError`` on a non-zero
status.  There is no fallback: if the library cannot be built or loaded,
importing a loop fails.  Device data are ``torch.Tensor`` objects on the
current CUDA device (PyTorch provides memory and streams only).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = [
    "MeshLoopError", "Plan", "lib", "loop_res_calc", "loop_bres_calc", "loop_adt_calc", "loop_save_soln",
    "loop_res_calc_host", "loop_update", "loop_update_noalloc", "loop_elem_assemble", "loop_adjoint",
    "loop_space_disc", "loop_getacc", "loop_face_flux", "mesh_map_renumber", "mp_check_device_status",
    "mp_grid_wait_test", "mp_recip_test",
    "REORDER", "COLORING", "LAYOUT", "MP_MAX_BLOCK_COLORS",
]

MP_OK = 0
MP_ERRORS = {-1: "MP_EINVAL", -2: "MP_EMAPRANGE", -3: "MP_ECOLORS", -4: "MP_ESMEM", -5: "MP_ECUDA",
             -6: "MP_ETIMEOUT", -7: "MP_ENOMEM", -8: "MP_EPLAN", -9: "MP_EIO", -10: "MP_ETOOBIG"}
MP_NOALLOC_MAX_CELLS = 4096 * 2048
MP_MAX_BLOCK_COLORS = 256
MP_MAX_MAPS = 4
MP_MAX_TOSETS = 2
REORDER = {"none": 0, "rcm": 1, "partition": 2}
STAGED = {None: -1, "pipelined": 0, "simple": 1, "smem_atomic": 2, "gather": 3, "inc_only": 4,
          "inc_only_gather": 5, "warp_agg": 6, "persistent": 7}
COLORING = {"hier": 0, "global": 1, "atomic": 2, "twostep": 3}
LAYOUT = {"aos": 0, "soa": 1}
DTYPE = {"f64": 0, "f32": 1, "f64dw": 2}
TABLES = {"block_offsets": 0, "color_offsets": 1, "block_color": 2, "thread_color": 3, "map": 4,
          "footprint": 5, "fp_start": 6, "fp_count": 7, "local_map": 8, "inv_offsets": 9, "inv_index": 10, "gather": 11}


class MeshLoopError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        self.name = MP_ERRORS.get(code, str(code))
        msg = lib().mp_error_string(code).decode() if _lib is not None else self.name
        super().__init__(f"{what}: {self.name} ({msg})" if what else f"{self.name} ({msg})")


class mp_map(ctypes.Structure):
    _fields_ = [("to_set", ctypes.c_int32), ("arity", ctypes.c_int32), ("to_size", ctypes.c_int64),
                ("idx", ctypes.c_void_p), ("written", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class mp_plan_opts(ctypes.Structure):
    _fields_ = [("block_size", ctypes.c_int32), ("reorder", ctypes.c_int32), ("coloring", ctypes.c_int32),
                ("layout", ctypes.c_int32), ("imbalance", ctypes.c_double), ("eps", ctypes.c_double),
                ("primary_map", ctypes.c_int32), ("data_reorder", ctypes.c_int32), ("staged", ctypes.c_int32),
                ("recolor", ctypes.c_int32), ("block_of", ctypes.c_void_p)]


class mp_plan_stats(ctypes.Structure):
    _fields_ = [("from_size", ctypes.c_int64), ("nblocks", ctypes.c_int32), ("nblock_colors", ctypes.c_int32),
                ("max_thread_colors", ctypes.c_int32), ("block_size", ctypes.c_int32), ("sprime", ctypes.c_int32),
                ("ntosets", ctypes.c_int32), ("lprime", ctypes.c_double), ("mean_thread_colors", ctypes.c_double),
                ("reuse", ctypes.c_double * MP_MAX_TOSETS), ("reuse_all", ctypes.c_double),
                ("footprint_total", ctypes.c_int64 * MP_MAX_TOSETS),
                ("footprint_max", ctypes.c_int32 * MP_MAX_TOSETS),
                ("to_set_id", ctypes.c_int32 * MP_MAX_TOSETS), ("to_set_size", ctypes.c_int64 * MP_MAX_TOSETS),
                ("plan_bytes", ctypes.c_int64),
                ("seconds_total", ctypes.c_double), ("seconds_reorder", ctypes.c_double),
                ("seconds_partition", ctypes.c_double), ("seconds_color", ctypes.c_double)]


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double

# name -> (restype, argtypes) for every entry point of include/meshloop.h
SIGNATURES = {
    "mp_plan_opts_default": (None, [ctypes.POINTER(mp_plan_opts)]),
    "mesh_plan_build": (_I32, [ctypes.POINTER(mp_map), _I32, _I64, ctypes.POINTER(mp_plan_opts),
                               ctypes.POINTER(_P)]),
    "mesh_plan_destroy": (None, [_P]),
    "mesh_plan_query": (_I32, [_P, ctypes.POINTER(mp_plan_stats)]),
    "mesh_plan_perm": (_I32, [_P, _I32, _P]),
    "mesh_plan_table": (_I32, [_P, _I32, _I32, _P, _I64, ctypes.POINTER(_I64)]),
    "mesh_map_renumber": (_I32, [_P, _I64, _I32, _P, _P, _I64, _P]),
    "mesh_plan_upload": (_I32, [_P]),
    "mesh_plan_set_staged": (_I32, [_P, _I32]),
    "mesh_batch_build": (_I32, [ctypes.POINTER(_P), _I32, ctypes.POINTER(_P)]),
    "mesh_plan_save": (_I32, [_P, ctypes.c_char_p]),
    "mesh_plan_load": (_I32, [ctypes.c_char_p, ctypes.POINTER(_P)]),
    "loop_res_calc": (_I32, [_P, _I32, _P, _P, _P, _P, _D, _D, _P]),
    "loop_res_calc_host": (_I32, [_P, _I32, _P, _P, _P, _P, _D, _D, _P]),
    "loop_bres_calc": (_I32, [_P, _I32, _P, _P, _P, _P, _P, _D, _D, _P]),
    "loop_adt_calc": (_I32, [_P, _I32, _P, _P, _P, _D, _D, _P]),
    "loop_save_soln": (_I32, [_I64, _I32, _I32, _P, _P, _P]),
    "loop_update": (_I32, [_I64, _I32, _I32, _P, _P, _P, _P, _P, _P]),
    "loop_update_noalloc": (_I32, [_I64, _I32, _I32, _P, _P, _P, _P, _P, _P]),
    "loop_elem_assemble": (_I32, [_P, _I32, _P, _P, _P, _P, _P, _D, _P]),
    "loop_adjoint": (_I32, [_P, _I32, _P, _P, _P, _P, _P, _P, _D, _D, _P]),
    "loop_space_disc": (_I32, [_P, _I32, _P, _P, _P, _P, _P]),
    "loop_getacc": (_I32, [_P, _I32, _P, _P, _P]),
    "loop_face_flux": (_I32, [_P, _I32, _P, _P, _P, _D, _D, _D, _P]),
    "mp_error_string": (ctypes.c_char_p, [_I32]),
    "mp_check_device_status": (_I32, [_P]),
    "mp_grid_wait_test": (_I32, [_I32, _I64, _I32, _P]),
    "mp_recip_test": (_I32, [_P, _P, _I64, _I32, _P]),
    "mp_version": (ctypes.c_char_p, []),
}


def lib():
    """Load (building first if needed) the in-tree libmeshloop.so."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name, None)
                if fn is None:
                    continue
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != MP_OK:
        raise MeshLoopError(rc, what)


def _np_ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ------------------------------------------------------------------ plans

class Plan:
    """A plan of one loop (``mesh_plan_build``).

    ``maps`` is a list of dicts ``{"to_set": id>=1, "idx": int32 [n, arity],
    "to_size": int, "written": bool}``; iterations are set 0.
    """

    def __init__(self, maps, from_size: int, block_size: int = 512, reorder: str = "partition",
                 coloring: str = "hier", layout: str = "aos", imbalance: float = 1.001, eps: float = 0.0,
                 primary_map: int = -1, data_reorder: int = -1, staged: str | None = None, block_of=None,
                 recolor: int = -1, _handle=None):
        L = lib()
        self._h = ctypes.c_void_p()
        if _handle is not None:
            self._h = _handle
            self.maps_meta = None
            return
        n = len(maps)
        arr = (mp_map * max(n, 1))()
        keep = []
        for i, m in enumerate(maps):
            idx = np.ascontiguousarray(m["idx"], dtype=np.int32)
            keep.append(idx)
            arity = idx.shape[1] if idx.ndim == 2 else 1
            arr[i] = mp_map(int(m["to_set"]), int(arity), int(m["to_size"]), idx.ctypes.data,
                            int(bool(m.get("written", False))), 0)
        o = mp_plan_opts()
        L.mp_plan_opts_default(ctypes.byref(o))
        o.block_size = int(block_size)
        o.reorder = REORDER[reorder]
        o.coloring = COLORING[coloring]
        o.layout = LAYOUT[layout]
        o.imbalance = float(imbalance)
        o.eps = float(eps)
        o.primary_map = int(primary_map)
        o.data_reorder = int(data_reorder)
        o.staged = STAGED[staged]
        o.recolor = int(recolor)
        if block_of is not None:
            bo = np.ascontiguousarray(block_of, dtype=np.int32)
            keep.append(bo)
            o.block_of = bo.ctypes.data
        _check(L.mesh_plan_build(arr, n, int(from_size), ctypes.byref(o), ctypes.byref(self._h)),
               "mesh_plan_build")
        self.maps_meta = [(int(m["to_set"]), int(m["to_size"])) for m in maps]

    @classmethod
    def batch(cls, plans) -> "Plan":
        """Fuse HIER plans of several meshes (``mesh_batch_build``)."""
        arr = (ctypes.c_void_p * len(plans))(*[p.handle.value for p in plans])
        h = ctypes.c_void_p()
        _check(lib().mesh_batch_build(arr, len(plans), ctypes.byref(h)), "mesh_batch_build")
        return cls(None, 0, _handle=h)

    @classmethod
    def load(cls, path: str) -> "Plan":
        h = ctypes.c_void_p()
        _check(lib().mesh_plan_load(path.encode(), ctypes.byref(h)), "mesh_plan_load")
        return cls(None, 0, _handle=h)

    def save(self, path: str):
        _check(lib().mesh_plan_save(self._h, path.encode()), "mesh_plan_save")

    @property
    def handle(self):
        return self._h

    def stats(self) -> dict:
        s = mp_plan_stats()
        _check(lib().mesh_plan_query(self._h, ctypes.byref(s)), "mesh_plan_query")
        out = {}
        for name, _ in s._fields_:
            v = getattr(s, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out

    def perm(self, set_id: int) -> np.ndarray:
        """new_to_old permutation of set ``set_id`` (0 = iterations)."""
        st = self.stats()
        if set_id == 0:
            n = st["from_size"]
        else:
            sizes = dict(zip(st["to_set_id"][:st["ntosets"]], st["to_set_size"][:st["ntosets"]]))
            if set_id not in sizes:
                raise MeshLoopError(-1, f"mesh_plan_perm: no set {set_id}")
            n = sizes[set_id]
        out = np.empty(n, dtype=np.int32)
        _check(lib().mesh_plan_perm(self._h, int(set_id), _np_ptr(out)), "mesh_plan_perm")
        return out

    def table(self, name: str, arg: int = 0) -> np.ndarray:
        cnt = ctypes.c_int64(0)
        t = TABLES[name]
        _check(lib().mesh_plan_table(self._h, t, int(arg), None, 0, ctypes.byref(cnt)), "mesh_plan_table")
        out = np.empty(cnt.value, dtype=np.int32)
        _check(lib().mesh_plan_table(self._h, t, int(arg), _np_ptr(out), cnt.value, ctypes.byref(cnt)),
               "mesh_plan_table")
        return out

    def set_staged(self, staged: str | None) -> None:
        """Switch the staged implementation (the tables do not change)."""
        _check(lib().mesh_plan_set_staged(self.handle, STAGED[staged]), "mesh_plan_set_staged")

    def upload(self):
        _check(lib().mesh_plan_upload(self._h), "mesh_plan_upload")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().mesh_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mesh_map_renumber(idx: np.ndarray, from_perm, to_perm, to_size: int) -> np.ndarray:
    """``out[i] = old_to_new_to[idx[from_perm[i]]]`` (C ``mesh_map_renumber``)."""
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    arity = idx.shape[1] if idx.ndim == 2 else 1
    out = np.empty_like(idx)
    fp = None if from_perm is None else np.ascontiguousarray(from_perm, dtype=np.int32)
    tp = None if to_perm is None else np.ascontiguousarray(to_perm, dtype=np.int32)
    _check(lib().mesh_map_renumber(_np_ptr(idx), idx.shape[0], arity, None if fp is None else _np_ptr(fp),
                                   None if tp is None else _np_ptr(tp), int(to_size), _np_ptr(out)),
           "mesh_map_renumber")
    return out


# ------------------------------------------------------------------ loops

def _stream(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_of(*tensors) -> int:
    import torch
    dt = tensors[0].dtype
    for t in tensors:
        if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
            raise MeshLoopError(-1, "tensors must be contiguous CUDA tensors of one dtype")
    if dt == torch.float64:
        return DTYPE["f64"]
    if dt == torch.float32:
        return DTYPE["f32"]
    raise MeshLoopError(-1, f"unsupported dtype {dt}")


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def loop_res_calc(plan: Plan, x, q, adt, res, gam: float = 1.4, eps: float = 0.05, stream=None,
                  compute: str | None = None):
    """``compute="dw"`` selects double-word arithmetic on FP64 data (HIER plans)."""
    dt = _dtype_of(x, q, adt, res)
    if compute == "dw":
        if dt != DTYPE["f64"]:
            raise MeshLoopError(-1, "double-word arithmetic needs float64 data")
        dt = DTYPE["f64dw"]
    _check(lib().loop_res_calc(plan.handle, dt, _ptr(x), _ptr(q), _ptr(adt), _ptr(res), gam, eps,
                               _stream(stream)), "loop_res_calc")


def loop_res_calc_host(plan: Plan, x, q, adt, res, gam: float = 1.4, eps: float = 0.05, stream=None,
                       compute: str | None = None):
    """res_calc on HOST tensors (pinned for asynchronous copies): the library
    copies x, q, adt, res in, runs the loop and copies res back, on
    ``stream``; the result is in ``res`` once the stream has completed."""
    import torch
    dt = x.dtype
    for t in (x, q, adt, res):
        if t.dtype != dt or t.is_cuda or not t.is_contiguous():
            raise MeshLoopError(-1, "tensors must be contiguous host tensors of one dtype")
    if dt == torch.float64:
        code = DTYPE["f64dw"] if compute == "dw" else DTYPE["f64"]
    elif dt == torch.float32 and compute is None:
        code = DTYPE["f32"]
    else:
        raise MeshLoopError(-1, f"unsupported dtype {dt} / compute {compute}")
    _check(lib().loop_res_calc_host(plan.handle, code, _ptr(x), _ptr(q), _ptr(adt), _ptr(res), gam, eps,
                                    _stream(stream)), "loop_res_calc_host")


def loop_bres_calc(plan: Plan, x, q, adt, res, qinf, gam: float = 1.4, eps: float = 0.05, stream=None):
    dt = _dtype_of(x, q, adt, res)
    qi = (ctypes.c_double * 4)(*[float(v) for v in qinf])
    _check(lib().loop_bres_calc(plan.handle, dt, _ptr(x), _ptr(q), _ptr(adt), _ptr(res), qi, gam, eps,
                                _stream(stream)), "loop_bres_calc")


def loop_adt_calc(plan: Plan, x, q, adt, gam: float = 1.4, cfl: float = 0.9, stream=None):
    dt = _dtype_of(x, q, adt)
    _check(lib().loop_adt_calc(plan.handle, dt, _ptr(x), _ptr(q), _ptr(adt), gam, cfl, _stream(stream)),
           "loop_adt_calc")


def loop_save_soln(q, qold, layout: str = "aos", stream=None):
    dt = _dtype_of(q, qold)
    ncell = q.numel() // 4
    _check(lib().loop_save_soln(ncell, dt, LAYOUT[layout], _ptr(q), _ptr(qold), _stream(stream)),
           "loop_save_soln")


def loop_update(qold, q, res, adt, rms, layout: str = "aos", stream=None):
    """rms: a CUDA float64 tensor with one element, incremented by sum d^2."""
    import torch
    dt = _dtype_of(qold, q, res, adt)
    if rms.dtype != torch.float64 or not rms.is_cuda:
        raise MeshLoopError(-1, "rms must be a CUDA float64 tensor")
    _check(lib().loop_update(adt.numel(), dt, LAYOUT[layout], _ptr(qold), _ptr(q), _ptr(res), _ptr(adt),
                             _ptr(rms), _stream(stream)), "loop_update")


def loop_update_noalloc(qold, q, res, adt, rms, layout: str = "aos", stream=None):
    """``loop_update`` without any device allocation: the library's fixed
    static scratch holds the partial sums (at most MP_NOALLOC_MAX_CELLS
    cells; calls that overlap on the GPU must be serialised)."""
    import torch
    dt = _dtype_of(qold, q, res, adt)
    if rms.dtype != torch.float64 or not rms.is_cuda:
        raise MeshLoopError(-1, "rms must be a CUDA float64 tensor")
    _check(lib().loop_update_noalloc(adt.numel(), dt, LAYOUT[layout], _ptr(qold), _ptr(q), _ptr(res), _ptr(adt),
                                     _ptr(rms), _stream(stream)), "loop_update_noalloc")


def loop_elem_assemble(plan: Plan, x, v, sig, f, vol, kappa: float = 0.01, stream=None,
                       compute: str | None = None):
    """``compute="dw"`` selects double-word arithmetic on FP64 data (HIER plans)."""
    dt = _dtype_of(x, v, sig, f, vol)
    if compute == "dw":
        if dt != DTYPE["f64"]:
            raise MeshLoopError(-1, "double-word arithmetic needs float64 data")
        dt = DTYPE["f64dw"]
    _check(lib().loop_elem_assemble(plan.handle, dt, _ptr(x), _ptr(v), _ptr(sig), _ptr(f), _ptr(vol), kappa,
                                    _stream(stream)), "loop_elem_assemble")


def loop_adjoint(plan: Plan, x, q, adt, res_bar, q_bar, x_bar, gam: float = 1.4, eps: float = 0.05,
                 stream=None, compute: str | None = None):
    """``compute="dw"`` selects double-word arithmetic on FP64 data (HIER,
    GLOBAL and ATOMIC plans)."""
    dt = _dtype_of(x, q, adt, res_bar, q_bar, x_bar)
    if compute == "dw":
        if dt != DTYPE["f64"]:
            raise MeshLoopError(-1, "double-word arithmetic needs float64 data")
        dt = DTYPE["f64dw"]
    _check(lib().loop_adjoint(plan.handle, dt, _ptr(x), _ptr(q), _ptr(adt), _ptr(res_bar), _ptr(q_bar),
                              _ptr(x_bar), gam, eps, _stream(stream)), "loop_adjoint")


def loop_space_disc(plan: Plan, edata, eflag, inv_area, res, stream=None):
    """Increment-only edge loop (Volna-style, Sec. 3.1.2); res +=."""
    import torch
    dt = _dtype_of(edata, inv_area, res)
    if eflag.dtype != torch.int32 or not eflag.is_cuda or not eflag.is_contiguous():
        raise MeshLoopError(-1, "eflag must be a contiguous int32 CUDA tensor")
    _check(lib().loop_space_disc(plan.handle, dt, _ptr(edata), _ptr(eflag), _ptr(inv_area), _ptr(res),
                                 _stream(stream)), "loop_space_disc")


def loop_getacc(plan: Plan, cdata, nd, stream=None):
    """Increment-only cell loop (BookLeaf-style, Sec. 3.1.3); nd +=."""
    dt = _dtype_of(cdata, nd)
    _check(lib().loop_getacc(plan.handle, dt, _ptr(cdata), _ptr(nd), _stream(stream)), "loop_getacc")


def loop_face_flux(plan: Plan, fdata, cdata, res, gam: float = 1.4, mu: float = 1e-3, pr: float = 0.72,
                   stream=None, compute: str | None = None):
    """Face flux (miniAero-style, Sec. 3.1.5); res [cells][5] +=.  ``compute="dw"``
    selects double-word arithmetic on FP64 data (HIER plans, block <= 128)."""
    dt = _dtype_of(fdata, cdata, res)
    if compute == "dw":
        if dt != DTYPE["f64"]:
            raise MeshLoopError(-1, "double-word arithmetic needs float64 data")
        dt = DTYPE["f64dw"]
    _check(lib().loop_face_flux(plan.handle, dt, _ptr(fdata), _ptr(cdata), _ptr(res), gam, mu, pr,
                                _stream(stream)), "loop_face_flux")


def mp_check_device_status(stream=None):
    _check(lib().mp_check_device_status(_stream(stream)), "mp_check_device_status")


def mp_grid_wait_test(nctas: int, wait_ns: int, missing: int = 0, stream=None):
    """Diagnostic of the bounded grid-wide wait (``mp_grid_wait_test``)."""
    _check(lib().mp_grid_wait_test(int(nctas), int(wait_ns), int(missing), _stream(stream)), "mp_grid_wait_test")


def mp_recip_test(x, y, mode: int = 0, stream=None):
    """The native FP64 flux kernels' helpers (``mp_recip_test``): mode 0
    y = 1/x, 1 y = 1/(2 x), 2 y = x/2; x, y contiguous float64 CUDA
    tensors."""
    if x.dtype != y.dtype or x.numel() != y.numel() or not (x.is_contiguous() and y.is_contiguous()):
        raise MeshLoopError(-1, "x and y: contiguous tensors of one dtype and size")
    if str(x.dtype) != "torch.float64" or not (x.is_cuda and y.is_cuda):
        raise MeshLoopError(-1, "float64 CUDA tensors expected")
    _check(lib().mp_recip_test(_ptr(x), _ptr(y), int(x.numel()), int(mode), _stream(stream)), "mp_recip_test")

"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Loaded only by ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
and reference legs of ``bench.py``.  It shares no code with the GPU library
(``paper_1802_03749_gb300``) and neither imports the other; both read their
inputs from ``meshgen``.

* ``oracle.c`` (compiled here with gcc, ISO C11, no FP contraction) holds the
  floating-point loops: res_calc, bres_calc, adt_calc, update, the time step,
  hex assembly, the hand-derived adjoint and a complex-step forward loop.
* ``plan.py`` holds plain-Python restatements of the planner's integer
  objects (first-fit colorings, the reverse Cuthill-McKee order, reuse
  factors and plan invariants) for bit-exact comparison.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against closed forms, invariants, brute force or an independent derivative
(see ``tests/test_oracle_*.py``); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

GAMMA = 1.4
EPS = 0.05
CFL = 0.9
KAPPA = 0.01


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so with gcc (no GPU involved)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double


def _declare(L):
    L.oracle_edge_flux.argtypes = [_P, _P, _P, _P, _D, _D, _D, _D, _P]
    L.oracle_res_calc.argtypes = [_I64, _P, _P, _P, _P, _P, _P, _D, _D]
    L.oracle_bres_calc.argtypes = [_I64, _P, _P, _P, _P, _P, _P, _P, _D, _D]
    L.oracle_adt_calc.argtypes = [_I64, _P, _P, _P, _P, _D, _D]
    L.oracle_save_soln.argtypes = [_I64, _P, _P]
    L.oracle_update.argtypes = [_I64, _P, _P, _P, _P, _P]
    L.oracle_step.argtypes = [_I64, _I64, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _D, _D, _D]
    L.oracle_step.restype = _D
    L.oracle_hex_element.argtypes = [_P, _P, _P, _D, _P, _P]
    L.oracle_hex_force.argtypes = [_I64, _P, _P, _P, _P, _P, _P, _D]
    L.oracle_res_calc_adjoint.argtypes = [_I64, _P, _P, _P, _P, _P, _P, _P, _P, _D, _D]
    L.oracle_res_calc_cstep.argtypes = [_I64, _I64, _P, _P, _P, _P, _P, _P, _P, _D, _P, _P, _D, _D]
    L.oracle_space_disc.argtypes = [_I64, _P, _P, _P, _P, _P]
    L.oracle_getacc.argtypes = [_I64, _P, _P, _P]
    L.oracle_face_flux.argtypes = [_I64, _P, _P, _P, _D, _D, _D, _P]


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data


def edge_flux(xa, xb, q1, q2, adt1, adt2, gam=GAMMA, eps=EPS):
    xa, pxa = _f64(xa)
    xb, pxb = _f64(xb)
    q1, pq1 = _f64(q1)
    q2, pq2 = _f64(q2)
    f = np.zeros(4)
    lib().oracle_edge_flux(pxa, pxb, pq1, pq2, float(adt1), float(adt2), gam, eps, f.ctypes.data)
    return f


def res_calc(edge2node, edge2cell, x, q, adt, res=None, gam=GAMMA, eps=EPS):
    """res += interior-edge increments; returns res ([ncell, 4])."""
    e2n, pe2n = _i32(edge2node)
    e2c, pe2c = _i32(edge2cell)
    x, px = _f64(x)
    q, pq = _f64(q)
    adt, padt = _f64(adt)
    if res is None:
        res = np.zeros((q.shape[0], 4))
    assert res.dtype == np.float64 and res.flags.c_contiguous
    lib().oracle_res_calc(e2n.shape[0], pe2n, pe2c, px, pq, padt, res.ctypes.data, gam, eps)
    return res


def bres_calc(bedge2node, bedge2cell, x, q, adt, qinf, res=None, gam=GAMMA, eps=EPS):
    b2n, pb2n = _i32(bedge2node)
    b2c, pb2c = _i32(bedge2cell)
    x, px = _f64(x)
    q, pq = _f64(q)
    adt, padt = _f64(adt)
    qinf, pqi = _f64(qinf)
    if res is None:
        res = np.zeros((q.shape[0], 4))
    lib().oracle_bres_calc(b2n.shape[0], pb2n, pb2c, px, pq, padt, res.ctypes.data, pqi, gam, eps)
    return res


def adt_calc(cell2node, x, q, gam=GAMMA, cfl=CFL):
    c2n, pc2n = _i32(cell2node)
    x, px = _f64(x)
    q, pq = _f64(q)
    adt = np.zeros(q.shape[0])
    lib().oracle_adt_calc(q.shape[0], pc2n, px, pq, adt.ctypes.data, gam, cfl)
    return adt


def update(qold, q, res, adt):
    """In place: q = qold - res/adt, res = 0.  Returns the sum of squared updates."""
    qold, pqo = _f64(qold)
    adt, padt = _f64(adt)
    assert q.dtype == np.float64 and q.flags.c_contiguous and res.flags.c_contiguous
    s = ctypes.c_double(0.0)
    lib().oracle_update(q.shape[0], pqo, q.ctypes.data, res.ctypes.data, padt, ctypes.byref(s))
    return s.value


def step(mesh, q, qinf, gam=GAMMA, eps=EPS, cfl=CFL, work=None):
    """One time step in place on q (save_soln, adt_calc, res_calc, bres_calc,
    update).  Returns (rms, adt, res_before_update_is_zeroed)."""
    assert q.dtype == np.float64 and q.flags.c_contiguous
    nc = q.shape[0]
    if work is None:
        work = {"qold": np.zeros((nc, 4)), "adt": np.zeros(nc), "res": np.zeros((nc, 4))}
    qinf, pqi = _f64(qinf)
    x, px = _f64(mesh.x)
    rms = lib().oracle_step(nc, mesh.nedge, mesh.nbedge, mesh.cell2node.ctypes.data,
                            mesh.edge2node.ctypes.data, mesh.edge2cell.ctypes.data,
                            mesh.bedge2node.ctypes.data, mesh.bedge2cell.ctypes.data, px,
                            q.ctypes.data, work["qold"].ctypes.data, work["adt"].ctypes.data,
                            work["res"].ctypes.data, pqi, gam, eps, cfl)
    return rms, work


def hex_element(xe, ve, sig, kappa=KAPPA):
    xe, pxe = _f64(np.reshape(xe, (8, 3)))
    ve, pve = _f64(np.reshape(ve, (8, 3)))
    sig, psig = _f64(sig)
    fe = np.zeros((8, 3))
    vol = ctypes.c_double(0.0)
    lib().oracle_hex_element(pxe, pve, psig, kappa, fe.ctypes.data, ctypes.byref(vol))
    return fe, vol.value


def hex_force(elem2node, x, v, sig, kappa=KAPPA, f=None):
    e2n, pe2n = _i32(elem2node)
    x, px = _f64(x)
    v, pv = _f64(v)
    sig, psig = _f64(sig)
    if f is None:
        f = np.zeros((x.shape[0], 3))
    vol = np.zeros(e2n.shape[0])
    lib().oracle_hex_force(e2n.shape[0], pe2n, px, pv, psig, f.ctypes.data, vol.ctypes.data, kappa)
    return f, vol


def res_calc_adjoint(edge2node, edge2cell, x, q, adt, res_bar, gam=GAMMA, eps=EPS):
    e2n, pe2n = _i32(edge2node)
    e2c, pe2c = _i32(edge2cell)
    x, px = _f64(x)
    q, pq = _f64(q)
    adt, padt = _f64(adt)
    rb, prb = _f64(res_bar)
    q_bar = np.zeros_like(q)
    x_bar = np.zeros_like(x)
    lib().oracle_res_calc_adjoint(e2n.shape[0], pe2n, pe2c, px, pq, padt, prb, q_bar.ctypes.data,
                                  x_bar.ctypes.data, gam, eps)
    return q_bar, x_bar


def res_calc_cstep(edge2node, edge2cell, x, dx, q, dq, adt, h=1e-30, gam=GAMMA, eps=EPS):
    """(res, J.(dq, dx)) by the complex step of size h."""
    e2n, pe2n = _i32(edge2node)
    e2c, pe2c = _i32(edge2cell)
    x, px = _f64(x)
    dx, pdx = _f64(dx)
    q, pq = _f64(q)
    dq, pdq = _f64(dq)
    adt, padt = _f64(adt)
    re = np.zeros_like(q)
    im = np.zeros_like(q)
    lib().oracle_res_calc_cstep(q.shape[0], e2n.shape[0], pe2n, pe2c, px, pdx, pq, pdq, padt, h,
                                re.ctypes.data, im.ctypes.data, gam, eps)
    return re, im / h


def space_disc(edge2cell, edata, eflag, inv_area, res=None):
    """Volna-style increment-only edge loop (Sec. 3.1.2); res [ncell, 4] +=."""
    e2c, pe = _i32(edge2cell)
    _, pd = _f64(edata)
    _, pf = _i32(eflag)
    ia, pa = _f64(inv_area)
    out = np.zeros((ia.shape[0], 4)) if res is None else np.array(res, dtype=np.float64)
    lib().oracle_space_disc(e2c.shape[0], pe, pd, pf, pa, out.ctypes.data)
    return out


def getacc(cell2node, cdata, nnode, nd=None):
    """BookLeaf-style increment-only cell loop (Sec. 3.1.3); nd [nnode, 4] +=."""
    c2n, pc = _i32(cell2node)
    _, pd = _f64(cdata)
    out = np.zeros((nnode, 4)) if nd is None else np.array(nd, dtype=np.float64)
    lib().oracle_getacc(c2n.shape[0], pc, pd, out.ctypes.data)
    return out


MU, PR = 1e-3, 0.72


def face_flux(face2cell, fdata, cdata, res=None, gam=GAMMA, mu=MU, pr=PR):
    """miniAero-style face flux (Sec. 3.1.5); res [ncell, 5] +=."""
    f2c, pf = _i32(face2cell)
    _, pd = _f64(fdata)
    cd, pc = _f64(cdata)
    out = np.zeros((cd.shape[0], 5)) if res is None else np.array(res, dtype=np.float64)
    lib().oracle_face_flux(f2c.shape[0], pf, pd, pc, gam, mu, pr, out.ctypes.data)
    return out

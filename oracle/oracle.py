"""FP64 CPU oracle for the AutoDiffGeo material map and adjoint gradient.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The product library
never loads it and shares no code with it.

This is a thin ctypes wrapper around ``adg_oracle.c`` (plain C, double
precision, straight loops over every cell x component x primitive).  It takes
the same plain design description (a dict of numpy arrays) that the seeded
input generators produce, and marshals it into its own C struct.

Functions and the passages of arXiv 2311.05646 they follow:

* :func:`sigma`         -- Table "Nonlinear function definitions" (sigma_k)
* :func:`prim`          -- Table "AutoDiffGeo definitions" (one primitive)
* :func:`fill`          -- Eq. eps (the forward composition p_P o ... o p_1)
* :func:`eps`           -- eps = eps_b + (eps_s - eps_b) fill, Sec. 5.1
* :func:`grad`          -- Eq. 1 (eps term) by the reverse sweep of Eqs. AD/jaceps
* :func:`grad_real`     -- the same sweep seeded with a real cotangent dL/deps
* :func:`loss`          -- L = Re sum w E_adj E eps (the scalar whose gradient is Eq. 1)
* :func:`grad_fd`       -- the paper's finite-difference baseline (Sec. 3)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

LOGIC = {"product": 0, "clamp": 1}


def build(force: bool = False) -> str:
    """Compile adg_oracle.c into liboracle.so (gcc, -O2, OpenMP)."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Design(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("ncomp", ctypes.c_int32),
        ("d", ctypes.c_double * 3), ("o", ctypes.c_double * 3), ("off", ctypes.c_double * 9),
        ("eps_bg", ctypes.c_double), ("eps_fg", ctypes.c_double),
        ("logic", ctypes.c_int32), ("nparam", ctypes.c_int32), ("nq", ctypes.c_int32),
        ("nprim", ctypes.c_int32), ("nops", ctypes.c_int32), ("pad_", ctypes.c_int32),
        ("q_base", ctypes.c_void_p), ("q_coeff", ctypes.c_void_p), ("q_param", ctypes.c_void_p),
        ("kind", ctypes.c_void_p), ("sigma", ctypes.c_void_p), ("flags", ctypes.c_void_p),
        ("q0", ctypes.c_void_p), ("nqp", ctypes.c_void_p), ("kr", ctypes.c_void_p),
        ("ops", ctypes.c_void_p),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.od_sigma.restype = ctypes.c_double
            lib.od_sigma.argtypes = [ctypes.c_int, ctypes.c_double, P]
            lib.od_prim.restype = ctypes.c_int
            lib.od_prim.argtypes = [P, ctypes.c_int, P, P, P, P]
            lib.od_validate.restype = ctypes.c_int
            lib.od_validate.argtypes = [P]
            lib.od_fill.restype = ctypes.c_int
            lib.od_fill.argtypes = [P, P, P]
            lib.od_fill_at.restype = ctypes.c_int
            lib.od_fill_at.argtypes = [P, P, ctypes.c_int64, P, P]
            lib.od_grad.restype = ctypes.c_int
            lib.od_grad.argtypes = [P, P, P, P, P, P, P]
            lib.od_grad_real.restype = ctypes.c_int
            lib.od_grad_real.argtypes = [P, P, P, P, P]
            lib.od_loss.restype = ctypes.c_double
            lib.od_loss.argtypes = [P, P, P, P, P]
            lib.od_grad_material.restype = ctypes.c_int
            lib.od_grad_material.argtypes = [P, P, P, P, P, P]
            lib.od_grad_fd.restype = ctypes.c_int
            lib.od_grad_fd.argtypes = [P, P, P, P, P, ctypes.c_double, P]
            lib.od_num_threads.restype = ctypes.c_int
            lib.od_set_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class _Marshalled:
    """Keeps the numpy buffers alive while the C struct points at them."""

    def __init__(self, desc: dict):
        g = desc["grid"]
        self.keep = []

        def arr(x, dt):
            a = np.ascontiguousarray(np.asarray(x, dtype=dt))
            self.keep.append(a)
            return a

        S = _Design()
        S.nx, S.ny, S.nz = (int(v) for v in g["n"])
        S.ncomp = int(g["ncomp"])
        for t in range(3):
            S.d[t] = float(g["d"][t])
            S.o[t] = float(g["o"][t])
        off = np.zeros((3, 3))
        off[: S.ncomp] = np.asarray(g["off"], dtype=np.float64).reshape(S.ncomp, 3)
        for t in range(9):
            S.off[t] = float(off.reshape(-1)[t])
        S.eps_bg = float(desc["eps_bg"])
        S.eps_fg = float(desc["eps_fg"])
        S.logic = LOGIC[desc["logic"]]
        S.nparam = int(len(desc["params"]))
        qb = arr(desc["q_base"], np.float64)
        S.nq = int(qb.size)
        pr = desc["prims"]
        S.nprim = int(len(pr["kind"]))
        ops = arr(desc["ops"], np.int32)
        S.nops = int(ops.size)
        S.q_base = _ptr(qb)
        S.q_coeff = _ptr(arr(desc["q_coeff"], np.float64))
        S.q_param = _ptr(arr(desc["q_param"], np.int32))
        S.kind = _ptr(arr(pr["kind"], np.int32))
        S.sigma = _ptr(arr(pr["sigma"], np.int32))
        S.flags = _ptr(arr(pr["flags"], np.int32))
        S.q0 = _ptr(arr(pr["q0"], np.int32))
        S.nqp = _ptr(arr(pr["nq"], np.int32))
        S.kr = _ptr(arr(pr["kr"], np.float64))
        S.ops = _ptr(ops)
        self.S = S
        self.shape = (S.ncomp, S.nz, S.ny, S.nx)

    @property
    def ref(self):
        return ctypes.byref(self.S)


def _params(desc, params):
    p = desc["params"] if params is None else params
    return np.ascontiguousarray(np.asarray(p, dtype=np.float64))


def set_threads(n: int) -> None:
    _load().od_set_threads(int(n))


def num_threads() -> int:
    return int(_load().od_num_threads())


def sigma(kind: int, u: float):
    """(sigma(u), d sigma / du) of the unit-scale building block."""
    d = ctypes.c_double(0.0)
    s = _load().od_sigma(int(kind), float(u), ctypes.byref(d))
    return s, d.value


def validate(desc: dict) -> int:
    m = _Marshalled(desc)
    return int(_load().od_validate(m.ref))


def q_of(desc: dict, params=None) -> np.ndarray:
    """Geometric scalars q_j = b_j + a_j p[idx_j] (the parameter map)."""
    p = _params(desc, params)
    q = np.asarray(desc["q_base"], dtype=np.float64).copy()
    idx = np.asarray(desc["q_param"])
    a = np.asarray(desc["q_coeff"], dtype=np.float64)
    for j in range(q.size):
        if idx[j] >= 0:
            q[j] += a[j] * p[idx[j]]
    return q


def prim(desc: dict, pi: int, r, params=None):
    """Value and local derivatives of primitive `pi` at physical point r."""
    m = _Marshalled(desc)
    q = q_of(desc, params)
    rr = np.ascontiguousarray(np.asarray(r, dtype=np.float64))
    nq = int(np.asarray(desc["prims"]["nq"])[pi])
    ds = np.zeros(max(nq, 1))
    s = ctypes.c_double(0.0)
    rc = _load().od_prim(m.ref, int(pi), _ptr(q), _ptr(rr), ctypes.byref(s), _ptr(ds))
    if rc:
        raise ValueError("od_prim failed (%d)" % rc)
    return s.value, ds[:nq].copy()


def fill(desc: dict, params=None) -> np.ndarray:
    m = _Marshalled(desc)
    p = _params(desc, params)
    out = np.zeros(m.shape, dtype=np.float64)
    rc = _load().od_fill(m.ref, _ptr(p), _ptr(out))
    if rc:
        raise ValueError("od_fill failed (%d)" % rc)
    return out


def fill_at(desc: dict, flat_idx, params=None) -> np.ndarray:
    m = _Marshalled(desc)
    p = _params(desc, params)
    idx = np.ascontiguousarray(np.asarray(flat_idx, dtype=np.int64))
    out = np.zeros(idx.size, dtype=np.float64)
    rc = _load().od_fill_at(m.ref, _ptr(p), idx.size, _ptr(idx), _ptr(out))
    if rc:
        raise ValueError("od_fill_at failed (%d)" % rc)
    return out


def eps(desc: dict, params=None) -> np.ndarray:
    f = fill(desc, params)
    return desc["eps_bg"] + (desc["eps_fg"] - desc["eps_bg"]) * f


def _field(a, shape):
    a = np.ascontiguousarray(np.asarray(a))
    if a.dtype != np.complex64:
        raise TypeError("fields must be complex64")
    if a.shape != shape:
        raise ValueError("field shape %s != %s" % (a.shape, shape))
    return a


def _w(desc, w):
    C = int(desc["grid"]["ncomp"])
    ww = np.zeros(2 * C, dtype=np.float64)
    wc = np.asarray(w, dtype=np.complex128).reshape(-1)
    if wc.size == 1:
        wc = np.repeat(wc, C)
    ww[0::2] = wc.real[:C]
    ww[1::2] = wc.imag[:C]
    return ww


def grad(desc: dict, efwd, eadj, w, params=None, return_loss: bool = False):
    """g_k = Re sum_c sum_cells w_c E_adj,c E_fwd,c d eps_c / d p_k (Eq. 1)."""
    m = _Marshalled(desc)
    p = _params(desc, params)
    ef = _field(efwd, m.shape)
    ea = _field(eadj, m.shape)
    ww = _w(desc, w)
    g = np.zeros(max(p.size, 1))
    L = ctypes.c_double(0.0)
    rc = _load().od_grad(m.ref, _ptr(p), _ptr(ef), _ptr(ea), _ptr(ww), _ptr(g), ctypes.byref(L))
    if rc:
        raise ValueError("od_grad failed (%d)" % rc)
    g = g[: p.size].copy()
    return (g, L.value) if return_loss else g


def grad_eh(desc_eps: dict, desc_mu: dict, efwd, eadj, w_e, hfwd, hadj, w_h, params=None):
    """Both terms of Eq. 1: the permittivity sweep seeded with E_adj E (Eq.
    jaceps) plus the permeability sweep seeded with H_adj H (Eqs. mu, jacmu),
    over the parameters the two compositions share."""
    return grad(desc_eps, efwd, eadj, w_e, params) + grad(desc_mu, hfwd, hadj, w_h, params)


def grad_real(desc: dict, G, params=None, return_loss: bool = False):
    """g_k = sum_c sum_cells G_c d eps_c / d p_k (real cotangent)."""
    m = _Marshalled(desc)
    p = _params(desc, params)
    GG = np.ascontiguousarray(np.asarray(G, dtype=np.float32))
    if GG.shape != m.shape:
        raise ValueError("G shape %s != %s" % (GG.shape, m.shape))
    g = np.zeros(max(p.size, 1))
    L = ctypes.c_double(0.0)
    rc = _load().od_grad_real(m.ref, _ptr(p), _ptr(GG), _ptr(g), ctypes.byref(L))
    if rc:
        raise ValueError("od_grad_real failed (%d)" % rc)
    g = g[: p.size].copy()
    return (g, L.value) if return_loss else g


def loss(desc: dict, efwd, eadj, w, params=None) -> float:
    m = _Marshalled(desc)
    p = _params(desc, params)
    ef = _field(efwd, m.shape)
    ea = _field(eadj, m.shape)
    return float(_load().od_loss(m.ref, _ptr(p), _ptr(ef), _ptr(ea), _ptr(_w(desc, w))))


def grad_material(desc: dict, efwd, eadj, w, params=None) -> np.ndarray:
    """[dL/d eps_bg, dL/d eps_fg] of L = Re sum w E_adj E_fwd eps (Sec. 5.1)."""
    m = _Marshalled(desc)
    p = _params(desc, params)
    ef = _field(efwd, m.shape)
    ea = _field(eadj, m.shape)
    out = np.zeros(2)
    rc = _load().od_grad_material(m.ref, _ptr(p), _ptr(ef), _ptr(ea), _ptr(_w(desc, w)), _ptr(out))
    if rc:
        raise ValueError("od_grad_material failed (%d)" % rc)
    return out


def grad_fd(desc: dict, efwd, eadj, w, h: float, params=None) -> np.ndarray:
    """Central finite differences of L, one parameter at a time."""
    m = _Marshalled(desc)
    p = _params(desc, params)
    ef = _field(efwd, m.shape)
    ea = _field(eadj, m.shape)
    g = np.zeros(max(p.size, 1))
    rc = _load().od_grad_fd(m.ref, _ptr(p), _ptr(ef), _ptr(ea), _ptr(_w(desc, w)), float(h), _ptr(g))
    if rc:
        raise ValueError("od_grad_fd failed (%d)" % rc)
    return g[: p.size].copy()

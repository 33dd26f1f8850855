"""Thin ctypes binding of libadg (include/adg.h), same names as the C ABI.

Argument marshalling only: every step of the method runs inside libadg's
CUDA kernels.  PyTorch supplies device memory and streams.  If libadg.so is
missing this module raises at import of the first call -- there is no CPU
fallback.

The calls, by the passage of arXiv 2311.05646 they follow:

* ``adg_build_eps``                       -- Eq. eps (step 2 of Sec. 2)
* ``adg_grad`` / ``adg_grad_real``        -- Eq. 1, eps term, by Eqs. AD / jaceps
* ``adg_grad_dense``                      -- the same, plus d/d eps_bg and d/d eps_fg (Sec. 5.1)
* ``adg_grad_eh``                         -- both terms of Eq. 1 (Eqs. mu, jacmu)
* ``adg_levels_eps`` / ``adg_levels_grad``   -- non-binary union (App. B, Alg. 1)
* ``adg_topo_eps`` / ``adg_topo_grad``       -- topology special case (Sec. 3.1)
* ``adg_grad_fd``                         -- the finite-difference baseline (Sec. 3)
* ``adg_mesh_fill`` / ``adg_mesh_grad_fd``   -- Prop. 2's exact mesher and its FD gradient
* ``adg_batch_submit`` / ``poll`` / ``wait`` -- many designs as one job table
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ADG_LIBRARY selects another build of the same library (the ADG_DEBUG build,
# libadg_debug.so, for the bound-check tests)
LIB_PATH = os.environ.get("ADG_LIBRARY") or os.path.join(_HERE, "libadg.so")
_lock = threading.Lock()
_lib = None

ADG_OK, ADG_EINVAL, ADG_ENOMEM, ADG_ECUDA, ADG_ETIMEOUT, ADG_EBUSY, ADG_EDEVICE = range(7)
_STATUS = {0: "ADG_OK", 1: "ADG_EINVAL", 2: "ADG_ENOMEM", 3: "ADG_ECUDA", 4: "ADG_ETIMEOUT",
           5: "ADG_EBUSY", 6: "ADG_EDEVICE"}
LOGIC = {"product": 0, "clamp": 1}


class AdgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class adg_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("ncomp", ctypes.c_int32), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.c_double), ("ox", ctypes.c_double), ("oy", ctypes.c_double),
                ("oz", ctypes.c_double), ("off", (ctypes.c_double * 3) * 3)]


class adg_topo_region(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_int32), ("y0", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("ny", ctypes.c_int32), ("z0", ctypes.c_int32), ("z1", ctypes.c_int32)]


class adg_mesh_layer(ctypes.Structure):
    _fields_ = [("n_polys", ctypes.c_int32), ("vert_off", ctypes.c_void_p),
                ("xy", ctypes.c_void_p), ("bound_z", ctypes.c_int32), ("z0", ctypes.c_double),
                ("z1", ctypes.c_double)]


class adg_design_desc(ctypes.Structure):
    _fields_ = [("grid", adg_grid), ("eps_bg", ctypes.c_double), ("eps_fg", ctypes.c_double),
                ("logic", ctypes.c_int32), ("n_params", ctypes.c_int32), ("n_q", ctypes.c_int32),
                ("n_prims", ctypes.c_int32), ("n_ops", ctypes.c_int32),
                ("reserved", ctypes.c_int32),
                ("q_base", ctypes.c_void_p), ("q_coeff", ctypes.c_void_p),
                ("q_param", ctypes.c_void_p), ("prim_kind", ctypes.c_void_p),
                ("prim_sigma", ctypes.c_void_p), ("prim_flags", ctypes.c_void_p),
                ("prim_q0", ctypes.c_void_p), ("prim_nq", ctypes.c_void_p),
                ("prim_kr", ctypes.c_void_p), ("ops", ctypes.c_void_p)]


class adg_tile_opts(ctypes.Structure):
    _fields_ = [("tx", ctypes.c_int32), ("ty", ctypes.c_int32), ("tz", ctypes.c_int32),
                ("fill_warps", ctypes.c_int32)]


K_NAMES = {0: "bin", 1: "build", 2: "vjp", 3: "finalize", 4: "prepare", 5: "fill", 6: "dense",
           7: "levels"}


class adg_profile_data(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 8), ("ms", ctypes.c_double * 8)]


class adg_stats(ctypes.Structure):
    _fields_ = [("tiles", ctypes.c_int64), ("program_tiles", ctypes.c_int64),
                ("cells", ctypes.c_int64), ("band_cells", ctypes.c_int64),
                ("tile", ctypes.c_int32 * 3), ("max_ops", ctypes.c_int32),
                ("active_samples", ctypes.c_int64)]


def lib():
    """Load libadg.so (fails loudly when it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError("libadg.so not found at %s: run __graft_entry__.build() (nvcc, "
                                  "sm_103a) first; there is no CPU fallback" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            P, I32 = ctypes.c_void_p, ctypes.c_int32
            sig = {
                "adg_ctx_create": [I32, ctypes.POINTER(P)],
                "adg_ctx_destroy": [P],
                "adg_design_create": [P, ctypes.POINTER(adg_design_desc),
                                      ctypes.POINTER(adg_tile_opts), ctypes.POINTER(P)],
                "adg_design_destroy": [P, P],
                "adg_build_eps": [P, P, P, P, P, P],
                "adg_grad": [P, P, P, P, P, P, P, P],
                "adg_grad_real": [P, P, P, P, P, P],
                "adg_grad_dense": [P, P, P, P, P, P, P, P, P, P],
                "adg_sync": [P, P],
                "adg_design_stats": [P, P, P, ctypes.POINTER(adg_stats)],
                "adg_profile_enable": [P, I32],
                "adg_profile_read": [P, ctypes.POINTER(adg_profile_data), I32],
                "adg_grad_fd": [P, P, P, P, P, P, ctypes.c_double, P, P],
                "adg_grad_eh": [P, P, P, P, P, P, P, P, P, P, P, P],
                "adg_levels_eps": [P, P, I32, P, ctypes.c_double, P, P, P],
                "adg_mesh_fill": [P, ctypes.POINTER(adg_grid), ctypes.POINTER(adg_mesh_layer), P,
                                  P, P],
                "adg_mesh_grad_fd": [P, ctypes.POINTER(adg_grid), I32, P, P, P, ctypes.c_double,
                                     ctypes.c_double, P, P, P, P, P],
                "adg_levels_grad": [P, P, I32, P, P, P, P, P, P, P],
                "adg_topo_eps": [P, ctypes.POINTER(adg_grid), ctypes.POINTER(adg_topo_region), P,
                                 ctypes.c_double, ctypes.c_double, P, P],
                "adg_topo_grad": [P, ctypes.POINTER(adg_grid), ctypes.POINTER(adg_topo_region), P,
                                  ctypes.c_double, P, P, P, P, P],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            L.adg_last_error.restype = ctypes.c_char_p
            L.adg_last_error.argtypes = []
            _lib = L
    return _lib


def _check(status):
    if status != ADG_OK:
        raise AdgError(status, lib().adg_last_error().decode())


def adg_last_error() -> str:
    return lib().adg_last_error().decode()


_RAW_STREAM = None  # torch's current-stream query (raw handle) for a device index


def _stream_ptr(stream, device=None):
    """The CUDA stream handle: the given stream, else torch's current stream on
    `device` (the context's device)."""
    global _RAW_STREAM
    if stream is None:
        import torch
        if device is not None:
            if _RAW_STREAM is None:
                _RAW_STREAM = getattr(torch._C, "_cuda_getCurrentRawStream", False)
            if _RAW_STREAM:
                return ctypes.c_void_p(_RAW_STREAM(device))
            return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dptr(t):
    if t is None:
        return ctypes.c_void_p(0)
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device tensors must be contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    def __init__(self, device: int = 0):
        self.handle = ctypes.c_void_p()
        _check(lib().adg_ctx_create(int(device), ctypes.byref(self.handle)))
        self.device = int(device)

    def close(self):
        if self.handle:
            lib().adg_ctx_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Design:
    """A compiled design (adg_design_create) built from a description dict."""

    def __init__(self, ctx: Context, desc: dict, tile=None):
        self.ctx = ctx
        self.desc = desc
        g = desc["grid"]
        self._keep = []

        def arr(x, dt):
            a = np.ascontiguousarray(np.asarray(x, dtype=dt))
            self._keep.append(a)
            return a.ctypes.data_as(ctypes.c_void_p)

        D = adg_design_desc()
        D.grid.nx, D.grid.ny, D.grid.nz = (int(v) for v in g["n"])
        D.grid.ncomp = int(g["ncomp"])
        D.grid.dx, D.grid.dy, D.grid.dz = (float(v) for v in g["d"])
        D.grid.ox, D.grid.oy, D.grid.oz = (float(v) for v in g["o"])
        for c in range(int(g["ncomp"])):
            for a in range(3):
                D.grid.off[c][a] = float(g["off"][c][a])
        D.eps_bg, D.eps_fg = float(desc["eps_bg"]), float(desc["eps_fg"])
        D.logic = LOGIC[desc["logic"]]
        D.n_params = int(len(desc["params"]))
        D.n_q = int(len(desc["q_base"]))
        pr = desc["prims"]
        D.n_prims = int(len(pr["kind"]))
        D.n_ops = int(len(desc["ops"]))
        D.reserved = 0
        D.q_base = arr(desc["q_base"], np.float64)
        D.q_coeff = arr(desc["q_coeff"], np.float64)
        D.q_param = arr(desc["q_param"], np.int32)
        D.prim_kind = arr(pr["kind"], np.int32)
        D.prim_sigma = arr(pr["sigma"], np.int32)
        D.prim_flags = arr(pr["flags"], np.int32)
        D.prim_q0 = arr(pr["q0"], np.int32)
        D.prim_nq = arr(pr["nq"], np.int32)
        D.prim_kr = arr(pr["kr"], np.float64)
        D.ops = arr(desc["ops"], np.int32)
        T = adg_tile_opts(0, 0, 0, 0)
        if tile is not None:  # (tx, ty, tz) or (tx, ty, tz, build fill warps)
            T.tx, T.ty, T.tz = (int(v) for v in tile[:3])
            if len(tile) > 3:
                T.fill_warps = int(tile[3])
        self.handle = ctypes.c_void_p()
        _check(lib().adg_design_create(ctx.handle, ctypes.byref(D), ctypes.byref(T),
                                       ctypes.byref(self.handle)))
        self._keep = []
        self.n_params = D.n_params
        self.ncomp = D.grid.ncomp
        self.shape = (D.grid.ncomp, D.grid.nz, D.grid.ny, D.grid.nx)

    def close(self):
        if self.handle:
            lib().adg_design_destroy(self.ctx.handle, self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _params(design: Design, params):
    p = params
    if not (isinstance(p, np.ndarray) and p.dtype == np.float64 and p.flags.c_contiguous):
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    if p.size != design.n_params:
        raise ValueError("expected %d parameters, got %d" % (design.n_params, p.size))
    return p


def _check_cell_tensor(design, t, name, dtype):
    import torch
    if t.dtype != dtype or tuple(t.shape) != design.shape:
        raise ValueError("%s must be %s of shape %s, got %s %s" % (name, dtype, design.shape,
                                                                    t.dtype, tuple(t.shape)))
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("%s must be a contiguous CUDA tensor" % name)
    del torch


def adg_build_eps(design: Design, params, eps, fill=None, stream=None):
    """eps (and fill, if given) <- the material map at `params` (Eq. eps)."""
    import torch
    p = _params(design, params)
    _check_cell_tensor(design, eps, "eps", torch.float32)
    if fill is not None:
        _check_cell_tensor(design, fill, "fill", torch.float32)
    _check(lib().adg_build_eps(design.ctx.handle, design.handle,
                               ctypes.c_void_p(p.ctypes.data), _dptr(fill), _dptr(eps),
                               _stream_ptr(stream, design.ctx.device)))


def _grad_args(design: Design, efwd, eadj, w, grad):
    import torch
    _check_cell_tensor(design, efwd, "efwd", torch.complex64)
    _check_cell_tensor(design, eadj, "eadj", torch.complex64)
    if grad.dtype != torch.float32 or grad.numel() != design.n_params or not grad.is_cuda:
        raise ValueError("grad must be a float32 CUDA tensor of n_params entries")
    C = design.ncomp
    # component c of a contiguous [C][nz][ny][nx] complex64 tensor starts c planes in
    bf, ba, pb = efwd.data_ptr(), eadj.data_ptr(), 8 * efwd.stride(0)
    ef = (ctypes.c_void_p * 3)(*[bf + c * pb if c < C else 0 for c in range(3)])
    ea = (ctypes.c_void_p * 3)(*[ba + c * pb if c < C else 0 for c in range(3)])
    if isinstance(w, (int, float, complex)):
        wl = [complex(w)] * C
    else:
        wl = [complex(v) for v in np.asarray(w).reshape(-1)]
        if len(wl) == 1:
            wl = wl * C
    ww = (ctypes.c_float * 6)()
    for c in range(C):
        ww[2 * c], ww[2 * c + 1] = wl[c].real, wl[c].imag
    return ef, ea, ww


def adg_grad(design: Design, params, efwd, eadj, w, grad, stream=None):
    """grad <- Re sum w_c E_adj,c E_fwd,c d eps_c / d p (Eq. 1, eps term)."""
    p = _params(design, params)
    ef, ea, ww = _grad_args(design, efwd, eadj, w, grad)
    _check(lib().adg_grad(design.ctx.handle, design.handle, ctypes.c_void_p(p.ctypes.data),
                          ef, ea, ww, _dptr(grad), _stream_ptr(stream, design.ctx.device)))


def adg_grad_eh(d_eps: Design, d_mu: Design, params, efwd, eadj, w_e, hfwd, hadj, w_h, grad,
                stream=None):
    """Both terms of Eq. 1: grad <- Re sum w_e E_adj E d eps/dp (through
    d_eps) + Re sum w_h H_adj H d mu/dp (through d_mu, the permeability
    composition of the same parameters at the H offsets)."""
    if d_mu.n_params != d_eps.n_params:
        raise ValueError("the two designs must share their parameters")
    p = _params(d_eps, params)
    ef, ea, we = _grad_args(d_eps, efwd, eadj, w_e, grad)
    hf, ha, wh = _grad_args(d_mu, hfwd, hadj, w_h, grad)
    _check(lib().adg_grad_eh(d_eps.ctx.handle, d_eps.handle, d_mu.handle,
                             ctypes.c_void_p(p.ctypes.data), ef, ea, we, hf, ha, wh, _dptr(grad),
                             _stream_ptr(stream, d_eps.ctx.device)))


def _level_sets(sets, levels):
    sets = list(sets)
    if not sets:
        raise ValueError("at least one set")
    lv = np.ascontiguousarray(np.asarray(levels, dtype=np.float64).reshape(-1))
    if lv.size != len(sets):
        raise ValueError("one material level per set")
    handles = (ctypes.c_void_p * len(sets))(*[d.handle for d in sets])
    return sets, lv, handles


def adg_levels_eps(sets, levels, eps_bg, params, eps, stream=None):
    """eps <- the union over non-binary material levels (App. B, Alg. 1) of
    the level sets `sets` (Designs, material slots 0 / 1) at `levels`."""
    import torch
    sets, lv, handles = _level_sets(sets, levels)
    p = _params(sets[0], params)
    _check_cell_tensor(sets[0], eps, "eps", torch.float32)
    _check(lib().adg_levels_eps(sets[0].ctx.handle, handles, len(sets),
                                lv.ctypes.data_as(ctypes.c_void_p), float(eps_bg),
                                p.ctypes.data_as(ctypes.c_void_p), _dptr(eps), _stream_ptr(stream)))


def adg_levels_grad(sets, levels, params, efwd, eadj, w, grad, stream=None):
    """grad <- Re sum w E_adj E d eps / dp (Eq. 1, eps term) with eps the map
    of adg_levels_eps."""
    sets, lv, handles = _level_sets(sets, levels)
    p = _params(sets[0], params)
    ef, ea, ww = _grad_args(sets[0], efwd, eadj, w, grad)
    _check(lib().adg_levels_grad(sets[0].ctx.handle, handles, len(sets),
                                 lv.ctypes.data_as(ctypes.c_void_p),
                                 p.ctypes.data_as(ctypes.c_void_p), ef, ea,
                                 ww, _dptr(grad),
                                 _stream_ptr(stream)))


def adg_grad_fd(design: Design, params, efwd, eadj, w, h, grad, stream=None):
    """The finite-difference baseline: grad <- central differences of the
    loss through two builds per parameter (step h), on the GPU."""
    p = _params(design, params)
    ef, ea, ww = _grad_args(design, efwd, eadj, w, grad)
    _check(lib().adg_grad_fd(design.ctx.handle, design.handle, p.ctypes.data_as(ctypes.c_void_p),
                             ef, ea, ww, float(h), _dptr(grad),
                             _stream_ptr(stream)))


def adg_grad_dense(design: Design, params, efwd, eadj, w, fill, grad, gmat, stream=None):
    """The dense form: grad as adg_grad, and gmat (2 float64 on the device)
    <- [dL/d eps_bg, dL/d eps_fg]; every cell's fields and `fill` (the fill at
    the same params) are streamed."""
    import torch
    p = _params(design, params)
    ef, ea, ww = _grad_args(design, efwd, eadj, w, grad)
    _check_cell_tensor(design, fill, "fill", torch.float32)
    if gmat.dtype != torch.float64 or gmat.numel() != 2 or not gmat.is_cuda or not gmat.is_contiguous():
        raise ValueError("gmat must be a contiguous float64 CUDA tensor of 2 entries")
    _check(lib().adg_grad_dense(design.ctx.handle, design.handle, p.ctypes.data_as(ctypes.c_void_p),
                                ef, ea, ww, _dptr(fill),
                                _dptr(grad), _dptr(gmat), _stream_ptr(stream)))


def adg_grad_real(design: Design, params, G, grad, stream=None):
    """grad <- sum G_c d eps_c / d p (real cotangent, the autograd form)."""
    import torch
    p = _params(design, params)
    _check_cell_tensor(design, G, "G", torch.float32)
    if grad.dtype != torch.float32 or grad.numel() != design.n_params or not grad.is_cuda:
        raise ValueError("grad must be a float32 CUDA tensor of n_params entries")
    _check(lib().adg_grad_real(design.ctx.handle, design.handle, p.ctypes.data_as(ctypes.c_void_p),
                               _dptr(G), _dptr(grad), _stream_ptr(stream)))


def adg_sync(ctx: Context, stream=None):
    _check(lib().adg_sync(ctx.handle, _stream_ptr(stream)))


def adg_design_stats(design: Design, stream=None) -> dict:
    s = adg_stats()
    _check(lib().adg_design_stats(design.ctx.handle, design.handle, _stream_ptr(stream),
                                  ctypes.byref(s)))
    return {"tiles": s.tiles, "program_tiles": s.program_tiles, "cells": s.cells,
            "band_cells": s.band_cells, "tile": tuple(s.tile), "max_ops": s.max_ops,
            "active_samples": s.active_samples}


def adg_profile_enable(ctx: Context, on: bool = True):
    _check(lib().adg_profile_enable(ctx.handle, 1 if on else 0))


def adg_profile_read(ctx: Context, reset: bool = True) -> dict:
    """{kernel name: (launches, total ms)} of the launches recorded while enabled."""
    d = adg_profile_data()
    _check(lib().adg_profile_read(ctx.handle, ctypes.byref(d), 1 if reset else 0))
    return {K_NAMES[k]: (int(d.launches[k]), float(d.ms[k])) for k in K_NAMES}


def adg_grad_noalloc(desc: dict, params, efwd, eadj, w, grad, tile=None, stream=None):
    """The Eq. 1 gradient without any allocation: for callers that cannot
    call cudaMalloc (a fixed device-memory arena owned by another runtime, a
    plug-in that must not grow its footprint, a strict budget).  It takes the
    design description directly, keeps all device scratch in libadg's static
    32 MiB array, and returns once the result is in `grad`.  Calls share that
    array: do not let two of them overlap on the GPU."""
    import torch
    keep = []

    def arr(x, dt):
        a = np.ascontiguousarray(np.asarray(x, dtype=dt))
        keep.append(a)
        return a.ctypes.data_as(ctypes.c_void_p)

    g = desc["grid"]
    D = adg_design_desc()
    D.grid.nx, D.grid.ny, D.grid.nz = (int(v) for v in g["n"])
    C = int(g["ncomp"])
    D.grid.ncomp = C
    D.grid.dx, D.grid.dy, D.grid.dz = (float(v) for v in g["d"])
    D.grid.ox, D.grid.oy, D.grid.oz = (float(v) for v in g["o"])
    for c in range(C):
        for a in range(3):
            D.grid.off[c][a] = float(g["off"][c][a])
    D.eps_bg, D.eps_fg = float(desc["eps_bg"]), float(desc["eps_fg"])
    D.logic = LOGIC[desc["logic"]]
    D.n_params = int(len(desc["params"]))
    D.n_q = int(len(desc["q_base"]))
    pr = desc["prims"]
    D.n_prims = int(len(pr["kind"]))
    D.n_ops = int(len(desc["ops"]))
    D.reserved = 0
    D.q_base = arr(desc["q_base"], np.float64)
    D.q_coeff = arr(desc["q_coeff"], np.float64)
    D.q_param = arr(desc["q_param"], np.int32)
    D.prim_kind = arr(pr["kind"], np.int32)
    D.prim_sigma = arr(pr["sigma"], np.int32)
    D.prim_flags = arr(pr["flags"], np.int32)
    D.prim_q0 = arr(pr["q0"], np.int32)
    D.prim_nq = arr(pr["nq"], np.int32)
    D.prim_kr = arr(pr["kr"], np.float64)
    D.ops = arr(desc["ops"], np.int32)
    T = adg_tile_opts(0, 0, 0, 0)
    if tile is not None:
        T.tx, T.ty, T.tz = (int(v) for v in tile[:3])
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    if p.size != D.n_params:
        raise ValueError("expected %d parameters, got %d" % (D.n_params, p.size))
    shape = (C, D.grid.nz, D.grid.ny, D.grid.nx)
    for t, name in ((efwd, "efwd"), (eadj, "eadj")):
        if t.dtype != torch.complex64 or tuple(t.shape) != shape or not t.is_cuda:
            raise ValueError("%s must be a complex64 CUDA tensor of shape %s" % (name, shape))
    if grad.dtype != torch.float32 or grad.numel() != D.n_params or not grad.is_cuda:
        raise ValueError("grad must be a float32 CUDA tensor of n_params entries")
    ef = (ctypes.c_void_p * 3)(*[efwd[c].data_ptr() if c < C else 0 for c in range(3)])
    ea = (ctypes.c_void_p * 3)(*[eadj[c].data_ptr() if c < C else 0 for c in range(3)])
    wc = np.asarray(w, dtype=np.complex128).reshape(-1)
    if wc.size == 1:
        wc = np.repeat(wc, C)
    ww = np.zeros(6, dtype=np.float32)
    ww[0:2 * C:2] = wc.real[:C]
    ww[1:2 * C:2] = wc.imag[:C]
    L = lib()
    f = L.adg_grad_noalloc
    f.argtypes = [ctypes.POINTER(adg_design_desc), ctypes.POINTER(adg_tile_opts),
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    _check(f(ctypes.byref(D), ctypes.byref(T), p.ctypes.data_as(ctypes.c_void_p), ef, ea,
             ww.ctypes.data_as(ctypes.c_void_p), _dptr(grad), _stream_ptr(stream)))


def adg_design_bytes(design: Design) -> int:
    """Device bytes the design holds (tables, bins, partial buffer, scratch of
    the optional calls); the caller's own buffers are not included."""
    b = ctypes.c_int64(0)
    L = lib()
    L.adg_design_bytes.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]
    L.adg_design_bytes.restype = ctypes.c_int
    _check(L.adg_design_bytes(design.ctx.handle, design.handle, ctypes.byref(b)))
    return int(b.value)


def adg_debug_alloc(fail_after: int = -2) -> int:
    """Host-side fault injection for tests: let `fail_after` more of libadg's
    allocations succeed and fail the next (-1: off, -2: unchanged).  Returns
    the number of allocations libadg holds now."""
    live = ctypes.c_int64(0)
    L = lib()
    L.adg_debug_alloc.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]
    L.adg_debug_alloc.restype = ctypes.c_int
    _check(L.adg_debug_alloc(int(fail_after), ctypes.byref(live)))
    return int(live.value)


BATCH_BUILD, BATCH_GRAD, BATCH_GRAD_REAL = 1, 2, 4
BATCH_GRAPH = 1


class adg_batch_item(ctypes.Structure):
    _fields_ = [("design", ctypes.c_void_p), ("ops", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("h_params", ctypes.c_void_p), ("d_fill", ctypes.c_void_p),
                ("d_eps", ctypes.c_void_p), ("d_efwd", ctypes.c_void_p * 3),
                ("d_eadj", ctypes.c_void_p * 3), ("w", ctypes.c_float * 6),
                ("d_G", ctypes.c_void_p), ("d_grad", ctypes.c_void_p)]


class BatchItem:
    """One (design, operations) entry of a batch; tensors are CUDA tensors
    shaped like the single-design calls."""

    def __init__(self, design: Design, params, eps=None, fill=None, efwd=None, eadj=None, w=None,
                 G=None, grad=None):
        self.design, self.params = design, np.ascontiguousarray(np.asarray(params, np.float64))
        self.eps, self.fill, self.efwd, self.eadj, self.w, self.G, self.grad = (
            eps, fill, efwd, eadj, w, G, grad)


def adg_batch_submit(ctx: Context, items, graph: bool = False, stream=None) -> int:
    """Enqueue all items as one job table (five launches); returns a ticket."""
    import torch
    arr = (adg_batch_item * len(items))()
    keep = []
    for k, it in enumerate(items):
        d = it.design
        if it.params.size != d.n_params:
            raise ValueError("item %d: expected %d parameters" % (k, d.n_params))
        e = arr[k]
        e.design = d.handle
        ops = 0
        keep.append(it.params)
        e.h_params = it.params.ctypes.data_as(ctypes.c_void_p)
        if it.eps is not None:
            _check_cell_tensor(d, it.eps, "eps", torch.float32)
            ops |= BATCH_BUILD
            e.d_eps = _dptr(it.eps)
            if it.fill is not None:
                _check_cell_tensor(d, it.fill, "fill", torch.float32)
                e.d_fill = _dptr(it.fill)
        if it.efwd is not None:
            _check_cell_tensor(d, it.efwd, "efwd", torch.complex64)
            _check_cell_tensor(d, it.eadj, "eadj", torch.complex64)
            ops |= BATCH_GRAD
            # component c of a contiguous [C][nz][ny][nx] complex64 tensor starts c planes in
            bf, ba, pb = it.efwd.data_ptr(), it.eadj.data_ptr(), 8 * it.efwd.stride(0)
            for c in range(d.ncomp):
                e.d_efwd[c] = bf + c * pb
                e.d_eadj[c] = ba + c * pb
            if isinstance(it.w, (int, float, complex)):
                wl = [complex(it.w)] * d.ncomp
            else:
                wl = [complex(v) for v in np.asarray(it.w).reshape(-1)]
                if len(wl) == 1:
                    wl = wl * d.ncomp
            for c in range(d.ncomp):
                e.w[2 * c] = wl[c].real
                e.w[2 * c + 1] = wl[c].imag
        elif it.G is not None:
            _check_cell_tensor(d, it.G, "G", torch.float32)
            ops |= BATCH_GRAD_REAL
            e.d_G = _dptr(it.G)
        if ops & (BATCH_GRAD | BATCH_GRAD_REAL):
            if it.grad is None or it.grad.dtype != torch.float32 or it.grad.numel() != d.n_params:
                raise ValueError("item %d: grad must be float32 with n_params entries" % k)
            e.d_grad = _dptr(it.grad)
        e.ops = ops
    f = _batch_fns().adg_batch_submit
    t = ctypes.c_uint64(0)
    _check(f(ctx.handle, arr, len(items), BATCH_GRAPH if graph else 0,
             _stream_ptr(stream, ctx.device), ctypes.byref(t)))
    return int(t.value)


_BATCH_L = None


def _batch_fns():
    """The library with the batch calls' signatures set (once)."""
    global _BATCH_L
    if _BATCH_L is None:
        L = lib()
        L.adg_batch_submit.argtypes = [ctypes.c_void_p, ctypes.POINTER(adg_batch_item),
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_uint64)]
        L.adg_batch_submit.restype = ctypes.c_int
        L.adg_batch_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32)]
        L.adg_batch_poll.restype = ctypes.c_int
        L.adg_batch_wait.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64]
        L.adg_batch_wait.restype = ctypes.c_int
        _BATCH_L = L
    return _BATCH_L


def adg_batch_poll(ctx: Context, ticket: int) -> bool:
    done = ctypes.c_int32(0)
    _check(_batch_fns().adg_batch_poll(ctx.handle, ticket, ctypes.byref(done)))
    return bool(done.value)


def adg_batch_wait(ctx: Context, ticket: int, timeout_s: float = 60.0) -> None:
    """Wait for a batch; raises AdgError(ADG_ETIMEOUT) when it is still running."""
    _check(_batch_fns().adg_batch_wait(ctx.handle, ticket, int(timeout_s * 1e9)))


# ------------------------------------------------------- topology (Sec. 3.1) --
def _topo_grid(n, ncomp):
    G = adg_grid()
    G.nx, G.ny, G.nz = (int(v) for v in n)
    G.ncomp = int(ncomp)
    return G


def _topo_region(region):
    R = adg_topo_region()
    R.x0, R.y0, R.nx, R.ny, R.z0, R.z1 = (int(v) for v in region)
    return R


def _topo_v(v, region, name="v"):
    import torch
    n = int(region[2]) * int(region[3])
    if v.dtype != torch.float32 or v.numel() != n or not v.is_cuda or not v.is_contiguous():
        raise ValueError("%s must be a contiguous float32 CUDA tensor of %d entries" % (name, n))


def adg_topo_eps(ctx: Context, n, ncomp, region, v, eps_l, deps, eps, stream=None):
    """eps (ncomp, nz, ny, nx) <- eps_l + deps sigmoid(v) over the region
    (x0, y0, nx, ny, z0, z1), broadcast along z (Eq. TO_example)."""
    import torch
    _topo_v(v, region)
    shape = (int(ncomp), int(n[2]), int(n[1]), int(n[0]))
    if eps.dtype != torch.float32 or tuple(eps.shape) != shape or not eps.is_cuda or not eps.is_contiguous():
        raise ValueError("eps must be a contiguous float32 CUDA tensor of shape %s" % (shape,))
    G, R = _topo_grid(n, ncomp), _topo_region(region)
    _check(lib().adg_topo_eps(ctx.handle, ctypes.byref(G), ctypes.byref(R), _dptr(v), float(eps_l),
                              float(deps), _dptr(eps), _stream_ptr(stream)))


def adg_topo_grad(ctx: Context, n, ncomp, region, v, deps, efwd, eadj, w, grad, stream=None):
    """grad (per pixel) <- deps sigmoid'(v) sum_c sum_z Re(w_c E_adj,c E_fwd,c)
    over the region (Eq. top_AD)."""
    import torch
    _topo_v(v, region)
    _topo_v(grad, region, "grad")
    C = int(ncomp)
    shape = (C, int(n[2]), int(n[1]), int(n[0]))
    for t, name in ((efwd, "efwd"), (eadj, "eadj")):
        if t.dtype != torch.complex64 or tuple(t.shape) != shape or not t.is_cuda or not t.is_contiguous():
            raise ValueError("%s must be a contiguous complex64 CUDA tensor of shape %s" % (name, shape))
    ef = (ctypes.c_void_p * 3)(*[efwd[c].data_ptr() if c < C else 0 for c in range(3)])
    ea = (ctypes.c_void_p * 3)(*[eadj[c].data_ptr() if c < C else 0 for c in range(3)])
    wc = np.asarray(w, dtype=np.complex128).reshape(-1)
    if wc.size == 1:
        wc = np.repeat(wc, C)
    ww = np.zeros(6, dtype=np.float32)
    ww[0:2 * C:2] = wc.real[:C]
    ww[1:2 * C:2] = wc.imag[:C]
    G, R = _topo_grid(n, ncomp), _topo_region(region)
    _check(lib().adg_topo_grad(ctx.handle, ctypes.byref(G), ctypes.byref(R), _dptr(v), float(deps),
                               ef, ea, ww.ctypes.data_as(ctypes.c_void_p), _dptr(grad),
                               _stream_ptr(stream)))


# ---- the exact polygon mesher (Prop. 2) and its FD gradient ------------------
def _grid_struct(grid: dict):
    G = adg_grid()
    G.nx, G.ny, G.nz = (int(v) for v in grid["n"])
    G.ncomp = int(grid["ncomp"])
    G.dx, G.dy, G.dz = (float(v) for v in grid["d"])
    G.ox, G.oy, G.oz = (float(v) for v in grid["o"])
    for c, row in enumerate(grid["off"][:3]):
        for a in range(3):
            G.off[c][a] = float(row[a])
    return G


def _layer_struct(layer: dict, keep: list):
    """{"polys": [(N, 2) vertices], "z": (z0, z1) or None} -> adg_mesh_layer;
    the arrays it points to are appended to `keep`."""
    polys = [np.ascontiguousarray(np.asarray(p, dtype=np.float64).reshape(-1, 2))
             for p in layer["polys"]]
    off = np.zeros(len(polys) + 1, dtype=np.int32)
    off[1:] = np.cumsum([p.shape[0] for p in polys])
    xy = np.ascontiguousarray(np.concatenate(polys) if polys else np.zeros((0, 2)))
    keep += [off, xy]
    L = adg_mesh_layer()
    L.n_polys = len(polys)
    L.vert_off = off.ctypes.data_as(ctypes.c_void_p)
    L.xy = xy.ctypes.data_as(ctypes.c_void_p)
    z = layer.get("z")
    L.bound_z = 0 if z is None else 1
    L.z0, L.z1 = (0.0, 0.0) if z is None else (float(z[0]), float(z[1]))
    return L


def _field_ptrs(grid: dict, efwd, eadj, w):
    import torch
    nx, ny, nz = (int(v) for v in grid["n"])
    C = int(grid["ncomp"])
    for t, name in ((efwd, "efwd"), (eadj, "eadj")):
        if (t.dtype != torch.complex64 or tuple(t.shape) != (C, nz, ny, nx) or not t.is_cuda
                or not t.is_contiguous()):
            raise ValueError("%s must be a contiguous complex64 CUDA tensor of shape %s"
                             % (name, (C, nz, ny, nx)))
    ef = (ctypes.c_void_p * 3)(*[efwd[c].data_ptr() if c < C else 0 for c in range(3)])
    ea = (ctypes.c_void_p * 3)(*[eadj[c].data_ptr() if c < C else 0 for c in range(3)])
    wc = np.asarray(w, dtype=np.complex128).reshape(-1)
    if wc.size == 1:
        wc = np.repeat(wc, C)
    ww = np.zeros(6, dtype=np.float32)
    ww[0:2 * C:2] = wc.real[:C]
    ww[1:2 * C:2] = wc.imag[:C]
    return ef, ea, ww


def adg_mesh_fill(ctx: Context, grid: dict, layer: dict, fill, region=None, stream=None):
    """fill (ncomp, nz, ny, nx) <- the exact volume-averaged fill of a polygon
    layer (Prop. 2's standard representation) over `region` (x0, y0, nx, ny,
    z0, z1; None: the whole grid)."""
    import torch
    nx, ny, nz = (int(v) for v in grid["n"])
    shape = (int(grid["ncomp"]), nz, ny, nx)
    if (fill.dtype != torch.float32 or tuple(fill.shape) != shape or not fill.is_cuda
            or not fill.is_contiguous()):
        raise ValueError("fill must be a contiguous float32 CUDA tensor of shape %s" % (shape,))
    keep = []
    G, L = _grid_struct(grid), _layer_struct(layer, keep)
    R = ctypes.byref(_topo_region(region)) if region is not None else None
    _check(lib().adg_mesh_fill(ctx.handle, ctypes.byref(G), ctypes.byref(L), R, _dptr(fill),
                               _stream_ptr(stream)))


class MeshLayers:
    """A list of polygon layers marshalled once into an adg_mesh_layer array
    (the arrays it points to are kept alive with it)."""

    def __init__(self, layers):
        self._keep = []
        self.n = len(layers)
        self.array = (adg_mesh_layer * max(self.n, 1))(*[_layer_struct(l, self._keep)
                                                          for l in layers])

    def __len__(self):
        return self.n


def adg_mesh_grad_fd(ctx: Context, grid: dict, plus, minus, regions, h, deps, efwd, eadj, w, grad,
                     stream=None):
    """The finite-difference gradient with the exact mesher: plus[k] / minus[k]
    are the layer at p +- h e_k (lists of layer dicts, or MeshLayers),
    regions[k] (or None) where they can differ."""
    import torch
    plus = plus if isinstance(plus, MeshLayers) else MeshLayers(plus)
    minus = minus if isinstance(minus, MeshLayers) else MeshLayers(minus)
    n = len(plus)
    if len(minus) != n or (regions is not None and len(regions) != n):
        raise ValueError("one plus layer, minus layer and region per parameter")
    if grad.dtype != torch.float32 or grad.numel() != n or not grad.is_cuda:
        raise ValueError("grad must be a float32 CUDA tensor of n_params entries")
    G = _grid_struct(grid)
    rr = None
    if regions is not None:
        rr = (adg_topo_region * max(n, 1))(*[_topo_region(r) for r in regions])
    ef, ea, ww = _field_ptrs(grid, efwd, eadj, w)
    _check(lib().adg_mesh_grad_fd(ctx.handle, ctypes.byref(G), n, plus.array, minus.array, rr,
                                  float(h), float(deps), ef, ea,
                                  ww.ctypes.data_as(ctypes.c_void_p), _dptr(grad),
                                  _stream_ptr(stream)))

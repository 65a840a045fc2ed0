"""Thin ctypes binding of libwavetile (include/wave.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device buffers are torch CUDA tensors (float32, contiguous); point
coordinates are host arrays.  The library is required: importing the
functions below on a machine without the built library raises instead of
falling back to anything else.
"""
import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

WAVE_OK = 0
WAVE_EINVAL = -1
WAVE_EUNSTABLE = -2
WAVE_ECUDA = -3
WAVE_ETIMEOUT = -4
WAVE_ENOSPACE = -5
WAVE_EUNSUPPORTED = -6
WAVE_OP_FWD, WAVE_OP_ADJ, WAVE_OP_GRAD, WAVE_OP_REVOLVE, WAVE_OP_BORN = 0, 1, 2, 3, 4
WAVE_ALLOW_UNSTABLE = 1
WAVE_TIME_SWEEPS = 2
WAVE_AUTOTUNE_SHAPE = 4
WAVE_BORN_TWO_SWEEPS = 8
WAVE_TEST_WITHHOLD = 256
WAVE_KERNEL_SHARED, WAVE_KERNEL_STAGED = 1, 2
WAVE_NOALLOC_MAX_BYTES = 32 * 1024 * 1024

EXPORTED = ["wave_version", "wave_strerror", "wave_fd_coefficients", "wave_cfl_dt",
            "wave_workspace_bytes", "wave_ckpt_bytes", "wave_fwd", "wave_adj", "wave_grad",
            "wave_status", "wave_describe_plan", "wave_sweep_stats", "wave_list_variants",
            "wave_autotune_stats", "wave_plan_bound",
            "wave_fwd_noalloc", "wave_measure_peaks", "wave_batch_workspace_bytes",
            "wave_fwd_batched", "wave_grad_batched", "wave_describe_batch_plan", "wave_heat",
            "wave_grad_revolve", "wave_revolve_forward_steps", "wave_revolve_schedule", "wave_born",
            "wave_heat_ab2", "wave_describe_grad_plan"]


class WaveError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, _lib().wave_strerror(code).decode(), code))


class _Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("h", ctypes.c_float * 3), ("dt", ctypes.c_float),
                ("nt", ctypes.c_int32), ("space_order", ctypes.c_int32)]


class _Points(ctypes.Structure):
    _fields_ = [("npts", ctypes.c_int32), ("xyz", ctypes.POINTER(ctypes.c_float))]


class _Shot(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_int32 * 3), ("n", ctypes.c_int32 * 3), ("src", _Points),
                ("rec", _Points)]


class _Tuning(ctypes.Structure):
    _fields_ = [("time_tile", ctypes.c_int32), ("tile_y", ctypes.c_int32),
                ("tile_x", ctypes.c_int32), ("vec", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("tile_z", ctypes.c_int32), ("kernel", ctypes.c_int32), ("rows", ctypes.c_int32)]


@dataclass
class Grid:
    """Grid shape (nx, ny, nz), spacing h (km), dt (s), nt steps, space order."""
    n: tuple
    h: tuple
    dt: float
    nt: int
    space_order: int

    def c(self):
        g = _Grid()
        g.n[:] = [int(v) for v in self.n]
        g.h[:] = [float(v) for v in self.h]
        g.dt = float(self.dt)
        g.nt = int(self.nt)
        g.space_order = int(self.space_order)
        return g


@dataclass
class Tuning:
    """time_tile: 0 autotune, 1 untiled, T >= 2 time-tile depth; tile_y, vec
    (z points per thread), tile_z, kernel (WAVE_KERNEL_SHARED / _STAGED) and
    rows (rows per thread) pick a compiled variant, tile_x its x-chunk."""
    time_tile: int = 0
    tile_y: int = 0
    tile_x: int = 0
    flags: int = 0
    vec: int = 0
    tile_z: int = 0
    kernel: int = 0
    rows: int = 0

    def c(self):
        return _Tuning(int(self.time_tile), int(self.tile_y), int(self.tile_x), int(self.vec),
                       int(self.flags), int(self.tile_z), int(self.kernel), int(self.rows))


_LIB = None


def library_path():
    return _build.LIB


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libwavetile is not built (%s); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
        lib = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        i32 = ctypes.c_int32
        gp = ctypes.POINTER(_Grid)
        pp = ctypes.POINTER(_Points)
        tp = ctypes.POINTER(_Tuning)
        lib.wave_version.restype = i32
        lib.wave_strerror.argtypes = [i32]
        lib.wave_strerror.restype = ctypes.c_char_p
        lib.wave_fd_coefficients.argtypes = [i32, ctypes.POINTER(ctypes.c_double)]
        lib.wave_fd_coefficients.restype = i32
        lib.wave_cfl_dt.argtypes = [i32, ctypes.POINTER(ctypes.c_float), ctypes.c_float]
        lib.wave_cfl_dt.restype = ctypes.c_double
        lib.wave_workspace_bytes.argtypes = [gp, i32, i32, i32, i32, tp]
        lib.wave_workspace_bytes.restype = ctypes.c_size_t
        lib.wave_ckpt_bytes.argtypes = [gp, i32]
        lib.wave_ckpt_bytes.restype = ctypes.c_size_t
        lib.wave_fwd.argtypes = [gp, vp, vp, pp, vp, pp, vp, vp, vp, i32, tp, vp, ctypes.c_size_t, vp]
        lib.wave_fwd.restype = i32
        lib.wave_adj.argtypes = [gp, vp, vp, pp, vp, pp, vp, vp, tp, vp, ctypes.c_size_t, vp]
        lib.wave_adj.restype = i32
        lib.wave_grad.argtypes = [gp, vp, vp, pp, vp, pp, vp, vp, i32, vp, tp, vp, ctypes.c_size_t, vp]
        lib.wave_grad.restype = i32
        lib.wave_born.argtypes = [gp, vp, vp, vp, pp, vp, pp, vp, vp, tp, vp, ctypes.c_size_t, vp]
        lib.wave_born.restype = i32
        lib.wave_grad_revolve.argtypes = [gp, vp, vp, pp, vp, pp, vp, i32, vp, tp, vp, ctypes.c_size_t, vp]
        lib.wave_grad_revolve.restype = i32
        lib.wave_revolve_forward_steps.argtypes = [i32, i32]
        lib.wave_revolve_forward_steps.restype = ctypes.c_int64
        lib.wave_revolve_schedule.argtypes = [i32, i32, ctypes.POINTER(i32), i32]
        lib.wave_revolve_schedule.restype = i32
        lib.wave_heat.argtypes = [gp, vp, vp, pp, vp, pp, vp, vp, tp, vp, ctypes.c_size_t, vp]
        lib.wave_heat_ab2.argtypes = [gp, vp, vp, pp, vp, pp, vp, vp, tp, vp, ctypes.c_size_t, vp]
        lib.wave_heat_ab2.restype = i32
        lib.wave_heat.restype = i32
        lib.wave_status.argtypes = [vp, vp]
        lib.wave_status.restype = i32
        lib.wave_describe_plan.argtypes = [gp, tp, ctypes.POINTER(i32)]
        lib.wave_describe_plan.restype = i32
        lib.wave_describe_grad_plan.argtypes = [gp, tp, i32, i32, i32, ctypes.POINTER(i32)]
        lib.wave_describe_grad_plan.restype = i32
        lib.wave_sweep_stats.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i32),
                                         ctypes.POINTER(i32)]
        lib.wave_sweep_stats.restype = i32
        lib.wave_autotune_stats.argtypes = [ctypes.POINTER(i32), ctypes.POINTER(i32)]
        lib.wave_autotune_stats.restype = i32
        lib.wave_plan_bound.argtypes = [gp, tp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.POINTER(ctypes.c_double)]
        lib.wave_plan_bound.restype = i32
        lib.wave_list_variants.argtypes = [i32, ctypes.POINTER(i32), i32]
        lib.wave_list_variants.restype = i32
        lib.wave_fwd_noalloc.argtypes = [gp, vp, vp, pp, vp, pp, vp, vp, tp, vp, ctypes.POINTER(i32)]
        lib.wave_fwd_noalloc.restype = i32
        lib.wave_measure_peaks.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp]
        lib.wave_measure_peaks.restype = i32
        sp_ = ctypes.POINTER(_Shot)
        lib.wave_batch_workspace_bytes.argtypes = [gp, i32, sp_, i32, i32]
        lib.wave_batch_workspace_bytes.restype = ctypes.c_size_t
        lib.wave_describe_batch_plan.argtypes = [gp, i32, sp_, i32, i32, tp, ctypes.POINTER(i32)]
        lib.wave_describe_batch_plan.restype = i32
        lib.wave_fwd_batched.argtypes = [gp, i32, sp_, vp, vp, vp, vp, i32, tp, vp, ctypes.c_size_t, vp]
        lib.wave_fwd_batched.restype = i32
        lib.wave_grad_batched.argtypes = [gp, i32, sp_, vp, vp, vp, vp, i32, vp, i32, tp, vp,
                                          ctypes.c_size_t, vp]
        lib.wave_grad_batched.restype = i32
        _LIB = lib
    return _LIB


def _check(code, what):
    if code != WAVE_OK:
        raise WaveError(code, what)


def fd_coefficients(space_order):
    out = (ctypes.c_double * (space_order // 2 + 1))()
    _check(_lib().wave_fd_coefficients(int(space_order), out), "wave_fd_coefficients")
    return np.array(list(out))


def cfl_dt(space_order, h, v_max):
    hh = (ctypes.c_float * 3)(*[float(v) for v in h])
    return float(_lib().wave_cfl_dt(int(space_order), hh, float(v_max)))


def workspace_bytes(grid, op, nsrc, nrec, ckpt_every=0, tuning=None):
    g = grid.c()
    t = tuning.c() if tuning is not None else None
    return int(_lib().wave_workspace_bytes(ctypes.byref(g), int(op), int(nsrc), int(nrec),
                                           int(ckpt_every), ctypes.byref(t) if t is not None else None))


def ckpt_bytes(grid, ckpt_every):
    g = grid.c()
    return int(_lib().wave_ckpt_bytes(ctypes.byref(g), int(ckpt_every)))


def list_variants(space_order):
    """Compiled sweep variants: dicts with time_tile, tile_y, tile_z, vec,
    prefetch, threads."""
    n = _lib().wave_list_variants(int(space_order), None, 0)
    if n < 0:
        raise WaveError(n, "wave_list_variants")
    out = (ctypes.c_int32 * (8 * max(n, 1)))()
    _lib().wave_list_variants(int(space_order), out, n)
    keys = ("time_tile", "tile_y", "tile_z", "vec", "prefetch", "threads", "kernel", "rows")
    return [dict(zip(keys, out[8 * i:8 * i + 8])) for i in range(n)]


def describe_plan(grid, tuning=None):
    g = grid.c()
    out = (ctypes.c_int32 * 8)()
    t = tuning.c() if tuning is not None else None
    _check(_lib().wave_describe_plan(ctypes.byref(g), ctypes.byref(t) if t else None, out),
           "wave_describe_plan")
    return dict(time_tile=out[0], tile_y=out[1], tile_x=out[2], tile_z=out[3], vec=out[4],
                prefetch=out[5], kernel=out[6], rows=out[7])


def describe_grad_plan(grid, nsrc, nrec, ckpt_every, tuning=None):
    """Shapes of the recompute and adjoint sweeps of the last wave_grad call
    with these arguments (raises WaveError when none has run)."""
    g = grid.c()
    out = (ctypes.c_int32 * 16)()
    t = tuning.c() if tuning is not None else None
    _check(_lib().wave_describe_grad_plan(ctypes.byref(g), ctypes.byref(t) if t else None, int(nsrc), int(nrec),
                                          int(ckpt_every), out), "wave_describe_grad_plan")
    keys = ("time_tile", "tile_y", "tile_x", "tile_z", "vec", "prefetch", "kernel", "rows")
    return {"recompute": {k: out[i] for i, k in enumerate(keys)},
            "adjoint": {k: out[8 + i] for i, k in enumerate(keys)}}


# --------------------------------------------------------------------------
# torch marshalling
# --------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def _dev_ptr(t, name, shape=None):
    torch = _torch()
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("%s must be a contiguous float32 tensor" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))
    return ctypes.c_void_p(t.data_ptr())


def _points(xyz):
    if xyz is None:
        return _Points(0, None), np.zeros((0, 3), np.float32)
    a = np.ascontiguousarray(np.asarray(xyz, dtype=np.float32).reshape(-1, 3))
    return _Points(a.shape[0], a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), a


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _workspace(nbytes, device, workspace):
    torch = _torch()
    if workspace is not None:
        if workspace.numel() * workspace.element_size() < nbytes:
            raise ValueError("workspace too small: need %d bytes" % nbytes)
        return workspace
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def fwd(grid, m, damp, src_xyz=None, src_traces=None, rec_xyz=None, *, tuning=None,
        want_u_last=False, ckpt_every=0, workspace=None, stream=None):
    """Forward modelling.  Returns (rec_traces [nt][nrec], u_last [2,...] or None,
    ckpt (flat float32 tensor) or None)."""
    torch = _torch()
    n = tuple(grid.n)
    sp, sa = _points(src_xyz)
    rp, ra = _points(rec_xyz)
    dev = m.device
    rec = torch.empty((grid.nt, rp.npts), dtype=torch.float32, device=dev)
    u_last = torch.empty((2,) + n, dtype=torch.float32, device=dev) if want_u_last else None
    ckpt = None
    if ckpt_every:
        ckpt = torch.empty(ckpt_bytes(grid, ckpt_every) // 4, dtype=torch.float32, device=dev)
    ws = _workspace(workspace_bytes(grid, WAVE_OP_FWD, sp.npts, rp.npts), dev, workspace)
    g = grid.c()
    t = tuning.c() if tuning is not None else None
    code = _lib().wave_fwd(
        ctypes.byref(g), _dev_ptr(m, "m", n), _dev_ptr(damp, "damp", n), ctypes.byref(sp),
        _dev_ptr(src_traces, "src_traces", (grid.nt, sp.npts)) if sp.npts else None,
        ctypes.byref(rp), _dev_ptr(rec, "rec") if rp.npts else None,
        _dev_ptr(u_last, "u_last") if u_last is not None else None,
        _dev_ptr(ckpt, "ckpt") if ckpt is not None else None, int(ckpt_every),
        ctypes.byref(t) if t is not None else None, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
        _stream(stream))
    del sa, ra
    _check(code, "wave_fwd")
    return rec, u_last, ckpt, ws


def adj(grid, m, damp, rec_xyz, rec_resid, src_xyz=None, *, tuning=None, want_v_last=False,
        workspace=None, stream=None):
    """Adjoint modelling.  Returns (src_adj [nt][nsrc], v_last [2,...] or None)."""
    torch = _torch()
    n = tuple(grid.n)
    rp, ra = _points(rec_xyz)
    sp, sa = _points(src_xyz)
    dev = m.device
    sadj = torch.empty((grid.nt, sp.npts), dtype=torch.float32, device=dev)
    v_last = torch.empty((2,) + n, dtype=torch.float32, device=dev) if want_v_last else None
    ws = _workspace(workspace_bytes(grid, WAVE_OP_ADJ, sp.npts, rp.npts), dev, workspace)
    g = grid.c()
    t = tuning.c() if tuning is not None else None
    code = _lib().wave_adj(
        ctypes.byref(g), _dev_ptr(m, "m", n), _dev_ptr(damp, "damp", n), ctypes.byref(rp),
        _dev_ptr(rec_resid, "rec_resid", (grid.nt, rp.npts)) if rp.npts else None,
        ctypes.byref(sp), _dev_ptr(sadj, "src_adj") if sp.npts else None,
        _dev_ptr(v_last, "v_last") if v_last is not None else None,
        ctypes.byref(t) if t is not None else None, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
        _stream(stream))
    del sa, ra
    _check(code, "wave_adj")
    return sadj, v_last, ws


def grad(grid, m, damp, src_xyz, src_traces, rec_xyz, rec_resid, ckpt, ckpt_every, *,
         tuning=None, workspace=None, stream=None):
    """dJ/dm for the residual rec_resid = dJ/dd, from wave_fwd checkpoints."""
    torch = _torch()
    n = tuple(grid.n)
    sp, sa = _points(src_xyz)
    rp, ra = _points(rec_xyz)
    dev = m.device
    g_out = torch.empty(n, dtype=torch.float32, device=dev)
    ws = _workspace(workspace_bytes(grid, WAVE_OP_GRAD, sp.npts, rp.npts, ckpt_every), dev,
                    workspace)
    g = grid.c()
    t = tuning.c() if tuning is not None else None
    code = _lib().wave_grad(
        ctypes.byref(g), _dev_ptr(m, "m", n), _dev_ptr(damp, "damp", n), ctypes.byref(sp),
        _dev_ptr(src_traces, "src_traces", (grid.nt, sp.npts)) if sp.npts else None,
        ctypes.byref(rp), _dev_ptr(rec_resid, "rec_resid", (grid.nt, rp.npts)) if rp.npts else None,
        _dev_ptr(ckpt, "ckpt"), int(ckpt_every), _dev_ptr(g_out, "grad"),
        ctypes.byref(t) if t is not None else None, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
        _stream(stream))
    del sa, ra
    _check(code, "wave_grad")
    return g_out, ws


def grad_revolve(grid, m, damp, src_xyz, src_traces, rec_xyz, rec_resid, nslots, *, tuning=None,
                 workspace=None, stream=None):
    """dJ/dm for the residual rec_resid = dJ/dd by binomial checkpointing
    with nslots stored states (wave_grad_revolve); no forward call first."""
    torch = _torch()
    n = tuple(grid.n)
    sp, sa = _points(src_xyz)
    rp, ra = _points(rec_xyz)
    dev = m.device
    g_out = torch.empty(n, dtype=torch.float32, device=dev)
    ws = _workspace(workspace_bytes(grid, WAVE_OP_REVOLVE, sp.npts, rp.npts, nslots), dev, workspace)
    g = grid.c()
    t = tuning.c() if tuning is not None else None
    code = _lib().wave_grad_revolve(
        ctypes.byref(g), _dev_ptr(m, "m", n), _dev_ptr(damp, "damp", n), ctypes.byref(sp),
        _dev_ptr(src_traces, "src_traces", (grid.nt, sp.npts)) if sp.npts else None,
        ctypes.byref(rp), _dev_ptr(rec_resid, "rec_resid", (grid.nt, rp.npts)) if rp.npts else None,
        int(nslots), _dev_ptr(g_out, "grad"), ctypes.byref(t) if t is not None else None,
        ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream))
    del sa, ra
    _check(code, "wave_grad_revolve")
    return g_out, ws


def born(grid, m, damp, dm, src_xyz, src_traces, rec_xyz, *, tuning=None, want_du_last=False,
         workspace=None, stream=None):
    """Born (linearised) modelling, the derivative of the traces in m in the
    direction dm (wave_born).  Returns (dd [nt][nrec], du_last [2,...] or
    None, workspace)."""
    torch = _torch()
    n = tuple(grid.n)
    sp, sa = _points(src_xyz)
    rp, ra = _points(rec_xyz)
    dev = m.device
    dd = torch.empty((grid.nt, rp.npts), dtype=torch.float32, device=dev)
    du = torch.empty((2,) + n, dtype=torch.float32, device=dev) if want_du_last else None
    ws = _workspace(workspace_bytes(grid, WAVE_OP_BORN, sp.npts, rp.npts), dev, workspace)
    g = grid.c()
    t = tuning.c() if tuning is not None else None
    code = _lib().wave_born(
        ctypes.byref(g), _dev_ptr(m, "m", n), _dev_ptr(damp, "damp", n), _dev_ptr(dm, "dm", n),
        ctypes.byref(sp), _dev_ptr(src_traces, "src_traces", (grid.nt, sp.npts)) if sp.npts else None,
        ctypes.byref(rp), _dev_ptr(dd, "rec") if rp.npts else None,
        _dev_ptr(du, "du_last") if du is not None else None,
        ctypes.byref(t) if t is not None else None, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
        _stream(stream))
    del sa, ra
    _check(code, "wave_born")
    return dd, du, ws


def revolve_forward_steps(nt, nslots):
    """Forward steps of the revolve schedule (-1: invalid arguments)."""
    return int(_lib().wave_revolve_forward_steps(int(nt), int(nslots)))


def revolve_schedule(nt, nslots):
    """The revolve schedule as a list of (kind, a, b): 0 advance a->b,
    1 takeshot (step a into slot b), 2 restore (step a from slot b, -1 = zero
    state), 3 youturn at a."""
    lib = _lib()
    n = int(lib.wave_revolve_schedule(int(nt), int(nslots), None, 0))
    if n < 0:
        _check(n, "wave_revolve_schedule")
    buf = (ctypes.c_int32 * (3 * max(n, 1)))()
    _check(min(0, int(lib.wave_revolve_schedule(int(nt), int(nslots), buf, n))), "wave_revolve_schedule")
    return [(buf[3 * i], buf[3 * i + 1], buf[3 * i + 2]) for i in range(n)]


def _heat(fn, grid, u0, kappa=None, src_xyz=None, src_traces=None, rec_xyz=None, *, tuning=None,
          workspace=None, stream=None):
    """Marshalling shared by wave_heat and wave_heat_ab2 (same arguments)."""
    torch = _torch()
    n = tuple(grid.n)
    sp, sa = _points(src_xyz)
    rp, ra = _points(rec_xyz)
    dev = u0.device
    rec = torch.empty((grid.nt, rp.npts), dtype=torch.float32, device=dev)
    u_out = torch.empty(n, dtype=torch.float32, device=dev)
    ws = _workspace(workspace_bytes(grid, WAVE_OP_FWD, sp.npts, rp.npts), dev, workspace)
    g = grid.c()
    t = tuning.c() if tuning is not None else None
    code = getattr(_lib(), fn)(
        ctypes.byref(g), _dev_ptr(kappa, "kappa", n) if kappa is not None else None,
        _dev_ptr(u0, "u0", n), ctypes.byref(sp),
        _dev_ptr(src_traces, "src_traces", (grid.nt, sp.npts)) if sp.npts else None,
        ctypes.byref(rp), _dev_ptr(rec, "rec") if rp.npts else None, _dev_ptr(u_out, "u_out"),
        ctypes.byref(t) if t is not None else None, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
        _stream(stream))
    del sa, ra
    _check(code, fn)
    return u_out, rec, ws


def heat(grid, u0, kappa=None, src_xyz=None, src_traces=None, rec_xyz=None, *, tuning=None,
         workspace=None, stream=None):
    """Heat (Laplace) operator, explicit Euler for u_t = kappa (lap u + f)
    (wave_heat).  u0: initial field; kappa: diffusivity field or None for 1.
    Returns (u^nt, rec_traces [nt][nrec], workspace)."""
    return _heat("wave_heat", grid, u0, kappa, src_xyz, src_traces, rec_xyz, tuning=tuning,
                 workspace=workspace, stream=stream)


def heat_ab2(grid, u0, kappa=None, src_xyz=None, src_traces=None, rec_xyz=None, *, tuning=None,
             workspace=None, stream=None):
    """The same operator by the two-step Adams-Bashforth scheme with an Euler
    first step (wave_heat_ab2).  Returns (u^nt, rec_traces, workspace)."""
    return _heat("wave_heat_ab2", grid, u0, kappa, src_xyz, src_traces, rec_xyz, tuning=tuning,
                 workspace=workspace, stream=stream)


@dataclass
class Shot:
    """One shot of a batch: a window [origin, origin + n) of the global grid,
    source and receiver coordinates (km) relative to the window origin."""
    origin: tuple
    n: tuple
    src_xyz: object = None
    rec_xyz: object = None


def _shots(shots):
    arr = (_Shot * len(shots))()
    keep = []
    for c, s in zip(arr, shots):
        c.origin[:] = [int(v) for v in s.origin]
        c.n[:] = [int(v) for v in s.n]
        sp, sa = _points(s.src_xyz)
        rp, ra = _points(s.rec_xyz)
        c.src, c.rec = sp, rp
        keep += [sa, ra]
    return arr, keep


def batch_workspace_bytes(grid, shots, ckpt_every=0, concurrency=0):
    arr, keep = _shots(shots)
    g = grid.c()
    n = int(_lib().wave_batch_workspace_bytes(ctypes.byref(g), len(shots), arr, int(ckpt_every),
                                              int(concurrency)))
    del keep
    return n


def describe_batch_plan(grid, shots, ckpt_every=0, concurrency=0, tuning=None):
    """Kernels of the first group of a batched call
    (wave_describe_batch_plan): None when the shots run one by one, else the
    forward kernel as the keys of describe_plan plus lockstep=True (time_tile
    0 while an autotuned group has not been timed yet), and for the gradient
    grad_kernel / grad_time_tile of its recompute and adjoint phases."""
    arr, keep = _shots(shots)
    g = grid.c()
    out = (ctypes.c_int32 * 11)()
    t = tuning.c() if tuning is not None else None
    _check(_lib().wave_describe_batch_plan(ctypes.byref(g), len(shots), arr, int(ckpt_every), int(concurrency),
                                           ctypes.byref(t) if t else None, out), "wave_describe_batch_plan")
    del keep
    if out[8] == 0:
        return None
    return dict(time_tile=out[0], tile_y=out[1], tile_x=out[2], tile_z=out[3], vec=out[4],
                prefetch=out[5], kernel=out[6], rows=out[7], lockstep=True,
                grad_kernel=out[9], grad_time_tile=out[10])


def _traces(x, name, nt, counts):
    """Per-shot [nt][k_s] blocks, one after another: a list of tensors or one
    flat tensor already in that layout."""
    torch = _torch()
    if isinstance(x, (list, tuple)):
        for t, k in zip(x, counts):
            if tuple(t.shape) != (nt, k):
                raise ValueError("%s block has shape %s, expected %s" % (name, tuple(t.shape), (nt, k)))
        x = torch.cat([t.reshape(-1) for t in x]) if x else None
    if x is not None and x.numel() != nt * sum(counts):
        raise ValueError("%s has %d values, expected %d" % (name, x.numel(), nt * sum(counts)))
    return x


def fwd_batched(grid, shots, m, damp, src_traces, *, concurrency=0, tuning=None, workspace=None,
                stream=None):
    """Forward modelling of every shot (wave_fwd_batched).  src_traces: list
    of [nt][nsrc_s] tensors (or their flat concatenation).  Returns the list
    of [nt][nrec_s] receiver traces and the workspace."""
    torch = _torch()
    n = tuple(grid.n)
    ns = [0 if s.src_xyz is None else len(s.src_xyz) for s in shots]
    nr = [0 if s.rec_xyz is None else len(s.rec_xyz) for s in shots]
    q = _traces(src_traces, "src_traces", grid.nt, ns)
    out = torch.empty(grid.nt * sum(nr), dtype=torch.float32, device=m.device)
    ws = _workspace(batch_workspace_bytes(grid, shots, 0, concurrency), m.device, workspace)
    arr, keep = _shots(shots)
    g = grid.c()
    t = tuning.c() if tuning is not None else None
    code = _lib().wave_fwd_batched(
        ctypes.byref(g), len(shots), arr, _dev_ptr(m, "m", n), _dev_ptr(damp, "damp", n),
        _dev_ptr(q, "src_traces") if q is not None and q.numel() else None,
        _dev_ptr(out, "rec_traces") if out.numel() else None, int(concurrency),
        ctypes.byref(t) if t is not None else None, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
        _stream(stream))
    del keep
    _check(code, "wave_fwd_batched")
    recs, o = [], 0
    for k in nr:
        recs.append(out[o:o + grid.nt * k].view(grid.nt, k))
        o += grid.nt * k
    return recs, ws


def grad_batched(grid, shots, m, damp, src_traces, rec_resid, ckpt_every, *, concurrency=0,
                 tuning=None, workspace=None, stream=None):
    """dJ/dm over all shots (wave_grad_batched); rec_resid: list of [nt][nrec_s]
    tensors of dJ/dd_s (or their flat concatenation).  Returns (grad, ws)."""
    torch = _torch()
    n = tuple(grid.n)
    ns = [0 if s.src_xyz is None else len(s.src_xyz) for s in shots]
    nr = [0 if s.rec_xyz is None else len(s.rec_xyz) for s in shots]
    q = _traces(src_traces, "src_traces", grid.nt, ns)
    r = _traces(rec_resid, "rec_resid", grid.nt, nr)
    g_out = torch.empty(n, dtype=torch.float32, device=m.device)
    ws = _workspace(batch_workspace_bytes(grid, shots, ckpt_every, concurrency), m.device, workspace)
    arr, keep = _shots(shots)
    g = grid.c()
    t = tuning.c() if tuning is not None else None
    code = _lib().wave_grad_batched(
        ctypes.byref(g), len(shots), arr, _dev_ptr(m, "m", n), _dev_ptr(damp, "damp", n),
        _dev_ptr(q, "src_traces") if q is not None and q.numel() else None,
        _dev_ptr(r, "rec_resid") if r is not None and r.numel() else None, int(ckpt_every),
        _dev_ptr(g_out, "grad"), int(concurrency), ctypes.byref(t) if t is not None else None,
        ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream))
    del keep
    _check(code, "wave_grad_batched")
    return g_out, ws


def fwd_noalloc(grid, m, damp, src_xyz, src_traces, rec_xyz, rec_out, u_last_out=None, *,
                tuning=None, stream=None, wait=True):
    """Forward modelling on the library's static workspace (wave_fwd_noalloc).
    The outputs are the caller's: rec_out [nt][nrec] and optionally
    u_last_out [2,...], both float32 on the device; nothing is allocated on
    the device here.  Returns the device status word when `wait`, else None."""
    n = tuple(grid.n)
    sp, sa = _points(src_xyz)
    rp, ra = _points(rec_xyz)
    g = grid.c()
    t = tuning.c() if tuning is not None else None
    st = ctypes.c_int32(0)
    code = _lib().wave_fwd_noalloc(
        ctypes.byref(g), _dev_ptr(m, "m", n), _dev_ptr(damp, "damp", n), ctypes.byref(sp),
        _dev_ptr(src_traces, "src_traces", (grid.nt, sp.npts)) if sp.npts else None,
        ctypes.byref(rp), _dev_ptr(rec_out, "rec_out", (grid.nt, rp.npts)) if rp.npts else None,
        _dev_ptr(u_last_out, "u_last_out", (2,) + n) if u_last_out is not None else None,
        ctypes.byref(t) if t is not None else None, _stream(stream),
        ctypes.byref(st) if wait else None)
    del sa, ra
    _check(code, "wave_fwd_noalloc")
    return int(st.value) if wait else None


def measure_peaks(stream=None):
    """Measured (FP32 FMA TFLOP/s with paired FMAs, shared-memory load TB/s)
    of the current device (wave_measure_peaks)."""
    f, m = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(_lib().wave_measure_peaks(ctypes.byref(f), ctypes.byref(m), _stream(stream)),
           "wave_measure_peaks")
    return f.value, m.value


def sweep_stats():
    """(ms, launches, steps) of the sweep launches of the last call made with
    Tuning.flags |= WAVE_TIME_SWEEPS on this thread."""
    ms = ctypes.c_float()
    nl = ctypes.c_int32()
    ns = ctypes.c_int32()
    _check(_lib().wave_sweep_stats(ctypes.byref(ms), ctypes.byref(nl), ctypes.byref(ns)),
           "wave_sweep_stats")
    return float(ms.value), int(nl.value), int(ns.value)


def autotune_stats():
    """(candidates, pruned) of the last autotuner run on this thread."""
    c, p = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib().wave_autotune_stats(ctypes.byref(c), ctypes.byref(p)), "wave_autotune_stats")
    return int(c.value), int(p.value)


def plan_bound(grid, tuning, hbm_gbs=0.0, lsu_gbs=0.0, l2_bytes=0.0):
    """Runtime bound (ms per time step) of the plan `tuning` selects
    (wave_plan_bound); zero arguments take the current device's figures."""
    g = grid.c()
    t = tuning.c()
    out = ctypes.c_double()
    _check(_lib().wave_plan_bound(ctypes.byref(g), ctypes.byref(t), float(hbm_gbs), float(lsu_gbs),
                                  float(l2_bytes), ctypes.byref(out)), "wave_plan_bound")
    return float(out.value)


def status(ws, stream=None):
    """Wait for the stream and return the device status word of workspace ws."""
    return int(_lib().wave_status(ctypes.c_void_p(ws.data_ptr()), _stream(stream)))

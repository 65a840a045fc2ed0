"""Plain FP64 CPU oracle for the time-tiled acoustic wave path.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
CPU-baseline / reference leg may import this package.  The product library
(paper_1806_08299_gb300) never imports it, and it imports nothing from the
product.  Inputs are numpy arrays; everything is computed in float64 by the C
code in wave_oracle.c (ctypes binding below) and by oracle/coeffs.py.

Functions and what pins them (see tests/test_oracle_*.py):
  fd2_central_weights  closed form and a published table           (pinned)
  cfl_dt               closed form at theta = pi                    (pinned)
  laplacian            exact on polynomials, order-2r convergence   (pinned)
  forward              discrete plane-wave dispersion (undamped and
                       damped), first-steps closed form, linearity,
                       trilinear exactness of receivers             (pinned)
  forward_tiled        bitwise equal to forward (the paper's test)  (pinned)
  adjoint              dot-product test against forward             (pinned)
  gradient             central finite differences of the misfit    (pinned)
  heat                 explicit Euler for the Laplace operator: exact decay
                       of a discrete Dirichlet sine mode (so 2), one step
                       of a quadratic exact away from the boundary, a
                       source on a node, linearity in u0 and f    (pinned)
  heat_ab2             two-step Adams-Bashforth for the Laplace operator:
                       exact amplification of a discrete Dirichlet sine
                       mode (the closed form of the two-step recurrence),
                       second-order convergence in dt to the exact decay,
                       Euler start, linearity                     (pinned)
  born                 linearised modelling (the derivative of forward
                       in m): central finite differences of forward,
                       the dot identity with gradient, linearity    (pinned)
  forward_batched,     per-shot forward / gradient on windows of one
  gradient_batched     model, window gradients summed into the global
                       grid; pinned by whole-grid shots, shot additivity
                       and central finite differences of the survey misfit
"""
import ctypes
import os

import numpy as np

from .coeffs import fd2_central_weights, symbol, symbol_max, cfl_dt  # noqa: F401
from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        i = ctypes.c_int
        d = ctypes.c_double
        lib.oracle_set_threads.argtypes = [i]
        lib.oracle_max_threads.restype = i
        lib.oracle_laplacian.argtypes = [ip, dp, i, dp, i, dp, dp]
        lib.oracle_forward.argtypes = [ip, dp, d, i, i, dp, dp, dp, i, dp, dp, i, dp, dp,
                                       i, dp, dp, dp, dp]
        lib.oracle_forward.restype = i
        lib.oracle_forward_tiled.argtypes = [ip, dp, d, i, i, dp, dp, dp, i, dp, dp, i, dp, dp,
                                             i, i, i, dp]
        lib.oracle_forward_tiled.restype = i
        lib.oracle_adjoint.argtypes = [ip, dp, d, i, i, dp, dp, dp, i, dp, dp, i, dp, dp, dp]
        lib.oracle_adjoint.restype = i
        lib.oracle_gradient.argtypes = [ip, dp, d, i, i, dp, dp, dp, i, dp, dp, i, dp, dp, dp]
        lib.oracle_gradient.restype = i
        lib.oracle_heat.argtypes = [ip, dp, d, i, i, dp, dp, dp, i, dp, dp, i, dp, dp, dp]
        lib.oracle_heat.restype = i
        lib.oracle_born.argtypes = [ip, dp, d, i, i, dp, dp, dp, dp, i, dp, dp, i, dp, dp, dp]
        lib.oracle_born.restype = i
        lib.oracle_heat_ab2.argtypes = [ip, dp, d, i, i, dp, dp, dp, i, dp, dp, i, dp, dp, dp]
        lib.oracle_heat_ab2.restype = i
        _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _arr(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ints(n):
    return (ctypes.c_int * 3)(*[int(v) for v in n])


def _coeffs(space_order):
    return np.array([float(v) for v in fd2_central_weights(space_order)], dtype=np.float64)


def _pts(xyz):
    if xyz is None:
        return 0, np.zeros((1, 3))
    a = _arr(xyz).reshape(-1, 3)
    return a.shape[0], a


def set_threads(n):
    """OpenMP thread count for the oracle's parallel loops."""
    _load().oracle_set_threads(int(n))


def max_threads():
    return int(_load().oracle_max_threads())


def laplacian(u, h, space_order, periodic=False):
    """L u with a zero halo outside the grid (or periodic wrap)."""
    u = _arr(u)
    out = np.empty_like(u)
    c = _coeffs(space_order)
    _load().oracle_laplacian(_ints(u.shape), _p(_arr(h)), space_order // 2, _p(c),
                             int(bool(periodic)), _p(u), _p(out))
    return out


def forward(m, damp, h, dt, nt, space_order, src_xyz=None, src_q=None, rec_xyz=None,
            periodic=False, u0=None, um1=None, keep_all=False):
    """Untiled leapfrog forward.  Returns (rec_d [nt][nrec], u_last [2][...], u_all).

    u_last = (u^nt, u^{nt-1}); u_all (if keep_all) = [u^-1, u^0, ..., u^nt]."""
    m = _arr(m)
    n = m.shape
    damp = _arr(damp, n)
    nsrc, sx = _pts(src_xyz)
    nrec, rx = _pts(rec_xyz)
    q = _arr(src_q, (nt, nsrc)) if nsrc else np.zeros((1,))
    d = np.zeros((nt, max(nrec, 1)))
    u_last = np.zeros((2,) + n)
    u_all = np.zeros((nt + 2,) + n) if keep_all else None
    c = _coeffs(space_order)
    rc = _load().oracle_forward(
        _ints(n), _p(_arr(h)), float(dt), int(nt), space_order // 2, _p(c), _p(m), _p(damp),
        nsrc, _p(sx), _p(q), nrec, _p(rx), _p(d), int(bool(periodic)),
        _p(_arr(u0, n)) if u0 is not None else None,
        _p(_arr(um1, n)) if um1 is not None else None,
        _p(u_last), _p(u_all))
    if rc:
        raise RuntimeError("oracle_forward failed (%d)" % rc)
    return d[:, :nrec], u_last, u_all


def forward_tiled(m, damp, h, dt, nt, space_order, src_xyz=None, src_q=None, rec_xyz=None,
                  tt=4, bx=8, by=8):
    """The paper's skewed time-tiled loop nest.  Returns (rec_d, u_last)."""
    m = _arr(m)
    n = m.shape
    damp = _arr(damp, n)
    nsrc, sx = _pts(src_xyz)
    nrec, rx = _pts(rec_xyz)
    q = _arr(src_q, (nt, nsrc)) if nsrc else np.zeros((1,))
    d = np.zeros((nt, max(nrec, 1)))
    u_last = np.zeros((2,) + n)
    c = _coeffs(space_order)
    rc = _load().oracle_forward_tiled(
        _ints(n), _p(_arr(h)), float(dt), int(nt), space_order // 2, _p(c), _p(m), _p(damp),
        nsrc, _p(sx), _p(q), nrec, _p(rx), _p(d), int(tt), int(bx), int(by), _p(u_last))
    if rc:
        raise RuntimeError("oracle_forward_tiled failed (%d)" % rc)
    return d[:, :nrec], u_last


def adjoint(m, damp, h, dt, nt, space_order, rec_xyz, res, src_xyz=None):
    """Transposed recursion.  Returns (src_grad [nt][nsrc], lam_last [2][...]).

    src_grad = dJ/dq for J = sum <res, d>; lam_last = (lambda^1, lambda^2)."""
    m = _arr(m)
    n = m.shape
    damp = _arr(damp, n)
    nrec, rx = _pts(rec_xyz)
    nsrc, sx = _pts(src_xyz)
    res = _arr(res, (nt, nrec))
    sg = np.zeros((nt, max(nsrc, 1)))
    lam = np.zeros((2,) + n)
    c = _coeffs(space_order)
    rc = _load().oracle_adjoint(
        _ints(n), _p(_arr(h)), float(dt), int(nt), space_order // 2, _p(c), _p(m), _p(damp),
        nrec, _p(rx), _p(res), nsrc, _p(sx), _p(sg), _p(lam))
    if rc:
        raise RuntimeError("oracle_adjoint failed (%d)" % rc)
    return sg[:, :nsrc], lam


def gradient(m, damp, h, dt, nt, space_order, src_xyz, src_q, rec_xyz, res):
    """dJ/dm for J = sum_n <res^n, d^n> with res held fixed (res = dJ/dd)."""
    m = _arr(m)
    n = m.shape
    damp = _arr(damp, n)
    nsrc, sx = _pts(src_xyz)
    nrec, rx = _pts(rec_xyz)
    q = _arr(src_q, (nt, nsrc))
    res = _arr(res, (nt, nrec))
    g = np.zeros(n)
    c = _coeffs(space_order)
    rc = _load().oracle_gradient(
        _ints(n), _p(_arr(h)), float(dt), int(nt), space_order // 2, _p(c), _p(m), _p(damp),
        nsrc, _p(sx), _p(q), nrec, _p(rx), _p(res), _p(g))
    if rc:
        raise RuntimeError("oracle_gradient failed (%d)" % rc)
    return g


def born(m, damp, dm, h, dt, nt, space_order, src_xyz, src_q, rec_xyz):
    """Born (linearised) modelling: the derivative of the receiver traces
    with respect to m in the direction dm.  Returns (dd [nt][nrec],
    du_last [2][...] = (du^nt, du^{nt-1})).  Not in the paper: the
    linearisation of the leapfrog scheme written out in wave_oracle.c."""
    m = _arr(m)
    n = m.shape
    damp = _arr(damp, n)
    dm = _arr(dm, n)
    nsrc, sx = _pts(src_xyz)
    nrec, rx = _pts(rec_xyz)
    q = _arr(src_q, (nt, nsrc)) if nsrc else np.zeros((1,))
    dd = np.zeros((nt, max(nrec, 1)))
    du_last = np.zeros((2,) + n)
    c = _coeffs(space_order)
    rc = _load().oracle_born(
        _ints(n), _p(_arr(h)), float(dt), int(nt), space_order // 2, _p(c), _p(m), _p(damp), _p(dm),
        nsrc, _p(sx), _p(q), nrec, _p(rx), _p(dd), _p(du_last))
    if rc:
        raise RuntimeError("oracle_born failed (%d)" % rc)
    return dd[:, :nrec], du_last


def heat(u0, h, dt, nt, space_order, kappa=None, src_xyz=None, src_q=None, rec_xyz=None):
    """Explicit Euler for u_t = kappa (lap u + f) (the Laplace operator of
    Sec. 5.7).  Returns (rec_d [nt][nrec], u^nt)."""
    u0 = _arr(u0)
    n = u0.shape
    nsrc, sx = _pts(src_xyz)
    nrec, rx = _pts(rec_xyz)
    q = _arr(src_q, (nt, nsrc)) if nsrc else np.zeros((1,))
    d = np.zeros((nt, max(nrec, 1)))
    u_last = np.zeros(n)
    c = _coeffs(space_order)
    rc = _load().oracle_heat(
        _ints(n), _p(_arr(h)), float(dt), int(nt), space_order // 2, _p(c),
        _p(_arr(kappa, n)) if kappa is not None else None, _p(u0),
        nsrc, _p(sx), _p(q), nrec, _p(rx), _p(d), _p(u_last))
    if rc:
        raise RuntimeError("oracle_heat failed (%d)" % rc)
    return d[:, :nrec], u_last


def heat_ab2(u0, h, dt, nt, space_order, kappa=None, src_xyz=None, src_q=None, rec_xyz=None):
    """Two-step Adams-Bashforth for u_t = kappa (lap u + f) with an Euler first
    step (a time dependence of two levels; the multi-step methods of Sec. 6).
    Returns (rec_d [nt][nrec], u^nt)."""
    u0 = _arr(u0)
    n = u0.shape
    nsrc, sx = _pts(src_xyz)
    nrec, rx = _pts(rec_xyz)
    q = _arr(src_q, (nt, nsrc)) if nsrc else np.zeros((1,))
    d = np.zeros((nt, max(nrec, 1)))
    u_last = np.zeros(n)
    c = _coeffs(space_order)
    rc = _load().oracle_heat_ab2(
        _ints(n), _p(_arr(h)), float(dt), int(nt), space_order // 2, _p(c),
        _p(_arr(kappa, n)) if kappa is not None else None, _p(u0),
        nsrc, _p(sx), _p(q), nrec, _p(rx), _p(d), _p(u_last))
    if rc:
        raise RuntimeError("oracle_heat_ab2 failed (%d)" % rc)
    return d[:, :nrec], u_last


def _window(shot):
    o, n = shot["origin"], shot["n"]
    return tuple(slice(int(o[a]), int(o[a]) + int(n[a])) for a in range(3))


def forward_batched(m, damp, h, dt, nt, space_order, shots, src_q):
    """Receiver traces of every shot of a survey.  Shot s (a dict with
    "origin", "n", "src", "rec"; coordinates relative to its window) sees the
    window of the global m and damp it names; src_q[s] is its [nt][nsrc_s]
    trace.  Returns the list of [nt][nrec_s] traces."""
    m, damp = _arr(m), _arr(damp)
    out = []
    for shot, q in zip(shots, src_q):
        w = _window(shot)
        d, _, _ = forward(m[w], damp[w], h, dt, nt, space_order, shot["src"], q, shot["rec"])
        out.append(d)
    return out


def gradient_batched(m, damp, h, dt, nt, space_order, shots, src_q, res):
    """Gradient of J = sum_s <res_s, d_s> with respect to the global m: the
    window gradient of each shot added into the global grid at its window
    (zero outside every window), summed in shot order."""
    m, damp = _arr(m), _arr(damp)
    g = np.zeros(m.shape)
    for shot, q, r in zip(shots, src_q, res):
        w = _window(shot)
        g[w] += gradient(m[w], damp[w], h, dt, nt, space_order, shot["src"], q, shot["rec"], r)
    return g

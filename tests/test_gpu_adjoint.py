"""GPU parity of the adjoint, the m-gradient and the autograd wrapper.

* wave_adj against the oracle's transposed recursion (source-side traces and
  the final adjoint field nu^1 = C lambda^1), and the FP32 dot-product test
  <F q, r> = <q, F^T r>;
* wave_grad (checkpoint every k steps, segment recompute, fused imaging
  condition) against the oracle gradient, rel-L2 <= 1e-5, with a ragged last
  segment, for untiled and time-tiled sweeps (bitwise equal to each other);
* every shape wave_grad can choose for its recompute and adjoint sweeps gives
  the same gradient bit for bit;
* the torch.autograd.Function gives the same gradient as wave_grad.
"""
import numpy as np
import pytest

from paper_1806_08299_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _t(x, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev)


def _f64(a):
    return np.asarray(a, dtype=np.float64)


def _setup(wavelib, n, so, nt, seed, nsrc=2, nrec=6):
    m, damp, src, q, rec = inputs.random_problem(n, so, nt, seed=seed, nsrc=nsrc, nrec=nrec)
    dt = 0.4 * wavelib.cfl_dt(so, (inputs.H,) * 3, 3.0)
    grid = wavelib.Grid(n, (inputs.H,) * 3, dt, nt, so)
    h = [float(np.float32(v)) for v in grid.h]
    return grid, h, float(np.float32(dt)), m, damp, src, q, rec


def _relerr(a, b):
    return float(np.linalg.norm(_f64(a) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("so,T", [(4, 1), (4, 3), (8, 2), (12, 1)])
def test_adjoint_vs_oracle(wavelib, cuda, oracle, so, T):
    import torch
    n = (39, 44, 37)
    nt = 27
    grid, h, dt, m, damp, src, q, rec = _setup(wavelib, n, so, nt, seed=3 + so)
    res = np.random.default_rng(1).standard_normal((nt, len(rec))).astype(np.float32)
    sadj, vl, ws = wavelib.adj(grid, _t(m, cuda), _t(damp, cuda), rec, _t(res, cuda), src,
                               tuning=wavelib.Tuning(time_tile=T), want_v_last=True)
    assert wavelib.status(ws) == 0
    sadj, vl = sadj.cpu().numpy(), vl.cpu().numpy()
    sg, lam = oracle.adjoint(_f64(m), _f64(damp), h, dt, nt, so, _f64(rec), _f64(res), src_xyz=_f64(src))
    C = dt * dt / (_f64(m) + _f64(damp) * dt / 2)
    assert _relerr(vl[0], C * lam[0]) <= TOL
    assert _relerr(vl[1], C * lam[1]) <= TOL
    assert np.abs(sadj - sg).max() <= TOL * np.abs(sg).max()
    # FP32 dot test: <F q, res> = <q, F^T res>
    d, _, _, _ = wavelib.fwd(grid, _t(m, cuda), _t(damp, cuda), src, _t(q, cuda), rec,
                             tuning=wavelib.Tuning(time_tile=T))
    torch.cuda.synchronize()
    lhs = float(np.sum(_f64(d.cpu().numpy()) * _f64(res)))
    rhs = float(np.sum(_f64(q) * _f64(sadj)))
    assert abs(lhs - rhs) <= TOL * abs(lhs)


@pytest.mark.parametrize("so,T,k", [(8, 1, 7), (8, 2, 8), (4, 4, 12), (4, 1, 40)])
def test_gradient_vs_oracle(wavelib, cuda, oracle, so, T, k):
    import torch
    n = (34, 31, 36)
    nt = 40
    grid, h, dt, m, damp, src, q, rec = _setup(wavelib, n, so, nt, seed=11, nsrc=1, nrec=8)
    res = np.random.default_rng(2).standard_normal((nt, len(rec))).astype(np.float32)
    tm, td, tq = _t(m, cuda), _t(damp, cuda), _t(q, cuda)
    tune = wavelib.Tuning(time_tile=T)
    _, _, ckpt, _ = wavelib.fwd(grid, tm, td, src, tq, rec, tuning=tune, ckpt_every=k)
    g, ws = wavelib.grad(grid, tm, td, src, tq, rec, _t(res, cuda), ckpt, k, tuning=tune)
    assert wavelib.status(ws) == 0
    g = g.cpu().numpy()
    gref = oracle.gradient(_f64(m), _f64(damp), h, dt, nt, so, _f64(src), _f64(q), _f64(rec), _f64(res))
    err = _relerr(g, gref)
    assert err <= TOL, err
    if T > 1:
        g1, _ = wavelib.grad(grid, tm, td, src, tq, rec, _t(res, cuda), ckpt, k,
                             tuning=wavelib.Tuning(time_tile=1))
        torch.cuda.synchronize()
        assert np.array_equal(g1.cpu().numpy(), g)


def test_autograd_matches_wave_grad(wavelib, cuda):
    import torch
    from paper_1806_08299_gb300.autograd import modeling
    n = (30, 32, 28)
    nt = 36
    grid, h, dt, m, damp, src, q, rec = _setup(wavelib, n, 8, nt, seed=21, nsrc=1, nrec=6)
    tm = _t(m, cuda).requires_grad_(True)
    td, tq = _t(damp, cuda), _t(q, cuda)
    d_obs = torch.zeros((nt, len(rec)), device=cuda)
    d = modeling(tm, grid, td, src, tq, rec, ckpt_every=10, tuning=wavelib.Tuning(time_tile=2))
    loss = 0.5 * ((d - d_obs) ** 2).sum()
    loss.backward()
    _, _, ckpt, _ = wavelib.fwd(grid, tm.detach(), td, src, tq, rec, ckpt_every=10,
                                tuning=wavelib.Tuning(time_tile=2))
    g, _ = wavelib.grad(grid, tm.detach(), td, src, tq, rec, (d - d_obs).detach().contiguous(),
                        ckpt, 10, tuning=wavelib.Tuning(time_tile=2))
    torch.cuda.synchronize()
    assert torch.equal(tm.grad, g)
    assert torch.isfinite(g).all() and g.abs().max() > 0


@pytest.mark.parametrize("so", [8, 4])
def test_staged_gradient_modes_bitwise(wavelib, cuda, oracle, so):
    """The gradient sweeps of the stage-specialised kernel (second differences
    stored by the recompute sweep, imaging condition fused into the adjoint
    sweep, at depth 1 and 2) give the untiled gradient of the shared-warp
    kernel bit for bit, which is at parity with the oracle; ragged last
    segment, x-chunks shorter and longer than the stencil reach."""
    import torch
    n = (37, 52, 45)
    nt, k = 23, 9
    grid, h, dt, m, damp, src, q, rec = _setup(wavelib, n, so, nt, seed=41 + so, nsrc=2, nrec=7)
    res = np.random.default_rng(5).standard_normal((nt, len(rec))).astype(np.float32)
    tm, td, tq, tr = _t(m, cuda), _t(damp, cuda), _t(q, cuda), _t(res, cuda)

    def grad(tune):
        _, _, ckpt, _ = wavelib.fwd(grid, tm, td, src, tq, rec, tuning=tune, ckpt_every=k)
        g, ws = wavelib.grad(grid, tm, td, src, tq, rec, tr, ckpt, k, tuning=tune)
        assert wavelib.status(ws) == 0
        torch.cuda.synchronize()
        return g.cpu().numpy()

    g1 = grad(wavelib.Tuning(time_tile=1, kernel=wavelib.WAVE_KERNEL_SHARED))
    gref = oracle.gradient(_f64(m), _f64(damp), h, dt, nt, so, _f64(src), _f64(q), _f64(rec), _f64(res))
    assert _relerr(g1, gref) <= TOL
    for T in (1, 2):
        shapes = [v for v in wavelib.list_variants(so)
                  if v["kernel"] == wavelib.WAVE_KERNEL_STAGED and v["time_tile"] == T]
        for v in shapes:
            for tile_x in (5, 17):
                tune = wavelib.Tuning(time_tile=T, tile_y=v["tile_y"], tile_z=v["tile_z"], tile_x=tile_x,
                                      kernel=wavelib.WAVE_KERNEL_STAGED, rows=v["rows"])
                assert np.array_equal(grad(tune), g1), (T, v, tile_x)


@pytest.mark.parametrize("so,T", [(8, 2), (8, 1), (4, 2)])
def test_every_gradient_shape_bitwise(wavelib, cuda, oracle, monkeypatch, so, T):
    """wave_grad times its candidate shapes for the recompute sweep and for the
    adjoint sweep separately.  Pinned one by one through the WAVE_GRAD_PIN
    test hook, every recompute candidate (with the first adjoint candidate)
    and every adjoint candidate (with the first recompute candidate) gives the
    gradient of the first pair bit for bit, which is at parity with the
    oracle; a ragged last segment."""
    import torch
    n = (37, 52, 45)
    nt, k = 23, 9
    grid, h, dt, m, damp, src, q, rec = _setup(wavelib, n, so, nt, seed=61 + so, nsrc=2, nrec=7)
    res = np.random.default_rng(7).standard_normal((nt, len(rec))).astype(np.float32)
    tm, td, tq, tr = _t(m, cuda), _t(damp, cuda), _t(q, cuda), _t(res, cuda)
    tune = wavelib.Tuning(time_tile=T, kernel=wavelib.WAVE_KERNEL_STAGED)
    _, _, ckpt, _ = wavelib.fwd(grid, tm, td, src, tq, rec, tuning=tune, ckpt_every=k)

    def grad(i, j):
        monkeypatch.setenv("WAVE_GRAD_PIN", "%d,%d" % (i, j))
        try:
            g, ws = wavelib.grad(grid, tm, td, src, tq, rec, tr, ckpt, k, tuning=tune)
        except wavelib.WaveError as e:
            assert e.code == wavelib.WAVE_EUNSUPPORTED
            return None
        assert wavelib.status(ws) == 0
        torch.cuda.synchronize()
        return g.cpu().numpy()

    g0 = grad(0, 0)
    gref = oracle.gradient(_f64(m), _f64(damp), h, dt, nt, so, _f64(src), _f64(q), _f64(rec), _f64(res))
    assert _relerr(g0, gref) <= TOL
    ran = [0, 0]
    for side in (0, 1):
        for c in range(1, 16):
            g = grad(c, 0) if side == 0 else grad(0, c)
            if g is None:
                break
            ran[side] += 1
            assert np.array_equal(g, g0), (side, c)
    # the shared-warp default and the staged shapes of depth T and 1
    assert ran[0] >= 2 and ran[1] >= 2, ran
    monkeypatch.delenv("WAVE_GRAD_PIN")
    g_auto, _ = wavelib.grad(grid, tm, td, src, tq, rec, tr, ckpt, k, tuning=tune)
    torch.cuda.synchronize()
    assert np.array_equal(g_auto.cpu().numpy(), g0)
    # the timed choice is reported per phase, among the candidates' depths
    gp = wavelib.describe_grad_plan(grid, len(src), len(rec), k, tuning=tune)
    for phase in ("recompute", "adjoint"):
        assert gp[phase]["time_tile"] in (1, T), gp
        assert gp[phase]["kernel"] in (wavelib.WAVE_KERNEL_SHARED, wavelib.WAVE_KERNEL_STAGED), gp
        assert gp[phase]["tile_x"] >= 1

"""GPU parity of wave_born (Born / linearised modelling).

* the linearised traces and the last two perturbation levels against the
  FP64 oracle's Born modelling, at every space order with a stage-specialised
  Born sweep (one per radius), within 1e-5 (traces: of max |dd|; fields:
  rel-L2);
* the FP32 dot identity with the gradient: <born(dm), r> = <dm, grad(r)>;
* linearity: born(2 dm) = 2 born(dm) to 1e-6 of max |dd| (every operation
  of the perturbation sweep is linear in dm and doubling is exact, except
  where a product P D rounds in the subnormal range ahead of the wavefront);
* the background plan (tiled or not) does not change the bits;
* the fused sweep (both fields in one pass) gives the bits of the two-sweep
  form (background storing D, then the perturbation sweep) at every order.
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


def _setup(wavelib, n, so, nt, seed):
    m, damp, src, q, rec = inputs.random_problem(n, so, nt, seed=seed, nsrc=2, nrec=9)
    rng = np.random.default_rng(seed + 100)
    dm = (0.05 * rng.standard_normal(n) * m.max()).astype(np.float32)
    dt = 0.4 * wavelib.cfl_dt(so, (inputs.H,) * 3, 3.0)
    grid = wavelib.Grid(n, (inputs.H,) * 3, dt, nt, so)
    return grid, m, damp, dm, src, q, rec


@pytest.mark.parametrize("so", [2, 4, 6, 8, 10, 12, 14, 16])
def test_born_vs_oracle(wavelib, cuda, oracle, so):
    n = (37, 41, 35)
    nt = 30
    grid, m, damp, dm, src, q, rec = _setup(wavelib, n, so, nt, 50 + so)
    dd, du, ws = wavelib.born(grid, _t(m, cuda), _t(damp, cuda), _t(dm, cuda), src, _t(q, cuda), rec,
                              want_du_last=True)
    assert wavelib.status(ws) == wavelib.WAVE_OK
    h = [float(np.float32(v)) for v in grid.h]
    ddr, dur = oracle.born(_f64(m), _f64(damp), _f64(dm), h, float(np.float32(grid.dt)), nt, so, _f64(src),
                           _f64(q), _f64(rec))
    dd2, du2, ws2 = wavelib.born(grid, _t(m, cuda), _t(damp, cuda), _t(dm, cuda), src, _t(q, cuda), rec,
                                 want_du_last=True, tuning=wavelib.Tuning(flags=wavelib.WAVE_BORN_TWO_SWEEPS))
    assert wavelib.status(ws2) == wavelib.WAVE_OK
    import torch
    torch.cuda.synchronize()
    assert torch.equal(dd, dd2) and torch.equal(du, du2)
    dd, du = dd.cpu().numpy(), du.cpu().numpy()
    assert np.abs(ddr).max() > 0
    assert np.abs(dd - ddr).max() <= TOL * np.abs(ddr).max()
    for k in range(2):
        err = np.linalg.norm(_f64(du[k]) - dur[k]) / np.linalg.norm(dur[k])
        assert err <= TOL, (k, err)


def test_born_adjoint_is_wave_grad(wavelib, cuda):
    import torch
    so, n, nt, k = 8, (34, 30, 33), 36, 6
    grid, m, damp, dm, src, q, rec = _setup(wavelib, n, so, nt, 9)
    r = np.random.default_rng(3).standard_normal((nt, len(rec))).astype(np.float32)
    tm, td, tq = _t(m, cuda), _t(damp, cuda), _t(q, cuda)
    dd, _, _ = wavelib.born(grid, tm, td, _t(dm, cuda), src, tq, rec)
    _, _, ck, _ = wavelib.fwd(grid, tm, td, src, tq, None, ckpt_every=k)
    g, _ = wavelib.grad(grid, tm, td, src, tq, rec, _t(r, cuda), ck, k)
    torch.cuda.synchronize()
    lhs = float(np.sum(_f64(dd.cpu().numpy()) * _f64(r)))
    rhs = float(np.sum(_f64(dm) * _f64(g.cpu().numpy())))
    assert abs(lhs - rhs) <= TOL * max(abs(lhs), abs(rhs)), (lhs, rhs)


def test_born_linear_and_plan_independent(wavelib, cuda):
    import torch
    so, n, nt = 4, (40, 36, 42), 25
    grid, m, damp, dm, src, q, rec = _setup(wavelib, n, so, nt, 4)
    tm, td, tq = _t(m, cuda), _t(damp, cuda), _t(q, cuda)
    d1, u1, _ = wavelib.born(grid, tm, td, _t(dm, cuda), src, tq, rec, want_du_last=True)
    d2, u2, _ = wavelib.born(grid, tm, td, _t(2 * dm, cuda), src, tq, rec, want_du_last=True)
    torch.cuda.synchronize()
    assert float((d2 - 2 * d1).abs().max()) <= 1e-6 * float(d2.abs().max())
    assert float((u2 - 2 * u1).abs().max()) <= 1e-6 * float(u2.abs().max())
    for tune in (wavelib.Tuning(time_tile=1, kernel=wavelib.WAVE_KERNEL_SHARED),
                 wavelib.Tuning(time_tile=2, kernel=wavelib.WAVE_KERNEL_STAGED)):
        d3, u3, _ = wavelib.born(grid, tm, td, _t(dm, cuda), src, tq, rec, tuning=tune, want_du_last=True)
        torch.cuda.synchronize()
        assert torch.equal(d3, d1) and torch.equal(u3, u1)

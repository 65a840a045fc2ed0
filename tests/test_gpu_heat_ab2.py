"""GPU parity of the two-step Adams-Bashforth Laplace operator
(wave_heat_ab2; a time dependence of two levels) through the C ABI.

* so 2, 4, 8, 16 against the FP64 oracle: rel-L2 of u^nt <= 1e-5, receiver
  traces within 1e-5 of max |d|, untiled and at depth 2 (an odd step count
  ends with an untiled step);
* the depth-2 sweep equals the untiled one bit for bit, field and traces
  (the depth-2 launch records the level between its steps from registers),
  for x-chunks shorter than the stencil reach and for the whole grid;
* one step agrees with wave_heat's Euler step to rounding;
* the stability check at dt kappa |L| > 1.
"""
import numpy as np
import pytest

import oracle
from paper_1806_08299_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5
H = (inputs.H,) * 3


def _t(x, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev)


def _lmax(so):
    lam = oracle.symbol_max(oracle.fd2_central_weights(so))
    return sum(lam / (float(np.float32(h)) ** 2) for h in H)


def _problem(so, nt, seed):
    rng = np.random.default_rng(seed)
    n = (38, 41, 45)
    u0 = rng.standard_normal(n).astype(np.float32)
    kappa = (0.5 + rng.random(n)).astype(np.float32)
    dt = float(np.float32(0.4 / (1.5 * _lmax(so))))  # within dt kappa |L| <= 1
    ext = np.array([(k - 1) * inputs.H for k in n])
    src = (rng.random((2, 3)) * ext).astype(np.float32)
    rec = (rng.random((6, 3)) * ext).astype(np.float32)
    q = rng.standard_normal((nt, 2)).astype(np.float32)
    return n, u0, kappa, dt, src, rec, q


@pytest.mark.parametrize("so,nt", [(2, 20), (4, 21), (8, 20), (16, 13)])
def test_ab2_vs_oracle_and_untiled(wavelib, cuda, so, nt):
    import torch
    n, u0, kappa, dt, src, rec, q = _problem(so, nt, seed=so + 7)
    grid = wavelib.Grid(n, H, dt, nt, so)
    h = [float(np.float32(v)) for v in grid.h]
    args = (np.float64(u0), h, float(np.float32(dt)), nt, so)
    dref, uref = oracle.heat_ab2(*args, kappa=np.float64(kappa), src_xyz=np.float64(src), src_q=np.float64(q),
                                 rec_xyz=np.float64(rec))
    # untiled, with receivers
    u1, d1, ws = wavelib.heat_ab2(grid, _t(u0, cuda), _t(kappa, cuda), src, _t(q, cuda), rec,
                                  tuning=wavelib.Tuning(time_tile=1))
    assert wavelib.status(ws) == wavelib.WAVE_OK
    torch.cuda.synchronize()
    u1n, d1n = u1.cpu().numpy(), d1.cpu().numpy()
    err = float(np.linalg.norm(u1n.astype(np.float64) - uref) / np.linalg.norm(uref))
    assert err <= TOL, err
    assert np.abs(d1n - dref).max() <= TOL * np.abs(dref).max()
    # depth 2 where compiled, bitwise the untiled sweep (field and traces)
    for tile_x in (0, 5, 13, n[0]):
        ub, db, ws = wavelib.heat_ab2(grid, _t(u0, cuda), _t(kappa, cuda), src, _t(q, cuda), rec,
                                      tuning=wavelib.Tuning(time_tile=2, tile_x=tile_x))
        assert wavelib.status(ws) == wavelib.WAVE_OK
        torch.cuda.synchronize()
        assert torch.equal(u1, ub) and torch.equal(d1, db), tile_x


def test_ab2_first_step_is_euler(wavelib, cuda):
    import torch
    so = 8
    n, u0, kappa, dt, src, rec, q = _problem(so, 1, seed=2)
    grid = wavelib.Grid(n, H, dt, 1, so)
    ua, da, _ = wavelib.heat_ab2(grid, _t(u0, cuda), _t(kappa, cuda), src, _t(q, cuda), rec)
    ue, de, _ = wavelib.heat(grid, _t(u0, cuda), _t(kappa, cuda), src, _t(q, cuda), rec,
                             tuning=wavelib.Tuning(time_tile=1))
    torch.cuda.synchronize()
    # the Euler step is u + C (L u + f) in both; the sweeps add the source to
    # the rate (Adams-Bashforth) or to the level (Euler), so they agree to rounding
    assert float((ua - ue).abs().max()) <= 1e-6 * float(ue.abs().max())
    assert float((da - de).abs().max()) <= 1e-6 * float(de.abs().max())


def test_ab2_stability_check(wavelib, cuda):
    import torch
    so, nt = 4, 4
    n, u0, kappa, _, src, rec, q = _problem(so, nt, seed=3)
    dt = float(np.float32(1.2 / (1.5 * _lmax(so))))  # dt kappa |L| up to 1.2 where kappa is largest
    grid = wavelib.Grid(n, H, dt, nt, so)
    _, _, ws = wavelib.heat_ab2(grid, _t(u0, cuda), _t(kappa, cuda), src, _t(q, cuda), rec)
    assert wavelib.status(ws) == wavelib.WAVE_EUNSTABLE
    u, _, ws = wavelib.heat_ab2(grid, _t(u0, cuda), _t(kappa, cuda), src, _t(q, cuda), rec,
                                tuning=wavelib.Tuning(flags=wavelib.WAVE_ALLOW_UNSTABLE))
    assert wavelib.status(ws) == wavelib.WAVE_OK
    torch.cuda.synchronize()
    assert np.all(np.isfinite(u.cpu().numpy()))

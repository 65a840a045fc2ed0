"""GPU parity of the Laplace (heat) operator (wave_heat, Sec. 5.7) through
the C ABI: explicit Euler for u_t = kappa (lap u + f) on the time-tiled
sweep (B = 0, C = dt kappa).

* every space order with a time-tiled shape and every compiled depth, against
  the FP64 oracle: rel-L2 of u^nt <= 1e-5, receiver traces within 1e-5 of
  max |d|; time-tiled == untiled bit for bit;
* the stability check: dt past 2 / (kappa |L|) is reported as
  WAVE_EUNSTABLE, and runs when WAVE_ALLOW_UNSTABLE is set.
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
    dt = float(np.float32(0.4 * 2.0 / (1.5 * _lmax(so))))
    ext = np.array([(k - 1) * inputs.H for k in n])
    src = (rng.random((2, 3)) * ext).astype(np.float32)
    rec = (rng.random((6, 3)) * ext).astype(np.float32)
    q = rng.standard_normal((nt, 2)).astype(np.float32)
    return n, u0, kappa, dt, src, rec, q


def _depths(wavelib, so):
    return sorted({v["time_tile"] for v in wavelib.list_variants(so)})


@pytest.mark.parametrize("so", [2, 4, 8, 16])
def test_heat_vs_oracle_and_untiled(wavelib, cuda, so):
    import torch
    nt = 20
    n, u0, kappa, dt, src, rec, q = _problem(so, nt, seed=so)
    grid = wavelib.Grid(n, H, dt, nt, so)
    h = [float(np.float32(v)) for v in grid.h]
    dref, uref = oracle.heat(np.float64(u0), h, float(np.float32(dt)), nt, so, kappa=np.float64(kappa),
                             src_xyz=np.float64(src), src_q=np.float64(q), rec_xyz=np.float64(rec))
    out = {}
    for T in _depths(wavelib, so):
        u, d, ws = wavelib.heat(grid, _t(u0, cuda), _t(kappa, cuda), src, _t(q, cuda), rec,
                                tuning=wavelib.Tuning(time_tile=T))
        assert wavelib.status(ws) == wavelib.WAVE_OK
        torch.cuda.synchronize()
        out[T] = (u.cpu().numpy(), d.cpu().numpy())
        err = float(np.linalg.norm(out[T][0].astype(np.float64) - uref) / np.linalg.norm(uref))
        assert err <= TOL, (T, err)
        assert np.abs(out[T][1] - dref).max() <= TOL * np.abs(dref).max()
    for T in out:
        assert np.array_equal(out[T][0], out[1][0]) and np.array_equal(out[T][1], out[1][1])


def test_heat_stability_check(wavelib, cuda):
    import torch
    so, nt = 8, 4
    n, u0, kappa, _, src, rec, q = _problem(so, nt, seed=3)
    dt = float(np.float32(1.2 * 2.0 / (1.5 * _lmax(so))))  # past the limit where kappa is largest
    grid = wavelib.Grid(n, H, dt, nt, so)
    _, _, ws = wavelib.heat(grid, _t(u0, cuda), _t(kappa, cuda), src, _t(q, cuda), rec,
                            tuning=wavelib.Tuning(time_tile=1))
    assert wavelib.status(ws) == wavelib.WAVE_EUNSTABLE
    u, _, ws = wavelib.heat(grid, _t(u0, cuda), _t(kappa, cuda), src, _t(q, cuda), rec,
                            tuning=wavelib.Tuning(time_tile=1, flags=wavelib.WAVE_ALLOW_UNSTABLE))
    assert wavelib.status(ws) == wavelib.WAVE_OK
    torch.cuda.synchronize()
    assert np.all(np.isfinite(u.cpu().numpy()))

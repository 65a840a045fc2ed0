"""Pins of the oracle's two-step Adams-Bashforth Laplace operator
(u_t = kappa (lap u + f), a time dependence of two levels).

* so 2: a discrete Dirichlet sine mode is an eigenvector of the zero-halo
  Laplacian (eigenvalue lambda), so u^n = s_n u^0 with s_n the solution of
  the scheme's two-step recurrence s_{n+1} = (1 + 3/2 mu) s_n - 1/2 mu s_{n-1}
  (mu = dt kappa lambda, s_0 = 1, s_1 = 1 + mu), written here in closed form
  from the roots of its characteristic polynomial z^2 - (1 + 3/2 mu) z + mu/2;
* the same mode against the exact decay exp(kappa lambda t) of the
  semi-discrete equation: the error at a fixed time falls by about 4 when dt
  is halved (second order; an Euler-like mistake in the weights falls by 2);
* one step is the Euler step of the (separately pinned) heat oracle, bit for
  bit;
* linearity in (u0, q).
"""
import numpy as np
import pytest

import oracle

H = (0.01, 0.012, 0.02)


def _mode(n, k):
    ax = [np.sin(np.pi * k[a] * (np.arange(n[a]) + 1) / (n[a] + 1)) for a in range(3)]
    u0 = ax[0][:, None, None] * ax[1][None, :, None] * ax[2][None, None, :]
    lam = sum((2 * np.cos(np.pi * k[a] / (n[a] + 1)) - 2) / H[a] ** 2 for a in range(3))
    return u0, lam


def _closed_form(mu, nt):
    b = 1 + 1.5 * mu
    disc = np.sqrt(complex(b * b - 2 * mu))
    z1, z2 = (b + disc) / 2, (b - disc) / 2
    # s_n = A z1^n + B z2^n with s_0 = 1, s_1 = 1 + mu
    A = ((1 + mu) - z2) / (z1 - z2)
    B = 1 - A
    return (A * z1 ** nt + B * z2 ** nt).real


@pytest.mark.parametrize("frac,nt", [(0.1, 9), (0.25, 12), (0.45, 7)])
def test_sine_mode_closed_form_so2(frac, nt):
    n = (13, 11, 9)
    u0, lam = _mode(n, (2, 3, 1))
    dt = frac * 2 / sum(4 / h ** 2 for h in H)
    _, u = oracle.heat_ab2(u0, H, dt, nt, 2)
    want = _closed_form(dt * lam, nt) * u0
    assert np.abs(u - want).max() <= 1e-12 * np.abs(u0).max()


def test_second_order_in_dt():
    n = (13, 11, 9)
    u0, lam = _mode(n, (3, 2, 1))
    # the longest step within the scheme's stability limit for every mode
    # (rounding excites all of them), then halved twice
    t_end = 40 * 0.8 / sum(4 / h ** 2 for h in H)
    errs = []
    for nt in (40, 80, 160):
        dt = t_end / nt
        _, u = oracle.heat_ab2(u0, H, dt, nt, 2)
        errs.append(np.abs(u - np.exp(lam * t_end) * u0).max())
    for a, b in zip(errs, errs[1:]):
        assert 3.6 < a / b < 4.4, errs


def test_first_step_is_the_euler_step():
    rng = np.random.default_rng(5)
    n = (12, 14, 10)
    u0 = rng.standard_normal(n)
    kappa = 0.5 + rng.random(n)
    src = [[0.05, 0.06, 0.07]]
    q = rng.standard_normal((1, 1))
    rec = [[0.03, 0.04, 0.05], [0.09, 0.1, 0.11]]
    for so in (2, 8):
        dt = 0.2 / sum(4 / h ** 2 for h in H)
        da, ua = oracle.heat_ab2(u0, H, dt, 1, so, kappa=kappa, src_xyz=src, src_q=q, rec_xyz=rec)
        de, ue = oracle.heat(u0, H, dt, 1, so, kappa=kappa, src_xyz=src, src_q=q, rec_xyz=rec)
        assert np.array_equal(ua, ue) and np.array_equal(da, de)


def test_linearity():
    rng = np.random.default_rng(8)
    n = (10, 11, 12)
    nt = 9
    dt = 0.2 / sum(4 / h ** 2 for h in H)
    src = [[0.04, 0.05, 0.06]]
    rec = [[0.02, 0.03, 0.04]]
    a0, b0 = rng.standard_normal(n), rng.standard_normal(n)
    qa, qb = rng.standard_normal((nt, 1)), rng.standard_normal((nt, 1))
    da, ua = oracle.heat_ab2(a0, H, dt, nt, 4, src_xyz=src, src_q=qa, rec_xyz=rec)
    db, ub = oracle.heat_ab2(b0, H, dt, nt, 4, src_xyz=src, src_q=qb, rec_xyz=rec)
    ds, us = oracle.heat_ab2(2 * a0 + b0, H, dt, nt, 4, src_xyz=src, src_q=2 * qa + qb, rec_xyz=rec)
    assert np.abs(us - (2 * ua + ub)).max() <= 1e-12 * np.abs(us).max()
    assert np.abs(ds - (2 * da + db)).max() <= 1e-12 * np.abs(ds).max()

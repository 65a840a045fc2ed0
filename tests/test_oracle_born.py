"""Pins for the oracle's Born (linearised) modelling.

Born modelling is the derivative of the forward map m -> d in a direction
dm.  It is pinned against things other than itself:
* central finite differences of the (separately pinned) forward oracle, whose
  error must fall as eps^2;
* the dot-product identity with the (separately pinned) gradient oracle:
  <B dm, r> = <dm, g(r)>, g(r) = dJ/dm of J = <r, d>, since g is B^T r;
* linearity: B(2 dm) = 2 B(dm) bit for bit, B(0) = 0.
"""
import numpy as np
import pytest


def _problem(so, n, seed, damp_scale=2.0):
    rng = np.random.default_rng(seed)
    h = (0.01, 0.011, 0.009)
    m = 0.25 + 0.2 * rng.random(n)
    damp = damp_scale * rng.random(n)
    return rng, h, m, damp


def _ricker(nt, dt, f0=40.0, t0=0.025):
    t = np.arange(nt) * dt
    a = (np.pi * f0 * (t - t0)) ** 2
    return ((1 - 2 * a) * np.exp(-a))[:, None]


@pytest.mark.parametrize("so", [4, 8])
def test_born_is_the_derivative_of_forward(oracle, so):
    n = (15, 14, 13)
    rng, h, m, damp = _problem(so, n, 3 + so)
    nt, dt = 50, 1e-3
    src = [[0.07, 0.07, 0.03]]
    rec = [[0.02 + 0.012 * i, 0.08, 0.09] for i in range(7)]
    q = _ricker(nt, dt)
    dm = rng.standard_normal(n)
    dm *= 0.05 * np.abs(m).max() / np.abs(dm).max()
    dd, _ = oracle.born(m, damp, dm, h, dt, nt, so, src, q, rec)
    errs = []
    for eps in (1e-1, 5e-2):
        dp, _, _ = oracle.forward(m + eps * dm, damp, h, dt, nt, so, src_xyz=src, src_q=q, rec_xyz=rec)
        dn, _, _ = oracle.forward(m - eps * dm, damp, h, dt, nt, so, src_xyz=src, src_q=q, rec_xyz=rec)
        fd = (dp - dn) / (2 * eps)
        errs.append(np.abs(fd - dd).max())
    scale = np.abs(dd).max()
    assert scale > 0
    assert errs[1] <= 1e-3 * scale
    # second order: halving eps divides the error by about 4
    assert 3.0 < errs[0] / errs[1] < 5.0


@pytest.mark.parametrize("so,n", [(2, (9, 10, 8)), (8, (13, 12, 11)), (16, (17, 18, 17))])
def test_born_dot_gradient(oracle, so, n):
    rng, h, m, damp = _problem(so, n, 20 + so, damp_scale=4.0)
    nt, dt = 30, 1e-3
    src = rng.random((2, 3)) * np.array(n) * np.array(h) * 0.9
    rec = rng.random((6, 3)) * np.array(n) * np.array(h) * 0.9
    q = rng.standard_normal((nt, 2))
    r = rng.standard_normal((nt, 6))
    dm = rng.standard_normal(n)
    dd, _ = oracle.born(m, damp, dm, h, dt, nt, so, src, q, rec)
    g = oracle.gradient(m, damp, h, dt, nt, so, src, q, rec, r)
    lhs = float(np.sum(dd * r))
    rhs = float(np.sum(dm * g))
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), abs(rhs))


def test_born_linear_in_dm(oracle):
    so, n = 4, (11, 10, 12)
    rng, h, m, damp = _problem(so, n, 7)
    nt, dt = 20, 1e-3
    src = [[0.05, 0.05, 0.05]]
    rec = [[0.02, 0.03, 0.04], [0.08, 0.07, 0.06]]
    q = rng.standard_normal((nt, 1))
    dm = rng.standard_normal(n)
    d1, u1 = oracle.born(m, damp, dm, h, dt, nt, so, src, q, rec)
    d2, u2 = oracle.born(m, damp, 2.0 * dm, h, dt, nt, so, src, q, rec)
    assert np.array_equal(d2, 2.0 * d1) and np.array_equal(u2, 2.0 * u1)
    d0, u0 = oracle.born(m, damp, np.zeros(n), h, dt, nt, so, src, q, rec)
    assert not d0.any() and not u0.any()
    assert np.abs(d1).max() > 0

"""Pins for the oracle's adjoint and gradient.

The adjoint is checked by the dot-product test against the forward and by the
time-reversal identity (the transposed recursion, rescaled, is the forward
scheme run with the residual as its source); the gradient by central finite
differences of the misfit, whose error must fall as eps^2.
"""
import numpy as np
import pytest


def _problem(so, n, seed, damp_scale=4.0):
    rng = np.random.default_rng(seed)
    h = (0.01, 0.011, 0.009)
    m = 0.25 + 0.2 * rng.random(n)
    damp = damp_scale * rng.random(n)
    return rng, h, m, damp


@pytest.mark.parametrize("so,n", [(2, (9, 8, 7)), (4, (11, 10, 9)), (8, (13, 12, 11)),
                                  (12, (15, 14, 13)), (16, (17, 18, 17))])
def test_dot_product(oracle, so, n):
    rng, h, m, damp = _problem(so, n, so)
    nt = 25
    dt = 1e-3
    src = rng.random((3, 3)) * np.array(n) * np.array(h) * 0.9
    rec = rng.random((5, 3)) * np.array(n) * np.array(h) * 0.9
    q = rng.standard_normal((nt, 3))
    res = rng.standard_normal((nt, 5))
    d, _, _ = oracle.forward(m, damp, h, dt, nt, so, src_xyz=src, src_q=q, rec_xyz=rec)
    sg, _ = oracle.adjoint(m, damp, h, dt, nt, so, rec, res, src_xyz=src)
    lhs = float(np.sum(d * res))
    rhs = float(np.sum(q * sg))
    assert abs(lhs) > 0
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("so", [4, 8])
def test_adjoint_is_forward_reversed(oracle, so):
    # nu^k = dt^2 alpha lambda^k obeys the forward scheme run backwards with the
    # residual injected at the receivers:  forward(src = rec, q^j = res^{nt-1-j})
    # ends at nu^1.
    n = (12, 11, 10)
    rng, h, m, damp = _problem(so, n, 7 + so)
    nt, dt = 30, 1e-3
    rec = rng.random((4, 3)) * np.array(n) * np.array(h) * 0.9
    res = rng.standard_normal((nt, 4))
    _, lam = oracle.adjoint(m, damp, h, dt, nt, so, rec, res)
    alpha = 1.0 / (m + damp * dt / 2)
    _, ul, _ = oracle.forward(m, damp, h, dt, nt, so, src_xyz=rec, src_q=res[::-1])
    nu1 = dt * dt * alpha * lam[0]
    nu2 = dt * dt * alpha * lam[1]
    assert np.abs(ul[0] - nu1).max() <= 1e-12 * np.abs(nu1).max()
    assert np.abs(ul[1] - nu2).max() <= 1e-12 * np.abs(nu2).max()


def test_gradient_finite_differences(oracle):
    so = 8
    n = (16, 15, 14)
    rng, h, m, damp = _problem(so, n, 11, damp_scale=2.0)
    nt, dt = 60, 1e-3
    src = [[0.08, 0.07, 0.03]]
    rec = [[0.03 + 0.01 * i, 0.08, 0.1] for i in range(8)]
    t = np.arange(nt) * dt
    q = ((1 - 2 * (np.pi * 40 * (t - 0.025)) ** 2)
         * np.exp(-(np.pi * 40 * (t - 0.025)) ** 2))[:, None]
    m_true = m.copy()
    m_true[6:10, 6:10, 5:9] *= 1.1
    d_obs, _, _ = oracle.forward(m_true, damp, h, dt, nt, so, src_xyz=src, src_q=q, rec_xyz=rec)

    def misfit(mm):
        d, _, _ = oracle.forward(mm, damp, h, dt, nt, so, src_xyz=src, src_q=q, rec_xyz=rec)
        return 0.5 * float(np.sum((d - d_obs) ** 2)), d

    j0, d0 = misfit(m)
    g = oracle.gradient(m, damp, h, dt, nt, so, src, q, rec, d0 - d_obs)
    for k in range(3):
        dm = rng.standard_normal(n)
        dm *= 0.01 * np.abs(m).max() / np.abs(dm).max()
        want = float(np.sum(g * dm))
        errs = []
        for eps in (1e-2, 5e-3):
            jp, _ = misfit(m + eps * dm)
            jm, _ = misfit(m - eps * dm)
            fd = (jp - jm) / (2 * eps)
            errs.append(abs(fd - want))
        assert errs[1] <= 1e-5 * abs(want)
        # second-order: halving eps divides the error by ~4
        assert errs[0] / errs[1] > 3.0

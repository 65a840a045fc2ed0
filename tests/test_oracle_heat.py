"""Pins of the oracle's Laplace (heat) operator, Sec. 5.7: explicit Euler
for u_t = kappa (lap u + f) with the zero-halo order-so Laplacian.

* so 2: a discrete Dirichlet sine mode is an eigenvector of the 7-point
  Laplacian with the zero halo, so nt steps scale it by (1 + dt lambda)^nt
  exactly, lambda = sum_a (2 cos(pi k_a / (n_a + 1)) - 2) / h_a^2;
* every order: L is exact on quadratics, so one step from x^2 + y^2 + z^2
  adds dt kappa 6 at every point at least r cells from the boundary;
* a source on a grid node adds dt kappa q there and nowhere else, and a
  receiver on that node records it;
* linearity in (u0, q).
"""
import numpy as np
import pytest

import oracle

H = (0.01, 0.012, 0.02)


def _lmax(so):
    """Largest |eigenvalue| of the zero-halo Laplacian's symbol over all modes."""
    lam = oracle.symbol_max(oracle.fd2_central_weights(so))
    return sum(lam / (h * h) for h in H)


def test_sine_mode_decays_exactly_so2():
    n = (13, 11, 9)
    k = (2, 3, 1)
    ax = [np.sin(np.pi * k[a] * (np.arange(n[a]) + 1) / (n[a] + 1)) for a in range(3)]
    u0 = ax[0][:, None, None] * ax[1][None, :, None] * ax[2][None, None, :]
    lam = sum((2 * np.cos(np.pi * k[a] / (n[a] + 1)) - 2) / H[a] ** 2 for a in range(3))
    dt = 0.3 * 2 / sum(4 / h ** 2 for h in H)
    nt = 7
    _, u = oracle.heat(u0, H, dt, nt, 2)
    want = (1 + dt * lam) ** nt * u0
    assert np.abs(u - want).max() <= 1e-12 * np.abs(u0).max()
    # and the mode really decays (a sign error in the update would grow it)
    assert np.abs(u).max() < np.abs(u0).max()


@pytest.mark.parametrize("so", [2, 4, 8, 12, 16])
def test_quadratic_one_step_interior(so):
    n = (24, 22, 26)
    r = so // 2
    X, Y, Z = np.meshgrid(*[np.arange(n[a]) * H[a] for a in range(3)], indexing="ij")
    u0 = X ** 2 + Y ** 2 + Z ** 2
    kappa = 0.5 + np.random.default_rng(so).random(n)
    dt = 1e-6
    _, u1 = oracle.heat(u0, H, dt, 1, so, kappa=kappa)
    inner = tuple(slice(r, n[a] - r) for a in range(3))
    want = u0 + dt * kappa * 6.0
    assert np.abs(u1[inner] - want[inner]).max() <= 1e-12 * np.abs(want[inner]).max()
    # the boundary cells feel the zero halo: not the interior value there
    assert np.abs(u1[0] - want[0]).max() > 1e-9


def test_source_on_node_and_receiver():
    n = (9, 10, 11)
    node = (4, 6, 3)
    hp = (0.0078125, 0.015625, 0.03125)  # powers of two: node coordinates divide exactly
    xyz = np.array([[node[a] * hp[a] for a in range(3)]])
    q = np.array([[2.5], [0.0]])
    kappa = np.full(n, 0.75)
    dt = 1e-4
    d, u1 = oracle.heat(np.zeros(n), hp, dt, 1, 4, kappa=kappa, src_xyz=xyz, src_q=q[:1],
                        rec_xyz=xyz)
    want = np.zeros(n)
    want[node] = dt * 0.75 * 2.5
    assert np.array_equal(u1, want)
    assert d[0, 0] == want[node]


def test_linearity():
    rng = np.random.default_rng(4)
    n = (12, 10, 14)
    nt = 5
    so = 8
    dt = 0.2 * 2 / _lmax(so)
    ua, ub = rng.standard_normal(n), rng.standard_normal(n)
    src = rng.random((3, 3)) * (np.array(n) - 1) * np.array(H)
    qa, qb = rng.standard_normal((nt, 3)), rng.standard_normal((nt, 3))
    rec = rng.random((4, 3)) * (np.array(n) - 1) * np.array(H)
    da, a = oracle.heat(ua, H, dt, nt, so, src_xyz=src, src_q=qa, rec_xyz=rec)
    db, b = oracle.heat(ub, H, dt, nt, so, src_xyz=src, src_q=qb, rec_xyz=rec)
    dc, c = oracle.heat(2 * ua - 3 * ub, H, dt, nt, so, src_xyz=src, src_q=2 * qa - 3 * qb, rec_xyz=rec)
    assert np.abs(c - (2 * a - 3 * b)).max() <= 1e-12 * np.abs(c).max()
    assert np.abs(dc - (2 * da - 3 * db)).max() <= 1e-12 * np.abs(dc).max()

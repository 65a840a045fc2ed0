"""Pins for the oracle's Laplacian and leapfrog forward.

Each test checks the oracle against something it does not compute itself:
exact derivatives of polynomials, the measured order of convergence, the
closed-form discrete solution of a plane wave (undamped and damped), the
hand-derived first two steps after a point source, exactness of trilinear
receivers, linearity, and the paper's own tiled == untiled rule.
"""
import cmath
import math

import numpy as np
import pytest


def _grid_coords(n, h):
    return np.meshgrid(*[np.arange(n[a]) * h[a] for a in range(3)], indexing="ij")


@pytest.mark.parametrize("so", [2, 4, 6, 8, 12, 16])
def test_laplacian_exact_on_polynomials(oracle, so):
    # The 1D stencil is exact for degree <= 2r+1, so L is exact on
    # p(x) + q(y) + s(z) + x^a y^b z^c with each axis degree <= 2r+1.
    r = so // 2
    n = (2 * r + 7, 2 * r + 6, 2 * r + 5)
    h = (0.5, 0.4, 0.25)
    x, y, z = _grid_coords(n, h)
    x, y, z = x - 1.0, y - 1.0, z - 1.0
    deg = 2 * r + 1
    rng = np.random.default_rng(so)
    a = rng.standard_normal(3)
    u = (a[0] * x ** deg + a[1] * y ** (deg - 1) + a[2] * z ** deg
         + x ** 2 * y ** 3 * z + 0.5 * x * y)
    exact = (a[0] * deg * (deg - 1) * x ** (deg - 2)
             + a[1] * (deg - 1) * (deg - 2) * y ** (deg - 3)
             + a[2] * deg * (deg - 1) * z ** (deg - 2)
             + 2 * y ** 3 * z + 6 * x ** 2 * y * z)
    got = oracle.laplacian(u, h, so)
    inner = tuple(slice(r, n[i] - r) for i in range(3))
    scale = np.abs(exact[inner]).max()
    assert np.abs(got[inner] - exact[inner]).max() <= 1e-9 * scale


@pytest.mark.parametrize("so", [2, 4, 6, 8])
def test_laplacian_convergence_order(oracle, so):
    # Periodic sin field: the error falls by 2^so per halving of h.
    errs = []
    for npt in (16, 32):
        n = (npt, 4, 4)
        h = (1.0 / npt, 0.25, 0.25)
        x, _, _ = _grid_coords(n, h)
        u = np.sin(2 * math.pi * x)
        got = oracle.laplacian(u, h, so, periodic=True)
        errs.append(np.abs(got + 4 * math.pi ** 2 * u).max())
    rate = math.log2(errs[0] / errs[1])
    assert rate == pytest.approx(so, abs=0.15)


def _plane_wave_setup(so, damp_val):
    n = (12, 10, 8)
    h = (0.01, 0.012, 0.015)
    v = 2.0
    m_val = 1.0 / v ** 2
    kk = [2 * math.pi * j / (n[a] * h[a]) for a, j in enumerate((1, 2, 1))]
    c = oracle_coeffs = None  # noqa: F841
    return n, h, m_val, kk


def _total_symbol(oracle, so, kk, h):
    c = oracle.fd2_central_weights(so)
    return sum(oracle.symbol(c, kk[a] * h[a]) / h[a] ** 2 for a in range(3))


@pytest.mark.parametrize("so", [4, 8, 16])
def test_plane_wave_dispersion_undamped(oracle, so):
    # u^n = cos(k.x - w n dt) solves the scheme exactly when
    # sin^2(w dt / 2) = (v^2 dt^2 / 4) sum_a Lambda(k_a h_a) / h_a^2.
    n, h, m_val, kk = _plane_wave_setup(so, 0.0)
    v = 1.0 / math.sqrt(m_val)
    dt = 0.4 * oracle.cfl_dt(so, h, v)
    lam = _total_symbol(oracle, so, kk, h)
    w = 2.0 / dt * math.asin(math.sqrt(v * v * dt * dt / 4.0 * lam))
    x, y, z = _grid_coords(n, h)
    phase = kk[0] * x + kk[1] * y + kk[2] * z
    nt = 1000
    m = np.full(n, m_val)
    _, ul, _ = oracle.forward(m, np.zeros(n), h, dt, nt, so, periodic=True,
                              u0=np.cos(phase), um1=np.cos(phase + w * dt))
    want = np.cos(phase - w * nt * dt)
    assert np.abs(ul[0] - want).max() < 1e-9
    # and the continuum limit: w -> v |k| as dt and h shrink (sanity of scale)
    assert w == pytest.approx(v * math.sqrt(sum(k * k for k in kk)), rel=0.05)


@pytest.mark.parametrize("so", [4, 8])
def test_plane_wave_damped(oracle, so):
    # With uniform damp, a Fourier mode obeys
    #   (m + eta) z^2 - (2 m - dt^2 Lam) z + (m - eta) = 0,  eta = damp dt / 2,
    # so u^n = Re(z^n e^{i k.x}) exactly.  This pins the centred damping term.
    n, h, m_val, kk = _plane_wave_setup(so, 0.0)
    v = 1.0 / math.sqrt(m_val)
    dt = 0.4 * oracle.cfl_dt(so, h, v)
    damp_val = 30.0
    eta = damp_val * dt / 2
    lam = _total_symbol(oracle, so, kk, h)
    a2, a1, a0 = m_val + eta, -(2 * m_val - dt * dt * lam), m_val - eta
    disc = cmath.sqrt(a1 * a1 - 4 * a2 * a0)
    zr = (-a1 + disc) / (2 * a2)
    x, y, z = _grid_coords(n, h)
    e = np.exp(1j * (kk[0] * x + kk[1] * y + kk[2] * z))
    nt = 300
    m = np.full(n, m_val)
    _, ul, _ = oracle.forward(m, np.full(n, damp_val), h, dt, nt, so, periodic=True,
                              u0=e.real, um1=(e / zr).real)
    want = (e * zr ** nt).real
    assert abs(zr) < 1.0
    assert np.abs(ul[0] - want).max() < 1e-10
    assert np.abs(ul[1] - (e * zr ** (nt - 1)).real).max() < 1e-10


def test_first_two_steps_after_point_source(oracle):
    # Source on node p: u^1 = alpha dt^2 q^0 e_p; u^2(p) and u^2(p + k e_a) by hand.
    so, r = 4, 2
    n = (11, 12, 13)
    h = (0.01, 0.02, 0.025)
    dt = 1e-3
    m_val, d_val = 0.3, 5.0
    p = (5, 6, 7)
    q = np.array([[2.0], [-1.0], [0.5]])
    m = np.full(n, m_val)
    damp = np.full(n, d_val)
    xyz = [[p[0] * h[0], p[1] * h[1], p[2] * h[2]]]
    _, _, ua = oracle.forward(m, damp, h, dt, 2, so, src_xyz=xyz, src_q=q[:2], keep_all=True)
    eta = d_val * dt / 2
    alpha = 1 / (m_val + eta)
    u1 = alpha * dt * dt * q[0, 0]
    got1 = ua[2]
    assert got1[p] == pytest.approx(u1, rel=1e-14)
    assert np.count_nonzero(got1) == 1
    c = [float(v) for v in oracle.fd2_central_weights(so)]
    lap_p = sum(c[0] / ha ** 2 for ha in h) * u1
    want_p = alpha * (2 * m_val * u1 + dt * dt * (lap_p + q[1, 0]))
    got2 = ua[3]
    assert got2[p] == pytest.approx(want_p, rel=1e-13)
    for a in range(3):
        for k in range(1, r + 1):
            for sgn in (1, -1):
                idx = list(p)
                idx[a] += sgn * k
                want = alpha * dt * dt * c[k] / h[a] ** 2 * u1
                assert got2[tuple(idx)] == pytest.approx(want, rel=1e-13)
    assert np.count_nonzero(got2) == 1 + 6 * r


def test_receivers_trilinear_and_time_alignment(oracle):
    # d^n records u^{n+1}: on a node it is the node value; at a cell centre it is
    # the mean of the 8 corners; on the upper face it is the face node.
    so = 4
    n = (10, 9, 8)
    h = (0.125, 0.125, 0.125)  # binary-exact spacing so node coordinates are exact
    rng = np.random.default_rng(3)
    m = 0.4 + 0.05 * rng.random(n)
    damp = rng.random(n)
    dt = 1e-2
    nt = 12
    src = [[4.5 * h[0], 4.1 * h[1], 3.3 * h[2]]]
    q = rng.standard_normal((nt, 1))
    rec = [[3 * h[0], 4 * h[1], 5 * h[2]], [3.5 * h[0], 4.5 * h[1], 5.5 * h[2]],
           [9 * h[0], 8 * h[1], 7 * h[2]]]
    d, _, ua = oracle.forward(m, damp, h, dt, nt, so, src_xyz=src, src_q=q, rec_xyz=rec,
                              keep_all=True)
    for s in range(nt):
        u = ua[s + 2]
        assert d[s, 0] == u[3, 4, 5]
        assert d[s, 1] == pytest.approx(u[3:5, 4:6, 5:7].mean(), rel=1e-12, abs=1e-30)
        assert d[s, 2] == u[9, 8, 7]
    assert np.all(d[-1] != 0)


def test_linearity_and_zero(oracle):
    so = 8
    n = (14, 13, 12)
    h = (0.01,) * 3
    rng = np.random.default_rng(5)
    m = 0.3 + 0.1 * rng.random(n)
    damp = 2 * rng.random(n)
    q = rng.standard_normal((20, 2))
    src = [[0.06, 0.05, 0.07], [0.031, 0.072, 0.044]]
    d1, u1, _ = oracle.forward(m, damp, h, 1e-3, 20, so, src_xyz=src, src_q=q)
    d2, u2, _ = oracle.forward(m, damp, h, 1e-3, 20, so, src_xyz=src, src_q=2 * q)
    assert np.array_equal(u2, 2 * u1)  # scaling by 2 is exact in binary FP
    assert np.array_equal(d2, 2 * d1) if d1.size else True
    _, u0, _ = oracle.forward(m, np.zeros(n), h, 1e-3, 20, so)
    assert not np.any(u0)
    assert np.all(np.isfinite(u1)) and np.any(u1)


@pytest.mark.parametrize("so,tt,bx,by", [(2, 2, 3, 5), (4, 3, 7, 4), (8, 5, 9, 6),
                                         (12, 2, 4, 11), (16, 4, 16, 3), (8, 1, 5, 5),
                                         (4, 16, 40, 40)])
def test_tiled_equals_untiled_bitwise(oracle, so, tt, bx, by):
    # The paper's correctness rule: the skewed time-tiled loop nest gives
    # bitwise the same field as the untiled loop (Sec. 4.3, Sec. 5.4.3).
    n = (13, 11, 9)
    h = (0.01, 0.011, 0.012)
    rng = np.random.default_rng(so * 100 + tt)
    m = 0.2 + 0.3 * rng.random(n)
    damp = 3 * rng.random(n)
    nt = 17
    src = [[0.05, 0.06, 0.04], [0.05, 0.06, 0.04], [0.1, 0.02, 0.09]]
    q = rng.standard_normal((nt, 3))
    rec = [[0.02, 0.03, 0.04], [0.12, 0.11, 0.096], [0.07, 0.05, 0.031]]
    d, ul, _ = oracle.forward(m, damp, h, 1e-3, nt, so, src_xyz=src, src_q=q, rec_xyz=rec)
    dt_, ult = oracle.forward_tiled(m, damp, h, 1e-3, nt, so, src_xyz=src, src_q=q,
                                    rec_xyz=rec, tt=tt, bx=bx, by=by)
    assert np.any(ul[0]) and np.all(np.isfinite(ul))
    assert np.array_equal(ul, ult)
    assert np.array_equal(d, dt_)

"""Pins for the oracle's stencil coefficients and stability limit.

The oracle solves the polynomial-exactness system (oracle/coeffs.py).  These
tests check it against things that system does not contain: a published table,
two independent closed forms, the order of accuracy of the Fourier symbol, and
the closed-form von Neumann limit.
"""
import math
import os
from fractions import Fraction

import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fd2_central_weights.txt")
ORDERS = [2, 4, 6, 8, 10, 12, 14, 16]


def _golden():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows[int(parts[0])] = [Fraction(p) for p in parts[1:]]
    return rows


def test_matches_published_table(oracle):
    rows = _golden()
    assert sorted(rows) == [2, 4, 6, 8]
    for so, want in rows.items():
        assert oracle.fd2_central_weights(so) == want


@pytest.mark.parametrize("so", ORDERS)
def test_closed_form_weights(oracle, so):
    # c_k = 2 (-1)^(k+1) (r!)^2 / (k^2 (r-k)! (r+k)!),  c_0 = -2 sum_{k<=r} 1/k^2
    r = so // 2
    c = oracle.fd2_central_weights(so)
    assert len(c) == r + 1
    f = math.factorial
    for k in range(1, r + 1):
        want = Fraction(2 * (-1) ** (k + 1) * f(r) ** 2, k * k * f(r - k) * f(r + k))
        assert c[k] == want
    assert c[0] == -2 * sum(Fraction(1, k * k) for k in range(1, r + 1))


@pytest.mark.parametrize("so", ORDERS)
def test_symbol_order_of_accuracy(oracle, so):
    # Lambda(theta) - theta^2 = K theta^(2r+2) + O(theta^(2r+4)) with K != 0:
    # the scaled error must tend to a nonzero constant as theta -> 0.
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 80
    c = [mp.mpf(v.numerator) / v.denominator for v in oracle.fd2_central_weights(so)]
    r = so // 2

    def lam(t):
        return -c[0] - 2 * sum(c[k] * mp.cos(k * t) for k in range(1, r + 1))

    e = [(lam(t) - t * t) / t ** (2 * r + 2) for t in (mp.mpf("1e-3"), mp.mpf("5e-4"))]
    assert abs(e[0]) > mp.mpf("1e-12")
    assert abs(e[0] - e[1]) / abs(e[1]) < mp.mpf("1e-5")


@pytest.mark.parametrize("so", ORDERS)
def test_symbol_max_at_nyquist(oracle, so):
    # The symbol is largest at theta = pi, where it equals -c_0 - 2 sum (-1)^k c_k.
    c = oracle.fd2_central_weights(so)
    at_pi = float(-c[0] - 2 * sum(c[k] * (-1) ** k for k in range(1, len(c))))
    assert oracle.symbol_max(c) == pytest.approx(at_pi, rel=1e-12)


def test_cfl_closed_form(oracle):
    # so=2: Lambda(pi) = 4, dt = 2 / (v sqrt(sum 4/h_a^2)).
    h = (0.01, 0.012, 0.015)
    want = 2.0 / (2.0 * math.sqrt(sum(4.0 / (a * a) for a in h)))
    assert oracle.cfl_dt(2, h, 2.0) == pytest.approx(want, rel=1e-12)
    # so=4: Lambda(pi) = 16/3, equal spacing: dt = 2h / (v sqrt(16)) = h / (2 v).
    assert oracle.cfl_dt(4, (0.01,) * 3, 1.5) == pytest.approx(0.01 / 3.0, rel=1e-12)

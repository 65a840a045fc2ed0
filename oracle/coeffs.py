"""Stencil coefficients and stability limit, exact, for the CPU oracle.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product library.

The paper only says the stencils follow from Taylor's theorem (Sec. 2.1,
"Terminology") with space orders 4..16 (Sec. 5.8.1) and radius r = so/2 (the
minimum skew factors of Table "AWE results", Sec. 5.8.2).  The oracle takes the plain definition of an order-2r central
second difference: the symmetric weights c_0..c_r that differentiate every
polynomial of degree <= 2r + 1 exactly.  Odd powers vanish by symmetry, so the
conditions on x^(2j), j = 0..r, give an (r+1)x(r+1) linear system that is
solved here in exact rational arithmetic by Gaussian elimination.
"""
from fractions import Fraction
import math


def fd2_central_weights(space_order):
    """Exact c_0..c_r (unit spacing) for the order-`space_order` central
    second derivative  u''(0) ~ c_0 u(0) + sum_k c_k (u(k) + u(-k)).

    Conditions, for u = x^(2j):
      j = 0:   c_0 + 2 sum_k c_k          = 0
      j >= 1:  2 sum_k c_k k^(2j)         = (2 if j == 1 else 0)
    """
    if space_order < 2 or space_order % 2:
        raise ValueError("space order must be even and >= 2")
    r = space_order // 2
    size = r + 1
    # rows j = 0..r, unknowns (c_0, c_1, ..., c_r)
    a = [[Fraction(0)] * size for _ in range(size)]
    b = [Fraction(0)] * size
    for j in range(size):
        a[j][0] = Fraction(1) if j == 0 else Fraction(0)
        for k in range(1, r + 1):
            a[j][k] = Fraction(2 * k ** (2 * j))
        b[j] = Fraction(2) if j == 1 else Fraction(0)
    # Gaussian elimination with row pivoting on exact rationals
    for col in range(size):
        piv = next(i for i in range(col, size) if a[i][col] != 0)
        a[col], a[piv] = a[piv], a[col]
        b[col], b[piv] = b[piv], b[col]
        for i in range(size):
            if i != col and a[i][col] != 0:
                fac = a[i][col] / a[col][col]
                for j in range(col, size):
                    a[i][j] -= fac * a[col][j]
                b[i] -= fac * b[col]
    return [b[i] / a[i][i] for i in range(size)]


def symbol(coeffs, theta):
    """Fourier symbol of the stencil, Lambda(theta) = -c_0 - 2 sum_k c_k cos(k theta),
    so that the stencil applied to exp(i k x) (unit spacing) gives
    -Lambda(k) exp(i k x); Lambda(theta) ~ theta^2 for small theta."""
    c = [float(v) for v in coeffs]
    return -c[0] - 2.0 * sum(c[k] * math.cos(k * theta) for k in range(1, len(c)))


def symbol_max(coeffs, samples=20001):
    """max over theta in [0, pi] of Lambda(theta), by dense sampling."""
    return max(symbol(coeffs, math.pi * i / (samples - 1)) for i in range(samples))


def cfl_dt(space_order, h, v_max):
    """Largest stable dt of the undamped leapfrog scheme (von Neumann): a
    Fourier mode grows unless dt^2 v^2 sum_a Lambda(theta_a)/h_a^2 <= 4 for all
    theta, i.e. dt <= 2 / (v_max sqrt(sum_a max Lambda / h_a^2))."""
    lam = symbol_max(fd2_central_weights(space_order))
    return 2.0 / (v_max * math.sqrt(sum(lam / (ha * ha) for ha in h)))

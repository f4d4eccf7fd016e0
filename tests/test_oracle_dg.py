"""Pins of the DG streaming oracle (oracle/dg.py) against facts that do not come
from it: exact differentiation of polynomials (numpy's polynomial routines),
reproduction of -c_x dp/dx for global polynomials of degree < K, the
telescoping of numerical fluxes (zero total mass change with zero-flux walls),
the exact equilibrium of a wall Maxwellian, upwinding, the h^(K-1) convergence
of the DG derivative, and the third-order Taylor identity of SSP-RK3 for a linear
operator."""
import numpy as np
import pytest
from numpy.polynomial import polynomial as Pn

import oracle as O
from oracle import dg as DG

rng = np.random.default_rng(77)
WALLS = ((1.0, (0.0, -0.3, 0.0)), (2.0, (0.0, 0.3, 0.0)))


def _slab(Ne=5, K=3, N=8, L=5.0, masses=(1.0, 2.0), walls=WALLS):
    return DG.Slab(Ne, K, 0.0, 1.0, N, L, masses, walls)


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5])
def test_derivative_matrix_differentiates_polynomials_exactly(K):
    xi, _ = O.gauss_legendre(K)
    D = DG.lagrange_derivative(xi)
    for _ in range(3):
        c = rng.normal(size=K)  # degree K - 1
        u = Pn.polyval(xi, c)
        du = Pn.polyval(xi, Pn.polyder(c)) if K > 1 else np.zeros(K)
        assert np.abs(D.T @ u - du).max() <= 1e-12 * max(1.0, np.abs(du).max())
    # the basis is a partition of unity
    assert np.abs(D.sum(axis=0)).max() < 1e-12
    for x in (-1.0, 0.3, 1.0):
        assert abs(DG.lagrange_values(xi, x).sum() - 1.0) < 1e-13


@pytest.mark.parametrize("K", [2, 3, 4])
def test_interior_elements_reproduce_polynomial_derivative(K):
    s = _slab(Ne=6, K=K)
    c = rng.normal(size=K)
    g = rng.uniform(0.5, 1.5, size=(s.S, s.N ** 3))
    f = Pn.polyval(s.x, c)[:, None, None] * g[None]
    r = s.streaming(f)
    dp = Pn.polyval(s.x, Pn.polyder(c))
    exact = -s.cx[None, None, :] * dp[:, None, None] * g[None]
    inner = slice(K, (s.Ne - 1) * K)  # elements 1 .. Ne-2
    err = np.abs(r[inner] - exact[inner]).max()
    assert err <= 1e-11 * np.abs(exact).max()


def test_zero_flux_walls_conserve_mass():
    s = _slab(Ne=4, K=3)
    f = rng.uniform(0.1, 1.0, size=(s.P, s.S, s.N ** 3))
    r = s.streaming(f)
    rate = s.mass_rate(r)
    scale = s.mass_rate(np.abs(r))
    assert np.all(np.abs(rate) <= 1e-13 * scale)


def test_wall_maxwellian_is_an_equilibrium():
    T = 1.3
    walls = ((T, (0.0, 0.0, 0.0)), (T, (0.0, 0.0, 0.0)))
    s = _slab(Ne=3, K=3, walls=walls)
    f = np.stack([np.stack([DG.maxwellian(s.N, s.L, m, 0.7, (0, 0, 0), T) for m in s.masses])] * s.P)
    r = s.streaming(f)
    scale = np.abs(s.cx[None, None, :] * f).max() / s.J
    assert np.abs(r).max() <= 1e-13 * scale


def test_upwinding_of_a_jump():
    s = _slab(Ne=4, K=3)
    f = np.zeros((s.P, s.S, s.N ** 3))
    f[: 2 * s.K] = 1.0  # elements 0, 1 hold 1, elements 2, 3 hold 0
    r = s.streaming(f)
    pos, neg = s.cx > 0, s.cx < 0
    e1, e2 = slice(s.K, 2 * s.K), slice(2 * s.K, 3 * s.K)
    assert np.abs(r[e1][..., pos]).max() < 1e-12  # constant state, left neighbour also 1
    assert np.abs(r[e2][..., neg]).max() < 1e-12  # zero state, right neighbour also 0
    assert np.abs(r[e2][..., pos]).max() > 1.0  # inflow of the jump
    assert np.abs(r[e1][..., neg]).max() > 1.0


def test_dg_derivative_converges_at_order_K_minus_1():
    # the derivative of a degree K-1 approximation is O(h^(K-1)) pointwise
    K = 3
    errs = []
    for Ne in (4, 8, 16):
        s = _slab(Ne=Ne, K=K, N=4)
        g = np.ones((s.S, s.N ** 3))
        f = np.sin(2 * np.pi * s.x)[:, None, None] * g[None]
        exact = -s.cx[None, None, :] * (2 * np.pi * np.cos(2 * np.pi * s.x))[:, None, None]
        inner = slice(K, (s.Ne - 1) * K)
        errs.append(np.abs(s.streaming(f)[inner] - exact[inner]).max())
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) >= K - 1 - 0.3, rates


def test_ssp_rk3_is_third_order_taylor_for_linear_streaming():
    s = _slab(Ne=3, K=2, N=4)
    f = rng.uniform(0.1, 1.0, size=(s.P, s.S, s.N ** 3))
    dt = 2e-3
    L1 = s.streaming(f)
    L2 = s.streaming(L1)
    L3 = s.streaming(L2)
    taylor = f + dt * L1 + dt ** 2 / 2 * L2 + dt ** 3 / 6 * L3
    step = s.ssp_rk3(f, dt)
    assert np.abs(step - taylor).max() <= 1e-13 * np.abs(f).max()

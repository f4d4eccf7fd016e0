"""Pins of the oracle's radial weight rho^{gamma+2} (gamma = 2(1 - omega)) and of
its moments, against results fixed by the mathematics rather than by the
oracle's own code.

Radial weight.  In the loss term of Algorithm 2, ifft(c . fft(f_q)) with
c_k = sum_rs w_r w_s rho_r^{gamma+2} E_eta(pi rho_r / L, k, sigma_s) (Algorithm 1,
Eq. 13) is, for VHS (eta = 0, so E_0 = 4 pi sinc and sum_s w_s = 4 pi), the
Gauss-Legendre form of the truncated collision frequency

    nu(x) = 4 pi int_{|u| <= R} |u|^{2(1 - omega)} f_q(x - u) du

(Eq. 3's kernel |u|^{2(1-omega)} in spherical coordinates: rho^gamma rho^2).
For a Maxwellian f_q the angular part of that integral is closed form, so
nu(x) reduces to a one-dimensional integral that scipy's adaptive quadrature
evaluates independently of the oracle's Gauss-Legendre nodes, designs,
Funk-Hecke series and FFT.  Algorithm 1's printed gamma = 2(omega - 1) changes
the exponent of rho by 4(1 - omega) and fails these tests by orders of
magnitude beyond their tolerances.

Moments.  For a shifted Maxwellian f = n (m/(pi T))^{3/2} exp(-m |c - u|^2 / T)
the velocity moments are n, n m u and n (m |u|^2 + 3 T / 2); on a grid wide
and fine enough the cell-centred midpoint rule reproduces them to ~1e-11, so a
missing h^3, a wrong mass factor or a grid-offset slip fails the test.
"""
import math
import os

import numpy as np
import pytest
import scipy.integrate

import oracle as O

O.set_threads(os.cpu_count() or 1)


def _grid(N, L):
    h = 2.0 * L / N
    c = -L + (np.arange(N) + 0.5) * h
    return np.meshgrid(c, c, c, indexing="ij")


def _maxwellian(N, L, n, m, u, T):
    cx, cy, cz = _grid(N, L)
    r2 = (cx - u[0]) ** 2 + (cy - u[1]) ** 2 + (cz - u[2]) ** 2
    return n * (m / (math.pi * T)) ** 1.5 * np.exp(-m * r2 / T)


def _collision_frequency(x, n, m, u, T, gamma, R):
    """4 pi int_{|w| <= R} |w|^gamma f_q(x - w) dw for the Maxwellian f_q, with
    the angular integral in closed form:
      int_{S^2} exp(-a |y - rho w^|^2) dw^ = exp(-a (|y|^2 + rho^2)) 4 pi sinh(2 a rho |y|) / (2 a rho |y|),
    a = m / T, y = x - u."""
    a = m / T
    y = math.sqrt(sum((x[i] - u[i]) ** 2 for i in range(3)))
    norm = n * (a / math.pi) ** 1.5

    def radial(rho):
        z = 2.0 * a * rho * y
        # sinh(z)/z times exp(-a (y^2 + rho^2)), written to avoid overflow
        if z < 1e-8:
            ang = math.exp(-a * (y * y + rho * rho))
        else:
            ang = (math.exp(-a * (y - rho) ** 2) - math.exp(-a * (y + rho) ** 2)) / (2.0 * z)
        return rho ** (gamma + 2.0) * 4.0 * math.pi * ang

    val, err = scipy.integrate.quad(radial, 0.0, R, epsabs=0.0, epsrel=1e-13, limit=400)
    return 4.0 * math.pi * norm * val


@pytest.mark.parametrize("omega", [0.5, 0.75, 0.81])
def test_loss_term_is_the_truncated_collision_frequency(omega):
    # N = 32 on [-8, 8]^3 (h = 0.5) resolves a T = 2 Maxwellian spectrally
    # (Fourier content at the Nyquist wavenumber ~ e^{-20}); the ball of radius
    # R = 7.25 around a central point stays where f_q < 1e-11 of its peak at the
    # boundary, so the periodic interpolant equals f_q there; VHS, equal masses.
    N, L, M, Nrho = 32, 8.0, 6, 32
    mq, n, T = 1.0, 1.0, 2.0
    u = (0.2, -0.1, 0.05)
    pair = O.Pair(N, L, M, Nrho, 1.0, mq, omega, 1.0, 1.0)
    assert abs(pair.gamma - 2.0 * (1.0 - omega)) < 1e-15
    fq = _maxwellian(N, L, n, mq, u, T)
    _, c, _ = pair.tables()
    nu = np.real(np.fft.ifftn(c * np.fft.fftn(fq)))
    cx, cy, cz = _grid(N, L)
    # interior points near the bulk velocity, where the ball of radius R
    # around x stays where f_q is below 1e-10 of its peak at the boundary
    idx = [(16, 16, 16), (15, 16, 17), (17, 15, 16), (14, 17, 15), (16, 14, 18)]
    for (i, j, k) in idx:
        x = (cx[i, j, k], cy[i, j, k], cz[i, j, k])
        ref = _collision_frequency(x, n, mq, u, T, 2.0 * (1.0 - omega), pair.R)
        got = nu[i, j, k]
        # Gauss-Legendre on rho^{gamma+2} g(rho) (gamma + 2 non-integer) with
        # 32 nodes is accurate to ~5e-9 (3e-7 with 16, 1e-3 with 8: algebraic
        # convergence), the spectral interpolant to ~1e-9; the printed
        # gamma = 2(omega - 1) is off by 0.37 (omega = 0.81) to 0.45 (omega = 0.75)
        assert abs(got - ref) < 3e-8 * abs(ref), (omega, (i, j, k), got, ref)


@pytest.mark.parametrize("omega,Nrho", [(0.5, 8), (0.75, 16), (0.81, 16), (1.0, 4)])
def test_c_at_k0_is_the_radial_moment(omega, Nrho):
    """c_0 = sum_r w_r rho_r^{gamma+2} sum_s w_s E_0(theta_r, 0) = (4 pi)^2 int_0^R rho^{gamma+2} drho
    for VHS, i.e. (4 pi)^2 R^{gamma+3} / (gamma + 3) up to the Gauss-Legendre error
    of a rho^{gamma+2} integrand (exact for omega = 1 and 0.5, where gamma + 2 is an integer)."""
    pair = O.Pair(8, 4.0, 6, Nrho, 1.0, 2.0, omega, 1.0, 1.0)
    _, c, _ = pair.tables()
    g = 2.0 * (1.0 - omega)
    ref = (4.0 * math.pi) ** 2 * pair.R ** (g + 3.0) / (g + 3.0)
    tol = 1e-13 if abs(g + 2 - round(g + 2)) < 1e-12 else 1e-5
    assert abs(c[0, 0, 0].real - ref) < tol * ref, (c[0, 0, 0], ref)
    assert abs(c[0, 0, 0].imag) < 1e-13 * ref


@pytest.mark.parametrize("m,n,u,T", [(1.0, 1.0, (0.0, 0.0, 0.0), 1.0), (2.0, 0.7, (0.4, -0.3, 0.25), 1.3),
                                     (4.0, 1.3, (-0.5, 0.2, 0.1), 0.8)])
def test_moments_of_a_maxwellian(m, n, u, T):
    N, L = 80, 10.0  # h = 0.25: midpoint-rule error ~ exp(-2 pi^2 T / (2 m h^2)) < 1e-11 for T / m >= 0.2
    f = _maxwellian(N, L, n, m, u, T)
    out = O.moments(N, L, m, f)
    uu = sum(x * x for x in u)
    ref = [n, n * m * u[0], n * m * u[1], n * m * u[2], n * (m * uu + 1.5 * T)]
    for i in range(5):
        assert abs(out[i] - ref[i]) < 1e-9 * max(1.0, abs(ref[i])), (i, out[i], ref[i])

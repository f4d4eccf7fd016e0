"""Pin of the unlike-mass pair operator Q^(pq) (Eq. 3 kernel, Algorithm 2 with
the mass ratios in its phases): linearised stress responses against their
closed forms.

With mu = m_p + m_q, kappa = m_q/mu, kappa' = m_p/mu, the p-particle's
post-collision velocity is v' = G + kappa |u| sigma with G = (m_p v + m_q v_*)/mu
and u = v - v_*, so v = G + kappa u and v_* = G - kappa' u.  For
phi = v_x^2 - v_y^2 the sigma-average of phi(v') - phi(v) with weight
b(t) = (1 + t)^{alpha-1} is

    -2 kappa c1 (G_x u_x - G_y u_y) - kappa^2 lambda (u_x^2 - u_y^2)   (+ an isotropic part),
    c1 = 2 pi int b (1 - t) dt = 2 pi 2^{alpha+1} / (alpha (alpha+1)),
    lambda = 3 pi int b (1 - t^2) dt = 3 pi 2^{alpha+2} / ((alpha+1)(alpha+2)).

About the Maxwellians M_s = (m_s/pi)^{3/2} exp(-m_s |v|^2), M_p(v) M_q(v_*) is a
Gaussian in G (variance 1/(2 mu)) times one in u (variance 1/(2 mu_r),
mu_r = m_p m_q / mu), so with A1 = <|u|^gamma u_x^2> = (2/(3 sqrt(pi)))
Gamma((gamma+5)/2) mu_r^{-(gamma+2)/2} and A2 = <|u|^gamma (u_x^2 - u_y^2)^2> =
(8/(15 sqrt(pi))) Gamma((gamma+7)/2) mu_r^{-(gamma+4)/2}:

    perturbing f_p by eps M_p phi:  <phi, Q>_lin = -eps beta [4 kappa^2 c1 A1 / mu + kappa^4 lambda A2],
    perturbing f_q by eps M_q phi:  <phi, Q>_lin =  eps beta [4 kappa kappa' c1 A1 / mu - kappa^2 kappa'^2 lambda A2],

and int M_s phi^2 = 1 / m_s^2 turns them into rates nu = -<phi, Q>_lin / (eps / m_s^2).
For m_p = m_q the G-u terms cancel in the sum and the single-species rate
returns.  The linear parts are taken as odd parts in eps of two evaluations.
Measured with m = (1, 2): within 1.2e-5 at N = 32 (L = 7) for (omega, alpha) =
(1, 1), (0.81, 1), (0.75, 1.4), and 2e-3 to 4e-3 at N = 24, where the
heavier species' Maxwellian is less resolved.  This pins the mass ratios in the
phases and the b table, R_pq and the unlike-pair beta's use, at omega and
alpha of the slab workload's kind."""
import math

import numpy as np
import pytest

import oracle as O

EPS = 0.05


def _closed(beta, omega, alpha, mp, mq):
    gamma = 2.0 * (1.0 - omega)
    mu, mur = mp + mq, mp * mq / (mp + mq)
    k, kp = mq / mu, mp / mu
    c1 = 2 * math.pi * 2 ** (alpha + 1) / (alpha * (alpha + 1))
    lam = 3 * math.pi * 2 ** (alpha + 2) / ((alpha + 1) * (alpha + 2))
    A1 = 2.0 / (3.0 * math.sqrt(math.pi)) * math.gamma((gamma + 5) / 2) * mur ** (-(gamma + 2) / 2)
    A2 = 8.0 / (15.0 * math.sqrt(math.pi)) * math.gamma((gamma + 7) / 2) * mur ** (-(gamma + 4) / 2)
    lin_p = -beta * (4 * k * k * c1 * A1 / mu + k ** 4 * lam * A2)
    lin_q = beta * (4 * k * kp * c1 * A1 / mu - k * k * kp * kp * lam * A2)
    return -lin_p * mp * mp, -lin_q * mq * mq


def _rates(N, L, M, Nrho, masses, omega, alpha):
    h = 2 * L / N
    c = -L + (np.arange(N) + 0.5) * h
    cx, cy, cz = np.meshgrid(c, c, c, indexing="ij")
    c2 = cx ** 2 + cy ** 2 + cz ** 2
    mp, mq = masses
    Mp = (mp / np.pi) ** 1.5 * np.exp(-mp * c2)
    Mq = (mq / np.pi) ** 1.5 * np.exp(-mq * c2)
    phi = cx ** 2 - cy ** 2
    pair = O.Problem(N, L, M, Nrho, list(masses), [dict(omega=omega, alpha=alpha, d=1.0)] * 4).pair(0, 1)
    na = nb = 0.0
    for s in (1.0, -1.0):
        Q, _ = pair.collide(Mp * (1 + s * EPS * phi), Mq)
        na += s * float((phi * Q).sum())
        Q, _ = pair.collide(Mp, Mq * (1 + s * EPS * phi))
        nb += s * float((phi * Q).sum())
    nu_p = -na / (2 * EPS * float((Mp * phi * phi).sum()))
    nu_q = -nb / (2 * EPS * float((Mq * phi * phi).sum()))
    return (nu_p, nu_q), _closed(pair.beta, omega, alpha, mp, mq)


@pytest.mark.parametrize("N,L,Nrho,omega,alpha,tol", [(32, 7.0, 16, 0.75, 1.4, 5e-5), (24, 7.0, 12, 0.81, 1.0, 5e-3)])
def test_unlike_mass_linearised_stress_responses(N, L, Nrho, omega, alpha, tol):
    got, want = _rates(N, L, 12, Nrho, (1.0, 2.0), omega, alpha)
    for g, w in zip(got, want):
        assert abs(g / w - 1.0) <= tol, (got, want)

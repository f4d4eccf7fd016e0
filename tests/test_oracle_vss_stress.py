"""Pin of the VSS (alpha != 1) operator: the relaxation rate of the traceless
stress of Maxwell molecules (omega = 1) against its closed form.

For a kernel that depends on the scattering angle only, B(|g|, t) = B(t),
t = sigma . g^ (Eq. 3 with omega = 1: |g|^{2(1 - omega)} = 1, and the VSS
factor (1 + t)^{alpha - 1} times beta), equal masses and zero mean velocity,
the weak form of Q with the post-collision velocity v' = (v + v_*)/2 + |g|
sigma/2 gives, for phi = v_x^2 - v_y^2 (any traceless quadratic),

    int phi Q(f, f) dv = -nu int phi f dv,
    nu = (n / 2) 2 pi int_{-1}^{1} B(t) (3/2) (1 - t^2) dt,

because the sigma-average of sigma_i sigma_j with weight B(t) is
2 pi int B [(1 - t^2)/2 (delta_ij - g^_i g^_j) + t^2 g^_i g^_j] dt and the
centre-of-mass cross terms cancel.  With B(t) = beta (1 + t)^{alpha - 1} the
integral is beta 2^{alpha + 2} / ((alpha + 1)(alpha + 2)), so

    nu(alpha) = 3 pi n beta 2^{alpha + 1} / ((alpha + 1)(alpha + 2)),

and with beta's VSS factor alpha / 2^{1 + alpha} (which keeps the total cross
section of Eq. 4-5 independent of alpha) the ratio to the VHS rate at the same
diameter is nu(alpha) / nu(1) = 6 alpha / ((alpha + 1)(alpha + 2)).

The discrete operator (Algorithm 2 with the 12-point design) reproduces the
continuous rate up to its angular quadrature error, which does not shrink
with N (about 2e-3 here, measured at N = 16, 24 and 32): the bounds are 1e-2
on each rate and 5e-3 on the ratio, which resolve the 3 % VSS effect at
alpha = 1.4 and fail for a wrong exponent sign (eta = 1 - alpha: 13 %), a
missing alpha or a wrong power of two in beta (factors 1.4 and 2)."""
import numpy as np
import pytest

import oracle as O

N, L, M, NRHO = 24, 7.0, 12, 12


def _rate(alpha):
    h = 2 * L / N
    c = -L + (np.arange(N) + 0.5) * h
    cx, cy, cz = np.meshgrid(c, c, c, indexing="ij")
    Tx, Ty, Tz = 1.3, 0.8, 1.0  # an anisotropic Maxwellian: traceless stress != 0
    f = np.exp(-(cx ** 2 / Tx + cy ** 2 / Ty + cz ** 2 / Tz)) / np.sqrt(np.pi ** 3 * Tx * Ty * Tz)
    pair = O.Problem(N, L, M, NRHO, [1.0], [dict(omega=1.0, alpha=alpha, d=1.0)]).pair(0, 0)
    Q, _ = pair.collide(f, f)
    phi = cx ** 2 - cy ** 2
    nu = -float((phi * Q).sum()) / float((phi * f).sum())
    n = float(f.sum()) * h ** 3
    nu_cf = 3.0 * np.pi * n * pair.beta * 2.0 ** (alpha + 1) / ((alpha + 1) * (alpha + 2))
    return nu, nu_cf


@pytest.fixture(scope="module")
def rates():
    return {a: _rate(a) for a in (1.0, 1.4, 0.8)}


@pytest.mark.parametrize("alpha", [1.0, 1.4, 0.8])
def test_stress_relaxation_rate_matches_closed_form(rates, alpha):
    nu, nu_cf = rates[alpha]
    assert abs(nu / nu_cf - 1.0) <= 1e-2, (alpha, nu, nu_cf)


@pytest.mark.parametrize("alpha", [1.4, 0.8])
def test_vss_to_vhs_rate_ratio(rates, alpha):
    got = rates[alpha][0] / rates[1.0][0]
    want = 6.0 * alpha / ((alpha + 1.0) * (alpha + 2.0))
    assert abs(got / want - 1.0) <= 5e-3, (alpha, got, want)
    # the VSS effect itself is resolved: the rate is not the VHS one
    assert abs(got - 1.0) > 5 * 5e-3 * want or alpha == 1.0

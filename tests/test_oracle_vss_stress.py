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
with N.  Two distributions: a near-equilibrium one, M (1 + eps (c_x^2 - c_y^2)),
whose rate the operator meets to 2e-5 at alpha = 1 and 1e-3 at alpha = 0.8,
1.4 (the design's error for the non-polynomial (1 + t)^{alpha-1}: 4 % with the
6-point design); and an anisotropic Maxwellian, far from equilibrium (2e-3,
measured at N = 16, 24 and 32).  Bounds: 2e-4 (alpha = 1) and 2e-3 (VSS) near
equilibrium, 1e-2 far from it, 2e-3 on the ratio to the VHS rate.  They
resolve the 3 % VSS effect at alpha = 1.4 and fail for a wrong exponent sign
(eta = 1 - alpha: 13 %), a missing alpha or a wrong power of two in beta
(factors 1.4 and 2)."""
import numpy as np
import pytest

import oracle as O

N, L, M, NRHO = 24, 7.0, 12, 12


def _grid():
    h = 2 * L / N
    c = -L + (np.arange(N) + 0.5) * h
    return np.meshgrid(c, c, c, indexing="ij")


def _rate(alpha, near):
    cx, cy, cz = _grid()
    if near:  # Maxwellian (T = 1) times 1 + eps (c_x^2 - c_y^2): zero mean velocity
        f = np.exp(-(cx ** 2 + cy ** 2 + cz ** 2)) / np.pi ** 1.5 * (1.0 + 0.1 * (cx ** 2 - cy ** 2))
    else:  # an anisotropic Maxwellian: traceless stress != 0
        Tx, Ty, Tz = 1.3, 0.8, 1.0
        f = np.exp(-(cx ** 2 / Tx + cy ** 2 / Ty + cz ** 2 / Tz)) / np.sqrt(np.pi ** 3 * Tx * Ty * Tz)
    pair = O.Problem(N, L, M, NRHO, [1.0], [dict(omega=1.0, alpha=alpha, d=1.0)]).pair(0, 0)
    Q, _ = pair.collide(f, f)
    phi = cx ** 2 - cy ** 2
    nu = -float((phi * Q).sum()) / float((phi * f).sum())
    n = float(f.sum()) * (2 * L / N) ** 3
    nu_cf = 3.0 * np.pi * n * pair.beta * 2.0 ** (alpha + 1) / ((alpha + 1) * (alpha + 2))
    return nu, nu_cf


@pytest.fixture(scope="module")
def rates():
    return {(a, near): _rate(a, near) for a in (1.0, 1.4, 0.8) for near in (True, False)}


@pytest.mark.parametrize("alpha", [1.0, 1.4, 0.8])
def test_stress_relaxation_rate_matches_closed_form(rates, alpha):
    nu, nu_cf = rates[(alpha, True)]
    assert abs(nu / nu_cf - 1.0) <= (2e-4 if alpha == 1.0 else 2e-3), (alpha, nu, nu_cf)
    nu, nu_cf = rates[(alpha, False)]
    assert abs(nu / nu_cf - 1.0) <= 1e-2, (alpha, nu, nu_cf)


@pytest.mark.parametrize("alpha", [1.4, 0.8])
def test_vss_to_vhs_rate_ratio(rates, alpha):
    got = rates[(alpha, True)][0] / rates[(1.0, True)][0]
    want = 6.0 * alpha / ((alpha + 1.0) * (alpha + 2.0))
    assert abs(got / want - 1.0) <= 2e-3, (alpha, got, want)
    # the VSS effect itself is resolved: the rate is not the VHS one
    assert abs(got - 1.0) > 10 * 2e-3 * want

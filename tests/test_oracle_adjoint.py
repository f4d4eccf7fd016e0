"""Pins of the oracle's adjoint of the bilinear map (f_p, f_q) -> Q^(pq) and of
its omega-derivative: dot-product tests (Q is bilinear, so <gbar, Q(d, f_q)> =
<dL/df_p, d> exactly) and central finite differences in omega."""
import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("M,alpha,masses", [(6, 1.0, (1.0, 2.0)), (12, 1.4, (1.0, 4.0)), (12, 0.8, (3.0, 1.0))])
def test_adjoint_dot_product(M, alpha, masses):
    N = 8
    rng = np.random.default_rng(M + int(10 * alpha))
    pair = O.Pair(N, 4.0, M, 4, masses[0], masses[1], 0.75, alpha, 1.0)
    fp, fq, g, dp, dq = (rng.normal(size=(N, N, N)) for _ in range(5))
    dfp, dfq, _ = pair.adjoint(fp, fq, g, domega=False)
    lhs_p = np.sum(g * pair.collide(dp, fq)[0])
    rhs_p = np.sum(dfp * dp)
    assert abs(lhs_p - rhs_p) < 1e-12 * (abs(lhs_p) + np.abs(dfp).sum() * 1e-3)
    lhs_q = np.sum(g * pair.collide(fp, dq)[0])
    rhs_q = np.sum(dfq * dq)
    assert abs(lhs_q - rhs_q) < 1e-12 * (abs(lhs_q) + np.abs(dfq).sum() * 1e-3)
    # dL/df_p does not depend on f_p (linearity in the first argument)
    dfp2, _, _ = pair.adjoint(2.0 * fp + 1.0, fq, g, domega=False)
    assert np.abs(dfp2 - dfp).max() < 1e-12 * np.abs(dfp).max()


@pytest.mark.parametrize("omega,alpha,override", [(0.81, 1.0, None), (0.75, 1.4, None), (0.7, 1.0, 0.05)])
def test_omega_derivative_finite_difference(omega, alpha, override):
    N, M, Nrho = 8, 6, 4
    rng = np.random.default_rng(5)
    fp = np.abs(rng.normal(size=(N, N, N)))
    fq = np.abs(rng.normal(size=(N, N, N)))
    g = rng.normal(size=(N, N, N))
    bo = float("nan") if override is None else override
    mk = lambda w: O.Pair(N, 4.0, M, Nrho, 1.0, 2.0, w, alpha, 1.1, bo)
    h = 1e-4
    Lp = np.sum(g * mk(omega + h).collide(fp, fq)[0])
    Lm = np.sum(g * mk(omega - h).collide(fp, fq)[0])
    fd = (Lp - Lm) / (2 * h)
    _, _, dw = mk(omega).adjoint(fp, fq, g)
    assert abs(dw - fd) < 1e-7 * max(1.0, abs(fd)), (dw, fd)
    # the elementwise dQ/domega against finite differences
    Q, _, dQ = mk(omega).collide(fp, fq, domega=True)
    Qp = mk(omega + h).collide(fp, fq)[0]
    Qm = mk(omega - h).collide(fp, fq)[0]
    assert np.abs(dQ - (Qp - Qm) / (2 * h)).max() < 1e-6 * np.abs(dQ).max()


def test_moment_weights_gradient():
    """For the moment loss L = sum_j w(c_j) Q_j, the gradient is <w, Q(., f_q)>'s
    representer; the dot-product identity holds for the physically relevant
    weights (1, v, |v|^2, v_x v_y) too."""
    N, L = 8, 4.0
    pair = O.Pair(N, L, 12, 4, 1.0, 2.0, 0.81, 1.0, 1.0)
    c = -L + (np.arange(N) + 0.5) * (2 * L / N)
    cx, cy, cz = np.meshgrid(c, c, c, indexing="ij")
    rng = np.random.default_rng(9)
    fp = np.exp(-(cx ** 2 + cy ** 2 + cz ** 2)) * (1 + 0.1 * rng.normal(size=(N, N, N)))
    fq = np.exp(-2 * (cx ** 2 + cy ** 2 + cz ** 2)) * (1 + 0.1 * rng.normal(size=(N, N, N)))
    for wgt in (np.ones_like(cx), cx, cx ** 2 + cy ** 2 + cz ** 2, cx * cy):
        dfp, dfq, _ = pair.adjoint(fp, fq, wgt, domega=False)
        d = rng.normal(size=(N, N, N))
        lhs = np.sum(wgt * pair.collide(d, fq)[0])
        assert abs(lhs - np.sum(dfp * d)) < 1e-11 * (abs(lhs) + np.abs(dfp).max())

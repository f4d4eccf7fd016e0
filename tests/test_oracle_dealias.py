"""Pin of the dealiased oracle (oracle/dealias.py): it equals the Galerkin sum
of Eq. (7) over l + m = k WITHOUT wrap-around, evaluated by brute force over
all pairs of retained wavenumbers (Nyquist planes zeroed on input and output),
and differs from the cyclic Algorithm 2 on rough input."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import dealias as DA


def brute_force_linear(pair, fp, fq):
    """X(k) = sum_{l+m=k} [sum_rs w_r w_s b_rs(k) e^{i cq a_rs(l)} e^{-i cp a_rs(m)} - c(m)] F_p(l) F_q(m) / n
    over integer l, m, k with all components in [-N/2, N/2), the -N/2 planes of
    F_p, F_q and X zeroed; Q = beta Re ifft(X).  Tables from the N-grid pair."""
    N, n = pair.N, pair.N ** 3
    rho, wrho, sig, wsig = pair.quadrature()
    b, c, _ = pair.tables()
    Fp = DA.zero_nyquist(np.fft.fftn(fp)).ravel()
    Fq = DA.zero_nyquist(np.fft.fftn(fq)).ravel()
    v = DA.wavenumbers(N)
    lv = np.stack(np.meshgrid(v, v, v, indexing="ij"), -1).reshape(n, 3)
    ksum = lv[:, None, :] + lv[None, :, :]  # integer l + m, (n, n, 3)
    inside = np.all((ksum >= -(N // 2)) & (ksum <= (N - 1) // 2), axis=-1)
    kidx = np.mod(ksum, N)
    kflat = (kidx[..., 0] * N + kidx[..., 1]) * N + kidx[..., 2]
    X = np.zeros(n, complex)

    def conv(prod):
        p = np.where(inside, prod, 0.0).ravel()
        return np.bincount(kflat.ravel(), p.real, n) + 1j * np.bincount(kflat.ravel(), p.imag, n)

    for r in range(pair.Nrho):
        for s in range(pair.M):
            a = math.pi / pair.L * rho[r] * (lv @ sig[s])
            t1 = np.exp(1j * pair.cq * a) * Fp
            t2 = np.exp(-1j * pair.cp * a) * Fq
            X += wrho[r] * wsig[s] * b[r, s].ravel() * conv(t1[:, None] * t2[None, :] / n)
    X -= conv(Fp[:, None] * (c.ravel() * Fq)[None, :] / n)
    X = DA.zero_nyquist(X.reshape(N, N, N))
    return pair.beta * np.real(np.fft.ifftn(X))


@pytest.mark.parametrize("N,M,Nrho,alpha", [(4, 6, 3, 1.4), (6, 12, 2, 1.0), (6, 6, 2, 0.8)])
def test_dealiased_oracle_equals_linear_galerkin_sum(N, M, Nrho, alpha):
    rng = np.random.default_rng(7 * N + M)
    args = (N, 3.0, M, Nrho, 1.0, 2.5, 0.75, alpha, 1.1)
    fp, fq = rng.normal(size=(N, N, N)), rng.normal(size=(N, N, N))
    Q = DA.DealiasedPair(*args).collide(fp, fq)
    ref = brute_force_linear(O.Pair(*args), fp, fq)
    assert np.abs(Q - ref).max() < 1e-12 * np.abs(ref).max()


def test_interpolation_is_exact_on_retained_modes_and_real():
    rng = np.random.default_rng(3)
    f = rng.normal(size=(8, 8, 8))
    g = DA.interpolate(f, 12)
    G = np.fft.fftn(g)
    F = DA.zero_nyquist(np.fft.fftn(f))
    e = np.mod(DA.wavenumbers(8), 12)
    assert np.abs(G[np.ix_(e, e, e)] * (8 / 12) ** 3 - F).max() < 1e-12 * np.abs(F).max()
    # and restriction undoes it
    assert np.abs(DA.restrict(g, 8) - np.real(np.fft.ifftn(F))).max() < 1e-13


def test_dealiased_differs_from_cyclic_on_rough_input():
    """On white-noise input the aliased terms are O(1): the variant is not the
    cyclic operator in disguise."""
    N, args = 8, (8, 4.0, 6, 3, 1.0, 2.0, 0.8, 1.0, 1.0)
    rng = np.random.default_rng(5)
    fp, fq = rng.normal(size=(N, N, N)), rng.normal(size=(N, N, N))
    Rd = DA.DealiasedPair(*args).collide(fp, fq)
    Rc, _ = O.Pair(*args).collide(fp, fq)
    assert np.abs(Rd - Rc).max() > 1e-3 * np.abs(Rc).max()

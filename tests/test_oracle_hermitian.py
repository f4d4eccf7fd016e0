"""Pins of the oracle's declared Hermitian variant (Algorithm 2 with the Nyquist
planes removed; orc_collide_hermitian): the direct O(n^2) Galerkin sum of
Eq. 7 over the Nyquist-free wavenumbers, its agreement with the literal
Algorithm 2 on every Nyquist-free output mode for band-limited inputs, the
projection's idempotence, and the equilibrium residual."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1903_04670_gb300 import workloads as W

O.set_threads(os.cpu_count() or 1)


def _nyquist_mask(N):
    idx = np.arange(N)
    nyq = idx == N // 2
    return nyq[:, None, None] | nyq[None, :, None] | nyq[None, None, :]


def _project(f):
    """f with every Fourier mode on a Nyquist plane removed (real)."""
    F = np.fft.fftn(f)
    F[_nyquist_mask(f.shape[0])] = 0
    return np.real(np.fft.ifftn(F))


def brute_force_hermitian(pair, fp, fq):
    """Eq. (7)'s low-rank gain as a DIRECT cyclic sum over all (l, m) with
    l + m = k (mod N) of the Nyquist-free spectra, restricted to Nyquist-free
    k, plus the loss of Eq. (13) with the projected f_p; numpy FFTs only for the
    outer transforms, the oracle's tables b, c (pinned separately)."""
    N = pair.N
    n = N ** 3
    rho, wrho, sig, wsig = pair.quadrature()
    b, c, _ = pair.tables()
    mask = _nyquist_mask(N).ravel()
    Ff = np.fft.fftn(fp).ravel()
    Fg = np.fft.fftn(fq).ravel()
    Ff[mask] = 0
    Fg[mask] = 0
    v = np.fft.fftfreq(N, 1.0 / N)
    lvec = np.stack(np.meshgrid(v, v, v, indexing="ij"), -1).reshape(n, 3)
    idx = np.stack(np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij"), -1).reshape(n, 3)
    kk = (idx[:, None, :] + idx[None, :, :]) % N
    kflat = (kk[..., 0] * N + kk[..., 1]) * N + kk[..., 2]
    QG = np.zeros(n, complex)
    for r in range(pair.Nrho):
        for s in range(pair.M):
            a = math.pi / pair.L * rho[r] * (lvec @ sig[s])
            t1 = np.exp(1j * pair.cq * a) * Ff
            t2 = np.exp(-1j * pair.cp * a) * Fg
            prod = (t1[:, None] * t2[None, :]).ravel() / n
            conv = (np.bincount(kflat.ravel(), prod.real, n) + 1j * np.bincount(kflat.ravel(), prod.imag, n))
            QG += wrho[r] * wsig[s] * b[r, s].ravel() * conv
    QG[mask] = 0
    fpt = np.real(np.fft.ifftn(Ff.reshape(N, N, N)))
    loss = fpt * np.fft.ifftn((c.ravel() * Fg).reshape(N, N, N))
    gain = np.fft.ifftn(QG.reshape(N, N, N))
    # both terms are real in exact arithmetic (Hermitian spectra)
    assert np.abs(gain.imag).max() <= 1e-12 * np.abs(gain.real).max()
    assert np.abs(loss.imag).max() <= 1e-12 * np.abs(loss.real).max()
    return pair.beta * np.real(gain - loss)


@pytest.mark.parametrize("N,M,Nrho,alpha", [(4, 6, 3, 1.4), (6, 12, 2, 1.4), (4, 12, 2, 1.0), (6, 6, 3, 0.7)])
def test_hermitian_variant_equals_direct_galerkin_sum(N, M, Nrho, alpha):
    rng = np.random.default_rng(N * 101 + M)
    pair = O.Pair(N, 3.0, M, Nrho, 1.0, 2.5, 0.75, alpha, 1.1)
    fp = rng.normal(size=(N, N, N))
    fq = rng.normal(size=(N, N, N))
    Q = pair.collide_hermitian(fp, fq)
    ref = brute_force_hermitian(pair, fp, fq)
    assert np.abs(Q - ref).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("N,alpha", [(8, 1.4), (16, 1.0)])
def test_agrees_with_literal_operator_off_the_nyquist_planes(N, alpha):
    """For band-limited inputs the two forms differ only by the Nyquist planes
    of the gain, so every Nyquist-free Fourier mode of the output agrees."""
    rng = np.random.default_rng(N)
    L = N / 3.2
    pair = O.Pair(N, L, 6, 4, 1.0, 2.0, 0.81, alpha, 1.0)
    fp = _project(W.two_maxwellians(rng, N, L, 1.0) * (1 + 0.1 * rng.normal(size=(N, N, N))))
    fq = _project(W.two_maxwellians(rng, N, L, 2.0))
    Qh = pair.collide_hermitian(fp, fq)
    Ql, _ = pair.collide(fp, fq)
    D = np.fft.fftn(Qh - Ql)
    keep = ~_nyquist_mask(N)
    scale = np.abs(np.fft.fftn(Ql)).max()
    assert np.abs(D[keep]).max() <= 1e-12 * scale
    assert np.abs(D[~keep]).max() > 1e-9 * scale  # the gain's Nyquist planes do differ


def test_projection_is_idempotent():
    rng = np.random.default_rng(5)
    N, L = 8, 2.5
    pair = O.Pair(N, L, 12, 3, 1.0, 4.0, 0.75, 1.4, 1.0)
    fp = W.two_maxwellians(rng, N, L, 1.0) + 0.05 * rng.normal(size=(N, N, N))
    fq = W.two_maxwellians(rng, N, L, 4.0) + 0.05 * rng.normal(size=(N, N, N))
    Q1 = pair.collide_hermitian(fp, fq)
    Q2 = pair.collide_hermitian(_project(fp), _project(fq))
    assert np.abs(Q1 - Q2).max() <= 1e-13 * np.abs(Q1).max()


def test_equilibrium_residual_decays_with_N():
    """Maxwellians with a common bulk velocity and temperature: the residual
    falls with N as for the literal operator (same setting as its pin)."""
    masses = [1.0, 2.0]
    res = []
    for N in (16, 24):
        pair = O.Pair(N, 8.0, 12, N // 2, masses[0], masses[1], 0.75, 1.4, 1.1)
        u, T = (0.2, -0.1, 0.3), 1.0
        fp = W.maxwellian(N, 8.0, masses[0], 1.0, u, T)
        fq = W.maxwellian(N, 8.0, masses[1], 0.7, u, T)
        Q = pair.collide_hermitian(fp, fq)
        _, d = pair.collide(fp, fq)
        res.append(np.abs(Q).max() / d["gain_max"])
    assert res[1] < 0.2 * res[0]
    assert res[1] < 0.05

"""FP64 CPU oracle of the dealiased collision operator (TEST INFRASTRUCTURE).

Test infrastructure only: ``tests/`` may import it; the CUDA library never does.

Algorithm 2 forms the product of the translates on the N-point grid, so its
Fourier coefficients are the cyclic sum over l + m = k (mod N), while the
Galerkin form of Eq. (7) sums over l + m = k without wrap-around.  The
dealiased operator follows Eq. (7) literally by the 3/2 rule:

1. spectral interpolation of f_p, f_q onto N' = 3N/2 points per axis: the
   coefficients at the N wavenumbers of each input, with the planes that
   carry the wavenumber -N/2 set to zero (for even N its partner +N/2 is not
   on the grid, so only with those planes zeroed is the interpolant real),
   and zero at every other wavenumber;
2. Algorithm 2 on the N' grid with the same L (the oracle's own Pair);
3. the Fourier coefficients of the result at the N original wavenumbers,
   the -N/2 planes again zeroed, transformed back on the N grid.

With N' >= 3N/2, no sum l + m of two retained wavenumbers (|l|, |m| < N/2)
wraps onto a retained wavenumber, so step 3 returns exactly the
linear-convolution coefficients of Eq. (7) over the retained wavenumbers.
numpy's FFT serves as the library primitive for the resampling steps.
"""
import numpy as np

from . import Pair


def wavenumbers(N):
    """Integer wavenumber of each index: 0, 1, ..., then negative (index >= N/2)."""
    return np.fft.fftfreq(N, 1.0 / N).astype(int)


def padded_size(N):
    return (3 * N + 1) // 2


def _embed(N, Np):
    """Index in the Np grid of each of the N grid's wavenumbers, per axis."""
    return np.mod(wavenumbers(N), Np)


def zero_nyquist(F):
    """Set the planes carrying wavenumber -N/2 (even N) of a spectrum to zero."""
    N = F.shape[0]
    F = F.copy()
    if N % 2 == 0:
        F[N // 2, :, :] = 0.0
        F[:, N // 2, :] = 0.0
        F[:, :, N // 2] = 0.0
    return F


def interpolate(f, Np):
    """Trigonometric interpolant (-N/2 planes zeroed) of the real N^3 samples f
    on Np^3 points; real up to rounding."""
    N = f.shape[0]
    F = zero_nyquist(np.fft.fftn(f))
    G = np.zeros((Np, Np, Np), complex)
    e = _embed(N, Np)
    G[np.ix_(e, e, e)] = F * (Np / N) ** 3
    return np.real(np.fft.ifftn(G))


def restrict(q, N):
    """Coefficients of the Np^3 field q at the N original wavenumbers, the
    -N/2 planes zeroed (even N), back on the N^3 grid."""
    Np = q.shape[0]
    X = np.fft.fftn(q)
    e = _embed(N, Np)
    Y = zero_nyquist(X[np.ix_(e, e, e)] * (N / Np) ** 3)
    return np.real(np.fft.ifftn(Y))


class DealiasedPair:
    """Q^(pq) with the linear convolution of Eq. (7), for one species pair."""

    def __init__(self, N, L, M, Nrho, mp, mq, omega, alpha, d, beta_override=float("nan")):
        self.N = int(N)
        self.Np = padded_size(self.N)
        self.pair = Pair(self.Np, L, M, Nrho, mp, mq, omega, alpha, d, beta_override)

    def collide(self, fp, fq):
        Qp, _ = self.pair.collide(interpolate(fp, self.Np), interpolate(fq, self.Np))
        return restrict(Qp, self.N)

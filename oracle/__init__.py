"""FP64 CPU oracle of the fast spectral collision operator (TEST INFRASTRUCTURE).

This package is test infrastructure, not part of the product path.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import it.  It shares no code with the CUDA library.

The arithmetic lives in ``dgfs_oracle.c`` (plain C99, FP64), which follows
Algorithm 1 (pre-computation) and Algorithm 2 (collision evaluation) of
Jaiswal et al., PASC'19 (arXiv 1903.04670) step by step; see that file's
header for the readings taken where the paper is silent.  This module only
marshals numpy arrays through ctypes.
"""
import ctypes
import math
import os

import numpy as np

from . import _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        sig = {
            "orc_set_threads": (None, [i]),
            "orc_get_threads": (i, []),
            "orc_dft_naive_line": (None, [i, p, p, i]),
            "orc_fft_line": (None, [i, p, i]),
            "orc_fft3": (None, [i, p, i]),
            "orc_gauss_legendre": (i, [i, d, d, p, p]),
            "orc_sphere_design": (i, [i, p, p]),
            "orc_knudsen": (d, [d, d, d]),
            "orc_knudsen_dim": (d, [d, d, d, d, d, d, d]),
            "orc_beta": (d, [d, d, d, d, d]),
            "orc_radius": (d, [d, d, d]),
            "orc_digamma": (d, [d]),
            "orc_dlogbeta_domega": (d, [d, d, d]),
            "orc_lambda": (d, [i, d]),
            "orc_angular_integral": (None, [d, p, p, d, p]),
            "orc_pair_create": (p, [i, d, i, i, d, d, d, d, d, d]),
            "orc_pair_destroy": (None, [p]),
            "orc_pair_scalars": (None, [p, p]),
            "orc_pair_quadrature": (None, [p, p, p, p, p]),
            "orc_pair_tables": (None, [p, p, p, p]),
            "orc_collide": (None, [p, p, p, p, p, p]),
            "orc_adjoint": (None, [p, p, p, p, p, p, p]),
            "orc_moments": (None, [i, d, d, p, p]),
            "orc_collide_batch": (None, [p, i, i, p, p]),
            "orc_collide_hermitian": (None, [p, p, p, p]),
            "orc_collide_hermitian_batch": (None, [p, i, i, p, p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def set_threads(n):
    lib().orc_set_threads(int(n))


def get_threads():
    return int(lib().orc_get_threads())


# ---------------------------------------------------------------- transforms
def dft_naive_line(x, sign=-1):
    x = _c128(x)
    out = np.empty_like(x)
    lib().orc_dft_naive_line(x.size, _ptr(x), _ptr(out), int(sign))
    return out


def fft_line(x, sign=-1):
    x = _c128(x).copy()
    lib().orc_fft_line(x.size, _ptr(x), int(sign))
    return x


def fft3(x, sign=-1):
    """Unnormalised 3-D transform of an (N, N, N) grid (x slowest)."""
    x = _c128(x).copy()
    N = x.shape[0]
    assert x.shape == (N, N, N)
    lib().orc_fft3(N, _ptr(x), int(sign))
    return x


# --------------------------------------------------------------- quadratures
def gauss_legendre(n, a=-1.0, b=1.0):
    x = np.empty(n)
    w = np.empty(n)
    if lib().orc_gauss_legendre(int(n), float(a), float(b), _ptr(x), _ptr(w)) != 0:
        raise ValueError("bad Gauss-Legendre order")
    return x, w


def sphere_design(M):
    s = np.empty((M, 3))
    w = np.empty(M)
    if lib().orc_sphere_design(int(M), _ptr(s), _ptr(w)) != 0:
        raise ValueError("only M = 6 (octahedron) and M = 12 (icosahedron) are defined")
    return s, w


# ------------------------------------------------------------ kernel constants
def knudsen(mp, mq, d):
    return lib().orc_knudsen(mp, mq, d)


def knudsen_dim(mp, mq, n0, d, tref_over_t0, omega, H0):
    return lib().orc_knudsen_dim(mp, mq, n0, d, tref_over_t0, omega, H0)


def beta(mp, mq, omega, alpha, d):
    return lib().orc_beta(mp, mq, omega, alpha, d)


def radius(L, mp, mq):
    return lib().orc_radius(L, mp, mq)


def digamma(x):
    return lib().orc_digamma(float(x))


def lambda_n(n, eta):
    return lib().orc_lambda(int(n), float(eta))


def angular_integral(theta, k, sigma, eta):
    k = _f64(k)
    s = _f64(sigma)
    out = np.empty(2)
    lib().orc_angular_integral(float(theta), _ptr(k), _ptr(s), float(eta), _ptr(out))
    return complex(out[0], out[1])


def moments(N, L, m, Q):
    Q = _f64(Q)
    out = np.empty(5)
    lib().orc_moments(int(N), float(L), float(m), _ptr(Q), _ptr(out))
    return out


# ------------------------------------------------------------------- per pair
class Pair:
    """Tables of Algorithm 1 and the evaluation of Algorithm 2 for one pair."""

    def __init__(self, N, L, M, Nrho, mp, mq, omega, alpha, d, beta_override=float("nan")):
        self.N, self.L, self.M, self.Nrho = int(N), float(L), int(M), int(Nrho)
        self.mp, self.mq = float(mp), float(mq)
        self._h = lib().orc_pair_create(self.N, self.L, self.M, self.Nrho, self.mp, self.mq,
                                        float(omega), float(alpha), float(d), float(beta_override))
        if not self._h:
            raise ValueError("oracle: invalid pair parameters")
        s = np.empty(8)
        lib().orc_pair_scalars(self._h, _ptr(s))
        self.R, self.beta, self.gamma, self.eta, self.dlogbeta = s[:5]
        self.cq, self.cp = s[5], s[6]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_pair_destroy(h)
            self._h = None

    @property
    def n(self):
        return self.N ** 3

    def quadrature(self):
        rho = np.empty(self.Nrho)
        wrho = np.empty(self.Nrho)
        sig = np.empty((self.M, 3))
        wsig = np.empty(self.M)
        lib().orc_pair_quadrature(self._h, _ptr(rho), _ptr(wrho), _ptr(sig), _ptr(wsig))
        return rho, wrho, sig, wsig

    def tables(self):
        N = self.N
        b = np.empty((self.Nrho, self.M, N, N, N), dtype=np.complex128)
        c = np.empty((N, N, N), dtype=np.complex128)
        c_om = np.empty((N, N, N), dtype=np.complex128)
        lib().orc_pair_tables(self._h, _ptr(b), _ptr(c), _ptr(c_om))
        return b, c, c_om

    def collide(self, fp, fq, domega=False):
        """Q^(pq)(f_p, f_q) by Algorithm 2.  Returns (Q, diag[, dQ/domega]).

        diag = {imag_max, gain_max, loss_max, q_max} (after beta)."""
        N = self.N
        fp = _f64(fp).reshape(N, N, N)
        fq = _f64(fq).reshape(N, N, N)
        Q = np.empty((N, N, N))
        dQ = np.empty((N, N, N)) if domega else None
        diag = np.empty(4)
        lib().orc_collide(self._h, _ptr(fp), _ptr(fq), _ptr(Q),
                          _ptr(dQ) if domega else None, _ptr(diag))
        keys = ("imag_max", "gain_max", "loss_max", "q_max")
        dd = dict(zip(keys, diag.tolist()))
        return (Q, dd, dQ) if domega else (Q, dd)

    def collide_hermitian(self, fp, fq):
        """The declared Hermitian variant: Algorithm 2 with the Nyquist planes
        removed from the inputs and from the gain (see dgfs_oracle.c)."""
        N = self.N
        fp = _f64(fp).reshape(N, N, N)
        fq = _f64(fq).reshape(N, N, N)
        Q = np.empty((N, N, N))
        lib().orc_collide_hermitian(self._h, _ptr(fp), _ptr(fq), _ptr(Q))
        return Q

    def adjoint(self, fp, fq, gbar, domega=True):
        N = self.N
        fp = _f64(fp).reshape(N, N, N)
        fq = _f64(fq).reshape(N, N, N)
        g = _f64(gbar).reshape(N, N, N)
        dfp = np.empty((N, N, N))
        dfq = np.empty((N, N, N))
        dw = np.zeros(1)
        lib().orc_adjoint(self._h, _ptr(fp), _ptr(fq), _ptr(g), _ptr(dfp), _ptr(dfq),
                          _ptr(dw) if domega else None)
        return dfp, dfq, (float(dw[0]) if domega else None)


class Problem:
    """All S*S pair operators of a multi-species problem (pair order p-major)."""

    def __init__(self, N, L, M, Nrho, masses, pairs):
        self.N, self.L, self.M, self.Nrho = N, L, M, Nrho
        self.masses = list(map(float, masses))
        S = self.S = len(self.masses)
        assert len(pairs) == S * S
        self.pairs = []
        for p in range(S):
            for q in range(S):
                pr = pairs[p * S + q]
                self.pairs.append(Pair(N, L, M, Nrho, self.masses[p], self.masses[q],
                                       pr["omega"], pr["alpha"], pr["d"],
                                       pr.get("beta_override", float("nan"))))

    def pair(self, p, q):
        return self.pairs[p * self.S + q]

    def collide_all_hermitian(self, f, points=None):
        """Like collide_all, for the declared Hermitian variant."""
        f = _f64(f)
        P = f.shape[0]
        N, S = self.N, self.S
        f = f.reshape(P, S, N ** 3)
        if points is not None:
            f = np.ascontiguousarray(f[list(points)])
            P = f.shape[0]
        Q = np.empty((P, S, S, N ** 3))
        arr = (ctypes.c_void_p * (S * S))(*[pr._h for pr in self.pairs])
        lib().orc_collide_hermitian_batch(arr, S, P, _ptr(f), _ptr(Q))
        return Q.reshape(P, S, S, N, N, N)

    def collide_all(self, f, points=None):
        """f: [P][S][N,N,N] -> Q: [P][S][S][N,N,N] (all pair operators)."""
        f = _f64(f)
        P = f.shape[0]
        N, S = self.N, self.S
        f = f.reshape(P, S, N ** 3)
        if points is not None:
            f = np.ascontiguousarray(f[list(points)])
            P = f.shape[0]
        Q = np.empty((P, S, S, N ** 3))
        arr = (ctypes.c_void_p * (S * S))(*[pr._h for pr in self.pairs])
        lib().orc_collide_batch(arr, S, P, _ptr(f), _ptr(Q))
        return Q.reshape(P, S, S, N, N, N)

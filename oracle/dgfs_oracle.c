/*
 * dgfs_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * A plain, slow, obviously-correct FP64 CPU implementation of the fast
 * Fourier spectral collision operator Q^(pq)(f_p, f_q) of Jaiswal, Hu,
 * Brillon & Alexeenko, "Fast Fourier spectral ... multi-species DGFS ...
 * on streaming multiprocessors" (PASC'19, arXiv 1903.04670).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference arm may load this library.  It shares no code, header, table or
 * constant generator with the CUDA library; neither includes the other.
 *
 * What it follows, step by step:
 *   - Sec. 2, Eq. (3)-(4) and the beta^(pq) prefactor definition: kernel constants.
 *   - Sec. 2.1, the truncation radius R and the Fourier series with
 *     k in [-N/2, N/2-1]^3.
 *   - Algorithm 1 (pre-computation): wavenumber map, the phase array a, the
 *     kernel-mode tables b^(pq) (Eq. 11) and c^(pq) (Eq. 12-13).  The
 *     pre-computation sphere sum over sigma^pre is taken to its limit
 *     (M^pre -> infinity), i.e. the exact angular integral, evaluated in closed
 *     form with the Funk-Hecke expansion of exp(-i theta k.u).
 *   - Algorithm 2 (collision evaluation), literally: FFT of f_p and f_q, the
 *     (rho, sigma) double loop with t1, t2, t3 and QG, then the loss term and
 *     the real part.  DFTs are unnormalised forward / 1/n inverse (numpy
 *     convention), with which Algorithm 2's normalisation closes exactly.
 *   - The adjoint of the bilinear map (f_p, f_q) -> Q (derived from Eq. 7)
 *     and the derivative with respect to the VHS/VSS exponent omega.
 *   - Moments of Q (mass, momentum, energy) on the cell-centred grid.
 *   - A declared variant that is not in the paper: Algorithm 2 with the
 *     Nyquist planes removed (orc_collide_hermitian), for the real-data form.
 *
 * Readings where the paper is silent or inconsistent (each also listed in the
 * design notes of the repository):
 *   - gamma = 2(1 - omega) (Eq. 3's |u|^{2(1-omega)}), not Algorithm 1's
 *     printed 2(omega - 1).
 *   - sigma runs over the FULL sphere with weights 4 pi / M: octahedron for
 *     M = 6, icosahedron for M = 12 (spherical designs of strength 3 and 5).
 *   - R, the Gauss-Legendre nodes and the phases are per pair (R depends on
 *     the masses of the pair).
 *   - The convolution is cyclic (Algorithm 2 uses FFTs without padding).
 *   - Index N/2 carries wavenumber -N/2 (Algorithm 1, first loop).
 *   - Velocity grid is cell centred: c_j = -L + (j + 1/2) h, h = 2L/N; index
 *     (ix*N + iy)*N + iz, x slowest.
 *   - Kn uses n0 = H0 = 1 and T_ref = T0 (non-dimensional inputs).
 *   - "ifft(QGs)" in Algorithm 2's last line is read as ifft(QG).
 *
 * Parity status: every function here is pinned by tests (FFT vs naive DFT,
 * Gauss-Legendre exactness, design exactness, Funk-Hecke vs direct
 * quadrature, Knudsen numbers of Table 2, brute-force Galerkin sum of Eq. 7,
 * Krook-Wu closed form, equilibrium, conservation, symmetries, dot-product
 * test of the adjoint, finite differences in omega, the loss term against an
 * independent quadrature of the truncated collision frequency for omega != 1
 * (pins the radial weight rho^{gamma+2}), moments of shifted Maxwellians
 * against their closed forms, the VSS (alpha != 1) operator of Maxwell
 * molecules through the closed-form relaxation rate of the traceless stress,
 * and the whole single-species operator at any omega and alpha through the
 * closed-form linearised stress relaxation rate, 2e-4, and the unlike-mass
 * pair operator through the closed-form linearised stress responses to a
 * perturbation of either species, 5e-5).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------ */
/* threads                                                                   */
/* ------------------------------------------------------------------------ */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Discrete Fourier transforms                                               */
/* sign = -1: forward  X_k = sum_j x_j exp(-2 pi i jk/N)   (unnormalised)    */
/* sign = +1: backward X_j = sum_k x_k exp(+2 pi i jk/N)   (unnormalised)    */
/* ------------------------------------------------------------------------ */

/* exp(sign * 2 pi i e / N) with the exponent reduced exactly mod N. */
static cplx unit_root(long e, int N, int sign)
{
    long r = e % N;
    if (r < 0) r += N;
    double ang = 2.0 * ORC_PI * (double)r / (double)N;
    return cos(ang) + (double)sign * sin(ang) * I;
}

/* Naive O(N^2) DFT of one line: the definition, used as the reference for
 * the FFT and as the fallback for prime factors other than 2 and 3. */
void orc_dft_naive_line(int N, const double *in, double *out, int sign)
{
    const cplx *x = (const cplx *)in;
    cplx *X = (cplx *)out;
    for (int k = 0; k < N; ++k) {
        cplx s = 0;
        for (int j = 0; j < N; ++j) s += x[j] * unit_root((long)j * k, N, sign);
        X[k] = s;
    }
}

/* Recursive mixed-radix decimation-in-time Cooley-Tukey: in (strided) ->
 * out (contiguous).  Radices 2 and 3; any other length is done naively. */
static void fft_rec(int N, const cplx *in, long is, cplx *out, int sign)
{
    if (N == 1) {
        out[0] = in[0];
        return;
    }
    int p = (N % 2 == 0) ? 2 : ((N % 3 == 0) ? 3 : 0);
    if (p == 0) {
        for (int k = 0; k < N; ++k) {
            cplx s = 0;
            for (int j = 0; j < N; ++j) s += in[j * is] * unit_root((long)j * k, N, sign);
            out[k] = s;
        }
        return;
    }
    int m = N / p;
    /* sub-transforms of the p interleaved subsequences x[p*j + a] */
    for (int a = 0; a < p; ++a) fft_rec(m, in + a * is, is * p, out + a * m, sign);
    /* butterflies: X[k + q m] = sum_a W_N^{a k} W_p^{a q} Y_a[k] */
    for (int k = 0; k < m; ++k) {
        cplx t[3];
        for (int a = 0; a < p; ++a) t[a] = out[a * m + k] * unit_root((long)a * k, N, sign);
        for (int q = 0; q < p; ++q) {
            cplx s = 0;
            for (int a = 0; a < p; ++a) s += t[a] * unit_root((long)a * q, p, sign);
            out[k + q * m] = s;
        }
    }
}

void orc_fft_line(int N, double *x, int sign)
{
    cplx *v = (cplx *)x;
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    fft_rec(N, v, 1, tmp, sign);
    memcpy(v, tmp, sizeof(cplx) * (size_t)N);
    free(tmp);
}

/* 3-D transform of an N^3 grid (x slowest, z fastest), unnormalised. */
static void fft3(int N, cplx *g, int sign)
{
    long n2 = (long)N * N;
    cplx *line = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    cplx *res = (cplx *)malloc(sizeof(cplx) * (size_t)N);
    /* along z (stride 1), y (stride N), x (stride N^2) */
    for (int axis = 0; axis < 3; ++axis) {
        long stride = (axis == 0) ? 1 : ((axis == 1) ? N : n2);
        for (long a = 0; a < N; ++a)
            for (long b = 0; b < N; ++b) {
                long base;
                if (axis == 0) base = a * n2 + b * N;
                else if (axis == 1) base = a * n2 + b;
                else base = a * N + b;
                for (int j = 0; j < N; ++j) line[j] = g[base + j * stride];
                fft_rec(N, line, 1, res, sign);
                for (int j = 0; j < N; ++j) g[base + j * stride] = res[j];
            }
    }
    free(line);
    free(res);
}

static void ifft3(int N, cplx *g)
{
    long n = (long)N * N * N;
    fft3(N, g, +1);
    double s = 1.0 / (double)n;
    for (long i = 0; i < n; ++i) g[i] *= s;
}

void orc_fft3(int N, double *x, int sign) { fft3(N, (cplx *)x, sign); }

/* ------------------------------------------------------------------------ */
/* Quadratures                                                               */
/* ------------------------------------------------------------------------ */

/* Gauss-Legendre nodes/weights on [a, b] (radial quadrature, Sec. 2.2):
 * Newton iteration on P_n from the three-term recurrence. */
int orc_gauss_legendre(int n, double a, double b, double *x, double *w)
{
    if (n < 1) return -1;
    for (int i = 0; i < n; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double pn = (n == 1) ? z : p1;
            double pm = (n == 1) ? 1.0 : p0;
            dp = n * (z * pn - pm) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        /* recompute derivative at the converged node */
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double pn = (n == 1) ? z : p1;
            double pm = (n == 1) ? 1.0 : p0;
            dp = n * (z * pn - pm) / (z * z - 1.0);
        }
        /* nodes in increasing order on [-1, 1] */
        double xi = -z;
        double wi = 2.0 / ((1.0 - z * z) * dp * dp);
        x[i] = 0.5 * (b - a) * xi + 0.5 * (b + a);
        w[i] = 0.5 * (b - a) * wi;
    }
    return 0;
}

/* Spherical designs on the full sphere (Sec. 2.2 uses Womersley's designs,
 * whose point files are not available here): M = 6 octahedron (strength 3),
 * M = 12 icosahedron (strength 5); weights 4 pi / M. */
int orc_sphere_design(int M, double *sig, double *w)
{
    if (M == 6) {
        static const double oct[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0},
                                         {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
        for (int s = 0; s < 6; ++s)
            for (int d = 0; d < 3; ++d) sig[3 * s + d] = oct[s][d];
    } else if (M == 12) {
        double phi = 0.5 * (1.0 + sqrt(5.0));
        double nrm = sqrt(1.0 + phi * phi);
        double a = 1.0 / nrm, b = phi / nrm;
        int s = 0;
        /* cyclic permutations of (0, +-1, +-phi)/|.| */
        for (int perm = 0; perm < 3; ++perm)
            for (int sg = 0; sg < 4; ++sg) {
                double v[3];
                v[0] = 0.0;
                v[1] = (sg & 2) ? -a : a;
                v[2] = (sg & 1) ? -b : b;
                for (int d = 0; d < 3; ++d) sig[3 * s + d] = v[(d - perm + 3) % 3];
                ++s;
            }
    } else {
        return -1;
    }
    for (int s = 0; s < M; ++s) w[s] = 4.0 * ORC_PI / (double)M;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Kernel constants: Eq. (3)-(4), the beta^(pq) prefactor and R (Sec. 2.1)   */
/* ------------------------------------------------------------------------ */

/* Eq. (4) with n0 = H0 = 1 and T_ref = T0 (non-dimensional diameter d). */
double orc_knudsen(double mp, double mq, double d)
{
    return 1.0 / (sqrt(1.0 + mp / mq) * ORC_PI * d * d);
}

/* Eq. (4) in dimensional form, used to reproduce Table 2's Knudsen numbers. */
double orc_knudsen_dim(double mp, double mq, double n0, double d, double Tref_over_T0,
                       double omega, double H0)
{
    return 1.0 / (sqrt(1.0 + mp / mq) * ORC_PI * n0 * d * d * pow(Tref_over_T0, omega - 0.5) * H0);
}

/* beta^(pq) = (1/Kn) (1 + mp/mq)^{-1/2} (mp mq / (mp + mq))^{-(omega - 1/2)}
 *            * alpha / (2^{1+alpha} Gamma(2.5 - omega) pi)                 */
double orc_beta(double mp, double mq, double omega, double alpha, double d)
{
    double kn = orc_knudsen(mp, mq, d);
    double mr = mp * mq / (mp + mq);
    return (1.0 / kn) / sqrt(1.0 + mp / mq) * pow(mr, -(omega - 0.5)) * alpha /
           (pow(2.0, 1.0 + alpha) * tgamma(2.5 - omega) * ORC_PI);
}

/* Truncation radius R = 4 L / (1 + max(4 mq/(mp+mq), 2) + sqrt(1 + mq/mp)). */
double orc_radius(double L, double mp, double mq)
{
    double t = 4.0 * mq / (mp + mq);
    if (t < 2.0) t = 2.0;
    return 4.0 * L / (1.0 + t + sqrt(1.0 + mq / mp));
}

/* Digamma from the asymptotic series (Abramowitz & Stegun 6.3.18) after
 * shifting the argument up with psi(x) = psi(x+1) - 1/x (A&S 6.3.5). */
double orc_digamma(double x)
{
    double acc = 0.0;
    while (x < 20.0) {
        acc -= 1.0 / x;
        x += 1.0;
    }
    double x2 = 1.0 / (x * x);
    double series = log(x) - 0.5 / x -
                    x2 * (1.0 / 12 - x2 * (1.0 / 120 - x2 * (1.0 / 252 - x2 * (1.0 / 240 - x2 * (1.0 / 132)))));
    return acc + series;
}

/* d ln beta / d omega: beta depends on omega through (mp mq/mu)^{-(omega-1/2)}
 * and 1/Gamma(2.5 - omega); Kn does not (T_ref = T0). */
double orc_dlogbeta_domega(double mp, double mq, double omega)
{
    return -log(mp * mq / (mp + mq)) + orc_digamma(2.5 - omega);
}

/* ------------------------------------------------------------------------ */
/* Angular integral E_eta(theta, k, sigma) = int_{S^2} (1 + sigma.u)^eta      */
/*                                            exp(-i theta k.u) du          */
/* This is the inner integral of Eq. (11) (with B's angular factor           */
/* (1 + cos chi)^{alpha-1}, eta = alpha - 1) and of Eq. (13).                */
/* Evaluated exactly by Funk-Hecke:                                          */
/*   E = 2 pi sum_n (-i)^n (2n+1) lambda_n j_n(theta |k|) P_n(sigma.k^)      */
/*   lambda_n = int_{-1}^{1} (1+t)^eta P_n(t) dt,                            */
/*   lambda_0 = 2^{eta+1}/(eta+1), lambda_{n+1} = lambda_n (eta-n)/(eta+n+2) */
/* ------------------------------------------------------------------------ */

double orc_lambda(int n, double eta)
{
    double lam = pow(2.0, eta + 1.0) / (eta + 1.0);
    for (int j = 0; j < n; ++j) lam *= (eta - j) / (eta + j + 2.0);
    return lam;
}

static cplx angular_integral(double theta, const double k[3], const double sig[3], double eta)
{
    double kn = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
    double x = theta * kn;
    double lam0 = pow(2.0, eta + 1.0) / (eta + 1.0);
    if (x == 0.0) return 2.0 * ORC_PI * lam0; /* only n = 0 survives (j_n(0) = delta_n0) */
    double t = (sig[0] * k[0] + sig[1] * k[1] + sig[2] * k[2]) / kn;
    if (t > 1.0) t = 1.0;
    if (t < -1.0) t = -1.0;

    int nmax = (int)(x + 20.0 + 10.0 * cbrt(x));
    /* lambda_n vanishes for n > eta when eta is a non-negative integer */
    if (eta >= 0.0 && eta == floor(eta) && (int)eta < nmax) nmax = (int)eta;

    /* upward: coef_n = (2n+1) lambda_n P_n(t) */
    double *coef = (double *)malloc(sizeof(double) * (size_t)(nmax + 1));
    {
        double lam = lam0, p0 = 1.0, p1 = t;
        for (int n = 0; n <= nmax; ++n) {
            double pn;
            if (n == 0) pn = 1.0;
            else if (n == 1) pn = t;
            else {
                double p2 = ((2.0 * n - 1.0) * t * p1 - (n - 1.0) * p0) / n;
                p0 = p1;
                p1 = p2;
                pn = p2;
            }
            coef[n] = (2.0 * n + 1.0) * lam * pn;
            lam *= (eta - n) / (eta + n + 2.0);
        }
    }

    /* downward (Miller) recurrence for the spherical Bessel functions
     * j_{n-1} = (2n+1)/x j_n - j_{n+1}, normalised by j_0 or j_1 */
    double top = (x > nmax) ? x : (double)nmax;
    int nstart = (int)top + 20 + (int)sqrt(40.0 * top);
    double jp1 = 0.0, jn = 1e-30;
    double sre = 0.0, sim = 0.0, j0u = 0.0, j1u = 0.0;
    for (int n = nstart; n >= 0; --n) {
        if (n <= nmax) {
            double term = coef[n] * jn;
            switch (n & 3) {
            case 0: sre += term; break;  /* (-i)^0 =  1 */
            case 1: sim -= term; break;  /* (-i)^1 = -i */
            case 2: sre -= term; break;  /* (-i)^2 = -1 */
            default: sim += term; break; /* (-i)^3 =  i */
            }
        }
        if (n == 1) j1u = jn;
        if (n == 0) {
            j0u = jn;
            break;
        }
        double jm1 = (2.0 * n + 1.0) / x * jn - jp1;
        jp1 = jn;
        jn = jm1;
        if (fabs(jn) > 1e200) {
            jn *= 1e-200;
            jp1 *= 1e-200;
            sre *= 1e-200;
            sim *= 1e-200;
            j1u *= 1e-200;
        }
    }
    free(coef);
    double j0 = sin(x) / x;
    double j1 = sin(x) / (x * x) - cos(x) / x;
    double scale = (fabs(j0) >= fabs(j1)) ? j0 / j0u : j1 / j1u;
    return 2.0 * ORC_PI * scale * (sre + sim * I);
}

void orc_angular_integral(double theta, const double *k, const double *sig, double eta, double *out2)
{
    cplx e = angular_integral(theta, k, sig, eta);
    out2[0] = creal(e);
    out2[1] = cimag(e);
}

/* ------------------------------------------------------------------------ */
/* Per-pair plan: quadratures and the tables of Algorithm 1                  */
/* ------------------------------------------------------------------------ */

typedef struct orc_pair {
    int N, M, Nrho;
    double L, mp, mq, omega, alpha, d;
    double gamma, eta, R, beta, dlogbeta;
    int beta_overridden;
    double *rho, *wrho; /* Nrho */
    double *sig, *wsig; /* 3M, M */
    cplx *b;            /* Nrho * M * N^3 : b_{rs}(k) */
    cplx *c;            /* N^3 */
    cplx *c_om;         /* N^3 : c with rho^{gamma+2} -> -2 ln(rho) rho^{gamma+2} */
} orc_pair;

/* wavenumber of grid index x: v_x = x - (x >= N/2) N (Algorithm 1, lines 1-3) */
static int wavenumber(int x, int N) { return x - ((x >= N / 2) ? N : 0); }

void orc_pair_destroy(orc_pair *P)
{
    if (!P) return;
    free(P->rho);
    free(P->wrho);
    free(P->sig);
    free(P->wsig);
    free(P->b);
    free(P->c);
    free(P->c_om);
    free(P);
}

/* beta_override: NaN -> beta from Eq. (4) and the beta^(pq) definition;
 * otherwise used as given (e.g. the constant Krook-Wu kernel). */
orc_pair *orc_pair_create(int N, double L, int M, int Nrho, double mp, double mq, double omega,
                          double alpha, double d, double beta_override)
{
    if (N < 2 || Nrho < 1 || !(L > 0)) return NULL;
    orc_pair *P = (orc_pair *)calloc(1, sizeof(orc_pair));
    P->N = N;
    P->M = M;
    P->Nrho = Nrho;
    P->L = L;
    P->mp = mp;
    P->mq = mq;
    P->omega = omega;
    P->alpha = alpha;
    P->d = d;
    P->gamma = 2.0 * (1.0 - omega); /* reading: Eq. (3)'s |u|^{2(1-omega)} */
    P->eta = alpha - 1.0;
    P->R = orc_radius(L, mp, mq);
    if (isnan(beta_override)) {
        P->beta = orc_beta(mp, mq, omega, alpha, d);
        P->dlogbeta = orc_dlogbeta_domega(mp, mq, omega);
        P->beta_overridden = 0;
    } else {
        P->beta = beta_override;
        P->dlogbeta = 0.0;
        P->beta_overridden = 1;
    }
    P->rho = (double *)malloc(sizeof(double) * Nrho);
    P->wrho = (double *)malloc(sizeof(double) * Nrho);
    P->sig = (double *)malloc(sizeof(double) * 3 * M);
    P->wsig = (double *)malloc(sizeof(double) * M);
    if (orc_sphere_design(M, P->sig, P->wsig) != 0) {
        orc_pair_destroy(P);
        return NULL;
    }
    orc_gauss_legendre(Nrho, 0.0, P->R, P->rho, P->wrho);

    long n = (long)N * N * N;
    P->b = (cplx *)calloc((size_t)Nrho * M * n, sizeof(cplx));
    P->c = (cplx *)calloc((size_t)n, sizeof(cplx));
    P->c_om = (cplx *)calloc((size_t)n, sizeof(cplx));
    double cq = mq / (mp + mq);

    /* b^(pq)_{rs}(k) = rho_r^{gamma+2} E_eta(pi/L rho_r mq/(mp+mq), k, sigma_s)
     * (Algorithm 1 line 13 with M^pre -> infinity; Eq. (11)) */
    for (int r = 0; r < Nrho; ++r)
        for (int s = 0; s < M; ++s) {
            cplx *brs = P->b + ((long)r * M + s) * n;
            double theta = ORC_PI / L * P->rho[r] * cq;
            double rg = pow(P->rho[r], P->gamma + 2.0);
#pragma omp parallel for schedule(dynamic, 64)
            for (long idx = 0; idx < n; ++idx) {
                int ix = (int)(idx / ((long)N * N)), iy = (int)((idx / N) % N), iz = (int)(idx % N);
                double k[3] = {wavenumber(ix, N), wavenumber(iy, N), wavenumber(iz, N)};
                brs[idx] = rg * angular_integral(theta, k, P->sig + 3 * s, P->eta);
            }
        }
    /* c^(pq)_k = sum_{r,s} w_r w_s rho_r^{gamma+2} E_eta(pi/L rho_r, k, sigma_s)
     * (Algorithm 1 line 14; Eq. (13)) */
#pragma omp parallel for schedule(dynamic, 64)
    for (long idx = 0; idx < n; ++idx) {
        int ix = (int)(idx / ((long)N * N)), iy = (int)((idx / N) % N), iz = (int)(idx % N);
        double k[3] = {wavenumber(ix, N), wavenumber(iy, N), wavenumber(iz, N)};
        cplx acc = 0, acc_om = 0;
        for (int r = 0; r < Nrho; ++r) {
            double theta = ORC_PI / L * P->rho[r];
            double rg = pow(P->rho[r], P->gamma + 2.0);
            for (int s = 0; s < M; ++s) {
                cplx e = P->wrho[r] * P->wsig[s] * rg * angular_integral(theta, k, P->sig + 3 * s, P->eta);
                acc += e;
                acc_om += -2.0 * log(P->rho[r]) * e;
            }
        }
        P->c[idx] = acc;
        P->c_om[idx] = acc_om;
    }
    return P;
}

/* Export the plan's scalars and tables (for tests and for brute force). */
void orc_pair_scalars(const orc_pair *P, double *out8)
{
    out8[0] = P->R;
    out8[1] = P->beta;
    out8[2] = P->gamma;
    out8[3] = P->eta;
    out8[4] = P->dlogbeta;
    out8[5] = P->mq / (P->mp + P->mq);
    out8[6] = P->mp / (P->mp + P->mq);
    out8[7] = (double)P->beta_overridden;
}

void orc_pair_quadrature(const orc_pair *P, double *rho, double *wrho, double *sig, double *wsig)
{
    memcpy(rho, P->rho, sizeof(double) * P->Nrho);
    memcpy(wrho, P->wrho, sizeof(double) * P->Nrho);
    memcpy(sig, P->sig, sizeof(double) * 3 * P->M);
    memcpy(wsig, P->wsig, sizeof(double) * P->M);
}

void orc_pair_tables(const orc_pair *P, double *b, double *c, double *c_om)
{
    long n = (long)P->N * P->N * P->N;
    if (b) memcpy(b, P->b, sizeof(cplx) * (size_t)P->Nrho * P->M * n);
    if (c) memcpy(c, P->c, sizeof(cplx) * (size_t)n);
    if (c_om) memcpy(c_om, P->c_om, sizeof(cplx) * (size_t)n);
}

/* a_{rs}(l) = pi/L rho_r (l . sigma_s)   (Algorithm 1, line 7) */
static double phase_arg(const orc_pair *P, int r, int s, long idx)
{
    int N = P->N;
    int ix = (int)(idx / ((long)N * N)), iy = (int)((idx / N) % N), iz = (int)(idx % N);
    const double *sg = P->sig + 3 * s;
    double ldots = wavenumber(ix, N) * sg[0] + wavenumber(iy, N) * sg[1] + wavenumber(iz, N) * sg[2];
    return ORC_PI / P->L * P->rho[r] * ldots;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2: one evaluation of Q^(pq)(f_p, f_q) at one spatial point      */
/*   Q     : out, N^3 real                                                   */
/*   dQdw  : optional out, dQ/d omega (N^3 real), may be NULL                */
/*   diag  : optional out[4] = {max|Im| of the final complex result,         */
/*           max|gain|, max|loss|, max|Q|}  (all after the beta factor)      */
/* ------------------------------------------------------------------------ */
void orc_collide(const orc_pair *P, const double *fp, const double *fq, double *Q, double *dQdw,
                 double *diag)
{
    int N = P->N;
    long n = (long)N * N * N;
    double cq = P->mq / (P->mp + P->mq), cp = P->mp / (P->mp + P->mq);
    cplx *FTf = (cplx *)malloc(sizeof(cplx) * n);
    cplx *FTg = (cplx *)malloc(sizeof(cplx) * n);
    cplx *QG = (cplx *)calloc((size_t)n, sizeof(cplx));
    cplx *QGw = (cplx *)calloc((size_t)n, sizeof(cplx));
    cplx *t1 = (cplx *)malloc(sizeof(cplx) * n);
    cplx *t2 = (cplx *)malloc(sizeof(cplx) * n);

    /* step 1: forward FFTs */
    for (long i = 0; i < n; ++i) {
        FTf[i] = fp[i];
        FTg[i] = fq[i];
    }
    fft3(N, FTf, -1);
    fft3(N, FTg, -1);

    /* steps 2-8: the (rho, sigma) loop */
    for (int r = 0; r < P->Nrho; ++r)
        for (int s = 0; s < P->M; ++s) {
            for (long i = 0; i < n; ++i) {
                double a = phase_arg(P, r, s, i);
                t1[i] = cexp(I * cq * a) * FTf[i];  /* step 4 */
                t2[i] = cexp(-I * cp * a) * FTg[i]; /* step 5 */
            }
            ifft3(N, t1); /* step 6: t3 = fft(ifft(t1) * ifft(t2)) */
            ifft3(N, t2);
            for (long i = 0; i < n; ++i) t1[i] *= t2[i];
            fft3(N, t1, -1);
            const cplx *brs = P->b + ((long)r * P->M + s) * n;
            double w = P->wrho[r] * P->wsig[s];
            double wl = -2.0 * log(P->rho[r]) * w;
            for (long i = 0; i < n; ++i) {
                QG[i] += w * brs[i] * t1[i]; /* step 7 */
                QGw[i] += wl * brs[i] * t1[i];
            }
        }

    /* step 10: Q = beta * real(ifft(QG) - f_p * ifft(c * FTg)) */
    ifft3(N, QG);
    for (long i = 0; i < n; ++i) t2[i] = P->c[i] * FTg[i];
    ifft3(N, t2);
    double imax = 0, gmax = 0, lmax = 0, qmax = 0;
    for (long i = 0; i < n; ++i) {
        cplx z = QG[i] - fp[i] * t2[i];
        Q[i] = P->beta * creal(z);
        double ai = fabs(P->beta * cimag(z));
        double ag = fabs(P->beta * creal(QG[i]));
        double al = fabs(P->beta * creal(fp[i] * t2[i]));
        if (ai > imax) imax = ai;
        if (ag > gmax) gmax = ag;
        if (al > lmax) lmax = al;
        if (fabs(Q[i]) > qmax) qmax = fabs(Q[i]);
    }
    if (dQdw) {
        /* dQ/domega = (dlnbeta/domega) Q + beta Re(ifft(QG_w) - f_p ifft(c_w FTg)) */
        ifft3(N, QGw);
        for (long i = 0; i < n; ++i) t2[i] = P->c_om[i] * FTg[i];
        ifft3(N, t2);
        for (long i = 0; i < n; ++i)
            dQdw[i] = P->dlogbeta * Q[i] + P->beta * creal(QGw[i] - fp[i] * t2[i]);
    }
    if (diag) {
        diag[0] = imax;
        diag[1] = gmax;
        diag[2] = lmax;
        diag[3] = qmax;
    }
    free(FTf);
    free(FTg);
    free(QG);
    free(QGw);
    free(t1);
    free(t2);
}

/* ------------------------------------------------------------------------ */
/* Declared variant (not in the paper): Algorithm 2 on the Hermitian          */
/* subspace.  With N even, the wavenumber -N/2 has no +N/2 partner on the     */
/* grid (Algorithm 1's wavenumber map), so a translate of a real f is not    */
/* exactly real.  Let P zero every Fourier mode with an index equal to N/2   */
/* (the Nyquist planes).  Then                                               */
/*   F~ = P fft(f),  f~ = ifft(F~) (real),                                   */
/*   QG = sum_rs w_r w_s b_rs . fft(ifft(e^{+i cq a} F~_p) . ifft(e^{-i cp a} F~_q)),  */
/*   Q  = beta ( ifft(P QG) - f~_p . ifft(c . F~_q) ).                        */
/* Every translate is real, and so are both terms of Q, because b_rs and c    */
/* satisfy X(-k) = conj X(k) on the Nyquist-free wavenumbers; the real part  */
/* taken at the end only drops rounding.                                     */
/* ------------------------------------------------------------------------ */
static int on_nyquist_plane(long idx, int N)
{
    int ix = (int)(idx / ((long)N * N)), iy = (int)((idx / N) % N), iz = (int)(idx % N);
    return (N % 2 == 0) && (ix == N / 2 || iy == N / 2 || iz == N / 2);
}

void orc_collide_hermitian(const orc_pair *P, const double *fp, const double *fq, double *Q)
{
    int N = P->N;
    long n = (long)N * N * N;
    double cq = P->mq / (P->mp + P->mq), cp = P->mp / (P->mp + P->mq);
    cplx *FTf = (cplx *)malloc(sizeof(cplx) * n);
    cplx *FTg = (cplx *)malloc(sizeof(cplx) * n);
    cplx *ft = (cplx *)malloc(sizeof(cplx) * n);
    cplx *QG = (cplx *)calloc((size_t)n, sizeof(cplx));
    cplx *t1 = (cplx *)malloc(sizeof(cplx) * n);
    cplx *t2 = (cplx *)malloc(sizeof(cplx) * n);

    /* F~_p, F~_q and f~_p */
    for (long i = 0; i < n; ++i) {
        FTf[i] = fp[i];
        FTg[i] = fq[i];
    }
    fft3(N, FTf, -1);
    fft3(N, FTg, -1);
    for (long i = 0; i < n; ++i)
        if (on_nyquist_plane(i, N)) FTf[i] = FTg[i] = 0;
    for (long i = 0; i < n; ++i) ft[i] = FTf[i];
    ifft3(N, ft);

    /* the (rho, sigma) loop of Algorithm 2 on the projected spectra */
    for (int r = 0; r < P->Nrho; ++r)
        for (int s = 0; s < P->M; ++s) {
            for (long i = 0; i < n; ++i) {
                double a = phase_arg(P, r, s, i);
                t1[i] = cexp(I * cq * a) * FTf[i];
                t2[i] = cexp(-I * cp * a) * FTg[i];
            }
            ifft3(N, t1);
            ifft3(N, t2);
            for (long i = 0; i < n; ++i) t1[i] *= t2[i];
            fft3(N, t1, -1);
            const cplx *brs = P->b + ((long)r * P->M + s) * n;
            double w = P->wrho[r] * P->wsig[s];
            for (long i = 0; i < n; ++i) QG[i] += w * brs[i] * t1[i];
        }

    /* Q = beta ( ifft(P QG) - f~_p . ifft(c . F~_q) ) */
    for (long i = 0; i < n; ++i)
        if (on_nyquist_plane(i, N)) QG[i] = 0;
    ifft3(N, QG);
    for (long i = 0; i < n; ++i) t2[i] = P->c[i] * FTg[i];
    ifft3(N, t2);
    for (long i = 0; i < n; ++i) Q[i] = P->beta * creal(QG[i] - creal(ft[i]) * t2[i]);
    free(FTf);
    free(FTg);
    free(ft);
    free(QG);
    free(t1);
    free(t2);
}

/* Batched driver of the Hermitian variant, like orc_collide_batch. */
void orc_collide_hermitian_batch(orc_pair **pairs, int S, int Pn, const double *f, double *Q)
{
    int N = pairs[0]->N;
    long n = (long)N * N * N;
    long total = (long)Pn * S * S;
#pragma omp parallel for schedule(dynamic, 1)
    for (long e = 0; e < total; ++e) {
        long pt = e / (S * S);
        int p = (int)((e / S) % S), q = (int)(e % S);
        orc_collide_hermitian(pairs[p * S + q], f + (pt * S + p) * n, f + (pt * S + q) * n, Q + e * n);
    }
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the bilinear map.  With K_rs = w_rs ifft3 diag(b_rs) fft3,     */
/* T+_rs = ifft3 diag(exp(+i cq a_rs)) fft3, T-_rs = ifft3 diag(exp(-i cp a_rs)) fft3, */
/* S = ifft3 diag(c) fft3:                                                   */
/*   Q = beta Re( sum_rs K_rs (T+ f_p . T- f_q) - f_p . S f_q )              */
/* and for a real upstream gbar, L = <gbar, Q>:                             */
/*   dL/df_p = beta Re sum_rs T+^H [ conj(T- f_q) . K^H gbar ]              */
/*             - beta gbar . Re(S f_q)                                       */
/*   dL/df_q = beta Re sum_rs T-^H [ conj(T+ f_p) . K^H gbar ]              */
/*             - beta Re( S^H (gbar . f_p) )                                 */
/* with K^H = w ifft3 diag(conj b) fft3, T^H = ifft3 diag(conj phase) fft3,  */
/* S^H = ifft3 diag(conj c) fft3.                                            */
/*   dL/domega = <gbar, dQ/domega>                                           */
/* ------------------------------------------------------------------------ */
void orc_adjoint(const orc_pair *P, const double *fp, const double *fq, const double *gbar,
                 double *dfp, double *dfq, double *domega)
{
    int N = P->N;
    long n = (long)N * N * N;
    double cq = P->mq / (P->mp + P->mq), cp = P->mp / (P->mp + P->mq);
    cplx *Fp = (cplx *)malloc(sizeof(cplx) * n);
    cplx *Fq = (cplx *)malloc(sizeof(cplx) * n);
    cplx *G = (cplx *)malloc(sizeof(cplx) * n);
    cplx *A = (cplx *)malloc(sizeof(cplx) * n);
    cplx *B = (cplx *)malloc(sizeof(cplx) * n);
    cplx *V = (cplx *)malloc(sizeof(cplx) * n);
    cplx *U = (cplx *)malloc(sizeof(cplx) * n);
    cplx *accp = (cplx *)calloc((size_t)n, sizeof(cplx));
    cplx *accq = (cplx *)calloc((size_t)n, sizeof(cplx));
    for (long i = 0; i < n; ++i) {
        Fp[i] = fp[i];
        Fq[i] = fq[i];
        G[i] = gbar[i];
    }
    fft3(N, Fp, -1);
    fft3(N, Fq, -1);
    fft3(N, G, -1);
    for (int r = 0; r < P->Nrho; ++r)
        for (int s = 0; s < P->M; ++s) {
            const cplx *brs = P->b + ((long)r * P->M + s) * n;
            double w = P->wrho[r] * P->wsig[s];
            for (long i = 0; i < n; ++i) {
                double a = phase_arg(P, r, s, i);
                A[i] = cexp(I * cq * a) * Fp[i];
                B[i] = cexp(-I * cp * a) * Fq[i];
                V[i] = w * conj(brs[i]) * G[i];
            }
            ifft3(N, A); /* A = T+ f_p */
            ifft3(N, B); /* B = T- f_q */
            ifft3(N, V); /* V = K^H gbar */
            /* p side: T+^H [conj(B) V] */
            for (long i = 0; i < n; ++i) U[i] = conj(B[i]) * V[i];
            fft3(N, U, -1);
            for (long i = 0; i < n; ++i) U[i] *= cexp(-I * cq * phase_arg(P, r, s, i));
            ifft3(N, U);
            for (long i = 0; i < n; ++i) accp[i] += U[i];
            /* q side: T-^H [conj(A) V] */
            for (long i = 0; i < n; ++i) U[i] = conj(A[i]) * V[i];
            fft3(N, U, -1);
            for (long i = 0; i < n; ++i) U[i] *= cexp(I * cp * phase_arg(P, r, s, i));
            ifft3(N, U);
            for (long i = 0; i < n; ++i) accq[i] += U[i];
        }
    /* loss terms */
    for (long i = 0; i < n; ++i) U[i] = P->c[i] * Fq[i];
    ifft3(N, U); /* S f_q */
    for (long i = 0; i < n; ++i) dfp[i] = P->beta * creal(accp[i]) - P->beta * gbar[i] * creal(U[i]);
    for (long i = 0; i < n; ++i) U[i] = gbar[i] * fp[i];
    fft3(N, U, -1);
    for (long i = 0; i < n; ++i) U[i] *= conj(P->c[i]);
    ifft3(N, U); /* S^H (gbar f_p) */
    for (long i = 0; i < n; ++i) dfq[i] = P->beta * creal(accq[i]) - P->beta * creal(U[i]);
    if (domega) {
        double *Q = (double *)malloc(sizeof(double) * n);
        double *dQ = (double *)malloc(sizeof(double) * n);
        orc_collide(P, fp, fq, Q, dQ, NULL);
        double s = 0;
        for (long i = 0; i < n; ++i) s += gbar[i] * dQ[i];
        *domega = s;
        free(Q);
        free(dQ);
    }
    free(Fp);
    free(Fq);
    free(G);
    free(A);
    free(B);
    free(V);
    free(U);
    free(accp);
    free(accq);
}

/* ------------------------------------------------------------------------ */
/* Moments of Q on the cell-centred grid c_j = -L + (j + 1/2) h, h = 2L/N:   */
/*   out = h^3 sum_j Q_j * {1, m c_x, m c_y, m c_z, m |c|^2}                 */
/* ------------------------------------------------------------------------ */
void orc_moments(int N, double L, double m, const double *Q, double *out5)
{
    double h = 2.0 * L / N;
    double acc[5] = {0, 0, 0, 0, 0};
    for (int ix = 0; ix < N; ++ix)
        for (int iy = 0; iy < N; ++iy)
            for (int iz = 0; iz < N; ++iz) {
                double cx = -L + (ix + 0.5) * h, cy = -L + (iy + 0.5) * h, cz = -L + (iz + 0.5) * h;
                double q = Q[((long)ix * N + iy) * N + iz];
                acc[0] += q;
                acc[1] += m * cx * q;
                acc[2] += m * cy * q;
                acc[3] += m * cz * q;
                acc[4] += m * (cx * cx + cy * cy + cz * cz) * q;
            }
    double h3 = h * h * h;
    for (int i = 0; i < 5; ++i) out5[i] = h3 * acc[i];
}

/* Batched driver: all (point, pair) evaluations of a multi-species problem.
 * f: [P][S][N^3], Q: [P][S][S][N^3] (p-major, q-minor).  pairs[p*S+q] must be
 * created with masses (m_p, m_q).  Evaluations run in parallel over
 * (point, pair) with OpenMP when available. */
void orc_collide_batch(orc_pair **pairs, int S, int Pn, const double *f, double *Q)
{
    int N = pairs[0]->N;
    long n = (long)N * N * N;
    long total = (long)Pn * S * S;
#pragma omp parallel for schedule(dynamic, 1)
    for (long e = 0; e < total; ++e) {
        long pt = e / (S * S);
        int p = (int)((e / S) % S), q = (int)(e % S);
        orc_collide(pairs[p * S + q], f + (pt * S + p) * n, f + (pt * S + q) * n, Q + e * n, NULL, NULL);
    }
}

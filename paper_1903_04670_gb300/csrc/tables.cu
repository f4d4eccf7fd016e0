// Pre-computation of Algorithm 1 (Sec. 2.2) on the device, in FP64.
//
//  - twiddles of the length-N DFT,
//  - separable phase vectors: the phase exp(i c a_rs(l)) with
//    a_rs(l) = pi/L rho_r (l . sigma_s) factorises over the three axes, so it
//    is stored as 3 vectors of N entries per (r, s) and side,
//  - b^(pq)_rs(k) = rho_r^{gamma+2} E_eta(pi/L rho_r m_q/(m_p+m_q), k, sigma_s)  (Eq. 11),
//  - c^(pq)_k = sum_rs w_r w_s rho_r^{gamma+2} E_eta(pi/L rho_r, k, sigma_s)      (Eq. 12-13),
// where E_eta(theta, k, sigma) = int_{S^2} (1 + sigma.u)^eta exp(-i theta k.u) du is the
// angular integral of Algorithm 1's pre-computation sphere taken to its limit
// (M^pre -> infinity), evaluated exactly with the Funk-Hecke expansion
//   E = 2 pi sum_n (-i)^n (2n+1) lambda_n j_n(theta|k|) P_n(sigma.k/|k|),
//   lambda_n = int_{-1}^{1} (1+t)^eta P_n(t) dt (two-term ratio recurrence),
// with the spherical Bessel functions from Miller's downward recurrence.
#include <cmath>

#include "dgfs_internal.h"

namespace dgfs {
namespace {

constexpr int kMaxTerms = 288;  // Funk-Hecke terms; theta|k| <= pi * sqrt(3) * 24 for N <= 48

__device__ __forceinline__ int wavenum(int i, int N) { return i < N / 2 ? i : i - N; }

// Funk-Hecke evaluation of E_eta.  `scratch` holds kMaxTerms doubles.
__device__ double2 angular_integral(double theta, double kx, double ky, double kz, const double *sig,
                                    double eta, double *scratch, int *overflow)
{
    const double kn = sqrt(kx * kx + ky * ky + kz * kz);
    const double x = theta * kn;
    const double lam0 = exp2(eta + 1.0) / (eta + 1.0);
    if (x == 0.0) return make_double2(2.0 * kPi * lam0, 0.0);
    double t = (sig[0] * kx + sig[1] * ky + sig[2] * kz) / kn;
    t = fmin(1.0, fmax(-1.0, t));

    int nmax = (int)(x + 20.0 + 10.0 * cbrt(x));
    if (eta >= 0.0 && eta == floor(eta) && (int)eta < nmax) nmax = (int)eta;
    if (nmax >= kMaxTerms) {
        *overflow = 1;
        nmax = kMaxTerms - 1;
    }
    // coefficient of j_n: (2n+1) lambda_n P_n(t), built upward
    double lam = lam0, pm1 = 0.0, p = 1.0;
    for (int n = 0; n <= nmax; ++n) {
        scratch[n] = (2.0 * n + 1.0) * lam * p;
        const double pn1 = ((2.0 * n + 1.0) * t * p - n * pm1) / (n + 1.0);
        pm1 = p;
        p = pn1;
        lam *= (eta - n) / (eta + n + 2.0);
    }
    // Miller: start well above max(x, nmax), recur downward, normalise by j0 or j1
    const double top = fmax(x, (double)nmax);
    const int nstart = (int)top + 20 + (int)sqrt(40.0 * top);
    double jp = 0.0, jc = 1e-30, re = 0.0, im = 0.0, j1u = 0.0, j0u = 1.0;
    for (int n = nstart; n >= 0; --n) {
        if (n <= nmax) {
            const double v = scratch[n] * jc;
            const int ph = n & 3;  // (-i)^n = 1, -i, -1, i
            if (ph == 0) re += v;
            else if (ph == 1) im -= v;
            else if (ph == 2) re -= v;
            else im += v;
        }
        if (n == 1) j1u = jc;
        if (n == 0) {
            j0u = jc;
            break;
        }
        const double jm = (2.0 * n + 1.0) / x * jc - jp;
        jp = jc;
        jc = jm;
        if (fabs(jc) > 1e200) {
            jc *= 1e-200;
            jp *= 1e-200;
            re *= 1e-200;
            im *= 1e-200;
            j1u *= 1e-200;
        }
    }
    double s, c;
    sincos(x, &s, &c);
    const double j0 = s / x, j1 = s / (x * x) - c / x;
    const double scale = (fabs(j0) >= fabs(j1)) ? j0 / j0u : j1 / j1u;
    return make_double2(2.0 * kPi * scale * re, 2.0 * kPi * scale * im);
}

__global__ void k_twiddle(double2 *tw, int N)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double s, c;
    sincospi(2.0 * j / N, &s, &c);
    tw[j] = make_double2(c, -s);
}

// quad: [rho(Nrho), wrho(Nrho), sigma(3M), wsig(M)]
__global__ void k_phase(double2 *phase, const double *quad, int N, int M, int Nrho, double L, double cq,
                        double cp)
{
    const int RS = Nrho * M;
    const long total = (long)RS * 2 * 3 * N;
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int l = (int)(i % N);
    const int ax = (int)((i / N) % 3);
    const int side = (int)((i / (3 * N)) % 2);
    const int rs = (int)(i / (6 * N));
    const int r = rs / M, s = rs % M;
    const double *rho = quad, *sig = quad + 2 * Nrho;
    // argument / pi = (+cq | -cp) * rho_r / L * sigma_{s,ax} * l
    const double coef = side == 0 ? cq : -cp;
    const double a = coef * rho[r] / L * sig[3 * s + ax] * (double)wavenum(l, N);
    double sn, cs;
    sincospi(a, &sn, &cs);
    phase[i] = make_double2(cs, sn);
}

__global__ void k_btable(double2 *b, const double *quad, int N, int M, int Nrho, double L, double cq,
                         double gamma, double eta, int *overflow)
{
    const long n = (long)N * N * N;
    const int RS = Nrho * M;
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * RS) return;
    double scratch[kMaxTerms];
    const long idx = i % n;
    const int rs = (int)(i / n);
    const int r = rs / M, s = rs % M;
    const double *rho = quad, *sig = quad + 2 * Nrho;
    const int ix = (int)(idx / ((long)N * N)), iy = (int)((idx / N) % N), iz = (int)(idx % N);
    const double theta = kPi / L * rho[r] * cq;
    const double e = pow(rho[r], gamma + 2.0);
    double2 v = angular_integral(theta, wavenum(ix, N), wavenum(iy, N), wavenum(iz, N), sig + 3 * s, eta,
                                 scratch, overflow);
    b[i] = make_double2(e * v.x, e * v.y);
}

__global__ void k_ctable(double2 *c, double2 *c_om, const double *quad, int N, int M, int Nrho, double L,
                         double gamma, double eta, int *overflow)
{
    const long n = (long)N * N * N;
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    double scratch[kMaxTerms];
    const double *rho = quad, *wrho = quad + Nrho, *sig = quad + 2 * Nrho, *wsig = quad + 2 * Nrho + 3 * M;
    const int ix = (int)(idx / ((long)N * N)), iy = (int)((idx / N) % N), iz = (int)(idx % N);
    double cr = 0, ci = 0, or_ = 0, oi = 0;
    for (int r = 0; r < Nrho; ++r) {
        const double theta = kPi / L * rho[r];
        const double e = pow(rho[r], gamma + 2.0) * wrho[r];
        const double lg = -2.0 * log(rho[r]);
        for (int s = 0; s < M; ++s) {
            double2 v = angular_integral(theta, wavenum(ix, N), wavenum(iy, N), wavenum(iz, N), sig + 3 * s,
                                         eta, scratch, overflow);
            const double f = e * wsig[s];
            cr += f * v.x;
            ci += f * v.y;
            or_ += lg * f * v.x;
            oi += lg * f * v.y;
        }
    }
    c[idx] = make_double2(cr, ci);
    c_om[idx] = make_double2(or_, oi);
}

__global__ void k_weights(double *w, double *wlog, const double *quad, int M, int Nrho)
{
    int rs = blockIdx.x * blockDim.x + threadIdx.x;
    if (rs >= Nrho * M) return;
    const double *rho = quad, *wrho = quad + Nrho, *wsig = quad + 2 * Nrho + 3 * M;
    const int r = rs / M, s = rs % M;
    w[rs] = wrho[r] * wsig[s];
    wlog[rs] = -2.0 * log(rho[r]) * wrho[r] * wsig[s];
}

unsigned blocks_for(long total, int threads) { return (unsigned)((total + threads - 1) / threads); }

}  // namespace

dgfs_status build_pair_tables(dgfs_plan_s *plan, int *d_over);

dgfs_status build_tables(dgfs_plan_s *plan)
{
    const int N = plan->N;
    DGFS_CUDA(dev_malloc(&plan->twiddle, sizeof(double2) * N));
    k_twiddle<<<1, 64>>>(plan->twiddle, N);
    DGFS_LAUNCHED(plan);

    int *d_over = nullptr;
    DGFS_CUDA(dev_malloc(&d_over, sizeof(int)));
    const dgfs_status st = build_pair_tables(plan, d_over);
    dev_free(d_over);
    return st;
}

// b, c, c_omega, phases and weights of every pair; d_over receives the
// overflow flag of the angular-integral kernels
dgfs_status build_pair_tables(dgfs_plan_s *plan, int *d_over)
{
    const int N = plan->N, M = plan->M, Nrho = plan->Nrho, RS = Nrho * M;
    const long n = (long)N * N * N;
    DGFS_CUDA(cudaMemset(d_over, 0, sizeof(int)));
    const size_t qn = 2 * Nrho + 4 * M;
    DGFS_CUDA(dev_malloc(&plan->quad_dev, sizeof(double) * qn));
    std::vector<double> quad(qn);
    for (auto &pt : plan->pairs) {
        for (int r = 0; r < Nrho; ++r) {
            quad[r] = pt.rho[r];
            quad[Nrho + r] = pt.wrho[r];
        }
        for (int i = 0; i < 3 * M; ++i) quad[2 * Nrho + i] = plan->sigma[i];
        for (int s = 0; s < M; ++s) quad[2 * Nrho + 3 * M + s] = plan->wsig[s];
        DGFS_CUDA(cudaMemcpy(plan->quad_dev, quad.data(), sizeof(double) * qn, cudaMemcpyHostToDevice));
        DGFS_CUDA(dev_malloc(&pt.b, sizeof(double2) * RS * n));
        DGFS_CUDA(dev_malloc(&pt.c, sizeof(double2) * n));
        DGFS_CUDA(dev_malloc(&pt.c_om, sizeof(double2) * n));
        DGFS_CUDA(dev_malloc(&pt.phase, sizeof(double2) * RS * 6 * N));
        DGFS_CUDA(dev_malloc(&pt.w, sizeof(double) * RS));
        DGFS_CUDA(dev_malloc(&pt.wlog, sizeof(double) * RS));
        plan->table_bytes += sizeof(double2) * (RS * n + 2 * n + RS * 6 * N) + 2 * sizeof(double) * RS;

        k_phase<<<blocks_for((long)RS * 6 * N, 256), 256>>>(pt.phase, plan->quad_dev, N, M, Nrho, plan->L,
                                                             pt.cq, pt.cp);
        DGFS_LAUNCHED(plan);
        k_btable<<<blocks_for(n * RS, 128), 128>>>(pt.b, plan->quad_dev, N, M, Nrho, plan->L, pt.cq,
                                                    pt.gamma, pt.eta, d_over);
        DGFS_LAUNCHED(plan);
        k_ctable<<<blocks_for(n, 128), 128>>>(pt.c, pt.c_om, plan->quad_dev, N, M, Nrho, plan->L, pt.gamma,
                                               pt.eta, d_over);
        DGFS_LAUNCHED(plan);
        k_weights<<<blocks_for(RS, 128), 128>>>(pt.w, pt.wlog, plan->quad_dev, M, Nrho);
        DGFS_LAUNCHED(plan);
        // quad_dev is reused by the next pair: finish this pair's kernels first
        DGFS_CUDA(cudaDeviceSynchronize());
    }
    int over = 0;
    DGFS_CUDA(cudaMemcpy(&over, d_over, sizeof(int), cudaMemcpyDeviceToHost));
    if (over) {
        set_error("angular integral needs more Funk-Hecke terms than the table kernel holds");
        return DGFS_EUNSUPPORTED;
    }
    return DGFS_OK;
}

}  // namespace dgfs

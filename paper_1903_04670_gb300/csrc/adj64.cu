// FP64 adjoint of the bilinear collision map (f_p, f_q) -> Q^(pq) and its
// derivative with respect to the VHS/VSS exponent omega.
//
// With K_rs = w_rs ifft3 diag(b_rs) fft3, the translates T+_rs = ifft3 diag(phi+) fft3,
// T-_rs = ifft3 diag(phi-) fft3 (Algorithm 2 steps 4-6) and S = ifft3 diag(c) fft3,
//   Q = beta Re( sum_rs K_rs (T+ f_p . T- f_q) - f_p . S f_q )          (Eq. 7, Algorithm 2)
// is bilinear, and for a real upstream gradient g, L = <g, Q>:
//   dL/df_p = beta Re sum_rs T+^H [conj(B_rs) V_rs] - beta g . Re(S f_q)
//   dL/df_q = beta Re sum_rs T-^H [conj(A_rs) V_rs] - beta Re(S^H (g . f_p))
//   V_rs = K^H g = w_rs ifft3(conj(b_rs) fft3(g)),  A = T+ f_p,  B = T- f_q,
// T^H = ifft3 diag(conj phi) fft3 factorises per axis.  The omega derivative:
//   d beta/d omega / beta = psi(2.5 - omega) - ln(m_p m_q / (m_p + m_q)),
//   d rho^{gamma+2} / d omega = -2 ln(rho) rho^{gamma+2}, so
//   <g, dQ/domega> = (dlnbeta) <g, Q>
//                    + beta ( sum_rs (wlog_rs / w_rs) Re<V_rs, A B> - <g f_p, Re(S_w f_q)> ),
//   <g, Q> = beta ( sum_rs Re<V_rs, A B> - <g f_p, Re(S f_q)> ),
// with S_w built from c_omega (c with -2 ln(rho_r) weights).
//
// Passes per (point, r, s), all FFTs unnormalised (scales folded in at the end):
//   J1 x: A = ifft_x(phi+_x F_p), B = ifft_x(phi-_x F_q), V = ifft_x(conj(b) G)
//   J2 y: the same three grids along y
//   J3 z: along z; then s_rs += Re sum conj(V) A B, U_p = conj(B) V, U_q = conj(A) V,
//         and the z factor of T^H: ifft_z(conj(phi_z) fft_z(U))
//   J4 y: y factor of T^H on U_p, U_q
//   J5 x: x factor of T^H, accumulated over all (r, s) in-thread, real parts kept.
// Per point: G = fft3(g), S f_q, S_w f_q, S^H (g f_p) and the final combination.
#include <algorithm>

#include "dgfs_internal.h"
#include "fftreg.cuh"

namespace dgfs {
namespace {

using reg::cmul;
using reg::cmulc;
using reg::fft;

__device__ __forceinline__ double2 conjd(double2 a) { return make_double2(a.x, -a.y); }

template <int N, int AXIS>
__device__ __forceinline__ long poff(int pi, int j)
{
    if constexpr (AXIS == 0) return (long)j * N * N + pi;
    else if constexpr (AXIS == 1) return (long)(pi / N) * N * N + (long)j * N + (pi % N);
    else return (long)pi * N + j;
}

enum AMode {
    G_FWD_REAL = 0,  // X = fft_axis(real src)       (g or g.f_p; grid.z = point)
    G_FWD,           // in-place forward on X
    J1,              // A, B, V from F_p, F_q, G (x)
    J2,              // A, B, V inverse along y
    J3,              // along z, products, dot, z factor of T^H
    J4,              // y factor of T^H on U_p, U_q
    J5,              // x factor of T^H, accumulate over (r, s)
    L1,              // loss grids: L = ifft(c F_q), Lw = ifft(c_w F_q), Y = ifft(conj(c) GF) (x)
    L2,              // the three loss grids along y (inverse)
    L3,              // along z, then combine into df and the omega dot
    X_INV,           // in-place inverse along the axis on X (grid.z = eval)
    X_INV_RE,        // inverse along the axis, xout = xscale Re(result)
};

constexpr int kAdjMaxPairs = 16;  // S * S, S <= 4

struct AdjArgs {
    long n;
    int S, p, q, pt0, RS;
    const double *f;       // [P][S][n] (double), or float when f32
    const void *dQ;        // [P][S][S][n] upstream gradient (same element type)
    int f32;
    const double2 *F;      // [P][S][n] forward transforms of f
    double2 *Gg;           // [E][n] fft3(g)
    double2 *GF;           // [E][n] fft3(g . f_p)
    double2 *A, *B, *V;    // [E][RS][n]
    double *accp, *accq;   // [E][n] real accumulators of the T^H sums
    double2 *L, *Lw, *Y;   // [E][n]
    double *dots;          // [E][RS][nblk] partial Re<V, A B> (if domega)
    double *lossdots;      // [E][2][nblk] partial <g f_p, Re L>, <g f_p, Re Lw>
    const double2 *phase;  // [RS][2][3][N]
    const double2 *b;      // [RS][n]
    const double2 *c, *c_om;
    const double *w;       // [RS]
    double beta;
    void *df;              // [P][S][n] output (accumulated)
    int want_omega;
    const double2 *tw;
    double2 *X;            // X_INV, X_INV_RE: [E][n] spectrum
    double *xout;          // X_INV_RE: [E][n]
    double xscale;
    // G_FWD_REAL and L1 over several pairs: grid.z = pair slot k * Ec + e, the
    // slot's pair (pk[k], qk[k]) and tables; every [E][n] buffer is indexed by grid.z
    int Ec;
    int pk[kAdjMaxPairs], qk[kAdjMaxPairs];
    const double2 *ck[kAdjMaxPairs], *comk[kAdjMaxPairs];
};

__device__ __forceinline__ double load_real(const void *base, int f32, long i)
{
    return f32 ? (double)reinterpret_cast<const float *>(base)[i] : reinterpret_cast<const double *>(base)[i];
}

// block reduction of one double per thread; thread 0 returns the sum
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

template <int N, int AXIS, int MODE>
__global__ void __launch_bounds__(64) k_adj(AdjArgs a)
{
    __shared__ double2 tw[N];
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = a.tw[i];
    extern __shared__ double acc_s[];  // J5: [2][N][blockDim]
    __syncthreads();
    const int pi = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = pi < N * N;
    const long n = a.n;
    double2 v[N];

    if constexpr (MODE == G_FWD_REAL) {
        // grid.y: 0 -> g, 1 -> g . f_p ; grid.z = (pair slot, eval)
        const int k = blockIdx.z / a.Ec, e = blockIdx.z % a.Ec, pt = a.pt0 + e;
        if (!act) return;
        const long qb = (((long)pt * a.S + a.pk[k]) * a.S + a.qk[k]) * n;
        const long fb = ((long)pt * a.S + a.pk[k]) * n;
        double2 *X = (blockIdx.y == 0 ? a.Gg : a.GF) + (long)blockIdx.z * n;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const long o = poff<N, AXIS>(pi, j);
            double gv = load_real(a.dQ, a.f32, qb + o);
            if (blockIdx.y == 1) gv *= load_real(a.f, a.f32, fb + o);
            v[j] = make_double2(gv, 0.0);
        }
        fft<N, -1>(v, tw);
#pragma unroll
        for (int k = 0; k < N; ++k) X[poff<N, AXIS>(pi, k)] = v[k];
    } else if constexpr (MODE == G_FWD) {
        if (!act) return;
        double2 *X = (blockIdx.y == 0 ? a.Gg : a.GF) + (long)blockIdx.z * n;
#pragma unroll
        for (int j = 0; j < N; ++j) v[j] = X[poff<N, AXIS>(pi, j)];
        fft<N, -1>(v, tw);
#pragma unroll
        for (int k = 0; k < N; ++k) X[poff<N, AXIS>(pi, k)] = v[k];
    } else if constexpr (MODE == J1 || MODE == J2) {
        if (!act) return;
        const int rs = blockIdx.y, e = blockIdx.z;
        const long gb = ((long)e * a.RS + rs) * n;
        const double2 *php = a.phase + ((long)rs * 6 + 0 + AXIS) * N;
        const double2 *phq = a.phase + ((long)rs * 6 + 3 + AXIS) * N;
        const double2 *sa = a.A + gb, *sb = a.B + gb, *sv = a.V + gb;
        if constexpr (MODE == J1) {
            const int pt = a.pt0 + e;
            sa = a.F + ((long)pt * a.S + a.p) * n;
            sb = a.F + ((long)pt * a.S + a.q) * n;
            sv = a.Gg + (long)e * n;
        }
#pragma unroll
        for (int j = 0; j < N; ++j) v[j] = cmul(sa[poff<N, AXIS>(pi, j)], php[j]);
        fft<N, +1>(v, tw);
#pragma unroll
        for (int k = 0; k < N; ++k) a.A[gb + poff<N, AXIS>(pi, k)] = v[k];
#pragma unroll
        for (int j = 0; j < N; ++j) v[j] = cmul(sb[poff<N, AXIS>(pi, j)], phq[j]);
        fft<N, +1>(v, tw);
#pragma unroll
        for (int k = 0; k < N; ++k) a.B[gb + poff<N, AXIS>(pi, k)] = v[k];
        if constexpr (MODE == J1) {
            const double2 *brs = a.b + (long)rs * n;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const long o = poff<N, AXIS>(pi, j);
                v[j] = cmulc(sv[o], brs[o]);  // G . conj(b)
            }
        } else {
#pragma unroll
            for (int j = 0; j < N; ++j) v[j] = sv[poff<N, AXIS>(pi, j)];
        }
        fft<N, +1>(v, tw);
#pragma unroll
        for (int k = 0; k < N; ++k) a.V[gb + poff<N, AXIS>(pi, k)] = v[k];
    } else if constexpr (MODE == J3) {
        const int rs = blockIdx.y, e = blockIdx.z;
        const long gb = ((long)e * a.RS + rs) * n;
        const double2 *php = a.phase + ((long)rs * 6 + 0 + AXIS) * N;
        const double2 *phq = a.phase + ((long)rs * 6 + 3 + AXIS) * N;
        double dot = 0.0;
        if (act) {
            double2 va[N], vb[N];
#pragma unroll
            for (int j = 0; j < N; ++j) va[j] = cmul(a.A[gb + poff<N, AXIS>(pi, j)], php[j]);
            fft<N, +1>(va, tw);
#pragma unroll
            for (int j = 0; j < N; ++j) vb[j] = cmul(a.B[gb + poff<N, AXIS>(pi, j)], phq[j]);
            fft<N, +1>(vb, tw);
#pragma unroll
            for (int j = 0; j < N; ++j) v[j] = a.V[gb + poff<N, AXIS>(pi, j)];
            fft<N, +1>(v, tw);
            // physical space: dot, U_p = conj(B) V, U_q = conj(A) V
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const double2 ab = cmul(va[j], vb[j]);
                dot += v[j].x * ab.x + v[j].y * ab.y;  // Re(conj(V) A B)
                const double2 up = cmul(conjd(vb[j]), v[j]);
                const double2 uq = cmul(conjd(va[j]), v[j]);
                va[j] = up;
                vb[j] = uq;
            }
            // z factor of T^H: ifft_z(conj(phi_z) fft_z(U))
            fft<N, -1>(va, tw);
            fft<N, -1>(vb, tw);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                va[j] = cmulc(va[j], php[j]);
                vb[j] = cmulc(vb[j], phq[j]);
            }
            fft<N, +1>(va, tw);
            fft<N, +1>(vb, tw);
#pragma unroll
            for (int k = 0; k < N; ++k) {
                a.A[gb + poff<N, AXIS>(pi, k)] = va[k];
                a.B[gb + poff<N, AXIS>(pi, k)] = vb[k];
            }
        }
        if (a.want_omega) {
            const double s = block_sum(dot);
            if (threadIdx.x == 0) a.dots[((long)e * a.RS + rs) * gridDim.x + blockIdx.x] = s;
        }
    } else if constexpr (MODE == J4) {
        if (!act) return;
        const int rs = blockIdx.y, e = blockIdx.z;
        const long gb = ((long)e * a.RS + rs) * n;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            double2 *X = side == 0 ? a.A : a.B;
            const double2 *ph = a.phase + ((long)rs * 6 + side * 3 + AXIS) * N;
#pragma unroll
            for (int j = 0; j < N; ++j) v[j] = X[gb + poff<N, AXIS>(pi, j)];
            fft<N, -1>(v, tw);
#pragma unroll
            for (int j = 0; j < N; ++j) v[j] = cmulc(v[j], ph[j]);
            fft<N, +1>(v, tw);
#pragma unroll
            for (int k = 0; k < N; ++k) X[gb + poff<N, AXIS>(pi, k)] = v[k];
        }
    } else if constexpr (MODE == J5) {
        const int e = blockIdx.z;
        const int T = blockDim.x, t = threadIdx.x;
        if (!act) return;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            acc_s[(0 * N + k) * T + t] = 0.0;
            acc_s[(1 * N + k) * T + t] = 0.0;
        }
        for (int rs = 0; rs < a.RS; ++rs) {
            const long gb = ((long)e * a.RS + rs) * n;
            const double wr = a.w[rs];
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const double2 *X = side == 0 ? a.A : a.B;
                const double2 *ph = a.phase + ((long)rs * 6 + side * 3 + AXIS) * N;
#pragma unroll
                for (int j = 0; j < N; ++j) v[j] = X[gb + poff<N, AXIS>(pi, j)];
                fft<N, -1>(v, tw);
#pragma unroll
                for (int j = 0; j < N; ++j) v[j] = cmulc(v[j], ph[j]);
                fft<N, +1>(v, tw);
#pragma unroll
                for (int k = 0; k < N; ++k) acc_s[(side * N + k) * T + t] += wr * v[k].x;
            }
        }
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const long o = (long)e * n + poff<N, AXIS>(pi, k);
            a.accp[o] = acc_s[(0 * N + k) * T + t];
            a.accq[o] = acc_s[(1 * N + k) * T + t];
        }
    } else if constexpr (MODE == X_INV || MODE == X_INV_RE) {
        if (!act) return;
        double2 *X = a.X + (long)blockIdx.z * n;
#pragma unroll
        for (int j = 0; j < N; ++j) v[j] = X[poff<N, AXIS>(pi, j)];
        fft<N, +1>(v, tw);
        if constexpr (MODE == X_INV) {
#pragma unroll
            for (int k = 0; k < N; ++k) X[poff<N, AXIS>(pi, k)] = v[k];
        } else {
            double *o = a.xout + (long)blockIdx.z * n;
#pragma unroll
            for (int k = 0; k < N; ++k) o[poff<N, AXIS>(pi, k)] = a.xscale * v[k].x;
        }
    } else if constexpr (MODE == L1 || MODE == L2) {
        if (!act) return;
        const int e = blockIdx.z, k = blockIdx.z / a.Ec;
        double2 *dst[3] = {a.L + (long)e * n, a.Lw + (long)e * n, a.Y + (long)e * n};
        const double2 *Fq = a.F + ((long)(a.pt0 + e % a.Ec) * a.S + a.qk[k]) * n;
        const double2 *Gf = a.GF + (long)e * n;
        const double2 *cc = a.ck[k], *cw = a.comk[k];
#pragma unroll
        for (int which = 0; which < 3; ++which) {
            if (which == 1 && !a.want_omega) continue;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const long o = poff<N, AXIS>(pi, j);
                if constexpr (MODE == L1) {
                    v[j] = which == 0 ? cmul(cc[o], Fq[o]) : which == 1 ? cmul(cw[o], Fq[o]) : cmulc(Gf[o], cc[o]);
                } else {
                    v[j] = dst[which][o];
                }
            }
            fft<N, +1>(v, tw);
#pragma unroll
            for (int k = 0; k < N; ++k) dst[which][poff<N, AXIS>(pi, k)] = v[k];
        }
    } else if constexpr (MODE == L3) {
        const int e = blockIdx.z, pt = a.pt0 + e;
        const double inv_n = 1.0 / (double)n;
        const double inv_n3 = inv_n * inv_n * inv_n;
        double ld0 = 0.0, ld1 = 0.0;
        if (act) {
            double2 vl[N], vy[N];
#pragma unroll
            for (int j = 0; j < N; ++j) vl[j] = a.L[(long)e * n + poff<N, AXIS>(pi, j)];
            fft<N, +1>(vl, tw);
#pragma unroll
            for (int j = 0; j < N; ++j) vy[j] = a.Y[(long)e * n + poff<N, AXIS>(pi, j)];
            fft<N, +1>(vy, tw);
            if (a.want_omega) {
#pragma unroll
                for (int j = 0; j < N; ++j) v[j] = a.Lw[(long)e * n + poff<N, AXIS>(pi, j)];
                fft<N, +1>(v, tw);
            }
            const long qb = (((long)pt * a.S + a.p) * a.S + a.q) * n;
            const long fbp = ((long)pt * a.S + a.p) * n, fbq = ((long)pt * a.S + a.q) * n;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const long o = poff<N, AXIS>(pi, k);
                const double g = load_real(a.dQ, a.f32, qb + o);
                const double fp = load_real(a.f, a.f32, fbp + o);
                const double gp = a.beta * (inv_n3 * a.accp[(long)e * n + o] - g * vl[k].x * inv_n);
                const double gq = a.beta * (inv_n3 * a.accq[(long)e * n + o] - vy[k].x * inv_n);
                if (a.f32) {
                    float *df = reinterpret_cast<float *>(a.df);
                    df[fbp + o] += (float)gp;
                    df[fbq + o] += (float)gq;
                } else {
                    double *df = reinterpret_cast<double *>(a.df);
                    df[fbp + o] += gp;
                    df[fbq + o] += gq;
                }
                ld0 += g * fp * vl[k].x * inv_n;
                if (a.want_omega) ld1 += g * fp * v[k].x * inv_n;
            }
        }
        if (a.want_omega) {
            const double s0 = block_sum(ld0);
            const double s1 = block_sum(ld1);
            if (threadIdx.x == 0) {
                a.lossdots[((long)e * 2 + 0) * gridDim.x + blockIdx.x] = s0;
                a.lossdots[((long)e * 2 + 1) * gridDim.x + blockIdx.x] = s1;
            }
        }
    }
}

// domega[pair] = sum over points of dlnbeta <g,Q> + beta (sum_rs (wlog/w) dot_rs - <g f_p, Re S_w f_q>)
// with <g,Q> = beta (sum_rs dot_rs - <g f_p, Re S f_q>) and dot_rs = w_rs dscale Re<V_u, A_u B_u>
// (V_u, A_u, B_u as the caller's passes leave them; dscale undoes their scale).
__global__ void __launch_bounds__(256) k_omega_reduce(double *domega, int pair, const double *dots, int dblk,
                                                      double dscale, const double *lossdots, int E, int RS, int nblk,
                                                      const double *w, const double *wlog, double beta, double dlnbeta,
                                                      int accumulate)
{
    // the sum is linear in every dot: each thread takes a share of the terms
    // with its weight, then one block reduction
    double v = 0.0;
    const long nd = dots ? (long)E * RS * dblk : 0;  // null: no gain terms in this call
    for (long i = threadIdx.x; i < nd; i += blockDim.x) {
        const int rs = (int)((i / dblk) % RS);
        v += (dlnbeta * beta * w[rs] + beta * wlog[rs]) * dscale * dots[i];
    }
    for (long i = threadIdx.x; lossdots && i < (long)E * nblk; i += blockDim.x) {
        const long e = i / nblk, b = i % nblk;
        v -= dlnbeta * beta * lossdots[(e * 2 + 0) * nblk + b] + beta * lossdots[(e * 2 + 1) * nblk + b];
    }
    const double total = block_sum(v);
    if (threadIdx.x == 0) domega[pair] = accumulate ? domega[pair] + total : total;
}

constexpr int kAdjThreads = 64;
template <int N> constexpr int adj64_nblk_n() { return (N * N + kAdjThreads - 1) / kAdjThreads; }

template <int N, int AXIS, int MODE>
dgfs_status alaunch(dgfs_plan_s *plan, dim3 grid, const AdjArgs &a, cudaStream_t st)
{
    static const char *names[] = {"adj_g_fwd_real", "adj_g_fwd", "adj_j1", "adj_j2",  "adj_j3",   "adj_j4",
                                  "adj_j5",         "adj_l1",    "adj_l2", "adj_l3",  "adj_x_inv", "adj_x_inv"};
    grid.x = (N * N + kAdjThreads - 1) / kAdjThreads;
    const size_t smem = MODE == J5 ? sizeof(double) * 2 * N * kAdjThreads : 0;
    if (smem > 0)
        DGFS_CUDA(cudaFuncSetAttribute(k_adj<N, AXIS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    {
        ProfScope ps(plan, names[MODE], st);
        k_adj<N, AXIS, MODE><<<grid, kAdjThreads, smem, st>>>(a);
    }
    DGFS_LAUNCHED(plan);
    return DGFS_OK;
}

template <int N>
dgfs_status backward_n(dgfs_plan_s *plan, int P, const void *f, const void *dQ, void *df, double *domega,
                       int domega_on_host, cudaStream_t st)
{
    const int S = plan->S, RS = plan->Nrho * plan->M;
    const long n = (long)N * N * N;
    const int nblk = (N * N + kAdjThreads - 1) / kAdjThreads;
    const size_t es = elem_size(plan);
    // workspace: F [maxP][S][n] | A, B, V [E][RS][n] | Gg, GF, L, Lw, Y [E][n] (complex)
    //            | accp, accq [E][n] | dots [E][RS][nblk] | lossdots [E][2][nblk] | dom [S*S]
    const long per_eval = (3L * RS + 5) * n * 16 + 2L * n * 8 + ((long)RS * nblk + 2L * nblk) * 8;
    const long fixed = (long)plan->max_points * S * n * 16 + (long)S * S * 8;
    int E = (int)std::max(1L, std::min((long)P, ((long)plan->ws_bytes - fixed) / per_eval));
    void *ws = plan->ws;
    size_t need = fixed + (size_t)E * per_eval;
    void *own = nullptr;
    if (need > plan->ws_bytes || E < 1) {
        // the adjoint needs more than the forward's workspace: allocate for this call
        E = 1;
        need = fixed + per_eval;
        DGFS_CUDA(dev_malloc_async(&own, need, st));
        ws = own;
    }
    char *base = reinterpret_cast<char *>(ws);
    double2 *F = reinterpret_cast<double2 *>(base);
    double2 *A = F + (long)plan->max_points * S * n;
    double2 *B = A + (long)E * RS * n;
    double2 *V = B + (long)E * RS * n;
    double2 *Gg = V + (long)E * RS * n;
    double2 *GF = Gg + (long)E * n;
    double2 *L = GF + (long)E * n;
    double2 *Lw = L + (long)E * n;
    double2 *Y = Lw + (long)E * n;
    double *accp = reinterpret_cast<double *>(Y + (long)E * n);
    double *accq = accp + (long)E * n;
    double *dots = accq + (long)E * n;
    double *lossdots = dots + (long)E * RS * nblk;
    double *dom = lossdots + (long)E * 2 * nblk;

    DGFS_CUDA(cudaMemsetAsync(df, 0, es * (size_t)P * S * n, st));
    DGFS_TRY(fp64_forward(plan, P, f, F, st));

    AdjArgs a{};
    a.n = n;
    a.S = S;
    a.RS = RS;
    a.f = reinterpret_cast<const double *>(f);
    a.dQ = dQ;
    a.f32 = plan->prec == DGFS_FP64 ? 0 : 1;
    a.F = F;
    a.Gg = Gg;
    a.GF = GF;
    a.A = A;
    a.B = B;
    a.V = V;
    a.accp = accp;
    a.accq = accq;
    a.L = L;
    a.Lw = Lw;
    a.Y = Y;
    a.dots = dots;
    a.lossdots = lossdots;
    a.df = df;
    a.want_omega = domega ? 1 : 0;
    a.tw = plan->twiddle;
    for (int p = 0; p < S; ++p)
        for (int q = 0; q < S; ++q) {
            const PairTables &pt = plan->pairs[p * S + q];
            a.p = p;
            a.q = q;
            a.phase = pt.phase;
            a.b = pt.b;
            a.c = pt.c;
            a.c_om = pt.c_om;
            a.w = pt.w;
            a.beta = pt.beta;
            a.pk[0] = p;
            a.qk[0] = q;
            a.ck[0] = pt.c;
            a.comk[0] = pt.c_om;
            for (int pt0 = 0; pt0 < P; pt0 += E) {
                const int Ec = std::min(E, P - pt0);
                a.pt0 = pt0;
                a.Ec = Ec;
                DGFS_TRY((alaunch<N, 0, G_FWD_REAL>(plan, dim3(1, 2, Ec), a, st)));
                DGFS_TRY((alaunch<N, 1, G_FWD>(plan, dim3(1, 2, Ec), a, st)));
                DGFS_TRY((alaunch<N, 2, G_FWD>(plan, dim3(1, 2, Ec), a, st)));
                DGFS_TRY((alaunch<N, 0, J1>(plan, dim3(1, RS, Ec), a, st)));
                DGFS_TRY((alaunch<N, 1, J2>(plan, dim3(1, RS, Ec), a, st)));
                DGFS_TRY((alaunch<N, 2, J3>(plan, dim3(1, RS, Ec), a, st)));
                DGFS_TRY((alaunch<N, 1, J4>(plan, dim3(1, RS, Ec), a, st)));
                DGFS_TRY((alaunch<N, 0, J5>(plan, dim3(1, 1, Ec), a, st)));
                DGFS_TRY((alaunch<N, 0, L1>(plan, dim3(1, 1, Ec), a, st)));
                DGFS_TRY((alaunch<N, 1, L2>(plan, dim3(1, 1, Ec), a, st)));
                DGFS_TRY((alaunch<N, 2, L3>(plan, dim3(1, 1, Ec), a, st)));
                if (domega) {
                    k_omega_reduce<<<1, 256, 0, st>>>(dom, p * S + q, dots, nblk, 1.0 / ((double)n * n * n),
                                                     lossdots, Ec, RS, nblk, pt.w, pt.wlog, pt.beta, pt.dlogbeta,
                                                     pt0 > 0 ? 1 : 0);
                    DGFS_LAUNCHED(plan);
                }
            }
        }
    if (domega) {
        DGFS_CUDA(cudaMemcpyAsync(domega, dom, sizeof(double) * S * S,
                                  domega_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
        if (domega_on_host) DGFS_CUDA(cudaStreamSynchronize(st));
    }
    if (own) DGFS_CUDA(dev_free_async(own, st));
    return DGFS_OK;
}

template <int N>
dgfs_status part_n(dgfs_plan_s *plan, int which, const AdjPart &x, cudaStream_t st)
{
    AdjArgs a{};
    a.n = (long)N * N * N;
    a.S = plan->S;
    a.RS = plan->Nrho * plan->M;
    a.pt0 = x.pt0;
    a.Ec = x.Ec;
    a.f = reinterpret_cast<const double *>(x.f);
    a.dQ = x.dQ;
    a.f32 = x.f32;
    a.F = x.F;
    a.df = x.df;
    a.want_omega = x.want_omega;
    a.tw = plan->twiddle;
    a.X = x.X;
    a.xout = x.xout;
    a.xscale = x.xscale;
    if (x.npairs < 1 || x.npairs > kAdjMaxPairs) {
        set_error("adjoint: bad pair count");
        return DGFS_EINVAL;
    }
    for (int k = 0; k < x.npairs; ++k) {
        const PairTables &pt = plan->pairs[x.pairs[k]];
        a.pk[k] = x.pairs[k] / plan->S;
        a.qk[k] = x.pairs[k] % plan->S;
        a.ck[k] = pt.c;
        a.comk[k] = pt.c_om;
    }
    const unsigned slots = (unsigned)(x.npairs * x.Ec);
    const long en = (long)x.Ec * a.n;  // one pair slot of an [E][n] buffer
    switch (which) {
    case ADJ_PART_G:
        a.Gg = x.Gg;
        a.GF = x.GF;
        DGFS_TRY((alaunch<N, 0, G_FWD_REAL>(plan, dim3(1, 2, slots), a, st)));
        DGFS_TRY((alaunch<N, 1, G_FWD>(plan, dim3(1, 2, slots), a, st)));
        return alaunch<N, 2, G_FWD>(plan, dim3(1, 2, slots), a, st);
    case ADJ_PART_INV:
        // x.Ec grids in X, no pairs involved
        DGFS_TRY((alaunch<N, 0, X_INV>(plan, dim3(1, 1, x.Ec), a, st)));
        DGFS_TRY((alaunch<N, 1, X_INV>(plan, dim3(1, 1, x.Ec), a, st)));
        return alaunch<N, 2, X_INV_RE>(plan, dim3(1, 1, x.Ec), a, st);
    case ADJ_PART_LOSS:
        a.GF = x.GF;
        a.L = x.L;
        a.Lw = x.Lw;
        a.Y = x.Y;
        DGFS_TRY((alaunch<N, 0, L1>(plan, dim3(1, 1, slots), a, st)));
        DGFS_TRY((alaunch<N, 1, L2>(plan, dim3(1, 1, slots), a, st)));
        // the combine adds into df[p] and df[q]: one pair per launch
        for (int k = 0; k < x.npairs; ++k) {
            const PairTables &pt = plan->pairs[x.pairs[k]];
            AdjArgs b = a;
            b.p = a.pk[k];
            b.q = a.qk[k];
            b.beta = pt.beta;
            b.L = x.L + k * en;
            b.Lw = x.Lw + k * en;
            b.Y = x.Y + k * en;
            b.accp = x.accp + 2 * k * en;
            b.accq = x.accp + (2 * k + 1) * en;
            b.lossdots = x.lossdots + (long)k * x.Ec * 2 * adj64_nblk_n<N>();
            DGFS_TRY((alaunch<N, 2, L3>(plan, dim3(1, 1, x.Ec), b, st)));
        }
        return DGFS_OK;
    default: set_error("adjoint: unknown part"); return DGFS_EINVAL;
    }
}

}  // namespace

int adj64_nblk(int N) { return (N * N + kAdjThreads - 1) / kAdjThreads; }

dgfs_status adj64_part(dgfs_plan_s *plan, int which, const AdjPart &x, cudaStream_t st)
{
    switch (plan->N) {
    case 8: return part_n<8>(plan, which, x, st);
    case 16: return part_n<16>(plan, which, x, st);
    case 24: return part_n<24>(plan, which, x, st);
    case 32: return part_n<32>(plan, which, x, st);
    case 48: return part_n<48>(plan, which, x, st);
    default: set_error("N not supported by the adjoint's FP64 parts"); return DGFS_EUNSUPPORTED;
    }
}

dgfs_status adj64_omega_gain(dgfs_plan_s *plan, double *dom, int p, int q, const double *dots, double dscale, int Ec,
                             int accumulate, cudaStream_t st)
{
    const PairTables &pt = plan->pairs[p * plan->S + q];
    k_omega_reduce<<<1, 256, 0, st>>>(dom, p * plan->S + q, dots, 1, dscale, nullptr, Ec, plan->Nrho * plan->M,
                                      adj64_nblk(plan->N), pt.w, pt.wlog, pt.beta, pt.dlogbeta, accumulate);
    DGFS_LAUNCHED(plan);
    return DGFS_OK;
}

dgfs_status adj64_omega_loss(dgfs_plan_s *plan, double *dom, int p, int q, const double *lossdots, int Ec,
                             cudaStream_t st)
{
    const PairTables &pt = plan->pairs[p * plan->S + q];
    k_omega_reduce<<<1, 256, 0, st>>>(dom, p * plan->S + q, nullptr, 1, 0.0, lossdots, Ec, plan->Nrho * plan->M,
                                      adj64_nblk(plan->N), pt.w, pt.wlog, pt.beta, pt.dlogbeta, 1);
    DGFS_LAUNCHED(plan);
    return DGFS_OK;
}

dgfs_status fp64_backward(dgfs_plan_s *plan, int P, const void *f, const void *dQ, void *df, double *domega,
                          int domega_on_host, cudaStream_t st)
{
    switch (plan->N) {
    case 4: return backward_n<4>(plan, P, f, dQ, df, domega, domega_on_host, st);
    case 6: return backward_n<6>(plan, P, f, dQ, df, domega, domega_on_host, st);
    case 8: return backward_n<8>(plan, P, f, dQ, df, domega, domega_on_host, st);
    case 12: return backward_n<12>(plan, P, f, dQ, df, domega, domega_on_host, st);
    case 16: return backward_n<16>(plan, P, f, dQ, df, domega, domega_on_host, st);
    case 24: return backward_n<24>(plan, P, f, dQ, df, domega, domega_on_host, st);
    case 32: return backward_n<32>(plan, P, f, dQ, df, domega, domega_on_host, st);
    case 48: return backward_n<48>(plan, P, f, dQ, df, domega, domega_on_host, st);
    default: set_error("N not supported by the FP64 adjoint"); return DGFS_EUNSUPPORTED;
    }
}

}  // namespace dgfs

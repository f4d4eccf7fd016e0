// Double-float passes around the tensor-core stages (Algorithm 2, steps 1
// and 10) for the FP32-class forms:
//   - forward transforms F = fft3(f) of every (point, species) (step 1),
//     needed by the loss term only (the gain stages transform f themselves);
//   - the finish of every species pair at once (step 10):
//     Q = beta/n Re( ifft3_u(QG) - f_p ifft3_u(c F_q) ).
// Both real parts come from one complex inverse transform of
// Z = Herm(QG) + i Herm(c F_q), Herm X(k) = (X(k) + conj X(-k)) / 2, because
// Re ifft3(X) = ifft3(Herm X).
//
// The gain and the loss term of step 10 nearly cancel: their magnitudes are
// 10 to 200 times that of Q on the benchmark workloads, so these transforms
// need more than FP32.  They run in double-float arithmetic (dfloat.cuh) on
// the FP32 pipes, about 48 significant bits, instead of FP64, whose rate on
// this GPU is a small fraction of FP32's.  One thread per pencil, the pencil
// in registers (the register FFT of fftreg.cuh on double-float complex
// values), one kernel per axis; complex double-floats are stored as float4.
#include "dgfs_internal.h"
#include "fftreg.cuh"
#include "dfloat.cuh"

namespace dgfs {
namespace {

enum ModeDf {
    D_FWD_REAL = 0,  // F = fft_axis(real f)    grid.y = species, grid.z = point
    D_FWD,           // F = fft_axis(F)         grid.y = species, grid.z = point
    D_INV,           // G = ifft_axis(G)        grid.y = pair p S + q, grid.z = point
    D_LAST,          // Q = beta/n (Re ifft(G) - f_p Im ifft(G))
    D_TOREAL         // out = Re ifft_axis(G) / n as float   grid.y = 1, grid.z = grid
};

struct PassDf {
    long n, pair_stride;  // pair_stride in complex elements
    int S;
    const float *f;     // [P][S][n]
    float4 *F;          // [P][S][n]
    float4 *G;          // pair p S + q at G + (p S + q) pair_stride, [P][n] each
    float *Q;           // [P][S][S][n]
    float *out;         // D_TOREAL: real grids, n apart
    dfl inv_n;          // D_TOREAL: 1 / n
    const float4 *tw;   // [N] exp(-2 pi i j / N)
    dfl scale[16];      // beta_pq / n per pair
};

template <int N, int AXIS>
__device__ __forceinline__ long off(int pi, int j)
{
    if constexpr (AXIS == 0) return (long)j * N * N + pi;
    else if constexpr (AXIS == 1) return (long)(pi / N) * N * N + (long)j * N + (pi % N);
    else return (long)pi * N + j;
}

template <int N, int AXIS, int MODE>
__global__ void __launch_bounds__(128) k_pass_df(PassDf a)
{
    __shared__ dcx tw[N];
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = ld_dcx(a.tw + i);
    __syncthreads();
    const int pi = blockIdx.x * blockDim.x + threadIdx.x;
    if (pi >= N * N) return;
    const long n = a.n;
    const dfl zero(0.f, 0.f);
    dcx v[N];
    if constexpr (MODE == D_FWD_REAL || MODE == D_FWD) {
        const long base = ((long)blockIdx.z * a.S + blockIdx.y) * n;
        float4 *F = a.F + base;
        if constexpr (MODE == D_FWD_REAL) {
            const float *fr = a.f + base;
#pragma unroll
            for (int j = 0; j < N; ++j) v[j] = dcx{dfl(fr[off<N, AXIS>(pi, j)], 0.f), zero};
        } else {
#pragma unroll
            for (int j = 0; j < N; ++j) v[j] = ld_dcx(F + off<N, AXIS>(pi, j));
        }
        reg::fft<N, -1>(v, tw);
#pragma unroll
        for (int k = 0; k < N; ++k) st_dcx(F + off<N, AXIS>(pi, k), v[k]);
    } else {
        const int pr = blockIdx.y, e = blockIdx.z;
        float4 *g = a.G + (long)pr * a.pair_stride + (long)e * n;
#pragma unroll
        for (int j = 0; j < N; ++j) v[j] = ld_dcx(g + off<N, AXIS>(pi, j));
        reg::fft<N, +1>(v, tw);
        if constexpr (MODE == D_INV) {
#pragma unroll
            for (int k = 0; k < N; ++k) st_dcx(g + off<N, AXIS>(pi, k), v[k]);
        } else if constexpr (MODE == D_TOREAL) {
            float *o = a.out + (long)e * n;
#pragma unroll
            for (int k = 0; k < N; ++k) o[off<N, AXIS>(pi, k)] = to_float(v[k].x * a.inv_n);
        } else {
            // ifft3_u(Z) = Re ifft3_u(QG) + i Re ifft3_u(c F_q)
            const int p = pr / a.S, q = pr % a.S;
            const float *fp = a.f + ((long)e * a.S + p) * n;
            float *Q = a.Q + (((long)e * a.S + p) * a.S + q) * n;
            const dfl sc = a.scale[pr];
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const long o = off<N, AXIS>(pi, k);
                Q[o] = to_float(sc * (v[k].x - dfl(fp[o], 0.f) * v[k].y));
            }
        }
    }
}

__device__ __forceinline__ dfl halve(dfl d) { return dfl(0.5f * d.hi, 0.5f * d.lo); }

struct PairCDf {
    const float4 *c[16];
};

// Z = Herm(QG) + i Herm(c F_q) in place for every pair and point: the thread of
// the smaller index of {k, -k mod N} forms Z(k) and Z(-k), using
// Herm X(-k) = conj Herm X(k).
__global__ void k_herm_df(float4 *G, long pair_stride, const float4 *F, PairCDf cs, int N, long n, int S, int P)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;  // over [S*S][P][n]
    if (i >= (long)S * S * P * n) return;
    const long k = i % n, pe = i / n;
    const int e = (int)(pe % P), pr = (int)(pe / P);
    const int kx = (int)(k / ((long)N * N)), ky = (int)((k / N) % N), kz = (int)(k % N);
    const long mk = ((long)((N - kx) % N) * N + (N - ky) % N) * N + (N - kz) % N;
    if (mk < k) return;
    float4 *g = G + (long)pr * pair_stride + (long)e * n;
    const float4 *Fq = F + ((long)e * S + pr % S) * n;
    const float4 *c = cs.c[pr];
    const dcx a0 = ld_dcx(g + k), a1 = ld_dcx(g + mk);
    const dcx l0 = reg::cmul(ld_dcx(c + k), ld_dcx(Fq + k)), l1 = reg::cmul(ld_dcx(c + mk), ld_dcx(Fq + mk));
    const dfl h1x = halve(a0.x + a1.x), h1y = halve(a0.y - a1.y);
    const dfl h2x = halve(l0.x + l1.x), h2y = halve(l0.y - l1.y);
    st_dcx(g + k, dcx{h1x - h2y, h1y + h2x});
    if (mk != k) st_dcx(g + mk, dcx{h1x + h2y, h2x - h1y});
}

// Hermitian form (declared variant): zero every mode with an index on a
// Nyquist plane (index N / 2 along any axis) of `grids` spectra of n points
__global__ void k_project_df(float4 *F, long grids, int N, long n)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= grids * n) return;
    const long k = i % n;
    const int kx = (int)(k / ((long)N * N)), ky = (int)((k / N) % N), kz = (int)(k % N);
    if (kx == N / 2 || ky == N / 2 || kz == N / 2) F[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Hermitian finish, first step, for every pair and packed slot e (points 2e
// and 2e + 1): Z1 = P QG in place (the gain's Nyquist planes removed) and
// Z2 = c (F~_q(2e) + i F~_q(2e + 1)) (the loss spectra of both points)
__global__ void k_herm_pack_df(float4 *G, long pair_stride, float4 *Z2, long z2_stride, const float4 *F,
                               PairCDf cs, int N, long n, int S, int P, int Ps)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;  // over [S*S][Ps][n]
    if (i >= (long)S * S * Ps * n) return;
    const long k = i % n, pe = i / n;
    const int e = (int)(pe % Ps), pr = (int)(pe / Ps), q = pr % S;
    const int kx = (int)(k / ((long)N * N)), ky = (int)((k / N) % N), kz = (int)(k % N);
    float4 *g = G + (long)pr * pair_stride + (long)e * n + k;
    if (kx == N / 2 || ky == N / 2 || kz == N / 2) *g = make_float4(0.f, 0.f, 0.f, 0.f);
    const dfl zero(0.f, 0.f);
    const dcx a = ld_dcx(F + ((long)(2 * e) * S + q) * n + k);
    const dcx b = 2 * e + 1 < P ? ld_dcx(F + ((long)(2 * e + 1) * S + q) * n + k) : dcx{zero, zero};
    const dcx packed{a.x - b.y, a.y + b.x};
    st_dcx(Z2 + (long)pr * z2_stride + (long)e * n + k, reg::cmul(ld_dcx(cs.c[pr] + k), packed));
}

struct PairScale {
    dfl sc[16];  // beta_pq / n
};

// Hermitian finish, last step: ifft3_u(Z1) = n (G(2e) + i G(2e+1)) and
// ifft3_u(Z2) = n (L(2e) + i L(2e+1)) separate into the two points:
// Q(point) = beta/n (n G - f~_p n L) for the real and the imaginary parts
__global__ void k_combine_pack_df(const float4 *G, long pair_stride, const float4 *Z2, long z2_stride, const float *ft,
                                  float *Q, PairScale ps, long n, int S, int P, int Ps)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)S * S * Ps * n) return;
    const long k = i % n, pe = i / n;
    const int e = (int)(pe % Ps), pr = (int)(pe / Ps), p = pr / S, q = pr % S;
    const dcx g = ld_dcx(G + (long)pr * pair_stride + (long)e * n + k);
    const dcx l = ld_dcx(Z2 + (long)pr * z2_stride + (long)e * n + k);
    const dfl sc = ps.sc[pr];
    const int i0 = 2 * e, i1 = 2 * e + 1;
    Q[(((long)i0 * S + p) * S + q) * n + k] = to_float(sc * (g.x - dfl(ft[((long)i0 * S + p) * n + k], 0.f) * l.x));
    if (i1 < P)
        Q[(((long)i1 * S + p) * S + q) * n + k] =
            to_float(sc * (g.y - dfl(ft[((long)i1 * S + p) * n + k], 0.f) * l.y));
}

constexpr int kT = 128;

template <int N, int AXIS, int MODE>
dgfs_status launch_df(dgfs_plan_s *plan, int gy, int gz, const PassDf &a, const char *name, cudaStream_t st)
{
    {
        ProfScope ps(plan, name, st);
        k_pass_df<N, AXIS, MODE><<<dim3((N * N + kT - 1) / kT, gy, gz), kT, 0, st>>>(a);
    }
    DGFS_LAUNCHED(plan);
    return DGFS_OK;
}

template <int N>
dgfs_status forward_df_n(dgfs_plan_s *plan, int P, const float *f, float4 *F, const float4 *tw, cudaStream_t st)
{
    PassDf a{};
    a.n = (long)N * N * N;
    a.S = plan->S;
    a.f = f;
    a.F = F;
    a.tw = tw;
    DGFS_TRY((launch_df<N, 0, D_FWD_REAL>(plan, plan->S, P, a, "df_fwd_real", st)));
    DGFS_TRY((launch_df<N, 1, D_FWD>(plan, plan->S, P, a, "df_fwd", st)));
    DGFS_TRY((launch_df<N, 2, D_FWD>(plan, plan->S, P, a, "df_fwd", st)));
    return DGFS_OK;
}

template <int N>
dgfs_status finish_df_n(dgfs_plan_s *plan, int P, float4 *G, long pair_stride, const float4 *F, const float *f,
                        float *Q, const float4 *tw, cudaStream_t st)
{
    const int S = plan->S;
    PassDf a{};
    a.n = (long)N * N * N;
    a.pair_stride = pair_stride;
    a.S = S;
    a.f = f;
    a.G = G;
    a.Q = Q;
    a.tw = tw;
    PairCDf cs{};
    for (int pr = 0; pr < S * S; ++pr) {
        cs.c[pr] = plan->pairs[pr].cdf;
        a.scale[pr] = dfl(plan->pairs[pr].beta / (double)a.n);
    }
    const long total = (long)S * S * P * a.n;
    {
        ProfScope ps(plan, "df_herm", st);
        k_herm_df<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(G, pair_stride, F, cs, N, a.n, S, P);
    }
    DGFS_LAUNCHED(plan);
    DGFS_TRY((launch_df<N, 0, D_INV>(plan, S * S, P, a, "df_inv", st)));
    DGFS_TRY((launch_df<N, 1, D_INV>(plan, S * S, P, a, "df_inv", st)));
    DGFS_TRY((launch_df<N, 2, D_LAST>(plan, S * S, P, a, "df_last", st)));
    return DGFS_OK;
}

// Hermitian form: project the spectra F [P][S][n] in place and write
// f~ = ifft3(P F) as float [P][S][n] to ft, through the scratch tmp (P S n float4)
template <int N>
dgfs_status herm_prepare_df_n(dgfs_plan_s *plan, int P, float4 *F, float4 *tmp, float *ft, const float4 *tw,
                              cudaStream_t st)
{
    const long n = (long)N * N * N, grids = (long)P * plan->S;
    {
        ProfScope ps(plan, "df_project", st);
        k_project_df<<<(unsigned)((grids * n + 255) / 256), 256, 0, st>>>(F, grids, N, n);
    }
    DGFS_LAUNCHED(plan);
    DGFS_CUDA(cudaMemcpyAsync(tmp, F, sizeof(float4) * grids * n, cudaMemcpyDeviceToDevice, st));
    PassDf a{};
    a.n = n;
    a.pair_stride = 0;
    a.S = plan->S;
    a.G = tmp;
    a.out = ft;
    a.inv_n = dfl(1.0 / (double)n);
    a.tw = tw;
    DGFS_TRY((launch_df<N, 0, D_INV>(plan, 1, (int)grids, a, "df_inv", st)));
    DGFS_TRY((launch_df<N, 1, D_INV>(plan, 1, (int)grids, a, "df_inv", st)));
    DGFS_TRY((launch_df<N, 2, D_TOREAL>(plan, 1, (int)grids, a, "df_toreal", st)));
    return DGFS_OK;
}

template <int N>
dgfs_status herm_finish_df_n(dgfs_plan_s *plan, int P, float4 *G, long pair_stride, float4 *Z2, long z2_stride,
                             const float4 *F, const float *ft, float *Q, const float4 *tw, cudaStream_t st)
{
    const int S = plan->S, Ps = (P + 1) / 2;
    const long n = (long)N * N * N;
    PairCDf cs{};
    PairScale psc{};
    for (int pr = 0; pr < S * S; ++pr) {
        cs.c[pr] = plan->pairs[pr].cdf;
        psc.sc[pr] = dfl(plan->pairs[pr].beta / (double)n);
    }
    const long total = (long)S * S * Ps * n;
    {
        ProfScope ps(plan, "df_herm_pack", st);
        k_herm_pack_df<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(G, pair_stride, Z2, z2_stride, F, cs, N, n,
                                                                          S, P, Ps);
    }
    DGFS_LAUNCHED(plan);
    PassDf a{};
    a.n = n;
    a.S = S;
    a.tw = tw;
    for (int which = 0; which < 2; ++which) {
        a.G = which == 0 ? G : Z2;
        a.pair_stride = which == 0 ? pair_stride : z2_stride;
        DGFS_TRY((launch_df<N, 0, D_INV>(plan, S * S, Ps, a, "df_inv", st)));
        DGFS_TRY((launch_df<N, 1, D_INV>(plan, S * S, Ps, a, "df_inv", st)));
        DGFS_TRY((launch_df<N, 2, D_INV>(plan, S * S, Ps, a, "df_inv", st)));
    }
    {
        ProfScope ps(plan, "df_combine", st);
        k_combine_pack_df<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(G, pair_stride, Z2, z2_stride, ft, Q, psc,
                                                                             n, S, P, Ps);
    }
    DGFS_LAUNCHED(plan);
    return DGFS_OK;
}

}  // namespace

dgfs_status df_herm_prepare(dgfs_plan_s *plan, int P, float4 *F, float4 *tmp, float *ft, const float4 *tw,
                            cudaStream_t st)
{
    switch (plan->N) {
    case 8: return herm_prepare_df_n<8>(plan, P, F, tmp, ft, tw, st);
    case 16: return herm_prepare_df_n<16>(plan, P, F, tmp, ft, tw, st);
    case 24: return herm_prepare_df_n<24>(plan, P, F, tmp, ft, tw, st);
    case 32: return herm_prepare_df_n<32>(plan, P, F, tmp, ft, tw, st);
    default: set_error("the Hermitian form of the tensor-core path supports N in {8, 16, 24, 32}");
        return DGFS_EUNSUPPORTED;
    }
}

dgfs_status df_herm_finish(dgfs_plan_s *plan, int P, float4 *G, long pair_stride, float4 *Z2, long z2_stride,
                           const float4 *F, const float *ft, float *Q, const float4 *tw, cudaStream_t st)
{
    switch (plan->N) {
    case 8: return herm_finish_df_n<8>(plan, P, G, pair_stride, Z2, z2_stride, F, ft, Q, tw, st);
    case 16: return herm_finish_df_n<16>(plan, P, G, pair_stride, Z2, z2_stride, F, ft, Q, tw, st);
    case 24: return herm_finish_df_n<24>(plan, P, G, pair_stride, Z2, z2_stride, F, ft, Q, tw, st);
    case 32: return herm_finish_df_n<32>(plan, P, G, pair_stride, Z2, z2_stride, F, ft, Q, tw, st);
    default: set_error("the Hermitian form of the tensor-core path supports N in {8, 16, 24, 32}");
        return DGFS_EUNSUPPORTED;
    }
}

// double -> double-float tables (plan creation)
__global__ void k_to_df(float4 *dst, const double2 *src, long count)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double2 v = src[i];
    const dfl x(v.x), y(v.y);
    dst[i] = make_float4(x.hi, x.lo, y.hi, y.lo);
}

dgfs_status df_forward(dgfs_plan_s *plan, int P, const float *f, float4 *F, const float4 *tw, cudaStream_t st)
{
    switch (plan->N) {
    case 8: return forward_df_n<8>(plan, P, f, F, tw, st);
    case 16: return forward_df_n<16>(plan, P, f, F, tw, st);
    case 24: return forward_df_n<24>(plan, P, f, F, tw, st);
    case 32: return forward_df_n<32>(plan, P, f, F, tw, st);
    case 48: return forward_df_n<48>(plan, P, f, F, tw, st);
    default: set_error("N not supported by the double-float passes"); return DGFS_EUNSUPPORTED;
    }
}

dgfs_status df_finish(dgfs_plan_s *plan, int P, float4 *G, long pair_stride, const float4 *F, const float *f,
                      float *Q, const float4 *tw, cudaStream_t st)
{
    switch (plan->N) {
    case 8: return finish_df_n<8>(plan, P, G, pair_stride, F, f, Q, tw, st);
    case 16: return finish_df_n<16>(plan, P, G, pair_stride, F, f, Q, tw, st);
    case 24: return finish_df_n<24>(plan, P, G, pair_stride, F, f, Q, tw, st);
    case 32: return finish_df_n<32>(plan, P, G, pair_stride, F, f, Q, tw, st);
    case 48: return finish_df_n<48>(plan, P, G, pair_stride, F, f, Q, tw, st);
    default: set_error("N not supported by the double-float passes"); return DGFS_EUNSUPPORTED;
    }
}

dgfs_status df_tables(dgfs_plan_s *plan, float4 **tw_out)
{
    const long n = (long)plan->N * plan->N * plan->N;
    for (auto &pt : plan->pairs) {
        DGFS_CUDA(dev_malloc(&pt.cdf, sizeof(float4) * n));
        plan->table_bytes += sizeof(float4) * n;
        k_to_df<<<(unsigned)((n + 255) / 256), 256>>>(pt.cdf, pt.c, n);
        DGFS_LAUNCHED(plan);
    }
    DGFS_CUDA(dev_malloc(tw_out, sizeof(float4) * plan->N));
    k_to_df<<<1, 64>>>(*tw_out, plan->twiddle, plan->N);
    DGFS_LAUNCHED(plan);
    return DGFS_OK;
}

}  // namespace dgfs

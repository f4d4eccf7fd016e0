// Dealiased collision operator (a declared variant; the paper's Algorithm 2
// is cyclic): the Galerkin sum of Eq. (7) over l + m = k without wrap-around,
// by the 3/2 rule.  A plan built at N' = 3N/2 evaluates Algorithm 2 on the
// spectral interpolants of the inputs; only the N original wavenumbers of the
// result are kept.
//
//   1. F = fft3_N(f); the planes carrying wavenumber -N/2 are zeroed (for even
//      N their partner +N/2 is not on the grid: only then is the interpolant
//      real), F is embedded at the same wavenumbers of the N' grid, zero
//      elsewhere, and f' = ifft3_N'(F) (real part);
//   2. Q' = Algorithm 2 on the N' grid (any precision form of the plan);
//   3. X = fft3_N'(Q') at the N original wavenumbers, -N/2 planes zeroed,
//      Q = Re ifft3_N(X).
// With N' >= 3N/2 no sum of two retained wavenumbers wraps onto a retained
// one, so step 3 yields the linear-convolution coefficients.
//
// The resampling runs in FP64: in-place pencil passes of the register FFT
// (one length-M pencil per thread) and elementwise embed / gather kernels.
#include <cmath>

#include "dgfs_internal.h"
#include "fftreg.cuh"

namespace dgfs {
namespace {

template <int M, int AXIS>
__device__ __forceinline__ long poff(int pi, int j)
{
    if constexpr (AXIS == 0) return (long)j * M * M + pi;
    else if constexpr (AXIS == 1) return (long)(pi / M) * M * M + (long)j * M + (pi % M);
    else return (long)pi * M + j;
}

// In-place transform of every length-M pencil along AXIS of `count` M^3 grids
// (SIGN -1 forward, +1 unnormalised inverse).
template <int M, int AXIS, int SIGN>
__global__ void __launch_bounds__(128) k_fft_axis(double2 *data)
{
    __shared__ double2 tw[M];
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        double s, c;
        sincospi(-2.0 * i / M, &s, &c);
        tw[i] = make_double2(c, s);
    }
    __syncthreads();
    const int pi = blockIdx.x * blockDim.x + threadIdx.x;
    if (pi >= M * M) return;
    double2 *g = data + (long)blockIdx.y * M * M * M;
    double2 v[M];
#pragma unroll
    for (int j = 0; j < M; ++j) v[j] = g[poff<M, AXIS>(pi, j)];
    reg::fft<M, SIGN>(v, tw);
#pragma unroll
    for (int k = 0; k < M; ++k) g[poff<M, AXIS>(pi, k)] = v[k];
}

template <typename T>
__global__ void k_to_complex(const T *x, double2 *y, long total)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) y[i] = make_double2((double)x[i], 0.0);
}

template <typename T>
__global__ void k_real_part(const double2 *x, T *y, long total, double scale)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) y[i] = (T)(x[i].x * scale);
}

__device__ __forceinline__ int wavenumber(int i, int M) { return 2 * i >= M ? i - M : i; }

// retained: every component strictly inside (-N/2, N/2)
__device__ __forceinline__ bool retained(int kx, int ky, int kz, int N)
{
    const int h = N / 2;
    return kx > -h && kx < h && ky > -h && ky < h && kz > -h && kz < h;
}

// G (Np^3 per grid) = F (N^3) at the same wavenumbers, scaled, zero elsewhere.
__global__ void k_embed(const double2 *F, double2 *G, int N, int Np, long count, double scale)
{
    const long np3 = (long)Np * Np * Np;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count * np3) return;
    const long gi = i / np3, k = i % np3;
    const int kx = wavenumber((int)(k / ((long)Np * Np)), Np), ky = wavenumber((int)((k / Np) % Np), Np),
              kz = wavenumber((int)(k % Np), Np);
    double2 v = make_double2(0.0, 0.0);
    if (retained(kx, ky, kz, N)) {
        const long src = (((long)((kx + N) % N) * N) + (ky + N) % N) * N + (kz + N) % N;
        const double2 u = F[gi * N * N * N + src];
        v = make_double2(u.x * scale, u.y * scale);
    }
    G[i] = v;
}

// Y (N^3 per grid) = X (Np^3) at the retained wavenumbers, scaled; zero on the
// -N/2 planes.
__global__ void k_gather(const double2 *X, double2 *Y, int N, int Np, long count, double scale)
{
    const long n3 = (long)N * N * N;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count * n3) return;
    const long gi = i / n3, k = i % n3;
    const int kx = wavenumber((int)(k / ((long)N * N)), N), ky = wavenumber((int)((k / N) % N), N),
              kz = wavenumber((int)(k % N), N);
    double2 v = make_double2(0.0, 0.0);
    if (retained(kx, ky, kz, N)) {
        const long src = (((long)((kx + Np) % Np) * Np) + (ky + Np) % Np) * Np + (kz + Np) % Np;
        const double2 u = X[gi * (long)Np * Np * Np + src];
        v = make_double2(u.x * scale, u.y * scale);
    }
    Y[i] = v;
}

unsigned blocks_for(long total) { return (unsigned)((total + 255) / 256); }

template <int M>
dgfs_status fft3(dgfs_plan_s *plan, double2 *data, long count, int sign, cudaStream_t st)
{
    const dim3 grid((M * M + 127) / 128, (unsigned)count);
    ProfScope ps(plan, "dealias_fft", st);
    if (sign < 0) {
        k_fft_axis<M, 0, -1><<<grid, 128, 0, st>>>(data);
        k_fft_axis<M, 1, -1><<<grid, 128, 0, st>>>(data);
        k_fft_axis<M, 2, -1><<<grid, 128, 0, st>>>(data);
    } else {
        k_fft_axis<M, 0, +1><<<grid, 128, 0, st>>>(data);
        k_fft_axis<M, 1, +1><<<grid, 128, 0, st>>>(data);
        k_fft_axis<M, 2, +1><<<grid, 128, 0, st>>>(data);
    }
    plan->launches += 2;  // the third is counted below
    DGFS_LAUNCHED(plan);
    return DGFS_OK;
}

dgfs_status fft3_any(dgfs_plan_s *plan, int M, double2 *data, long count, int sign, cudaStream_t st)
{
    switch (M) {
    case 4: return fft3<4>(plan, data, count, sign, st);
    case 6: return fft3<6>(plan, data, count, sign, st);
    case 8: return fft3<8>(plan, data, count, sign, st);
    case 12: return fft3<12>(plan, data, count, sign, st);
    case 16: return fft3<16>(plan, data, count, sign, st);
    case 24: return fft3<24>(plan, data, count, sign, st);
    case 32: return fft3<32>(plan, data, count, sign, st);
    case 48: return fft3<48>(plan, data, count, sign, st);
    }
    set_error("dealias: grid size not supported");
    return DGFS_EUNSUPPORTED;
}

bool dealias_sizes(const dgfs_plan_s *plan, int N)
{
    return N >= 4 && N % 2 == 0 && (3 * N) % 2 == 0 && 3 * N / 2 == plan->N;
}

struct DealiasWork {
    double2 *A;  // [P][S*S][N^3]: F, later Y
    double2 *B;  // [P][S*S][N'^3]: G, later X
    void *fpad;  // [P][S][N'^3] plan element type
    void *Qpad;  // [P][S][S][N'^3] plan element type
};

size_t work_bytes(const dgfs_plan_s *plan, int P, int N, DealiasWork *w, void *base)
{
    const long n = (long)N * N * N, np3 = (long)plan->N * plan->N * plan->N;
    const long S = plan->S, es = (long)elem_size(plan);
    const size_t a = sizeof(double2) * (size_t)P * S * S * n, b = sizeof(double2) * (size_t)P * S * S * np3;
    const size_t c = (size_t)es * P * S * np3, d = (size_t)es * P * S * S * np3;
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    if (w) {
        uint8_t *p = reinterpret_cast<uint8_t *>(base);
        w->A = reinterpret_cast<double2 *>(p);
        w->B = reinterpret_cast<double2 *>(p + up(a));
        w->fpad = p + up(a) + up(b);
        w->Qpad = p + up(a) + up(b) + up(c);
    }
    return up(a) + up(b) + up(c) + up(d);
}

template <typename T>
dgfs_status dealiased(dgfs_plan_s *plan, int P, int N, const void *f, void *Q, void *work, cudaStream_t st)
{
    const int Np = plan->N, S = plan->S;
    const long n = (long)N * N * N, np3 = (long)Np * Np * Np;
    DealiasWork w{};
    work_bytes(plan, P, N, &w, work);
    const double up3 = std::pow((double)Np / N, 3), down3 = std::pow((double)N / Np, 3);
    // 1. spectrum of f, embedded on the N' grid, back to physical space
    {
        const long tot = (long)P * S * n;
        ProfScope ps(plan, "dealias_resample", st);
        k_to_complex<T><<<blocks_for(tot), 256, 0, st>>>(reinterpret_cast<const T *>(f), w.A, tot);
        DGFS_LAUNCHED(plan);
    }
    dgfs_status s = fft3_any(plan, N, w.A, (long)P * S, -1, st);
    if (s != DGFS_OK) return s;
    {
        const long tot = (long)P * S * np3;
        ProfScope ps(plan, "dealias_resample", st);
        k_embed<<<blocks_for(tot), 256, 0, st>>>(w.A, w.B, N, Np, (long)P * S, up3);
        DGFS_LAUNCHED(plan);
    }
    s = fft3_any(plan, Np, w.B, (long)P * S, +1, st);
    if (s != DGFS_OK) return s;
    {
        const long tot = (long)P * S * np3;
        ProfScope ps(plan, "dealias_resample", st);
        k_real_part<T><<<blocks_for(tot), 256, 0, st>>>(w.B, reinterpret_cast<T *>(w.fpad), tot, 1.0 / np3);
        DGFS_LAUNCHED(plan);
    }
    // 2. Algorithm 2 on the N' grid
    s = dgfs_collide(plan, P, w.fpad, w.Qpad, st);
    if (s != DGFS_OK) return s;
    // 3. the retained wavenumbers of the result, back on the N grid
    {
        const long tot = (long)P * S * S * np3;
        ProfScope ps(plan, "dealias_resample", st);
        k_to_complex<T><<<blocks_for(tot), 256, 0, st>>>(reinterpret_cast<const T *>(w.Qpad), w.B, tot);
        DGFS_LAUNCHED(plan);
    }
    s = fft3_any(plan, Np, w.B, (long)P * S * S, -1, st);
    if (s != DGFS_OK) return s;
    {
        const long tot = (long)P * S * S * n;
        ProfScope ps(plan, "dealias_resample", st);
        k_gather<<<blocks_for(tot), 256, 0, st>>>(w.B, w.A, N, Np, (long)P * S * S, down3);
        DGFS_LAUNCHED(plan);
    }
    s = fft3_any(plan, N, w.A, (long)P * S * S, +1, st);
    if (s != DGFS_OK) return s;
    {
        const long tot = (long)P * S * S * n;
        ProfScope ps(plan, "dealias_resample", st);
        k_real_part<T><<<blocks_for(tot), 256, 0, st>>>(w.A, reinterpret_cast<T *>(Q), tot, 1.0 / n);
        DGFS_LAUNCHED(plan);
    }
    return DGFS_OK;
}

}  // namespace
}  // namespace dgfs

using namespace dgfs;

extern "C" {

dgfs_status dgfs_dealias_work_bytes(dgfs_plan plan, int P, int N, size_t *bytes)
{
    if (!plan || !bytes || P < 1 || P > plan->max_points || !dealias_sizes(plan, N)) {
        set_error("dgfs_dealias_work_bytes: bad plan, P, or N (the plan's N must be 3N/2)");
        return DGFS_EINVAL;
    }
    *bytes = work_bytes(plan, P, N, nullptr, nullptr);
    return DGFS_OK;
}

dgfs_status dgfs_collide_dealiased(dgfs_plan plan, int P, int N, const void *f_dev, void *Q_dev, void *work_dev,
                                   size_t work_bytes_given, void *stream)
{
    if (!plan || !f_dev || !Q_dev || !work_dev || P < 1 || P > plan->max_points || !dealias_sizes(plan, N) ||
        work_bytes_given < work_bytes(plan, P, N, nullptr, nullptr) ||
        (reinterpret_cast<uintptr_t>(work_dev) & 255)) {
        set_error("dgfs_collide_dealiased: bad plan, pointer, P, N (the plan's N must be 3N/2), or work "
                  "buffer (256-byte aligned, at least dgfs_dealias_work_bytes)");
        return DGFS_EINVAL;
    }
    if (plan->hermitian) {
        set_error("dgfs_collide_dealiased: runs the literal operator; switch the plan's Hermitian form off");
        return DGFS_EUNSUPPORTED;
    }
    dgfs_status st = plan_entry_check(plan);
    if (st != DGFS_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (plan->prec == DGFS_FP64) return dealiased<double>(plan, P, N, f_dev, Q_dev, work_dev, s);
    return dealiased<float>(plan, P, N, f_dev, Q_dev, work_dev, s);
}

}  // extern "C"

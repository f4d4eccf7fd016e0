// Tensor-core (tcgen05) FP32 path of the collision operator (Algorithm 2).
//
// Reformulation.  With the separable phase of Algorithm 1 (a_rs(l) =
// pi/L rho_r l.sigma_s), the translate ifft(t1) of Algorithm 2 step 6 is the
// tensor product of three length-N operators acting on the physical samples
// of f_p:  A_rs = (T^p_x (x) T^p_y (x) T^p_z) f_p,  T^p_d = F^-1 diag(phi^p_d) F,
// phi^p_d(l) = exp(+i m_q/(m_p+m_q) pi/L rho_r sigma_{s,d} l); likewise B_rs from
// f_q with exp(-i m_p/(m_p+m_q) ...).  Each T is a dense N x N complex matrix, so
// every 1-D stage of the method is a dense contraction: (lines x K) x (K x 2N),
// run on the 5th-generation tensor cores with complex numbers as real 2x2
// blocks.  The gain of step 6-7 is then
//   QG = sum_rs w_rs b_rs . F_x F_y F_z (A_rs . B_rs).
//
// Kernels per (point, pair) chunk:
//   stage A (plane, per x-plane):  A' = T_y T_z f_p,  B' = T_y T_z f_q        (tcgen05)
//   stage B (pencil along x):      H  = F_x ( (T^p_x A') . (T^q_x B') )      (tcgen05)
//   stage C (plane, per kx-plane): QG_part += w_rs b_rs . F_y F_z H           (tcgen05, loop over (r, s))
//   finish (FP64 SIMT FFTs):       Q = beta/n Re( ifft3_u(sum QG_part) - f_p ifft3_u(c . F_q) )
// The finish is ~1% of the transforms; doing it in FP64 keeps the loss term
// and the gain-loss cancellation out of the FP32 error budget.
//
// Precision: operands are split x = hi + lo with hi = round-to-nearest TF32 and
// lo = x - hi (exact in FP32); the 3-term product hi*hi + hi*lo + lo*hi with FP32
// accumulation in TMEM gives FP32-level results ("3xTF32").  DGFS_TF32 uses
// the single hi*hi product.
//
// Every mbarrier wait is bounded; on expiry the kernel raises the plan's error
// flag, frees its TMEM and returns (reported as DGFS_ETIMEOUT by dgfs_plan_check).
#include <algorithm>
#include <cstdint>

#include "dgfs_internal.h"
#include "fftreg.cuh"
#include "umma.cuh"

namespace dgfs {
namespace {

using namespace umma;

constexpr int kRows = 128;             // MMA M: data rows per CTA
constexpr int kThreads = 128;          // one thread per data row / TMEM lane
constexpr long kWaitLimit = 1L << 22;  // mbarrier polls before declaring a timeout
constexpr int kErrTimeout = 1;

struct TcState {
    float *Fm = nullptr;      // forward DFT as B operand [2 terms][2N][2N]
    float2 *tw32 = nullptr;   // [N] exp(-2 pi i j/N)
    int *err = nullptr;       // device error flag
    int nterms = 3;
    int chunk = 4;            // evaluations per launch
    int rsb = 8;              // (r, s) blocks of stage C
};

struct TcArgs {
    long n;
    int S, p, q, pt0, RS, nterms, rs_per_block, rsb;
    const float *f;      // [P][S][n]
    float2 *Ap, *Bq, *H; // [E][RS][n]
    float2 *QGp;         // [E][rsb][n]
    const float *tmat;   // pair: [RS][2 sides][2 terms][10 N^2]
    const float *Fm;     // [2 terms][4 N^2]
    const float2 *b32;   // [RS][n]
    const double *w;     // [RS]
    int *err;
};

__host__ __device__ constexpr int atoms(int kfloats) { return (kfloats * 4 + 127) / 128; }
__host__ __device__ constexpr int pow2_cols(int c) { return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512; }

__device__ __forceinline__ uint8_t *align1024(uint8_t *p)
{
    return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo)
{
    hi = tf32_rna(x);
    lo = tf32_rna(x - hi);
}

// Copy a row-major [rows][K] FP32 matrix pair (hi, lo) from global memory into
// SW128 K-major operands (K a multiple of 4).
__device__ __forceinline__ void load_bop(uint8_t *dh, uint8_t *dl, const float *gh, const float *gl, int rows, int K,
                                         int nterms)
{
    const int q = K / 4;
    for (int i = threadIdx.x; i < rows * q; i += blockDim.x) {
        const int r = i / q, kb = (i % q) * 16;
        const uint32_t o = sw128_off(r, kb, rows);
        *reinterpret_cast<float4 *>(dh + o) = reinterpret_cast<const float4 *>(gh)[i];
        if (nterms > 1) *reinterpret_cast<float4 *>(dl + o) = reinterpret_cast<const float4 *>(gl)[i];
    }
}

// store a split complex value at (row, complex index k) of a K-major operand
__device__ __forceinline__ void st_c(uint8_t *ah, uint8_t *al, int row, int k, float re, float im)
{
    float h0, l0, h1, l1;
    split_tf32(re, h0, l0);
    split_tf32(im, h1, l1);
    const uint32_t o = sw128_off(row, 8 * k, kRows);
    *reinterpret_cast<float2 *>(ah + o) = make_float2(h0, h1);
    *reinterpret_cast<float2 *>(al + o) = make_float2(l0, l1);
}

// Issue D = A * B^T over K bytes with 1 or 3 split terms (small terms first).
__device__ __forceinline__ void gemm(uint32_t d, const uint8_t *ah, const uint8_t *al, const uint8_t *bh,
                                     const uint8_t *bl, int brows, int kbytes, int nterms, uint32_t idesc)
{
    const uint8_t *as[3] = {al, ah, ah};
    const uint8_t *bs[3] = {bh, bl, bh};
    const int t0 = nterms == 3 ? 0 : 2;
    uint32_t acc = 0;
    for (int t = t0; t < 3; ++t) {
        const uint32_t a0 = smem_u32(as[t]), b0 = smem_u32(bs[t]);
        for (int kb = 0; kb < kbytes; kb += 32) {
            const uint32_t ao = (kb >> 7) * (kRows * 128) + (kb & 127);
            const uint32_t bo = (kb >> 7) * (brows * 128) + (kb & 127);
            mma_tf32(d, desc_sw128(a0 + ao), desc_sw128(b0 + bo), idesc, acc);
            acc = 1;
        }
    }
}

// Block-wide: thread 0 issues `issue()`, commits to mbar; all threads wait.
// Returns false (for every thread) if the wait expired.
template <typename F>
__device__ __forceinline__ bool run_mma(uint64_t *mbar, uint32_t &phase, F issue)
{
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x == 0) {
        issue();
        commit(mbar);
    }
    const bool ok = mbar_wait(mbar, phase, kWaitLimit);
    phase ^= 1u;
    const int all = __syncthreads_and(ok ? 1 : 0);
    fence_after();
    return all != 0;
}

__device__ __forceinline__ uint32_t lane_base(uint32_t tbase) { return tbase + ((uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16); }

// ------------------------------------------------------------------ stage A
// CTA: G = 128/N x-planes of one (eval, r, s).  For each side (p: f_p, T^p;
// q: f_q, T^q): z-pass (real in) then y-pass, both on the tensor cores.
template <int N>
__global__ void __launch_bounds__(kThreads) k_stage_a(TcArgs a)
{
    constexpr int G = kRows / N, KR = N, KC = 2 * N, NO = 2 * N;
    constexpr int ABYTES = atoms(KC) * kRows * 128, BBYTES = atoms(KC) * NO * 128;
    constexpr int MSZ = 10 * N * N;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align1024(smem_raw);
    uint8_t *Ah = sm, *Al = Ah + ABYTES, *Bh = Al + ABYTES, *Bl = Bh + BBYTES;
    __shared__ uint64_t mbar;
    __shared__ uint32_t tslot;
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * G, rs = blockIdx.y, e = blockIdx.z;
    const int nvalid = min(G, N - x0);
    const long n = a.n;
    const int pt = a.pt0 + e;
    if (t < 32) tmem_alloc(&tslot, pow2_cols(2 * NO));
    if (t == 0) mbar_init(&mbar, 1);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tb = tslot, tl = lane_base(tb);
    uint32_t phase = 0;
    bool ok = true;
    const int g = t / N, yl = t % N;  // row t = (plane g, line y) before the y-pass
    for (int side = 0; side < 2 && ok; ++side) {
        const int sp = side == 0 ? a.p : a.q;
        const float *fs = a.f + ((long)pt * a.S + sp) * n + (long)x0 * N * N;
        const float *tm = a.tmat + (long)(rs * 2 + side) * 2 * MSZ;
        // data: rows (g, y), K = z (real)
        for (int i = t; i < nvalid * N * N / 4; i += kThreads) {
            const float4 v = reinterpret_cast<const float4 *>(fs)[i];
            const int row = (4 * i) / N, kb = ((4 * i) % N) * 4;
            float4 h, l;
            split_tf32(v.x, h.x, l.x);
            split_tf32(v.y, h.y, l.y);
            split_tf32(v.z, h.z, l.z);
            split_tf32(v.w, h.w, l.w);
            const uint32_t o = sw128_off(row, kb, kRows);
            *reinterpret_cast<float4 *>(Ah + o) = h;
            *reinterpret_cast<float4 *>(Al + o) = l;
        }
        load_bop(Bh, Bl, tm, tm + MSZ, NO, KR, a.nterms);  // T_z (real in)
        ok = run_mma(&mbar, phase, [&] { gemm(tb, Ah, Al, Bh, Bl, NO, KR * 4, a.nterms, idesc_tf32(kRows, NO)); });
        if (!ok) break;
        // transpose within each plane: row (g, y) holds z' -> rows (g, z'), K = y
#pragma unroll
        for (int c0 = 0; c0 < NO; c0 += 16) {
            float v[16];
            tmem_ld16(tl + c0, v);
            if (t < nvalid * N) {
#pragma unroll
                for (int j = 0; j < 8; ++j) st_c(Ah, Al, g * N + c0 / 2 + j, yl, v[2 * j], v[2 * j + 1]);
            }
        }
        __syncthreads();
        load_bop(Bh, Bl, tm + 2 * N * N, tm + MSZ + 2 * N * N, NO, KC, a.nterms);  // T_y
        ok = run_mma(&mbar, phase, [&] { gemm(tb + NO, Ah, Al, Bh, Bl, NO, KC * 4, a.nterms, idesc_tf32(kRows, NO)); });
        if (!ok) break;
        // row t = (g, z'): y' values -> global [x][y'][z']
        float2 *dst = (side == 0 ? a.Ap : a.Bq) + ((long)e * a.RS + rs) * n + (long)(x0 + g) * N * N + yl;
#pragma unroll
        for (int c0 = 0; c0 < NO; c0 += 16) {
            float v[16];
            tmem_ld16(tl + NO + c0, v);
            if (t < nvalid * N) {
#pragma unroll
                for (int j = 0; j < 8; ++j) dst[(long)(c0 / 2 + j) * N] = make_float2(v[2 * j], v[2 * j + 1]);
            }
        }
        fence_before();
        __syncthreads();
        fence_after();
    }
    if (!ok && t == 0) atomicExch(a.err, kErrTimeout);
    fence_before();
    __syncthreads();
    if (t < 32) tmem_dealloc(tb, pow2_cols(2 * NO));
}

// ------------------------------------------------------------------ stage B
// CTA: 128 pencils (y, z) of one (eval, r, s).  H = F_x ((T^p_x A') . (T^q_x B')).
template <int N>
__global__ void __launch_bounds__(kThreads) k_stage_b(TcArgs a)
{
    constexpr int KC = 2 * N, NO = 2 * N;
    constexpr int ABYTES = atoms(KC) * kRows * 128, BBYTES = atoms(KC) * NO * 128;
    constexpr int MSZ = 10 * N * N;
    constexpr int NN = N * N;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align1024(smem_raw);
    uint8_t *Ah = sm, *Al = Ah + ABYTES, *Bh = Al + ABYTES, *Bl = Bh + BBYTES;
    __shared__ uint64_t mbar;
    __shared__ uint32_t tslot;
    const int t = threadIdx.x;
    const int p0 = blockIdx.x * kRows, rs = blockIdx.y, e = blockIdx.z;
    const int nvalid = min(kRows, NN - p0);
    const long n = a.n;
    constexpr uint32_t NCOL = pow2_cols(3 * NO);
    if (t < 32) tmem_alloc(&tslot, NCOL);
    if (t == 0) mbar_init(&mbar, 1);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tb = tslot, tl = lane_base(tb);
    uint32_t phase = 0;
    bool ok = true;
    const long gbase = ((long)e * a.RS + rs) * n + p0;
    for (int side = 0; side < 2 && ok; ++side) {
        const float2 *src = (side == 0 ? a.Ap : a.Bq) + gbase;
        const float *tm = a.tmat + (long)(rs * 2 + side) * 2 * MSZ + 6 * NN;  // T_x
        if (t < nvalid) {
#pragma unroll 4
            for (int x = 0; x < N; ++x) {
                const float2 v = src[(long)x * NN + t];
                st_c(Ah, Al, t, x, v.x, v.y);
            }
        }
        load_bop(Bh, Bl, tm, tm + MSZ, NO, KC, a.nterms);
        ok = run_mma(&mbar, phase,
                     [&] { gemm(tb + side * NO, Ah, Al, Bh, Bl, NO, KC * 4, a.nterms, idesc_tf32(kRows, NO)); });
    }
    if (ok) {
        // P = A . B (complex), back into the data operand
#pragma unroll
        for (int c0 = 0; c0 < NO; c0 += 16) {
            float va[16], vb[16];
            tmem_ld16(tl + c0, va);
            tmem_ld16(tl + NO + c0, vb);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float re = va[2 * j] * vb[2 * j] - va[2 * j + 1] * vb[2 * j + 1];
                const float im = va[2 * j] * vb[2 * j + 1] + va[2 * j + 1] * vb[2 * j];
                st_c(Ah, Al, t, c0 / 2 + j, re, im);
            }
        }
        __syncthreads();
        load_bop(Bh, Bl, a.Fm, a.Fm + 4 * NN, NO, KC, a.nterms);
        ok = run_mma(&mbar, phase,
                     [&] { gemm(tb + 2 * NO, Ah, Al, Bh, Bl, NO, KC * 4, a.nterms, idesc_tf32(kRows, NO)); });
    }
    if (ok) {
        float2 *dst = a.H + gbase + t;
#pragma unroll
        for (int c0 = 0; c0 < NO; c0 += 16) {
            float v[16];
            tmem_ld16(tl + 2 * NO + c0, v);
            if (t < nvalid) {
#pragma unroll
                for (int j = 0; j < 8; ++j) dst[(long)(c0 / 2 + j) * NN] = make_float2(v[2 * j], v[2 * j + 1]);
            }
        }
    }
    if (!ok && t == 0) atomicExch(a.err, kErrTimeout);
    fence_before();
    __syncthreads();
    if (t < 32) tmem_dealloc(tb, NCOL);
}

// ------------------------------------------------------------------ stage C
// CTA: G kx-planes of one eval and one block of (r, s).  For every (r, s):
// t3 = F_y F_z H on the tensor cores, QG_part += w_rs b_rs . t3 in registers.
template <int N>
__global__ void __launch_bounds__(kThreads) k_stage_c(TcArgs a)
{
    constexpr int G = kRows / N, KC = 2 * N, NO = 2 * N;
    constexpr int ABYTES = atoms(KC) * kRows * 128, BBYTES = atoms(KC) * NO * 128;
    constexpr int NN = N * N;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align1024(smem_raw);
    uint8_t *Ah = sm, *Al = Ah + ABYTES, *Bh = Al + ABYTES, *Bl = Bh + BBYTES;
    __shared__ uint64_t mbar;
    __shared__ uint32_t tslot;
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * G, rb = blockIdx.y, e = blockIdx.z;
    const int nvalid = min(G, N - x0);
    const long n = a.n;
    if (t < 32) tmem_alloc(&tslot, pow2_cols(2 * NO));
    if (t == 0) mbar_init(&mbar, 1);
    load_bop(Bh, Bl, a.Fm, a.Fm + 4 * NN, NO, KC, a.nterms);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tb = tslot, tl = lane_base(tb);
    uint32_t phase = 0;
    bool ok = true;
    const int g = t / N, yl = t % N;
    float2 acc[N];
#pragma unroll
    for (int k = 0; k < N; ++k) acc[k] = make_float2(0.f, 0.f);
    const int rs0 = rb * a.rs_per_block, rs1 = min(a.RS, rs0 + a.rs_per_block);
    for (int rs = rs0; rs < rs1 && ok; ++rs) {
        const float2 *src = a.H + ((long)e * a.RS + rs) * n + (long)x0 * NN;
        // rows (g, y), K = z (complex): contiguous planes
        for (int i = t; i < nvalid * NN / 2; i += kThreads) {
            const float4 v = reinterpret_cast<const float4 *>(src)[i];
            const int c = 2 * i;
            const int row = c / N, kb = (c % N) * 8;
            float4 h, l;
            split_tf32(v.x, h.x, l.x);
            split_tf32(v.y, h.y, l.y);
            split_tf32(v.z, h.z, l.z);
            split_tf32(v.w, h.w, l.w);
            const uint32_t o = sw128_off(row, kb, kRows);
            *reinterpret_cast<float4 *>(Ah + o) = h;
            *reinterpret_cast<float4 *>(Al + o) = l;
        }
        ok = run_mma(&mbar, phase, [&] { gemm(tb, Ah, Al, Bh, Bl, NO, KC * 4, a.nterms, idesc_tf32(kRows, NO)); });
        if (!ok) break;
#pragma unroll
        for (int c0 = 0; c0 < NO; c0 += 16) {
            float v[16];
            tmem_ld16(tl + c0, v);
            if (t < nvalid * N) {
#pragma unroll
                for (int j = 0; j < 8; ++j) st_c(Ah, Al, g * N + c0 / 2 + j, yl, v[2 * j], v[2 * j + 1]);
            }
        }
        ok = run_mma(&mbar, phase, [&] { gemm(tb + NO, Ah, Al, Bh, Bl, NO, KC * 4, a.nterms, idesc_tf32(kRows, NO)); });
        if (!ok) break;
        // row t = (g, kz): t3(kx0+g, ky, kz) for all ky
        const float wr = (float)a.w[rs];
        const float2 *brs = a.b32 + (long)rs * n + (long)(x0 + g) * NN + yl;
#pragma unroll
        for (int c0 = 0; c0 < NO; c0 += 16) {
            float v[16];
            tmem_ld16(tl + NO + c0, v);
            if (t < nvalid * N) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int ky = c0 / 2 + j;
                    const float2 bb = brs[(long)ky * N];
                    const float tr = v[2 * j], ti = v[2 * j + 1];
                    acc[ky].x = fmaf(wr, bb.x * tr - bb.y * ti, acc[ky].x);
                    acc[ky].y = fmaf(wr, bb.x * ti + bb.y * tr, acc[ky].y);
                }
            }
        }
        fence_before();
        __syncthreads();
        fence_after();
    }
    if (ok && t < nvalid * N) {
        float2 *dst = a.QGp + ((long)e * a.rsb + rb) * n + (long)(x0 + g) * NN + yl;
#pragma unroll
        for (int ky = 0; ky < N; ++ky) dst[(long)ky * N] = acc[ky];
    }
    if (!ok && t == 0) atomicExch(a.err, kErrTimeout);
    fence_before();
    __syncthreads();
    if (t < 32) tmem_dealloc(tb, pow2_cols(2 * NO));
}

// ------------------------------------------------- partial sums of the gain
// QG64[pt0 + e][k] = sum_rb QGp[e][rb][k]  (FP32 partials summed in FP64)
__global__ void k_sum_partials(double2 *QG64, const float2 *QGp, int rsb, long n, int pt0, int E)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)E * n) return;
    const long e = i / n, k = i % n;
    double sx = 0.0, sy = 0.0;
    for (int rb = 0; rb < rsb; ++rb) {
        const float2 v = QGp[(e * rsb + rb) * n + k];
        sx += v.x;
        sy += v.y;
    }
    QG64[(pt0 + e) * n + k] = make_double2(sx, sy);
}

// ------------------------------------------------------ table preparation
// T_d[j][j'] = (1/N) sum_l exp(2 pi i l (j - j') / N) phi_d(l), written as split
// B operands: z (real input) [2N][N]; y, x (complex input) [2N][2N].
__global__ void k_tmat(float *out, const double2 *phase, int N, int RS)
{
    const long total = (long)RS * 2 * 3 * N * N;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int jp = (int)(i % N), j = (int)((i / N) % N), ax = (int)((i / ((long)N * N)) % 3);
    const int side = (int)((i / (3L * N * N)) % 2), rs = (int)(i / (6L * N * N));
    const double2 *ph = phase + ((long)rs * 6 + side * 3 + ax) * N;
    double tr = 0, ti = 0;
    for (int l = 0; l < N; ++l) {
        const int m = ((l * (j - jp)) % N + N) % N;
        double s, c;
        sincospi(2.0 * m / N, &s, &c);
        tr += c * ph[l].x - s * ph[l].y;
        ti += c * ph[l].y + s * ph[l].x;
    }
    tr /= N;
    ti /= N;
    const long MSZ = 10L * N * N;
    float *hi = out + ((long)rs * 2 + side) * 2 * MSZ;
    float *lo = hi + MSZ;
    auto put = [&](long idx, double v) {
        const float h = tf32_rna((float)v);
        hi[idx] = h;
        lo[idx] = tf32_rna((float)(v - (double)h));
    };
    if (ax == 2) {  // z: real input, [2N][N]
        put((long)(2 * j) * N + jp, tr);
        put((long)(2 * j + 1) * N + jp, ti);
    } else {
        const long off = ax == 1 ? 2L * N * N : 6L * N * N;
        const int K = 2 * N;
        put(off + (long)(2 * j) * K + 2 * jp, tr);
        put(off + (long)(2 * j) * K + 2 * jp + 1, -ti);
        put(off + (long)(2 * j + 1) * K + 2 * jp, ti);
        put(off + (long)(2 * j + 1) * K + 2 * jp + 1, tr);
    }
}

// forward DFT F[k][j] = exp(-2 pi i jk/N) as a split complex-input B operand
__global__ void k_fmat(float *out, int N)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * N) return;
    const int j = i % N, k = i / N;
    double s, c;
    sincospi(2.0 * ((j * k) % N) / N, &s, &c);
    const double fr = c, fi = -s;
    const int K = 2 * N;
    float *hi = out, *lo = out + 4 * N * N;
    auto put = [&](long idx, double v) {
        const float h = tf32_rna((float)v);
        hi[idx] = h;
        lo[idx] = tf32_rna((float)(v - (double)h));
    };
    put((long)(2 * k) * K + 2 * j, fr);
    put((long)(2 * k) * K + 2 * j + 1, -fi);
    put((long)(2 * k + 1) * K + 2 * j, fi);
    put((long)(2 * k + 1) * K + 2 * j + 1, fr);
}

__global__ void k_to_f32(float2 *dst, const double2 *src, long count)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}

unsigned nblk(long total, int t) { return (unsigned)((total + t - 1) / t); }

template <int N>
size_t stage_smem()
{
    return 1024 + 2 * (size_t)atoms(2 * N) * kRows * 128 + 2 * (size_t)atoms(2 * N) * (2 * N) * 128;
}

#define DGFS_TRY(x)                   \
    do {                              \
        dgfs_status s_ = (x);         \
        if (s_ != DGFS_OK) return s_; \
    } while (0)

template <int N>
dgfs_status collide_n(dgfs_plan_s *plan, int P, const void *f, void *Qout, cudaStream_t st)
{
    TcState *ts = reinterpret_cast<TcState *>(plan->tc);
    const int S = plan->S, RS = plan->Nrho * plan->M;
    const long n = (long)N * N * N;
    const int E = ts->chunk, RSB = ts->rsb;
    // workspace: F64 [maxP][S][n] d2 | QG64, G2 [maxP][n] d2 | Ap, Bq, H [E][RS][n] f2 | QGp [E][RSB][n] f2
    double2 *F64 = reinterpret_cast<double2 *>(plan->ws);
    double2 *QG64 = F64 + (long)plan->max_points * S * n;
    double2 *G2 = QG64 + (long)plan->max_points * n;
    float2 *Ap = reinterpret_cast<float2 *>(G2 + (long)plan->max_points * n);
    float2 *Bq = Ap + (long)E * RS * n;
    float2 *H = Bq + (long)E * RS * n;
    float2 *QGp = H + (long)E * RS * n;

    TcArgs a{};
    a.n = n;
    a.S = S;
    a.RS = RS;
    a.nterms = ts->nterms;
    a.rsb = RSB;
    a.rs_per_block = (RS + RSB - 1) / RSB;
    a.f = reinterpret_cast<const float *>(f);
    a.Ap = Ap;
    a.Bq = Bq;
    a.H = H;
    a.QGp = QGp;
    a.Fm = ts->Fm;
    a.err = ts->err;

    const size_t smem = stage_smem<N>();
    // FP64 forward transforms of f for the loss term (step 1 of Algorithm 2)
    DGFS_TRY(fp64_forward(plan, P, f, F64, st));
    constexpr int G = kRows / N;
    for (int p = 0; p < S; ++p)
        for (int q = 0; q < S; ++q) {
            const PairTables &pt = plan->pairs[p * S + q];
            a.p = p;
            a.q = q;
            a.tmat = pt.tmat;
            a.b32 = pt.b32;
            a.w = pt.w;
            for (int pt0 = 0; pt0 < P; pt0 += E) {
                const int Ec = std::min(E, P - pt0);
                a.pt0 = pt0;
                {
                    ProfScope ps(plan, "tc_stage_a", st);
                    k_stage_a<N><<<dim3((N + G - 1) / G, RS, Ec), kThreads, smem, st>>>(a);
                }
                DGFS_LAUNCHED(plan);
                {
                    ProfScope ps(plan, "tc_stage_b", st);
                    k_stage_b<N><<<dim3((N * N + kRows - 1) / kRows, RS, Ec), kThreads, smem, st>>>(a);
                }
                DGFS_LAUNCHED(plan);
                {
                    ProfScope ps(plan, "tc_stage_c", st);
                    k_stage_c<N><<<dim3((N + G - 1) / G, RSB, Ec), kThreads, smem, st>>>(a);
                }
                DGFS_LAUNCHED(plan);
                {
                    ProfScope ps(plan, "tc_sum_partials", st);
                    k_sum_partials<<<nblk((long)Ec * n, 256), 256, 0, st>>>(QG64, QGp, RSB, n, pt0, Ec);
                }
                DGFS_LAUNCHED(plan);
            }
            // step 10 in FP64 for this pair over all points
            DGFS_TRY(fp64_finish(plan, p, q, P, QG64, G2, F64, f, Qout, st));
        }
    return DGFS_OK;
}

template <int N>
dgfs_status set_smem_attrs()
{
    const int smem = (int)stage_smem<N>();
    DGFS_CUDA(cudaFuncSetAttribute(k_stage_a<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    DGFS_CUDA(cudaFuncSetAttribute(k_stage_b<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    DGFS_CUDA(cudaFuncSetAttribute(k_stage_c<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    return DGFS_OK;
}

bool tc_supported_N(int N) { return N == 8 || N == 16 || N == 24 || N == 32 || N == 48; }

}  // namespace

dgfs_status tc_prepare(dgfs_plan_s *plan)
{
    const int N = plan->N, RS = plan->Nrho * plan->M;
    const long n = (long)N * N * N;
    if (!tc_supported_N(N)) {
        set_error("tensor-core plans support N in {8, 16, 24, 32, 48}");
        return DGFS_EUNSUPPORTED;
    }
    if (plan->prec == DGFS_BF16X3) {
        set_error("the split-BF16 form is not built yet");
        return DGFS_EUNSUPPORTED;
    }
    TcState *ts = new TcState();
    plan->tc = ts;
    ts->nterms = plan->prec == DGFS_TF32 ? 1 : 3;
    ts->chunk = std::max(1, std::min(plan->max_points, 8));
    ts->rsb = std::min(RS, 8);
    DGFS_CUDA(cudaMalloc(&ts->Fm, sizeof(float) * 8 * N * N));
    DGFS_CUDA(cudaMalloc(&ts->tw32, sizeof(float2) * N));
    DGFS_CUDA(cudaMalloc(&ts->err, sizeof(int)));
    DGFS_CUDA(cudaMemset(ts->err, 0, sizeof(int)));
    k_fmat<<<nblk((long)N * N, 256), 256>>>(ts->Fm, N);
    DGFS_LAUNCHED(plan);
    k_to_f32<<<1, 64>>>(ts->tw32, plan->twiddle, N);
    DGFS_LAUNCHED(plan);
    for (auto &pt : plan->pairs) {
        DGFS_CUDA(cudaMalloc(&pt.tmat, sizeof(float) * (size_t)RS * 2 * 2 * 10 * N * N));
        DGFS_CUDA(cudaMemset(pt.tmat, 0, sizeof(float) * (size_t)RS * 2 * 2 * 10 * N * N));
        DGFS_CUDA(cudaMalloc(&pt.b32, sizeof(float2) * RS * n));
        plan->table_bytes += sizeof(float) * (size_t)RS * 40 * N * N + sizeof(float2) * RS * n;
        k_tmat<<<nblk((long)RS * 6 * N * N, 256), 256>>>(pt.tmat, pt.phase, N, RS);
        DGFS_LAUNCHED(plan);
        k_to_f32<<<nblk(RS * n, 256), 256>>>(pt.b32, pt.b, RS * n);
        DGFS_LAUNCHED(plan);
    }
    switch (N) {
    case 8: DGFS_TRY(set_smem_attrs<8>()); break;
    case 16: DGFS_TRY(set_smem_attrs<16>()); break;
    case 24: DGFS_TRY(set_smem_attrs<24>()); break;
    case 32: DGFS_TRY(set_smem_attrs<32>()); break;
    case 48: DGFS_TRY(set_smem_attrs<48>()); break;
    }
    DGFS_CUDA(cudaDeviceSynchronize());
    return DGFS_OK;
}

void tc_release(dgfs_plan_s *plan)
{
    TcState *ts = reinterpret_cast<TcState *>(plan->tc);
    if (!ts) return;
    cudaFree(ts->Fm);
    cudaFree(ts->tw32);
    cudaFree(ts->err);
    delete ts;
    plan->tc = nullptr;
}

size_t tc_workspace_bytes(const dgfs_plan_s *plan)
{
    const TcState *ts = reinterpret_cast<const TcState *>(plan->tc);
    const long n = (long)plan->N * plan->N * plan->N;
    const long RS = (long)plan->Nrho * plan->M;
    const long E = ts ? ts->chunk : 1, RSB = ts ? ts->rsb : 1;
    return sizeof(double2) * ((long)plan->max_points * (plan->S + 2) * n) + sizeof(float2) * (3 * E * RS * n + E * RSB * n);
}

dgfs_status tc_collide(dgfs_plan_s *plan, int P, const void *f, void *Q, cudaStream_t st)
{
    switch (plan->N) {
    case 8: return collide_n<8>(plan, P, f, Q, st);
    case 16: return collide_n<16>(plan, P, f, Q, st);
    case 24: return collide_n<24>(plan, P, f, Q, st);
    case 32: return collide_n<32>(plan, P, f, Q, st);
    case 48: return collide_n<48>(plan, P, f, Q, st);
    default: set_error("N not supported by the tensor-core path"); return DGFS_EUNSUPPORTED;
    }
}

void tc_info(const dgfs_plan_s *plan, double *info)
{
    const TcState *ts = reinterpret_cast<const TcState *>(plan->tc);
    if (!ts) return;
    info[9] = ts->chunk;
    info[10] = ts->rsb;
    info[11] = ts->nterms;
}

dgfs_status tc_check(dgfs_plan_s *plan)
{
    TcState *ts = reinterpret_cast<TcState *>(plan->tc);
    if (!ts) return DGFS_OK;
    int v = 0;
    DGFS_CUDA(cudaMemcpy(&v, ts->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (v) {
        DGFS_CUDA(cudaMemset(ts->err, 0, sizeof(int)));
        set_error("a bounded tensor-core wait expired");
        return DGFS_ETIMEOUT;
    }
    return DGFS_OK;
}

}  // namespace dgfs

// Tensor-core (tcgen05) path of the collision operator (Algorithm 2).
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
// Kernels per (pair, chunk of points):
//   stage A (plane, per x-plane):  A' = T_y T_z f_p,  B' = T_y T_z f_q        (tcgen05)
//   stage B (pencil along x):      H  = F_x ( (T^p_x A') . (T^q_x B') )      (tcgen05)
//   stage C (plane, per kx-plane): QG_part += w_rs b_rs . F_y F_z H           (tcgen05, loop over (r, s))
//   finish (FP64 SIMT FFTs):       Q = beta/n Re( ifft3_u(sum QG_part) - f_p ifft3_u(c . F_q) )
// The finish is ~1% of the transforms; doing it in FP64 keeps the loss term
// and the gain-loss cancellation out of the FP32 error budget.
//
// Stage A and B CTAs are matrix-stationary: a CTA owns one (r, s) (and side),
// keeps that (r, s)'s matrices in shared memory (loaded once with one bulk
// copy per pre-swizzled image) and runs several independent 128-thread
// pipelines, each looping over work items (point, plane group or pencil tile)
// and prefetching the next item's data into registers while the current
// item's contractions run.
//
// Precision: operands are split into TF32 (hi + lo) or BF16 (three terms)
// parts, see tcfmt.cuh; accumulation is FP32 in TMEM.
//
// Every mbarrier wait is bounded; on expiry the kernel raises the plan's error
// flag, frees its TMEM and returns (reported as DGFS_ETIMEOUT by dgfs_plan_check).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "dfloat.cuh"
#include "dgfs_internal.h"
#include "tcfmt.cuh"
#include "umma.cuh"
#include "tcstage.cuh"

namespace dgfs {
namespace {

// ------------------------------------------- stage A, two threads per row
// The plane stage with 256-thread pipelines: the two threads of a row split
// its columns (TMEM lanes are shared by warps w and w + 4), halving the work
// and registers per thread so that twice the warps fit on an SM.
template <int COUNT>
__device__ __forceinline__ void pbar_n(int id)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(COUNT) : "memory");
}

template <int COUNT>
__device__ __forceinline__ bool pbar_and_n(int id, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)(v ? 1 : 0)), "r"(id), "n"(COUNT)
        : "memory");
    return r != 0;
}

template <int COUNT, typename F>
__device__ __forceinline__ bool run_mma_n(uint64_t *mbar, uint32_t &phase, int bar_id, F issue)
{
    fence_proxy_async();
    fence_before();
    pbar_n<COUNT>(bar_id);
    fence_after();
    if ((threadIdx.x % COUNT) == 0) {
        issue();
        commit(mbar);
    }
    const bool ok = mbar_wait(mbar, phase, kWaitLimit);
    phase ^= 1u;
    const bool all = pbar_and_n<COUNT>(bar_id, ok);
    fence_after();
    return all;
}

template <int N, int FMT> struct A2 {
    static constexpr int NP = NPipes<N, FMT>::A;
    static constexpr bool OK = Smem<N, FMT>::RES_A && (2 * N) % 32 == 0 && NP * 2 * kRows <= 1024;
};

template <int N, int FMT>
__global__ void __launch_bounds__(2 * kRows * NPipes<N, FMT>::A, 1) k_stage_a2(TcArgs a)
{
    using SM = Smem<N, FMT>;
    constexpr int NP = NPipes<N, FMT>::A, NT = SM::NT, AB = SM::AB, IR = SM::IR, IC = SM::IC;
    constexpr int PT = 2 * kRows;  // threads per pipeline
    constexpr int G = kRows / N, KC = 2 * N, NO = 2 * N, NH = N, NG = (N + G - 1) / G;  // NH: columns per thread
    constexpr int KR = FMT == 1 ? (N + 15) / 16 * 16 : N;
    constexpr int NN = N * N;
    constexpr int FPT = (G * NN / 4 + PT - 1) / PT;  // float4 per thread for one group
    constexpr uint32_t NCOL = pow2_cols(NP * 2 * NO);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align1024(smem_raw);
    const int pp = threadIdx.x / PT, tt = threadIdx.x % PT, t = tt % kRows, hf = tt / kRows, bar = 1 + pp;
    uint8_t *Bz = sm;
    uint8_t *By = Bz + NT * IR;
    uint8_t *A0 = sm + NT * (IR + IC) + pp * NT * AB;
    __shared__ uint64_t mb[NP + 1];
    __shared__ uint32_t tslot;
    const int rs = blockIdx.y, side = blockIdx.z;
    const long n = a.n;
    const int items = a.Ec * NG;
    const bool ident_y = a.idmask && (a.idmask[rs] & 2);
    cta_setup(&tslot, NCOL, mb, NP + 1);
    const uint32_t tb = tslot + pp * 2 * NO, tl = lane_base(tb) + hf * NH;  // this thread's column half
    uint32_t ph_mma = 0, ph_cp = 0;
    const int sp = side == 0 ? a.p : a.q;
    const int g = t / N, yl = t % N;
    float4 pf[FPT];
    auto prefetch = [&](int it) {
        const int e = it / NG, x0 = (it % NG) * G, nval = min(G, N - x0);
        const float4 *fs =
            reinterpret_cast<const float4 *>(a.f + ((long)(a.pt0 + e) * a.S + sp) * n + (long)x0 * NN);
#pragma unroll
        for (int j = 0; j < FPT; ++j) {
            const int i = tt + PT * j;
            pf[j] = (4 * i < nval * NN) ? fs[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    const int stride = gridDim.x * NP;
    int it = blockIdx.x * NP + pp;
    if (it < items) prefetch(it);
    if (threadIdx.x == 0) {
        mbar_expect_tx(&mb[NP], NT * (IR + IC));
        copy_terms(Bz, IR, timg_at<FMT>(a.timg, N, rs, side, 2), IC, IR, NT, &mb[NP]);
        copy_terms(By, IC, timg_at<FMT>(a.timg, N, rs, side, 1), IC, IC, NT, &mb[NP]);
    }
    bool ok = wait_copy_cta(&mb[NP], ph_cp);
    for (; it < items && ok; it += stride) {
        const int e = it / NG, x0 = (it % NG) * G, nval = min(G, N - x0);
#pragma unroll
        for (int j = 0; j < FPT; ++j) {
            const int i = tt + PT * j;
            if (4 * i < nval * NN) tcfmt::st_f4<FMT>(A0, AB, (4 * i) / N, (4 * i) % N, pf[j]);
        }
        if constexpr (KR > N) {  // zero the pad of the row (first thread of the row)
            if (hf == 0 && t < nval * N)
#pragma unroll
                for (int term = 0; term < NT; ++term)
#pragma unroll
                    for (int e0 = N; e0 < KR; e0 += 8)
                        *reinterpret_cast<uint4 *>(A0 + term * AB + sw128_off(t, e0 * Fmt<FMT>::ESZ, kRows)) =
                            make_uint4(0u, 0u, 0u, 0u);
        }
        if (it + stride < items) prefetch(it + stride);
        ok = run_mma_n<PT>(&mb[pp], ph_mma, bar, [&] { tcfmt::gemm<FMT>(tb, A0, AB, Bz, IR, NO, KR, a.nterms); });
        if (!ok) break;
        if (ident_y) {
            float2 *dst = (side == 0 ? a.Ap : a.Bq) + ((long)e * a.RS + rs) * n + (long)(x0 + g) * NN + yl * N +
                          hf * (NH / 2);
            tmem_visit<NH>(tl, [&](int c0, const float *v) {
                if (t < nval * N) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        *reinterpret_cast<float4 *>(dst + c0 / 2 + 2 * j) =
                            make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                }
            });
            continue;
        }
        // transpose within each plane: row (g, y) holds z' -> rows (g, z'), K = y
        tmem_visit<NH>(tl, [&](int c0, const float *v) {
            if (t < nval * N) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    tcfmt::st_c<FMT>(A0, AB, g * N + hf * (NH / 2) + c0 / 2 + j, yl, v[2 * j], v[2 * j + 1]);
            }
        });
        ok = run_mma_n<PT>(&mb[pp], ph_mma, bar,
                           [&] { tcfmt::gemm<FMT>(tb + NO, A0, AB, By, IC, NO, KC, a.nterms); });
        if (!ok) break;
        // row t = (g, z'): this thread's half of the y' values -> global [x][y'][z']
        float2 *dstp = (side == 0 ? a.Ap : a.Bq) + ((long)e * a.RS + rs) * n + (long)(x0 + g) * NN + (yl & ~1) +
                       (long)hf * (NH / 2) * N;
        tmem_visit<NH>(tl + NO, [&](int c0, const float *v) {
            float2 h[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) h[j] = make_float2(v[2 * j], v[2 * j + 1]);
            store_pair<8>(dstp + (long)(c0 / 2) * N, h, N, t < nval * N);
        });
    }
    cta_teardown(tslot, NCOL, ok, a.err);
}

// ------------------------------------------------- stage A, warp-specialised
// The same plane stage with its three kinds of work on separate warpgroups of
// one CTA, so that the tensor core works on one item while the CUDA cores
// prepare the next and drain the previous:
//   WG0 (load):         f tile -> split -> A_z[slot]; its thread 0 issues the
//                       z-pass into TMEM D1[slot];
//   WG1, WG2 (transpose): D1[slot] -> in-plane transpose -> A_y, each half of
//                       the columns; the first thread issues the y-pass into
//                       D2[slot] (sigma_y = 0: D1 goes straight to global
//                       memory instead);
//   WG3 (store):        D2[slot] -> A' / B' in global memory.
// Two slots for A_z, D1, D2 and one A_y; every handoff is an mbarrier
// (full: the MMA's commit or the producer; empty: the consumer) waited on
// with a bound.  A role whose wait expires raises a CTA-wide abort flag that
// the other roles' waits observe; each wait is followed by a vote over the
// role's 128 threads, so a role always leaves its loop as a whole.
template <int N, int FMT> struct WsA {
    static constexpr int NT = Fmt<FMT>::NT;
    static constexpr int KR = FMT == 1 ? (N + 15) / 16 * 16 : N;
    static constexpr int AZB = tcfmt::atoms_b(KR * Fmt<FMT>::ESZ) * kRows * 128;  // one term of A_z
    static constexpr int AB = tcfmt::abytes<FMT>(N), IC = tcfmt::img_c<FMT>(N), IR = tcfmt::img_r<FMT>(N);
    static constexpr size_t BYTES = 1024 + (size_t)NT * (IR + IC) + 2 * (size_t)NT * AZB + (size_t)NT * AB;
    static constexpr bool OK = BYTES <= kSmemMax && N >= 16 && N % 16 == 0;
};

// bounded wait that also gives up when another role has aborted
__device__ __forceinline__ bool ws_wait(uint64_t *mbar, uint32_t parity, volatile int *abort)
{
    for (long it = 0; it < kWaitLimit; it += 64) {
        if (mbar_wait(mbar, parity, 64)) return true;
        if (*abort) return false;
    }
    return false;
}

template <int N, int FMT>
__global__ void __launch_bounds__(4 * kRows, 1) k_stage_a_ws(TcArgs a)
{
    using W = WsA<N, FMT>;
    constexpr int NT = W::NT, AB = W::AB, IR = W::IR, IC = W::IC, AZB = W::AZB, KR = W::KR;
    constexpr int G = kRows / N, KC = 2 * N, NO = 2 * N, NH = N, NG = (N + G - 1) / G, NN = N * N;
    constexpr int FPT = (G * NN / 4 + kRows - 1) / kRows;
    constexpr uint32_t NCOL = pow2_cols(4 * NO);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align1024(smem_raw);
    uint8_t *Bz = sm, *By = sm + NT * IR;
    uint8_t *AZ0 = sm + NT * (IR + IC);  // slot s at AZ0 + s * NT * AZB
    uint8_t *AY = AZ0 + 2 * NT * AZB;
    // [0] images, [1..2] az_empty, [3..4] d1_full, [5..6] d1_empty, [7] ay_empty,
    // [8..9] d2_full, [10..11] d2_empty, [12..13] drain of the two issuing threads
    __shared__ uint64_t mb[14];
    __shared__ uint32_t tslot;
    __shared__ int abort_flag;
    uint64_t *az_empty = mb + 1, *d1_full = mb + 3, *d1_empty = mb + 5, *ay_empty = mb + 7, *d2_full = mb + 8,
             *d2_empty = mb + 10, *drain = mb + 12;
    // roles: 0 load, 1 and 2 transpose (column halves, one 256-thread barrier), 3 store
    const int wg = threadIdx.x / kRows, t = threadIdx.x % kRows;
    const int role = wg == 0 ? 0 : wg == 3 ? 2 : 1, hf = wg - 1, bar = 1 + role;
    const int rs = blockIdx.y, side = blockIdx.z;
    const long n = a.n;
    const int items = a.Ec * NG;
    const bool ident_y = a.idmask && (a.idmask[rs] & 2);
    if (threadIdx.x == 0) abort_flag = 0;
    cta_setup(&tslot, NCOL, mb, 14);
    const uint32_t tb = tslot, tl = lane_base(tb);  // D1[s]: tb + s NO, D2[s]: tb + (2 + s) NO
    volatile int *abort_p = &abort_flag;
    uint32_t ph_img = 0;
    if (threadIdx.x == 0) {
        mbar_expect_tx(&mb[0], NT * (IR + IC));
        copy_terms(Bz, IR, timg_at<FMT>(a.timg, N, rs, side, 2), IC, IR, NT, &mb[0]);
        copy_terms(By, IC, timg_at<FMT>(a.timg, N, rs, side, 1), IC, IC, NT, &mb[0]);
    }
    bool ok = wait_copy_cta(&mb[0], ph_img);
    const int sp = side == 0 ? a.p : a.q;
    const int g = t / N, yl = t % N;
    auto fail = [&]() {
        ok = false;
        *abort_p = 1;
    };

    if (role == 0 && ok) {
        // ---------------------------------------------------------- load
        float4 pf[FPT];
        auto prefetch = [&](int it) {
            const int e = it / NG, x0 = (it % NG) * G, nval = min(G, N - x0);
            const float4 *fs =
                reinterpret_cast<const float4 *>(a.f + ((long)(a.pt0 + e) * a.S + sp) * n + (long)x0 * NN);
#pragma unroll
            for (int j = 0; j < FPT; ++j) {
                const int i = t + kRows * j;
                pf[j] = (4 * i < nval * NN) ? fs[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        int it = blockIdx.x;
        if (it < items) prefetch(it);
        for (int j = 0; it < items; ++j, it += gridDim.x) {
            const int slot = j & 1;
            const uint32_t use = (uint32_t)(j >> 1) & 1u;
            const int x0 = (it % NG) * G, nval = min(G, N - x0);
            uint8_t *AZ = AZ0 + slot * NT * AZB;
            // every wait is followed by a vote, so that the role's threads leave together
            if (!pbar_and(bar, ws_wait(&az_empty[slot], use ^ 1u, abort_p) && !*abort_p)) { fail(); break; }
#pragma unroll
            for (int jj = 0; jj < FPT; ++jj) {
                const int i = t + kRows * jj;
                if (4 * i < nval * NN) tcfmt::st_f4<FMT>(AZ, AZB, (4 * i) / N, (4 * i) % N, pf[jj]);
            }
            if constexpr (KR > N) {
                if (t < nval * N)
#pragma unroll
                    for (int term = 0; term < NT; ++term)
#pragma unroll
                        for (int e0 = N; e0 < KR; e0 += 8)
                            *reinterpret_cast<uint4 *>(AZ + term * AZB + sw128_off(t, e0 * Fmt<FMT>::ESZ, kRows)) =
                                make_uint4(0u, 0u, 0u, 0u);
            }
            if (it + (int)gridDim.x < items) prefetch(it + gridDim.x);
            fence_proxy_async();
            if (!pbar_and(bar, !*abort_p)) { fail(); break; }
            if (t == 0) {
                if (!ws_wait(&d1_empty[slot], use ^ 1u, abort_p)) {
                    fail();
                } else {
                    fence_after();
                    tcfmt::gemm<FMT>(tb + slot * NO, AZ, AZB, Bz, IR, NO, KR, a.nterms);
                    commit(&d1_full[slot]);
                    commit(&az_empty[slot]);
                }
            }
        }
        if (t == 0) {  // every z-pass issued by this thread has completed
            commit(&drain[0]);
            if (!mbar_wait(&drain[0], 0, kWaitLimit)) ok = false;
        }
    } else if (role == 1 && ok) {
        // ---------------------------------------------------- transpose
        int it = blockIdx.x;
        for (int j = 0; it < items; ++j, it += gridDim.x) {
            const int slot = j & 1;
            const uint32_t use = (uint32_t)(j >> 1) & 1u;
            const int e = it / NG, x0 = (it % NG) * G, nval = min(G, N - x0);
            if (!pbar_and_n<2 * kRows>(bar, ws_wait(&d1_full[slot], use, abort_p) && !*abort_p)) { fail(); break; }
            fence_after();
            if (ident_y) {
                // sigma_y = 0: T_y = I, row t = (g, y) holds A'(x0+g, y, z') for all z'
                float2 *dst = (side == 0 ? a.Ap : a.Bq) + ((long)e * a.RS + rs) * n + (long)(x0 + g) * NN +
                              yl * N + hf * (NH / 2);
                tmem_visit<NH>(tl + slot * NO + hf * NH, [&](int c0, const float *v) {
                    if (t < nval * N) {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            *reinterpret_cast<float4 *>(dst + c0 / 2 + 2 * q) =
                                make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    }
                });
                fence_before();
                pbar_n<2 * kRows>(bar);
                if (hf == 0 && t == 0) mbar_arrive(&d1_empty[slot]);
                continue;
            }
            if (!pbar_and_n<2 * kRows>(bar, ws_wait(ay_empty, ((uint32_t)j & 1u) ^ 1u, abort_p) && !*abort_p)) {
                fail();
                break;
            }
            tmem_visit<NH>(tl + slot * NO + hf * NH, [&](int c0, const float *v) {
                if (t < nval * N) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        tcfmt::st_c<FMT>(AY, AB, g * N + hf * (NH / 2) + c0 / 2 + q, yl, v[2 * q], v[2 * q + 1]);
                }
            });
            fence_before();
            fence_proxy_async();
            pbar_n<2 * kRows>(bar);
            if (hf == 0 && t == 0) {
                mbar_arrive(&d1_empty[slot]);
                if (!ws_wait(&d2_empty[slot], use ^ 1u, abort_p)) {
                    fail();
                } else {
                    fence_after();
                    tcfmt::gemm<FMT>(tb + (2 + slot) * NO, AY, AB, By, IC, NO, KC, a.nterms);
                    commit(&d2_full[slot]);
                    commit(ay_empty);
                }
            }
        }
        if (hf == 0 && t == 0) {
            commit(&drain[1]);
            if (!mbar_wait(&drain[1], 0, kWaitLimit)) ok = false;
        }
    } else if (role == 2 && ok && !ident_y) {
        // -------------------------------------------------------- store
        int it = blockIdx.x;
        for (int j = 0; it < items; ++j, it += gridDim.x) {
            const int slot = j & 1;
            const uint32_t use = (uint32_t)(j >> 1) & 1u;
            const int e = it / NG, x0 = (it % NG) * G, nval = min(G, N - x0);
            if (!pbar_and(bar, ws_wait(&d2_full[slot], use, abort_p) && !*abort_p)) { fail(); break; }
            fence_after();
            // row t = (g, z'): y' values -> global [x][y'][z']
            float2 *dstp =
                (side == 0 ? a.Ap : a.Bq) + ((long)e * a.RS + rs) * n + (long)(x0 + g) * NN + (yl & ~1);
            tmem_visit<NO>(tl + (2 + slot) * NO, [&](int c0, const float *v) {
                float2 h[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) h[q] = make_float2(v[2 * q], v[2 * q + 1]);
                store_pair<8>(dstp + (long)(c0 / 2) * N, h, N, t < nval * N);
            });
            fence_before();
            pbar(bar);
            if (t == 0) mbar_arrive(&d2_empty[slot]);
        }
    }
    if (*abort_p) ok = false;
    cta_teardown(tslot, NCOL, __syncthreads_and(ok ? 1 : 0) != 0, a.err);
}

// ------------------------------------------------- partial sums of the gain
// ------------------------------------------------------- batched work list
// One launch of a stage kernel over the jobs (instance, pair, chunk of points)
// of several plans with the same N and operand format: CTA b belongs to the
// job whose first CTA is the largest start <= b, and runs that job's kernel
// body with its own block index and grid.
struct JobGrid {
    uint32_t start, gx, gy, gz;
};

// Jobs of one batched launch, passed by value: the arguments then sit in the
// constant bank like a plain launch's, instead of global memory that every
// store of the kernel may alias.
constexpr int kJobsPerLaunch = 48;
struct JobTable {
    TcArgs job[kJobsPerLaunch];
    JobGrid grid[kJobsPerLaunch];
    int njobs;
};

__device__ __forceinline__ int find_job(const JobTable &t, uint32_t b)
{
    int lo = 0, hi = t.njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (t.grid[mid].start <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint3 job_block(const JobGrid &g, uint32_t b)
{
    const uint32_t l = b - g.start;
    return make_uint3(l % g.gx, (l / g.gx) % g.gy, l / (g.gx * g.gy));
}

template <int N, int FMT>
__global__ void __launch_bounds__(kRows *NPipes<N, FMT>::A, 1) k_stage_a_batch(const __grid_constant__ JobTable t)
{
    const int j = find_job(t, blockIdx.x);
    const JobGrid &g = t.grid[j];
    k_stage_a_body<N, FMT>(t.job[j], job_block(g, blockIdx.x), make_uint3(g.gx, g.gy, g.gz));
}

template <int N, int FMT>
__global__ void __launch_bounds__(kRows *NPipes<N, FMT>::B, 1) k_stage_b_batch(const __grid_constant__ JobTable t)
{
    const int j = find_job(t, blockIdx.x);
    const JobGrid &g = t.grid[j];
    k_stage_b_body<N, FMT>(t.job[j], job_block(g, blockIdx.x), make_uint3(g.gx, g.gy, g.gz));
}

template <int N, int FMT>
__global__ void __launch_bounds__(kRows *NPipes<N, FMT>::C, 1) k_stage_c_batch(const __grid_constant__ JobTable t)
{
    const int j = find_job(t, blockIdx.x);
    const JobGrid &g = t.grid[j];
    k_stage_c_body<N, FMT>(t.job[j], job_block(g, blockIdx.x), make_uint3(g.gx, g.gy, g.gz));
}

// QG[pt0 + e][k] = sum_rb QGp[e][rb][k]  (FP32 partials summed in double-float)
__device__ __forceinline__ void sum_partial(float4 *QG, const float2 *QGp, int rsb, long n, int pt0, long i)
{
    const long e = i / n, k = i % n;
    dfl sx(0.f, 0.f), sy(0.f, 0.f);
    for (int rb = 0; rb < rsb; ++rb) {
        const float2 v = QGp[(e * rsb + rb) * n + k];
        sx = add_f(sx, v.x);
        sy = add_f(sy, v.y);
    }
    st_dcx(QG + (pt0 + e) * n + k, dcx{sx, sy});
}

__global__ void k_sum_partials(float4 *QG, const float2 *QGp, int rsb, long n, int pt0, int E)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)E * n) return;
    sum_partial(QG, QGp, rsb, n, pt0, i);
}

// -------------------------------------------------------- work list
// One launch of k_worklist runs every stage of a list of jobs (a job: one
// species pair and chunk of points of one plan).  A task is one CTA of a plain
// launch's stage A, B or C grid, run by the same body with the same block
// index, or one slice of the partial sums.  CTAs claim tasks from a queue in
// global memory (see k_worklist), wait until the tasks they depend on are
// complete, run them and publish their completion in per-job counters.  With
// prev the job of the same plan queued before job j (whose workspace slots j
// overwrites):
//   A(j, rs)  after B(prev, rs), and B(prev, rs') if prev reads B' from A' at rs' = bmap[rs]
//   B(j, rs)  after A(j, rs) (and A(j, bmap[rs]) when j reads B' from A') and C(prev, g(rs))
//   C(j, g)   after B(j, rs) for every rs of g, and S(prev)
//   S(j)      after C(j, every g)
// where g(rs) is the stage C grid index y whose (r, s)-blocks hold rs.  Tasks
// are queued so that every task's dependencies come before it.  Every wait is
// bounded (global timer); on expiry the CTA raises the job's error flag and
// the launch's abort flag, and every CTA stops taking tasks.
constexpr int kWlJobs = 96;    // jobs per launch
constexpr int kWlSegs = 1024;  // task segments per launch
constexpr long kWlSumChunk = 8192;  // grid points per partial-sum task
constexpr uint64_t kWlWaitNs = 4000000000ull;  // bound of one dependency wait
enum { WL_A = 0, WL_B = 1, WL_C = 2, WL_S = 3 };

struct WlJob {
    TcArgs a;
    float4 *qg;            // QG of the job's pair, as in k_sum_partials
    const uint16_t *bmap;  // same-species pair: B' read from A' at bmap[rs] (null: both sides computed)
    int prev;              // job of the same plan queued before this one in this launch, or -1
    uint32_t cnt;          // first counter of the job: A[RS] B[RS] Bg[gyc] C[gyc] Ctot S
    uint16_t ga, sides, gb, ngc, gyc, ec;  // grids (ga, RS, sides), (gb, RS), (ngc, gyc, ec)
    uint32_t ns;           // partial-sum tasks
};

// Passed by value (constant bank).  seg[i]: x = first task of the segment,
// y = job | stage << 12 | first linear block index << 14; a segment's tasks are
// consecutive linear block indices of one stage grid of one job.
struct WlTable {
    WlJob job[kWlJobs];
    uint2 seg[kWlSegs];
    // ctr: [0] queue head, [1] abort flag, [2] tasks handed on, [3] handed-on
    // tasks taken, [4] claims resolved (run or handed on), from [8] the jobs'
    // counters, from [8 + ring] the ring of handed-on tasks (task + 1; zero at launch)
    uint32_t *ctr;
    uint32_t ring;
    int nseg;
    uint32_t ntasks;
    // optional task trace (dgfs_debug_worklist_trace): per task, the global
    // timer when it was taken, when its dependencies were met and when it
    // ended, and (SM << 8 | stage); tasks beyond trace_cap are not recorded
    unsigned long long *trace;
    uint32_t trace_cap;
};
static_assert(sizeof(WlTable) <= 32764, "a kernel's parameters are limited to 32764 bytes");

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// thread 0: wait until *c >= target; false on abort or when the bound expires
__device__ __noinline__ bool wl_wait(const uint32_t *c, uint32_t target, const uint32_t *abort_flag)
{
    if (ld_acquire_u32(c) >= target) return true;
    const uint64_t t_end = global_ns() + kWlWaitNs;
    for (;;) {
        __nanosleep(128);
        if (ld_acquire_u32(c) >= target) return true;
        if (ld_acquire_u32(abort_flag) || global_ns() > t_end) return false;
    }
}

// counters of a job
struct WlCtr {
    uint32_t *A, *B, *Bg, *C, *Ctot, *S;
};
__device__ __forceinline__ WlCtr wl_ctr(const WlTable &t, const WlJob &J)
{
    WlCtr c;
    c.A = t.ctr + 8 + J.cnt;
    c.B = c.A + J.a.RS;
    c.Bg = c.B + J.a.RS;
    c.C = c.Bg + J.gyc;
    c.Ctot = c.C + J.gyc;
    c.S = c.Ctot + 1;
    return c;
}

// stage C grid index y whose (r, s)-blocks hold rs, and the rs range of index g
template <int NPC> __device__ __forceinline__ int wl_g(const TcArgs &a, int rs) { return rs / a.rs_per_block / NPC; }
template <int NPC> __device__ __forceinline__ int2 wl_grange(const TcArgs &a, int g)
{
    const int lo = g * NPC * a.rs_per_block;
    const int hi = min(a.RS, min(a.rsb, (g + 1) * NPC) * a.rs_per_block);
    return make_int2(lo, max(lo, hi));
}

// thread 0: wait for the dependencies of task (job j, stage, linear block v)
template <int NPC> __device__ bool wl_deps(const WlTable &t, int j, int stage, uint32_t v)
{
    const WlJob &J = t.job[j];
    const WlCtr c = wl_ctr(t, J);
    const uint32_t *ab = t.ctr + 1;
    const bool hp = J.prev >= 0;
    const WlJob &P = t.job[hp ? J.prev : j];
    const WlCtr pc = wl_ctr(t, P);
    if (stage == WL_A) {
        const int rs = (int)(v / J.ga / J.sides);
        if (hp && !wl_wait(pc.B + rs, P.gb, ab)) return false;
        if (hp && P.bmap && !wl_wait(pc.B + __ldg(P.bmap + rs), P.gb, ab)) return false;
    } else if (stage == WL_B) {
        const int rs = (int)(v / J.gb);
        const uint32_t na = (uint32_t)J.ga * J.sides;
        if (!wl_wait(c.A + rs, na, ab)) return false;
        if (J.bmap && !wl_wait(c.A + __ldg(J.bmap + rs), na, ab)) return false;
        if (hp && !wl_wait(pc.C + wl_g<NPC>(P.a, rs), (uint32_t)P.ngc * P.ec, ab)) return false;
    } else if (stage == WL_C) {
        const int g = (int)(v / J.ngc / J.ec);
        const int2 r = wl_grange<NPC>(J.a, g);
        if (!wl_wait(c.Bg + g, (uint32_t)J.gb * (r.y - r.x), ab)) return false;
        if (hp && !wl_wait(pc.S, P.ns, ab)) return false;
    } else {
        if (!wl_wait(c.Ctot, (uint32_t)J.ngc * J.gyc * J.ec, ab)) return false;
    }
    return true;
}

// thread 0, after the task's writes: publish its completion
template <int NPC> __device__ __forceinline__ void wl_done(const WlTable &t, int j, int stage, uint32_t v)
{
    const WlJob &J = t.job[j];
    const WlCtr c = wl_ctr(t, J);
    if (stage == WL_A) {
        atomicAdd(c.A + v / J.ga / J.sides, 1u);
    } else if (stage == WL_B) {
        const int rs = (int)(v / J.gb);
        atomicAdd(c.B + rs, 1u);
        atomicAdd(c.Bg + wl_g<NPC>(J.a, rs), 1u);
    } else if (stage == WL_C) {
        atomicAdd(c.C + v / J.ngc / J.ec, 1u);
        atomicAdd(c.Ctot, 1u);
    } else {
        atomicAdd(c.S, 1u);
    }
}

// (job, stage, linear block index) of task h
__device__ __forceinline__ void wl_decode(const WlTable &t, uint32_t h, int &job, int &stage, uint32_t &v)
{
    int lo = 0, hi = t.nseg - 1;  // the last segment starting at or before h
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (t.seg[mid].x <= h) lo = mid;
        else hi = mid - 1;
    }
    const uint2 sg = t.seg[lo];
    job = (int)(sg.y & 0xFFFu);
    stage = (int)((sg.y >> 12) & 3u);
    v = (sg.y >> 14) + (h - sg.x);
}

// thread 0, a CTA running tasks of one kind (stage `want`; for stage B also
// whether the job reads B' from A', want_share): claim the next task.  True if
// it is of that kind; a task of another kind is handed on through the ring
// (a fresh CTA takes it) and false returned, as when the queue is exhausted
// or the launch aborted.
__device__ bool wl_claim_same(const WlTable &t, int want, int want_share, int &job, int &stage, uint32_t &v,
                              uint32_t &task)
{
    if (ld_acquire_u32(t.ctr + 1)) return false;
    const uint32_t h = atomicAdd(t.ctr, 1u);
    if (h >= t.ntasks) return false;
    wl_decode(t, h, job, stage, v);
    const bool same =
        stage == want && (want_share < 0 || (t.job[job].bmap != nullptr) == (want_share != 0));
    if (!same) {
        const uint32_t i = atomicAdd(t.ctr + 2, 1u);
        atomicExch(t.ctr + 8 + t.ring + i, h + 1);
        __threadfence();
    }
    atomicAdd(t.ctr + 4, 1u);
    task = h;
    return same;
}

// thread 0, a fresh CTA: its first task, a handed-on one if any is waiting,
// else the next one in the queue.  False when no work is left (every task
// claimed and run or handed on, and every handed-on task taken), on abort, or
// when the bounded wait for work expires (the launch is then aborted).
__device__ bool wl_claim_first(const WlTable &t, int &job, int &stage, uint32_t &v, uint32_t &task)
{
    const uint64_t t_end = global_ns() + kWlWaitNs;
    const uint32_t *ring = t.ctr + 8 + t.ring;
    for (;;) {
        if (ld_acquire_u32(t.ctr + 1)) return false;
        const uint32_t r = ld_acquire_u32(t.ctr + 3), w = ld_acquire_u32(t.ctr + 2);
        if (r < w) {
            if (atomicCAS(t.ctr + 3, r, r + 1) == r) {
                // slot r was reserved by the CTA that hands the task on; it writes it next
                uint32_t x;
                while ((x = ld_acquire_u32(ring + r)) == 0) {
                    if (global_ns() > t_end) {
                        atomicExch(t.job[0].a.err, kErrTimeout);
                        atomicExch(t.ctr + 1, 1u);
                        return false;
                    }
                    __nanosleep(32);
                }
                task = x - 1;
                wl_decode(t, task, job, stage, v);
                return true;
            }
            continue;
        }
        if (ld_acquire_u32(t.ctr) < t.ntasks) {
            const uint32_t h = atomicAdd(t.ctr, 1u);
            if (h < t.ntasks) {
                atomicAdd(t.ctr + 4, 1u);
                task = h;
                wl_decode(t, h, job, stage, v);
                return true;
            }
        }
        // the queue is exhausted: done once every claim is resolved and every handed-on task taken
        if (ld_acquire_u32(t.ctr + 4) >= t.ntasks && ld_acquire_u32(t.ctr + 3) >= ld_acquire_u32(t.ctr + 2))
            return false;
        if (global_ns() > t_end) {
            atomicExch(t.job[0].a.err, kErrTimeout);
            atomicExch(t.ctr + 1, 1u);
            return false;
        }
        __nanosleep(256);
    }
}

// The work-list kernel.  A fresh CTA takes a handed-on task or the next one in
// the queue, then keeps claiming tasks while they are of the same kind (stage,
// and for stage B the body), and leaves when it claims one of another kind,
// handing it on through the ring.  The grid has one CTA per task, more than
// can ever be needed (each CTA's first task is one no other CTA took first),
// so a fresh CTA always takes the place of one that left.  Every claim is a
// fetch-and-add on the queue head, so claims do not serialise.  Each kind's
// loop is a branch of its own, not one loop over all the bodies: the bodies use
// nearly all 255 registers, and one loop around all of them makes the register
// allocator spill inside them.
//
// No deadlock: a task's dependencies are earlier in the queue, so they were
// claimed before it; a claimed task runs on its claiming CTA or waits in the
// ring, and every hand-on is followed by the handing CTA leaving, which lets a
// fresh CTA, which takes handed-on tasks first, start.
template <int N, int FMT>
__global__ void __launch_bounds__(kRows *NPipes<N, FMT>::A, 1) k_worklist(const __grid_constant__ WlTable t)
{
    constexpr int NP = NPipes<N, FMT>::A;
    static_assert(NP == NPipes<N, FMT>::B && NP == NPipes<N, FMT>::C, "one pipeline count for every stage");
    __shared__ uint32_t s_tm;
    __shared__ int s_job, s_stage;
    __shared__ uint32_t s_v;
    // thread 0 takes a task (of stage `want`, or any when want < 0) and waits
    // for its dependencies; every thread returns its stage, or -1
    __shared__ uint32_t s_task;
    // want < 0: a fresh CTA's first task; else the next task of this kind
    auto next = [&](int want, int want_share) -> int {
        // the previous task's generic shared-memory writes before the next
        // task's bulk copies into the same bytes
        fence_proxy_async();
        if (threadIdx.x == 0) {
            int job = -1, stage = -1;
            uint32_t v = 0, task = 0;
            const bool got = want < 0 ? wl_claim_first(t, job, stage, v, task)
                                      : wl_claim_same(t, want, want_share, job, stage, v, task);
            if (!got) stage = -1;
            if (got) {
                const uint64_t t0 = t.trace ? global_ns() : 0;
                const bool ready = wl_deps<NP>(t, job, stage, v);
                if (t.trace && task < t.trace_cap) {
                    uint32_t smid;
                    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
                    t.trace[4 * task] = t0;
                    t.trace[4 * task + 1] = global_ns();
                    t.trace[4 * task + 3] = (unsigned long long)(smid << 8 | (uint32_t)stage);
                }
                s_task = task;
                if (ready) {
                    __threadfence();
                } else {
                    atomicExch(t.job[job].a.err, kErrTimeout);
                    atomicExch(t.ctr + 1, 1u);
                    stage = -1;
                }
            }
            s_job = job;
            s_stage = stage;
            s_v = v;
        }
        __syncthreads();
        return s_stage;
    };
    // thread 0: publish a finished task (or abort the launch)
    auto done = [&](bool ok, int stage) {
        if (threadIdx.x == 0) {
            if (t.trace && s_task < t.trace_cap) t.trace[4 * s_task + 2] = global_ns();
            if (ok) {
                __threadfence();
                wl_done<NP>(t, s_job, stage, s_v);
            } else {
                atomicExch(t.ctr + 1, 1u);
            }
        }
    };
    const int first = next(-1, -1);
    if (first < 0) return;
    const bool share = t.job[s_job].bmap != nullptr;
    if (threadIdx.x < 32) tmem_alloc(&s_tm, 512);
    fence_before();
    __syncthreads();
    fence_after();
    const Persist ps{s_tm};
    if (first == WL_A) {
        for (int st = first; st == WL_A; st = next(WL_A, -1)) {
            const WlJob &J = t.job[s_job];
            const uint32_t v = s_v, r = v / J.ga;
            done(k_stage_a_body<N, FMT>(J.a, make_uint3(v % J.ga, r / J.sides, r % J.sides),
                                        make_uint3(J.ga, J.a.RS, J.sides), &ps),
                 WL_A);
        }
    } else if (first == WL_B && share) {
        for (int st = first; st == WL_B; st = next(WL_B, 1)) {
            const WlJob &J = t.job[s_job];
            const uint32_t v = s_v;
            done(k_stage_b_body<N, FMT, false, true>(J.a, make_uint3(v % J.gb, v / J.gb, 0),
                                                     make_uint3(J.gb, J.a.RS, 1), J.bmap, &ps),
                 WL_B);
        }
    } else if (first == WL_B) {
        for (int st = first; st == WL_B; st = next(WL_B, 0)) {
            const WlJob &J = t.job[s_job];
            const uint32_t v = s_v;
            done(k_stage_b_body<N, FMT>(J.a, make_uint3(v % J.gb, v / J.gb, 0), make_uint3(J.gb, J.a.RS, 1),
                                        nullptr, &ps),
                 WL_B);
        }
    } else if (first == WL_C) {
        for (int st = first; st == WL_C; st = next(WL_C, -1)) {
            const WlJob &J = t.job[s_job];
            const uint32_t v = s_v, r = v / J.ngc;
            done(k_stage_c_body<N, FMT>(J.a, make_uint3(v % J.ngc, r / J.ec, r % J.ec),
                                        make_uint3(J.ngc, J.gyc, J.ec), &ps),
                 WL_C);
        }
    } else {
        for (int st = first; st == WL_S; st = next(WL_S, -1)) {
            const WlJob &J = t.job[s_job];
            const long total = (long)J.ec * J.a.n, lo = (long)s_v * kWlSumChunk;
            const long hi = min(total, lo + kWlSumChunk);
            for (long i = lo + threadIdx.x; i < hi; i += blockDim.x)
                sum_partial(J.qg, J.a.QGp, J.a.rsb, J.a.n, J.a.pt0, i);
            __syncthreads();
            done(true, WL_S);
        }
    }
    fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tmem_dealloc(s_tm, 512);
}

// ------------------------------------------------------ table preparation
// T_d[j][j'] = (1/N) sum_l exp(2 pi i l (j - j') / N) phi_d(l), written into
// pre-swizzled B-operand images (terms IMGC apart): z (real input) rows 2j,
// 2j+1, K = j'; y, x (complex input) the real 2x2 block [Re -Im; Im Re] at
// K = 2j', 2j'+1.
template <int FMT>
__global__ void k_timg(uint8_t *out, const double2 *phase, int N, int RS)
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
    const int NO = 2 * N;
    const long IC = tcfmt::img_c<FMT>(N);
    uint8_t *img = out + (((long)rs * 2 + side) * 3 + ax) * Fmt<FMT>::NT * IC;
    if (ax == 2) {
        tcfmt::put_img<FMT>(img, IC, 2 * j, jp, NO, tr);
        tcfmt::put_img<FMT>(img, IC, 2 * j + 1, jp, NO, ti);
    } else {
        tcfmt::put_img<FMT>(img, IC, 2 * j, 2 * jp, NO, tr);
        tcfmt::put_img<FMT>(img, IC, 2 * j, 2 * jp + 1, NO, -ti);
        tcfmt::put_img<FMT>(img, IC, 2 * j + 1, 2 * jp, NO, ti);
        tcfmt::put_img<FMT>(img, IC, 2 * j + 1, 2 * jp + 1, NO, tr);
    }
}

// Hermitian form: T_z of every (r, s) and side as a complex-input image (the
// real 2x2 block [Re -Im; Im Re] at K = 2j', 2j'+1), out [RS][2 sides][terms][IMGC]
template <int FMT>
__global__ void k_timg_zc(uint8_t *out, const double2 *phase, int N, int RS)
{
    const long total = (long)RS * 2 * N * N;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int jp = (int)(i % N), j = (int)((i / N) % N), side = (int)((i / ((long)N * N)) % 2);
    const int rs = (int)(i / (2L * N * N));
    const double2 *ph = phase + ((long)rs * 6 + side * 3 + 2) * N;
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
    const int NO = 2 * N;
    const long IC = tcfmt::img_c<FMT>(N);
    uint8_t *img = out + ((long)rs * 2 + side) * Fmt<FMT>::NT * IC;
    tcfmt::put_img<FMT>(img, IC, 2 * j, 2 * jp, NO, tr);
    tcfmt::put_img<FMT>(img, IC, 2 * j, 2 * jp + 1, NO, -ti);
    tcfmt::put_img<FMT>(img, IC, 2 * j + 1, 2 * jp, NO, ti);
    tcfmt::put_img<FMT>(img, IC, 2 * j + 1, 2 * jp + 1, NO, tr);
}

// forward DFT F[k][j] = exp(-2 pi i jk/N) as pre-swizzled complex-input images
template <int FMT>
__global__ void k_fimg(uint8_t *out, int N)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * N) return;
    const int j = i % N, k = i / N;
    double s, c;
    sincospi(2.0 * ((j * k) % N) / N, &s, &c);
    const double fr = c, fi = -s;
    const int NO = 2 * N;
    const long IC = tcfmt::img_c<FMT>(N);
    tcfmt::put_img<FMT>(out, IC, 2 * k, 2 * j, NO, fr);
    tcfmt::put_img<FMT>(out, IC, 2 * k, 2 * j + 1, NO, -fi);
    tcfmt::put_img<FMT>(out, IC, 2 * k + 1, 2 * j, NO, fi);
    tcfmt::put_img<FMT>(out, IC, 2 * k + 1, 2 * j + 1, NO, fr);
}

__global__ void k_to_f32(float2 *dst, const double2 *src, long count)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}

// Workspace of the Hermitian form (dgfs_plan_set_hermitian), per plan:
//   ft [maxP][S][n] float (f~) | Z2 [S*S][Ps_max][n] float4 | zimg [S*S][RS][2][terms][IMGC]
struct HermWs {
    float *ft;
    float4 *z2;
    long z2_stride;
    uint8_t *zimg;
    long zimg_pair;  // bytes per pair
};

template <int FMT> long zimg_pair_bytes(const dgfs_plan_s *plan)
{
    return (long)plan->Nrho * plan->M * 2 * Fmt<FMT>::NT * tcfmt::img_c<FMT>(plan->N);
}

HermWs herm_ws_of(const dgfs_plan_s *plan)
{
    const TcState *ts = reinterpret_cast<const TcState *>(plan->tc);
    const long n = (long)plan->N * plan->N * plan->N;
    const long Psmax = (plan->max_points + 1) / 2;
    HermWs h;
    h.ft = reinterpret_cast<float *>(plan->herm_ws);
    h.z2 = reinterpret_cast<float4 *>(h.ft + (long)plan->max_points * plan->S * n);
    h.z2_stride = Psmax * n;
    h.zimg = reinterpret_cast<uint8_t *>(h.z2 + (long)plan->S * plan->S * h.z2_stride);
    h.zimg_pair = ts->fmt == 0 ? zimg_pair_bytes<0>(plan) : zimg_pair_bytes<1>(plan);
    return h;
}


// -------------------------------------------------- work list (host)
// N with one pipeline count for stages A, B and C (the work-list kernel runs
// all three bodies in one CTA shape)
bool wl_supported(int N) { return N == 24 || N == 32 || N == 48; }

// One job of a schedule.
struct WlSpec {
    TcArgs a;
    float4 *qg;
    const uint16_t *bmap;
    const void *key;  // the plan: jobs with one key reuse one workspace
    dim3 gA, gB, gC;
    int M;
};

template <int N, int FMT>
WlSpec wl_spec(const dgfs_plan_s *plan, const void *f, int p, int q, int pt0, int Ec)
{
    const TcWs w = ws_of(plan);
    WlSpec s;
    s.a = job_args(plan, f, p, q, pt0, Ec);
    const Share sh = job_share(plan, p, q);
    s.bmap = sh.on ? sh.bmap : nullptr;
    s.qg = w.QG + (p * plan->S + q) * w.qg_stride;
    s.key = plan;
    s.M = plan->M;
    job_grids<N, FMT>(plan, Ec, sh.on, s.gA, s.gB, s.gC);
    return s;
}

// Counter words of the work list's launches for jobs of RS (r, s) and gyc stage C grid rows.
// task trace of the work-list launches (dgfs_debug_worklist_trace); off when null
unsigned long long *g_wl_trace = nullptr;
uint32_t g_wl_trace_cap = 0;
// (r, s) per wave of the work-list queue (dgfs_debug_worklist_chunk)
int g_wl_chunk = 48;

// Counter words of a work-list launch: the control words, the jobs'
// counters and one ring slot per task.
size_t wl_words_for(int RS, int gyc, size_t tasks) { return 8 + (size_t)kWlJobs * (2 * RS + 2 * gyc + 2) + tasks; }

// An upper bound of the tasks of one job of a plan over every launch
// configuration the autotuner tries (CTA groups for up to 16 waves, chunks of
// up to chunk_max points, up to rsb_max (r, s)-blocks).
size_t wl_job_tasks_max(const dgfs_plan_s *plan, int sms, int chunk_max, int rsb_max)
{
    const long RS = (long)plan->Nrho * plan->M, N = plan->N, n = N * N * N;
    const long ga = std::max(1L, (16L * sms + RS) / (2 * RS)), gb = std::max(1L, (16L * sms + RS / 2) / RS);
    const long G = kRows / N, ngc = (N + G - 1) / G;
    return (size_t)(2 * RS * ga + RS * gb + ngc * rsb_max * chunk_max + (chunk_max * n + kWlSumChunk - 1) / kWlSumChunk);
}

// Queue the jobs of `rounds` (a round holds at most one job per plan) into
// work-list launches.  Within a round the tasks go in waves over chunks of
// about twelve (r, s) (whole radial nodes): wave c holds stage A of chunk c,
// stage B of chunk c - 2 and stage C of every grid row whose (r, s) had their
// stage B queued in an earlier wave; the partial sums of a round follow at
// wave 2 of the next round.  Every task's dependencies are queued before it.
// Returns false if a launch's tables cannot hold one job.
bool wl_build(const std::vector<std::vector<WlSpec>> &rounds, int npc, uint32_t *ctr, std::vector<WlTable> &L,
              std::vector<uint32_t> &words, int chunk = g_wl_chunk)
{
    constexpr int LAG = 2;
    L.clear();
    words.clear();
    bool open = false, fits = true;
    uint32_t nw = 0;
    int nj = 0;
    std::vector<std::pair<const void *, int>> last;  // plan -> its latest job in the open launch
    std::vector<int> pend;                           // jobs whose partial sums are not queued yet
    auto T = [&]() -> WlTable & { return L.back(); };
    auto seg = [&](int j, int stage, uint32_t v0, uint32_t cnt) {
        if (!cnt) return;
        WlTable &t = T();
        if (t.nseg >= kWlSegs || v0 >= (1u << 18) || j > 0xFFF) {
            fits = false;
            return;
        }
        t.seg[t.nseg++] = make_uint2(t.ntasks, (uint32_t)j | ((uint32_t)stage << 12) | (v0 << 14));
        t.ntasks += cnt;
    };
    auto close = [&] {
        if (!open) return;
        for (int j : pend) seg(j, WL_S, 0, T().job[j].ns);
        pend.clear();
        T().ring = nw;
        words.push_back(8 + nw + T().ntasks);
        open = false;
    };
    auto start = [&] {
        L.emplace_back();
        memset(&L.back(), 0, sizeof(WlTable));
        L.back().ctr = ctr;
        nw = 0;
        nj = 0;
        last.clear();
        open = true;
    };
    auto chunk_rs = [chunk](const WlSpec &s) { return s.M * std::max(1, (chunk + s.M - 1) / s.M); };
    auto nchunks = [&](const WlSpec &s) { return (s.a.RS + chunk_rs(s) - 1) / chunk_rs(s); };
    auto est = [&](const WlSpec &s) { return 2 * nchunks(s) + (int)s.gC.y + 1; };
    // rs range of stage C grid row g, as wl_grange on the device
    auto grange_hi = [&](const TcArgs &a, int g) {
        return std::min(a.RS, std::min(a.rsb, (g + 1) * npc) * a.rs_per_block);
    };
    for (const auto &round : rounds) {
        size_t r0 = 0;
        while (r0 < round.size()) {
            if (!open) start();
            int segs = T().nseg + (int)pend.size();
            size_t r1 = r0;
            while (r1 < round.size() && nj + (int)(r1 - r0) < kWlJobs && segs + est(round[r1]) <= kWlSegs)
                segs += est(round[r1++]);
            if (r1 == r0) {
                if (nj == 0) return false;
                close();
                continue;
            }
            std::vector<int> idx;
            for (size_t i = r0; i < r1; ++i) {
                const WlSpec &s = round[i];
                WlJob &J = T().job[nj];
                J.a = s.a;
                J.qg = s.qg;
                J.bmap = s.bmap;
                J.prev = -1;
                for (auto &kv : last)
                    if (kv.first == s.key) J.prev = kv.second;
                J.cnt = nw;
                nw += 2u * s.a.RS + 2u * s.gC.y + 2u;
                J.ga = (uint16_t)s.gA.x;
                J.sides = (uint16_t)s.gA.z;
                J.gb = (uint16_t)s.gB.x;
                J.ngc = (uint16_t)s.gC.x;
                J.gyc = (uint16_t)s.gC.y;
                J.ec = (uint16_t)s.gC.z;
                J.ns = (uint32_t)(((long)J.ec * s.a.n + kWlSumChunk - 1) / kWlSumChunk);
                idx.push_back(nj++);
            }
            int maxch = 0;
            std::vector<int> gnext(idx.size(), 0);
            for (size_t i = r0; i < r1; ++i) maxch = std::max(maxch, nchunks(round[i]));
            for (int c = 0; c <= maxch + LAG; ++c) {
                for (size_t k = 0; k < idx.size(); ++k) {
                    const WlSpec &s = round[r0 + k];
                    const WlJob &J = T().job[idx[k]];
                    const int RC = chunk_rs(s), lo = c * RC, hi = std::min(s.a.RS, lo + RC);
                    if (c < nchunks(s)) seg(idx[k], WL_A, (uint32_t)lo * J.sides * J.ga, (uint32_t)(hi - lo) * J.sides * J.ga);
                }
                if (c == LAG) {
                    for (int j : pend) seg(j, WL_S, 0, T().job[j].ns);
                    pend.clear();
                }
                // stage B of the jobs that compute both sides, then of those
                // that read B' from A' (one stage B body per run of tasks)
                for (int kind = 0; kind < 2; ++kind)
                    for (size_t k = 0; k < idx.size(); ++k) {
                        const WlSpec &s = round[r0 + k];
                        const WlJob &J = T().job[idx[k]];
                        const int RC = chunk_rs(s), cb = c - LAG;
                        if ((s.bmap != nullptr) == (kind == 1) && cb >= 0 && cb < nchunks(s)) {
                            const int lo = cb * RC, hi = std::min(s.a.RS, lo + RC);
                            seg(idx[k], WL_B, (uint32_t)lo * J.gb, (uint32_t)(hi - lo) * J.gb);
                        }
                    }
                for (size_t k = 0; k < idx.size(); ++k) {
                    const WlSpec &s = round[r0 + k];
                    const WlJob &J = T().job[idx[k]];
                    const int RC = chunk_rs(s);
                    // stage C rows whose stage B was queued in earlier waves
                    const long lim = (long)(c - LAG) * RC;
                    while (c > LAG && gnext[k] < (int)J.gyc && grange_hi(s.a, gnext[k]) <= lim) {
                        seg(idx[k], WL_C, (uint32_t)gnext[k] * J.ec * J.ngc, (uint32_t)J.ec * J.ngc);
                        ++gnext[k];
                    }
                }
            }
            for (size_t k = 0; k < idx.size(); ++k) {
                bool found = false;
                for (auto &kv : last)
                    if (kv.first == round[r0 + k].key) {
                        kv.second = idx[k];
                        found = true;
                    }
                if (!found) last.emplace_back(round[r0 + k].key, idx[k]);
                pend.push_back(idx[k]);
            }
            r0 = r1;
        }
    }
    close();
    return fits;
}


template <int N, int FMT> constexpr size_t wl_smem()
{
    using SM = Smem<N, FMT>;
    return std::max(SM::A, std::max(SM::B, SM::C));
}

template <int N, int FMT>
dgfs_status wl_launch(dgfs_plan_s *plan, const std::vector<WlTable> &L, const std::vector<uint32_t> &words, int sms,
                      cudaStream_t st)
{
    for (size_t l = 0; l < L.size(); ++l) {
        if (!L[l].ntasks) continue;
        DGFS_CUDA(cudaMemsetAsync(L[l].ctr, 0, sizeof(uint32_t) * words[l], st));
        const unsigned grid = L[l].ntasks;  // one CTA per task at most (see k_worklist)
        {
            ProfScope ps(plan, "tc_worklist", st);
            if (g_wl_trace) {
                WlTable tt = L[l];
                tt.trace = g_wl_trace;
                tt.trace_cap = g_wl_trace_cap;
                k_worklist<N, FMT><<<grid, kRows * NPipes<N, FMT>::A, wl_smem<N, FMT>(), st>>>(tt);
            } else {
                k_worklist<N, FMT><<<grid, kRows * NPipes<N, FMT>::A, wl_smem<N, FMT>(), st>>>(L[l]);
            }
        }
        DGFS_LAUNCHED(plan);
    }
    return DGFS_OK;
}

// A plain call as one work-list launch (TcState::sched = 1).  The jobs
// (species pair, chunk of points) share the plan's workspace, so each is a
// round of its own; the dependencies let the next job's stage A start as soon
// as the current job's stage B has read the grids it overwrites.
template <int N, int FMT>
dgfs_status collide_wl(dgfs_plan_s *plan, int P, const void *f, void *Qout, cudaStream_t st)
{
    TcState *ts = reinterpret_cast<TcState *>(plan->tc);
    const TcWs w = ws_of(plan);
    std::vector<std::vector<WlSpec>> rounds;
    for (int p = 0; p < plan->S; ++p)
        for (int q = 0; q < plan->S; ++q)
            for (int pt0 = 0; pt0 < P; pt0 += ts->chunk)
                rounds.push_back({wl_spec<N, FMT>(plan, f, p, q, pt0, std::min(ts->chunk, P - pt0))});
    std::vector<WlTable> L;
    std::vector<uint32_t> words;
    if (!wl_build(rounds, NPipes<N, FMT>::C, ts->wl_ctr, L, words)) {
        set_error("dgfs_collide: the work list cannot hold this plan's jobs");
        return DGFS_EUNSUPPORTED;
    }
    for (uint32_t wd : words)
        if (wd > ts->wl_words) {
            set_error("dgfs_collide: work-list counters exceed their buffer");
            return DGFS_EUNSUPPORTED;
        }
    DGFS_TRY(df_forward(plan, P, reinterpret_cast<const float *>(f), w.F, ts->tw_df, st));
    DGFS_TRY((wl_launch<N, FMT>(plan, L, words, ts->sms, st)));
    return df_finish(plan, P, w.QG, w.qg_stride, w.F, reinterpret_cast<const float *>(f),
                     reinterpret_cast<float *>(Qout), ts->tw_df, st);
}

template <int N, int FMT>
dgfs_status collide_n(dgfs_plan_s *plan, int P, const void *f, void *Qout, cudaStream_t st)
{
    using SM = Smem<N, FMT>;
    TcState *ts = reinterpret_cast<TcState *>(plan->tc);
    if constexpr (N == 24 || N == 32 || N == 48)
        if (ts->sched == 1) return collide_wl<N, FMT>(plan, P, f, Qout, st);
    const int S = plan->S;
    const long n = (long)N * N * N;
    const int E = ts->chunk, RSB = rs_blocks(plan);
    const TcWs w = ws_of(plan);

    // Stage A runs on the plan's side stream: job k's stage A waits for job
    // k-1's stage B (the last reader of A', B'), so it overlaps job k-1's
    // stage C; stage B waits for stage A.  With H double-buffered (hslots 2),
    // stage B runs on a third stream and waits only for its stage A and for
    // the stage C two jobs back (the last reader of its H slot), so that job
    // k's stage B also runs beside job k-1's stage C; stage C and the partial
    // sums stay on the caller's stream.  The first stage A waits for the
    // caller's stream at entry, and every side-stream launch is joined back
    // through the stage C that consumes it (graph capture sees a closed fork).
    // (serial when the plan's per-kernel profiler is on, so that every kernel's
    // event-bracketed time is its own)
    cudaStream_t sa = plan->prof ? st : ts->side;
    const bool fork = sa != st;
    const int nh = fork ? ts->hslots : 1;
    cudaStream_t sb = nh == 2 ? ts->side_b : st;
    float2 *const Hslot[2] = {w.H, w.H2};
    if (fork) DGFS_CUDA(cudaEventRecord(ts->ev_entry, st));
    int job = 0;
    // forward transforms of f for the loss term (step 1 of Algorithm 2)
    DGFS_TRY(df_forward(plan, P, reinterpret_cast<const float *>(f), w.F, ts->tw_df, st));
    for (int p = 0; p < S; ++p)
        for (int q = 0; q < S; ++q) {
            for (int pt0 = 0; pt0 < P; pt0 += E, ++job) {
                const int Ec = std::min(E, P - pt0);
                TcArgs a = job_args(plan, f, p, q, pt0, Ec);
                a.H = Hslot[job % nh];
                const Share sh = job_share(plan, p, q);
                dim3 gA, gB, gC;
                job_grids<N, FMT>(plan, Ec, sh.on, gA, gB, gC);
                if (fork) DGFS_CUDA(cudaStreamWaitEvent(sa, job == 0 ? ts->ev_entry : ts->ev_b, 0));
                {
                    ProfScope ps(plan, "tc_stage_a", sa);
                    if (WsA<N, FMT>::OK && ts->ws_a == 1)
                        k_stage_a_ws<N, FMT><<<gA, 4 * kRows, WsA<N, FMT>::BYTES, sa>>>(a);
                    else if (A2<N, FMT>::OK && ts->ws_a == 2)
                        k_stage_a2<N, FMT><<<gA, 2 * kRows * NPipes<N, FMT>::A, SM::A, sa>>>(a);
                    else
                        k_stage_a<N, FMT><<<gA, kRows * NPipes<N, FMT>::A, SM::A, sa>>>(a);
                }
                DGFS_LAUNCHED(plan);
                if (fork) {
                    DGFS_CUDA(cudaEventRecord(ts->ev_a, sa));
                    DGFS_CUDA(cudaStreamWaitEvent(sb, ts->ev_a, 0));
                }
                if (nh == 2 && job >= 2) DGFS_CUDA(cudaStreamWaitEvent(sb, ts->ev_c[job % 2], 0));
                {
                    ProfScope ps(plan, "tc_stage_b", sb);
                    if (sh.on)
                        k_stage_b_share<N, FMT, false><<<gB, kRows * NPipes<N, FMT>::B, SM::B, sb>>>(a, sh.bmap);
                    else
                        k_stage_b<N, FMT><<<gB, kRows * NPipes<N, FMT>::B, SM::B, sb>>>(a);
                }
                DGFS_LAUNCHED(plan);
                if (fork) DGFS_CUDA(cudaEventRecord(ts->ev_b, sb));
                if (nh == 2) DGFS_CUDA(cudaStreamWaitEvent(st, ts->ev_b, 0));
                {
                    ProfScope ps(plan, "tc_stage_c", st);
                    k_stage_c<N, FMT><<<gC, kRows * NPipes<N, FMT>::C, SM::C, st>>>(a);
                }
                DGFS_LAUNCHED(plan);
                {
                    ProfScope ps(plan, "tc_sum_partials", st);
                    k_sum_partials<<<nblk((long)Ec * n, 256), 256, 0, st>>>(w.QG + (p * S + q) * w.qg_stride,
                                                                           w.QGp, RSB, n, pt0, Ec);
                }
                DGFS_LAUNCHED(plan);
                if (nh == 2) DGFS_CUDA(cudaEventRecord(ts->ev_c[job % 2], st));
            }
        }
    // step 10 for every pair and point
    return df_finish(plan, P, w.QG, w.qg_stride, w.F, reinterpret_cast<const float *>(f),
                     reinterpret_cast<float *>(Qout), ts->tw_df, st);
}

// Hermitian form (declared variant, dgfs_plan_set_hermitian): Algorithm 2
// with the Nyquist planes removed.  Every translate is then real, so a grid
// slot carries two points, point 2e as the real part and 2e + 1 as the
// imaginary part, and each (r, s) step serves both: the stage kernels run
// over ceil(P/2) slots.  Stage A packs the two Nyquist-free inputs into its
// complex z-pass, stage B multiplies the two real translates of each point
// separately, stage C and the partial sums are unchanged; the finish removes
// the gain's Nyquist planes and separates the two points.
template <int N, int FMT>
dgfs_status collide_herm_n(dgfs_plan_s *plan, int P, const void *f, void *Qout, cudaStream_t st)
{
    using SM = Smem<N, FMT>;
    TcState *ts = reinterpret_cast<TcState *>(plan->tc);
    const int S = plan->S;
    const long n = (long)N * N * N;
    const int E = ts->chunk, RSB = rs_blocks(plan), Ps = (P + 1) / 2;
    const TcWs w = ws_of(plan);
    const HermWs h = herm_ws_of(plan);
    constexpr int NT = Fmt<FMT>::NT;
    constexpr size_t smem_a = SM::A + (size_t)NT * (tcfmt::img_c<FMT>(N) - tcfmt::img_r<FMT>(N));
    cudaStream_t sa = plan->prof ? st : ts->side;
    const bool fork = sa != st;
    bool first = true;
    // F = fft3(f), projected; f~ = ifft3(P F) (the QG region is free until the first partial sum)
    DGFS_TRY(df_forward(plan, P, reinterpret_cast<const float *>(f), w.F, ts->tw_df, st));
    DGFS_TRY(df_herm_prepare(plan, P, w.F, w.QG, h.ft, ts->tw_df, st));
    // the side stream's first stage A reads f~: fork after it is written
    if (fork) DGFS_CUDA(cudaEventRecord(ts->ev_entry, st));
    for (int p = 0; p < S; ++p)
        for (int q = 0; q < S; ++q) {
            for (int pt0 = 0; pt0 < Ps; pt0 += E) {
                const int Ec = std::min(E, Ps - pt0);
                TcArgs a = job_args(plan, h.ft, p, q, pt0, Ec);
                const Share sh = job_share(plan, p, q);
                a.herm = 1;
                a.npts = P;
                a.zimg = h.zimg + (long)(p * S + q) * h.zimg_pair;
                dim3 gA, gB, gC;
                job_grids<N, FMT>(plan, Ec, sh.on, gA, gB, gC);
                if (fork) DGFS_CUDA(cudaStreamWaitEvent(sa, first ? ts->ev_entry : ts->ev_b, 0));
                first = false;
                {
                    ProfScope ps(plan, "tc_stage_a", sa);
                    k_stage_a_herm<N, FMT><<<gA, kRows * NPipes<N, FMT>::A, smem_a, sa>>>(a);
                }
                DGFS_LAUNCHED(plan);
                if (fork) {
                    DGFS_CUDA(cudaEventRecord(ts->ev_a, sa));
                    DGFS_CUDA(cudaStreamWaitEvent(st, ts->ev_a, 0));
                }
                {
                    ProfScope ps(plan, "tc_stage_b", st);
                    if (sh.on)
                        k_stage_b_share<N, FMT, true><<<gB, kRows * NPipes<N, FMT>::B, SM::B, st>>>(a, sh.bmap);
                    else
                        k_stage_b_herm<N, FMT><<<gB, kRows * NPipes<N, FMT>::B, SM::B, st>>>(a);
                }
                DGFS_LAUNCHED(plan);
                if (fork) DGFS_CUDA(cudaEventRecord(ts->ev_b, st));
                {
                    ProfScope ps(plan, "tc_stage_c", st);
                    k_stage_c<N, FMT><<<gC, kRows * NPipes<N, FMT>::C, SM::C, st>>>(a);
                }
                DGFS_LAUNCHED(plan);
                {
                    ProfScope ps(plan, "tc_sum_partials", st);
                    k_sum_partials<<<nblk((long)Ec * n, 256), 256, 0, st>>>(w.QG + (p * S + q) * w.qg_stride,
                                                                           w.QGp, RSB, n, pt0, Ec);
                }
                DGFS_LAUNCHED(plan);
            }
        }
    return df_herm_finish(plan, P, w.QG, w.qg_stride, h.z2, h.z2_stride, w.F, h.ft, reinterpret_cast<float *>(Qout),
                          ts->tw_df, st);
}

template <int N, int FMT>
dgfs_status set_smem_attrs()
{
    using SM = Smem<N, FMT>;
    DGFS_CUDA(cudaFuncSetAttribute(k_stage_a<N, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::A));
    if constexpr (WsA<N, FMT>::OK)
        DGFS_CUDA(cudaFuncSetAttribute(k_stage_a_ws<N, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)WsA<N, FMT>::BYTES));
    if constexpr (A2<N, FMT>::OK)
        DGFS_CUDA(cudaFuncSetAttribute(k_stage_a2<N, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::A));
    DGFS_CUDA(cudaFuncSetAttribute(k_stage_b<N, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::B));
    DGFS_CUDA(cudaFuncSetAttribute(k_stage_b_share<N, FMT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)SM::B));
    DGFS_CUDA(cudaFuncSetAttribute(k_stage_c<N, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::C));
    if constexpr (N <= 32) {
        DGFS_CUDA(cudaFuncSetAttribute(k_stage_a_herm<N, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(SM::A + (size_t)Fmt<FMT>::NT *
                                                         (tcfmt::img_c<FMT>(N) - tcfmt::img_r<FMT>(N)))));
        DGFS_CUDA(cudaFuncSetAttribute(k_stage_b_herm<N, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::B));
        DGFS_CUDA(cudaFuncSetAttribute(k_stage_b_share<N, FMT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SM::B));
    }
    DGFS_CUDA(cudaFuncSetAttribute(k_stage_a_batch<N, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::A));
    DGFS_CUDA(cudaFuncSetAttribute(k_stage_b_batch<N, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::B));
    DGFS_CUDA(cudaFuncSetAttribute(k_stage_c_batch<N, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::C));
    if constexpr (N == 24 || N == 32 || N == 48)
        DGFS_CUDA(cudaFuncSetAttribute(k_worklist<N, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)wl_smem<N, FMT>()));
    return DGFS_OK;
}

// ------------------------------------------------------------ batches
// A batch holds, per (N, operand format) group of tensor-core plans, rounds of
// jobs: round k runs the k-th job (species pair, chunk of points) of every
// plan of the group, each stage as one launch over all of them.  The FP64
// forward transforms, partial sums and finishing passes stay per plan; the
// finishing passes run once per plan after the last round.
struct BatchJob {
    dgfs_plan_s *plan;
    int p, q, pt0, Ec, P;
    const void *f;
    void *Q;
};

struct BatchRound {
    std::vector<BatchJob> jobs;
    // per launch of at most kJobsPerLaunch jobs: the tables of stages A, B, C
    std::vector<JobTable> tabs;
    std::vector<uint32_t> ctas;
};

struct BatchGroup {
    int N = 0, fmt = 0;
    std::vector<BatchRound> rounds;
};

template <int N, int FMT>
dgfs_status round_build(BatchRound &r)
{
    const int nj = (int)r.jobs.size();
    for (int j0 = 0; j0 < nj; j0 += kJobsPerLaunch) {
        const int cnt = std::min(kJobsPerLaunch, nj - j0);
        JobTable t[3];
        uint32_t c[3] = {0, 0, 0};
        for (int k = 0; k < 3; ++k) {
            memset(&t[k], 0, sizeof(JobTable));
            t[k].njobs = cnt;
        }
        for (int j = 0; j < cnt; ++j) {
            const BatchJob &b = r.jobs[j0 + j];
            // the batched work list computes both sides of every pair
            const TcArgs a = job_args(b.plan, b.f, b.p, b.q, b.pt0, b.Ec);
            dim3 g[3];
            job_grids<N, FMT>(b.plan, b.Ec, false, g[0], g[1], g[2]);
            for (int k = 0; k < 3; ++k) {
                t[k].job[j] = a;
                t[k].grid[j] = JobGrid{c[k], g[k].x, g[k].y, g[k].z};
                c[k] += g[k].x * g[k].y * g[k].z;
            }
        }
        for (int k = 0; k < 3; ++k) {
            r.tabs.push_back(t[k]);
            r.ctas.push_back(c[k]);
        }
    }
    return DGFS_OK;
}

// Stage A of a launch on a side stream, as in collide_n: it waits for the
// previous launch's stage B (the last reader of A', B'), so it overlaps that
// launch's stage C; stage B waits for it.
struct Fork {
    cudaStream_t sa;
    cudaEvent_t ev_entry, ev_a, ev_b;
    bool on, first;
};

template <int N, int FMT>
dgfs_status round_launch(const BatchRound &r, cudaStream_t st, Fork &fk)
{
    using SM = Smem<N, FMT>;
    dgfs_plan_s *lead = r.jobs[0].plan;  // launch counting and profiling
    const cudaStream_t sa = fk.on ? fk.sa : st;
    // N = 8: each job's own stage kernels instead of the job-table kernels (the
    // N = 8 job-table stage B kernel disagreed with the plain kernel on the same
    // job in some builds; see the design notes)
    constexpr bool per_job = N == 8;
    auto grid_of = [](const JobGrid &g) { return dim3(g.gx, g.gy, g.gz); };
    for (size_t l = 0; l < r.tabs.size(); l += 3) {
        const int nj = r.tabs[l].njobs;
        if (fk.on) DGFS_CUDA(cudaStreamWaitEvent(sa, fk.first ? fk.ev_entry : fk.ev_b, 0));
        fk.first = false;
        {
            ProfScope ps(lead, "tc_stage_a", sa);
            if (per_job)
                for (int j = 0; j < nj; ++j)
                    k_stage_a<N, FMT><<<grid_of(r.tabs[l].grid[j]), kRows * NPipes<N, FMT>::A, SM::A, sa>>>(
                        r.tabs[l].job[j]);
            else
                k_stage_a_batch<N, FMT><<<r.ctas[l], kRows * NPipes<N, FMT>::A, SM::A, sa>>>(r.tabs[l]);
        }
        DGFS_LAUNCHED(lead);
        if (fk.on) {
            DGFS_CUDA(cudaEventRecord(fk.ev_a, sa));
            DGFS_CUDA(cudaStreamWaitEvent(st, fk.ev_a, 0));
        }
        {
            ProfScope ps(lead, "tc_stage_b", st);
            if (per_job)
                for (int j = 0; j < nj; ++j)
                    k_stage_b<N, FMT><<<grid_of(r.tabs[l + 1].grid[j]), kRows * NPipes<N, FMT>::B, SM::B, st>>>(
                        r.tabs[l + 1].job[j]);
            else
                k_stage_b_batch<N, FMT><<<r.ctas[l + 1], kRows * NPipes<N, FMT>::B, SM::B, st>>>(r.tabs[l + 1]);
        }
        DGFS_LAUNCHED(lead);
        if (fk.on) DGFS_CUDA(cudaEventRecord(fk.ev_b, st));
        {
            ProfScope ps(lead, "tc_stage_c", st);
            if (per_job)
                for (int j = 0; j < nj; ++j)
                    k_stage_c<N, FMT><<<grid_of(r.tabs[l + 2].grid[j]), kRows * NPipes<N, FMT>::C, SM::C, st>>>(
                        r.tabs[l + 2].job[j]);
            else
                k_stage_c_batch<N, FMT><<<r.ctas[l + 2], kRows * NPipes<N, FMT>::C, SM::C, st>>>(r.tabs[l + 2]);
        }
        DGFS_LAUNCHED(lead);
    }
    for (const BatchJob &b : r.jobs) {
        const TcWs w = ws_of(b.plan);
        const long n = (long)N * N * N;
        {
            ProfScope ps(b.plan, "tc_sum_partials", st);
            k_sum_partials<<<nblk((long)b.Ec * n, 256), 256, 0, st>>>(
                w.QG + (b.p * b.plan->S + b.q) * w.qg_stride, w.QGp, rs_blocks(b.plan), n, b.pt0, b.Ec);
        }
        DGFS_LAUNCHED(b.plan);
    }
    return DGFS_OK;
}

template <int FMT>
dgfs_status round_dispatch(int N, BatchRound &r, bool build, cudaStream_t st, Fork *fk)
{
    switch (N) {
    case 8: return build ? round_build<8, FMT>(r) : round_launch<8, FMT>(r, st, *fk);
    case 16: return build ? round_build<16, FMT>(r) : round_launch<16, FMT>(r, st, *fk);
    case 24: return build ? round_build<24, FMT>(r) : round_launch<24, FMT>(r, st, *fk);
    case 32: return build ? round_build<32, FMT>(r) : round_launch<32, FMT>(r, st, *fk);
    case 48: return build ? round_build<48, FMT>(r) : round_launch<48, FMT>(r, st, *fk);
    default: set_error("batch: N not supported by the tensor-core path"); return DGFS_EUNSUPPORTED;
    }
}

template <int FMT>
dgfs_status dispatch_collide(dgfs_plan_s *plan, int P, const void *f, void *Q, cudaStream_t st)
{
    if (plan->hermitian) {
        switch (plan->N) {
        case 8: return collide_herm_n<8, FMT>(plan, P, f, Q, st);
        case 16: return collide_herm_n<16, FMT>(plan, P, f, Q, st);
        case 24: return collide_herm_n<24, FMT>(plan, P, f, Q, st);
        case 32: return collide_herm_n<32, FMT>(plan, P, f, Q, st);
        default: set_error("the Hermitian form of the tensor-core path supports N <= 32"); return DGFS_EUNSUPPORTED;
        }
    }
    switch (plan->N) {
    case 8: return collide_n<8, FMT>(plan, P, f, Q, st);
    case 16: return collide_n<16, FMT>(plan, P, f, Q, st);
    case 24: return collide_n<24, FMT>(plan, P, f, Q, st);
    case 32: return collide_n<32, FMT>(plan, P, f, Q, st);
    case 48: return collide_n<48, FMT>(plan, P, f, Q, st);
    default: set_error("N not supported by the tensor-core path"); return DGFS_EUNSUPPORTED;
    }
}

template <int FMT>
dgfs_status dispatch_attrs(int N)
{
    switch (N) {
    case 8: return set_smem_attrs<8, FMT>();
    case 16: return set_smem_attrs<16, FMT>();
    case 24: return set_smem_attrs<24, FMT>();
    case 32: return set_smem_attrs<32, FMT>();
    case 48: return set_smem_attrs<48, FMT>();
    default: set_error("N not supported by the tensor-core path"); return DGFS_EUNSUPPORTED;
    }
}

template <int FMT>
dgfs_status build_images(dgfs_plan_s *plan, TcState *ts)
{
    const int N = plan->N, RS = plan->Nrho * plan->M;
    const long n = (long)N * N * N;
    const long IC = tcfmt::img_c<FMT>(N);
    constexpr int NT = Fmt<FMT>::NT;
    DGFS_CUDA(dev_malloc(&ts->Fimg, NT * IC));
    DGFS_CUDA(cudaMemset(ts->Fimg, 0, NT * IC));
    k_fimg<FMT><<<nblk((long)N * N, 256), 256>>>(ts->Fimg, N);
    DGFS_LAUNCHED(plan);
    for (auto &pt : plan->pairs) {
        const size_t tbytes = (size_t)RS * 2 * 3 * NT * IC;
        DGFS_CUDA(dev_malloc(&pt.tmat, tbytes));
        DGFS_CUDA(cudaMemset(pt.tmat, 0, tbytes));
        DGFS_CUDA(dev_malloc(&pt.b32, sizeof(float2) * RS * n));
        plan->table_bytes += tbytes + sizeof(float2) * RS * n;
        k_timg<FMT><<<nblk((long)RS * 6 * N * N, 256), 256>>>(reinterpret_cast<uint8_t *>(pt.tmat), pt.phase, N, RS);
        DGFS_LAUNCHED(plan);
        k_to_f32<<<nblk(RS * n, 256), 256>>>(pt.b32, pt.b, RS * n);
        DGFS_LAUNCHED(plan);
    }
    DGFS_TRY(df_tables(plan, &ts->tw_df));
    return dispatch_attrs<FMT>(N);
}

bool tc_supported_N(int N) { return N == 8 || N == 16 || N == 24 || N == 32 || N == 48; }

// The kernels' bounded-wait path on an mbarrier that nothing completes
// (expire != 0) or that the kernel completes itself (expire == 0).
__global__ void k_wait_selftest(int *err, int expire, long polls)
{
    __shared__ uint64_t mb;
    if (threadIdx.x == 0) mbar_init(&mb, 1);
    __syncthreads();
    if (!expire && threadIdx.x == 0)
        asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(smem_u32(&mb))
                     : "memory");
    const bool ok = mbar_wait(&mb, 0, polls);
    if (!__syncthreads_and(ok ? 1 : 0) && threadIdx.x == 0) atomicExch(err, kErrTimeout);
}

}  // namespace

dgfs_status tc_prepare(dgfs_plan_s *plan)
{
    const int N = plan->N, RS = plan->Nrho * plan->M;
    if (!tc_supported_N(N)) {
        set_error("tensor-core plans support N in {8, 16, 24, 32, 48}");
        return DGFS_EUNSUPPORTED;
    }
    TcState *ts = host_new<TcState>();
    if (!ts) {
        set_error("tc_prepare: out of host memory");
        return DGFS_ENOMEM;
    }
    plan->tc = ts;
    ts->fmt = plan->prec == DGFS_BF16X3 ? 1 : 0;
    ts->nterms = plan->prec == DGFS_TF32 ? 1 : (plan->prec == DGFS_BF16X3 ? 6 : 3);
    ts->chunk_max = std::max(1, std::min(plan->max_points, 24));
    ts->chunk = ts->chunk_max;
    ts->rsb_max = std::min(RS, 16);
    ts->rsb = std::min(RS, 4);
    // CTA groups: about four waves of CTAs over the GPU
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, plan->device);
    // about 8 waves of CTAs per stage (the autotuner's usual choice at N = 32)
    ts->groups_a = std::max(1, (8 * sms + RS) / (2 * RS));
    ts->groups_b = std::max(1, (8 * sms + RS / 2) / RS);
    ts->sms = sms;
    DGFS_CUDA(dev_malloc(&ts->err, sizeof(int)));
    if (wl_supported(N)) {  // counters of the work list (stage C grid rows <= rsb_max)
        // jobs of one call: S^2 pairs times the chunks of points (chunks of at
        // least min(chunk_max, 8) points, the autotuner's smaller candidate)
        const int cmin = std::min(ts->chunk_max, 8);
        const size_t jobs = std::min<size_t>(kWlJobs, (size_t)plan->S * plan->S * ((plan->max_points + cmin - 1) / cmin));
        ts->wl_words = wl_words_for(RS, ts->rsb_max, jobs * wl_job_tasks_max(plan, sms, ts->chunk_max, ts->rsb_max));
        DGFS_CUDA(dev_malloc(&ts->wl_ctr, sizeof(uint32_t) * ts->wl_words));
    }
    DGFS_CUDA(cudaMemset(ts->err, 0, sizeof(int)));
    DGFS_CUDA(cudaStreamCreateWithFlags(&ts->side, cudaStreamNonBlocking));
    DGFS_CUDA(cudaEventCreateWithFlags(&ts->ev_entry, cudaEventDisableTiming));
    DGFS_CUDA(cudaEventCreateWithFlags(&ts->ev_a, cudaEventDisableTiming));
    DGFS_CUDA(cudaEventCreateWithFlags(&ts->ev_b, cudaEventDisableTiming));
    // H double-buffered where its second slot takes at most 2 GiB
    ts->hslots = sizeof(float2) * (size_t)ts->chunk_max * RS * ((size_t)N * N * N) <= (size_t(2) << 30) ? 2 : 1;
    DGFS_CUDA(cudaStreamCreateWithFlags(&ts->side_b, cudaStreamNonBlocking));
    DGFS_CUDA(cudaEventCreateWithFlags(&ts->ev_c[0], cudaEventDisableTiming));
    DGFS_CUDA(cudaEventCreateWithFlags(&ts->ev_c[1], cudaEventDisableTiming));
    // axes along which the design direction has no component: the translate
    // there is exp(i 0) = 1 in k-space, i.e. the identity, and is skipped
    {
        std::vector<uint8_t> mask(RS);
        for (int rs = 0; rs < RS; ++rs) {
            const double *sg = plan->sigma + 3 * (rs % plan->M);
            mask[rs] = (uint8_t)((sg[0] == 0.0 ? 1 : 0) | (sg[1] == 0.0 ? 2 : 0) | (sg[2] == 0.0 ? 4 : 0));
        }
        DGFS_CUDA(dev_malloc(&ts->idmask, RS));
        DGFS_CUDA(cudaMemcpy(ts->idmask, mask.data(), RS, cudaMemcpyHostToDevice));
    }
    // the reflected direction of every (r, s), for the same-species pairs
    {
        const int M = plan->M;
        std::vector<uint16_t> map(RS);
        int found = 0;
        for (int s = 0; s < M; ++s) {
            const double *sg = plan->sigma + 3 * s;
            for (int t = 0; t < M; ++t) {
                const double *sr = plan->sigma + 3 * t;
                if (sr[0] == -sg[0] && sr[1] == -sg[1] && sr[2] == -sg[2]) {
                    for (int r = 0; r < plan->Nrho; ++r) map[r * M + s] = (uint16_t)(r * M + t);
                    ++found;
                    break;
                }
            }
        }
        if (found == M) {  // both designs are centrally symmetric
            DGFS_CUDA(dev_malloc(&ts->bmap, sizeof(uint16_t) * RS));
            DGFS_CUDA(cudaMemcpy(ts->bmap, map.data(), sizeof(uint16_t) * RS, cudaMemcpyHostToDevice));
        }
    }
    dgfs_status st = ts->fmt == 0 ? build_images<0>(plan, ts) : build_images<1>(plan, ts);
    if (st != DGFS_OK) return st;
    DGFS_CUDA(cudaDeviceSynchronize());
    return DGFS_OK;
}

void tc_release(dgfs_plan_s *plan)
{
    TcState *ts = reinterpret_cast<TcState *>(plan->tc);
    if (!ts) return;
    dev_free(ts->Fimg);
    dev_free(ts->err);
    dev_free(ts->wl_ctr);
    dev_free(ts->idmask);
    dev_free(ts->bmap);
    dev_free(ts->tw_df);
    dev_free(ts->adjmul);
    if (ts->side) cudaStreamDestroy(ts->side);
    if (ts->side_b) cudaStreamDestroy(ts->side_b);
    for (cudaEvent_t e : ts->ev_c)
        if (e) cudaEventDestroy(e);
    if (ts->ev_entry) cudaEventDestroy(ts->ev_entry);
    if (ts->ev_a) cudaEventDestroy(ts->ev_a);
    if (ts->ev_b) cudaEventDestroy(ts->ev_b);
    delete ts;
    plan->tc = nullptr;
}

size_t tc_workspace_bytes(const dgfs_plan_s *plan)
{
    const TcState *ts = reinterpret_cast<const TcState *>(plan->tc);
    const long n = (long)plan->N * plan->N * plan->N;
    const long RS = (long)plan->Nrho * plan->M;
    const long E = ts ? ts->chunk_max : 1, RSB = ts ? ts->rsb_max : 1;
    const long hs = ts ? ts->hslots : 1;
    return sizeof(float4) * ((long)plan->max_points * (plan->S + plan->S * plan->S) * n) +
           sizeof(float2) * ((2 + hs) * E * RS * n + E * RSB * n);
}

struct BatchPlan {
    dgfs_plan_s *plan;
    int P;
    const void *f;
    void *Q;
};

struct TcBatch {
    std::vector<BatchGroup> groups;
    std::vector<BatchPlan> plans;  // forward transforms before the rounds, finishing passes after them
    cudaStream_t side = nullptr;   // stage A launches (see Fork)
    cudaEvent_t ev_entry = nullptr, ev_a = nullptr, ev_b = nullptr;
    // work list per group (empty where N has none): the group's
    // rounds queued into k_worklist launches, which share one counter buffer
    // (sched = 1; the default 0 runs the rounds as per-stage launches)
    int sched = 0;
    std::vector<std::vector<WlTable>> wl;
    std::vector<std::vector<uint32_t>> wl_words;
    uint32_t *wl_ctr = nullptr;
    int sms = 148;
};

void tc_batch_free(void *handle)
{
    TcBatch *b = reinterpret_cast<TcBatch *>(handle);
    if (!b) return;
    dev_free(b->wl_ctr);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->ev_entry) cudaEventDestroy(b->ev_entry);
    if (b->ev_a) cudaEventDestroy(b->ev_a);
    if (b->ev_b) cudaEventDestroy(b->ev_b);
    delete b;
}

// Jobs of `count` tensor-core plans (distinct; each with its own f, Q and P)
// grouped by (N, operand format) into rounds.
dgfs_status tc_batch_build(int count, dgfs_plan_s *const *plans, const int *P, void *const *f, void *const *Q,
                           void **out)
{
    TcBatch *b = host_new<TcBatch>();
    if (!b) {
        set_error("dgfs_batch_create: out of host memory");
        return DGFS_ENOMEM;
    }
    for (int i = 0; i < count; ++i) {
        dgfs_plan_s *plan = plans[i];
        const TcState *ts = reinterpret_cast<const TcState *>(plan->tc);
        if (reinterpret_cast<uintptr_t>(f[i]) & 15) {
            set_error("dgfs_batch_create: f must be 16-byte aligned for tensor-core plans");
            tc_batch_free(b);
            return DGFS_EINVAL;
        }
        b->plans.push_back(BatchPlan{plan, P[i], f[i], Q[i]});
        BatchGroup *g = nullptr;
        for (auto &x : b->groups)
            if (x.N == plan->N && x.fmt == ts->fmt) g = &x;
        if (!g) {
            b->groups.push_back(BatchGroup{});
            g = &b->groups.back();
            g->N = plan->N;
            g->fmt = ts->fmt;
        }
        int k = 0;
        for (int p = 0; p < plan->S; ++p)
            for (int q = 0; q < plan->S; ++q)
                for (int pt0 = 0; pt0 < P[i]; pt0 += ts->chunk, ++k) {
                    if ((int)g->rounds.size() <= k) g->rounds.emplace_back();
                    const int Ec = std::min(ts->chunk, P[i] - pt0);
                    g->rounds[k].jobs.push_back(BatchJob{plan, p, q, pt0, Ec, P[i], f[i], Q[i]});
                }
    }
    for (auto &g : b->groups)
        for (auto &r : g.rounds) {
            const dgfs_status st = g.fmt == 0 ? round_dispatch<0>(g.N, r, true, nullptr, nullptr)
                                              : round_dispatch<1>(g.N, r, true, nullptr, nullptr);
            if (st != DGFS_OK) {
                tc_batch_free(b);
                return st;
            }
        }
    // the same rounds as work lists (groups of N = 24, 32, 48)
    size_t words = 0;
    b->wl.resize(b->groups.size());
    b->wl_words.resize(b->groups.size());
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        const BatchGroup &g = b->groups[gi];
        if (!wl_supported(g.N)) continue;
        std::vector<std::vector<WlSpec>> rounds;
        for (const BatchRound &r : g.rounds) {
            rounds.emplace_back();
            for (const BatchJob &j : r.jobs) {
                WlSpec sp;
                switch (g.N * 2 + g.fmt) {
                case 48: sp = wl_spec<24, 0>(j.plan, j.f, j.p, j.q, j.pt0, j.Ec); break;
                case 49: sp = wl_spec<24, 1>(j.plan, j.f, j.p, j.q, j.pt0, j.Ec); break;
                case 64: sp = wl_spec<32, 0>(j.plan, j.f, j.p, j.q, j.pt0, j.Ec); break;
                case 65: sp = wl_spec<32, 1>(j.plan, j.f, j.p, j.q, j.pt0, j.Ec); break;
                case 96: sp = wl_spec<48, 0>(j.plan, j.f, j.p, j.q, j.pt0, j.Ec); break;
                default: sp = wl_spec<48, 1>(j.plan, j.f, j.p, j.q, j.pt0, j.Ec); break;
                }
                rounds.back().push_back(sp);
            }
        }
        const int npc = g.N == 48 ? NPipes<48, 0>::C : NPipes<32, 0>::C;
        if (!wl_build(rounds, npc, nullptr, b->wl[gi], b->wl_words[gi])) {
            b->wl[gi].clear();  // this group runs its rounds as launches
            b->wl_words[gi].clear();
            continue;
        }
        for (uint32_t wd : b->wl_words[gi]) words = std::max(words, (size_t)wd);
    }
    if (words) {
        cudaError_t ea = dev_malloc(&b->wl_ctr, sizeof(uint32_t) * words);
        if (ea != cudaSuccess) {
            tc_batch_free(b);
            return cuda_status(ea, "dgfs_batch_create: work-list counters");
        }
        for (auto &L : b->wl)
            for (WlTable &t : L) t.ctr = b->wl_ctr;
    }
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, plans[0]->device);
    cudaError_t e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_entry, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_a, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_b, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        tc_batch_free(b);
        return cuda_status(e, "batch stream and events");
    }
    *out = b;
    return DGFS_OK;
}

dgfs_status tc_batch_launch(void *handle, cudaStream_t st)
{
    TcBatch *b = reinterpret_cast<TcBatch *>(handle);
    // serial when a plan's per-kernel profiler is on (as in collide_n)
    bool prof = false;
    for (const BatchPlan &bp : b->plans) prof |= bp.plan->prof != nullptr;
    Fork fk{b->side, b->ev_entry, b->ev_a, b->ev_b, !prof, true};
    if (fk.on) DGFS_CUDA(cudaEventRecord(fk.ev_entry, st));
    for (const BatchPlan &bp : b->plans) {
        const TcState *ts = reinterpret_cast<const TcState *>(bp.plan->tc);
        DGFS_TRY(df_forward(bp.plan, bp.P, reinterpret_cast<const float *>(bp.f), ws_of(bp.plan).F, ts->tw_df, st));
    }
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        const BatchGroup &g = b->groups[gi];
        if (b->sched == 1 && !b->wl[gi].empty()) {
            dgfs_plan_s *lead = g.rounds[0].jobs[0].plan;
            const auto &L = b->wl[gi];
            const auto &W = b->wl_words[gi];
            switch (g.N * 2 + g.fmt) {
            case 48: DGFS_TRY((wl_launch<24, 0>(lead, L, W, b->sms, st))); break;
            case 49: DGFS_TRY((wl_launch<24, 1>(lead, L, W, b->sms, st))); break;
            case 64: DGFS_TRY((wl_launch<32, 0>(lead, L, W, b->sms, st))); break;
            case 65: DGFS_TRY((wl_launch<32, 1>(lead, L, W, b->sms, st))); break;
            case 96: DGFS_TRY((wl_launch<48, 0>(lead, L, W, b->sms, st))); break;
            default: DGFS_TRY((wl_launch<48, 1>(lead, L, W, b->sms, st))); break;
            }
            continue;
        }
        for (auto &r : b->groups[gi].rounds)
            DGFS_TRY(g.fmt == 0 ? round_dispatch<0>(g.N, r, false, st, &fk)
                                : round_dispatch<1>(g.N, r, false, st, &fk));
    }
    for (const BatchPlan &bp : b->plans) {
        const TcWs w = ws_of(bp.plan);
        const TcState *ts = reinterpret_cast<const TcState *>(bp.plan->tc);
        DGFS_TRY(df_finish(bp.plan, bp.P, w.QG, w.qg_stride, w.F, reinterpret_cast<const float *>(bp.f),
                           reinterpret_cast<float *>(bp.Q), ts->tw_df, st));
    }
    return DGFS_OK;
}

// 0: every group runs its rounds as per-stage launches (the default); 1:
// groups of N = 24, 32 and 48 run as work lists
dgfs_status tc_batch_set_schedule(void *handle, int mode)
{
    TcBatch *b = reinterpret_cast<TcBatch *>(handle);
    if (mode != 0 && mode != 1) {
        set_error("dgfs_batch_set_schedule: mode must be 0 or 1");
        return DGFS_EINVAL;
    }
    if (b) b->sched = mode;
    return DGFS_OK;
}

// Hermitian form: bytes of the plan's extra workspace (see HermWs), and the
// complex-input z images written into it
size_t tc_herm_bytes(const dgfs_plan_s *plan)
{
    const TcState *ts = reinterpret_cast<const TcState *>(plan->tc);
    const long n = (long)plan->N * plan->N * plan->N, S = plan->S;
    const long Psmax = (plan->max_points + 1) / 2;
    const long zi = ts->fmt == 0 ? zimg_pair_bytes<0>(plan) : zimg_pair_bytes<1>(plan);
    return sizeof(float) * plan->max_points * S * n + sizeof(float4) * S * S * Psmax * n + (size_t)(S * S) * zi;
}

bool tc_herm_supported(const dgfs_plan_s *plan) { return plan->N <= 32; }

dgfs_status tc_herm_build(dgfs_plan_s *plan)
{
    const TcState *ts = reinterpret_cast<const TcState *>(plan->tc);
    const HermWs h = herm_ws_of(plan);
    const int N = plan->N, RS = plan->Nrho * plan->M, S = plan->S;
    DGFS_CUDA(cudaMemset(h.zimg, 0, (size_t)S * S * h.zimg_pair));
    for (int pr = 0; pr < S * S; ++pr) {
        uint8_t *dst = h.zimg + (long)pr * h.zimg_pair;
        if (ts->fmt == 0)
            k_timg_zc<0><<<nblk((long)RS * 2 * N * N, 256), 256>>>(dst, plan->pairs[pr].phase, N, RS);
        else
            k_timg_zc<1><<<nblk((long)RS * 2 * N * N, 256), 256>>>(dst, plan->pairs[pr].phase, N, RS);
        DGFS_LAUNCHED(plan);
    }
    DGFS_CUDA(cudaDeviceSynchronize());
    return DGFS_OK;
}

dgfs_status tc_collide(dgfs_plan_s *plan, int P, const void *f, void *Q, cudaStream_t st)
{
    const TcState *ts = reinterpret_cast<const TcState *>(plan->tc);
    if (reinterpret_cast<uintptr_t>(f) & 15) {  // f tiles are read with 16-byte loads
        set_error("dgfs_collide: f must be 16-byte aligned for tensor-core plans");
        return DGFS_EINVAL;
    }
    return ts->fmt == 0 ? dispatch_collide<0>(plan, P, f, Q, st) : dispatch_collide<1>(plan, P, f, Q, st);
}

// Time candidate launch configurations on the caller's data (each candidate:
// one untimed call, then the best of two timed calls) and keep the fastest.
dgfs_status tc_autotune(dgfs_plan_s *plan, int P, const void *f, void *Q, cudaStream_t st, double *best_ms)
{
    TcState *ts = reinterpret_cast<TcState *>(plan->tc);
    if (!ts) {
        set_error("dgfs_plan_autotune: only tensor-core plans have launch parameters to tune");
        return DGFS_EUNSUPPORTED;
    }
    const int RS = plan->Nrho * plan->M;
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, plan->device);
    struct Cand { int chunk, rsb, ga, gb, ws; };
    std::vector<Cand> cands;
    const bool ws_fits = plan->N == 16 || plan->N == 32;  // WsA<N, FMT>::OK
    const bool a2_fits = plan->N == 16 || plan->N == 32 || plan->N == 48;  // A2<N, FMT>::OK
    const int chunks[] = {ts->chunk_max, std::min(ts->chunk_max, 8)};
    const int rsbs[] = {std::min(RS, 2), std::min(RS, 4), std::min(RS, 6), std::min(RS, 8),
                        std::min(RS, 12), std::min(RS, 16)};
    const int waves[] = {4, 8, 16};
    for (int c : chunks)
        for (int r : rsbs)
            for (int w : waves)
                for (int ws = 0; ws < 3; ++ws) {
                    if ((ws == 1 && !ws_fits) || (ws == 2 && !a2_fits)) continue;
                    const Cand k{c, std::min(r, ts->rsb_max), std::max(1, (w * sms + RS) / (2 * RS)),
                                 std::max(1, (w * sms + RS / 2) / RS), ws};
                    bool dup = false;
                    for (auto &o : cands)
                        dup |= o.chunk == k.chunk && o.rsb == k.rsb && o.ga == k.ga && o.gb == k.gb && o.ws == k.ws;
                    if (!dup) cands.push_back(k);
                }
    cudaEvent_t e0, e1;
    DGFS_CUDA(cudaEventCreate(&e0));
    DGFS_CUDA(cudaEventCreate(&e1));
    const TcState saved = *ts;
    double best = 1e300;
    TcState bestcfg = saved;
    dgfs_status status = DGFS_OK;
    for (const Cand &k : cands) {
        ts->chunk = k.chunk;
        ts->rsb = k.rsb;
        ts->groups_a = k.ga;
        ts->groups_b = k.gb;
        ts->ws_a = k.ws;
        status = tc_collide(plan, P, f, Q, st);
        if (status != DGFS_OK) break;
        double t = 1e300;
        for (int rep = 0; rep < 2 && status == DGFS_OK; ++rep) {
            cudaEventRecord(e0, st);
            status = tc_collide(plan, P, f, Q, st);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) status = cuda_status(cudaGetLastError(), "autotune");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            t = std::min(t, (double)ms);
        }
        if (status != DGFS_OK) break;
        if (t < best) {
            best = t;
            bestcfg = *ts;
        }
    }
    // the work-list schedule with the best launch parameters (variant 0)
    if (status == DGFS_OK && wl_supported(plan->N)) {
        *ts = bestcfg;
        ts->ws_a = 0;
        ts->sched = 1;
        status = tc_collide(plan, P, f, Q, st);
        double t = 1e300;
        for (int rep = 0; rep < 2 && status == DGFS_OK; ++rep) {
            cudaEventRecord(e0, st);
            status = tc_collide(plan, P, f, Q, st);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) status = cuda_status(cudaGetLastError(), "autotune");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            t = std::min(t, (double)ms);
        }
        if (status == DGFS_OK && t < best) {
            best = t;
            bestcfg = *ts;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != DGFS_OK) {
        *ts = saved;
        return status;
    }
    *ts = bestcfg;
    ts->tuned = 1;
    plan->config_gen++;
    if (best_ms) *best_ms = best;
    return tc_check(plan);
}

void tc_info(const dgfs_plan_s *plan, double *info)
{
    const TcState *ts = reinterpret_cast<const TcState *>(plan->tc);
    if (!ts) return;
    info[9] = ts->chunk;
    info[10] = ts->rsb;
    info[11] = ts->nterms;
    info[12] = ts->groups_a;
    info[13] = ts->groups_b;
    info[14] = ts->tuned;
}

dgfs_status tc_selftest_wait(dgfs_plan_s *plan, int expire, cudaStream_t st)
{
    TcState *ts = reinterpret_cast<TcState *>(plan->tc);
    if (!ts) {
        set_error("dgfs_plan_selftest_wait: only tensor-core plans have bounded device waits");
        return DGFS_EUNSUPPORTED;
    }
    k_wait_selftest<<<1, 32, 0, st>>>(ts->err, expire, 4096);
    DGFS_LAUNCHED(plan);
    return DGFS_OK;
}

// the plane stage sums the tiles of a radial node's directions (stage C)
bool tc_supports_collapse(const dgfs_plan_s *) { return true; }

// Select the plane-stage-A kernel (0 two-pipeline, 1 warp-specialised, 2 two
// threads per row); the autotuner times all that fit.
dgfs_status tc_set_variant(dgfs_plan_s *plan, int variant)
{
    TcState *ts = reinterpret_cast<TcState *>(plan->tc);
    if (!ts) {
        set_error("dgfs_plan_set_kernel_variant: only tensor-core plans have kernel variants");
        return DGFS_EUNSUPPORTED;
    }
    const int N = plan->N;
    const bool fits = variant == 0 || (variant == 1 && (N == 16 || N == 32)) ||
                      (variant == 2 && (N == 16 || N == 32 || N == 48));
    if (!fits) {
        set_error("dgfs_plan_set_kernel_variant: variant not available for this N");
        return variant < 0 || variant > 2 ? DGFS_EINVAL : DGFS_EUNSUPPORTED;
    }
    ts->ws_a = variant;
    plan->config_gen++;
    return DGFS_OK;
}

void tc_debug_worklist_chunk(int rs) { g_wl_chunk = std::max(1, rs); }

void tc_debug_worklist_trace(void *buf, size_t bytes)
{
    g_wl_trace = reinterpret_cast<unsigned long long *>(buf);
    g_wl_trace_cap = buf ? (uint32_t)std::min<size_t>(bytes / 32, 0xFFFFFFFFu) : 0;
}

// Select how a call runs its stages: 0 one launch per stage and job (two
// streams), 1 one work-list launch (N = 24, 32, 48).
dgfs_status tc_set_schedule(dgfs_plan_s *plan, int mode)
{
    TcState *ts = reinterpret_cast<TcState *>(plan->tc);
    if (!ts) {
        set_error("dgfs_plan_set_schedule: only tensor-core plans have a stage schedule");
        return DGFS_EUNSUPPORTED;
    }
    if (mode != 0 && mode != 1) {
        set_error("dgfs_plan_set_schedule: mode must be 0 or 1");
        return DGFS_EINVAL;
    }
    if (mode == 1 && !wl_supported(plan->N)) {
        set_error("dgfs_plan_set_schedule: the work list needs N in {24, 32, 48}");
        return DGFS_EUNSUPPORTED;
    }
    ts->sched = mode;
    plan->config_gen++;
    return DGFS_OK;
}

int tc_schedule(const dgfs_plan_s *plan)
{
    const TcState *ts = reinterpret_cast<const TcState *>(plan->tc);
    return ts ? ts->sched : 0;
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

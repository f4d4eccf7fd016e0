// Shared device and host pieces of the tensor-core path: the plan state,
// the stage arguments, the tcgen05 helpers, the stage A/B/C kernel bodies
// and the workspace/argument helpers.  Included by tc32.cu (forward) and
// tcadj.cu (adjoint); everything sits in an unnamed namespace, so each
// translation unit compiles and launches its own kernel instantiations.
#pragma once
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "dfloat.cuh"
#include "dgfs_internal.h"
#include "tcfmt.cuh"
#include "umma.cuh"

namespace dgfs {
namespace {

using namespace umma;
using tcfmt::kRows;
using tcfmt::Fmt;

constexpr long kWaitLimit = 1L << 22;  // mbarrier polls before declaring a timeout
constexpr int kErrTimeout = 1;
constexpr int kSmemMax = 227 * 1024;

struct TcState {
    int fmt = 0;              // operand format: 0 TF32 split, 1 BF16 three-term split
    uint8_t *Fimg = nullptr;  // forward DFT as pre-swizzled B-operand images [terms][IMGC]
    int *err = nullptr;       // device error flag
    int nterms = 3;           // products per contraction (TF32: 1 or 3; BF16: 6)
    int chunk = 8;            // evaluations per launch (<= chunk_max, the workspace's)
    int rsb = 8;              // (r, s) blocks of stage C (<= rsb_max)
    int chunk_max = 8, rsb_max = 16;
    int groups_a = 2, groups_b = 4;  // CTA groups per (r, s) in stages A and B
    int tuned = 0;
    uint8_t *idmask = nullptr;  // [RS] bit d set when sigma_{s,d} == 0 (T_d is the identity; x and y are skipped)
    uint16_t *bmap = nullptr;   // [RS] r M + s' with sigma_s' = -sigma_s (null if the design is not centrally symmetric)
    int skip_identity = 1;
    int ws_a = 0;  // stage A variant: 0 two-pipeline, 1 warp-specialised, 2 two threads per row (autotuner)
    float4 *tw_df = nullptr;  // [N] exp(-2 pi i j / N) as double-float (findf.cu)
    // stage A of the next job runs on a second stream while stage C of the
    // current one drains (it only has to wait for stage B to have read A', B')
    cudaStream_t side = nullptr;
    cudaEvent_t ev_entry = nullptr, ev_a = nullptr, ev_b = nullptr;
    // 1: every stage of a call runs in one work-list launch
    // (k_worklist) instead of one launch per stage and job
    int sched = 0;
    int sms = 148;
    uint32_t *wl_ctr = nullptr;  // dependency counters of the work list
    size_t wl_words = 0;
    // plain calls: 2 when H is double-buffered (stage B of job j + 1 on a third
    // stream then runs beside stage C of job j, see collide_n)
    int hslots = 1;
    cudaStream_t side_b = nullptr;
    cudaEvent_t ev_c[2] = {nullptr, nullptr};
    // adjoint (tcadj.cu): per pair [2 sides][RS][n] conj(phi_rs(k)) of the
    // transposed translates, built at the first backward call
    float2 *adjmul = nullptr;
};

struct TcArgs {
    long n;
    int S, p, q, pt0, Ec, RS, nterms, rs_per_block, rsb;
    int collapse_M;        // > 1: stage C sums the M directions of each radial node first (sigma collapse)
    const float *f;        // [P][S][n]
    float2 *Ap, *Bq, *H;   // [E][RS][n]
    float2 *QGp;           // [E][rsb][n]
    const uint8_t *timg;   // pair: [RS][2 sides][3 axes][terms][IMGC] pre-swizzled B images
    const uint8_t *Fimg;   // [terms][IMGC]
    const float2 *b32;     // [RS][n]
    const double *w;       // [RS]
    const uint8_t *idmask; // [RS] identity-axis bits (x: 1, y: 2, z: 4), null = none
    int *err;
    // Hermitian form (declared variant): grid slot e carries points 2(pt0 + e)
    // (real part) and 2(pt0 + e) + 1 (imaginary part, absent beyond npts) of
    // the Nyquist-free f~ in a.f; stage A's z-pass takes that complex input
    // with the complex-input images zimg [RS][2 sides][terms][IMGC], and stage
    // B multiplies real parts and imaginary parts separately
    int herm, npts;
    const uint8_t *zimg;
};

// Same-species pair (p = q): the B-side translate at (r, s) equals the A-side
// translate at (r, s') with sigma_s' = -sigma_s (m_p = m_q), so stage A computes
// the A side only and stage B reads B' from A' at bmap[rs] = r M + s'.  Kept
// apart from TcArgs (the batched work list passes 48 TcArgs by value and does
// not use this).
struct Share {
    bool on = false;
    const uint16_t *bmap = nullptr;  // [RS], device
};

__host__ __device__ constexpr int pow2_cols(int c)
{
    return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512;
}

__device__ __forceinline__ uint8_t *align1024(uint8_t *p)
{
    return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

// Named barrier of one 128-thread pipeline: id 1 + pipeline (id 0 is __syncthreads).
__device__ __forceinline__ void pbar(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

// AND-vote over one pipeline's 128 threads (also a barrier).
__device__ __forceinline__ bool pbar_and(int id, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, %2, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)(v ? 1 : 0)), "r"(id)
        : "memory");
    return r != 0;
}

// One pipeline: its thread 0 issues `issue()` and commits to mbar; the
// pipeline's threads wait.  Returns false (for every thread of the pipeline)
// if the wait expired.
template <typename F>
__device__ __forceinline__ bool run_mma(uint64_t *mbar, uint32_t &phase, int bar_id, F issue)
{
    fence_proxy_async();
    fence_before();
    pbar(bar_id);
    fence_after();
    if ((threadIdx.x & (kRows - 1)) == 0) {
        issue();
        commit(mbar);
    }
    const bool ok = mbar_wait(mbar, phase, kWaitLimit);
    phase ^= 1u;
    const bool all = pbar_and(bar_id, ok);
    fence_after();
    return all;
}

// Whole-CTA bounded wait for a bulk-copy phase.
__device__ __forceinline__ bool wait_copy_cta(uint64_t *mbar, uint32_t &phase)
{
    const bool ok = mbar_wait(mbar, phase, kWaitLimit);
    phase ^= 1u;
    return __syncthreads_and(ok ? 1 : 0) != 0;
}

// One pipeline's bounded wait for a bulk-copy phase.
__device__ __forceinline__ bool wait_copy_pipe(uint64_t *mbar, uint32_t &phase, int bar_id)
{
    const bool ok = mbar_wait(mbar, phase, kWaitLimit);
    phase ^= 1u;
    return pbar_and(bar_id, ok);
}

// Pencils held one per thread, adjacent lanes (2k, 2k+1) holding adjacent
// pencils whose elements lie `stride` float2 apart in global memory: one
// 16-byte access covers one element of both pencils of a lane pair (the even
// lane takes the even elements, the odd lane the odd ones) and a shuffle hands
// each lane the value of its own pencil.  This halves the global memory
// instructions of 8-byte per-thread accesses.  base: element 0 of the even
// lane's pencil (16-byte aligned).  Every lane of the warp must call these.
template <int CNT>
__device__ __forceinline__ void load_pair(float2 *dst, const float2 *base, long stride, bool valid)
{
    const bool odd = threadIdx.x & 1;
#pragma unroll
    for (int x = 0; x < CNT; x += 2) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (valid) v = *reinterpret_cast<const float4 *>(base + (long)(x + (odd ? 1 : 0)) * stride);
        // even lane: v = (x of own, x of partner); odd lane: v = (x+1 of partner, x+1 of own)
        const float gx = odd ? v.x : v.z, gy = odd ? v.y : v.w;
        const float rx = __shfl_xor_sync(0xffffffffu, gx, 1), ry = __shfl_xor_sync(0xffffffffu, gy, 1);
        dst[x] = odd ? make_float2(rx, ry) : make_float2(v.x, v.y);
        dst[x + 1] = odd ? make_float2(v.z, v.w) : make_float2(rx, ry);
    }
}

// The same access split in two, so that a prefetch stays asynchronous: the
// raw 16-byte loads first, the shuffles when the values are needed.
template <int CNT>
__device__ __forceinline__ void load_pair_raw(float4 *raw, const float2 *base, long stride, bool valid)
{
    const bool odd = threadIdx.x & 1;
#pragma unroll
    for (int x = 0; x < CNT; x += 2)
        raw[x / 2] = valid ? *reinterpret_cast<const float4 *>(base + (long)(x + (odd ? 1 : 0)) * stride)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
}

template <int CNT>
__device__ __forceinline__ void unpack_pair(float2 *dst, const float4 *raw)
{
    const bool odd = threadIdx.x & 1;
#pragma unroll
    for (int x = 0; x < CNT; x += 2) {
        const float4 v = raw[x / 2];
        const float gx = odd ? v.x : v.z, gy = odd ? v.y : v.w;
        const float rx = __shfl_xor_sync(0xffffffffu, gx, 1), ry = __shfl_xor_sync(0xffffffffu, gy, 1);
        dst[x] = odd ? make_float2(rx, ry) : make_float2(v.x, v.y);
        dst[x + 1] = odd ? make_float2(v.z, v.w) : make_float2(rx, ry);
    }
}

template <int CNT>
__device__ __forceinline__ void store_pair(float2 *base, const float2 *val, long stride, bool valid)
{
    const bool odd = threadIdx.x & 1;
#pragma unroll
    for (int x = 0; x < CNT; x += 2) {
        const float2 give = odd ? val[x] : val[x + 1];
        const float rx = __shfl_xor_sync(0xffffffffu, give.x, 1), ry = __shfl_xor_sync(0xffffffffu, give.y, 1);
        const float4 w =
            odd ? make_float4(rx, ry, val[x + 1].x, val[x + 1].y) : make_float4(val[x].x, val[x].y, rx, ry);
        if (valid) *reinterpret_cast<float4 *>(base + (long)(x + (odd ? 1 : 0)) * stride) = w;
    }
}

__device__ __forceinline__ uint32_t lane_base(uint32_t tbase)
{
    return tbase + ((uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16);
}

// first term of the image of (r, s, side, axis); terms are IMGC bytes apart
template <int FMT>
__device__ __forceinline__ const uint8_t *timg_at(const uint8_t *timg, int N, int rs, int side, int ax)
{
    return timg + (((long)rs * 2 + side) * 3 + ax) * Fmt<FMT>::NT * (long)tcfmt::img_c<FMT>(N);
}

// Bulk-copy `terms` blocks of `bytes` (source blocks `sstride` apart) to
// shared memory blocks `dstride` apart, completing on mbar (thread 0 only).
__device__ __forceinline__ void copy_terms(uint8_t *dst, int dstride, const uint8_t *src, long sstride, int bytes,
                                           int terms, uint64_t *mbar)
{
    for (int t = 0; t < terms; ++t) bulk_g2s(dst + t * dstride, src + t * sstride, bytes, mbar);
}

// A stage body run as one task of the work list (k_worklist): the CTA, which
// may run several tasks, allocated all of TMEM once, at its start, and its
// mbarriers are initialised per task and invalidated after it.
struct Persist {
    uint32_t tmem;  // TMEM base address of the CTA's allocation
};

// Allocate ncols TMEM columns for the CTA (or take the work-list CTA's
// allocation) and initialise `nb` mbarriers.
__device__ __forceinline__ void cta_setup(uint32_t *slot, uint32_t ncols, uint64_t *mb, int nb,
                                          const Persist *ps = nullptr)
{
    if (ps) {
        if (threadIdx.x == 0) *slot = ps->tmem;
    } else if (threadIdx.x < 32) {
        tmem_alloc(slot, ncols);
    }
    if (threadIdx.x == 0)
        for (int i = 0; i < nb; ++i) mbar_init(mb + i, 1);
    fence_before();
    __syncthreads();
    fence_after();
}

__device__ __forceinline__ void cta_teardown(uint32_t tb, uint32_t ncols, bool ok, int *err, uint64_t *mb = nullptr,
                                             int nb = 0, const Persist *ps = nullptr)
{
    if (!ok) atomicExch(err, kErrTimeout);
    fence_before();
    __syncthreads();
    if (ps) {
        if (threadIdx.x == 0)
            for (int i = 0; i < nb; ++i) mbar_inval(mb + i);
    } else if (threadIdx.x < 32) {
        tmem_dealloc(tb, ncols);
    }
}

// Pipelines per CTA: each pipeline is 128 threads with its own data operand,
// TMEM columns, mbarrier and named barrier; the matrix images are shared.
// Chosen so that shared memory, TMEM (512 columns) and registers fit.
template <int N, int FMT> struct NPipes {
    static constexpr int A = N <= 16 ? 4 : (N <= 32 ? 2 : 1);
    static constexpr int B = N <= 16 ? (FMT == 0 ? 4 : 3) : (N <= 32 ? 2 : 1);
    static constexpr int C = N <= 8 ? 4 : (N <= 32 ? 2 : 1);
};

// Shared-memory layout sizes of the three stages.
template <int N, int FMT> struct Smem {
    static constexpr int NT = Fmt<FMT>::NT;
    static constexpr int AB = tcfmt::abytes<FMT>(N), IC = tcfmt::img_c<FMT>(N), IR = tcfmt::img_r<FMT>(N);
    static constexpr bool RES_A = NPipes<N, FMT>::A > 1 || 1024 + NT * (AB + IR + IC) <= kSmemMax;
    static constexpr bool RES_B = NPipes<N, FMT>::B > 1 || 1024 + NT * (AB + 3 * IC) <= kSmemMax;
    static constexpr size_t A = 1024 + (size_t)NPipes<N, FMT>::A * NT * AB + (RES_A ? NT * (IR + IC) : NT * IC);
    static constexpr size_t B = 1024 + (size_t)NPipes<N, FMT>::B * NT * AB + (RES_B ? 3 : 1) * NT * IC;
    static constexpr size_t C = 1024 + (size_t)NPipes<N, FMT>::C * NT * AB + NT * IC;
    static_assert(A <= kSmemMax && B <= kSmemMax && C <= kSmemMax, "shared memory");
};

// ------------------------------------------------------------------ stage A
// grid (groups, RS, sides: 2, or 1 for a same-species pair, whose B side stage B
// reads from the A side at the reflected direction).  A CTA holds T_z, T_y of
// its (r, s, side); each of
// its NP pipelines loops over items (point e, group of G x-planes): z-pass
// (real input), an in-plane transpose through shared memory, y-pass, result A'
// or B' to global.
template <int N, int FMT, bool HC = false>
__device__ __forceinline__ bool k_stage_a_body(const TcArgs &a, const uint3 bid, const uint3 gdim,
                                               const Persist *ps = nullptr)
{
    using SM = Smem<N, FMT>;
    constexpr int NP = NPipes<N, FMT>::A, NT = SM::NT, AB = SM::AB, IR = SM::IR, IC = SM::IC;
    constexpr bool RESIDENT = SM::RES_A;
    constexpr int G = kRows / N, KC = 2 * N, NO = 2 * N, NG = (N + G - 1) / G;
    // real-input K padded to whole 32-byte MMA steps (16 BF16 elements); the pad is zero
    constexpr int KR = FMT == 1 ? (N + 15) / 16 * 16 : N;
    constexpr int NN = N * N;
    constexpr int FPT = (G * NN / 4 + kRows - 1) / kRows;  // float4 per thread for one group
    constexpr uint32_t NCOL = pow2_cols(NP * 2 * NO);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align1024(smem_raw);
    const int pp = threadIdx.x / kRows, t = threadIdx.x % kRows, bar = 1 + pp;
    // the z image: real input (K = N) in the literal form, complex input
    // (K = 2N, IZ = IC bytes per term) in the Hermitian form
    constexpr bool herm = HC;
    constexpr int IZ = herm ? IC : IR;
    uint8_t *Bz = sm;                            // NT terms, IZ apart
    uint8_t *By = RESIDENT ? Bz + NT * IZ : Bz;  // NT terms, IC apart (one reloaded slot if not resident)
    uint8_t *A0 = sm + (RESIDENT ? NT * (IR + IC) + (herm ? NT * (IC - IR) : 0) : NT * IC) + pp * NT * AB;
    __shared__ uint64_t mb[NP + 1];  // [0, NP): MMA per pipeline, NP: copies
    __shared__ uint32_t tslot;
    const int rs = bid.y, side = bid.z;
    const long n = a.n;
    const int items = a.Ec * NG;
    const bool ident_y = a.idmask && (a.idmask[rs] & 2);
    // sigma_z = 0: T_z = I, so the y-pass operand is built from f directly; a
    // thread then loads its own row's z-pencil (needs N / 4 <= FPT float4)
    constexpr bool ZSKIP = N % 4 == 0 && N / 4 <= FPT;
    const bool ident_z = ZSKIP && a.idmask && (a.idmask[rs] & 4);
    cta_setup(&tslot, NCOL, mb, NP + 1, ps);
    const uint32_t tb = tslot + pp * 2 * NO, tl = lane_base(tb);
    uint32_t ph_mma = 0, ph_cp = 0;
    auto load_imgs = [&](int which) {  // 0: z, 1: y, 2: both
        if (threadIdx.x == 0) {
            const uint32_t bytes = which == 0 ? NT * IZ : which == 1 ? NT * IC : NT * (IZ + IC);
            mbar_expect_tx(&mb[NP], bytes);
            if (which != 1) {
                if (herm)
                    copy_terms(Bz, IZ, a.zimg + ((long)rs * 2 + side) * NT * (long)IC, IC, IZ, NT, &mb[NP]);
                else
                    copy_terms(Bz, IR, timg_at<FMT>(a.timg, N, rs, side, 2), IC, IR, NT, &mb[NP]);
            }
            if (which != 0) copy_terms(By, IC, timg_at<FMT>(a.timg, N, rs, side, 1), IC, IC, NT, &mb[NP]);
        }
    };
    const int sp = side == 0 ? a.p : a.q;
    const int g = t / N, yl = t % N;
    float4 pf[FPT];
    float4 pf2[HC ? FPT : 1];  // Hermitian form: the slot's second point
    auto prefetch = [&](int it) {
        const int e = it / NG, x0 = (it % NG) * G, nval = min(G, N - x0);
        const int pt = herm ? 2 * (a.pt0 + e) : a.pt0 + e;
        const float4 *fs = reinterpret_cast<const float4 *>(a.f + ((long)pt * a.S + sp) * n + (long)x0 * NN);
        const bool second = HC && herm && pt + 1 < a.npts;
        const float4 *fs2 = fs + (long)a.S * n / 4;
        const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ident_z) {  // row t = (g, y): f(x0 + g, y, z) for all z
#pragma unroll
            for (int j = 0; j < FPT; ++j) {
                const bool ok = j < N / 4 && t < nval * N;
                pf[j] = ok ? fs[t * (N / 4) + j] : zero4;
                if constexpr (HC) pf2[j] = (ok && second) ? fs2[t * (N / 4) + j] : zero4;
            }
            return;
        }
#pragma unroll
        for (int j = 0; j < FPT; ++j) {
            const int i = t + kRows * j;
            pf[j] = (4 * i < nval * NN) ? fs[i] : zero4;
            if constexpr (HC) pf2[j] = (4 * i < nval * NN && second) ? fs2[i] : zero4;
        }
    };
    const int stride = gdim.x * NP;
    int it = bid.x * NP + pp;
    if (it < items) prefetch(it);
    bool ok = true;
    if (RESIDENT && !(ident_z && ident_y)) {  // only the images this (r, s) uses
        load_imgs(ident_z ? 1 : (ident_y ? 0 : 2));
        ok = wait_copy_cta(&mb[NP], ph_cp);
    }
    for (; it < items && ok; it += stride) {
        const int e = it / NG, x0 = (it % NG) * G, nval = min(G, N - x0);
        if (ident_z) {
            if (ident_y) {
                // sigma_y = sigma_z = 0: A'(x0+g, y, z) = f for all z
                float4 *dst = reinterpret_cast<float4 *>((side == 0 ? a.Ap : a.Bq) + ((long)e * a.RS + rs) * n +
                                                         (long)(x0 + g) * NN + yl * N);
                if (t < nval * N) {
#pragma unroll
                    for (int j = 0; j < N / 4; ++j) {
                        float4 im = make_float4(0.f, 0.f, 0.f, 0.f);
                        if constexpr (HC) im = pf2[j];
                        dst[2 * j] = make_float4(pf[j].x, im.x, pf[j].y, im.y);
                        dst[2 * j + 1] = make_float4(pf[j].z, im.z, pf[j].w, im.w);
                    }
                }
                if (it + stride < items) prefetch(it + stride);
                continue;
            }
            // the y-pass operand, rows (g, z), K = y, straight from this row's f values
            if (t < nval * N) {
#pragma unroll
                for (int j = 0; j < N / 4; ++j) {
                    float4 im = make_float4(0.f, 0.f, 0.f, 0.f);
                    if constexpr (HC) im = pf2[j];
                    tcfmt::st_c<FMT>(A0, AB, g * N + 4 * j, yl, pf[j].x, im.x);
                    tcfmt::st_c<FMT>(A0, AB, g * N + 4 * j + 1, yl, pf[j].y, im.y);
                    tcfmt::st_c<FMT>(A0, AB, g * N + 4 * j + 2, yl, pf[j].z, im.z);
                    tcfmt::st_c<FMT>(A0, AB, g * N + 4 * j + 3, yl, pf[j].w, im.w);
                }
            }
            if (it + stride < items) prefetch(it + stride);
        } else {
        if constexpr (HC) {  // complex input: (point 2e, point 2e + 1) at K = 2 z, 2 z + 1
#pragma unroll
            for (int j = 0; j < FPT; ++j) {
                const int i = t + kRows * j;
                if (4 * i < nval * NN) {
                    const int row = (4 * i) / N, z = (4 * i) % N;
                    tcfmt::st_c2<FMT>(A0, AB, row, z, make_float2(pf[j].x, pf2[j].x), make_float2(pf[j].y, pf2[j].y));
                    tcfmt::st_c2<FMT>(A0, AB, row, z + 2, make_float2(pf[j].z, pf2[j].z),
                                      make_float2(pf[j].w, pf2[j].w));
                }
            }
        } else {
#pragma unroll
        for (int j = 0; j < FPT; ++j) {
            const int i = t + kRows * j;
            if (4 * i < nval * NN) tcfmt::st_f4<FMT>(A0, AB, (4 * i) / N, (4 * i) % N, pf[j]);
        }
        }
        if constexpr (KR > N && !HC) {  // zero the pad of this thread's row in every term
            if (t < nval * N)
#pragma unroll
                for (int term = 0; term < NT; ++term)
#pragma unroll
                    for (int e0 = N; e0 < KR; e0 += 8)
                        *reinterpret_cast<uint4 *>(A0 + term * AB + sw128_off(t, e0 * Fmt<FMT>::ESZ, kRows)) =
                            make_uint4(0u, 0u, 0u, 0u);
        }
        if (it + stride < items) prefetch(it + stride);
        if (!RESIDENT) {
            load_imgs(0);
            ok = wait_copy_pipe(&mb[NP], ph_cp, bar);
            if (!ok) break;
        }
        ok = run_mma(&mb[pp], ph_mma, bar, [&] {
            if constexpr (HC) tcfmt::gemm<FMT>(tb, A0, AB, Bz, IC, NO, KC, a.nterms);
            else tcfmt::gemm<FMT>(tb, A0, AB, Bz, IR, NO, KR, a.nterms);
        });
        if (!ok) break;
        if (ident_y) {
            // sigma_y = 0: T_y = I, row t = (g, y) already holds A'(x0+g, y, z') for all z'
            float2 *dst = (side == 0 ? a.Ap : a.Bq) + ((long)e * a.RS + rs) * n + (long)(x0 + g) * NN + yl * N;
            tmem_visit<NO>(tl, [&](int c0, const float *v) {
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
        tmem_visit<NO>(tl, [&](int c0, const float *v) {
            if (t < nval * N) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    tcfmt::st_c<FMT>(A0, AB, g * N + c0 / 2 + j, yl, v[2 * j], v[2 * j + 1]);
            }
        });
        }  // z-pass
        if (!RESIDENT) {
            load_imgs(1);
            ok = wait_copy_pipe(&mb[NP], ph_cp, bar);
            if (!ok) break;
        }
        ok = run_mma(&mb[pp], ph_mma, bar, [&] { tcfmt::gemm<FMT>(tb + NO, A0, AB, By, IC, NO, KC, a.nterms); });
        if (!ok) break;
        // row t = (g, z'): y' values -> global [x][y'][z']
        float2 *dstp = (side == 0 ? a.Ap : a.Bq) + ((long)e * a.RS + rs) * n + (long)(x0 + g) * NN + (yl & ~1);
        tmem_visit<NO>(tl + NO, [&](int c0, const float *v) {
            float2 h[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) h[j] = make_float2(v[2 * j], v[2 * j + 1]);
            store_pair<8>(dstp + (long)(c0 / 2) * N, h, N, t < nval * N);
        });
    }
    cta_teardown(tslot, NCOL, ok, a.err, mb, NP + 1, ps);
    return ok;
}

template <int N, int FMT>
__global__ void __launch_bounds__(kRows *NPipes<N, FMT>::A, 1) k_stage_a(TcArgs a)
{
    k_stage_a_body<N, FMT>(a, blockIdx, dim3(gridDim.x, gridDim.y, gridDim.z));
}

// Stage A of the Hermitian form (complex z-pass input, two points per slot)
template <int N, int FMT>
__global__ void __launch_bounds__(kRows *NPipes<N, FMT>::A, 1) k_stage_a_herm(TcArgs a)
{
    k_stage_a_body<N, FMT, true>(a, blockIdx, dim3(gridDim.x, gridDim.y, gridDim.z));
}

// ------------------------------------------------------------------ stage B
// grid (groups, RS).  A CTA holds T^p_x, T^q_x and F of its (r, s) when they
// fit next to the data operands (else it reloads one image slot per
// contraction); each of its NP pipelines loops over items (point e, tile of
// 128 (y, z) pencils): H = F_x ((T^p_x A') . (T^q_x B')).
template <int N, int FMT, bool HP = false, bool SH = false>
__device__ __forceinline__ bool k_stage_b_body(const TcArgs &a, const uint3 bid, const uint3 gdim,
                                               const uint16_t *bmap = nullptr, const Persist *ps = nullptr)
{
    using SM = Smem<N, FMT>;
    constexpr int NP = NPipes<N, FMT>::B, NT = SM::NT, AB = SM::AB, IC = SM::IC;
    constexpr bool RESIDENT = SM::RES_B;
    constexpr int KC = 2 * N, NO = 2 * N, NN = N * N, NT_TILES = (NN + kRows - 1) / kRows;
    constexpr uint32_t NCOL = pow2_cols(NP * 3 * NO);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align1024(smem_raw);
    const int pp = threadIdx.x / kRows, t = threadIdx.x % kRows, bar = 1 + pp;
    uint8_t *B0 = sm;  // image slots [T^p_x][T^q_x][F], NT terms each, or one reloaded slot
    uint8_t *A0 = B0 + (RESIDENT ? 3 : 1) * NT * IC + pp * NT * AB;
    __shared__ uint64_t mb[NP + 1];
    __shared__ uint32_t tslot;
    const int rs = bid.y;
    const long n = a.n;
    const int items = a.Ec * NT_TILES;
    const bool ident_x = a.idmask && (a.idmask[rs] & 1);
    cta_setup(&tslot, NCOL, mb, NP + 1, ps);
    const uint32_t tb = tslot + pp * 3 * NO, tl = lane_base(tb);
    uint32_t ph_mma = 0, ph_cp = 0;
    auto src_img = [&](int which) -> const uint8_t * {
        return which < 2 ? timg_at<FMT>(a.timg, N, rs, which, 0) : a.Fimg;
    };
    auto slot = [&](int which) -> uint8_t * { return RESIDENT ? B0 + which * NT * IC : B0; };
    auto load_images = [&](int first, int count) {
        if (threadIdx.x == 0) {
            mbar_expect_tx(&mb[NP], NT * IC * count);
            for (int w = first; w < first + count; ++w) copy_terms(slot(w), IC, src_img(w), IC, IC, NT, &mb[NP]);
        }
    };
    // this thread's pencil p0 + t, loaded with 16-byte accesses shared with the
    // neighbouring lane (raw; unpack_pair when used)
    float4 pa_raw[N / 2];
    auto load_pencil = [&](float4 *raw, const float2 *src, bool valid) {
        load_pair_raw<N>(raw, src - (t & 1), NN, valid);
    };
    const int stride = gdim.x * NP;
    int it = bid.x * NP + pp;
    if (it < items) {
        const int e = it / NT_TILES, p0 = (it % NT_TILES) * kRows;
        load_pencil(pa_raw, a.Ap + ((long)e * a.RS + rs) * n + p0 + t, p0 + t < NN);
    }
    bool ok = true;
    if (RESIDENT) {  // sigma_x = 0 needs only F
        if (ident_x) load_images(2, 1);
        else load_images(0, 3);
        ok = wait_copy_cta(&mb[NP], ph_cp);
    }
    // B' of this (r, s): its own grid, or A' at the reflected direction (same species)
    const float2 *bsrc = SH ? a.Ap : a.Bq;
    const long boff = SH ? ((long)bmap[rs] - rs) * n : 0;
    for (; it < items && ok; it += stride) {
        const int e = it / NT_TILES, p0 = (it % NT_TILES) * kRows;
        const bool valid = p0 + t < NN;
        const long gbase = ((long)e * a.RS + rs) * n + p0 + t;
        float4 pb_raw[N / 2];
        if (ident_x) {
            // sigma_x = 0: T^p_x = T^q_x = I, so P = A' . B' directly
            load_pencil(pb_raw, bsrc + (gbase + boff), valid);
            float2 pa[N], pb[N];
            unpack_pair<N>(pa, pa_raw);
            unpack_pair<N>(pb, pb_raw);
#pragma unroll
            for (int x = 0; x < N; x += 2) {
                const float2 u = HP ? make_float2(pa[x].x * pb[x].x, pa[x].y * pb[x].y)
                                        : make_float2(pa[x].x * pb[x].x - pa[x].y * pb[x].y,
                                                      pa[x].x * pb[x].y + pa[x].y * pb[x].x);
                const float2 v = HP ? make_float2(pa[x + 1].x * pb[x + 1].x, pa[x + 1].y * pb[x + 1].y)
                                        : make_float2(pa[x + 1].x * pb[x + 1].x - pa[x + 1].y * pb[x + 1].y,
                                                      pa[x + 1].x * pb[x + 1].y + pa[x + 1].y * pb[x + 1].x);
                tcfmt::st_c2<FMT>(A0, AB, t, x, u, v);
            }
            const int nx = it + stride;
            if (nx < items) {
                const int e2 = nx / NT_TILES, q0 = (nx % NT_TILES) * kRows;
                load_pencil(pa_raw, a.Ap + ((long)e2 * a.RS + rs) * n + q0 + t, q0 + t < NN);
            }
        } else {
        {
            float2 pa[N];
            unpack_pair<N>(pa, pa_raw);
#pragma unroll
            for (int x = 0; x < N; x += 2) tcfmt::st_c2<FMT>(A0, AB, t, x, pa[x], pa[x + 1]);
        }
        load_pencil(pb_raw, bsrc + (gbase + boff), valid);
        if (!RESIDENT) {
            load_images(0, 1);
            ok = wait_copy_pipe(&mb[NP], ph_cp, bar);
            if (!ok) break;
        }
        ok = run_mma(&mb[pp], ph_mma, bar, [&] { tcfmt::gemm<FMT>(tb, A0, AB, slot(0), IC, NO, KC, a.nterms); });
        if (!ok) break;
        {
            float2 pb[N];
            unpack_pair<N>(pb, pb_raw);
#pragma unroll
            for (int x = 0; x < N; x += 2) tcfmt::st_c2<FMT>(A0, AB, t, x, pb[x], pb[x + 1]);
        }
        const int nx = it + stride;
        if (nx < items) {
            const int e2 = nx / NT_TILES, q0 = (nx % NT_TILES) * kRows;
            load_pencil(pa_raw, a.Ap + ((long)e2 * a.RS + rs) * n + q0 + t, q0 + t < NN);
        }
        if (!RESIDENT) {
            load_images(1, 1);
            ok = wait_copy_pipe(&mb[NP], ph_cp, bar);
            if (!ok) break;
        }
        ok = run_mma(&mb[pp], ph_mma, bar,
                     [&] { tcfmt::gemm<FMT>(tb + NO, A0, AB, slot(1), IC, NO, KC, a.nterms); });
        if (!ok) break;
        // P = A . B (complex), back into the data operand
#pragma unroll
        for (int c0 = 0; c0 < NO; c0 += 16) {
            float va[16], vb[16];
            tmem_ld16x2(tl + c0, tl + NO + c0, va, vb);
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
                // literal: the complex product; Hermitian form: the two real
                // translates of each packed point multiply separately
                const float2 p0v =
                    HP ? make_float2(va[2 * j] * vb[2 * j], va[2 * j + 1] * vb[2 * j + 1])
                           : make_float2(va[2 * j] * vb[2 * j] - va[2 * j + 1] * vb[2 * j + 1],
                                         va[2 * j] * vb[2 * j + 1] + va[2 * j + 1] * vb[2 * j]);
                const float2 p1v =
                    HP ? make_float2(va[2 * j + 2] * vb[2 * j + 2], va[2 * j + 3] * vb[2 * j + 3])
                           : make_float2(va[2 * j + 2] * vb[2 * j + 2] - va[2 * j + 3] * vb[2 * j + 3],
                                         va[2 * j + 2] * vb[2 * j + 3] + va[2 * j + 3] * vb[2 * j + 2]);
                tcfmt::st_c2<FMT>(A0, AB, t, c0 / 2 + j, p0v, p1v);
            }
        }
        }  // translates along x
        if (!RESIDENT) {
            load_images(2, 1);
            ok = wait_copy_pipe(&mb[NP], ph_cp, bar);
            if (!ok) break;
        }
        ok = run_mma(&mb[pp], ph_mma, bar,
                     [&] { tcfmt::gemm<FMT>(tb + 2 * NO, A0, AB, slot(2), IC, NO, KC, a.nterms); });
        if (!ok) break;
        float2 *dstp = a.H + gbase - (t & 1);
        tmem_visit<NO>(tl + 2 * NO, [&](int c0, const float *v) {
            float2 h[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) h[j] = make_float2(v[2 * j], v[2 * j + 1]);
            store_pair<8>(dstp + (long)(c0 / 2) * NN, h, NN, valid);
        });
    }
    cta_teardown(tslot, NCOL, ok, a.err, mb, NP + 1, ps);
    return ok;
}

template <int N, int FMT>
__global__ void __launch_bounds__(kRows *NPipes<N, FMT>::B, 1) k_stage_b(TcArgs a)
{
    k_stage_b_body<N, FMT>(a, blockIdx, dim3(gridDim.x, gridDim.y, gridDim.z));
}

// Stage B of the Hermitian form (products of the packed real translates)
template <int N, int FMT>
__global__ void __launch_bounds__(kRows *NPipes<N, FMT>::B, 1) k_stage_b_herm(TcArgs a)
{
    k_stage_b_body<N, FMT, true>(a, blockIdx, dim3(gridDim.x, gridDim.y, gridDim.z));
}

// Stage B of a same-species pair: B' read from A' at the reflected direction
template <int N, int FMT, bool HP>
__global__ void __launch_bounds__(kRows *NPipes<N, FMT>::B, 1) k_stage_b_share(TcArgs a, const uint16_t *bmap)
{
    k_stage_b_body<N, FMT, HP, true>(a, blockIdx, dim3(gridDim.x, gridDim.y, gridDim.z), bmap);
}

// ------------------------------------------------------------------ stage C
// grid (plane groups, ceil(RSB / NP), Ec).  Each pipeline owns one block of
// (r, s) and, for every (r, s) of it, computes t3 = F_y F_z H on the tensor
// cores and QG_part += w_rs b_rs . t3 in registers; the next (r, s)'s H tile
// is prefetched into registers meanwhile.
template <int N, int FMT>
__device__ __forceinline__ bool k_stage_c_body(const TcArgs &a, const uint3 bid, const uint3 gdim,
                                               const Persist *ps = nullptr)
{
    using SM = Smem<N, FMT>;
    constexpr int NP = NPipes<N, FMT>::C, NT = SM::NT, AB = SM::AB, IC = SM::IC;
    constexpr int G = kRows / N, KC = 2 * N, NO = 2 * N, NN = N * N;
    constexpr int HPT = (G * NN / 2 + kRows - 1) / kRows;  // float4 (2 complex) per thread per tile
    constexpr bool PREFETCH = N <= 32;
    constexpr uint32_t NCOL = pow2_cols(NP * 2 * NO);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align1024(smem_raw);
    const int pp = threadIdx.x / kRows, t = threadIdx.x % kRows, bar = 1 + pp;
    uint8_t *Bf = sm;  // F, NT terms IC apart
    uint8_t *A0 = Bf + NT * IC + pp * NT * AB;
    __shared__ uint64_t mb[NP + 1];
    __shared__ uint32_t tslot;
    const int x0 = bid.x * G, rb = bid.y * NP + pp, e = bid.z;
    const int nval = min(G, N - x0);
    const long n = a.n;
    cta_setup(&tslot, NCOL, mb, NP + 1, ps);
    const uint32_t tb = tslot + pp * 2 * NO, tl = lane_base(tb);
    uint32_t ph_mma = 0, ph_cp = 0;
    if (threadIdx.x == 0) {
        mbar_expect_tx(&mb[NP], NT * IC);
        copy_terms(Bf, IC, a.Fimg, IC, IC, NT, &mb[NP]);
    }
    const int g = t / N, yl = t % N;
    float2 acc[N];
#pragma unroll
    for (int k = 0; k < N; ++k) acc[k] = make_float2(0.f, 0.f);
    const int rs0 = rb * a.rs_per_block, rs1 = rb < a.rsb ? min(a.RS, rs0 + a.rs_per_block) : rs0;
    float4 hp[PREFETCH ? HPT : 1];
    auto tile = [&](int rs) {
        return reinterpret_cast<const float4 *>(a.H + ((long)e * a.RS + rs) * n + (long)x0 * NN);
    };
    if (PREFETCH && a.collapse_M == 1 && rs0 < rs1) {
        const float4 *src = tile(rs0);
#pragma unroll
        for (int j = 0; j < HPT; ++j) {
            const int i = t + kRows * j;
            hp[j] = (2 * i < nval * NN) ? src[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    bool ok = wait_copy_cta(&mb[NP], ph_cp);
    // sigma collapse: b_rs and w_rs do not depend on s, so the M tiles of one
    // radial node are summed (FP32, in registers) and transformed once
    constexpr int HS = (G * NN / 2 + kRows - 1) / kRows;  // float4 per thread per tile
    for (int r0 = rs0; a.collapse_M > 1 && r0 < rs1 && ok; r0 += a.collapse_M) {
        float4 hs[HS];
#pragma unroll
        for (int j = 0; j < HS; ++j) hs[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int sd = 0; sd < a.collapse_M; ++sd) {
            const float4 *src = tile(r0 + sd);
#pragma unroll
            for (int j = 0; j < HS; ++j) {
                const int i = t + kRows * j;
                if (2 * i < nval * NN) {
                    const float4 v = src[i];
                    hs[j].x += v.x;
                    hs[j].y += v.y;
                    hs[j].z += v.z;
                    hs[j].w += v.w;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < HS; ++j) {
            const int i = t + kRows * j;
            if (2 * i < nval * NN) tcfmt::st_f4<FMT>(A0, AB, (2 * i) / N, 2 * ((2 * i) % N), hs[j]);
        }
        ok = run_mma(&mb[pp], ph_mma, bar, [&] { tcfmt::gemm<FMT>(tb, A0, AB, Bf, IC, NO, KC, a.nterms); });
        if (!ok) break;
        tmem_visit<NO>(tl, [&](int c0, const float *v) {
            if (t < nval * N) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    tcfmt::st_c<FMT>(A0, AB, g * N + c0 / 2 + j, yl, v[2 * j], v[2 * j + 1]);
            }
        });
        ok = run_mma(&mb[pp], ph_mma, bar, [&] { tcfmt::gemm<FMT>(tb + NO, A0, AB, Bf, IC, NO, KC, a.nterms); });
        if (!ok) break;
        const float wr = (float)a.w[r0];
        const float2 *brsp = a.b32 + (long)r0 * n + (long)(x0 + g) * NN + (yl & ~1);
        tmem_visit<NO>(tl + NO, [&](int c0, const float *v) {
            float2 bb[8];
            load_pair<8>(bb, brsp + (long)(c0 / 2) * N, N, t < nval * N);
            if (t < nval * N) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int ky = c0 / 2 + j;
                    const float tr = v[2 * j], ti = v[2 * j + 1];
                    acc[ky].x = fmaf(wr, bb[j].x * tr - bb[j].y * ti, acc[ky].x);
                    acc[ky].y = fmaf(wr, bb[j].x * ti + bb[j].y * tr, acc[ky].y);
                }
            }
        });
    }
    for (int rs = rs0; a.collapse_M == 1 && rs < rs1 && ok; ++rs) {
        // rows (g, y), K = z (complex): contiguous planes; float4 i holds complex 2i, 2i+1
        if constexpr (PREFETCH) {
#pragma unroll
            for (int j = 0; j < HPT; ++j) {
                const int i = t + kRows * j;
                if (2 * i < nval * NN) tcfmt::st_f4<FMT>(A0, AB, (2 * i) / N, 2 * ((2 * i) % N), hp[j]);
            }
            if (rs + 1 < rs1) {
                const float4 *src = tile(rs + 1);
#pragma unroll
                for (int j = 0; j < HPT; ++j) {
                    const int i = t + kRows * j;
                    hp[j] = (2 * i < nval * NN) ? src[i] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        } else {
            const float4 *src = tile(rs);
            for (int i = t; i < nval * NN / 2; i += kRows)
                tcfmt::st_f4<FMT>(A0, AB, (2 * i) / N, 2 * ((2 * i) % N), src[i]);
        }
        ok = run_mma(&mb[pp], ph_mma, bar, [&] { tcfmt::gemm<FMT>(tb, A0, AB, Bf, IC, NO, KC, a.nterms); });
        if (!ok) break;
        tmem_visit<NO>(tl, [&](int c0, const float *v) {
            if (t < nval * N) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    tcfmt::st_c<FMT>(A0, AB, g * N + c0 / 2 + j, yl, v[2 * j], v[2 * j + 1]);
            }
        });
        ok = run_mma(&mb[pp], ph_mma, bar, [&] { tcfmt::gemm<FMT>(tb + NO, A0, AB, Bf, IC, NO, KC, a.nterms); });
        if (!ok) break;
        // row t = (g, kz): t3(kx0+g, ky, kz) for all ky
        const float wr = (float)a.w[rs];
        const float2 *brsp = a.b32 + (long)rs * n + (long)(x0 + g) * NN + (yl & ~1);
        tmem_visit<NO>(tl + NO, [&](int c0, const float *v) {
            float2 bb[8];
            load_pair<8>(bb, brsp + (long)(c0 / 2) * N, N, t < nval * N);
            if (t < nval * N) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int ky = c0 / 2 + j;
                    const float tr = v[2 * j], ti = v[2 * j + 1];
                    acc[ky].x = fmaf(wr, bb[j].x * tr - bb[j].y * ti, acc[ky].x);
                    acc[ky].y = fmaf(wr, bb[j].x * ti + bb[j].y * tr, acc[ky].y);
                }
            }
        });
    }
    if (ok && rb < a.rsb) {  // uniform over the pipeline
        float2 *dstp = a.QGp + ((long)e * a.rsb + rb) * n + (long)(x0 + g) * NN + (yl & ~1);
        store_pair<N>(dstp, acc, N, t < nval * N);
    }
    cta_teardown(tslot, NCOL, ok, a.err, mb, NP + 1, ps);
    return ok;
}

template <int N, int FMT>
__global__ void __launch_bounds__(kRows *NPipes<N, FMT>::C, 1) k_stage_c(TcArgs a)
{
    k_stage_c_body<N, FMT>(a, blockIdx, dim3(gridDim.x, gridDim.y, gridDim.z));
}


unsigned nblk(long total, int t) { return (unsigned)((total + t - 1) / t); }

// Workspace of a tensor-core plan:
//   F [maxP][S][n] | QG [S*S][maxP][n] (complex double-floats, float4) | Ap, Bq, H [Emax][RS][n] f2 |
//   QGp [Emax][RSBmax][n] f2 | H2 [Emax][RS][n] f2 (when H is double-buffered)
struct TcWs {
    float4 *F, *QG;  // QG: pair p S + q at QG + (p S + q) qg_stride
    long qg_stride;
    float2 *Ap, *Bq, *H, *QGp;
    float2 *H2;  // the second H slot (H itself when H is not double-buffered)
};

TcWs ws_of(const dgfs_plan_s *plan)
{
    const TcState *ts = reinterpret_cast<const TcState *>(plan->tc);
    const long n = (long)plan->N * plan->N * plan->N, RS = (long)plan->Nrho * plan->M;
    TcWs w;
    w.F = reinterpret_cast<float4 *>(plan->ws);
    w.QG = w.F + (long)plan->max_points * plan->S * n;
    w.qg_stride = (long)plan->max_points * n;
    w.Ap = reinterpret_cast<float2 *>(w.QG + (long)plan->S * plan->S * w.qg_stride);
    w.Bq = w.Ap + (long)ts->chunk_max * RS * n;
    w.H = w.Bq + (long)ts->chunk_max * RS * n;
    w.QGp = w.H + (long)ts->chunk_max * RS * n;
    w.H2 = ts->hslots == 2 ? w.QGp + (long)ts->chunk_max * ts->rsb_max * n : w.H;
    return w;
}


// accumulation blocks of (r, s); with the sigma collapse every block holds whole radial nodes
int rs_blocks(const dgfs_plan_s *plan)
{
    const TcState *ts = reinterpret_cast<const TcState *>(plan->tc);
    if (!plan->collapse) return ts->rsb;
    const int per = (plan->Nrho + ts->rsb - 1) / ts->rsb;
    return (plan->Nrho + per - 1) / per;
}

// Arguments of one job: species pair (p, q), points [pt0, pt0 + Ec).
TcArgs job_args(const dgfs_plan_s *plan, const void *f, int p, int q, int pt0, int Ec)
{
    const TcState *ts = reinterpret_cast<const TcState *>(plan->tc);
    const TcWs w = ws_of(plan);
    const int RS = plan->Nrho * plan->M, RSB = rs_blocks(plan);
    const PairTables &pt = plan->pairs[p * plan->S + q];
    TcArgs a{};
    a.n = (long)plan->N * plan->N * plan->N;
    a.S = plan->S;
    a.RS = RS;
    a.nterms = ts->nterms;
    a.rsb = RSB;
    a.rs_per_block = plan->collapse ? plan->M * ((plan->Nrho + ts->rsb - 1) / ts->rsb) : (RS + RSB - 1) / RSB;
    a.collapse_M = plan->collapse ? plan->M : 1;
    a.f = reinterpret_cast<const float *>(f);
    a.Ap = w.Ap;
    a.Bq = w.Bq;
    a.H = w.H;
    a.QGp = w.QGp;
    a.Fimg = ts->Fimg;
    a.err = ts->err;
    a.p = p;
    a.q = q;
    a.timg = reinterpret_cast<const uint8_t *>(pt.tmat);
    a.b32 = pt.b32;
    a.w = pt.w;
    a.idmask = ts->skip_identity ? ts->idmask : nullptr;
    a.pt0 = pt0;
    a.Ec = Ec;
    return a;
}

// The translate sharing of a same-species pair (plain calls only)
Share job_share(const dgfs_plan_s *plan, int p, int q)
{
    const TcState *ts = reinterpret_cast<const TcState *>(plan->tc);
    Share sh;
    sh.on = p == q && ts->bmap != nullptr;
    sh.bmap = sh.on ? ts->bmap : nullptr;
    return sh;
}

// Grids of the three stage kernels for one job.
template <int N, int FMT>
void job_grids(const dgfs_plan_s *plan, int Ec, bool share, dim3 &gA, dim3 &gB, dim3 &gC)
{
    const TcState *ts = reinterpret_cast<const TcState *>(plan->tc);
    const int RS = plan->Nrho * plan->M, RSB = rs_blocks(plan);
    constexpr int G = kRows / N;
    gA = dim3(ts->groups_a, RS, share ? 1 : 2);
    gB = dim3(ts->groups_b, RS);
    gC = dim3((N + G - 1) / G, (RSB + NPipes<N, FMT>::C - 1) / NPipes<N, FMT>::C, Ec);
}

}  // namespace
}  // namespace dgfs

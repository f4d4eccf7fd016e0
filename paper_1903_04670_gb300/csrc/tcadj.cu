// Tensor-core adjoint of the bilinear collision map (f_p, f_q) -> Q^(pq)
// (bilinearity of Eq. (7); the forward is Algorithm 2).
//
// With D the unnormalised 3-D DFT, the translates A_rs = T+_rs f_p, B_rs = T-_rs f_q
// (T = D^-1 diag(phi) D, phi separable per axis) and
//   Q = beta Re( D^-1 sum_rs w_rs b_rs . D(A_rs . B_rs) - f_p . D^-1(c . D f_q) ),
// an upstream gradient g (real) gives, since T^H = D^-1 diag(conj phi) D,
//   dL/df_p = beta Re D^-1 sum_rs w_rs conj(phi+_rs) . D( conj(B_rs) . V_rs ) - loss term,
//   dL/df_q = beta Re D^-1 sum_rs w_rs conj(phi-_rs) . D( conj(A_rs) . V_rs ) - loss term,
//   V_rs = D^-1( conj(b_rs) . D g ).
// So the (r, s) loop has the shape of the forward's: a per-(r, s) 3-D transform
// of a product of two grids, multiplied by a per-(r, s) table in k-space and
// summed over (r, s).  It runs on the forward's stage kernels plus two:
//   stage A (forward kernel):  A' = T+_y T+_z f_p, B' = T-_y T-_z f_q
//   stage Z (here):            W  = F_y F_z (b_rs . conj(G)),  G = D g,
//                              so that conj(F_x W) = n V_rs (unnormalised inverse
//                              as the conjugate of the forward DFT image)
//   stage B adjoint (here):    X = F_x W, A = T+_x A', B = T-_x B';
//                              dot_rs += Re sum X A B  (= n Re<V, A B>, for d/d omega),
//                              H_p = F_x conj(B X), H_q = F_x conj(A X); a
//                              same-species pair reads B' from A' at the reflected
//                              direction, as the forward's stage B
//   stage C (forward kernel) with the table w_rs conj(phi_rs(k)) in place of
//                              w_rs b_rs: the (r, s) sums of both gradients
// The parts outside the (r, s) loop (D g, D(g f_p), the loss-term adjoint, the
// final inverse transforms and the omega reduction) run in FP64 (adj64.cu).
// Every wait in the stage kernels is bounded, as in the forward.
#include "tcstage.cuh"

namespace dgfs {
namespace {

// ------------------------------------------------------------------ stage Z
// grid (plane groups, ceil(RSB / NP), Ec), as stage C.  Each pipeline loads the
// tile of G = D g of its point and x-planes once, then for every (r, s) of its
// block forms b_rs . conj(G), applies F_z and F_y on the tensor cores and
// stores W_rs in the natural layout [x][y][z] for the x-pencils of stage B.
template <int N, int FMT>
__device__ __forceinline__ bool k_stage_z_body(const TcArgs &a, const double2 *Gg, const uint3 bid)
{
    using SM = Smem<N, FMT>;
    constexpr int NP = NPipes<N, FMT>::C, NT = SM::NT, AB = SM::AB, IC = SM::IC;
    constexpr int G = kRows / N, KC = 2 * N, NO = 2 * N, NN = N * N;
    constexpr int HPT = (G * NN / 2 + kRows - 1) / kRows;  // float4 (2 complex) per thread per tile
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
    cta_setup(&tslot, NCOL, mb, NP + 1);
    const uint32_t tb = tslot + pp * 2 * NO, tl = lane_base(tb);
    uint32_t ph_mma = 0, ph_cp = 0;
    if (threadIdx.x == 0) {
        mbar_expect_tx(&mb[NP], NT * IC);
        copy_terms(Bf, IC, a.Fimg, IC, IC, NT, &mb[NP]);
    }
    const int g = t / N, yl = t % N;
    const int rs0 = rb * a.rs_per_block, rs1 = rb < a.rsb ? min(a.RS, rs0 + a.rs_per_block) : rs0;
    // this thread's elements of the G tile: complex 2i, 2i + 1, i = t + 128 j
    float4 gt[HPT];
    const double2 *gsrc = Gg + (long)e * n + (long)x0 * NN;
#pragma unroll
    for (int j = 0; j < HPT; ++j) {
        const int i = t + kRows * j;
        gt[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (rs0 < rs1 && 2 * i < nval * NN) {
            const double2 u = gsrc[2 * i], v = gsrc[2 * i + 1];
            gt[j] = make_float4((float)u.x, (float)u.y, (float)v.x, (float)v.y);
        }
    }
    float4 bp[HPT];
    auto load_b = [&](int rs) {
        const float4 *src = reinterpret_cast<const float4 *>(a.b32 + (long)rs * n + (long)x0 * NN);
#pragma unroll
        for (int j = 0; j < HPT; ++j) {
            const int i = t + kRows * j;
            bp[j] = (2 * i < nval * NN) ? src[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    if (rs0 < rs1) load_b(rs0);
    bool ok = wait_copy_cta(&mb[NP], ph_cp);
    for (int rs = rs0; rs < rs1 && ok; ++rs) {
        // rows (g, y), K = z (complex): b . conj(G)
#pragma unroll
        for (int j = 0; j < HPT; ++j) {
            const int i = t + kRows * j;
            if (2 * i < nval * NN) {
                const float4 b = bp[j], u = gt[j];
                const float4 v = make_float4(b.x * u.x + b.y * u.y, b.y * u.x - b.x * u.y, b.z * u.z + b.w * u.w,
                                             b.w * u.z - b.z * u.w);
                tcfmt::st_f4<FMT>(A0, AB, (2 * i) / N, 2 * ((2 * i) % N), v);
            }
        }
        if (rs + 1 < rs1) load_b(rs + 1);
        ok = run_mma(&mb[pp], ph_mma, bar, [&] { tcfmt::gemm<FMT>(tb, A0, AB, Bf, IC, NO, KC, a.nterms); });
        if (!ok) break;
        // transpose within each plane: row (g, y) holds z' -> rows (g, z'), K = y
        tmem_visit<NO>(tl, [&](int c0, const float *v) {
            if (t < nval * N) {
#pragma unroll
                for (int j = 0; j < 8; ++j) tcfmt::st_c<FMT>(A0, AB, g * N + c0 / 2 + j, yl, v[2 * j], v[2 * j + 1]);
            }
        });
        ok = run_mma(&mb[pp], ph_mma, bar, [&] { tcfmt::gemm<FMT>(tb + NO, A0, AB, Bf, IC, NO, KC, a.nterms); });
        if (!ok) break;
        // row t = (g, z'): y' values -> W [x][y'][z']
        float2 *dstp = a.H + ((long)e * a.RS + rs) * n + (long)(x0 + g) * NN + (yl & ~1);
        tmem_visit<NO>(tl + NO, [&](int c0, const float *v) {
            float2 h[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) h[j] = make_float2(v[2 * j], v[2 * j + 1]);
            store_pair<8>(dstp + (long)(c0 / 2) * N, h, N, t < nval * N);
        });
    }
    cta_teardown(tslot, NCOL, ok, a.err, mb, NP + 1);
    return ok;
}

template <int N, int FMT>
__global__ void __launch_bounds__(kRows *NPipes<N, FMT>::C, 1) k_stage_z(TcArgs a, const double2 *Gg)
{
    k_stage_z_body<N, FMT>(a, Gg, blockIdx);
}

// --------------------------------------------------------- stage B, adjoint
// grid (groups, RS).  A CTA holds T+_x, T-_x and F of its (r, s); each
// pipeline loops over items (point e, tile of 128 (y, z) pencils):
//   X = F_x W,  A = T+_x A',  B = T-_x B'          (three contractions)
//   dot_rs(e) += Re sum_x X A B
//   H_p = F_x conj(B X)  -> written over W (a.H)
//   H_q = F_x conj(A X)  -> written over B' (a.Bq)
// Every item reads its pencils before it writes the same pencils, and no other
// item touches them, so the outputs can overwrite the inputs.  A same-species
// pair (SH) reads B' from A' at the reflected direction bmap[rs] (stage A then
// computes the A side only, as in the forward); A' is only read here, and its
// B' buffer is free for H_q.
template <int N, int FMT, bool SH>
__device__ __forceinline__ bool k_stage_b_adj_body(const TcArgs &a, double *dots, const uint16_t *bmap,
                                                   const uint3 bid, const uint3 gdim)
{
    using SM = Smem<N, FMT>;
    constexpr int NP = NPipes<N, FMT>::B, NT = SM::NT, AB = SM::AB, IC = SM::IC;
    constexpr bool RESIDENT = SM::RES_B;
    constexpr int KC = 2 * N, NO = 2 * N, NN = N * N, NT_TILES = (NN + kRows - 1) / kRows;
    constexpr uint32_t NCOL = pow2_cols(NP * 3 * NO);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = align1024(smem_raw);
    const int pp = threadIdx.x / kRows, t = threadIdx.x % kRows, bar = 1 + pp;
    uint8_t *B0 = sm;  // image slots [T+_x][T-_x][F], NT terms each, or one reloaded slot
    uint8_t *A0 = B0 + (RESIDENT ? 3 : 1) * NT * IC + pp * NT * AB;
    __shared__ uint64_t mb[NP + 1];
    __shared__ uint32_t tslot;
    const int rs = bid.y;
    const long n = a.n;
    const int items = a.Ec * NT_TILES;
    cta_setup(&tslot, NCOL, mb, NP + 1);
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
    // one contraction of the data operand with image `which` into TMEM column offset d
    auto contract = [&](uint32_t d, int which) -> bool {
        if (!RESIDENT) {
            load_images(which, 1);
            if (!wait_copy_pipe(&mb[NP], ph_cp, bar)) return false;
        }
        return run_mma(&mb[pp], ph_mma, bar,
                       [&] { tcfmt::gemm<FMT>(tb + d, A0, AB, slot(which), IC, NO, KC, a.nterms); });
    };
    auto load_pencil = [&](float4 *raw, const float2 *src, bool valid) {
        load_pair_raw<N>(raw, src - (t & 1), NN, valid);
    };
    auto stage_pencil = [&](const float4 *raw) {
        float2 v[N];
        unpack_pair<N>(v, raw);
#pragma unroll
        for (int x = 0; x < N; x += 2) tcfmt::st_c2<FMT>(A0, AB, t, x, v[x], v[x + 1]);
    };
    auto store_out = [&](float2 *dst, bool valid) {
        tmem_visit<NO>(tl + 2 * NO, [&](int c0, const float *v) {
            float2 h[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) h[j] = make_float2(v[2 * j], v[2 * j + 1]);
            store_pair<8>(dst + (long)(c0 / 2) * NN, h, NN, valid);
        });
    };
    const int stride = gdim.x * NP;
    int it = bid.x * NP + pp;
    float4 pw_raw[N / 2];
    if (it < items) {
        const int e = it / NT_TILES, p0 = (it % NT_TILES) * kRows;
        load_pencil(pw_raw, a.H + ((long)e * a.RS + rs) * n + p0 + t, p0 + t < NN);
    }
    bool ok = true;
    if (RESIDENT) {
        load_images(0, 3);
        ok = wait_copy_cta(&mb[NP], ph_cp);
    }
    for (; it < items && ok; it += stride) {
        const int e = it / NT_TILES, p0 = (it % NT_TILES) * kRows;
        const bool valid = p0 + t < NN;
        const long gbase = ((long)e * a.RS + rs) * n + p0 + t;
        float4 pa_raw[N / 2];
        // X = F_x W (region 0)
        stage_pencil(pw_raw);
        load_pencil(pa_raw, a.Ap + gbase, valid);
        ok = contract(0, 2);
        if (!ok) break;
        // A = T+_x A' (region 1)
        stage_pencil(pa_raw);
        load_pencil(pa_raw, (SH ? a.Ap + ((long)bmap[rs] - rs) * n : a.Bq) + gbase, valid);
        ok = contract(NO, 0);
        if (!ok) break;
        // B = T-_x B' (region 2)
        stage_pencil(pa_raw);
        const int nx = it + stride;
        if (nx < items) {
            const int e2 = nx / NT_TILES, q0 = (nx % NT_TILES) * kRows;
            load_pencil(pw_raw, a.H + ((long)e2 * a.RS + rs) * n + q0 + t, q0 + t < NN);
        }
        ok = contract(2 * NO, 1);
        if (!ok) break;
        // dot and P_p = conj(B X) into the data operand
        float dot = 0.f;
#pragma unroll
        for (int c0 = 0; c0 < NO; c0 += 16) {
            float vx[16], va[16], vb[16];
            tmem_ld16x2(tl + c0, tl + NO + c0, vx, va);
            tmem_ld16(tl + 2 * NO + c0, vb);
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
                float2 pr[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = 2 * (j + h);
                    const float xr = vx[k], xi = vx[k + 1], ar = va[k], ai = va[k + 1], br = vb[k], bi = vb[k + 1];
                    const float bxr = br * xr - bi * xi, bxi = br * xi + bi * xr;  // B X
                    dot = fmaf(ar, bxr, fmaf(-ai, bxi, dot));                      // Re(A B X)
                    pr[h] = make_float2(bxr, -bxi);
                }
                tcfmt::st_c2<FMT>(A0, AB, t, c0 / 2 + j, pr[0], pr[1]);
            }
        }
        ok = contract(2 * NO, 2);  // H_p = F_x P_p (region 2; B is consumed)
        if (!ok) break;
        store_out(a.H + gbase - (t & 1), valid);
        // P_q = conj(A X)
#pragma unroll
        for (int c0 = 0; c0 < NO; c0 += 16) {
            float vx[16], va[16];
            tmem_ld16x2(tl + c0, tl + NO + c0, vx, va);
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
                float2 pr[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = 2 * (j + h);
                    const float xr = vx[k], xi = vx[k + 1], ar = va[k], ai = va[k + 1];
                    pr[h] = make_float2(ar * xr - ai * xi, -(ar * xi + ai * xr));
                }
                tcfmt::st_c2<FMT>(A0, AB, t, c0 / 2 + j, pr[0], pr[1]);
            }
        }
        ok = contract(2 * NO, 2);  // H_q = F_x P_q
        if (!ok) break;
        store_out(a.Bq + gbase - (t & 1), valid);
        // this warp's pencils belong to one (point, r, s)
        if (!valid) dot = 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(dots + (long)e * a.RS + rs, (double)dot);
    }
    cta_teardown(tslot, NCOL, ok, a.err, mb, NP + 1);
    return ok;
}

template <int N, int FMT, bool SH>
__global__ void __launch_bounds__(kRows *NPipes<N, FMT>::B, 1)
    k_stage_b_adj(TcArgs a, double *dots, const uint16_t *bmap)
{
    k_stage_b_adj_body<N, FMT, SH>(a, dots, bmap, blockIdx, dim3(gridDim.x, gridDim.y, gridDim.z));
}

// out[side][rs][k] = conj(phi_side,x(kx) phi_side,y(ky) phi_side,z(kz)) in FP32, from
// the FP64 per-axis phases [RS][2][3][N] (the transposed translates' k-space factor)
__global__ void k_adjmul(float2 *out, const double2 *phase, int N, int RS)
{
    const long n = (long)N * N * N;
    const long total = 2L * RS * n;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const long k = i % n;
    const int rs = (int)((i / n) % RS), side = (int)(i / (n * RS));
    const int kx = (int)(k / ((long)N * N)), ky = (int)((k / N) % N), kz = (int)(k % N);
    const double2 *ph = phase + ((long)rs * 2 + side) * 3 * N;
    const double2 px = ph[kx], py = ph[N + ky], pz = ph[2 * N + kz];
    const double xyr = px.x * py.x - px.y * py.y, xyi = px.x * py.y + px.y * py.x;
    const double r = xyr * pz.x - xyi * pz.y, im = xyr * pz.y + xyi * pz.x;
    out[i] = make_float2((float)r, (float)-im);
}

// acc[e][k] = sum_rb QGp[e][rb][k] in FP64
__global__ void k_sum_partials_d(double2 *acc, const float2 *QGp, int rsb, long n, int E)
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
    acc[i] = make_double2(sx, sy);
}

constexpr int kZBlock = 8;  // (r, s) per stage Z pipeline

dgfs_status ensure_adjmul(dgfs_plan_s *plan, TcState *ts, cudaStream_t st)
{
    if (ts->adjmul) return DGFS_OK;
    const int S = plan->S, RS = plan->Nrho * plan->M;
    const long n = (long)plan->N * plan->N * plan->N;
    const long per_pair = 2L * RS * n;
    DGFS_CUDA(dev_malloc(&ts->adjmul, sizeof(float2) * per_pair * S * S));
    for (int pq = 0; pq < S * S; ++pq) {
        k_adjmul<<<nblk(per_pair, 256), 256, 0, st>>>(ts->adjmul + pq * per_pair, plan->pairs[pq].phase, plan->N,
                                                       RS);
        DGFS_LAUNCHED(plan);
    }
    return DGFS_OK;
}

template <int N, int FMT>
dgfs_status backward_n(dgfs_plan_s *plan, int P, const void *f, const void *dQ, void *df, double *domega,
                       int domega_on_host, cudaStream_t st)
{
    using SM = Smem<N, FMT>;
    TcState *ts = reinterpret_cast<TcState *>(plan->tc);
    const int S = plan->S, RS = plan->Nrho * plan->M, E = ts->chunk;
    const long n = (long)N * N * N;
    const int lblk = adj64_nblk(N);
    const TcWs w = ws_of(plan);
    DGFS_TRY(ensure_adjmul(plan, ts, st));
    DGFS_CUDA(cudaFuncSetAttribute(k_stage_a<N, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::A));
    DGFS_CUDA(cudaFuncSetAttribute(k_stage_z<N, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::C));
    DGFS_CUDA(
        cudaFuncSetAttribute(k_stage_b_adj<N, FMT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::B));
    DGFS_CUDA(
        cudaFuncSetAttribute(k_stage_b_adj<N, FMT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::B));
    DGFS_CUDA(cudaFuncSetAttribute(k_stage_c<N, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::C));

    // per call: F [P][S][n] | Gg, GF, L, Lw, Y [S*S][E][n], ACC [S*S][2][E][n] (complex FP64) |
    //           acc [S*S][2][E][n] | dots [E][RS] | lossdots [S*S][E][2][lblk] | dom [S*S]
    const long SS = (long)S * S, En = (long)E * n;
    const size_t bytes = sizeof(double2) * ((size_t)P * S * n + 7 * SS * En) +
                         sizeof(double) * (2 * SS * En + (size_t)E * RS + 2 * SS * E * lblk + SS);
    void *own = nullptr;
    DGFS_CUDA(dev_malloc_async(&own, bytes, st));
    double2 *F = reinterpret_cast<double2 *>(own);
    double2 *Gg = F + (long)P * S * n, *GF = Gg + SS * En, *Lb = GF + SS * En, *Lw = Lb + SS * En;
    double2 *Y = Lw + SS * En, *ACC = Y + SS * En;
    double *acc = reinterpret_cast<double *>(ACC + 2 * SS * En);
    double *dots = acc + 2 * SS * En, *lossdots = dots + (long)E * RS, *dom = lossdots + 2 * SS * E * lblk;

    auto run = [&]() -> dgfs_status {
        DGFS_CUDA(cudaMemsetAsync(df, 0, sizeof(float) * (size_t)P * S * n, st));
        DGFS_TRY(fp64_forward(plan, P, f, F, st));
        // (r, s) blocks of stages Z and C: the plan's block count, no sigma collapse
        const int rsb = std::min(ts->rsb, RS), rpb = (RS + rsb - 1) / rsb;
        const int RSB = (RS + rpb - 1) / rpb;
        constexpr int G = kRows / N;
        const dim3 gB(ts->groups_b, RS);
        for (int pt0 = 0; pt0 < P; pt0 += E) {
            const int Ec = std::min(E, P - pt0);
            const long ecn = (long)Ec * n;  // one pair slot of this chunk's buffers
            AdjPart x;
            x.pt0 = pt0;
            x.Ec = Ec;
            x.f32 = 1;
            x.want_omega = domega ? 1 : 0;
            x.npairs = (int)SS;
            for (int k = 0; k < SS; ++k) x.pairs[k] = k;
            x.f = f;
            x.dQ = dQ;
            x.df = df;
            x.F = F;
            x.Gg = Gg;
            x.GF = GF;
            x.L = Lb;
            x.Lw = Lw;
            x.Y = Y;
            x.accp = acc;
            x.lossdots = lossdots;
            // G = D g and D(g f_p) of every pair
            DGFS_TRY(adj64_part(plan, ADJ_PART_G, x, st));
            for (int p = 0; p < S; ++p)
                for (int q = 0; q < S; ++q) {
                    const long pq = p * S + q;
                    TcArgs a = job_args(plan, f, p, q, pt0, Ec);
                    const Share sh = job_share(plan, p, q);
                    const dim3 gA(ts->groups_a, RS, sh.on ? 1 : 2);
                    a.collapse_M = 1;
                    a.rsb = RSB;
                    a.rs_per_block = rpb;
                    const dim3 gC((N + G - 1) / G, (RSB + NPipes<N, FMT>::C - 1) / NPipes<N, FMT>::C, Ec);
                    {
                        ProfScope ps(plan, "tc_stage_a", st);
                        k_stage_a<N, FMT><<<gA, kRows * NPipes<N, FMT>::A, SM::A, st>>>(a);
                    }
                    DGFS_LAUNCHED(plan);
                    {
                        // stage Z's (r, s) are independent (no accumulation): blocks of
                        // kZBlock, so that its grid fills the SMs at a few points too
                        TcArgs z = a;
                        z.rs_per_block = std::min(kZBlock, RS);
                        z.rsb = (RS + z.rs_per_block - 1) / z.rs_per_block;
                        const dim3 gZ((N + G - 1) / G, (z.rsb + NPipes<N, FMT>::C - 1) / NPipes<N, FMT>::C, Ec);
                        ProfScope ps(plan, "tc_adj_stage_z", st);
                        k_stage_z<N, FMT><<<gZ, kRows * NPipes<N, FMT>::C, SM::C, st>>>(z, Gg + pq * ecn);
                    }
                    DGFS_LAUNCHED(plan);
                    if (domega) DGFS_CUDA(cudaMemsetAsync(dots, 0, sizeof(double) * (size_t)Ec * RS, st));
                    {
                        ProfScope ps(plan, "tc_adj_stage_b", st);
                        if (sh.on)
                            k_stage_b_adj<N, FMT, true><<<gB, kRows * NPipes<N, FMT>::B, SM::B, st>>>(a, dots, sh.bmap);
                        else
                            k_stage_b_adj<N, FMT, false><<<gB, kRows * NPipes<N, FMT>::B, SM::B, st>>>(a, dots, nullptr);
                    }
                    DGFS_LAUNCHED(plan);
                    // the two (r, s) sums: H_p (in H) with conj(phi+), H_q (in B') with conj(phi-)
                    for (int side = 0; side < 2; ++side) {
                        TcArgs c = a;
                        c.H = side == 0 ? w.H : w.Bq;
                        c.b32 = ts->adjmul + (pq * 2 + side) * (long)RS * n;
                        {
                            ProfScope ps(plan, "tc_stage_c", st);
                            k_stage_c<N, FMT><<<gC, kRows * NPipes<N, FMT>::C, SM::C, st>>>(c);
                        }
                        DGFS_LAUNCHED(plan);
                        {
                            ProfScope ps(plan, "tc_adj_sum", st);
                            k_sum_partials_d<<<nblk(ecn, 256), 256, 0, st>>>(ACC + (pq * 2 + side) * ecn, w.QGp, RSB,
                                                                              n, Ec);
                        }
                        DGFS_LAUNCHED(plan);
                    }
                    // dots hold n Re<V, A B> per (point, r, s); the reduction waits for
                    // the loss dots of this pair below
                    if (domega) {
                        // keep this pair's dots: the next pair's stage B overwrites the buffer
                        DGFS_TRY(adj64_omega_gain(plan, dom, p, q, dots, 1.0 / (double)n, Ec, pt0 > 0 ? 1 : 0, st));
                    }
                }
            // acc = n Re ifft3_u(sum) of every pair and side: the FP64 adjoint's scale (n^3
            // times the gain sum); the stage outputs carry n (V from the unnormalised
            // conjugate transform)
            AdjPart xi = x;
            xi.Ec = (int)(2 * SS * Ec);
            xi.X = ACC;
            xi.xout = acc;
            xi.xscale = (double)n;
            DGFS_TRY(adj64_part(plan, ADJ_PART_INV, xi, st));
            // loss-term adjoint and df += beta (acc / n^3 - ...), per species
            DGFS_TRY(adj64_part(plan, ADJ_PART_LOSS, x, st));
            if (domega)
                for (int k = 0; k < SS; ++k)
                    DGFS_TRY(adj64_omega_loss(plan, dom, (int)(k / S), (int)(k % S),
                                              lossdots + (long)k * Ec * 2 * lblk, Ec, st));
        }
        if (domega) {
            DGFS_CUDA(cudaMemcpyAsync(domega, dom, sizeof(double) * S * S,
                                      domega_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
            if (domega_on_host) DGFS_CUDA(cudaStreamSynchronize(st));
        }
        return DGFS_OK;
    };
    const dgfs_status status = run();
    const cudaError_t fe = dev_free_async(own, st);
    if (status == DGFS_OK && fe != cudaSuccess) return cuda_status(fe, "dgfs_collide_backward");
    return status;
}

template <int FMT>
dgfs_status backward_fmt(dgfs_plan_s *plan, int P, const void *f, const void *dQ, void *df, double *domega,
                         int domega_on_host, cudaStream_t st)
{
    switch (plan->N) {
    case 8: return backward_n<8, FMT>(plan, P, f, dQ, df, domega, domega_on_host, st);
    case 16: return backward_n<16, FMT>(plan, P, f, dQ, df, domega, domega_on_host, st);
    case 24: return backward_n<24, FMT>(plan, P, f, dQ, df, domega, domega_on_host, st);
    case 32: return backward_n<32, FMT>(plan, P, f, dQ, df, domega, domega_on_host, st);
    case 48: return backward_n<48, FMT>(plan, P, f, dQ, df, domega, domega_on_host, st);
    default: set_error("N not supported by the tensor-core adjoint"); return DGFS_EUNSUPPORTED;
    }
}

}  // namespace

dgfs_status tc_backward(dgfs_plan_s *plan, int P, const void *f, const void *dQ, void *df, double *domega,
                        int domega_on_host, cudaStream_t st)
{
    const TcState *ts = reinterpret_cast<const TcState *>(plan->tc);
    if (!ts) {
        set_error("dgfs_collide_backward: the plan has no tensor-core state");
        return DGFS_EINVAL;
    }
    return ts->fmt == 0 ? backward_fmt<0>(plan, P, f, dQ, df, domega, domega_on_host, st)
                        : backward_fmt<1>(plan, P, f, dQ, df, domega, domega_on_host, st);
}

}  // namespace dgfs

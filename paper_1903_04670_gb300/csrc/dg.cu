// 1-D nodal DG streaming term, purely diffuse walls and the SSP-RK3 step
// around the collision operator: Eq. (1), df_p/dt + c . grad_x f_p =
// sum_q Q^(pq), solved by Runge-Kutta discontinuous Galerkin in one space
// dimension (Sec. 3.3; diffuse walls as in the Couette case of Table 2).  The
// paper names the scheme and defers its formulas to its references; this is
// the textbook nodal form:
//
//  - Ne equal elements on [x0, x1]; on each, the K Gauss-Legendre nodes xi_j
//    of [-1, 1] carry the Lagrange interpolant and are the quadrature, so the
//    element mass matrix is J diag(w), J = h_e / 2, and
//      J w_i df_i/dt = c_x sum_j w_j phi_i'(xi_j) f_j - phi_i(+1) F_R + phi_i(-1) F_L
//    with the upwind flux F = c_x f taken from the side the velocity comes from;
//  - at a wall, velocities entering the domain see n_w M_w(c), the wall
//    Maxwellian (m/(pi T_w))^{3/2} exp(-m |c - u_w|^2 / T_w) scaled so that
//    the discrete net mass flux sum_c c_x f(c) through the wall is zero;
//  - SSP-RK3 in Shu-Osher form with L(f) = streaming(f) + sum_q Q^(pq)(f).
//
// Work per stage: one deterministic reduction of the outgoing wall fluxes
// (32 blocks per wall and species, partials added in a fixed order) and one
// elementwise kernel over
// (element, species, velocity) that forms the K nodal right-hand sides and
// the Runge-Kutta combination in registers.  Both are HBM-bound.
#include <cmath>
#include <new>
#include <vector>

#include "dgfs_internal.h"

struct dgfs_dg_s {
    dgfs_plan_s *plan = nullptr;
    int Ne = 0, K = 0, P = 0;
    double x0 = 0, x1 = 0, J = 0;
    double walls[8] = {0};         // {T, ux, uy, uz} left, right
    std::vector<double> xi, w;     // Gauss-Legendre nodes / weights on [-1, 1]
    double A[5][5] = {{0}};        // w_j phi_i'(xi_j) / (J w_i)
    double bL[5] = {0}, bR[5] = {0};  // phi_i(-1) / (J w_i), phi_i(+1) / (J w_i)
    double tL[5] = {0}, tR[5] = {0};  // phi_j(-1), phi_j(+1): traces
    std::vector<double> inflow;    // [2][S] sum over entering velocities of c_x M_w
    double *Mw = nullptr;          // device [2][S][n] unit-density wall Maxwellians
    double *wsum = nullptr;        // device [2][S][chunks] partial outgoing flux sums
    void *f1 = nullptr, *f2 = nullptr, *Q = nullptr;  // SSP-RK3 stage buffers
};

namespace dgfs {
namespace {

constexpr int kMaxK = 5;

struct DgCoef {
    double A[kMaxK][kMaxK], bL[kMaxK], bR[kMaxK], tL[kMaxK], tR[kMaxK];
    double nwL[4], nwR[4];  // 1 / (sum over entering velocities of c_x M_w) per species (S <= 4)
};

__device__ __forceinline__ double cx_of(long v, int N, double L)
{
    const int ix = (int)((uint32_t)v / (uint32_t)(N * N));  // n = N^3 < 2^31
    return -L + (ix + 0.5) * (2.0 * L / N);
}

constexpr int kWallChunks = 32;  // blocks per (wall, species) in the flux reduction

// Outgoing mass-flux sums at the two walls: block (side, p, chunk) reduces
// sum_{c leaving the domain} c_x f_trace(c) over its contiguous share of the
// n velocities in a fixed order and writes one partial sum; the partials are
// added in chunk order where they are used.  Left wall: trace of element 0
// at xi = -1, leaving = c_x < 0.
template <typename T, int K>
__global__ void k_wall_out(const T *f, DgCoef cf, int Ne, int S, int N, double L, long n, double *wsum)
{
    const int side = blockIdx.x, p = blockIdx.y;
    const int e = side == 0 ? 0 : Ne - 1;
    const long per = (n + kWallChunks - 1) / kWallChunks;
    const long v0 = blockIdx.z * per, v1 = min(n, v0 + per);
    double acc = 0.0;
    for (long v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        const double cx = cx_of(v, N, L);
        if (side == 0 ? cx < 0.0 : cx > 0.0) {
            double u = 0.0;
#pragma unroll
            for (int j = 0; j < K; ++j)
                u += (side == 0 ? cf.tL[j] : cf.tR[j]) * (double)f[((long)(e * K + j) * S + p) * n + v];
            acc += cx * u;
        }
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) wsum[(side * S + p) * kWallChunks + blockIdx.z] = red[0];
}

__device__ __forceinline__ double wall_sum(const double *wsum, int side, int S, int p)
{
    const double *w = wsum + (side * S + p) * kWallChunks;
    double s = 0.0;
    for (int i = 0; i < kWallChunks; ++i) s += w[i];
    return s;
}

// One thread per (element, species, velocity): the K nodal right-hand sides
//   r_i = c_x sum_j A_ij f_j - bR_i F_R + bL_i F_L (+ sum_q Q^(pq) at node i)
// then out_i = r_i (STAGE = false) or out_i = a0 f0_i + a1 (f_i + dt r_i).
// out may alias f0 (each element's f0 is read only by the thread writing it),
// never f.
template <typename T, int K, bool STAGE>
__global__ void k_dg(const T *f, const T *Q, const T *f0, T *out, DgCoef cf, const double *Mw, const double *wsum,
                     const double *halo_l, const double *halo_r, int Ne, int S, int N, double L, long n, double a0,
                     double a1, double dt)
{
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long)Ne * S * n) return;
    // 32-bit index arithmetic: Ne S n < 2^31 (checked when the DG object is created)
    const uint32_t g32 = (uint32_t)gid, n32 = (uint32_t)n, ps = g32 / n32;
    const long v = g32 - ps * n32;
    const int p = (int)(ps % (uint32_t)S), e = (int)(ps / (uint32_t)S);
    const double cx = cx_of(v, N, L);
    auto at = [&](int node) { return ((long)node * S + p) * n + v; };
    double u[K];
#pragma unroll
    for (int j = 0; j < K; ++j) u[j] = (double)f[at(e * K + j)];
    double uL_in = 0.0, uR_in = 0.0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        uL_in += cf.tL[j] * u[j];
        uR_in += cf.tR[j] * u[j];
    }
    double FL, FR;
    if (cx > 0.0) {  // comes from the left
        double up;
        if (e > 0) {
            up = 0.0;
#pragma unroll
            for (int j = 0; j < K; ++j) up += cf.tR[j] * (double)f[at((e - 1) * K + j)];
        } else {
            up = halo_l ? halo_l[(long)p * n + v] : -wall_sum(wsum, 0, S, p) * cf.nwL[p] * Mw[(long)p * n + v];
        }
        FL = cx * up;
        FR = cx * uR_in;
    } else {  // comes from the right
        double dn;
        if (e < Ne - 1) {
            dn = 0.0;
#pragma unroll
            for (int j = 0; j < K; ++j) dn += cf.tL[j] * (double)f[at((e + 1) * K + j)];
        } else {
            dn = halo_r ? halo_r[(long)p * n + v]
                        : -wall_sum(wsum, 1, S, p) * cf.nwR[p] * Mw[((long)S + p) * n + v];
        }
        FL = cx * uL_in;
        FR = cx * dn;
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
        double r = 0.0;
#pragma unroll
        for (int j = 0; j < K; ++j) r += cf.A[i][j] * u[j];
        r = cx * r - cf.bR[i] * FR + cf.bL[i] * FL;
        if (Q) {
            const long qb = ((long)(e * K + i) * S + p) * S * n + v;
            for (int q = 0; q < S; ++q) r += (double)Q[qb + (long)q * n];
        }
        const long o = at(e * K + i);
        if (STAGE) {
            const double nx = u[i] + dt * r;
            out[o] = (T)(a0 == 0.0 ? a1 * nx : a0 * (double)f0[o] + a1 * nx);
        } else {
            out[o] = (T)r;
        }
    }
}

// Boundary traces of this slab, FP64 [S][n]: element 0 at xi = -1 (left) and
// element Ne - 1 at xi = +1 (right), the values a neighbouring slab needs.
template <typename T, int K>
__global__ void k_traces(const T *f, DgCoef cf, int Ne, int S, long n, double *left, double *right)
{
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long)S * n) return;
    const long v = gid % n;
    const int p = (int)(gid / n);
    double l = 0.0, r = 0.0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        l += cf.tL[j] * (double)f[((long)j * S + p) * n + v];
        r += cf.tR[j] * (double)f[((long)((Ne - 1) * K + j) * S + p) * n + v];
    }
    if (left) left[gid] = l;
    if (right) right[gid] = r;
}

DgCoef coef_of(const dgfs_dg_s *dg)
{
    DgCoef c{};
    for (int i = 0; i < dg->K; ++i) {
        for (int j = 0; j < dg->K; ++j) c.A[i][j] = dg->A[i][j];
        c.bL[i] = dg->bL[i];
        c.bR[i] = dg->bR[i];
        c.tL[i] = dg->tL[i];
        c.tR[i] = dg->tR[i];
    }
    const int S = dg->plan->S;
    for (int p = 0; p < S; ++p) {
        c.nwL[p] = 1.0 / dg->inflow[p];
        c.nwR[p] = 1.0 / dg->inflow[S + p];
    }
    return c;
}

struct DgCall {
    const void *f, *Q, *f0;
    void *out;
    bool stage;
    double a0, a1, dt;
    const double *halo_l, *halo_r;  // null: wall at that side
};

template <typename T, int K>
dgfs_status dg_launch_k(dgfs_dg_s *dg, const DgCall &c, cudaStream_t st)
{
    const void *f = c.f, *Q = c.Q, *f0 = c.f0;
    void *out = c.out;
    const bool stage = c.stage;
    const double a0 = c.a0, a1 = c.a1, dt = c.dt;
    dgfs_plan_s *plan = dg->plan;
    const int N = plan->N, S = plan->S;
    const long n = (long)N * N * N;
    const DgCoef cf = coef_of(dg);
    {
        ProfScope ps(plan, "dg_wall_flux", st);
        k_wall_out<T, K><<<dim3(2, S, kWallChunks), 256, 0, st>>>(reinterpret_cast<const T *>(f), cf, dg->Ne, S, N, plan->L, n,
                                                     dg->wsum);
        DGFS_LAUNCHED(plan);
    }
    const long total = (long)dg->Ne * S * n;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    ProfScope ps(plan, "dg_rhs", st);
    if (stage)
        k_dg<T, K, true><<<blocks, 256, 0, st>>>(reinterpret_cast<const T *>(f), reinterpret_cast<const T *>(Q),
                                                 reinterpret_cast<const T *>(f0), reinterpret_cast<T *>(out), cf,
                                                 dg->Mw, dg->wsum, c.halo_l, c.halo_r, dg->Ne, S, N, plan->L, n, a0,
                                                 a1, dt);
    else
        k_dg<T, K, false><<<blocks, 256, 0, st>>>(reinterpret_cast<const T *>(f), reinterpret_cast<const T *>(Q),
                                                  nullptr, reinterpret_cast<T *>(out), cf, dg->Mw, dg->wsum, c.halo_l,
                                                  c.halo_r, dg->Ne, S, N, plan->L, n, 0.0, 0.0, 0.0);
    DGFS_LAUNCHED(plan);
    return DGFS_OK;
}

template <typename T, int K>
dgfs_status traces_k(dgfs_dg_s *dg, const void *f, double *left, double *right, cudaStream_t st)
{
    dgfs_plan_s *plan = dg->plan;
    const long n = (long)plan->N * plan->N * plan->N, total = (long)plan->S * n;
    ProfScope ps(plan, "dg_traces", st);
    k_traces<T, K><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(reinterpret_cast<const T *>(f), coef_of(dg),
                                                                     dg->Ne, plan->S, n, left, right);
    DGFS_LAUNCHED(plan);
    return DGFS_OK;
}

template <typename T>
dgfs_status dg_launch_t(dgfs_dg_s *dg, const DgCall &c, cudaStream_t st)
{
    switch (dg->K) {
    case 1: return dg_launch_k<T, 1>(dg, c, st);
    case 2: return dg_launch_k<T, 2>(dg, c, st);
    case 3: return dg_launch_k<T, 3>(dg, c, st);
    case 4: return dg_launch_k<T, 4>(dg, c, st);
    case 5: return dg_launch_k<T, 5>(dg, c, st);
    }
    set_error("dg: K out of range");
    return DGFS_EINVAL;
}

dgfs_status dg_launch(dgfs_dg_s *dg, const DgCall &c, cudaStream_t st)
{
    if (dg->plan->prec == DGFS_FP64) return dg_launch_t<double>(dg, c, st);
    return dg_launch_t<float>(dg, c, st);
}

template <typename T>
dgfs_status traces_t(dgfs_dg_s *dg, const void *f, double *left, double *right, cudaStream_t st)
{
    switch (dg->K) {
    case 1: return traces_k<T, 1>(dg, f, left, right, st);
    case 2: return traces_k<T, 2>(dg, f, left, right, st);
    case 3: return traces_k<T, 3>(dg, f, left, right, st);
    case 4: return traces_k<T, 4>(dg, f, left, right, st);
    case 5: return traces_k<T, 5>(dg, f, left, right, st);
    }
    set_error("dg: K out of range");
    return DGFS_EINVAL;
}

// One Runge-Kutta stage: out = a0 f0 + a1 (f_in + dt L(f_in)), with the
// collision operator of the plan evaluated on f_in when requested.
dgfs_status dg_stage(dgfs_dg_s *dg, const void *f_in, const void *f0, void *out, double a0, double a1, double dt,
                     int with_collisions, const double *halo_l, const double *halo_r, cudaStream_t st)
{
    if (with_collisions) {
        const dgfs_status s = dgfs_collide(dg->plan, dg->P, f_in, dg->Q, st);
        if (s != DGFS_OK) return s;
    }
    const DgCall c{f_in, with_collisions ? dg->Q : nullptr, f0, out, true, a0, a1, dt, halo_l, halo_r};
    return dg_launch(dg, c, st);
}

void dg_free(dgfs_dg_s *dg)
{
    if (!dg) return;
    dev_free(dg->Mw);
    dev_free(dg->wsum);
    dev_free(dg->f1);
    dev_free(dg->f2);
    dev_free(dg->Q);
    delete dg;
}

dgfs_status dg_build(dgfs_dg_s *dg)
{
    dgfs_plan_s *plan = dg->plan;
    const int K = dg->K, S = plan->S, N = plan->N;
    const long n = (long)N * N * N;
    host_gauss_legendre(K, -1.0, 1.0, dg->xi, dg->w);
    dg->J = 0.5 * (dg->x1 - dg->x0) / dg->Ne;
    const std::vector<double> &x = dg->xi;
    auto phi = [&](int i, double t) {
        double v = 1.0;
        for (int m = 0; m < K; ++m)
            if (m != i) v *= (t - x[m]) / (x[i] - x[m]);
        return v;
    };
    auto dphi = [&](int i, double t) {  // product rule
        double den = 1.0;
        for (int m = 0; m < K; ++m)
            if (m != i) den *= x[i] - x[m];
        double s = 0.0;
        for (int l = 0; l < K; ++l) {
            if (l == i) continue;
            double p = 1.0;
            for (int m = 0; m < K; ++m)
                if (m != i && m != l) p *= t - x[m];
            s += p;
        }
        return s / den;
    };
    for (int i = 0; i < K; ++i) {
        const double jw = dg->J * dg->w[i];
        for (int j = 0; j < K; ++j) dg->A[i][j] = dg->w[j] * dphi(i, x[j]) / jw;
        dg->tL[i] = phi(i, -1.0);
        dg->tR[i] = phi(i, 1.0);
        dg->bL[i] = dg->tL[i] / jw;
        dg->bR[i] = dg->tR[i] / jw;
    }
    // wall Maxwellians (unit density) and their entering fluxes
    const double L = plan->L, h = 2.0 * L / N;
    std::vector<double> Mw((size_t)2 * S * n);
    dg->inflow.assign(2 * S, 0.0);
    for (int side = 0; side < 2; ++side) {
        const double T = dg->walls[4 * side];
        const double *u = dg->walls + 4 * side + 1;
        for (int p = 0; p < S; ++p) {
            const double m = plan->masses[p];
            const double pre = std::pow(m / (kPi * T), 1.5);
            double in = 0.0;
            for (long v = 0; v < n; ++v) {
                const int ix = (int)(v / ((long)N * N)), iy = (int)((v / N) % N), iz = (int)(v % N);
                const double cx = -L + (ix + 0.5) * h, cy = -L + (iy + 0.5) * h, cz = -L + (iz + 0.5) * h;
                const double e2 = (cx - u[0]) * (cx - u[0]) + (cy - u[1]) * (cy - u[1]) + (cz - u[2]) * (cz - u[2]);
                const double M = pre * std::exp(-m * e2 / T);
                Mw[((size_t)side * S + p) * n + v] = M;
                if (side == 0 ? cx > 0.0 : cx < 0.0) in += cx * M;
            }
            if (!(std::fabs(in) > 0.0)) {
                set_error("dgfs_dg_create: the wall Maxwellian has no entering flux on this grid");
                return DGFS_EINVAL;
            }
            dg->inflow[side * S + p] = in;
        }
    }
    DGFS_CUDA(cudaSetDevice(plan->device));
    DGFS_CUDA(dev_malloc(&dg->Mw, sizeof(double) * Mw.size()));
    DGFS_CUDA(cudaMemcpy(dg->Mw, Mw.data(), sizeof(double) * Mw.size(), cudaMemcpyHostToDevice));
    DGFS_CUDA(dev_malloc(&dg->wsum, sizeof(double) * 2 * S * kWallChunks));
    const size_t es = elem_size(plan);
    DGFS_CUDA(dev_malloc(&dg->f1, es * dg->P * S * n));
    DGFS_CUDA(dev_malloc(&dg->f2, es * dg->P * S * n));
    DGFS_CUDA(dev_malloc(&dg->Q, es * dg->P * S * S * n));
    return DGFS_OK;
}

}  // namespace
}  // namespace dgfs

using namespace dgfs;

extern "C" {

dgfs_status dgfs_dg_create(dgfs_dg *out, dgfs_plan plan, int Ne, int K, double x0, double x1, const double *walls)
{
    if (!out) return DGFS_EINVAL;
    *out = nullptr;
    if (!plan || !walls || Ne < 1 || K < 1 || K > kMaxK || !(x1 > x0) || plan->S > 4 ||
        (long)Ne * K > plan->max_points || (long)Ne * K * plan->S * plan->N * plan->N * plan->N >= (1L << 31)) {
        set_error("dgfs_dg_create: bad plan, walls, Ne, K (1..5), interval or Ne*K > max_points");
        return DGFS_EINVAL;
    }
    for (int s = 0; s < 2; ++s) {
        if (!(walls[4 * s] > 0.0) || !std::isfinite(walls[4 * s]) || !std::isfinite(walls[4 * s + 1]) ||
            !std::isfinite(walls[4 * s + 2]) || !std::isfinite(walls[4 * s + 3])) {
            set_error("dgfs_dg_create: wall temperature must be > 0 and velocities finite");
            return DGFS_EINVAL;
        }
    }
    dgfs_dg_s *dg = host_new<dgfs_dg_s>();
    if (!dg) {
        set_error("dgfs_dg_create: out of host memory");
        return DGFS_ENOMEM;
    }
    dg->plan = plan;
    dg->Ne = Ne;
    dg->K = K;
    dg->P = Ne * K;
    dg->x0 = x0;
    dg->x1 = x1;
    for (int i = 0; i < 8; ++i) dg->walls[i] = walls[i];
    const dgfs_status st = dg_build(dg);
    if (st != DGFS_OK) {
        dg_free(dg);
        return st;
    }
    *out = dg;
    return DGFS_OK;
}

dgfs_status dgfs_dg_destroy(dgfs_dg dg)
{
    if (!dg) return DGFS_OK;
    cudaSetDevice(dg->plan->device);
    cudaDeviceSynchronize();
    dg_free(dg);
    return DGFS_OK;
}

dgfs_status dgfs_dg_nodes(dgfs_dg dg, double *x_host)
{
    if (!dg || !x_host) return DGFS_EINVAL;
    for (int e = 0; e < dg->Ne; ++e)
        for (int j = 0; j < dg->K; ++j)
            x_host[e * dg->K + j] = dg->x0 + (e + 0.5) * (2.0 * dg->J) + dg->J * dg->xi[j];
    return DGFS_OK;
}

dgfs_status dgfs_dg_rhs(dgfs_dg dg, const void *f_dev, const void *Q_dev, void *rhs_dev, void *stream)
{
    if (!dg || !f_dev || !rhs_dev || f_dev == rhs_dev) {
        set_error("dgfs_dg_rhs: bad handle or pointer (rhs must not alias f)");
        return DGFS_EINVAL;
    }
    dgfs_status st = plan_entry_check(dg->plan);
    if (st != DGFS_OK) return st;
    const DgCall c{f_dev, Q_dev, nullptr, rhs_dev, false, 0.0, 0.0, 0.0, nullptr, nullptr};
    return dg_launch(dg, c, reinterpret_cast<cudaStream_t>(stream));
}

dgfs_status dgfs_dg_rhs_halo(dgfs_dg dg, const void *f_dev, const void *Q_dev, void *rhs_dev,
                             const double *halo_left_dev, const double *halo_right_dev, void *stream)
{
    if (!dg || !f_dev || !rhs_dev || f_dev == rhs_dev) {
        set_error("dgfs_dg_rhs_halo: bad handle or pointer (rhs must not alias f)");
        return DGFS_EINVAL;
    }
    dgfs_status st = plan_entry_check(dg->plan);
    if (st != DGFS_OK) return st;
    const DgCall c{f_dev, Q_dev, nullptr, rhs_dev, false, 0.0, 0.0, 0.0, halo_left_dev, halo_right_dev};
    return dg_launch(dg, c, reinterpret_cast<cudaStream_t>(stream));
}

dgfs_status dgfs_dg_traces(dgfs_dg dg, const void *f_dev, double *left_dev, double *right_dev, void *stream)
{
    if (!dg || !f_dev || (!left_dev && !right_dev)) {
        set_error("dgfs_dg_traces: bad handle or pointer");
        return DGFS_EINVAL;
    }
    dgfs_status st = plan_entry_check(dg->plan);
    if (st != DGFS_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (dg->plan->prec == DGFS_FP64) return traces_t<double>(dg, f_dev, left_dev, right_dev, s);
    return traces_t<float>(dg, f_dev, left_dev, right_dev, s);
}

dgfs_status dgfs_dg_stage(dgfs_dg dg, const void *f_in_dev, const void *f0_dev, void *out_dev, double a0, double a1,
                          double dt, int with_collisions, const double *halo_left_dev,
                          const double *halo_right_dev, void *stream)
{
    if (!dg || !f_in_dev || !out_dev || f_in_dev == out_dev || (a0 != 0.0 && !f0_dev) || !std::isfinite(dt)) {
        set_error("dgfs_dg_stage: bad handle, pointer (out must not alias f_in) or coefficient");
        return DGFS_EINVAL;
    }
    dgfs_status st = plan_entry_check(dg->plan);
    if (st != DGFS_OK) return st;
    return dg_stage(dg, f_in_dev, f0_dev, out_dev, a0, a1, dt, with_collisions, halo_left_dev, halo_right_dev,
                    reinterpret_cast<cudaStream_t>(stream));
}

dgfs_status dgfs_dg_step(dgfs_dg dg, void *f_dev, double dt, int with_collisions, void *stream)
{
    if (!dg || !f_dev || !std::isfinite(dt)) {
        set_error("dgfs_dg_step: bad handle, pointer or dt");
        return DGFS_EINVAL;
    }
    dgfs_status st = plan_entry_check(dg->plan);
    if (st != DGFS_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    struct Stage { const void *in; void *out; double a0, a1; };
    const Stage stages[3] = {{f_dev, dg->f1, 0.0, 1.0}, {dg->f1, dg->f2, 0.75, 0.25}, {dg->f2, f_dev, 1.0 / 3.0, 2.0 / 3.0}};
    for (const Stage &sg : stages) {
        st = dg_stage(dg, sg.in, f_dev, sg.out, sg.a0, sg.a1, dt, with_collisions, nullptr, nullptr, s);
        if (st != DGFS_OK) return st;
    }
    return DGFS_OK;
}

}  // extern "C"

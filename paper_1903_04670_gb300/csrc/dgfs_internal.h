// Internal declarations of the CUDA collision library (not installed, not
// shared with anything outside csrc/).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <new>
#include <string>
#include <vector>

#include "../../include/dgfs.h"

namespace dgfs {

constexpr double kPi = 3.14159265358979323846264338327950288;

// Per-pair tables (Algorithm 1).  Device arrays are owned by the plan.
struct PairTables {
    // scalars (host)
    double R = 0, beta = 0, gamma = 0, eta = 0, dlogbeta = 0, cq = 0, cp = 0;
    int overridden = 0;
    std::vector<double> rho, wrho;  // N_rho Gauss-Legendre nodes/weights on [0, R]
    // FP64 device tables, natural k layout (x slowest)
    double2 *b = nullptr;      // [RS][n]   b_rs(k), RS = N_rho * M, rs = r*M + s
    double2 *c = nullptr;      // [n]       c_k
    double2 *c_om = nullptr;   // [n]       c with rho^{gamma+2} -> -2 ln(rho) rho^{gamma+2}
    double2 *phase = nullptr;  // [RS][2][3][N]  exp(+i cq theta_r sigma_sd l), exp(-i cp theta_r sigma_sd l)
    double *w = nullptr;       // [RS]  w_r w_s
    double *wlog = nullptr;    // [RS]  -2 ln(rho_r) w_r w_s
    // FP32 tensor-core form (built only for non-FP64 plans)
    float2 *b32 = nullptr;     // [RS][n]
    float *tmat = nullptr;     // translate / DFT matrices, see tc32.cu
    float4 *cdf = nullptr;     // [n] c as double-float (findf.cu)
};

}  // namespace dgfs

struct dgfs_plan_s {
    int N = 0, M = 0, Nrho = 0, S = 0, max_points = 0, device = 0;
    double L = 0;
    dgfs_precision prec = DGFS_FP64;
    std::vector<double> masses;
    std::vector<dgfs_pair> pair_params;
    double sigma[12 * 3] = {0};
    double wsig[12] = {0};
    std::vector<dgfs::PairTables> pairs;  // S*S, p-major

    double2 *twiddle = nullptr;  // [N] exp(-2 pi i j / N)
    double *quad_dev = nullptr;  // scratch copy of rho/w/sigma for table kernels
    double *masses_dev = nullptr;  // [S]

    // workspace (owned)
    void *ws = nullptr;
    size_t ws_bytes = 0;
    int chunk = 1;            // evaluations per pass launch
    void *stage_f = nullptr;  // host-call staging [max_points][S][n]
    void *stage_Q = nullptr;  // host-call staging [max_points][S][S][n]
    size_t table_bytes = 0;
    long long launches = 0;
    // tensor-core form state (tc32.cu)
    void *tc = nullptr;
    // 1: sum over design directions before the forward transforms (VHS only)
    int collapse = 0;
    // bumped whenever the launch configuration changes (collapse, kernel
    // variant, autotuning); a batch built on an older configuration is stale
    unsigned config_gen = 0;
    // per-kernel CUDA-event profiler (capi.cu), null unless enabled
    void *prof = nullptr;
    // 1: the declared Hermitian form (Nyquist planes removed, two points per
    // grid slot); herm_ws is its extra workspace (dgfs_plan_set_hermitian)
    int hermitian = 0;
    void *herm_ws = nullptr;
    size_t herm_bytes = 0;
};

namespace dgfs {

// error detail for dgfs_last_error(); thread local
void set_error(const std::string &msg);
dgfs_status cuda_status(cudaError_t e, const char *what);

#define DGFS_CUDA(call)                                                    \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return ::dgfs::cuda_status(e_, #call);      \
    } while (0)

#define DGFS_LAUNCHED(plan)                                                \
    do {                                                                   \
        (plan)->launches++;                                                \
        cudaError_t e_ = cudaGetLastError();                               \
        if (e_ != cudaSuccess) return ::dgfs::cuda_status(e_, "kernel launch"); \
    } while (0)

#define DGFS_TRY(x)                   \
    do {                              \
        dgfs_status s_ = (x);         \
        if (s_ != DGFS_OK) return s_; \
    } while (0)

size_t elem_size(const dgfs_plan_s *plan);

// Allocations of the library (capi.cu).  Device memory goes through
// dev_malloc / dev_free (and the stream-ordered pair), which count the live
// allocations; the library's host objects through host_new.  Both honour the
// host-side allocation-failure hook (dgfs_debug_fail_alloc): the allocation
// it selects reports failure without allocating.
bool alloc_fault_injected();
cudaError_t dev_malloc_raw(void **p, size_t bytes);
cudaError_t dev_malloc_async_raw(void **p, size_t bytes, cudaStream_t st);
cudaError_t dev_free(void *p);
cudaError_t dev_free_async(void *p, cudaStream_t st);
template <typename T> inline cudaError_t dev_malloc(T **p, size_t bytes)
{
    return dev_malloc_raw(reinterpret_cast<void **>(p), bytes);
}
template <typename T> inline cudaError_t dev_malloc_async(T **p, size_t bytes, cudaStream_t st)
{
    return dev_malloc_async_raw(reinterpret_cast<void **>(p), bytes, st);
}
template <typename T> inline T *host_new() { return alloc_fault_injected() ? nullptr : new (std::nothrow) T(); }

// Brackets one kernel launch with CUDA events on its stream when the plan's
// profiler is on (dgfs_plan_profile); no-op otherwise.
class ProfScope {
  public:
    ProfScope(dgfs_plan_s *plan, const char *kernel_class, cudaStream_t st);
    ~ProfScope();

  private:
    void *slot_;
    cudaStream_t st_;
};

// capi.cu: whether the sigma collapse is exact and implemented for the plan
bool collapse_eligible(const dgfs_plan_s *plan);
// capi.cu: Gauss-Legendre nodes (increasing) and weights on [a, b]
void host_gauss_legendre(int n, double a, double b, std::vector<double> &x, std::vector<double> &w);
// tables.cu
dgfs_status build_tables(dgfs_plan_s *plan);
// fft64.cu
size_t fp64_workspace_bytes(const dgfs_plan_s *plan, int chunk);
size_t fp64_scratch_bytes(const dgfs_plan_s *plan, int Fcap, int chunk);
dgfs_status fp64_collide_ws(dgfs_plan_s *plan, int P, const void *f, void *Q, void *ws, int Fcap, int chunk,
                            cudaStream_t st);
dgfs_status plan_entry_check(dgfs_plan_s *plan);
dgfs_status fp64_collide(dgfs_plan_s *plan, int P, const void *f, void *Q, cudaStream_t st);
dgfs_status fp64_backward(dgfs_plan_s *plan, int P, const void *f, const void *dQ, void *df,
                          double *domega, int domega_on_host, cudaStream_t st);
dgfs_status fp64_forward(dgfs_plan_s *plan, int P, const void *f, double2 *F, cudaStream_t st);
// adj64.cu: the parts of the adjoint outside its (r, s) loop, in FP64, for one
// chunk of points [pt0, pt0 + Ec) and a list of species pairs (also used by the
// tensor-core adjoint).  Buffers hold one [Ec][n] slot per listed pair, in list
// order (accp: two slots per pair, the f_p then the f_q sum).
struct AdjPart {
    int pt0 = 0, Ec = 0, f32 = 1, want_omega = 0;
    int npairs = 1;
    int pairs[16] = {0};                     // p S + q of each listed pair (S <= 4)
    const void *f = nullptr, *dQ = nullptr;  // [P][S][n], [P][S][S][n]
    void *df = nullptr;                      // [P][S][n], accumulated
    const double2 *F = nullptr;              // [P][S][n] fft3(f)
    double2 *Gg = nullptr, *GF = nullptr, *L = nullptr, *Lw = nullptr, *Y = nullptr;  // [pairs][Ec][n]
    double *accp = nullptr;                   // [pairs][2][Ec][n] gain sums of the f_p, f_q gradients (scale n^3)
    double *lossdots = nullptr;               // [pairs][Ec][2][adj64_nblk(N)]
    double2 *X = nullptr;                     // ADJ_PART_INV: [Ec][n] spectra (Ec counts grids here)
    double *xout = nullptr;                   // ADJ_PART_INV: [Ec][n] = xscale Re ifft3_u(X)
    double xscale = 1.0;
};
enum { ADJ_PART_G = 0, ADJ_PART_INV = 1, ADJ_PART_LOSS = 2 };
int adj64_nblk(int N);
dgfs_status adj64_part(dgfs_plan_s *plan, int which, const AdjPart &x, cudaStream_t st);
// dL/d omega_pq (dom[p S + q]): the gain terms from per-(point, r, s) dots [Ec][RS] of
// dscale^-1 Re<V, A B> (set, or added when accumulate), and the loss terms (added)
dgfs_status adj64_omega_gain(dgfs_plan_s *plan, double *dom, int p, int q, const double *dots, double dscale, int Ec,
                             int accumulate, cudaStream_t st);
dgfs_status adj64_omega_loss(dgfs_plan_s *plan, double *dom, int p, int q, const double *lossdots, int Ec,
                             cudaStream_t st);
// tcadj.cu: the adjoint of a tensor-core plan
dgfs_status tc_backward(dgfs_plan_s *plan, int P, const void *f, const void *dQ, void *df, double *domega,
                        int domega_on_host, cudaStream_t st);
dgfs_status df_forward(dgfs_plan_s *plan, int P, const float *f, float4 *F, const float4 *tw, cudaStream_t st);
dgfs_status df_finish(dgfs_plan_s *plan, int P, float4 *G, long pair_stride, const float4 *F, const float *f,
                      float *Q, const float4 *tw, cudaStream_t st);
dgfs_status df_tables(dgfs_plan_s *plan, float4 **tw_out);
dgfs_status df_herm_prepare(dgfs_plan_s *plan, int P, float4 *F, float4 *tmp, float *ft, const float4 *tw,
                            cudaStream_t st);
dgfs_status df_herm_finish(dgfs_plan_s *plan, int P, float4 *G, long pair_stride, float4 *Z2, long z2_stride,
                           const float4 *F, const float *ft, float *Q, const float4 *tw, cudaStream_t st);
// moments (fft64.cu)
dgfs_status moments(dgfs_plan_s *plan, int P, const void *Q, double *out, cudaStream_t st);
// tc32.cu
dgfs_status tc_prepare(dgfs_plan_s *plan);
void tc_release(dgfs_plan_s *plan);
dgfs_status tc_collide(dgfs_plan_s *plan, int P, const void *f, void *Q, cudaStream_t st);
size_t tc_workspace_bytes(const dgfs_plan_s *plan);
dgfs_status tc_check(dgfs_plan_s *plan);
bool tc_supports_collapse(const dgfs_plan_s *plan);
size_t tc_herm_bytes(const dgfs_plan_s *plan);
bool tc_herm_supported(const dgfs_plan_s *plan);
dgfs_status tc_herm_build(dgfs_plan_s *plan);
size_t fp64_herm_bytes(const dgfs_plan_s *plan);
dgfs_status tc_set_variant(dgfs_plan_s *plan, int variant);
dgfs_status tc_set_schedule(dgfs_plan_s *plan, int mode);
int tc_schedule(const dgfs_plan_s *plan);
dgfs_status tc_batch_set_schedule(void *batch, int mode);
void tc_debug_worklist_trace(void *buf, size_t bytes);
void tc_debug_worklist_chunk(int rs);
dgfs_status tc_batch_build(int count, dgfs_plan_s *const *plans, const int *P, void *const *f, void *const *Q,
                           void **out);
dgfs_status tc_batch_launch(void *batch, cudaStream_t st);
void tc_batch_free(void *batch);
dgfs_status tc_selftest_wait(dgfs_plan_s *plan, int expire, cudaStream_t st);
void tc_info(const dgfs_plan_s *plan, double *info);
dgfs_status tc_autotune(dgfs_plan_s *plan, int P, const void *f, void *Q, cudaStream_t st, double *best_ms);
dgfs_status relax_step(dgfs_plan_s *plan, int P, void *f, const void *Q, double dt, cudaStream_t st);

}  // namespace dgfs

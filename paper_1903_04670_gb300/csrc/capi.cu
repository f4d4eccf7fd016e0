// C-ABI entry points (include/dgfs.h): argument checking, plan construction
// (host scalars of Sec. 2 and 2.2: truncation radius, Gauss-Legendre radial
// quadrature, spherical designs, beta^(pq)), dispatch to the FP64 and
// tensor-core paths, host-buffer variant, moments and introspection.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "dgfs_internal.h"

namespace dgfs {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

dgfs_status cuda_status(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? DGFS_ENOMEM : DGFS_ECUDA;
}

size_t elem_size(const dgfs_plan_s *plan) { return plan->prec == DGFS_FP64 ? sizeof(double) : sizeof(float); }

// ------------------------------------------------- allocation accounting
namespace {
std::atomic<long long> g_live_device_allocs{0};
std::atomic<int> g_fail_countdown{0};  // > 0: that many allocations from now, the last one fails
}  // namespace

bool alloc_fault_injected()
{
    int c = g_fail_countdown.load();
    while (c > 0)
        if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
    return false;
}

cudaError_t dev_malloc_raw(void **p, size_t bytes)
{
    *p = nullptr;
    if (alloc_fault_injected()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) g_live_device_allocs++;
    return e;
}

cudaError_t dev_malloc_async_raw(void **p, size_t bytes, cudaStream_t st)
{
    *p = nullptr;
    if (alloc_fault_injected()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e == cudaSuccess) g_live_device_allocs++;
    return e;
}

cudaError_t dev_free(void *p)
{
    if (!p) return cudaSuccess;
    g_live_device_allocs--;
    return cudaFree(p);
}

cudaError_t dev_free_async(void *p, cudaStream_t st)
{
    if (!p) return cudaSuccess;
    g_live_device_allocs--;
    return cudaFreeAsync(p, st);
}

long long live_device_allocations() { return g_live_device_allocs.load(); }
void set_fail_countdown(int n) { g_fail_countdown.store(n > 0 ? n : 0); }

// ------------------------------------------------------------- profiler
namespace {
struct ProfSlot {
    cudaEvent_t a = nullptr, b = nullptr;
    int cls = -1;
};
struct Profiler {
    std::vector<ProfSlot> slots;
    size_t used = 0;
    long long dropped = 0;
    std::vector<std::string> names;
    int class_id(const char *name)
    {
        for (size_t i = 0; i < names.size(); ++i)
            if (names[i] == name) return (int)i;
        names.emplace_back(name);
        return (int)names.size() - 1;
    }
};
constexpr size_t kProfSlots = 16384;
}  // namespace

ProfScope::ProfScope(dgfs_plan_s *plan, const char *kernel_class, cudaStream_t st) : slot_(nullptr), st_(st)
{
    Profiler *pr = reinterpret_cast<Profiler *>(plan->prof);
    if (!pr) return;
    if (pr->used >= pr->slots.size()) {
        pr->dropped++;
        return;
    }
    ProfSlot &sl = pr->slots[pr->used++];
    sl.cls = pr->class_id(kernel_class);
    cudaEventRecord(sl.a, st);
    slot_ = &sl;
}

ProfScope::~ProfScope()
{
    if (slot_) cudaEventRecord(reinterpret_cast<ProfSlot *>(slot_)->b, st_);
}

static void prof_free(dgfs_plan_s *plan)
{
    Profiler *pr = reinterpret_cast<Profiler *>(plan->prof);
    if (!pr) return;
    for (auto &s : pr->slots) {
        if (s.a) cudaEventDestroy(s.a);
        if (s.b) cudaEventDestroy(s.b);
    }
    delete pr;
    plan->prof = nullptr;
}

namespace {

// Gauss-Legendre nodes and weights on [a, b]: Newton's method on P_n with the
// three-term recurrence, nodes in increasing order.
void gauss_legendre(int n, double a, double b, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (n - i - 0.25) / (n + 0.5));  // i-th smallest root
        double dp = 1.0;
        for (int it = 0; it < 200; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            // P_n = p1 (or z when n == 1), P_{n-1} = p0
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) <= 1e-16 * std::fabs(z) + 1e-300) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = 0.5 * (b - a) * z + 0.5 * (b + a);
        w[i] = 0.5 * (b - a) * 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Digamma: recurrence psi(x) = psi(x+1) - 1/x up to x >= 20, then the
// asymptotic series of Abramowitz & Stegun 6.3.18.
double digamma(double x)
{
    double r = 0.0;
    for (; x < 20.0; x += 1.0) r -= 1.0 / x;
    const double z = 1.0 / (x * x);
    const double tail = z * (1.0 / 12 - z * (1.0 / 120 - z * (1.0 / 252 - z * (1.0 / 240 - z / 132))));
    return r + std::log(x) - 0.5 / x - tail;
}

// Full-sphere spherical designs with weights 4 pi / M: M = 6 octahedron, M = 12
// icosahedron (cyclic permutations of (0, +-1, +-golden)/norm).
bool design(int M, double *sig, double *w)
{
    if (M == 6) {
        for (int s = 0; s < 6; ++s) {
            for (int d = 0; d < 3; ++d) sig[3 * s + d] = 0.0;
            sig[3 * s + s / 2] = (s & 1) ? -1.0 : 1.0;
        }
    } else if (M == 12) {
        const double g = 0.5 * (1.0 + std::sqrt(5.0));
        const double nrm = std::sqrt(1.0 + g * g);
        int s = 0;
        for (int perm = 0; perm < 3; ++perm)
            for (int sg = 0; sg < 4; ++sg, ++s) {
                const double v[3] = {0.0, ((sg & 2) ? -1.0 : 1.0) / nrm, ((sg & 1) ? -g : g) / nrm};
                for (int d = 0; d < 3; ++d) sig[3 * s + d] = v[(d + 3 - perm) % 3];
            }
    } else {
        return false;
    }
    for (int s = 0; s < M; ++s) w[s] = 4.0 * kPi / M;
    return true;
}

bool supported_N(int N)
{
    return N == 4 || N == 6 || N == 8 || N == 12 || N == 16 || N == 24 || N == 32 || N == 48;
}

void free_plan(dgfs_plan_s *plan)
{
    if (!plan) return;
    prof_free(plan);
    tc_release(plan);
    for (auto &pt : plan->pairs) {
        dev_free(pt.b);
        dev_free(pt.c);
        dev_free(pt.c_om);
        dev_free(pt.phase);
        dev_free(pt.w);
        dev_free(pt.wlog);
        dev_free(pt.b32);
        dev_free(pt.cdf);
        dev_free(pt.tmat);
    }
    dev_free(plan->twiddle);
    dev_free(plan->quad_dev);
    dev_free(plan->masses_dev);
    dev_free(plan->ws);
    dev_free(plan->stage_f);
    dev_free(plan->stage_Q);
    dev_free(plan->herm_ws);
    delete plan;
}

// checks that precede every launch on a plan: sticky async faults surface here
dgfs_status entry_check(dgfs_plan_s *plan)
{
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return cuda_status(e, "cudaSetDevice");
    e = cudaPeekAtLastError();
    if (e != cudaSuccess) return cuda_status(e, "pending device error");
    return DGFS_OK;
}

}  // namespace

dgfs_status plan_entry_check(dgfs_plan_s *plan) { return entry_check(plan); }

// The sum over design directions may move before the forward transforms when
// b_rs does not depend on s: eta = alpha - 1 = 0 for every pair (the angular
// integral is then 4 pi sinc(theta abs(k)), Sec. 2.2) and equal design weights.
bool collapse_eligible(const dgfs_plan_s *plan)
{
    for (const dgfs_pair &pp : plan->pair_params)
        if (pp.alpha != 1.0) return false;
    for (int s = 1; s < plan->M; ++s)
        if (plan->wsig[s] != plan->wsig[0]) return false;
    return plan->prec == DGFS_FP64 || tc_supports_collapse(plan);
}

void host_gauss_legendre(int n, double a, double b, std::vector<double> &x, std::vector<double> &w)
{
    gauss_legendre(n, a, b, x, w);
}

}  // namespace dgfs

using namespace dgfs;

extern "C" {

const char *dgfs_version(void) { return "dgfs-gb300 0.1 (sm_103a)"; }

void dgfs_debug_fail_alloc(int n) { set_fail_countdown(n); }

long long dgfs_debug_live_allocations(void) { return live_device_allocations(); }

const char *dgfs_status_string(dgfs_status s)
{
    switch (s) {
    case DGFS_OK: return "DGFS_OK";
    case DGFS_EINVAL: return "DGFS_EINVAL";
    case DGFS_ENOMEM: return "DGFS_ENOMEM";
    case DGFS_ECUDA: return "DGFS_ECUDA";
    case DGFS_ETIMEOUT: return "DGFS_ETIMEOUT";
    case DGFS_EUNSUPPORTED: return "DGFS_EUNSUPPORTED";
    }
    return "DGFS_UNKNOWN";
}

const char *dgfs_last_error(void) { return g_last_error.c_str(); }

dgfs_status dgfs_plan_create(dgfs_plan *out, int N, double L, int M, int N_rho, int S, const double *masses,
                             const dgfs_pair *pairs, dgfs_precision prec, int max_points, int device)
{
    if (!out) {
        set_error("out is NULL");
        return DGFS_EINVAL;
    }
    *out = nullptr;
    if (!supported_N(N)) {
        set_error("N must be one of 4, 6, 8, 12, 16, 24, 32, 48");
        return N < 2 ? DGFS_EINVAL : DGFS_EUNSUPPORTED;
    }
    if (!(L > 0.0) || !std::isfinite(L) || (M != 6 && M != 12) || N_rho < 1 || N_rho > 64 || S < 1 || S > 4 ||
        max_points < 1 || max_points > 65535 || !masses || !pairs) {
        set_error("invalid plan arguments (L > 0, M in {6, 12}, 1 <= N_rho <= 64, 1 <= S <= 4, "
                  "1 <= max_points <= 65535)");
        return DGFS_EINVAL;
    }
    if (prec != DGFS_FP64 && prec != DGFS_FP32_TC && prec != DGFS_TF32 && prec != DGFS_BF16X3) {
        set_error("unknown precision");
        return DGFS_EINVAL;
    }
    for (int s = 0; s < S; ++s)
        if (!(masses[s] > 0.0) || !std::isfinite(masses[s])) {
            set_error("masses must be positive and finite");
            return DGFS_EINVAL;
        }
    for (int i = 0; i < S * S; ++i) {
        const dgfs_pair &pp = pairs[i];
        const bool ov = !std::isnan(pp.beta_override);
        if (!(pp.alpha > 0.0) || !(pp.omega < 2.5) || !std::isfinite(pp.omega) ||
            (!ov && !(pp.d > 0.0)) || (ov && !std::isfinite(pp.beta_override))) {
            set_error("invalid pair parameters (alpha > 0, omega < 2.5, d > 0 unless beta is overridden)");
            return DGFS_EINVAL;
        }
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        set_error("no such CUDA device");
        return DGFS_EINVAL;
    }
    DGFS_CUDA(cudaSetDevice(device));

    dgfs_plan_s *plan = host_new<dgfs_plan_s>();
    if (!plan) {
        set_error("dgfs_plan_create: out of host memory");
        return DGFS_ENOMEM;
    }
    plan->N = N;
    plan->L = L;
    plan->M = M;
    plan->Nrho = N_rho;
    plan->S = S;
    plan->prec = prec;
    plan->max_points = max_points;
    plan->device = device;
    plan->masses.assign(masses, masses + S);
    plan->pair_params.assign(pairs, pairs + S * S);
    design(M, plan->sigma, plan->wsig);

    plan->pairs.resize(S * S);
    for (int p = 0; p < S; ++p)
        for (int q = 0; q < S; ++q) {
            PairTables &pt = plan->pairs[p * S + q];
            const dgfs_pair &pp = pairs[p * S + q];
            const double mp = masses[p], mq = masses[q], mu = mp + mq;
            pt.cq = mq / mu;
            pt.cp = mp / mu;
            // truncation radius R = 4L / (1 + max(4 mq/mu, 2) + sqrt(1 + mq/mp)) (Sec. 2.1)
            pt.R = 4.0 * L / (1.0 + std::fmax(4.0 * mq / mu, 2.0) + std::sqrt(1.0 + mq / mp));
            pt.gamma = 2.0 * (1.0 - pp.omega);  // |u|^{2(1-omega)} of Eq. (3)
            pt.eta = pp.alpha - 1.0;            // (1 + cos chi)^{alpha-1} of Eq. (3)
            if (std::isnan(pp.beta_override)) {
                // Eq. (4) with n0 = H0 = 1, T_ref = T0, and the beta^(pq) definition
                const double kn = 1.0 / (std::sqrt(1.0 + mp / mq) * kPi * pp.d * pp.d);
                const double mr = mp * mq / mu;
                pt.beta = (1.0 / kn) / std::sqrt(1.0 + mp / mq) * std::pow(mr, -(pp.omega - 0.5)) * pp.alpha /
                          (std::pow(2.0, 1.0 + pp.alpha) * std::tgamma(2.5 - pp.omega) * kPi);
                pt.dlogbeta = -std::log(mr) + digamma(2.5 - pp.omega);
                pt.overridden = 0;
            } else {
                pt.beta = pp.beta_override;
                pt.dlogbeta = 0.0;
                pt.overridden = 1;
            }
            gauss_legendre(N_rho, 0.0, pt.R, pt.rho, pt.wrho);
        }
    plan->collapse = collapse_eligible(plan) ? 1 : 0;

    dgfs_status st = build_tables(plan);
    if (st == DGFS_OK) {
        cudaError_t e = dev_malloc(&plan->masses_dev, sizeof(double) * S);
        if (e == cudaSuccess) e = cudaMemcpy(plan->masses_dev, masses, sizeof(double) * S, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = cuda_status(e, "masses");
    }
    if (st == DGFS_OK && prec != DGFS_FP64) st = tc_prepare(plan);
    if (st == DGFS_OK) {
        // workspace: bounded to ~1 GiB of per-(r,s) intermediates per pass
        if (prec == DGFS_FP64) {
            const long n = (long)N * N * N;
            const long per_eval = 2L * N_rho * M * n * (long)sizeof(double2);
            int chunk = (int)std::max(1L, std::min((long)max_points, (1L << 30) / per_eval));
            plan->chunk = chunk;
            plan->ws_bytes = fp64_workspace_bytes(plan, chunk);
        } else {
            plan->ws_bytes = tc_workspace_bytes(plan);
        }
        cudaError_t e = dev_malloc(&plan->ws, plan->ws_bytes);
        if (e != cudaSuccess) st = cuda_status(e, "workspace");
    }
    if (st == DGFS_OK) {
        const long n = (long)N * N * N;
        const size_t es = elem_size(plan);
        cudaError_t e = dev_malloc(&plan->stage_f, es * (size_t)max_points * S * n);
        if (e == cudaSuccess) e = dev_malloc(&plan->stage_Q, es * (size_t)max_points * S * S * n);
        if (e != cudaSuccess) st = cuda_status(e, "staging buffers");
    }
    if (st == DGFS_OK) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) st = cuda_status(e, "plan tables");
    }
    if (st != DGFS_OK) {
        free_plan(plan);
        return st;
    }
    *out = plan;
    return DGFS_OK;
}

dgfs_status dgfs_plan_destroy(dgfs_plan plan)
{
    if (!plan) return DGFS_OK;
    cudaSetDevice(plan->device);
    cudaDeviceSynchronize();
    free_plan(plan);
    return DGFS_OK;
}

dgfs_status dgfs_collide(dgfs_plan plan, int P, const void *f_dev, void *Q_dev, void *stream)
{
    if (!plan || !f_dev || !Q_dev || P < 1 || P > plan->max_points) {
        set_error("dgfs_collide: bad plan, pointer or P (1 <= P <= max_points)");
        return DGFS_EINVAL;
    }
    dgfs_status st = entry_check(plan);
    if (st != DGFS_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (plan->prec == DGFS_FP64) return fp64_collide(plan, P, f_dev, Q_dev, s);
    return tc_collide(plan, P, f_dev, Q_dev, s);
}

dgfs_status dgfs_plan_set_kernel_variant(dgfs_plan plan, int variant)
{
    if (!plan) return DGFS_EINVAL;
    return tc_set_variant(plan, variant);
}

dgfs_status dgfs_plan_set_schedule(dgfs_plan plan, int mode)
{
    if (!plan) return DGFS_EINVAL;
    return tc_set_schedule(plan, mode);
}

dgfs_status dgfs_debug_worklist_trace(void *trace_dev, size_t bytes)
{
    tc_debug_worklist_trace(trace_dev, bytes);
    return DGFS_OK;
}

dgfs_status dgfs_debug_worklist_chunk(int rs_per_wave)
{
    if (rs_per_wave < 1) return DGFS_EINVAL;
    tc_debug_worklist_chunk(rs_per_wave);
    return DGFS_OK;
}

dgfs_status dgfs_plan_get_schedule(dgfs_plan plan, int *mode)
{
    if (!plan || !mode) return DGFS_EINVAL;
    *mode = tc_schedule(plan);
    return DGFS_OK;
}

dgfs_status dgfs_plan_set_collapse(dgfs_plan plan, int enable)
{
    if (!plan) return DGFS_EINVAL;
    if (enable && !collapse_eligible(plan)) {
        set_error("dgfs_plan_set_collapse: needs alpha = 1 for every pair (b independent of the design "
                  "direction) and a path that implements it");
        return DGFS_EUNSUPPORTED;
    }
    plan->collapse = enable ? 1 : 0;
    plan->config_gen++;
    return DGFS_OK;
}

dgfs_status dgfs_plan_set_hermitian(dgfs_plan plan, int enable)
{
    if (!plan) return DGFS_EINVAL;
    if (!enable) {
        if (plan->herm_ws) {
            DGFS_CUDA(cudaSetDevice(plan->device));
            DGFS_CUDA(cudaDeviceSynchronize());
            dev_free(plan->herm_ws);
        }
        plan->herm_ws = nullptr;
        plan->herm_bytes = 0;
        plan->hermitian = 0;
        plan->config_gen++;
        return DGFS_OK;
    }
    if (plan->N % 2 != 0 || (plan->prec != DGFS_FP64 && !tc_herm_supported(plan))) {
        set_error("dgfs_plan_set_hermitian: needs even N, and N <= 32 for the tensor-core forms");
        return DGFS_EUNSUPPORTED;
    }
    dgfs_status st = entry_check(plan);
    if (st != DGFS_OK) return st;
    if (!plan->herm_ws) {
        const size_t bytes = plan->prec == DGFS_FP64 ? fp64_herm_bytes(plan) : tc_herm_bytes(plan);
        void *p = nullptr;
        cudaError_t e = dev_malloc(&p, bytes);
        if (e != cudaSuccess) return cuda_status(e, "dgfs_plan_set_hermitian: workspace");
        plan->herm_ws = p;
        plan->herm_bytes = bytes;
        if (plan->prec != DGFS_FP64) {
            st = tc_herm_build(plan);
            if (st != DGFS_OK) {
                dev_free(plan->herm_ws);
                plan->herm_ws = nullptr;
                plan->herm_bytes = 0;
                return st;
            }
        }
    }
    plan->hermitian = 1;
    plan->config_gen++;
    return DGFS_OK;
}

dgfs_status dgfs_collide_host(dgfs_plan plan, int P, const void *f_host, void *Q_host, void *stream)
{
    if (!plan || !f_host || !Q_host || P < 1 || P > plan->max_points) {
        set_error("dgfs_collide_host: bad plan, pointer or P");
        return DGFS_EINVAL;
    }
    dgfs_status st = entry_check(plan);
    if (st != DGFS_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const long n = (long)plan->N * plan->N * plan->N;
    const size_t es = elem_size(plan);
    const size_t fb = es * (size_t)P * plan->S * n, qb = es * (size_t)P * plan->S * plan->S * n;
    DGFS_CUDA(cudaMemcpyAsync(plan->stage_f, f_host, fb, cudaMemcpyHostToDevice, s));
    st = dgfs_collide(plan, P, plan->stage_f, plan->stage_Q, stream);
    if (st != DGFS_OK) return st;
    DGFS_CUDA(cudaMemcpyAsync(Q_host, plan->stage_Q, qb, cudaMemcpyDeviceToHost, s));
    DGFS_CUDA(cudaStreamSynchronize(s));
    return tc_check(plan);
}

dgfs_status dgfs_plan_selftest_wait(dgfs_plan plan, int expire, void *stream)
{
    if (!plan) return DGFS_EINVAL;
    dgfs_status st = entry_check(plan);
    if (st != DGFS_OK) return st;
    return tc_selftest_wait(plan, expire, reinterpret_cast<cudaStream_t>(stream));
}

dgfs_status dgfs_plan_check(dgfs_plan plan)
{
    if (!plan) return DGFS_EINVAL;
    dgfs_status st = entry_check(plan);
    if (st != DGFS_OK) return st;
    DGFS_CUDA(cudaDeviceSynchronize());
    return tc_check(plan);
}

dgfs_status dgfs_collide_backward(dgfs_plan plan, int P, const void *f_dev, const void *dQ_dev, void *df_dev,
                                  double *domega, int domega_on_host, void *stream)
{
    if (!plan || !f_dev || !dQ_dev || !df_dev || P < 1 || P > plan->max_points) {
        set_error("dgfs_collide_backward: bad plan, pointer or P");
        return DGFS_EINVAL;
    }
    dgfs_status st = entry_check(plan);
    if (st != DGFS_OK) return st;
    if (plan->hermitian) {
        set_error("dgfs_collide_backward: the adjoint is of the literal operator; switch the Hermitian form off");
        return DGFS_EUNSUPPORTED;
    }
    if (plan->prec != DGFS_FP64)
        return tc_backward(plan, P, f_dev, dQ_dev, df_dev, domega, domega_on_host,
                           reinterpret_cast<cudaStream_t>(stream));
    return fp64_backward(plan, P, f_dev, dQ_dev, df_dev, domega, domega_on_host,
                         reinterpret_cast<cudaStream_t>(stream));
}

dgfs_status dgfs_moments(dgfs_plan plan, int P, const void *Q_dev, double *out_dev, void *stream)
{
    if (!plan || !Q_dev || !out_dev || P < 1 || P > plan->max_points) {
        set_error("dgfs_moments: bad plan, pointer or P");
        return DGFS_EINVAL;
    }
    dgfs_status st = entry_check(plan);
    if (st != DGFS_OK) return st;
    return moments(plan, P, Q_dev, out_dev, reinterpret_cast<cudaStream_t>(stream));
}

dgfs_status dgfs_plan_info(dgfs_plan plan, double *info)
{
    if (!plan || !info) return DGFS_EINVAL;
    for (int i = 0; i < 16; ++i) info[i] = 0.0;
    info[0] = plan->N;
    info[1] = plan->L;
    info[2] = plan->M;
    info[3] = plan->Nrho;
    info[4] = plan->S;
    info[5] = (double)plan->prec;
    info[6] = plan->max_points;
    info[7] = (double)plan->ws_bytes;
    info[8] = (double)plan->table_bytes;
    info[9] = plan->chunk;
    tc_info(plan, info);
    info[15] = plan->collapse;
    return DGFS_OK;
}

dgfs_status dgfs_plan_pair_tables(dgfs_plan plan, int p, int q, double *scalars, double *rho, double *w_rho,
                                  double *sigma, double *w_sigma, double *b, double *c)
{
    if (!plan || p < 0 || q < 0 || p >= plan->S || q >= plan->S) return DGFS_EINVAL;
    dgfs_status st = entry_check(plan);
    if (st != DGFS_OK) return st;
    const PairTables &pt = plan->pairs[p * plan->S + q];
    if (scalars) {
        const double v[8] = {pt.R, pt.beta, pt.gamma, pt.eta, pt.dlogbeta, pt.cq, pt.cp, (double)pt.overridden};
        std::memcpy(scalars, v, sizeof(v));
    }
    if (rho) std::memcpy(rho, pt.rho.data(), sizeof(double) * plan->Nrho);
    if (w_rho) std::memcpy(w_rho, pt.wrho.data(), sizeof(double) * plan->Nrho);
    if (sigma) std::memcpy(sigma, plan->sigma, sizeof(double) * 3 * plan->M);
    if (w_sigma) std::memcpy(w_sigma, plan->wsig, sizeof(double) * plan->M);
    const long n = (long)plan->N * plan->N * plan->N;
    if (b) DGFS_CUDA(cudaMemcpy(b, pt.b, sizeof(double2) * plan->Nrho * plan->M * n, cudaMemcpyDeviceToHost));
    if (c) DGFS_CUDA(cudaMemcpy(c, pt.c, sizeof(double2) * n, cudaMemcpyDeviceToHost));
    return DGFS_OK;
}

dgfs_status dgfs_plan_profile(dgfs_plan plan, int enable)
{
    if (!plan) return DGFS_EINVAL;
    dgfs_status st = entry_check(plan);
    if (st != DGFS_OK) return st;
    if (!enable) {
        DGFS_CUDA(cudaDeviceSynchronize());
        prof_free(plan);
        return DGFS_OK;
    }
    if (!plan->prof) {
        Profiler *pr = new (std::nothrow) Profiler();
        if (!pr) return DGFS_ENOMEM;
        pr->slots.resize(kProfSlots);
        for (auto &sl : pr->slots) {
            if (cudaEventCreate(&sl.a) != cudaSuccess || cudaEventCreate(&sl.b) != cudaSuccess) {
                plan->prof = pr;
                prof_free(plan);
                set_error("cudaEventCreate failed");
                return DGFS_ECUDA;
            }
        }
        plan->prof = pr;
    }
    Profiler *pr = reinterpret_cast<Profiler *>(plan->prof);
    pr->used = 0;
    pr->dropped = 0;
    return DGFS_OK;
}

dgfs_status dgfs_plan_profile_read(dgfs_plan plan, int max_classes, char *names, long long *counts,
                                   double *total_ms, int *n_classes)
{
    if (!plan || !n_classes || max_classes < 0) return DGFS_EINVAL;
    Profiler *pr = reinterpret_cast<Profiler *>(plan->prof);
    *n_classes = 0;
    if (!pr) return DGFS_OK;
    dgfs_status st = entry_check(plan);
    if (st != DGFS_OK) return st;
    DGFS_CUDA(cudaDeviceSynchronize());
    const int nc = (int)pr->names.size();
    std::vector<long long> cnt(nc, 0);
    std::vector<double> ms(nc, 0.0);
    for (size_t i = 0; i < pr->used; ++i) {
        float t = 0.f;
        DGFS_CUDA(cudaEventElapsedTime(&t, pr->slots[i].a, pr->slots[i].b));
        cnt[pr->slots[i].cls] += 1;
        ms[pr->slots[i].cls] += t;
    }
    const int out = nc < max_classes ? nc : max_classes;
    for (int c = 0; c < out; ++c) {
        if (names) {
            std::strncpy(names + 64 * c, pr->names[c].c_str(), 63);
            names[64 * c + 63] = 0;
        }
        if (counts) counts[c] = cnt[c];
        if (total_ms) total_ms[c] = ms[c];
    }
    *n_classes = out;
    if (pr->dropped) {
        set_error("profiler slots exhausted; later launches were not timed");
        return DGFS_EINVAL;
    }
    return DGFS_OK;
}

dgfs_status dgfs_plan_autotune(dgfs_plan plan, int P, const void *f_dev, void *Q_dev, void *stream,
                               double *best_ms)
{
    if (!plan || !f_dev || !Q_dev || P < 1 || P > plan->max_points) {
        set_error("dgfs_plan_autotune: bad plan, pointer or P");
        return DGFS_EINVAL;
    }
    dgfs_status st = entry_check(plan);
    if (st != DGFS_OK) return st;
    return tc_autotune(plan, P, f_dev, Q_dev, reinterpret_cast<cudaStream_t>(stream), best_ms);
}

dgfs_status dgfs_plan_launch_count(dgfs_plan plan, long long *count)
{
    if (!plan || !count) return DGFS_EINVAL;
    *count = plan->launches;
    return DGFS_OK;
}

}  // extern "C"

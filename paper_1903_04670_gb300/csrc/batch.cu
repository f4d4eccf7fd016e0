// Batching and scheduling around the collision operator:
//  - dgfs_relax_step: homogeneous relaxation f_p += dt sum_q Q^(pq) (the
//    spatially homogeneous form of Eq. (1), explicit Euler as in Table 2),
//  - dgfs_graph_capture / _launch / _destroy: one CUDA graph holding the
//    collision calls (and optional relaxation steps) of a batch of uneven
//    instances, i.e. several plans with different N, S, M, N_rho and point
//    counts, replayed with a single launch,
//  - dgfs_batch_create / _launch / _destroy: a batched work list over uneven
//    instances; each tensor-core stage runs as one launch over the jobs of
//    all instances that share N and the operand format,
//  - dgfs_plan_autotune: times candidate launch configurations of a
//    tensor-core plan on the caller's data and keeps the fastest.
#include <algorithm>
#include <new>
#include <vector>

#include "dgfs_internal.h"

namespace dgfs {
namespace {

template <typename T>
__global__ void k_relax(T *f, const T *Q, int S, long n, long total, double dt)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;  // over [P][S][n]
    if (i >= total) return;
    const long k = i % n;
    const long ps = i / n;  // pt * S + p
    const long pt = ps / S;
    const int p = (int)(ps % S);
    double s = 0.0;
    for (int q = 0; q < S; ++q) s += (double)Q[((pt * S + p) * S + q) * n + k];
    f[i] = (T)((double)f[i] + dt * s);
}

}  // namespace

dgfs_status relax_step(dgfs_plan_s *plan, int P, void *f, const void *Q, double dt, cudaStream_t st)
{
    const long n = (long)plan->N * plan->N * plan->N;
    const long total = (long)P * plan->S * n;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    ProfScope ps(plan, "relax_step", st);
    if (plan->prec == DGFS_FP64)
        k_relax<double><<<blocks, 256, 0, st>>>(reinterpret_cast<double *>(f), reinterpret_cast<const double *>(Q),
                                                plan->S, n, total, dt);
    else
        k_relax<float><<<blocks, 256, 0, st>>>(reinterpret_cast<float *>(f), reinterpret_cast<const float *>(Q),
                                               plan->S, n, total, dt);
    DGFS_LAUNCHED(plan);
    return DGFS_OK;
}

}  // namespace dgfs

struct dgfs_graph_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture_stream = nullptr;
    int device = 0;
    long long kernels = 0;
};

struct dgfs_batch_s {
    std::vector<dgfs_plan_s *> plans;
    std::vector<unsigned> gens;  // config_gen of each plan at creation
    std::vector<int> P;
    std::vector<const void *> f;
    std::vector<void *> Q;
    double dt = 0.0;
    void *tc = nullptr;  // tensor-core work list (tc32.cu), null without TC plans
    int device = 0;
};

using namespace dgfs;

extern "C" {

dgfs_status dgfs_relax_step(dgfs_plan plan, int P, void *f_dev, const void *Q_dev, double dt, void *stream)
{
    if (!plan || !f_dev || !Q_dev || P < 1 || P > plan->max_points) {
        set_error("dgfs_relax_step: bad plan, pointer or P");
        return DGFS_EINVAL;
    }
    dgfs_status st = plan_entry_check(plan);
    if (st != DGFS_OK) return st;
    return relax_step(plan, P, f_dev, Q_dev, dt, reinterpret_cast<cudaStream_t>(stream));
}

dgfs_status dgfs_graph_capture(int count, const dgfs_plan *plans, const int *P, void *const *f_dev,
                               void *const *Q_dev, double dt, int steps, dgfs_graph *out)
{
    if (!out || count < 1 || !plans || !P || !f_dev || !Q_dev || steps < 1) {
        set_error("dgfs_graph_capture: bad arguments");
        return DGFS_EINVAL;
    }
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !f_dev[i] || !Q_dev[i] || P[i] < 1 || P[i] > plans[i]->max_points ||
            plans[i]->device != plans[0]->device) {
            set_error("dgfs_graph_capture: bad instance (plan, pointers, P, or plans on different devices)");
            return DGFS_EINVAL;
        }
    }
    dgfs_status st = plan_entry_check(plans[0]);
    if (st != DGFS_OK) return st;
    dgfs_graph_s *g = host_new<dgfs_graph_s>();
    if (!g) {
        set_error("dgfs_graph_capture: out of host memory");
        return DGFS_ENOMEM;
    }
    g->device = plans[0]->device;
    cudaError_t e = cudaStreamCreateWithFlags(&g->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete g;
        return cuda_status(e, "cudaStreamCreate");
    }
    std::vector<long long> before(count);
    for (int i = 0; i < count; ++i) before[i] = plans[i]->launches;
    e = cudaStreamBeginCapture(g->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int s = 0; s < steps && st == DGFS_OK; ++s)
            for (int i = 0; i < count && st == DGFS_OK; ++i) {
                st = dgfs_collide(plans[i], P[i], f_dev[i], Q_dev[i], g->capture_stream);
                if (st == DGFS_OK && dt != 0.0)
                    st = relax_step(plans[i], P[i], f_dev[i], Q_dev[i], dt, g->capture_stream);
            }
        cudaError_t e2 = cudaStreamEndCapture(g->capture_stream, &g->graph);
        if (st == DGFS_OK && e2 != cudaSuccess) st = cuda_status(e2, "cudaStreamEndCapture");
    } else {
        st = cuda_status(e, "cudaStreamBeginCapture");
    }
    if (st == DGFS_OK) {
        e = cudaGraphInstantiate(&g->exec, g->graph, 0);
        if (e != cudaSuccess) st = cuda_status(e, "cudaGraphInstantiate");
    }
    for (int i = 0; i < count; ++i) {
        g->kernels += plans[i]->launches - before[i];
        plans[i]->launches = before[i];  // captured, not launched
    }
    if (st != DGFS_OK) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        cudaStreamDestroy(g->capture_stream);
        delete g;
        return st;
    }
    *out = g;
    return DGFS_OK;
}

dgfs_status dgfs_batch_create(int count, const dgfs_plan *plans, const int *P, void *const *f_dev,
                              void *const *Q_dev, double dt, dgfs_batch *out)
{
    if (!out || count < 1 || !plans || !P || !f_dev || !Q_dev) {
        set_error("dgfs_batch_create: bad arguments");
        return DGFS_EINVAL;
    }
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !f_dev[i] || !Q_dev[i] || P[i] < 1 || P[i] > plans[i]->max_points ||
            plans[i]->device != plans[0]->device) {
            set_error("dgfs_batch_create: bad instance (plan, pointers, P, or plans on different devices)");
            return DGFS_EINVAL;
        }
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) {
                set_error("dgfs_batch_create: a plan appears twice (each instance needs its own workspace)");
                return DGFS_EINVAL;
            }
        if (plans[i]->hermitian) {
            set_error("dgfs_batch_create: the work list runs the literal operator (a plan is in the Hermitian form)");
            return DGFS_EUNSUPPORTED;
        }
    }
    dgfs_status st = plan_entry_check(plans[0]);
    if (st != DGFS_OK) return st;
    dgfs_batch_s *b = host_new<dgfs_batch_s>();
    if (!b) {
        set_error("dgfs_batch_create: out of host memory");
        return DGFS_ENOMEM;
    }
    b->device = plans[0]->device;
    b->dt = dt;
    std::vector<dgfs_plan_s *> tcp;
    std::vector<int> tcP;
    std::vector<void *> tcf, tcQ;
    for (int i = 0; i < count; ++i) {
        b->plans.push_back(plans[i]);
        b->gens.push_back(plans[i]->config_gen);
        b->P.push_back(P[i]);
        b->f.push_back(f_dev[i]);
        b->Q.push_back(Q_dev[i]);
        if (plans[i]->prec != DGFS_FP64) {
            tcp.push_back(plans[i]);
            tcP.push_back(P[i]);
            tcf.push_back(f_dev[i]);
            tcQ.push_back(Q_dev[i]);
        }
    }
    if (!tcp.empty()) {
        st = tc_batch_build((int)tcp.size(), tcp.data(), tcP.data(), tcf.data(), tcQ.data(), &b->tc);
        if (st != DGFS_OK) {
            delete b;
            return st;
        }
    }
    *out = b;
    return DGFS_OK;
}

dgfs_status dgfs_batch_launch(dgfs_batch b, void *stream)
{
    if (!b) return DGFS_EINVAL;
    for (size_t i = 0; i < b->plans.size(); ++i)
        if (b->plans[i]->config_gen != b->gens[i]) {
            set_error("dgfs_batch_launch: a plan's launch configuration changed after the batch was created");
            return DGFS_EINVAL;
        }
    dgfs_status st = plan_entry_check(b->plans[0]);
    if (st != DGFS_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (size_t i = 0; i < b->plans.size(); ++i)
        if (b->plans[i]->prec == DGFS_FP64) DGFS_TRY(fp64_collide(b->plans[i], b->P[i], b->f[i], b->Q[i], s));
    if (b->tc) DGFS_TRY(tc_batch_launch(b->tc, s));
    if (b->dt != 0.0)
        for (size_t i = 0; i < b->plans.size(); ++i)
            DGFS_TRY(relax_step(b->plans[i], b->P[i], const_cast<void *>(b->f[i]), b->Q[i], b->dt, s));
    return DGFS_OK;
}

dgfs_status dgfs_batch_set_schedule(dgfs_batch b, int mode)
{
    if (!b) return DGFS_EINVAL;
    return tc_batch_set_schedule(b->tc, mode);
}

dgfs_status dgfs_batch_destroy(dgfs_batch b)
{
    if (!b) return DGFS_OK;
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    tc_batch_free(b->tc);
    delete b;
    return DGFS_OK;
}

dgfs_status dgfs_graph_launch(dgfs_graph g, void *stream)
{
    if (!g) return DGFS_EINVAL;
    DGFS_CUDA(cudaSetDevice(g->device));
    DGFS_CUDA(cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream)));
    return DGFS_OK;
}

dgfs_status dgfs_graph_kernel_count(dgfs_graph g, long long *count)
{
    if (!g || !count) return DGFS_EINVAL;
    *count = g->kernels;
    return DGFS_OK;
}

dgfs_status dgfs_graph_destroy(dgfs_graph g)
{
    if (!g) return DGFS_OK;
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->capture_stream) cudaStreamDestroy(g->capture_stream);
    delete g;
    return DGFS_OK;
}

}  // extern "C"

// Peak issue rate of the 5th-generation tensor cores on this GPU
// (instrumentation for the roofline; no counterpart in the paper).
//
// One CTA per SM: thread 0 issues `iters` back-to-back MMAs of the shape that
// keeps the pipe busy (M = 128, N = 256, one 32-byte K step each) from zeroed
// SW128 K-major operands in shared memory into one TMEM accumulator, commits
// once and the CTA waits (bounded) for the commit.  The host times the launch
// with CUDA events; the rate is 2 M N K iters SMs / time.  kind::tf32 (K = 8)
// is the denominator of the 3xTF32 and TF32 forms, kind::f16 with BF16
// operands (K = 16) that of the split-BF16 form.
#include <algorithm>

#include "dgfs_internal.h"
#include "umma.cuh"

namespace dgfs {
namespace {

using namespace umma;

constexpr int kPM = 128, kPN = 256;
constexpr int kProbeSmem = 120 * 1024;  // more than half of an SM: one CTA per SM

template <int KIND>
__global__ void __launch_bounds__(128, 1) k_mma_probe(int iters, int *err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm =
        reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *A = sm;               // 128 rows x 128 B (one SW128 atom)
    uint8_t *Bop = sm + kPM * 128;  // 256 rows x 128 B
    __shared__ uint64_t mb;
    __shared__ uint32_t slot;
    for (int i = threadIdx.x; i < (kPM + kPN) * 128 / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x < 32) tmem_alloc(&slot, kPN);
    if (threadIdx.x == 0) mbar_init(&mb, 1);
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tb = slot;
    if (threadIdx.x == 0) {
        const uint32_t idesc = KIND == 0 ? idesc_tf32(kPM, kPN) : idesc_bf16(kPM, kPN);
        const uint32_t a0 = smem_u32(A), b0 = smem_u32(Bop);
        for (int it = 0; it < iters; ++it) {
            const uint32_t kb = (uint32_t)(it & 3) * 32;  // the four K steps of the atom in turn
            if (KIND == 0)
                mma_tf32(tb, desc_sw128(a0 + kb), desc_sw128(b0 + kb), idesc, it > 0 ? 1u : 0u);
            else
                mma_bf16(tb, desc_sw128(a0 + kb), desc_sw128(b0 + kb), idesc, it > 0 ? 1u : 0u);
        }
        commit(&mb);
    }
    const bool ok = mbar_wait(&mb, 0, 1L << 24);
    if (!__syncthreads_and(ok ? 1 : 0) && threadIdx.x == 0) atomicExch(err, 1);
    fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tmem_dealloc(tb, kPN);
}

}  // namespace
}  // namespace dgfs

using namespace dgfs;

extern "C" dgfs_status dgfs_probe_mma_rate(int device, int kind, int iters, double *tflops)
{
    if (!tflops || (kind != 0 && kind != 1) || iters < 64 || iters > (1 << 16)) {
        set_error("dgfs_probe_mma_rate: kind 0 (tf32) or 1 (bf16), 64 <= iters <= 65536, tflops not NULL");
        return DGFS_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        set_error("no such CUDA device");
        return DGFS_EINVAL;
    }
    DGFS_CUDA(cudaSetDevice(device));
    int sms = 0;
    DGFS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    auto kern = kind == 0 ? k_mma_probe<0> : k_mma_probe<1>;
    DGFS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem));
    int *err = nullptr;
    DGFS_CUDA(dev_malloc(&err, sizeof(int)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
        e = cudaEventRecord(e0, 0);
        if (e == cudaSuccess) {
            kern<<<sms, 128, kProbeSmem>>>(iters, err);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&flag, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(err);
    if (e != cudaSuccess) return cuda_status(e, "dgfs_probe_mma_rate");
    if (flag) {
        set_error("dgfs_probe_mma_rate: the bounded wait for the MMAs expired");
        return DGFS_ETIMEOUT;
    }
    const double k = kind == 0 ? 8.0 : 16.0;
    *tflops = 2.0 * kPM * kPN * k * (double)iters * sms / (best * 1e-3) / 1e12;
    return DGFS_OK;
}

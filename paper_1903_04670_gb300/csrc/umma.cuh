// tcgen05 (5th-generation tensor core) building blocks for sm_103a, in inline
// PTX: shared-memory matrix descriptors for K-major operands in the 128-byte
// swizzled layout, instruction descriptors for kind::tf32 and kind::f16 (bf16)
// with FP32 accumulation, MMA issue, commit to an mbarrier, bounded mbarrier
// waits, and tensor-memory (TMEM) allocation and loads.
//
// Operand layout ("SW128 K-major"): an operand of R rows and K elements per row
// is stored as ceil(K*esz/128) column blocks ("atoms") of R x 128 bytes; inside
// an atom, row r occupies bytes [128 r, 128 r + 128) and its 16-byte chunk c is
// stored at chunk c ^ (r mod 8).  Every atom starts on a 1024-byte boundary.
// One MMA consumes 32 bytes of K (8 tf32 or 16 bf16 values); its descriptor
// points at byte (k mod 128) of atom k / 128, the stride between 8-row groups
// (SBO) is 1024 bytes.
#pragma once

#include <cstdint>

namespace dgfs {
namespace umma {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of (row r, byte kb of the row) inside an SW128 K-major operand with R rows
__device__ __forceinline__ uint32_t sw128_off(int r, int kb, int R)
{
    const int atom = kb >> 7, in = kb & 127;
    return (uint32_t)(atom * (R * 128) + r * 128 + ((((in >> 4) ^ (r & 7))) << 4) + (in & 15));
}

__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);  // start address >> 4
    d |= (uint64_t)1 << 16;                  // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                  // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                  // 128-byte swizzle
    return d;
}

// instruction descriptors: D = F32, A/B K-major, M and N of the MMA
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// invalidate an idle mbarrier (every phase complete) so that its shared
// memory can be initialised again
__device__ __forceinline__ void mbar_inval(uint64_t *mbar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

// Waits for the phase with the given parity to complete; gives up after
// `limit` polls (each poll may suspend briefly) and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, long limit)
{
    uint32_t done = 0;
    for (long it = 0; it < limit; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// make generic-proxy shared-memory writes visible to the tensor core
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// warp-collective TMEM allocation of ncols (power of two >= 32); the address is
// written to *slot (shared memory)
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane; the warp reads lanes
// [32 (warp % 4), +32).  taddr must already carry the warp's lane offset.
// The load and its wait are one asm statement: tcgen05.ld is asynchronous, so
// nothing (a spill or a move of a destination register) may come between it
// and tcgen05.wait::ld.  The destinations are early-clobber: the load writes
// them asynchronously, so none may share a register with an address operand.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=&r"(r[0]), "=&r"(r[1]), "=&r"(r[2]), "=&r"(r[3]), "=&r"(r[4]), "=&r"(r[5]), "=&r"(r[6]), "=&r"(r[7]),
          "=&r"(r[8]), "=&r"(r[9]), "=&r"(r[10]), "=&r"(r[11]), "=&r"(r[12]), "=&r"(r[13]), "=&r"(r[14]), "=&r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Two 16-column TMEM loads (any two column offsets of this lane) completed by
// one wait, all in one asm statement (see tmem_ld16).
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, float *va, float *vb)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, "
        "[%33];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=&r"(r[0]), "=&r"(r[1]), "=&r"(r[2]), "=&r"(r[3]), "=&r"(r[4]), "=&r"(r[5]), "=&r"(r[6]), "=&r"(r[7]),
          "=&r"(r[8]), "=&r"(r[9]), "=&r"(r[10]), "=&r"(r[11]), "=&r"(r[12]), "=&r"(r[13]), "=&r"(r[14]), "=&r"(r[15]),
          "=&r"(r[16]), "=&r"(r[17]), "=&r"(r[18]), "=&r"(r[19]), "=&r"(r[20]), "=&r"(r[21]), "=&r"(r[22]),
          "=&r"(r[23]), "=&r"(r[24]), "=&r"(r[25]), "=&r"(r[26]), "=&r"(r[27]), "=&r"(r[28]), "=&r"(r[29]),
          "=&r"(r[30]), "=&r"(r[31])
        : "r"(ta), "r"(tb)
        : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        va[j] = __uint_as_float(r[j]);
        vb[j] = __uint_as_float(r[16 + j]);
    }
}

// Visit NO consecutive FP32 columns of this lane in chunks of 16 columns,
// f(c0, v) with v[j] = column c0 + j; two chunks share one wait.
template <int NO, typename F>
__device__ __forceinline__ void tmem_visit(uint32_t taddr, F &&f)
{
#pragma unroll
    for (int c0 = 0; c0 < NO; c0 += 32) {
        if (c0 + 32 <= NO) {
            float a[16], b[16];
            tmem_ld16x2(taddr + c0, taddr + c0 + 16, a, b);
            f(c0, a);
            f(c0 + 16, b);
        } else {
            float a[16];
            tmem_ld16(taddr + c0, a);
            f(c0, a);
        }
    }
}

// round-to-nearest TF32 value of x (low 13 mantissa bits cleared)
__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

}  // namespace umma
}  // namespace dgfs

namespace dgfs {
namespace umma {

// arrive on mbar and add tx_bytes to the transaction count it waits for
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t tx_bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(tx_bytes)
                 : "memory");
}

// asynchronous bulk copy global -> shared (16-byte aligned, size a multiple of
// 16), completion counted on mbar
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(mbar))
        : "memory");
}

}  // namespace umma
}  // namespace dgfs

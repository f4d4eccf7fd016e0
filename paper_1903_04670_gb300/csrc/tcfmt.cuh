// Operand formats of the tensor-core path.
//
// An FP32 value x enters the tensor cores as a sum of narrower terms and the
// products of the terms are accumulated in FP32 in TMEM:
//   FMT 0 (TF32): x = hi + lo, hi and lo rounded to TF32 (stored as 32-bit);
//                 products lo*hi + hi*lo + hi*hi ("3xTF32", kind::tf32), or the
//                 single hi*hi product for the plain TF32 form.
//   FMT 1 (BF16): x = b0 + b1 + b2, each rounded to BF16 (stored as 16-bit; the
//                 three terms carry 24 significand bits); the six products of
//                 total order <= 2, b2*b0 + b1*b1 + b0*b2 + b1*b0 + b0*b1 + b0*b0
//                 (kind::f16 with bf16 inputs), smallest first.
// Operands are SW128 K-major (see umma.cuh); one MMA consumes 32 bytes of K:
// 8 TF32 or 16 BF16 values.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "umma.cuh"

namespace dgfs {
namespace tcfmt {

using namespace umma;

constexpr int kRows = 128;  // MMA M: data rows per pipeline

template <int FMT> struct Fmt;
template <> struct Fmt<0> {
    static constexpr int ESZ = 4;  // bytes per stored element
    static constexpr int NT = 2;   // stored terms
};
template <> struct Fmt<1> {
    static constexpr int ESZ = 2;
    static constexpr int NT = 3;
};

__host__ __device__ constexpr int atoms_b(int bytes) { return (bytes + 127) / 128; }
// bytes of one term of the data operand (128 rows, K = 2N elements)
template <int FMT> __host__ __device__ constexpr int abytes(int N) { return atoms_b(2 * N * Fmt<FMT>::ESZ) * kRows * 128; }
// bytes of one term of a B-operand image: 2N rows, K = 2N (complex input) or N (real input)
template <int FMT> __host__ __device__ constexpr int img_c(int N) { return atoms_b(2 * N * Fmt<FMT>::ESZ) * 2 * N * 128; }
template <int FMT> __host__ __device__ constexpr int img_r(int N) { return atoms_b(N * Fmt<FMT>::ESZ) * 2 * N * 128; }

// x rounded to TF32 (10 mantissa bits), to nearest with ties away from zero:
// add half a TF32 unit to the magnitude bits and clear the 13 low bits.  The
// same bits as cvt.rna.tf32.f32 for every finite x, on the full-rate integer
// pipe (the split runs for every operand element the CUDA cores write).
__device__ __forceinline__ float tf32_round(float x)
{
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo)
{
    hi = tf32_round(x);
    lo = tf32_round(x - hi);
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &b0, __nv_bfloat16 &b1, __nv_bfloat16 &b2)
{
    b0 = __float2bfloat16_rn(x);
    float r = x - __bfloat162float(b0);  // exact in FP32
    b1 = __float2bfloat16_rn(r);
    r -= __bfloat162float(b1);  // exact in FP32
    b2 = __float2bfloat16_rn(r);
}

// Store NV (2 or 4) consecutive elements v[] starting at element e of `row`
// of a data operand whose terms are `ab` bytes apart, splitting each value.
template <int FMT, int NV>
__device__ __forceinline__ void st_elems(uint8_t *a0, int ab, int row, int e, const float *v)
{
    const uint32_t o = sw128_off(row, e * Fmt<FMT>::ESZ, kRows);
    if constexpr (FMT == 0) {
        float h[NV], l[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) split_tf32(v[i], h[i], l[i]);
        if constexpr (NV == 2) {
            *reinterpret_cast<float2 *>(a0 + o) = make_float2(h[0], h[1]);
            *reinterpret_cast<float2 *>(a0 + ab + o) = make_float2(l[0], l[1]);
        } else {
            *reinterpret_cast<float4 *>(a0 + o) = make_float4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<float4 *>(a0 + ab + o) = make_float4(l[0], l[1], l[2], l[3]);
        }
    } else {
        __nv_bfloat16 b[3][NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) split_bf16(v[i], b[0][i], b[1][i], b[2][i]);
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            if constexpr (NV == 2) {
                *reinterpret_cast<__nv_bfloat162 *>(a0 + t * ab + o) = __halves2bfloat162(b[t][0], b[t][1]);
            } else {
                __nv_bfloat162 lo2 = __halves2bfloat162(b[t][0], b[t][1]);
                __nv_bfloat162 hi2 = __halves2bfloat162(b[t][2], b[t][3]);
                uint2 u;
                u.x = *reinterpret_cast<uint32_t *>(&lo2);
                u.y = *reinterpret_cast<uint32_t *>(&hi2);
                *reinterpret_cast<uint2 *>(a0 + t * ab + o) = u;
            }
        }
    }
}

// one complex value at complex index k
template <int FMT>
__device__ __forceinline__ void st_c(uint8_t *a0, int ab, int row, int k, float re, float im)
{
    const float v[2] = {re, im};
    st_elems<FMT, 2>(a0, ab, row, 2 * k, v);
}

// two complex values at complex indices k, k+1 (k even)
template <int FMT>
__device__ __forceinline__ void st_c2(uint8_t *a0, int ab, int row, int k, float2 u, float2 w)
{
    const float v[4] = {u.x, u.y, w.x, w.y};
    st_elems<FMT, 4>(a0, ab, row, 2 * k, v);
}

// four consecutive real elements at element e (e a multiple of 4)
template <int FMT>
__device__ __forceinline__ void st_f4(uint8_t *a0, int ab, int row, int e, float4 x)
{
    const float v[4] = {x.x, x.y, x.z, x.w};
    st_elems<FMT, 4>(a0, ab, row, e, v);
}

// Issue D (128 x brows, FP32 in TMEM) = sum of the term products A_i * B_j^T
// over K = kelems elements.  a0 / b0: first term of the data operand and of the
// B image; their terms are ab / ib bytes apart.  For FMT 0, nterms is 1 or 3.
template <int FMT>
__device__ __forceinline__ void gemm(uint32_t d, const uint8_t *a0, int ab, const uint8_t *b0, int ib, int brows,
                                     int kelems, int nterms)
{
    const int kbytes = kelems * Fmt<FMT>::ESZ;
    uint32_t acc = 0;
    if constexpr (FMT == 0) {
        const int ta[3] = {1, 0, 0}, tb[3] = {0, 1, 0};
        const uint32_t idesc = idesc_tf32(kRows, brows);
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            if (nterms == 1 && t < 2) continue;
            const uint32_t A = smem_u32(a0 + ta[t] * ab), B = smem_u32(b0 + tb[t] * ib);
            for (int kb = 0; kb < kbytes; kb += 32) {
                const uint32_t ao = (kb >> 7) * (kRows * 128) + (kb & 127);
                const uint32_t bo = (kb >> 7) * (brows * 128) + (kb & 127);
                mma_tf32(d, desc_sw128(A + ao), desc_sw128(B + bo), idesc, acc);
                acc = 1;
            }
        }
    } else {
        const int ta[6] = {2, 1, 0, 1, 0, 0}, tb[6] = {0, 1, 2, 0, 1, 0};
        const uint32_t idesc = idesc_bf16(kRows, brows);
#pragma unroll
        for (int t = 0; t < 6; ++t) {
            const uint32_t A = smem_u32(a0 + ta[t] * ab), B = smem_u32(b0 + tb[t] * ib);
            for (int kb = 0; kb < kbytes; kb += 32) {
                const uint32_t ao = (kb >> 7) * (kRows * 128) + (kb & 127);
                const uint32_t bo = (kb >> 7) * (brows * 128) + (kb & 127);
                mma_bf16(d, desc_sw128(A + ao), desc_sw128(B + bo), idesc, acc);
                acc = 1;
            }
        }
    }
}

// Write the split terms of an FP64 matrix entry v at (row, element k) of a
// B-operand image with `rows` rows; terms are ib bytes apart.
template <int FMT>
__device__ __forceinline__ void put_img(uint8_t *img0, long ib, int row, int k, int rows, double v)
{
    const uint32_t off = sw128_off(row, k * Fmt<FMT>::ESZ, rows);
    if constexpr (FMT == 0) {
        const float h = tf32_rna((float)v);
        *reinterpret_cast<float *>(img0 + off) = h;
        *reinterpret_cast<float *>(img0 + ib + off) = tf32_rna((float)(v - (double)h));
    } else {
        double r = v;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const __nv_bfloat16 b = __float2bfloat16_rn((float)r);
            *reinterpret_cast<__nv_bfloat16 *>(img0 + t * ib + off) = b;
            r -= (double)__bfloat162float(b);
        }
    }
}

}  // namespace tcfmt
}  // namespace dgfs

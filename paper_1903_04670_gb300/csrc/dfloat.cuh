// Double-float ("float-float") arithmetic: a value is the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi) / 2, about 48 significant bits.
// The operations are the error-free transformations TwoSum (Knuth), Fast2Sum
// (Dekker) and the FMA-based exact product, combined as in the accurate
// double-word addition and multiplication of Joldes, Muller and Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic" (ACM TOMS 44, 2017): relative error below 3u^2 for the sum and
// 5u^2 for the product, u = 2^-24.  The explicit _rn intrinsics keep the
// compiler from contracting or reordering the steps, which the error-free
// transformations rely on.
//
// With these types the register FFT of fftreg.cuh runs on the FP32 pipes
// with close to FP64 accuracy; FP64 throughput on this GPU is a small
// fraction of FP32's.
#pragma once

#include <cuda_runtime.h>

namespace dgfs {

struct dfl {
    float hi, lo;
    dfl() = default;
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    // nearest float, then the float nearest to the remainder
    __host__ __device__ explicit dfl(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};

struct dcx {
    dfl x, y;
};

__device__ __forceinline__ dfl two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dfl(s, e);
}

__device__ __forceinline__ dfl fast_two_sum(float a, float b)  // |a| >= |b| or a == 0
{
    const float s = __fadd_rn(a, b);
    return dfl(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b)
{
    const dfl s = two_sum(a.hi, b.hi);
    const dfl t = two_sum(a.lo, b.lo);
    const dfl v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }

__device__ __forceinline__ dfl operator*(dfl a, dfl b)
{
    const float ch = __fmul_rn(a.hi, b.hi);
    const float cl1 = __fmaf_rn(a.hi, b.hi, -ch);
    const float tl1 = __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.lo));
    const float cl2 = __fmaf_rn(a.lo, b.hi, tl1);
    return fast_two_sum(ch, __fadd_rn(cl1, cl2));
}

__device__ __forceinline__ dfl fma(dfl a, dfl b, dfl c) { return a * b + c; }

// a float added exactly into a double-float accumulator
__device__ __forceinline__ dfl add_f(dfl a, float b)
{
    const dfl s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ float to_float(dfl a) { return __fadd_rn(a.hi, a.lo); }

// storage: one complex double-float as a float4 (x.hi, x.lo, y.hi, y.lo)
__device__ __forceinline__ dcx ld_dcx(const float4 *p)
{
    const float4 v = *p;
    return dcx{dfl(v.x, v.y), dfl(v.z, v.w)};
}
__device__ __forceinline__ void st_dcx(float4 *p, dcx v) { *p = make_float4(v.x.hi, v.x.lo, v.y.hi, v.y.lo); }

// found by argument-dependent lookup from the generic complex helpers of fftreg.cuh
__device__ __forceinline__ dcx mk(dfl x, dfl y) { return dcx{x, y}; }

namespace reg {
template <typename T2> struct Scalar;
template <> struct Scalar<dcx> { using type = dfl; };
}  // namespace reg

}  // namespace dgfs

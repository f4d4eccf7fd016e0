// Register-resident, compile-time-unrolled mixed-radix (4, 2, 3) decimation-in-
// time Cooley-Tukey FFT of one length-N pencil per thread, for double2 and
// float2 data.  Twiddles come from a table tw[e] = exp(-2 pi i e / N) of the
// same element type (held in shared memory by the caller).
#pragma once

#include <cuda_runtime.h>

namespace dgfs {
namespace reg {

template <typename T2> struct Scalar;
template <> struct Scalar<double2> { using type = double; };
template <> struct Scalar<float2> { using type = float; };

__device__ __forceinline__ double2 mk(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ float2 mk(float x, float y) { return make_float2(x, y); }

template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b)
{
    return mk(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
template <typename T2>
__device__ __forceinline__ T2 cmulc(T2 a, T2 b)  // a * conj(b)
{
    return mk(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { return mk(a.x - b.x, a.y - b.y); }
template <int SIGN, typename T2>
__device__ __forceinline__ T2 mul_si(T2 a)  // multiply by SIGN * i
{
    return SIGN < 0 ? mk(a.y, -a.x) : mk(-a.y, a.x);
}

template <int P, int SIGN, typename T2>
__device__ __forceinline__ void bfly(const T2 *t, T2 *y, int m)
{
    using R = typename Scalar<T2>::type;
    if constexpr (P == 2) {
        y[0] = cadd(t[0], t[1]);
        y[m] = csub(t[0], t[1]);
    } else if constexpr (P == 4) {
        const T2 u0 = cadd(t[0], t[2]), u1 = csub(t[0], t[2]);
        const T2 u2 = cadd(t[1], t[3]), u3 = mul_si<SIGN>(csub(t[1], t[3]));
        y[0] = cadd(u0, u2);
        y[2 * m] = csub(u0, u2);
        y[m] = cadd(u1, u3);
        y[3 * m] = csub(u1, u3);
    } else {  // P == 3
        const R h3 = (R)0.86602540378443864676;  // sqrt(3)/2
        const T2 s = cadd(t[1], t[2]);
        const T2 d = csub(t[1], t[2]);
        const T2 r = mk(t[0].x - (R)0.5 * s.x, t[0].y - (R)0.5 * s.y);
        const T2 q = mul_si<SIGN>(mk(h3 * d.x, h3 * d.y));
        y[0] = cadd(t[0], s);
        y[m] = cadd(r, q);
        y[2 * m] = csub(r, q);
    }
}

// y[k] = sum_j x[j*S] exp(SIGN 2 pi i j k / N), k < N; TOPN is the top-level length.
template <int N, int SIGN, int TOPN, typename T2>
struct Dft {
    template <int S>
    __device__ static __forceinline__ void run(const T2 *x, T2 *y, const T2 *tw)
    {
        if constexpr (N == 1) {
            y[0] = x[0];
        } else {
            constexpr int P = (N % 4 == 0) ? 4 : ((N % 2 == 0) ? 2 : 3);
            constexpr int m = N / P;
            T2 sub[N];
#pragma unroll
            for (int a = 0; a < P; ++a) Dft<m, SIGN, TOPN, T2>::template run<S * P>(x + a * S, sub + a * m, tw);
#pragma unroll
            for (int k = 0; k < m; ++k) {
                T2 t[P];
#pragma unroll
                for (int a = 0; a < P; ++a) {
                    const int e = (a * k * (TOPN / N)) % TOPN;
                    if (e == 0) {
                        t[a] = sub[a * m + k];
                    } else {
                        const T2 w = tw[e];
                        t[a] = SIGN < 0 ? cmul(sub[a * m + k], w) : cmulc(sub[a * m + k], w);
                    }
                }
                bfly<P, SIGN>(t, y + k, m);
            }
        }
    }
};

// in-place unnormalised transform of v[0..N-1]; SIGN -1 forward, +1 backward
template <int N, int SIGN, typename T2>
__device__ __forceinline__ void fft(T2 *v, const T2 *tw)
{
    T2 out[N];
    Dft<N, SIGN, N, T2>::template run<1>(v, out, tw);
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = out[k];
}

}  // namespace reg
}  // namespace dgfs

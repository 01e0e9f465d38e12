// Double-float numbers for the TSYLV_DF64 solve: a value is the unevaluated
// sum h + l of two floats with |l| <= ulp(h) / 2 after normalisation (the
// "double-word" numbers of T. J. Dekker, "A floating-point technique for
// extending the available precision", Numer. Math. 18, 1971, with the
// fused-multiply-add product of M. Joldes, J.-M. Muller, V. Popescu, "Tight
// and rigorous error bounds for basic building blocks of double-word
// arithmetic", ACM TOMS 44(2), 2017).  About 48 significant bits on the FP32
// pipes, which on this GPU issue 64 times the FP64 pipes' rate.
//
// Error-free transformations used below:
//   two_sum(a, b)      = (s, e) with s = fl(a + b), s + e = a + b exactly
//   fast_two_sum(a, b) = the same when |a| >= |b| (or a = 0)
//   two_prod(a, b)     = (p, e) with p = fl(a b), e = fma(a, b, -p) exact
// The sum, product and quotient normalise their result.  The multiply-add of
// the block products (dev::fmadd) leaves its pair unnormalised -- the pair
// still holds the sum exactly up to the products' roundings, with the low word
// a few ulps of the high one -- and dev::settle normalises an accumulator
// after its run of products.
#pragma once

#include "complex_z.h"

namespace tsylv {

struct alignas(8) dfl {
    float h, l;
    __host__ __device__ constexpr dfl() : h(0.f), l(0.f) {}
    __host__ __device__ constexpr dfl(float hi, float lo) : h(hi), l(lo) {}
    // nearest pair to a double: the float nearest to x, then the float nearest to the rest
    __host__ __device__ dfl(double x) : h(static_cast<float>(x)), l(static_cast<float>(x - static_cast<double>(h))) {}
    __host__ __device__ explicit operator double() const { return static_cast<double>(h) + static_cast<double>(l); }
};

#if defined(__CUDACC__)
namespace dfl_detail {
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dfl(s, __fsub_rn(b, __fsub_rn(s, a)));
}
}  // namespace dfl_detail

// (x + y): two_sum of the high words, the low words added to the error
// ("sloppy" sum: its error is bounded by the magnitudes of the summands,
// which is what the backward-stable triangular solve needs)
__device__ __forceinline__ dfl operator+(dfl x, dfl y) {
    float s, e;
    dfl_detail::two_sum(x.h, y.h, s, e);
    e = __fadd_rn(e, __fadd_rn(x.l, y.l));
    return dfl_detail::fast_two_sum(s, e);
}
__device__ __forceinline__ dfl operator-(dfl x) { return dfl(-x.h, -x.l); }
__device__ __forceinline__ dfl operator-(dfl x, dfl y) { return x + (-y); }
// x y: exact product of the high words by FMA, the cross terms added to its error
__device__ __forceinline__ dfl operator*(dfl x, dfl y) {
    const float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fmaf_rn(x.h, y.l, e);
    e = __fmaf_rn(x.l, y.h, e);
    return dfl_detail::fast_two_sum(p, e);
}
// x / y: a float quotient, corrected once by the double-float remainder
__device__ __forceinline__ dfl operator/(dfl x, dfl y) {
    const float q1 = __fdiv_rn(x.h, y.h);
    const dfl r = x - y * dfl(q1, 0.f);
    const float q2 = __fdiv_rn(r.h, y.h);
    return dfl_detail::fast_two_sum(q1, q2);
}
__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { a = a + b; return a; }
__device__ __forceinline__ dfl& operator-=(dfl& a, dfl b) { a = a - b; return a; }
__device__ __forceinline__ dfl& operator*=(dfl& a, dfl b) { a = a * b; return a; }
__device__ __forceinline__ bool operator==(dfl a, dfl b) { return a.h == b.h && a.l == b.l; }
__device__ __forceinline__ bool operator!=(dfl a, dfl b) { return !(a == b); }
// magnitude used by the pivot and singularity tests (normalised pairs: |h|)
__device__ __forceinline__ float fabs(dfl a) { return ::fabsf(a.h); }
__device__ __forceinline__ bool isfinite(dfl a) { return ::isfinite(a.h) && ::isfinite(a.l); }
#endif

template <typename T>
struct IsDoubleFloat { static constexpr bool value = false; };
template <>
struct IsDoubleFloat<dfl> { static constexpr bool value = true; };

template <>
struct RealOf<dfl> { using type = float; };

}  // namespace tsylv

// Double-precision complex numbers of the complex-triangular variant (the
// complex Schur forms of Sec. 2.4): a plain pair of doubles, laid out as
// interleaved (re, im) -- the memory layout of C99 double complex, of
// std::complex<double> and of torch.complex128 -- with the arithmetic the
// block kernels use.  Products and multiply-adds expand into real fused
// multiply-adds; the quotient uses Smith's algorithm (R. L. Smith, "Algorithm
// 116: Complex division", CACM 5(8), 1962), which avoids the overflow of the
// textbook formula.
#pragma once

namespace tsylv {

struct alignas(16) zd {
    double re, im;
    __host__ __device__ constexpr zd() : re(0), im(0) {}
    __host__ __device__ constexpr zd(double r) : re(r), im(0) {}
    __host__ __device__ constexpr zd(double r, double i) : re(r), im(i) {}
};

#if defined(__CUDACC__)
__device__ __forceinline__ zd operator+(zd a, zd b) { return zd(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ zd operator-(zd a, zd b) { return zd(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ zd operator-(zd a) { return zd(-a.re, -a.im); }
__device__ __forceinline__ zd operator*(zd a, zd b) {
    return zd(fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re));
}
__device__ __forceinline__ zd operator*(zd a, double s) { return zd(a.re * s, a.im * s); }
__device__ __forceinline__ zd operator/(zd a, zd b) {
    if (fabs(b.re) >= fabs(b.im)) {
        const double r = b.im / b.re, den = b.re + b.im * r;
        return zd((a.re + a.im * r) / den, (a.im - a.re * r) / den);
    }
    const double r = b.re / b.im, den = b.re * r + b.im;
    return zd((a.re * r + a.im) / den, (a.im * r - a.re) / den);
}
__device__ __forceinline__ zd& operator+=(zd& a, zd b) { a.re += b.re; a.im += b.im; return a; }
__device__ __forceinline__ zd& operator-=(zd& a, zd b) { a.re -= b.re; a.im -= b.im; return a; }
__device__ __forceinline__ zd& operator*=(zd& a, zd b) { a = a * b; return a; }
__device__ __forceinline__ bool operator==(zd a, zd b) { return a.re == b.re && a.im == b.im; }
__device__ __forceinline__ bool operator!=(zd a, zd b) { return !(a == b); }
// magnitude used by the pivot and singularity tests: |re| + |im| (within a
// factor sqrt(2) of the modulus)
__device__ __forceinline__ double fabs(zd a) { return ::fabs(a.re) + ::fabs(a.im); }
__device__ __forceinline__ bool isfinite(zd a) { return ::isfinite(a.re) && ::isfinite(a.im); }
// the real types' own (exact matches inside this namespace, ahead of the
// element types' overloads, which a double or float would otherwise reach by
// conversion)
__device__ __forceinline__ double fabs(double a) { return ::fabs(a); }
__device__ __forceinline__ float fabs(float a) { return ::fabsf(a); }
__device__ __forceinline__ bool isfinite(double a) { return ::isfinite(a); }
__device__ __forceinline__ bool isfinite(float a) { return ::isfinite(a); }
#endif

template <typename T>
struct IsComplex { static constexpr bool value = false; };
template <>
struct IsComplex<zd> { static constexpr bool value = true; };

// Real type of the magnitudes of T.
template <typename T>
struct RealOf { using type = T; };
template <>
struct RealOf<zd> { using type = double; };

}  // namespace tsylv

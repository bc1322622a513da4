// scalar.cuh -- the storage scalars of the kernels: float, double and their
// complex counterparts (time evolution makes the MPS complex, Sec. 2.2).
//
// cplx<R> is a plain aggregate (no constructors), so it can live in shared
// memory and in register arrays like a built-in type.  The helpers below are
// the only operations the kernels use on a scalar T besides + - *: for real T
// they are the identity or the obvious real operation, so the real kernels
// compile to the same instructions as before.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace thc {

template <class R>
struct cplx {
    R x, y;  // real and imaginary parts
};
using c32 = cplx<float>;
using c64 = cplx<double>;

template <class T> struct ScalarOf { using real = T; static constexpr bool complex = false; };
template <class R> struct ScalarOf<cplx<R>> { using real = R; static constexpr bool complex = true; };
template <class T> using real_t = typename ScalarOf<T>::real;
template <class T> constexpr bool is_complex_v = ScalarOf<T>::complex;

// float64 accumulator of a storage type: double for real, c64 for complex
template <class T> struct Wide { using type = double; };
template <class R> struct Wide<cplx<R>> { using type = c64; };

#define THC_HD __host__ __device__ __forceinline__

template <class R> THC_HD cplx<R> operator+(cplx<R> a, cplx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <class R> THC_HD cplx<R> operator-(cplx<R> a, cplx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <class R> THC_HD cplx<R> operator-(cplx<R> a) { return {-a.x, -a.y}; }
template <class R> THC_HD cplx<R> operator*(cplx<R> a, cplx<R> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class R> THC_HD cplx<R> operator*(R a, cplx<R> b) { return {a * b.x, a * b.y}; }
template <class R> THC_HD cplx<R> operator*(cplx<R> a, R b) { return {a.x * b, a.y * b}; }
template <class R> THC_HD cplx<R>& operator+=(cplx<R>& a, cplx<R> b) { a.x += b.x; a.y += b.y; return a; }
template <class R> THC_HD cplx<R>& operator-=(cplx<R>& a, cplx<R> b) { a.x -= b.x; a.y -= b.y; return a; }
template <class R> THC_HD cplx<R>& operator*=(cplx<R>& a, cplx<R> b) { a = a * b; return a; }
template <class R> THC_HD cplx<R>& operator*=(cplx<R>& a, R b) { a.x *= b; a.y *= b; return a; }
template <class R> THC_HD bool operator==(cplx<R> a, cplx<R> b) { return a.x == b.x && a.y == b.y; }
template <class R> THC_HD bool operator!=(cplx<R> a, cplx<R> b) { return !(a == b); }

// zero, one and a real value in type T
template <class T> THC_HD T tzero() {
    if constexpr (is_complex_v<T>) return T{0, 0};
    else return T(0);
}
template <class T> THC_HD T tone() {
    if constexpr (is_complex_v<T>) return T{1, 0};
    else return T(1);
}
template <class T> THC_HD T treal(real_t<T> r) {
    if constexpr (is_complex_v<T>) return T{r, 0};
    else return r;
}

// conversion between storage and accumulator types (real -> complex adds a
// zero imaginary part; complex -> real is not used)
template <class D, class S> THC_HD D cvt(S s) {
    if constexpr (is_complex_v<D> && is_complex_v<S>) return D{real_t<D>(s.x), real_t<D>(s.y)};
    else if constexpr (is_complex_v<D>) return D{real_t<D>(s), real_t<D>(0)};
    else {
        static_assert(!is_complex_v<S>, "complex to real conversion");
        return D(s);
    }
}

template <class T> THC_HD T tconj(T a) {
    if constexpr (is_complex_v<T>) return T{a.x, -a.y};
    else return a;
}
// |a|^2 in the real type of T
template <class T> THC_HD real_t<T> tabs2(T a) {
    if constexpr (is_complex_v<T>) return a.x * a.x + a.y * a.y;
    else return a * a;
}
// largest |component| (real and imaginary parts separately)
template <class T> THC_HD real_t<T> tmaxabs(T a) {
    if constexpr (is_complex_v<T>) return fmax(fabs(a.x), fabs(a.y));
    else return fabs(a);
}
template <class T> THC_HD real_t<T> treal_part(T a) {
    if constexpr (is_complex_v<T>) return a.x;
    else return a;
}
template <class T> THC_HD bool tisfinite_sq(T a) {  // |a|^2 is a finite number
    const real_t<T> v = tabs2(a);
    return v == v && v < real_t<T>(1e300);
}
// conj(a) * b
template <class T> THC_HD T tconj_mul(T a, T b) {
    if constexpr (is_complex_v<T>) return T{a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
    else return a * b;
}
// a * r for a real r
template <class T> THC_HD T tscale(T a, real_t<T> r) {
    if constexpr (is_complex_v<T>) return T{a.x * r, a.y * r};
    else return a * r;
}

// warp shuffles of a scalar (both parts of a complex value)
template <class T> __device__ __forceinline__ T shfl_xor(T v, int o) {
    if constexpr (is_complex_v<T>)
        return T{__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)};
    else return __shfl_xor_sync(0xffffffffu, v, o);
}
template <class T> __device__ __forceinline__ T shfl(T v, int src) {
    if constexpr (is_complex_v<T>)
        return T{__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)};
    else return __shfl_sync(0xffffffffu, v, src);
}

// warp-wide sum of a complex value (every lane gets the total)
template <class R> __device__ __forceinline__ cplx<R> warp_sum(cplx<R> v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
    return v;
}

#undef THC_HD

}  // namespace thc

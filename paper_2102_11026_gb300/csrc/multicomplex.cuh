// Exact multicomplex arithmetic in FP32, for the untruncated activation (an ablation of
// the truncated Taylor form of the epilogue).  A number of level n + 1 is X + i Y with X,
// Y of level n and a new imaginary unit i (i^2 = -1) commuting with the units below:
// level 1 the complex numbers in i2 over the reals, level 2 the bicomplex numbers in i3
// over level 1, level 3 the tricomplex numbers in i1 over level 2 (Sec. 4.1, Eq. 16: the
// multicomplex step puts every perturbation on its own unit).  Functions of X + i Y come
// from the addition theorems, which hold for commuting arguments:
//   sin(X + iY)  = sin X cosh Y + i cos X sinh Y      cos(X + iY)  = cos X cosh Y - i sin X sinh Y
//   sinh(X + iY) = sinh X cos Y + i cosh X sin Y      cosh(X + iY) = cosh X cos Y + i sinh X sin Y
//   tanh(X + iY) = (sinh 2X + i sin 2Y) / (cosh 2X + cos 2Y)
// and (X + iY)^-1 = (X - iY) (X^2 + Y^2)^-1.  No form here splits a number into
// idempotent parts (that reintroduces cancellation in the mixed components); every
// component is a sum of products of components of its own order.
#pragma once
#include <cuda_runtime.h>

namespace dae {
namespace mc {

template <class T>
struct M {
    T x, y;   // x + i y
};

__device__ __forceinline__ float neg(float a) { return -a; }
template <class T>
__device__ __forceinline__ M<T> neg(const M<T>& a) { return {neg(a.x), neg(a.y)}; }

__device__ __forceinline__ float add(float a, float b) { return a + b; }
template <class T>
__device__ __forceinline__ M<T> add(const M<T>& a, const M<T>& b) { return {add(a.x, b.x), add(a.y, b.y)}; }

__device__ __forceinline__ float sub(float a, float b) { return a - b; }
template <class T>
__device__ __forceinline__ M<T> sub(const M<T>& a, const M<T>& b) { return {sub(a.x, b.x), sub(a.y, b.y)}; }

__device__ __forceinline__ float mul(float a, float b) { return a * b; }
template <class T>
__device__ __forceinline__ M<T> mul(const M<T>& a, const M<T>& b) {
    return {sub(mul(a.x, b.x), mul(a.y, b.y)), add(mul(a.x, b.y), mul(a.y, b.x))};
}

__device__ __forceinline__ float scale(float s, float a) { return s * a; }
template <class T>
__device__ __forceinline__ M<T> scale(float s, const M<T>& a) { return {scale(s, a.x), scale(s, a.y)}; }

__device__ __forceinline__ float inv(float a) { return 1.0f / a; }
template <class T>
__device__ __forceinline__ M<T> inv(const M<T>& a) {
    const T n = inv(add(mul(a.x, a.x), mul(a.y, a.y)));
    return {mul(a.x, n), neg(mul(a.y, n))};
}

__device__ __forceinline__ float fsin(float a) { return sinf(a); }
__device__ __forceinline__ float fcos(float a) { return cosf(a); }
__device__ __forceinline__ float fsinh(float a) { return sinhf(a); }
__device__ __forceinline__ float fcosh(float a) { return coshf(a); }
__device__ __forceinline__ float ftanh(float a) { return tanhf(a); }

template <class T>
__device__ __forceinline__ M<T> fsin(const M<T>& a) {
    return {mul(fsin(a.x), fcosh(a.y)), mul(fcos(a.x), fsinh(a.y))};
}
template <class T>
__device__ __forceinline__ M<T> fcos(const M<T>& a) {
    return {mul(fcos(a.x), fcosh(a.y)), neg(mul(fsin(a.x), fsinh(a.y)))};
}
template <class T>
__device__ __forceinline__ M<T> fsinh(const M<T>& a) {
    return {mul(fsinh(a.x), fcos(a.y)), mul(fcosh(a.x), fsin(a.y))};
}
template <class T>
__device__ __forceinline__ M<T> fcosh(const M<T>& a) {
    return {mul(fcosh(a.x), fcos(a.y)), mul(fsinh(a.x), fsin(a.y))};
}
template <class T>
__device__ __forceinline__ M<T> ftanh(const M<T>& a) {
    const T x2 = scale(2.0f, a.x), y2 = scale(2.0f, a.y);
    const T d = inv(add(fcosh(x2), fcos(y2)));
    return {mul(fsinh(x2), d), mul(fsin(y2), d)};
}

using C1 = M<float>;   // x + i2 y
using C2 = M<C1>;      // X + i3 Y
using C3 = M<C2>;      // X + i1 Y

// The activation (dae_act) of a multicomplex argument.
template <class T>
__device__ __forceinline__ T act(int a, const T& z) {
    if (a == DAE_ACT_TANH) return ftanh(z);
    if (a == DAE_ACT_SIN) return fsin(z);
    return z;
}

}  // namespace mc
}  // namespace dae

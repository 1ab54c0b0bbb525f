// common.cuh -- complex scalar type and small device helpers shared by the
// sm_103a kernels of the mixed-precision matrix square root.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace sqm {

// Interleaved complex value (same layout as torch.complex64 / complex128).
template <class R>
struct alignas(2 * sizeof(R)) cplx {
    R x, y;
};

template <class R> __host__ __device__ __forceinline__ cplx<R> mk(R a, R b) { return cplx<R>{a, b}; }
template <class R> __host__ __device__ __forceinline__ cplx<R> operator+(cplx<R> a, cplx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <class R> __host__ __device__ __forceinline__ cplx<R> operator-(cplx<R> a, cplx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <class R> __host__ __device__ __forceinline__ cplx<R> operator-(cplx<R> a) { return {-a.x, -a.y}; }
template <class R> __host__ __device__ __forceinline__ cplx<R> operator*(cplx<R> a, cplx<R> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class R> __host__ __device__ __forceinline__ cplx<R> operator*(R s, cplx<R> a) { return {s * a.x, s * a.y}; }
template <class R> __host__ __device__ __forceinline__ cplx<R> &operator+=(cplx<R> &a, cplx<R> b) { a.x += b.x; a.y += b.y; return a; }
template <class R> __host__ __device__ __forceinline__ cplx<R> &operator-=(cplx<R> &a, cplx<R> b) { a.x -= b.x; a.y -= b.y; return a; }
template <class R> __host__ __device__ __forceinline__ cplx<R> conj(cplx<R> a) { return {a.x, -a.y}; }
template <class R> __host__ __device__ __forceinline__ R abs2(cplx<R> a) { return a.x * a.x + a.y * a.y; }
template <class R> __device__ __forceinline__ R cabs_(cplx<R> a) { return hypot(a.x, a.y); }

// acc += a * b (complex fused multiply-add, 4 real FMAs)
template <class R> __device__ __forceinline__ void cfma(cplx<R> &acc, cplx<R> a, cplx<R> b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc -= a * b
template <class R> __device__ __forceinline__ void cfms(cplx<R> &acc, cplx<R> a, cplx<R> b) {
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}

// Complex division a / b by Smith's method (R. L. Smith, CACM 5(8), 1962):
// scale by the larger component of b to avoid overflow in |b|^2.
template <class R> __device__ __forceinline__ cplx<R> cdiv(cplx<R> a, cplx<R> b) {
    if (fabs(b.x) >= fabs(b.y)) {
        R r = b.y / b.x, den = b.x + b.y * r;
        return {(a.x + a.y * r) / den, (a.y - a.x * r) / den};
    }
    R r = b.x / b.y, den = b.x * r + b.y;
    return {(a.x * r + a.y) / den, (a.y * r - a.x) / den};
}

// Principal square root: for z = x + iy, t = sqrt((|x| + |z|) / 2);
// x >= 0: t + i y/(2t); x < 0: |y|/(2t) + i sign(y) t.  Both branches avoid
// cancellation, and the real part is >= 0 (principal branch).
template <class R> __device__ __forceinline__ cplx<R> csqrt_(cplx<R> z) {
    if (z.x == R(0) && z.y == R(0)) return {R(0), R(0)};
    R t = sqrt(R(0.5) * (fabs(z.x) + hypot(z.x, z.y)));
    if (z.x >= R(0)) return {t, z.y / (R(2) * t)};
    return {fabs(z.y) / (R(2) * t), copysign(t, z.y)};
}

template <class R> struct num;
template <> struct num<float> {
    static constexpr float eps = 5.9604644775390625e-08f;  // 2^-24
};
template <> struct num<double> {
    static constexpr double eps = 1.1102230246251565e-16;  // 2^-53
};

// Asynchronous global -> shared copy of one complex element (Ampere-style
// cp.async; the thread does not wait for the load).  Complete with
// cp_async_wait_all() followed by a barrier.
template <class R> __device__ __forceinline__ void cp_async_elem(cplx<R> *smem, const cplx<R> *gmem);
template <> __device__ __forceinline__ void cp_async_elem<float>(cplx<float> *smem, const cplx<float> *gmem)
{
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
template <> __device__ __forceinline__ void cp_async_elem<double>(cplx<double> *smem, const cplx<double> *gmem)
{
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <class T> __device__ __forceinline__ T shfl_xor(T v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
template <class R> __device__ __forceinline__ cplx<R> shfl_xor(cplx<R> v, int m) {
    return {__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m)};
}

template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += shfl_xor(v, m);
    return v;
}

__host__ __device__ __forceinline__ int64_t cdiv_i(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace sqm

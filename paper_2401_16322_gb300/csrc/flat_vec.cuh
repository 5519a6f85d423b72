// 16-byte vector helpers of the flat Krylov passes (kernels_aux.cu) and the Gram-Schmidt
// column kernel (kernels_mgs.cu).  Both take their products, updates and dot products from
// here, so that the two forms of a pass compute the same values bit for bit.
#pragma once

#include "ewave_internal.cuh"

namespace ewv {

template <typename T>
__device__ __forceinline__ T* vptr(const ProblemDev* P, int k) {
    return k == 0 ? (T*)P->state : (T*)P->work + (long long)(k - 1) * P->vec_stride;
}

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
    static constexpr int N = 4;
};
template <>
struct Vec16<double> {
    using type = double2;
    static constexpr int N = 2;
};

__device__ __forceinline__ float dot16(const float4& a, const float4& b) {
    return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)));
}
__device__ __forceinline__ double dot16d(const double2& a, const double2& b) {
    return fma(a.y, b.y, a.x * b.x);
}
__device__ __forceinline__ float4 axpy16(const float4& w, float c, const float4& q) {
    return make_float4(fmaf(-c, q.x, w.x), fmaf(-c, q.y, w.y), fmaf(-c, q.z, w.z), fmaf(-c, q.w, w.w));
}
__device__ __forceinline__ double2 axpy16(const double2& w, double c, const double2& q) {
    return make_double2(fma(-c, q.x, w.x), fma(-c, q.y, w.y));
}
__device__ __forceinline__ void fma16(float4& acc, float c, const float4& q) {
    acc.x = fmaf(c, q.x, acc.x);
    acc.y = fmaf(c, q.y, acc.y);
    acc.z = fmaf(c, q.z, acc.z);
    acc.w = fmaf(c, q.w, acc.w);
}
__device__ __forceinline__ void fma16(double2& acc, double c, const double2& q) {
    acc.x = fma(c, q.x, acc.x);
    acc.y = fma(c, q.y, acc.y);
}
// dot product of one 16-byte vector, widened to FP64 for the accumulation
__device__ __forceinline__ double dotv(const float4& a, const float4& b) { return (double)dot16(a, b); }
__device__ __forceinline__ double dotv(const double2& a, const double2& b) { return dot16d(a, b); }

}  // namespace ewv

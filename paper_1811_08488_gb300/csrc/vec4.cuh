// Flat element-wise access to native fields in groups of four reals, and the
// per-thread compensated sums of the BLAS-1 kernels (blas.cu, eig.cu).
#pragma once

#include <type_traits>

#include "dwf_internal.cuh"

namespace dwf {

// Group i of a native field: the 4 reals [4c, 4c+4) of element e = site*Ls + s,
// numbered in FP32 order i = c * cs + e (cs = nsite * Ls, chunk-major). In an
// FP32 field this is the float4 at index i; in an FP64 field it is the double2
// chunks 2c and 2c+1 of e, at (2c) * cs + e and (2c + 1) * cs + e. Kernels that
// mix precisions therefore meet the same (site, s, component) on both sides.
template <class S, class U>
__device__ __forceinline__ void ld4(const char *p, long long i, long long cs, U v[4]) {
  if constexpr (std::is_same<S, F32>::value) {
    float4 q = reinterpret_cast<const float4 *>(p)[i];
    v[0] = (U)q.x; v[1] = (U)q.y; v[2] = (U)q.z; v[3] = (U)q.w;
  } else {
    const long long c = i / cs, e = i - c * cs;
    const long long j = 2 * c * cs + e;
    double2 a = reinterpret_cast<const double2 *>(p)[j];
    double2 b = reinterpret_cast<const double2 *>(p)[j + cs];
    v[0] = (U)a.x; v[1] = (U)a.y; v[2] = (U)b.x; v[3] = (U)b.y;
  }
}
template <class S, class U>
__device__ __forceinline__ void st4(char *p, long long i, long long cs, const U v[4]) {
  if constexpr (std::is_same<S, F32>::value) {
    reinterpret_cast<float4 *>(p)[i] =
        make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
  } else {
    const long long c = i / cs, e = i - c * cs;
    const long long j = 2 * c * cs + e;
    reinterpret_cast<double2 *>(p)[j] = make_double2((double)v[0], (double)v[1]);
    reinterpret_cast<double2 *>(p)[j + cs] = make_double2((double)v[2], (double)v[3]);
  }
}
#define FLAT_LOOP(n4)                                                              \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n4); \
       i += (long long)gridDim.x * blockDim.x)

// Per-thread sums: compensated (Kahan) in FP32 for FP32 fields, plain FP64 for
// FP64 fields; the cross-thread and cross-CTA sums are FP64. FP64 arithmetic
// per element would run on GB300's small FP64 pipe and make these
// bandwidth-bound kernels compute-bound.
struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
struct SumD {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <class SL> struct Acc { using T = KahanF; using R = float; };
template <> struct Acc<F64> { using T = SumD; using R = double; };

template <class R>
__device__ __forceinline__ R sq4(const R v[4]) {
  return v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
}

}  // namespace dwf

// Device helpers shared by the kernels: native-field loads and stores, link
// records, and the Ls-direction operator applied by one thread per
// (site, spin-colour component).
#pragma once

#include "dwf_internal.cuh"

namespace dwf {

// ---------------------------------------------------------------------------
// Native field access. Spinor reals are ordered [spin][colour][re, im]; the
// upper chirality (P_+, spins 0-1) is reals 0..11, the lower (P_-) 12..23.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 h2f(const __half2 h) { return __half22float2(h); }
__device__ __forceinline__ float2 h2f(const __nv_bfloat162 h) { return __bfloat1622float2(h); }

template <class S> struct Half2Of { using T = __half2; };
template <> struct Half2Of<BF16> { using T = __nv_bfloat162; };

__device__ __forceinline__ __half2 f2h(float a, float b, __half2 *) { return __floats2half2_rn(a, b); }
__device__ __forceinline__ __nv_bfloat162 f2h(float a, float b, __nv_bfloat162 *) {
  return __floats2bfloat162_rn(a, b);
}

template <class S>
__device__ __forceinline__ void unpack8(const uint4 q, float *v) {
  using H2 = typename Half2Of<S>::T;
  const H2 *h = reinterpret_cast<const H2 *>(&q);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float2 f = h2f(h[i]);
    v[2 * i] = f.x;
    v[2 * i + 1] = f.y;
  }
}

template <class S>
__device__ __forceinline__ uint4 pack8(const float *v, float scl) {
  using H2 = typename Half2Of<S>::T;
  uint4 q;
  H2 *h = reinterpret_cast<H2 *>(&q);
#pragma unroll
  for (int i = 0; i < 4; ++i) h[i] = f2h(v[2 * i] * scl, v[2 * i + 1] * scl, (H2 *)nullptr);
  return q;
}

// Load the 24 reals of (site, s).
template <class S>
__device__ __forceinline__ void load24(const char *base, long long soff, int site, int s, int Ls,
                                       typename S::R *v) {
  if constexpr (std::is_same<S, F32>::value) {
    const float4 *p = reinterpret_cast<const float4 *>(base) + (size_t)site * 6 * Ls + s;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float4 q = __ldg(p + k * Ls);
      v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
    }
  } else if constexpr (std::is_same<S, F64>::value) {
    const double2 *p = reinterpret_cast<const double2 *>(base) + (size_t)site * 12 * Ls + s;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double2 q = __ldg(p + k * Ls);
      v[2 * k] = q.x; v[2 * k + 1] = q.y;
    }
  } else {
    const uint4 *p = reinterpret_cast<const uint4 *>(base) + (size_t)site * 3 * Ls + s;
    const float scl = __ldg(reinterpret_cast<const float *>(base + soff) + (size_t)site * Ls + s);
#pragma unroll
    for (int k = 0; k < 3; ++k) unpack8<S>(__ldg(p + k * Ls), v + 8 * k);
#pragma unroll
    for (int k = 0; k < 24; ++k) v[k] *= scl;
  }
}

// Load one chirality (UPPER: reals 0..11, else 12..23) of (site, s) into v[0..12).
template <class S, bool UPPER>
__device__ __forceinline__ void load12(const char *base, long long soff, int site, int s, int Ls,
                                       typename S::R *v) {
  if constexpr (std::is_same<S, F32>::value) {
    const float4 *p = reinterpret_cast<const float4 *>(base) + (size_t)site * 6 * Ls + s +
                      (UPPER ? 0 : 3 * Ls);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float4 q = __ldg(p + k * Ls);
      v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
    }
  } else if constexpr (std::is_same<S, F64>::value) {
    const double2 *p = reinterpret_cast<const double2 *>(base) + (size_t)site * 12 * Ls + s +
                       (UPPER ? 0 : 6 * Ls);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      double2 q = __ldg(p + k * Ls);
      v[2 * k] = q.x; v[2 * k + 1] = q.y;
    }
  } else {
    const uint4 *p = reinterpret_cast<const uint4 *>(base) + (size_t)site * 3 * Ls + s;
    const float scl = __ldg(reinterpret_cast<const float *>(base + soff) + (size_t)site * Ls + s);
    float w[16];
    if (UPPER) {
      unpack8<S>(__ldg(p), w);
      unpack8<S>(__ldg(p + Ls), w + 8);
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = w[k] * scl;
    } else {
      unpack8<S>(__ldg(p + Ls), w);
      unpack8<S>(__ldg(p + 2 * Ls), w + 8);
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = w[k + 4] * scl;
    }
  }
}

// Store the 24 reals of (site, s); FP16/BF16 stores v / max|v| and the scale.
template <class S>
__device__ __forceinline__ void store24(char *base, long long soff, int site, int s, int Ls,
                                        const typename S::R *v) {
  if constexpr (std::is_same<S, F32>::value) {
    float4 *p = reinterpret_cast<float4 *>(base) + (size_t)site * 6 * Ls + s;
#pragma unroll
    for (int k = 0; k < 6; ++k)
      p[k * Ls] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  } else if constexpr (std::is_same<S, F64>::value) {
    double2 *p = reinterpret_cast<double2 *>(base) + (size_t)site * 12 * Ls + s;
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k * Ls] = make_double2(v[2 * k], v[2 * k + 1]);
  } else {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 24; ++k) m = fmaxf(m, fabsf(v[k]));
    const float inv = m > 0.f ? 1.0f / m : 0.f;
    uint4 *p = reinterpret_cast<uint4 *>(base) + (size_t)site * 3 * Ls + s;
#pragma unroll
    for (int k = 0; k < 3; ++k) p[k * Ls] = pack8<S>(v + 8 * k, inv);
    reinterpret_cast<float *>(base + soff)[(size_t)site * Ls + s] = m;
  }
}

// ---------------------------------------------------------------------------
// Link records: 18 reals of U[a][b] (row-major complex) per (owner, mu).
// ---------------------------------------------------------------------------
template <class S>
__device__ __forceinline__ void load_link(const char *links, int owner, int mu,
                                          typename S::R *u) {
  const size_t rec = (size_t)owner * 4 + mu;
  if constexpr (std::is_same<S, F64>::value) {
    const double2 *p = reinterpret_cast<const double2 *>(links) + rec * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double2 q = __ldg(p + k);
      u[2 * k] = q.x; u[2 * k + 1] = q.y;
    }
  } else if constexpr (std::is_same<S, F32>::value) {
    const float4 *p = reinterpret_cast<const float4 *>(links) + rec * 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float4 q = __ldg(p + k);
      u[4 * k] = q.x; u[4 * k + 1] = q.y; u[4 * k + 2] = q.z; u[4 * k + 3] = q.w;
    }
    float2 q = __ldg(reinterpret_cast<const float2 *>(p + 4));
    u[16] = q.x; u[17] = q.y;
  } else {
    const uint4 *p = reinterpret_cast<const uint4 *>(links) + rec * 3;
    float w[24];
#pragma unroll
    for (int k = 0; k < 3; ++k) unpack8<F16>(__ldg(p + k), w + 8 * k);
#pragma unroll
    for (int k = 0; k < 18; ++k) u[k] = w[k];
  }
}

// ---------------------------------------------------------------------------
// Ls-direction operator on one (site, component) column T[0..Ls) in shared
// memory (stride 1):
//     T <- q0 (p0 + p1 S) [(1 - r S)^-1 if inv] T  +  (a0 + a1 S) X  (if X)
// S is the chiral shift; `down` selects (S v)_j = v_{j-1}, (S v)_0 = -mf v_{Ls-1},
// otherwise (S v)_j = v_{j+1}, (S v)_{Ls-1} = -mf v_0. The inverse uses the
// closed form y_0 = (v_0 - mf sum_{k=1}^{Ls-1} r^k v_{Ls-k}) / (1 + mf r^Ls),
// y_j = v_j + r y_{j-1} (in the shift's own index order).
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void ls_column(R *T, const R *X, int Ls, bool down, bool inv,
                                          const LsCoef &c) {
  auto ix = [&](int j) { return down ? j : Ls - 1 - j; };
  const R mf = (R)c.mf;
  if (inv) {
    const R r = (R)c.r;
    R acc = 0, rk = r;
    for (int k = 1; k < Ls; ++k) {
      acc += rk * T[ix(Ls - k)];
      rk *= r;
    }
    R y = (T[ix(0)] - mf * acc) * (R)c.inv_den;
    T[ix(0)] = y;
    for (int j = 1; j < Ls; ++j) {
      y = T[ix(j)] + r * y;
      T[ix(j)] = y;
    }
  }
  const R p0 = (R)(c.q0 * c.p0), p1 = (R)(c.q0 * c.p1);
  const R last = T[ix(Ls - 1)];
  for (int j = Ls - 1; j >= 1; --j) T[ix(j)] = p0 * T[ix(j)] + p1 * T[ix(j - 1)];
  T[ix(0)] = p0 * T[ix(0)] - p1 * mf * last;
  if (X) {
    const R a0 = (R)c.a0, a1 = (R)c.a1;
    for (int j = 1; j < Ls; ++j) T[ix(j)] += a0 * X[ix(j)] + a1 * X[ix(j - 1)];
    T[ix(0)] += a0 * X[ix(0)] - a1 * mf * X[ix(Ls - 1)];
  }
}

// ---------------------------------------------------------------------------
// Deterministic CTA reduction of one double per thread; result in thread 0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double cta_sum(double v, double *sh /* >= 32 */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) t += sh[i];
  }
  return t;
}

// Publish one CTA partial. The last CTA of the group to arrive sums all
// partials in a fixed order; the call returns true in its thread 0 with the sum
// in `total` (false everywhere else). Must be called by all threads of the CTA.
__device__ __forceinline__ bool group_reduce(double cta_val, double *partials, int ntiles,
                                             int tile, unsigned int *counter, double &total) {
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    partials[tile] = cta_val;
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    s_last = (prev == (unsigned int)ntiles - 1u);
  }
  __syncthreads();
  bool last = false;
  if (s_last && threadIdx.x < 32) {
    __threadfence();
    double a = 0.0;
    const volatile double *vp = partials;
    for (int i = threadIdx.x; i < ntiles; i += 32) a += vp[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (threadIdx.x == 0) {
      total = a;
      *counter = 0u;
      last = true;
    }
  }
  return last;
}

}  // namespace dwf

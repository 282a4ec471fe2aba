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

// Native layout of one right-hand side (of one block): element e = site*Ls + s,
// 16-byte chunk c of element e at chunk index c * cs + e with cs = nsite*Ls
// (chunk-major), so the chunk c of consecutive (site, s) is contiguous and a
// warp's load of one chunk is a contiguous 512-byte segment. FP16/BF16 scales
// are one float per element at byte offset soff.
template <class S>
__device__ __forceinline__ void load24(const char *base, long long soff, int cs, int e,
                                       typename S::R *v) {
  if constexpr (std::is_same<S, F32>::value) {
    const float4 *p = reinterpret_cast<const float4 *>(base) + e;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float4 q = __ldg(p + (size_t)k * cs);
      v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
    }
  } else if constexpr (std::is_same<S, F64>::value) {
    const double2 *p = reinterpret_cast<const double2 *>(base) + e;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double2 q = __ldg(p + (size_t)k * cs);
      v[2 * k] = q.x; v[2 * k + 1] = q.y;
    }
  } else {
    const uint4 *p = reinterpret_cast<const uint4 *>(base) + e;
    const float scl = __ldg(reinterpret_cast<const float *>(base + soff) + e);
#pragma unroll
    for (int k = 0; k < 3; ++k) unpack8<S>(__ldg(p + (size_t)k * cs), v + 8 * k);
#pragma unroll
    for (int k = 0; k < 24; ++k) v[k] *= scl;
  }
}

// Load one chirality (UPPER: reals 0..11, else 12..23) of element e into v[0..12).
template <class S, bool UPPER>
__device__ __forceinline__ void load12(const char *base, long long soff, int cs, int e,
                                       typename S::R *v) {
  if constexpr (std::is_same<S, F32>::value) {
    const float4 *p = reinterpret_cast<const float4 *>(base) + e + (UPPER ? 0 : (size_t)3 * cs);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float4 q = __ldg(p + (size_t)k * cs);
      v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
    }
  } else if constexpr (std::is_same<S, F64>::value) {
    const double2 *p = reinterpret_cast<const double2 *>(base) + e + (UPPER ? 0 : (size_t)6 * cs);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      double2 q = __ldg(p + (size_t)k * cs);
      v[2 * k] = q.x; v[2 * k + 1] = q.y;
    }
  } else {
    const uint4 *p = reinterpret_cast<const uint4 *>(base) + e;
    const float scl = __ldg(reinterpret_cast<const float *>(base + soff) + e);
    float w[16];
    if (UPPER) {
      unpack8<S>(__ldg(p), w);
      unpack8<S>(__ldg(p + cs), w + 8);
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = w[k] * scl;
    } else {
      unpack8<S>(__ldg(p + cs), w);
      unpack8<S>(__ldg(p + (size_t)2 * cs), w + 8);
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = w[k + 4] * scl;
    }
  }
}

// Store the 24 reals of element e; FP16/BF16 stores v / max|v| and the scale.
template <class S>
__device__ __forceinline__ void store24(char *base, long long soff, int cs, int e,
                                        const typename S::R *v) {
  if constexpr (std::is_same<S, F32>::value) {
    float4 *p = reinterpret_cast<float4 *>(base) + e;
#pragma unroll
    for (int k = 0; k < 6; ++k)
      p[(size_t)k * cs] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  } else if constexpr (std::is_same<S, F64>::value) {
    double2 *p = reinterpret_cast<double2 *>(base) + e;
#pragma unroll
    for (int k = 0; k < 12; ++k) p[(size_t)k * cs] = make_double2(v[2 * k], v[2 * k + 1]);
  } else {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 24; ++k) m = fmaxf(m, fabsf(v[k]));
    const float inv = m > 0.f ? 1.0f / m : 0.f;
    uint4 *p = reinterpret_cast<uint4 *>(base) + e;
#pragma unroll
    for (int k = 0; k < 3; ++k) p[(size_t)k * cs] = pack8<S>(v + 8 * k, inv);
    reinterpret_cast<float *>(base + soff)[e] = m;
  }
}

// ---------------------------------------------------------------------------
// Pairs of adjacent elements (e, e+1), e even: chunk c of both is one 32-byte
// word, moved with a single 256-bit load or store (sm_100 and later). A warp
// request of 32 such words is one contiguous kilobyte.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ldg256(const void *p, uint32_t (&a)[8]) {
  asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]),
                 "=r"(a[6]), "=r"(a[7])
               : "l"(p));
}
__device__ __forceinline__ void stg256(void *p, const uint32_t (&a)[8]) {
  asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(a[0]),
               "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7])
               : "memory");
}

// Load the 24 reals of elements e (v0) and e+1 (v1); e even. FP32/FP16/BF16.
template <class S>
__device__ __forceinline__ void load24x2(const char *base, long long soff, int cs, int e,
                                         float *v0, float *v1) {
  const uint4 *p = reinterpret_cast<const uint4 *>(base) + e;
  if constexpr (std::is_same<S, F32>::value) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      uint32_t a[8];
      ldg256(p + (size_t)k * cs, a);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        v0[4 * k + i] = __uint_as_float(a[i]);
        v1[4 * k + i] = __uint_as_float(a[4 + i]);
      }
    }
  } else {
    const float2 scl = __ldg(reinterpret_cast<const float2 *>(base + soff) + e / 2);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint32_t a[8];
      ldg256(p + (size_t)k * cs, a);
      unpack8<S>(make_uint4(a[0], a[1], a[2], a[3]), v0 + 8 * k);
      unpack8<S>(make_uint4(a[4], a[5], a[6], a[7]), v1 + 8 * k);
    }
#pragma unroll
    for (int k = 0; k < 24; ++k) {
      v0[k] *= scl.x;
      v1[k] *= scl.y;
    }
  }
}

// One chirality (UPPER: reals 0..11, else 12..23) of elements e (v0) and e+1
// (v1); e even. FP32/FP16/BF16, 256-bit loads as in load24x2.
template <class S, bool UPPER>
__device__ __forceinline__ void load12x2(const char *base, long long soff, int cs, int e,
                                         float *v0, float *v1) {
  const uint4 *p = reinterpret_cast<const uint4 *>(base) + e;
  if constexpr (std::is_same<S, F32>::value) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint32_t a[8];
      ldg256(p + (size_t)(UPPER ? k : 3 + k) * cs, a);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        v0[4 * k + i] = __uint_as_float(a[i]);
        v1[4 * k + i] = __uint_as_float(a[4 + i]);
      }
    }
  } else {
    const float2 scl = __ldg(reinterpret_cast<const float2 *>(base + soff) + e / 2);
    float t0[16], t1[16];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      uint32_t a[8];
      ldg256(p + (size_t)(UPPER ? k : 1 + k) * cs, a);
      unpack8<S>(make_uint4(a[0], a[1], a[2], a[3]), t0 + 8 * k);
      unpack8<S>(make_uint4(a[4], a[5], a[6], a[7]), t1 + 8 * k);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      v0[k] = t0[UPPER ? k : 4 + k] * scl.x;
      v1[k] = t1[UPPER ? k : 4 + k] * scl.y;
    }
  }
}

// FP16/BF16: the stored values of elements e and e+1 (e even) without their
// scales, which are returned in scl (the caller folds them in later).
template <class S>
__device__ __forceinline__ void load24x2_unscaled(const char *base, long long soff, int cs, int e,
                                                  float *v0, float *v1, float2 &scl) {
  const uint4 *p = reinterpret_cast<const uint4 *>(base) + e;
  scl = __ldg(reinterpret_cast<const float2 *>(base + soff) + e / 2);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    uint32_t a[8];
    ldg256(p + (size_t)k * cs, a);
    unpack8<S>(make_uint4(a[0], a[1], a[2], a[3]), v0 + 8 * k);
    unpack8<S>(make_uint4(a[4], a[5], a[6], a[7]), v1 + 8 * k);
  }
}

// Store the 24 reals of elements e (v0) and e+1 (v1); e even. FP16/BF16 store
// each element relative to its own maximum.
template <class S>
__device__ __forceinline__ void store24x2(char *base, long long soff, int cs, int e,
                                          const float *v0, const float *v1) {
  uint4 *p = reinterpret_cast<uint4 *>(base) + e;
  if constexpr (std::is_same<S, F32>::value) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      uint32_t a[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = __float_as_uint(v0[4 * k + i]);
        a[4 + i] = __float_as_uint(v1[4 * k + i]);
      }
      stg256(p + (size_t)k * cs, a);
    }
  } else {
    float m0 = 0.f, m1 = 0.f;
#pragma unroll
    for (int k = 0; k < 24; ++k) {
      m0 = fmaxf(m0, fabsf(v0[k]));
      m1 = fmaxf(m1, fabsf(v1[k]));
    }
    const float i0 = m0 > 0.f ? 1.0f / m0 : 0.f, i1 = m1 > 0.f ? 1.0f / m1 : 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const uint4 q0 = pack8<S>(v0 + 8 * k, i0), q1 = pack8<S>(v1 + 8 * k, i1);
      const uint32_t a[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
      stg256(p + (size_t)k * cs, a);
    }
    reinterpret_cast<float2 *>(base + soff)[e / 2] = make_float2(m0, m1);
  }
}

// ---------------------------------------------------------------------------
// Link records: 18 reals of U[a][b] (row-major complex) per (owner, mu), in
// kLinkChunks 16-byte words (FP64 9, FP32 5, FP16 3).
// ---------------------------------------------------------------------------
// Third row of a reconstruct-12 link: u[0..11] hold sg * (row 0, row 1) of an
// SU(3) matrix, so sg * conj(row0 x row1) = sg * row 2 (the cross product of
// the signed rows carries sg^2 = 1).
template <class R>
__device__ __forceinline__ void reconstruct_row2(R *u, R sg) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int a = (c + 1) % 3, b = (c + 2) % 3;
    const R ar = u[2 * a], ai = u[2 * a + 1], br = u[2 * b], bi = u[2 * b + 1];          // row 0
    const R cr = u[6 + 2 * a], ci = u[6 + 2 * a + 1], dr = u[6 + 2 * b], di = u[6 + 2 * b + 1];  // row 1
    // (row0 x row1)_c = row0_a row1_b - row0_b row1_a
    const R re = (ar * dr - ai * di) - (br * cr - bi * ci);
    const R im = (ar * di + ai * dr) - (br * ci + bi * cr);
    u[12 + 2 * c] = sg * re;
    u[12 + 2 * c + 1] = -sg * im;
  }
}

// Load the link record whose word 0 is at w; word k is at w[k * ws] (the
// chunk-major link layout: ws = number of link owners). recon: the record
// holds two rows and a sign (reconstruct-12, FP32/FP16/BF16 only).
template <class S>
__device__ __forceinline__ void load_link(const uint4 *w, size_t ws, typename S::R *u,
                                          int recon = 0) {
  if constexpr (std::is_same<S, F64>::value) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double2 q = __ldg(reinterpret_cast<const double2 *>(w + k * ws));
      u[2 * k] = q.x; u[2 * k + 1] = q.y;
    }
  } else if constexpr (std::is_same<S, F32>::value) {
    if (recon) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(w + k * ws));
        u[4 * k] = q.x; u[4 * k + 1] = q.y; u[4 * k + 2] = q.z; u[4 * k + 3] = q.w;
      }
      reconstruct_row2<float>(u, __ldg(reinterpret_cast<const float *>(w + 3 * ws)));
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(w + k * ws));
        u[4 * k] = q.x; u[4 * k + 1] = q.y; u[4 * k + 2] = q.z; u[4 * k + 3] = q.w;
      }
      const float2 q = __ldg(reinterpret_cast<const float2 *>(w + 4 * ws));
      u[16] = q.x; u[17] = q.y;
    }
  } else {
    if (recon) {
      float t[16];
      unpack8<F16>(__ldg(w), t);
      unpack8<F16>(__ldg(w + ws), t + 8);
#pragma unroll
      for (int k = 0; k < 12; ++k) u[k] = t[k];
      reconstruct_row2<float>(u, t[12]);
    } else {
      float t[24];
#pragma unroll
      for (int k = 0; k < 3; ++k) unpack8<F16>(__ldg(w + k * ws), t + 8 * k);
#pragma unroll
      for (int k = 0; k < 18; ++k) u[k] = t[k];
    }
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
__device__ __forceinline__ const LsK<R> &kc(const LsCoef &c) {
  if constexpr (std::is_same<R, float>::value)
    return c.f;
  else
    return c.d;
}

// The column is first read into registers (LM >= Ls, loops unrolled over LM
// with j < Ls guards, so no register array is indexed at run time) and the
// recursions run there; shared memory is read once and written once.
template <class R, int LM>
__device__ __forceinline__ void ls_column_reg(R *T, const R *X, int Ls, bool down, bool inv,
                                              const LsK<R> &c) {
  auto ix = [&](int j) { return down ? j : Ls - 1 - j; };
  const R mf = c.mf;
  R v[LM];
#pragma unroll
  for (int j = 0; j < LM; ++j) v[j] = j < Ls ? T[ix(j)] : (R)0;
  if (inv) {
    // y_0 = (v_0 - mf sum_{j=1}^{Ls-1} r^(Ls-j) v_j) / (1 + mf r^Ls) by Horner,
    // then y_j = v_j + r y_{j-1}
    const R r = c.r;
    R h = 0;
#pragma unroll
    for (int j = 1; j < LM; ++j)
      if (j < Ls) h = h * r + v[j];
    v[0] = (v[0] - mf * r * h) * c.inv_den;
#pragma unroll
    for (int j = 1; j < LM; ++j)
      if (j < Ls) v[j] = v[j] + r * v[j - 1];
  }
  const R p0 = c.p0q, p1 = c.p1q;
  R last = 0;
#pragma unroll
  for (int j = 0; j < LM; ++j)
    if (j == Ls - 1) last = v[j];
  R out_prev = v[0];
  v[0] = p0 * v[0] - p1 * mf * last;
#pragma unroll
  for (int j = 1; j < LM; ++j)
    if (j < Ls) {
      const R t = v[j];
      v[j] = p0 * t + p1 * out_prev;
      out_prev = t;
    }
  if (X) {
    const R a0 = c.a0, a1 = c.a1;
    R xlast = X[ix(Ls - 1)], xprev = X[ix(0)];
    v[0] += a0 * xprev - a1 * mf * xlast;
#pragma unroll
    for (int j = 1; j < LM; ++j)
      if (j < Ls) {
        const R xj = X[ix(j)];
        v[j] += a0 * xj + a1 * xprev;
        xprev = xj;
      }
  }
#pragma unroll
  for (int j = 0; j < LM; ++j)
    if (j < Ls) T[ix(j)] = v[j];
}

// In-place walk over the shared-memory column.
template <class R>
__device__ __forceinline__ void ls_column_smem(R *T, const R *X, int Ls, bool down, bool inv,
                                               const LsK<R> &c) {
  auto ix = [&](int j) { return down ? j : Ls - 1 - j; };
  const R mf = c.mf;
  if (inv) {
    const R r = c.r;
    R acc = 0, rk = r;
    for (int k = 1; k < Ls; ++k) {
      acc += rk * T[ix(Ls - k)];
      rk *= r;
    }
    R y = (T[ix(0)] - mf * acc) * c.inv_den;
    T[ix(0)] = y;
    for (int j = 1; j < Ls; ++j) {
      y = T[ix(j)] + r * y;
      T[ix(j)] = y;
    }
  }
  const R p0 = c.p0q, p1 = c.p1q;
  const R last = T[ix(Ls - 1)];
  for (int j = Ls - 1; j >= 1; --j) T[ix(j)] = p0 * T[ix(j)] + p1 * T[ix(j - 1)];
  T[ix(0)] = p0 * T[ix(0)] - p1 * mf * last;
  if (X) {
    const R a0 = c.a0, a1 = c.a1;
    for (int j = 1; j < Ls; ++j) T[ix(j)] += a0 * X[ix(j)] + a1 * X[ix(j - 1)];
    T[ix(0)] += a0 * X[ix(0)] - a1 * mf * X[ix(Ls - 1)];
  }
}

// Columns of up to 16 slices run in registers, longer ones in place.
template <class R>
__device__ __forceinline__ void ls_column(R *T, const R *X, int Ls, bool down, bool inv,
                                          const LsK<R> &c) {
  if (Ls <= 16)
    ls_column_reg<R, 16>(T, X, Ls, down, inv, c);
  else
    ls_column_smem<R>(T, X, Ls, down, inv, c);
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

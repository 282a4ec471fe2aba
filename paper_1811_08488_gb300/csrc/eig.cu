// Low modes of the normal operator A and deflation of the outer solve.
//
// Paper Sec. 1: in the measurement phase many right-hand sides are solved with
// one Dirac matrix, and eigen-space methods (EigCG; Lanczos with a Chebyshev
// polynomial) compute low-lying eigenvectors once to lower the effective
// condition number of every solve. Here the low modes come from Chebyshev-
// filtered subspace iteration with a Rayleigh-Ritz step, and they enter
// Algorithm 1 as the start x_0 = V Lambda^-1 V^+ b and as an additive coarse
// correction z += V Lambda^-1 V^+ r of the multisplitting preconditioner.
//
// Kernels: a multi-dot (Gram) kernel over tiles of vector pairs, a
// linear-combination kernel, the Chebyshev three-term update, Ritz residual
// norms, and one single-CTA kernel for the small dense problem of the
// Rayleigh-Ritz step (Cholesky, two triangular solves, cyclic Jacobi
// rotations in parallel round-robin order, back substitution, sorting) in
// FP64. The vector kernels are HBM-bound; the dense kernel works on at most
// 64 x 64 matrices.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <type_traits>
#include <vector>

#include "device_common.cuh"
#include "eig.cuh"
#include "solver.cuh"
#include "vec4.cuh"

namespace dwf {

constexpr int kEigThreads = 256;
constexpr int kEigCtas = 152 * 4;  // CTAs of one vector-kernel launch over all its tiles
constexpr int kMaxTiles = (kMaxEig / 4) * (kMaxEig / 4);

constexpr int kMaxValues = 128;  // partial sums per CTA of one multi-dot launch at most

size_t dot_scratch_bytes() {
  // partials: at most max(kEigCtas, kMaxTiles) CTAs x kMaxValues values;
  // counters: one per tile
  return align_up(sizeof(double) * kMaxValues * (size_t)std::max(kEigCtas, kMaxTiles), 256) +
         align_up(sizeof(unsigned int) * kMaxTiles, 256);
}
DotScratch dot_scratch_at(char *base) {
  DotScratch w;
  w.partials = reinterpret_cast<double *>(base);
  w.counters = reinterpret_cast<unsigned int *>(
      base + align_up(sizeof(double) * kMaxValues * (size_t)std::max(kEigCtas, kMaxTiles), 256));
  return w;
}

// CTAs of one full wave of kernel K (kEigThreads threads, no dynamic shared
// memory) on the current device: the grid-stride vector kernels are launched
// with one wave, split over their tiles, so that no partial second wave
// trails them.
template <auto K>
static int wave_ctas() {
  constexpr int kDevices = 64;
  static std::atomic<int> cache[kDevices];  // per device; 0 until computed
  int dev = 0;
  DWF_CUDA_TRY(cudaGetDevice(&dev));
  std::atomic<int> *slot = dev < kDevices ? &cache[dev] : nullptr;
  if (slot) {
    const int n = slot->load(std::memory_order_relaxed);
    if (n > 0) return n;
  }
  int nsm = 0, per = 0;
  DWF_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  DWF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, K, kEigThreads, 0));
  const int n = std::max(1, per) * std::max(1, nsm);
  if (slot) slot->store(n, std::memory_order_relaxed);
  return n;
}

// CTAs per tile: one wave over all tiles (at least one CTA per tile), at most
// one CTA per `per_cta` work items of a tile, and at most kEigCtas in all
// (the partial-sum scratch holds kEigCtas CTAs).
static int ctas_per_tile(int wave, int tiles, long long items, int per_cta) {
  const long long want = (items + per_cta - 1) / per_cta;
  const int cap = std::max(1, std::min(wave, kEigCtas) / tiles);
  return (int)std::max(1LL, std::min<long long>(cap, want));
}

// Item k = c cs + e (c = 0, 1, 2) of a native field: the 8 reals [8c, 8c + 8)
// of element e, i.e. 4 complex numbers. FP32/FP64: the groups 2c and 2c + 1
// of element e; FP16: chunk c of element e (one 16-byte load) times e's scale.
template <class S, class U>
__device__ __forceinline__ void ld8(const char *p, long long soff, long long k, long long cs,
                                    U v[8]) {
  const long long c = k / cs, e = k - c * cs;
  if constexpr (std::is_same<S, F16>::value) {
    float f[8];
    unpack8<F16>(__ldg(reinterpret_cast<const uint4 *>(p) + k), f);
    const float scl = __ldg(reinterpret_cast<const float *>(p + soff) + e);
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = (U)(f[q] * scl);
  } else {
    ld4<S>(p, 2 * c * cs + e, cs, v);
    ld4<S>(p, (2 * c + 1) * cs + e, cs, v + 4);
  }
}
template <class S, class U>
__device__ __forceinline__ void st8(char *p, long long k, long long cs, const U v[8]) {
  const long long c = k / cs, e = k - c * cs;
  st4<S>(p, 2 * c * cs + e, cs, v);
  st4<S>(p, (2 * c + 1) * cs + e, cs, v + 4);
}

// ---------------------------------------------------------------------------
// Multi-dot: G[i][j] = <X_i, Y_j> over tiles of TI x TJ vector pairs.
// ---------------------------------------------------------------------------
struct GramArgs {
  const char *x = nullptr;
  long long xvs = 0;
  long long xsoff = 0;  // FP16 X: byte offset of the scales within a vector
  int nx = 0;
  const char *y = nullptr;
  long long yvs = 0;
  int ny = 0;
  long long n4 = 0, cs = 0;
  double2 *G = nullptr;
  int ldg = 0;
  double *partials = nullptr;
  unsigned int *counters = nullptr;
};

// One CTA accumulates the 2 TI TJ real sums (re, im of each pair) over its
// share of the elements; the last CTA of the tile to finish adds the partials
// of all CTAs in CTA order and writes the tile of G.
template <int TI, int TJ, class SY>
__global__ void __launch_bounds__(kEigThreads) gram_kernel(const GramArgs a) {
  constexpr int NV = 2 * TI * TJ;
  __shared__ double sh[kEigThreads / 32][NV];
  __shared__ int s_last;
  const int ntj = (a.ny + TJ - 1) / TJ;
  const int tile = blockIdx.y, ti = tile / ntj, tj = tile - ti * ntj;
  const int i0 = ti * TI, j0 = tj * TJ;
  KahanF acc[NV];
  FLAT_LOOP(a.n4) {
    float y[TJ][4];
#pragma unroll
    for (int j = 0; j < TJ; ++j) {
      if (j0 + j < a.ny)
        ld4<SY>(a.y + (j0 + j) * a.yvs, i, a.cs, y[j]);
      else
        y[j][0] = y[j][1] = y[j][2] = y[j][3] = 0.f;
    }
#pragma unroll
    for (int t = 0; t < TI; ++t) {
      if (i0 + t < a.nx) {
        float x[4];
        ld4<F32>(a.x + (i0 + t) * a.xvs, i, a.cs, x);
#pragma unroll
        for (int j = 0; j < TJ; ++j) {
          // conj(x) y on the two complex numbers of the group
          acc[2 * (t * TJ + j)].add(x[0] * y[j][0] + x[1] * y[j][1] + x[2] * y[j][2] +
                                    x[3] * y[j][3]);
          acc[2 * (t * TJ + j) + 1].add(x[0] * y[j][1] - x[1] * y[j][0] + x[2] * y[j][3] -
                                        x[3] * y[j][2]);
        }
      }
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double d = acc[v].value();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
    if (lane == 0) sh[w][v] = d;
  }
  __syncthreads();
  double *part = a.partials + (size_t)tile * gridDim.x * NV;
  if (threadIdx.x < NV) {
    double t = 0.0;
    for (int k = 0; k < kEigThreads / 32; ++k) t += sh[k][threadIdx.x];
    part[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = t;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int prev = atomicAdd(a.counters + tile, 1u);
    s_last = prev == gridDim.x - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < NV) {
    const volatile double *vp = part + (size_t)threadIdx.x * gridDim.x;
    double t = 0.0;
    for (unsigned int k = 0; k < gridDim.x; ++k) t += vp[k];
    const int v = threadIdx.x >> 1, gi = i0 + v / TJ, gj = j0 + v % TJ;
    if (gi < a.nx && gj < a.ny)
      reinterpret_cast<double *>(a.G + (size_t)gi * a.ldg + gj)[threadIdx.x & 1] = t;
  }
  if (threadIdx.x == 0) a.counters[tile] = 0u;
}

// Few Y vectors (ny <= NJ <= 4) against many X (FP32, or FP16 with scales):
// the 8 warps of a CTA walk the same stretch of 32 elements (groups of 4 reals
// or 16-byte chunks of 8 reals), warp w taking X vectors
// ibase + w + 8 t (t < NI) and every Y vector, so each X vector is read once
// per launch and the Y vectors once per tile of 8 NI X vectors (the other
// warps' Y loads hit L1).
template <int NI, int NJ, class SX, class SY>
__global__ void __launch_bounds__(kEigThreads) gram_skinny_kernel(const GramArgs a) {
  constexpr int NV = 8 * NI * NJ * 2;
  static_assert(NV <= kMaxValues, "too many partial sums per CTA");
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int tile = blockIdx.y, ibase = tile * 8 * NI;
  KahanF acc[NI][NJ][2];
  if constexpr (std::is_same<SX, F32>::value && NJ > 1) {
    // FP32 X against several Y: groups of 4 reals, all Y of the group loaded
    // up front (two groups' loads in flight per thread); measured faster than
    // the chunk loop below for 4 Y, slower for one
#pragma unroll 2
    for (long long i = blockIdx.x * 32LL + lane; i < a.n4; i += gridDim.x * 32LL) {
      float y[NJ][4];
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        if (j < a.ny)
          ld4<SY>(a.y + j * a.yvs, i, a.cs, y[j]);
        else
          y[j][0] = y[j][1] = y[j][2] = y[j][3] = 0.f;
      }
#pragma unroll
      for (int t = 0; t < NI; ++t) {
        const int xi = ibase + w + 8 * t;
        if (xi < a.nx) {
          float x[4];
          ld4<F32>(a.x + xi * a.xvs, i, a.cs, x);
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            acc[t][j][0].add(x[0] * y[j][0] + x[1] * y[j][1] + x[2] * y[j][2] + x[3] * y[j][3]);
            acc[t][j][1].add(x[0] * y[j][1] - x[1] * y[j][0] + x[2] * y[j][3] - x[3] * y[j][2]);
          }
        }
      }
    }
  } else {
    // FP16 X, or FP32 X against one Y: 16-byte chunks of 8 reals (FP32: two
    // groups; FP16: one chunk and its scale)
    const long long n8 = 3 * a.cs;
    for (long long k = blockIdx.x * 32LL + lane; k < n8; k += gridDim.x * 32LL) {
      // this warp's X items first, then one Y item at a time (few registers:
      // the Y loads of the 8 warps hit L1 after the first)
      float x[NI][8];
#pragma unroll
      for (int t = 0; t < NI; ++t) {
        const int xi = ibase + w + 8 * t;
        if (xi < a.nx) {
          ld8<SX>(a.x + xi * a.xvs, a.xsoff, k, a.cs, x[t]);
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q) x[t][q] = 0.f;
        }
      }
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        if (j < a.ny) {
          float y[8];
          ld8<SY>(a.y + j * a.yvs, 0, k, a.cs, y);
#pragma unroll
          for (int t = 0; t < NI; ++t) {
            // conj(x) y on the item's four complex numbers
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int q = 0; q < 8; q += 2) {
              re += x[t][q] * y[q] + x[t][q + 1] * y[q + 1];
              im += x[t][q] * y[q + 1] - x[t][q + 1] * y[q];
            }
            acc[t][j][0].add(re);
            acc[t][j][1].add(im);
          }
        }
      }
    }
  }
  // value v = ((w NI + t) NJ + j) 2 + c: warp sums, written by lane 0 of warp w
  double *part = a.partials + (size_t)tile * gridDim.x * NV;
#pragma unroll
  for (int t = 0; t < NI; ++t)
#pragma unroll
    for (int j = 0; j < NJ; ++j)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        double d = acc[t][j][c].value();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
        if (lane == 0)
          part[(size_t)(((w * NI + t) * NJ + j) * 2 + c) * gridDim.x + blockIdx.x] = d;
      }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int prev = atomicAdd(a.counters + tile, 1u);
    s_last = prev == gridDim.x - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < NV) {
    const int v = threadIdx.x, c = v & 1, j = (v >> 1) % NJ, wt = (v >> 1) / NJ;
    const int t = wt % NI, ww = wt / NI;
    const volatile double *vp = part + (size_t)v * gridDim.x;
    double sum = 0.0;
    for (unsigned int k = 0; k < gridDim.x; ++k) sum += vp[k];
    const int gi = ibase + ww + 8 * t;
    if (gi < a.nx && j < a.ny)
      reinterpret_cast<double *>(a.G + (size_t)gi * a.ldg + j)[c] = sum;
  }
  if (threadIdx.x == 0) a.counters[tile] = 0u;
}

template <int NI, int NJ, class SX, class SY>
static void gram_skinny_go(const GramArgs &a, cudaStream_t st) {
  const int tiles = (a.nx + 8 * NI - 1) / (8 * NI);
  dim3 grid(ctas_per_tile(wave_ctas<gram_skinny_kernel<NI, NJ, SX, SY>>(), tiles, 3 * a.cs, 32),
            tiles);
  gram_skinny_kernel<NI, NJ, SX, SY><<<grid, kEigThreads, 0, st>>>(a);
  DWF_CUDA_TRY(cudaGetLastError());
}
template <int NI, int NJ>
static void gram_skinny_launch(const GramArgs &a, dwf_prec xprec, dwf_prec yprec,
                               cudaStream_t st) {
  if (xprec == DWF_FP16)
    yprec == DWF_FP64 ? gram_skinny_go<NI, NJ, F16, F64>(a, st)
                      : gram_skinny_go<NI, NJ, F16, F32>(a, st);
  else
    yprec == DWF_FP64 ? gram_skinny_go<NI, NJ, F32, F64>(a, st)
                      : gram_skinny_go<NI, NJ, F32, F32>(a, st);
}

template <int TI, int TJ>
static void gram_launch(const GramArgs &a, dwf_prec yprec, cudaStream_t st) {
  const int tiles = ((a.nx + TI - 1) / TI) * ((a.ny + TJ - 1) / TJ);
  if (yprec == DWF_FP64) {
    dim3 grid(ctas_per_tile(wave_ctas<gram_kernel<TI, TJ, F64>>(), tiles, a.n4, kEigThreads),
              tiles);
    gram_kernel<TI, TJ, F64><<<grid, kEigThreads, 0, st>>>(a);
  } else {
    dim3 grid(ctas_per_tile(wave_ctas<gram_kernel<TI, TJ, F32>>(), tiles, a.n4, kEigThreads),
              tiles);
    gram_kernel<TI, TJ, F32><<<grid, kEigThreads, 0, st>>>(a);
  }
  DWF_CUDA_TRY(cudaGetLastError());
}

void gram(const VecSet &X, const VecSet &Y, long long cs, double2 *G, int ldg,
          const DotScratch &w, cudaStream_t st) {
  DWF_REQUIRE((X.prec == DWF_FP32 || (X.prec == DWF_FP16 && Y.n <= 4)) &&
                  (Y.prec == DWF_FP32 || Y.prec == DWF_FP64),
              DWF_ERR_INVALID_ARG,
              "gram: X must be FP32 (or FP16 against at most 4 Y), Y FP32 or FP64");
  DWF_REQUIRE(X.n >= 1 && X.n <= kMaxEig && Y.n >= 1 && Y.n <= kMaxEig, DWF_ERR_INVALID_ARG,
              "gram: 1 .. 64 vectors per side");
  GramArgs a;
  a.x = X.p;
  a.xvs = X.vs;
  a.xsoff = X.soff;
  a.nx = X.n;
  a.y = Y.p;
  a.yvs = Y.vs;
  a.ny = Y.n;
  a.n4 = 6 * cs;
  a.cs = cs;
  a.G = G;
  a.ldg = ldg;
  a.partials = w.partials;
  a.counters = w.counters;
  if (Y.n == 1)
    gram_skinny_launch<2, 1>(a, X.prec, Y.prec, st);
  else if (Y.n == 2)
    gram_skinny_launch<2, 2>(a, X.prec, Y.prec, st);
  else if (Y.n <= 4)
    gram_skinny_launch<2, 4>(a, X.prec, Y.prec, st);
  else
    gram_launch<4, 4>(a, Y.prec, st);
}

// ---------------------------------------------------------------------------
// Linear combination: out_j = base_j + sum_i X_i C_ij w_i.
// ---------------------------------------------------------------------------
struct CombineArgs {
  const char *x = nullptr;
  long long xvs = 0;
  long long xsoff = 0;  // FP16 X: byte offset of the scales within a vector
  int nx = 0;
  const double2 *C = nullptr;
  int ldc = 0;
  const double *wi = nullptr;
  const char *base = nullptr;
  char *out = nullptr;
  long long ovs = 0;
  int nout = 0;
  const int *skip = nullptr;
  long long n4 = 0, cs = 0;
};

// One item (8 reals) of every output per thread and grid-stride step; X is
// FP32 or FP16 with scales, the outputs FP32 or FP64.
template <int TJ, class SX, class SO>
__global__ void __launch_bounds__(kEigThreads) combine_kernel(const CombineArgs a) {
  using R = typename std::conditional<std::is_same<SO, F64>::value, double, float>::type;
  __shared__ R cr[kMaxEig][TJ], ci[kMaxEig][TJ];
  const int j0 = blockIdx.y * TJ;
  for (int k = threadIdx.x; k < a.nx * TJ; k += blockDim.x) {
    const int i = k / TJ, j = k - i * TJ;
    double2 v = make_double2(0.0, 0.0);
    if (j0 + j < a.nout) {
      v = a.C[(size_t)i * a.ldc + j0 + j];
      if (a.wi) {
        v.x *= a.wi[i];
        v.y *= a.wi[i];
      }
    }
    cr[i][j] = (R)v.x;
    ci[i][j] = (R)v.y;
  }
  __syncthreads();
  bool live[TJ];
#pragma unroll
  for (int j = 0; j < TJ; ++j)
    live[j] = j0 + j < a.nout && !(a.skip && a.skip[j0 + j]);
  const long long n8 = 3 * a.cs;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n8;
       k += (long long)gridDim.x * blockDim.x) {
    R acc[TJ][8];
#pragma unroll
    for (int j = 0; j < TJ; ++j) {
      if (a.base && live[j]) {
        ld8<SO>(a.base + (j0 + j) * a.ovs, 0, k, a.cs, acc[j]);
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[j][q] = (R)0;
      }
    }
    for (int t = 0; t < a.nx; ++t) {
      float x[8];
      ld8<SX>(a.x + t * a.xvs, a.xsoff, k, a.cs, x);
#pragma unroll
      for (int j = 0; j < TJ; ++j) {
        const R r = cr[t][j], m = ci[t][j];
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
          acc[j][q] += (R)x[q] * r - (R)x[q + 1] * m;
          acc[j][q + 1] += (R)x[q] * m + (R)x[q + 1] * r;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < TJ; ++j)
      if (live[j]) st8<SO>(a.out + (j0 + j) * a.ovs, k, a.cs, acc[j]);
  }
}

template <int TJ, class SX, class SO>
static void combine_go(const CombineArgs &a, cudaStream_t st) {
  const int tiles = (a.nout + TJ - 1) / TJ;
  dim3 grid(ctas_per_tile(wave_ctas<combine_kernel<TJ, SX, SO>>(), tiles, 3 * a.cs, kEigThreads),
            tiles);
  combine_kernel<TJ, SX, SO><<<grid, kEigThreads, 0, st>>>(a);
  DWF_CUDA_TRY(cudaGetLastError());
}
// FP64 outputs take at most 4 per tile (8 doubles of accumulators each).
template <int TJ>
static void combine_launch(const CombineArgs &a, dwf_prec xprec, dwf_prec oprec,
                           cudaStream_t st) {
  if (oprec == DWF_FP64) {
    constexpr int T = TJ > 4 ? 4 : TJ;
    xprec == DWF_FP16 ? combine_go<T, F16, F64>(a, st) : combine_go<T, F32, F64>(a, st);
  } else {
    xprec == DWF_FP16 ? combine_go<TJ, F16, F32>(a, st) : combine_go<TJ, F32, F32>(a, st);
  }
}

void combine(const VecSet &X, const double2 *C, int ldc, const double *wi, const char *base,
             char *out, long long ovs, dwf_prec oprec, int nout, const int *skip, long long cs,
             cudaStream_t st) {
  DWF_REQUIRE((X.prec == DWF_FP32 || X.prec == DWF_FP16) &&
                  (oprec == DWF_FP32 || oprec == DWF_FP64),
              DWF_ERR_INVALID_ARG, "combine: X must be FP32 or FP16, the output FP32 or FP64");
  DWF_REQUIRE(X.n >= 1 && X.n <= kMaxEig && nout >= 1 && nout <= kMaxEig, DWF_ERR_INVALID_ARG,
              "combine: 1 .. 64 vectors per side");
  CombineArgs a;
  a.x = X.p;
  a.xvs = X.vs;
  a.xsoff = X.soff;
  a.nx = X.n;
  a.C = C;
  a.ldc = ldc;
  a.wi = wi;
  a.base = base;
  a.out = out;
  a.ovs = ovs;
  a.nout = nout;
  a.skip = skip;
  a.n4 = 6 * cs;
  a.cs = cs;
  if (nout == 1)
    combine_launch<1>(a, X.prec, oprec, st);
  else if (nout == 2)
    combine_launch<2>(a, X.prec, oprec, st);
  else if (nout <= 4)
    combine_launch<4>(a, X.prec, oprec, st);
  else
    combine_launch<8>(a, X.prec, oprec, st);
}

// ---------------------------------------------------------------------------
// Chebyshev step and Ritz residuals (FP32 fields)
// ---------------------------------------------------------------------------
// out = s1 (A y - c y) - s2 y_prev on nvec vectors (y_prev may be null; out
// may be A y or y_prev).
struct ChebArgs {
  const char *ay = nullptr, *y = nullptr, *yprev = nullptr;
  char *out = nullptr;
  long long vs = 0, n4 = 0;
  float s1 = 0.f, c = 0.f, s2 = 0.f;
};

__global__ void __launch_bounds__(kEigThreads) cheb_kernel(const ChebArgs a) {
  const long long o = blockIdx.y * a.vs;
  const float4 *ay = reinterpret_cast<const float4 *>(a.ay + o);
  const float4 *y = reinterpret_cast<const float4 *>(a.y + o);
  const float4 *yp = a.yprev ? reinterpret_cast<const float4 *>(a.yprev + o) : nullptr;
  float4 *out = reinterpret_cast<float4 *>(a.out + o);
  FLAT_LOOP(a.n4) {
    const float4 q = ay[i], v = y[i];
    float4 r = make_float4(a.s1 * (q.x - a.c * v.x), a.s1 * (q.y - a.c * v.y),
                           a.s1 * (q.z - a.c * v.z), a.s1 * (q.w - a.c * v.w));
    if (yp) {
      const float4 p = yp[i];
      r.x -= a.s2 * p.x;
      r.y -= a.s2 * p.y;
      r.z -= a.s2 * p.z;
      r.w -= a.s2 * p.w;
    }
    out[i] = r;
  }
}

static void cheb_step(const char *ay, const char *y, const char *yprev, char *out, long long vs,
                      int nvec, long long n4, double s1, double c, double s2, cudaStream_t st) {
  ChebArgs a;
  a.ay = ay;
  a.y = y;
  a.yprev = yprev;
  a.out = out;
  a.vs = vs;
  a.n4 = n4;
  a.s1 = (float)s1;
  a.c = (float)c;
  a.s2 = (float)s2;
  const int ctas = ctas_per_tile(wave_ctas<cheb_kernel>(), nvec, n4, kEigThreads);
  cheb_kernel<<<dim3(ctas, nvec), kEigThreads, 0, st>>>(a);
  DWF_CUDA_TRY(cudaGetLastError());
}

// out[j] = |AV_j - theta_j V_j| (FP32 fields, FP64 sums).
struct ResidArgs {
  const char *av = nullptr, *v = nullptr;
  long long vs = 0, n4 = 0, cs = 0;
  const double *theta = nullptr;
  double *out = nullptr;
  double *partials = nullptr;
  unsigned int *counters = nullptr;
};

__global__ void __launch_bounds__(kEigThreads) resid_kernel(const ResidArgs a) {
  __shared__ double red[32];
  const int j = blockIdx.y;
  const float th = (float)a.theta[j];
  KahanF acc;
  FLAT_LOOP(a.n4) {
    float p[4], q[4];
    ld4<F32>(a.av + j * a.vs, i, a.cs, p);
    ld4<F32>(a.v + j * a.vs, i, a.cs, q);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float d = p[k] - th * q[k];
      s += d * d;
    }
    acc.add(s);
  }
  const double t = cta_sum(acc.value(), red);
  double tot;
  if (group_reduce(t, a.partials + (size_t)j * gridDim.x, gridDim.x, blockIdx.x, a.counters + j,
                   tot))
    a.out[j] = sqrt(tot);
}

// ---------------------------------------------------------------------------
// The small dense problem of the Rayleigh-Ritz step, one CTA, FP64:
// G = W^+ W = L L^+ (Cholesky), H' = L^-1 (W^+ A W) L^-+, H' = Q diag(theta) Q^+
// (cyclic Jacobi), S = L^-+ Q, columns sorted by ascending theta. Then W S
// holds orthonormal Ritz vectors with Ritz values theta. Row-major m x m.
// ---------------------------------------------------------------------------
struct DenseArgs {
  int m = 0;
  const double2 *G = nullptr, *H = nullptr;
  double2 *L = nullptr, *X = nullptr, *Q = nullptr, *T = nullptr;  // m x m scratch each
  double *theta = nullptr;  // [m]
  double2 *S = nullptr;     // m x m
  int *status = nullptr;    // 0 ok, 1 G not positive definite
  int max_sweeps = 0;
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

__global__ void __launch_bounds__(kEigThreads) dense_rr_kernel(const DenseArgs a) {
  const int m = a.m, tid = threadIdx.x, nt = blockDim.x;
  __shared__ double s_red[kEigThreads / 32][2];
  __shared__ double rc[kMaxEig / 2], rs[kMaxEig / 2];
  __shared__ double2 rph[kMaxEig / 2];  // e^{-i phi}
  __shared__ int rp[kMaxEig / 2], rq[kMaxEig / 2];
  __shared__ int s_stop, s_bad;
  __shared__ int rank[kMaxEig];
  double2 *L = a.L, *X = a.X, *Q = a.Q, *T = a.T;
  if (tid == 0) s_bad = 0;
  // Cholesky G = L L^+ (left-looking, lower triangle)
  for (int k = tid; k < m * m; k += nt) {
    const int i = k / m, j = k - i * m;
    L[k] = j <= i ? a.G[k] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  double gmax = 0.0;
  for (int i = 0; i < m; ++i) gmax = fmax(gmax, a.G[i * m + i].x);
  for (int k = 0; k < m; ++k) {
    if (tid == 0) {
      double d = L[k * m + k].x;
      for (int j = 0; j < k; ++j) d -= L[k * m + j].x * L[k * m + j].x + L[k * m + j].y * L[k * m + j].y;
      if (!(d > 1e-15 * gmax)) {
        s_bad = 1;
        d = 1e-15 * gmax + 1e-300;
      }
      L[k * m + k] = make_double2(sqrt(d), 0.0);
    }
    __syncthreads();
    const double lkk = L[k * m + k].x;
    for (int i = k + 1 + tid; i < m; i += nt) {
      double2 s = L[i * m + k];
      for (int j = 0; j < k; ++j) {
        const double2 p = cmul(L[i * m + j], cconj(L[k * m + j]));
        s.x -= p.x;
        s.y -= p.y;
      }
      L[i * m + k] = make_double2(s.x / lkk, s.y / lkk);
    }
    __syncthreads();
  }
  // X = L^-1 H (forward substitution, one column per thread)
  for (int j = tid; j < m; j += nt) {
    for (int i = 0; i < m; ++i) {
      double2 s = a.H[i * m + j];
      for (int k = 0; k < i; ++k) {
        const double2 p = cmul(L[i * m + k], X[k * m + j]);
        s.x -= p.x;
        s.y -= p.y;
      }
      X[i * m + j] = make_double2(s.x / L[i * m + i].x, s.y / L[i * m + i].x);
    }
  }
  __syncthreads();
  // T = X^+; X = L^-1 T = L^-1 H L^-+
  for (int k = tid; k < m * m; k += nt) {
    const int i = k / m, j = k - i * m;
    T[k] = cconj(X[j * m + i]);
  }
  __syncthreads();
  for (int j = tid; j < m; j += nt) {
    for (int i = 0; i < m; ++i) {
      double2 s = T[i * m + j];
      for (int k = 0; k < i; ++k) {
        const double2 p = cmul(L[i * m + k], X[k * m + j]);
        s.x -= p.x;
        s.y -= p.y;
      }
      X[i * m + j] = make_double2(s.x / L[i * m + i].x, s.y / L[i * m + i].x);
    }
  }
  __syncthreads();
  // Hermitian part; Q = 1
  for (int k = tid; k < m * m; k += nt) {
    const int i = k / m, j = k - i * m;
    Q[k] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    if (i < j) {
      const double2 u = X[i * m + j], v = X[j * m + i];
      const double2 h = make_double2(0.5 * (u.x + v.x), 0.5 * (u.y - v.y));
      X[i * m + j] = h;
      X[j * m + i] = cconj(h);
    } else if (i == j) {
      X[k].y = 0.0;
    }
  }
  __syncthreads();
  // Cyclic Jacobi, pairs in round-robin order (n = m rounded up to even;
  // index m is a dummy when m is odd): in round r, position 0 holds index 0
  // and position p > 0 holds 1 + (p - 1 + r) mod (n - 1); positions k and
  // n - 1 - k form a pair.
  const int n = m + (m & 1), npair = n / 2;
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    // converged when the off-diagonal |X|^2 is below 1e-26 of the diagonal's
    // (off-diagonal entries about 1e-13 of the largest eigenvalue)
    double off = 0.0, dia = 0.0;
    for (int k = tid; k < m * m; k += nt) {
      const int i = k / m, j = k - i * m;
      const double v = X[k].x * X[k].x + X[k].y * X[k].y;
      if (i == j)
        dia += v;
      else
        off += v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_down_sync(0xffffffffu, off, o);
      dia += __shfl_down_sync(0xffffffffu, dia, o);
    }
    if ((tid & 31) == 0) {
      s_red[tid >> 5][0] = off;
      s_red[tid >> 5][1] = dia;
    }
    __syncthreads();
    if (tid == 0) {
      double o2 = 0.0, d2 = 0.0;
      for (int w = 0; w < (nt + 31) / 32; ++w) {
        o2 += s_red[w][0];
        d2 += s_red[w][1];
      }
      s_stop = o2 <= 1e-26 * d2;
    }
    __syncthreads();
    if (s_stop) break;
    for (int r = 0; r < n - 1; ++r) {
      for (int k = tid; k < npair; k += nt) {
        const int pa = k, pb = n - 1 - k;
        int p = pa == 0 ? 0 : 1 + (pa - 1 + r) % (n - 1);
        int q = 1 + (pb - 1 + r) % (n - 1);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        rp[k] = p;
        rq[k] = q;
        double c = 1.0, s = 0.0;
        double2 ph = make_double2(1.0, 0.0);
        if (q < m) {
          const double2 z = X[p * m + q];
          const double az = sqrt(z.x * z.x + z.y * z.y);
          const double app = X[p * m + p].x, aqq = X[q * m + q].x;
          if (az > 1e-300 && az > 1e-18 * (fabs(app) + fabs(aqq))) {
            ph = make_double2(z.x / az, -z.y / az);
            const double th = (aqq - app) / (2.0 * az);
            const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        rc[k] = c;
        rs[k] = s;
        rph[k] = ph;
      }
      __syncthreads();
      // columns: X <- X J and Q <- Q J, J_pp = c, J_pq = s, J_qp = -s e^{-i phi},
      // J_qq = c e^{-i phi}
      for (int idx = tid; idx < m * npair; idx += nt) {
        const int i = idx / npair, k = idx - i * npair;
        const int p = rp[k], q = rq[k];
        if (q >= m || rs[k] == 0.0) continue;
        const double c = rc[k], s = rs[k];
        const double2 ph = rph[k];
#pragma unroll
        for (int mat = 0; mat < 2; ++mat) {
          double2 *M = mat ? Q : X;
          const double2 xp = M[i * m + p], xq = cmul(M[i * m + q], ph);
          M[i * m + p] = make_double2(c * xp.x - s * xq.x, c * xp.y - s * xq.y);
          M[i * m + q] = make_double2(s * xp.x + c * xq.x, s * xp.y + c * xq.y);
        }
      }
      __syncthreads();
      // rows: X <- J^+ X
      for (int idx = tid; idx < m * npair; idx += nt) {
        const int j = idx / npair, k = idx - j * npair;
        const int p = rp[k], q = rq[k];
        if (q >= m || rs[k] == 0.0) continue;
        const double c = rc[k], s = rs[k];
        const double2 phc = cconj(rph[k]);
        const double2 xp = X[p * m + j], xq = cmul(X[q * m + j], phc);
        X[p * m + j] = make_double2(c * xp.x - s * xq.x, c * xp.y - s * xq.y);
        X[q * m + j] = make_double2(s * xp.x + c * xq.x, s * xp.y + c * xq.y);
      }
      __syncthreads();
    }
  }
  // S = L^-+ Q (back substitution, one column per thread) into T
  for (int j = tid; j < m; j += nt) {
    for (int i = m - 1; i >= 0; --i) {
      double2 s = Q[i * m + j];
      for (int k = i + 1; k < m; ++k) {
        const double2 p = cmulc(L[k * m + i], T[k * m + j]);
        s.x -= p.x;
        s.y -= p.y;
      }
      T[i * m + j] = make_double2(s.x / L[i * m + i].x, s.y / L[i * m + i].x);
    }
  }
  // ascending order: rank of each Ritz value (ties by index)
  for (int i = tid; i < m; i += nt) {
    const double ti = X[i * m + i].x;
    int r = 0;
    for (int j = 0; j < m; ++j) {
      const double tj = X[j * m + j].x;
      r += (tj < ti) || (tj == ti && j < i);
    }
    rank[i] = r;
  }
  __syncthreads();
  for (int i = tid; i < m; i += nt) a.theta[rank[i]] = X[i * m + i].x;
  for (int k = tid; k < m * m; k += nt) {
    const int i = k / m, j = k - i * m;
    a.S[i * m + rank[j]] = T[k];
  }
  if (tid == 0) *a.status = s_bad;
}

// Power iteration: c = 1 / |y| from G = <y, y> (device scalars).
__global__ void inv_norm_kernel(const double2 *g, double2 *c) {
  if (threadIdx.x == 0) *c = make_double2(g->x > 0.0 ? 1.0 / sqrt(g->x) : 0.0, 0.0);
}

// ---------------------------------------------------------------------------
// The subspace iteration (host driver)
// ---------------------------------------------------------------------------
namespace {
struct EigSmall {  // layout of the small device buffer
  double2 *G, *H, *L, *X, *Q, *T, *S, *pw;
  double *theta, *resid;
  int *status;
  DotScratch dw;
  double *rpart;
  unsigned int *rcount;
};
}  // namespace

void eig_lowmodes(dwf_ctx *ctx, char *V, int m, double mf, const dwf_eig_params &p,
                  double *theta_h, double *resid_h, dwf_eig_info *info, cudaStream_t st) {
  const auto t0 = std::chrono::steady_clock::now();
  const int Vh = ctx->geo.Vh, Ls = ctx->act.Ls;
  const long long cs = (long long)Vh * Ls, n4 = 6 * cs;
  const long long vs = (long long)field_rhs_bytes(DWF_FP32, Vh, Ls);
  const int batch = kMaxRhs;
  ctx->eig_w.ensure((size_t)vs * m);
  ctx->eig_aw.ensure((size_t)vs * m);
  ctx->eig_t.ensure((size_t)vs * 3 * batch);
  char *W = ctx->eig_w.c(), *AW = ctx->eig_aw.c();
  char *Tb[3] = {ctx->eig_t.c(), ctx->eig_t.c() + vs * batch, ctx->eig_t.c() + 2 * vs * batch};
  // small buffer: 8 m x m complex matrices (the last holds power-iteration
  // scalars), theta, resid, status, dot and residual scratch
  const size_t mm = (size_t)kMaxEig * kMaxEig * sizeof(double2);
  const size_t rpart_bytes = align_up(sizeof(double) * (size_t)kMaxEig * kEigCtas, 256);
  ctx->eig_small.ensure(8 * mm + 3 * 256 * 4 + dot_scratch_bytes() + rpart_bytes +
                        align_up(sizeof(unsigned int) * kMaxEig, 256));
  char *sb = ctx->eig_small.c();
  EigSmall E;
  E.G = reinterpret_cast<double2 *>(sb);
  E.H = reinterpret_cast<double2 *>(sb + mm);
  E.L = reinterpret_cast<double2 *>(sb + 2 * mm);
  E.X = reinterpret_cast<double2 *>(sb + 3 * mm);
  E.Q = reinterpret_cast<double2 *>(sb + 4 * mm);
  E.T = reinterpret_cast<double2 *>(sb + 5 * mm);
  E.S = reinterpret_cast<double2 *>(sb + 6 * mm);
  E.pw = reinterpret_cast<double2 *>(sb + 7 * mm);
  char *tail = sb + 8 * mm;
  E.theta = reinterpret_cast<double *>(tail);
  E.resid = reinterpret_cast<double *>(tail + 256 * 4);
  E.status = reinterpret_cast<int *>(tail + 2 * 256 * 4);
  E.dw = dot_scratch_at(tail + 3 * 256 * 4);
  E.rpart = reinterpret_cast<double *>(tail + 3 * 256 * 4 + dot_scratch_bytes());
  E.rcount = reinterpret_cast<unsigned int *>(tail + 3 * 256 * 4 + dot_scratch_bytes() +
                                              rpart_bytes);
  DWF_CUDA_TRY(cudaMemsetAsync(E.dw.counters, 0, sizeof(unsigned int) * kMaxTiles, st));
  DWF_CUDA_TRY(cudaMemsetAsync(E.rcount, 0, sizeof(unsigned int) * kMaxEig, st));

  long long matvecs = 0;
  const double mfs[kMaxRhs] = {mf, mf, mf, mf, mf, mf, mf, mf, mf, mf, mf, mf, mf, mf, mf, mf};
  auto matvec = [&](char *out, const char *in, int nvec) {
    for (int b0 = 0; b0 < nvec; b0 += batch) {
      const int nb = std::min(batch, nvec - b0);
      apply_mdagm(ctx, out + b0 * vs, in + b0 * vs, DWF_FP32, nb, mfs,
                  op_work(ctx, DWF_FP32, nb), nullptr, nullptr, st, p.schur);
    }
    matvecs += nvec;
  };
  auto set = [&](const char *ptr, int nvec) {
    VecSet s;
    s.p = ptr;
    s.vs = vs;
    s.n = nvec;
    s.prec = DWF_FP32;
    return s;
  };

  // upper bound of the spectrum
  double lam_max = p.lambda_max;
  if (!(lam_max > 0.0)) {
    char *y = Tb[0], *ay = Tb[1];
    DWF_CUDA_TRY(cudaMemcpyAsync(y, V, vs, cudaMemcpyDeviceToDevice, st));
    gram(set(y, 1), set(y, 1), cs, E.pw, 1, E.dw, st);
    inv_norm_kernel<<<1, 32, 0, st>>>(E.pw, E.pw + 1);
    combine(set(y, 1), E.pw + 1, 1, nullptr, nullptr, y, vs, DWF_FP32, 1, nullptr, cs, st);
    for (int k = 0; k < p.power_steps; ++k) {
      matvec(ay, y, 1);
      gram(set(y, 1), set(ay, 1), cs, E.pw + 2, 1, E.dw, st);  // <y, A y>, |y| = 1
      gram(set(ay, 1), set(ay, 1), cs, E.pw, 1, E.dw, st);
      inv_norm_kernel<<<1, 32, 0, st>>>(E.pw, E.pw + 1);
      combine(set(ay, 1), E.pw + 1, 1, nullptr, nullptr, y, vs, DWF_FP32, 1, nullptr, cs, st);
    }
    double2 q;
    DWF_CUDA_TRY(cudaMemcpyAsync(&q, E.pw + 2, sizeof(q), cudaMemcpyDeviceToHost, st));
    DWF_CUDA_TRY(cudaStreamSynchronize(st));
    DWF_REQUIRE(std::isfinite(q.x) && q.x > 0.0, DWF_ERR_NAN,
                "eig: power iteration gave no positive Rayleigh quotient");
    lam_max = 1.1 * q.x;
  }

  std::vector<double> theta(m), resid(m);
  // Rayleigh-Ritz on span(W): V = W S, W <- A V, residual norms
  auto rayleigh_ritz = [&]() {
    matvec(AW, W, m);
    gram(set(W, m), set(W, m), cs, E.G, m, E.dw, st);
    gram(set(W, m), set(AW, m), cs, E.H, m, E.dw, st);
    DenseArgs d;
    d.m = m;
    d.G = E.G;
    d.H = E.H;
    d.L = E.L;
    d.X = E.X;
    d.Q = E.Q;
    d.T = E.T;
    d.theta = E.theta;
    d.S = E.S;
    d.status = E.status;
    d.max_sweeps = 40;
    dense_rr_kernel<<<1, kEigThreads, 0, st>>>(d);
    DWF_CUDA_TRY(cudaGetLastError());
    combine(set(W, m), E.S, m, nullptr, nullptr, V, vs, DWF_FP32, m, nullptr, cs, st);
    combine(set(AW, m), E.S, m, nullptr, nullptr, W, vs, DWF_FP32, m, nullptr, cs, st);
    ResidArgs ra;
    ra.av = W;
    ra.v = V;
    ra.vs = vs;
    ra.n4 = n4;
    ra.cs = cs;
    ra.theta = E.theta;
    ra.out = E.resid;
    ra.partials = E.rpart;
    ra.counters = E.rcount;
    const int ctas = (int)std::min<long long>(kEigCtas / 4, (n4 + kEigThreads - 1) / kEigThreads);
    resid_kernel<<<dim3(std::max(1, ctas), m), kEigThreads, 0, st>>>(ra);
    DWF_CUDA_TRY(cudaGetLastError());
    int status = 0;
    DWF_CUDA_TRY(cudaMemcpyAsync(theta.data(), E.theta, sizeof(double) * m,
                                 cudaMemcpyDeviceToHost, st));
    DWF_CUDA_TRY(cudaMemcpyAsync(resid.data(), E.resid, sizeof(double) * m,
                                 cudaMemcpyDeviceToHost, st));
    DWF_CUDA_TRY(cudaMemcpyAsync(&status, E.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    DWF_CUDA_TRY(cudaStreamSynchronize(st));
    DWF_REQUIRE(status == 0, DWF_ERR_NAN,
                "eig: the filtered subspace lost rank (Gram matrix not positive definite)");
    for (int j = 0; j < m; ++j)
      DWF_REQUIRE(std::isfinite(theta[j]) && std::isfinite(resid[j]), DWF_ERR_NAN,
                  "eig: non-finite Ritz value or residual");
  };

  DWF_CUDA_TRY(cudaMemcpyAsync(W, V, (size_t)vs * m, cudaMemcpyDeviceToDevice, st));
  rayleigh_ritz();
  auto converged = [&]() {
    if (!(p.tol > 0.0)) return false;
    for (int j = 0; j < p.n_ev; ++j)
      if (resid[j] > p.tol * lam_max) return false;
    return true;
  };
  int passes = 0;
  while (passes < p.max_passes && !converged()) {
    // filter V -> W with T_d on [a, lam_max], a = the largest Ritz value
    const double a = std::min(theta[m - 1], 0.5 * lam_max);
    const double c = 0.5 * (a + lam_max), e = 0.5 * (lam_max - a);
    for (int b0 = 0; b0 < m; b0 += batch) {
      const int nb = std::min(batch, m - b0);
      char *vb = V + b0 * vs, *wb = W + b0 * vs;
      char *Z = Tb[2];  // A applied to the current term
      const char *tprev = vb;
      char *tcur = p.degree == 1 ? wb : Tb[0];
      matvec(Z, vb, nb);
      cheb_step(Z, vb, nullptr, tcur, vs, nb, n4, 1.0 / e, c, 0.0, st);
      for (int k = 2; k <= p.degree; ++k) {
        matvec(Z, tcur, nb);
        char *out = k == p.degree ? wb : (tprev == vb ? Tb[1] : const_cast<char *>(tprev));
        cheb_step(Z, tcur, tprev, out, vs, nb, n4, 2.0 / e, c, 1.0, st);
        tprev = tcur;
        tcur = out;
      }
    }
    rayleigh_ritz();
    ++passes;
  }
  for (int j = 0; j < m; ++j) {
    theta_h[j] = theta[j];
    resid_h[j] = resid[j];
  }
  if (info) {
    info->passes = passes;
    info->converged = converged() ? 1 : 0;
    info->matvecs = matvecs;
    info->lambda_max = lam_max;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
}

// ---------------------------------------------------------------------------
// Deflation of the outer solve
// ---------------------------------------------------------------------------
void deflate_start(const Deflation &d, const char *b64, char *x64, long long stride64, int nrhs,
                   long long cs, cudaStream_t st) {
  VecSet Vs;
  Vs.p = d.V;
  Vs.vs = d.vs;
  Vs.n = d.n_ev;
  Vs.prec = d.vprec;
  Vs.soff = d.vsoff;
  VecSet Bs;
  Bs.p = b64;
  Bs.vs = stride64;
  Bs.n = nrhs;
  Bs.prec = DWF_FP64;
  gram(Vs, Bs, cs, d.c, nrhs, d.dw, st);
  combine(Vs, d.c, nrhs, d.inv_lam, nullptr, x64, stride64, DWF_FP64, nrhs, nullptr, cs, st);
}

// rz_new += sum_j |c_j|^2 / lambda_j (or rr + that sum).
__global__ void defl_rz_kernel(const double2 *c, const double *inv_lam, int n_ev, int nrhs,
                               int z_from_r, OuterScalars *scal, const int *skip) {
  const int r = threadIdx.x;
  if (r >= nrhs || (skip && skip[r])) return;
  double s = 0.0;
  for (int j = 0; j < n_ev; ++j) {
    const double2 v = c[j * nrhs + r];
    s += (v.x * v.x + v.y * v.y) * inv_lam[j];
  }
  scal[r].rz_new = (z_from_r ? scal[r].rr : scal[r].rz_new) + s;
}

void deflate_correct(const Deflation &d, dwf_prec lo, const char *r, char *z, long long stride,
                     int nrhs, int z_from_r, OuterScalars *scal, const int *skip, long long cs,
                     cudaStream_t st) {
  VecSet Vs;
  Vs.p = d.V;
  Vs.vs = d.vs;
  Vs.n = d.n_ev;
  Vs.prec = d.vprec;
  Vs.soff = d.vsoff;
  VecSet Rs;
  Rs.p = r;
  Rs.vs = stride;
  Rs.n = nrhs;
  Rs.prec = lo;
  gram(Vs, Rs, cs, d.c, nrhs, d.dw, st);
  combine(Vs, d.c, nrhs, d.inv_lam, z_from_r ? r : z, z, stride, lo, nrhs, skip, cs, st);
  defl_rz_kernel<<<1, 32, 0, st>>>(d.c, d.inv_lam, d.n_ev, nrhs, z_from_r, scal, skip);
  DWF_CUDA_TRY(cudaGetLastError());
}

}  // namespace dwf

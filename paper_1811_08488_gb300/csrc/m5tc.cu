// M_5^-1 (and its adjoint) as a tensor-core GEMM batched over right-hand sides
// (paper Sec. 2.2: M_5 = alpha + beta C is Ls-local, so M_5^-1 is one dense
// Ls x Ls real matrix per chirality).
//
// For one chirality chi and one right-hand side, every (site, spin, colour,
// re/im) of that chirality is an Ls-vector, and
//     out[(h, r), s] = sum_s' in[(h, r), s'] (M_5^-1)_chi[s, s']
// is a real GEMM D = A B with M = 12 * sites (rows (h, r)), K = N = Ls.
// A CTA takes 32 sites of one right-hand side: 2 chiralities x 384 rows =
// six M = 128 tiles; each tile is one tcgen05.mma of kind::f16 per K step of
// 16 (Ls padded to LP = 16 or 32 with zero rows of B and zero columns of A),
// accumulated in FP32 in tensor memory (TMEM). A is written in the MN-major
// operand layout straight from coalesced global loads (the four rows of one
// 16-byte input chunk are contiguous there), B (host-built) is K-major.
//
// Precision. Operands are FP16. Every (site, chirality) slab of A is first
// scaled by a power of two so that its largest entry lies in [0.5, 1), and B
// (M_5^-1 for that right-hand side, built and inverted on the host in FP64)
// likewise; the scales are undone exactly in the epilogue. FP32 fields split
// both operands into hi + lo FP16 parts (the three products hi*hi, hi*lo,
// lo*hi; split-precision tensor-core products as in Markidis et al., IPDPSW
// 2018), about 2^-21 of each slab's largest entry. FP16/BF16 fields take
// A hi and B hi + lo, at the 2^-11 of their own storage.
//
// The path is HBM-bound: it moves 2 * 96 B (FP32) per (site, s) for
// 2 * 24 * Ls flops, far below the tensor pipe's ridge.
#include <cuda_fp16.h>

#include <cmath>
#include <cstdlib>
#include <vector>

#include "device_common.cuh"

namespace dwf {
namespace {

constexpr int kTcSites = 32;    // sites per CTA
constexpr int kTcThreads = 256;
constexpr int kTcTiles = 6;     // 2 chiralities x (12 rows x 32 sites / 128)

struct TcParams {
  const char *in;
  char *out;
  long long rstride;  // bytes between right-hand sides
  long long soff;     // FP16/BF16: byte offset of the scale array
  const uint4 *bimg;  // [rhs][chi][term] B operands in the canonical smem layout
  float b_unscale[kMaxRhs][2];
  int nsite, Ls;
  int *status;        // set to 1 when a bounded wait gave up
  int starve;                  // test hook: also wait for a phase nothing completes
  unsigned long long wait_ns;  // limit of the bounded wait
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// tcgen05 shared-memory matrix descriptor: start address, leading (K) and
// stride (M/N) byte offsets between 8 x 16-byte core matrices, version 1,
// no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) |
         (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of an mbarrier, giving up after limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t addr, uint32_t parity,
                                                  uint64_t limit_ns) {
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&d)[N]);
template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, uint32_t (&d)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]),
        "=r"(d[7]), "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]),
        "=r"(d[14]), "=r"(d[15])
      : "r"(taddr));
}
template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t taddr, uint32_t (&d)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]),
        "=r"(d[7]), "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]),
        "=r"(d[14]), "=r"(d[15]), "=r"(d[16]), "=r"(d[17]), "=r"(d[18]), "=r"(d[19]),
        "=r"(d[20]), "=r"(d[21]), "=r"(d[22]), "=r"(d[23]), "=r"(d[24]), "=r"(d[25]),
        "=r"(d[26]), "=r"(d[27]), "=r"(d[28]), "=r"(d[29]), "=r"(d[30]), "=r"(d[31])
      : "r"(taddr));
}

// Power of two 2^k as a float, k clamped to the normal range.
__device__ __forceinline__ float pow2f(int k) {
  k = max(-126, min(127, k));
  return __int_as_float((k + 127) << 23);
}

template <int LP>
__host__ __device__ constexpr int tc_cols() {
  return kTcTiles * LP <= 128 ? 128 : 256;
}

// Bytes of the shared region that holds the A operands and, once the MMAs
// are done, the FP32 output staging [chunk][site][s][4] (chunks padded by 16 B).
template <int LP, bool SPLIT>
__host__ __device__ inline int tc_region_bytes(int Ls) {
  const int a = (SPLIT ? 2 : 1) * kTcTiles * 128 * LP * 2;
  const int stg = 6 * (kTcSites * Ls * 4 + 4) * 4;
  const int r = a > stg ? a : stg;
  return (r + 127) / 128 * 128;
}

// Load the 4 reals 4c .. 4c+3 of element e (FP32 chunk c of the FP32 layout;
// for FP16/BF16 the halves 4(c % 2) .. +3 of chunk c / 2, times the scale).
template <class S>
__device__ __forceinline__ float4 load_quad(const char *ip, long long soff, int cs, int c, int e) {
  if constexpr (std::is_same<S, F32>::value) {
    return __ldg(reinterpret_cast<const float4 *>(ip) + (size_t)c * cs + e);
  } else {
    const uint2 q = __ldg(reinterpret_cast<const uint2 *>(
                              reinterpret_cast<const uint4 *>(ip) + (size_t)(c >> 1) * cs + e) +
                          (c & 1));
    float w[8];
    unpack8<S>(make_uint4(q.x, q.y, 0u, 0u), w);
    const float f = __ldg(reinterpret_cast<const float *>(ip + soff) + e);
    return make_float4(w[0] * f, w[1] * f, w[2] * f, w[3] * f);
  }
}

template <class S, int LP, bool SPLIT>
__global__ void __launch_bounds__(kTcThreads, 4) m5inv_gemm_kernel(const __grid_constant__ TcParams P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int kTileBytes = 128 * LP * 2;    // one M = 128 tile, K = LP FP16
  constexpr int kABytes = kTcTiles * kTileBytes;
  constexpr int kBImg = LP * LP * 2;          // one N x K image
  constexpr uint32_t kCols = tc_cols<LP>();
  const int Ls = P.Ls;
  const int chs = kTcSites * Ls * 4 + 4;      // staging floats per chunk (padded)

  unsigned char *A = smem;
  float *stg = reinterpret_cast<float *>(smem);
  unsigned char *B = smem + tc_region_bytes<LP, SPLIT>(Ls);
  float *sig_inv = reinterpret_cast<float *>(B + 4 * kBImg);  // [site][chi]: 2^e
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sig_inv + 2 * kTcSites);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rhs = blockIdx.y;
  const int h0 = blockIdx.x * kTcSites;
  const int nh = min(kTcSites, P.nsite - h0);
  const int cs = P.nsite * Ls;
  const char *ip = P.in + rhs * P.rstride;
  char *op = P.out + rhs * P.rstride;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B operands of this right-hand side (four images: chi x {hi, lo})
  {
    const uint4 *src = P.bimg + (size_t)rhs * (4 * kBImg / 16);
    uint4 *dst = reinterpret_cast<uint4 *>(B);
    for (int i = tid; i < 4 * kBImg / 16; i += kTcThreads) dst[i] = __ldg(src + i);
  }
  // A operands in the canonical MN-major layout without swizzle: element
  // (row m, K index k) of tile t at t*kTileBytes + (m/8)*128 + (k/8)*2048 +
  // (k%8)*16 + (m%8)*2, so the four consecutive rows of one 16-byte input
  // chunk at one s are one 8-byte store. K indices s >= Ls are zero.
  for (int i = tid; i < 2 * kTcTiles * 16 * (LP - Ls); i += kTcThreads) {
    const int term = i / (kTcTiles * 16 * (LP - Ls)), r = i % (kTcTiles * 16 * (LP - Ls));
    const int t = r / (16 * (LP - Ls)), g = (r / (LP - Ls)) % 16, k = Ls + r % (LP - Ls);
    if (term == 0 || SPLIT)
      *reinterpret_cast<uint4 *>(A + term * kABytes + t * kTileBytes + g * 128 + (k >> 3) * 2048 +
                                 (k & 7) * 16) = make_uint4(0u, 0u, 0u, 0u);
  }
  // Thread (site h = tid / 8, lane q = tid % 8) owns the quads of its site at
  // s = q + 8j: the eight lanes of a site read its chunk rows as contiguous
  // 128-byte pieces, and hold the whole (site, chirality) slab between them.
  {
    constexpr int KJ = LP / 8;  // s values per lane
    const int h = tid >> 3, q = tid & 7;
    const bool hv = h < nh;
#pragma unroll 1
    for (int chi = 0; chi < 2; ++chi) {
      float m = 0.f;
      float4 v[3][KJ];
#pragma unroll
      for (int cc = 0; cc < 3; ++cc)
#pragma unroll
        for (int j = 0; j < KJ; ++j) {
          const int k = q + 8 * j;
          v[cc][j] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (hv && k < Ls) {
            v[cc][j] = load_quad<S>(ip, P.soff, cs, chi * 3 + cc, (h0 + h) * Ls + k);
            m = fmaxf(m, fmaxf(fmaxf(fabsf(v[cc][j].x), fabsf(v[cc][j].y)),
                               fmaxf(fabsf(v[cc][j].z), fabsf(v[cc][j].w))));
          }
        }
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      // m = f 2^e with f in [0.5, 1): the scaled slab has its maximum in [0.5, 1)
      const int ex = (m > 0.f && m < INFINITY) ? ((__float_as_int(m) >> 23) & 0xFF) - 126 : 0;
      const float sc = pow2f(-ex);
      if (q == 0) sig_inv[h * 2 + chi] = pow2f(ex);
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        const int rho0 = h * 12 + 4 * cc;  // first of the four rows within the chirality
        const int t = chi * 3 + rho0 / 128, m0 = rho0 % 128;
#pragma unroll
        for (int j = 0; j < KJ; ++j) {
          const int k = q + 8 * j;
          if (k >= Ls) continue;
          const float4 w = make_float4(v[cc][j].x * sc, v[cc][j].y * sc, v[cc][j].z * sc,
                                       v[cc][j].w * sc);
          const __half2 a0 = __floats2half2_rn(w.x, w.y), a1 = __floats2half2_rn(w.z, w.w);
          const int off = t * kTileBytes + (m0 >> 3) * 128 + (k >> 3) * 2048 + (k & 7) * 16 +
                          (m0 & 7) * 2;
          uint2 hi;
          *reinterpret_cast<__half2 *>(&hi.x) = a0;
          *reinterpret_cast<__half2 *>(&hi.y) = a1;
          *reinterpret_cast<uint2 *>(A + off) = hi;
          if (SPLIT) {
            const float2 f0 = __half22float2(a0), f1 = __half22float2(a1);
            uint2 lo;
            *reinterpret_cast<__half2 *>(&lo.x) = __floats2half2_rn(w.x - f0.x, w.y - f0.y);
            *reinterpret_cast<__half2 *>(&lo.y) = __floats2half2_rn(w.z - f1.x, w.w - f1.y);
            *reinterpret_cast<uint2 *>(A + kABytes + off) = lo;
          }
        }
      }
    }
  }

  // make the generic-proxy smem writes visible to the tensor core, then issue
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *tslot;
  if (tid == 0) {
    // kind::f16, D FP32, A and B FP16, A MN-major, B K-major, N = LP, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 15) | ((uint32_t)(LP >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);
    const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
    for (int t = 0; t < kTcTiles; ++t) {
      const int chi = t / 3;
      uint32_t acc = 0;
      // products hi*hi, hi*lo (B), lo*hi (A, FP32 fields only)
      for (int term = 0; term < (SPLIT ? 3 : 2); ++term) {
        const int at = term == 2 ? 1 : 0, bt = term == 1 ? 1 : 0;
        for (int kk = 0; kk < LP / 16; ++kk) {
          // A: K groups 2048 bytes apart (LBO), M groups 128 bytes apart (SBO)
          const uint64_t ad = umma_desc(a0 + at * kABytes + t * kTileBytes + kk * 4096, 2048, 128);
          const uint64_t bd = umma_desc(b0 + (chi * 2 + bt) * kBImg + kk * 256, 128, LP * 16);
          umma_f16(tbase + t * LP, ad, bd, idesc, acc);
          acc = 1;
        }
      }
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(mbar))
        : "memory");
  }
  const bool mma_done = __syncthreads_and(mbar_wait_bounded(smem_u32(mbar), 0, P.wait_ns));
  // test hook: the second phase is never completed (no further arrival), so
  // this wait runs out after the MMAs have finished (phase 0 above)
  bool hook_ok = true;
  if (P.starve && mma_done) hook_ok = mbar_wait_bounded(smem_u32(mbar), 1, P.wait_ns);
  const bool ok = __syncthreads_and(mma_done && hook_ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // status 1: only the test hook's wait expired (the MMAs had completed);
  // status 2: the MMA commit itself did not arrive in time, so MMAs may still
  // be reading this CTA's shared memory and writing its TMEM columns
  if (!ok && tid == 0) atomicMax(P.status, mma_done ? 1 : 2);

  if (ok) {
    // TMEM -> staging (the A region is free once the MMAs completed): warp w
    // reads lanes 32 (w % 4) .. +31 of tiles t = w/4, w/4 + 2, ...
    const int sub = warp & 3;
    for (int t = warp >> 2; t < kTcTiles; t += 2) {
      uint32_t d[LP];
      tmem_ld<LP>(tbase + ((uint32_t)(sub * 32) << 16) + (uint32_t)(t * LP), d);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int m = sub * 32 + lane;
      const int chi = t / 3, rho = (t % 3) * 128 + m, h = rho / 12, r = rho - h * 12;
      const int c = chi * 3 + (r >> 2), j = r & 3;
      if (h < nh) {
        const float us = sig_inv[h * 2 + chi] * P.b_unscale[rhs][chi];
#pragma unroll
        for (int s = 0; s < LP; ++s)
          if (s < Ls) stg[c * chs + (h * Ls + s) * 4 + j] = __uint_as_float(d[s]) * us;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  if constexpr (std::is_same<S, F32>::value) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kCols)
                 : "memory");
  if (!ok) return;
  if constexpr (std::is_same<S, F32>::value) {
    // each chunk's sites are one contiguous run in global memory: bulk copies
    if (tid == 0) {
      const uint32_t bytes = (uint32_t)nh * Ls * 16;
      for (int c = 0; c < 6; ++c) {
        char *dst = op + ((size_t)c * cs + (size_t)h0 * Ls) * 16;
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                     "r"(smem_u32(stg + c * chs)), "r"(bytes)
                     : "memory");
      }
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
  } else {
    for (int e = tid; e < nh * Ls; e += kTcThreads) {
      float v[24];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const float4 q = *reinterpret_cast<const float4 *>(stg + c * chs + e * 4);
        v[4 * c] = q.x; v[4 * c + 1] = q.y; v[4 * c + 2] = q.z; v[4 * c + 3] = q.w;
      }
      store24<S>(op, P.soff, cs, h0 * Ls + e, v);
    }
  }
}

template <int LP, bool SPLIT>
size_t tc_smem_bytes(int Ls) {
  const size_t b = 4u * LP * LP * 2;
  const size_t bytes = (size_t)tc_region_bytes<LP, SPLIT>(Ls) + b + 2u * kTcSites * 4 + 16;
  // at least 48 KB: at most four CTAs (4 x 128 TMEM columns) share an SM
  return bytes < 48u * 1024 ? 48u * 1024 : bytes;
}

// Dense M_5 of one chirality (Sec. 2.2): alpha on the diagonal, beta on the
// chiral shift, -m_f on its wrap; `down` = the shift takes s-1 (P_+ with the
// chiral basis gamma_5 = diag(1, 1, -1, -1)).
void m5_dense(const dwf_action &a, double mf, bool down, std::vector<double> &M) {
  const int L = a.Ls;
  const double al = a.b * (4.0 - a.M5) + 1.0, be = a.c * (4.0 - a.M5) - 1.0;
  M.assign((size_t)L * L, 0.0);
  for (int s = 0; s < L; ++s) {
    M[(size_t)s * L + s] = al;
    if (down) {
      if (s > 0) M[(size_t)s * L + s - 1] += be;
      else M[(size_t)s * L + L - 1] += -mf * be;
    } else {
      if (s < L - 1) M[(size_t)s * L + s + 1] += be;
      else M[(size_t)s * L] += -mf * be;
    }
  }
}

// Gauss-Jordan inverse with partial pivoting (FP64, Ls <= 32).
void invert(std::vector<double> M, int L, std::vector<double> &X) {
  X.assign((size_t)L * L, 0.0);
  for (int i = 0; i < L; ++i) X[(size_t)i * L + i] = 1.0;
  for (int col = 0; col < L; ++col) {
    int piv = col;
    for (int r = col + 1; r < L; ++r)
      if (std::fabs(M[(size_t)r * L + col]) > std::fabs(M[(size_t)piv * L + col])) piv = r;
    DWF_REQUIRE(M[(size_t)piv * L + col] != 0.0, DWF_ERR_INVALID_ARG, "M_5 is singular");
    if (piv != col)
      for (int k = 0; k < L; ++k) {
        std::swap(M[(size_t)piv * L + k], M[(size_t)col * L + k]);
        std::swap(X[(size_t)piv * L + k], X[(size_t)col * L + k]);
      }
    const double d = 1.0 / M[(size_t)col * L + col];
    for (int k = 0; k < L; ++k) {
      M[(size_t)col * L + k] *= d;
      X[(size_t)col * L + k] *= d;
    }
    for (int r = 0; r < L; ++r) {
      if (r == col) continue;
      const double f = M[(size_t)r * L + col];
      if (f == 0.0) continue;
      for (int k = 0; k < L; ++k) {
        M[(size_t)r * L + k] -= f * M[(size_t)col * L + k];
        X[(size_t)r * L + k] -= f * X[(size_t)col * L + k];
      }
    }
  }
}

}  // namespace

void launch_m5inv_gemm(dwf_ctx *ctx, dwf_prec p, char *out, const char *in, int dagger, int nrhs,
                       const double *mf, cudaStream_t st) {
  const int Ls = ctx->act.Ls, nsite = ctx->geo.Vh;
  DWF_REQUIRE(Ls <= 32, DWF_ERR_UNSUPPORTED, "the tensor-core M_5^-1 takes Ls <= 32");
  DWF_REQUIRE(p == DWF_FP32 || p == DWF_FP16 || p == DWF_BF16, DWF_ERR_UNSUPPORTED,
              "the tensor-core M_5^-1 takes FP32, FP16 or BF16 fields");
  const int LP = Ls <= 16 ? 16 : 32;
  const size_t img = (size_t)LP * LP;  // halves per image
  TcParams P{};
  // B operands: rebuilt only when the masses or the adjoint flag change
  std::vector<double> key(mf, mf + nrhs);
  key.push_back(dagger ? 1.0 : 0.0);
  ctx->tc_aux.ensure(256 + (size_t)kMaxRhs * 4 * 32 * 32 * 2);
  if (key != ctx->tc_key) {
    std::vector<__half> B((size_t)nrhs * 4 * img, __float2half_rn(0.f));
    std::vector<double> M, X;
    for (int r = 0; r < nrhs; ++r)
      for (int chi = 0; chi < 2; ++chi) {
        // reals 0..11 (P_+) shift down; the adjoint is the transpose, which
        // shifts the other way
        m5_dense(ctx->act, mf[r], (chi == 0) != (dagger != 0), M);
        invert(M, Ls, X);
        double mx = 0.0;
        for (double v : X) mx = std::fmax(mx, std::fabs(v));
        int e = 0;
        if (mx > 0.0) std::frexp(mx, &e);
        const double sc = std::ldexp(1.0, -e);
        ctx->tc_unscale[r][chi] = (float)std::ldexp(1.0, e);
        for (int n = 0; n < Ls; ++n)
          for (int k = 0; k < Ls; ++k) {
            // B[k][n] = X[n][k], stored K-major: row n, K contiguous
            const double v = X[(size_t)n * Ls + k] * sc;
            const __half hi = __float2half_rn((float)v);
            const __half lo = __float2half_rn((float)(v - (double)__half2float(hi)));
            const size_t o = (size_t)(n / 8) * (LP * 8) + (k / 8) * 64 + (n % 8) * 8 + (k % 8);
            B[((size_t)r * 4 + chi * 2 + 0) * img + o] = hi;
            B[((size_t)r * 4 + chi * 2 + 1) * img + o] = lo;
          }
      }
    // a pageable source: the copy is staged before cudaMemcpyAsync returns
    DWF_CUDA_TRY(cudaMemcpyAsync(ctx->tc_aux.c() + 256, B.data(), B.size() * sizeof(__half),
                                 cudaMemcpyHostToDevice, st));
    ctx->tc_key = key;
  }
  for (int r = 0; r < nrhs; ++r)
    for (int chi = 0; chi < 2; ++chi) P.b_unscale[r][chi] = ctx->tc_unscale[r][chi];
  int *status = ctx->tc_aux.as<int>();
  DWF_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
  P.in = in;
  P.out = out;
  P.rstride = (long long)field_rhs_bytes(p, nsite, Ls);
  P.soff = (long long)align_up(field_data_bytes(p, nsite, Ls), 256);
  P.bimg = reinterpret_cast<const uint4 *>(ctx->tc_aux.c() + 256);
  P.nsite = nsite;
  P.Ls = Ls;
  P.status = status;
  P.starve = 0;
  P.wait_ns = 1000000000ull;  // 1 s
  // Failure-detection test hook: with DWF_TEST_STARVE_WAIT=1 every CTA, after
  // its MMAs have completed, also waits for a barrier phase that nothing
  // completes; the wait gives up after 1 ms, the CTA frees its TMEM and
  // returns, and the call reports DWF_ERR_TIMEOUT.
  if (const char *t = std::getenv("DWF_TEST_STARVE_WAIT")) {
    if (t[0] == '1') {
      P.starve = 1;
      P.wait_ns = 1000000ull;
    }
  }
  dim3 grid((nsite + kTcSites - 1) / kTcSites, nrhs), block(kTcThreads);
#define TCK(ST, L, SP)                                                                     \
  do {                                                                                     \
    const size_t smem = tc_smem_bytes<L, SP>(Ls);                                          \
    DWF_CUDA_TRY(cudaFuncSetAttribute(m5inv_gemm_kernel<ST, L, SP>,                        \
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    m5inv_gemm_kernel<ST, L, SP><<<grid, block, smem, st>>>(P);                            \
  } while (0)
  if (p == DWF_FP32) {
    if (LP == 16) TCK(F32, 16, true); else TCK(F32, 32, true);
  } else if (p == DWF_FP16) {
    if (LP == 16) TCK(F16, 16, false); else TCK(F16, 32, false);
  } else {
    if (LP == 16) TCK(BF16, 16, false); else TCK(BF16, 32, false);
  }
#undef TCK
  DWF_CUDA_TRY(cudaGetLastError());
  int h_status = 0;
  DWF_CUDA_TRY(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  DWF_CUDA_TRY(cudaStreamSynchronize(st));
  if (h_status == 2) {
    // after a genuine expiry the abandoned MMAs may still write TMEM and read
    // shared memory that later CTAs reuse: nothing on this context is trusted
    ctx->unusable = 1;
    throw Error{DWF_ERR_TIMEOUT,
                "tensor-core M_5^-1: the MMA completion wait expired; the context is unusable "
                "and must be destroyed"};
  }
  DWF_REQUIRE(h_status == 0, DWF_ERR_TIMEOUT,
              "tensor-core M_5^-1: a bounded wait expired after the MMAs completed");
}

}  // namespace dwf

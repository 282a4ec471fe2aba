// The 4D Wilson hop with the fifth dimension, the one kernel behind every
// operator application of the solver (paper Sec. 2.2, M^4 = D^w M_phi and
// eq. for D^w; Sec. 2.3 for its use inside the Dirichlet block operator).
//
// Two kernels. hop2_kernel (FP32/FP16/BF16 fields, even Ls): one thread per
// pair of slices (s0, s0 + 1) of one output site; the Ls/2 threads of a site
// are consecutive lanes of one warp (a warp holds whole sites), so the links
// of a site are loaded once per warp line, and everything that couples
// neighbouring slices -- M_phi on load (s0 - 1, s0 + 2), the Ls epilogue
// (M_phi^+, M_5^-1, K = M_phi M_5^-1 and their adjoints) and the x-term of the
// epilogue -- is exchanged between those lanes with warp shuffles; the
// epilogue's (1 - r S)^-1 is a scan over the site's lanes. It uses no shared
// memory outside its reductions, so the unified L1 serves the neighbour
// gather. hop_kernel (FP64 fields, odd Ls): one thread per output (site, s),
// the Ls epilogue walks columns in shared memory.
//
// For output site x and direction mu (chiral basis, g_mu = [[0, A],[A^+, 0]]):
//   forward : (1 - sg g_mu) U_mu(x)      chi(x+mu)
//   backward: (1 + sg g_mu) U_mu(x-mu)^+ chi(x-mu)
// with sg = +1 for Dhop and sg = -1 for Dhop^+. (1 - g)v = [h; -A^+ h] with
// h = v_u - A v_l, so only the two-spinor h is multiplied by the link.
// With PRE, the input is chi = M_phi psi = b psi + c C psi, formed on load:
// chi_u(s) = b psi_u(s) + c psi_u(s-1), chi_l(s) = b psi_l(s) + c psi_l(s+1),
// with the wrap factor -m_f.
#include <type_traits>

#include "device_common.cuh"

namespace dwf {

template <class R>
struct Cx {
  R re, im;
};

// (A v_l) for the two lower spins v2, v3 -> a0, a1 (per colour).
template <int MU, class R>
__device__ __forceinline__ void a_times(const Cx<R> v2, const Cx<R> v3, Cx<R> &a0, Cx<R> &a1) {
  if constexpr (MU == 0) {  // A = -i sigma_1
    a0 = {v3.im, -v3.re};
    a1 = {v2.im, -v2.re};
  } else if constexpr (MU == 1) {  // A = -i sigma_2 = [[0,-1],[1,0]]
    a0 = {-v3.re, -v3.im};
    a1 = {v2.re, v2.im};
  } else if constexpr (MU == 2) {  // A = -i sigma_3 = diag(-i, i)
    a0 = {v2.im, -v2.re};
    a1 = {-v3.im, v3.re};
  } else {  // A = 1
    a0 = v2;
    a1 = v3;
  }
}

// (A^+ w) for the two projected spins w0, w1 -> b0, b1.
template <int MU, class R>
__device__ __forceinline__ void adag_times(const Cx<R> w0, const Cx<R> w1, Cx<R> &b0, Cx<R> &b1) {
  if constexpr (MU == 0) {  // A^+ = i sigma_1
    b0 = {-w1.im, w1.re};
    b1 = {-w0.im, w0.re};
  } else if constexpr (MU == 1) {  // A^+ = [[0,1],[-1,0]]
    b0 = w1;
    b1 = {-w0.re, -w0.im};
  } else if constexpr (MU == 2) {  // A^+ = diag(i, -i)
    b0 = {-w0.im, w0.re};
    b1 = {w1.im, -w1.re};
  } else {
    b0 = w0;
    b1 = w1;
  }
}

template <class R, int MU, bool FWD, bool DAG>
__device__ __forceinline__ void proj_mul_acc(R *acc, const R *v, const R *u);

// One direction of the hop: project, multiply by U or U^+, reconstruct, add.
// `lk` is the link record.
template <class S, int MU, bool FWD, bool DAG, bool PRE, bool RC>
__device__ __forceinline__ void hop_dir(typename S::R *acc, const char *in, long long soff,
                                        int cs, int j, int s, int Ls, const uint4 *lk,
                                        size_t ls, const LsCoef &cf) {
  using R = typename S::R;
  R v[24];
  load24<S>(in, soff, cs, j * Ls + s, v);
  if constexpr (PRE) {
    R w[12];
    const LsK<R> &kk = kc<R>(cf);
    const R b = kk.pre_b, c = kk.pre_c, mf = kk.mf;
    const int sm = s == 0 ? Ls - 1 : s - 1;
    const R fm = s == 0 ? -mf : (R)1;
    load12<S, true>(in, soff, cs, j * Ls + sm, w);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = b * v[k] + c * fm * w[k];
    const int sp = s == Ls - 1 ? 0 : s + 1;
    const R fp = s == Ls - 1 ? -mf : (R)1;
    load12<S, false>(in, soff, cs, j * Ls + sp, w);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[12 + k] = b * v[12 + k] + c * fp * w[k];
  }
  R u[18];
  load_link<S>(lk, ls, u, RC ? 1 : 0);
  proj_mul_acc<R, MU, FWD, DAG>(acc, v, u);
}

// Project v with (1 - sg g_mu), multiply the two-spinor by U (forward) or U^+
// (backward), reconstruct and add to acc.
template <class R, int MU, bool FWD, bool DAG>
__device__ __forceinline__ void proj_mul_acc(R *acc, const R *v, const R *u) {
  constexpr R sg = (FWD != DAG) ? (R)1 : (R)-1;  // projector (1 - sg g_mu)
  Cx<R> h[2][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Cx<R> v0{v[0 * 6 + 2 * c], v[0 * 6 + 2 * c + 1]};
    Cx<R> v1{v[1 * 6 + 2 * c], v[1 * 6 + 2 * c + 1]};
    Cx<R> v2{v[2 * 6 + 2 * c], v[2 * 6 + 2 * c + 1]};
    Cx<R> v3{v[3 * 6 + 2 * c], v[3 * 6 + 2 * c + 1]};
    Cx<R> a0, a1;
    a_times<MU>(v2, v3, a0, a1);
    h[0][c] = {v0.re - sg * a0.re, v0.im - sg * a0.im};
    h[1][c] = {v1.re - sg * a1.re, v1.im - sg * a1.im};
  }
  Cx<R> w[2][3];
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      R re = 0, im = 0;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        // forward: U[a][b]; backward: conj(U[b][a])
        const R ur = FWD ? u[2 * (3 * a + b)] : u[2 * (3 * b + a)];
        const R ui = FWD ? u[2 * (3 * a + b) + 1] : -u[2 * (3 * b + a) + 1];
        re += ur * h[sp][b].re - ui * h[sp][b].im;
        im += ur * h[sp][b].im + ui * h[sp][b].re;
      }
      w[sp][a] = {re, im};
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Cx<R> b0, b1;
    adag_times<MU>(w[0][c], w[1][c], b0, b1);
    acc[0 * 6 + 2 * c] += w[0][c].re;
    acc[0 * 6 + 2 * c + 1] += w[0][c].im;
    acc[1 * 6 + 2 * c] += w[1][c].re;
    acc[1 * 6 + 2 * c + 1] += w[1][c].im;
    acc[2 * 6 + 2 * c] -= sg * b0.re;
    acc[2 * 6 + 2 * c + 1] -= sg * b0.im;
    acc[3 * 6 + 2 * c] -= sg * b1.re;
    acc[3 * 6 + 2 * c + 1] -= sg * b1.im;
  }
}

template <class S, int MU, bool DAG, bool PRE, bool RC>
__device__ __forceinline__ void hop_mu(typename S::R *acc, const HopParams &P, const char *in,
                                       const uint4 *links, const int *nb, int site, int s,
                                       const LsCoef &cf) {
  constexpr int LC = RC ? S::kLinkChunksRecon : S::kLinkChunks;
  const int jf = nb[2 * MU], jb = nb[2 * MU + 1];
  const size_t ls = (size_t)P.link_cs;
  const uint4 *lmu = links + (size_t)MU * LC * ls;
  if (jf >= 0 && jf < P.in_limit)
    hop_dir<S, MU, true, DAG, PRE, RC>(acc, in, P.in.scale_off, P.in.cs, jf, s, P.Ls,
                                   lmu + P.out_link_off + site, ls, cf);
  if (jb >= 0 && jb < P.in_limit)
    hop_dir<S, MU, false, DAG, PRE, RC>(acc, in, P.in.scale_off, P.in.cs, jb, s, P.Ls,
                                    lmu + P.in_link_off + jb, ls, cf);
}

// Shared memory of one CTA for the Ls epilogue: the hop result T and the
// own-site input X as [site][component][Ls + 1] columns.
template <class R>
__device__ __forceinline__ void epilogue_columns(R *T, const R *X, int nsites, int site0,
                                                 int n_out, int Ls, bool dag, int inv,
                                                 const LsCoef &cf) {
  const int col = Ls + 1;
  for (int w = threadIdx.x; w < nsites * 24; w += blockDim.x) {
    if (site0 + w / 24 >= n_out) continue;
    const bool down = ((w % 24) < 12) != dag;
    ls_column<R>(T + w * col, X ? X + w * col : nullptr, Ls, down, inv != 0, kc<R>(cf));
  }
}

// One thread's part of the fused <dotv, out> of the global dot products. The
// FP32 products are summed with Kahan compensation, so the sum's error is at
// most about 3 * 2^-24 * sum |d_k a_k| (one rounding per product, two for the
// compensated sum) whatever the count; the partials are then added in FP64.
// FP64 fields sum in FP64.
template <class R>
__device__ __forceinline__ double dot_compensated(const R *d, const R *a, int n) {
  if constexpr (std::is_same<R, double>::value) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 24; ++k)
      if (k < n) s += d[k] * a[k];
    return s;
  } else {
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int k = 0; k < 24; ++k)
      if (k < n) {
        const float y = d[k] * a[k] - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
      }
    return (double)s - (double)c;
  }
}

// Publish the CTA's part of Re<dotv, out> (both summed per (rhs, block)).
__device__ __forceinline__ void hop_dot(const HopParams &P, double d, double *red, int rhs,
                                        int blk) {
  d = cta_sum(d, red);
  const int ntiles = gridDim.x;
  const int grp = rhs * P.nblocks + blk;
  double total;
  if (group_reduce(d, P.partials + (size_t)grp * ntiles, ntiles, blockIdx.x, P.counters + grp,
                   total))
    P.dot_out[(size_t)rhs * P.dot_rstride + blk] = total;
}

// Kernel timer (only when P.prof is set). CTA 0 reads the global timer at
// entry (CTAs are dispatched in index order, so it starts first); every CTA
// takes a ticket when it has finished, and the CTA with the last ticket reads
// the timer again, adds the span to the slot and resets it for the next
// launch. One atomic per CTA. Launches of one slot must not overlap in time
// (one stream at a time), which stream order guarantees.
__device__ __forceinline__ unsigned long long gtimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool first_cta() {
  return blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
}
__device__ __noinline__ void prof_enter(const HopParams &P) {
  if (P.prof && threadIdx.x == 0 && first_cta()) {
    P.prof->start = gtimer_ns();
    __threadfence();
  }
}
__device__ __noinline__ void prof_exit(const HopParams &P) {
  if (!P.prof) return;
  __syncthreads();
  if (threadIdx.x != 0) return;
  KernProf *k = P.prof;
  const unsigned int nct = gridDim.x * gridDim.y * gridDim.z;
  if (atomicAdd(&k->done, 1u) != nct - 1) return;
  __threadfence();
  const unsigned long long t1 = gtimer_ns();
  const unsigned long long t0 = *reinterpret_cast<volatile unsigned long long *>(&k->start);
  k->total_ns += t1 - t0;
  k->launches += 1;
  k->bytes += P.alg_bytes;
  k->done = 0;
  __threadfence();
}

// One thread per output (site, s): used for FP64 fields and odd Ls.
template <class S, bool DAG, bool PRE, bool RC>
__device__ __forceinline__ void hop_body(const HopParams &P) {
  using R = typename S::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  const int rhs = blockIdx.z, blk = blockIdx.y;
  if (P.skip && P.skip[rhs]) return;
  if (P.bskip && P.bskip[rhs * P.nblocks + blk]) return;
  const int Ls = P.Ls;
  const int nsites = P.nsites;  // blockDim.x is nsites * Ls rounded up to whole warps
  const int tid = threadIdx.x;
  const int s = tid % Ls, sl = tid / Ls;
  const int site0 = blockIdx.x * nsites;
  const int site = site0 + sl;
  const bool active = (sl < nsites) && (site < P.n_out);
  const LsCoef &cf = P.coef[rhs];

  const char *in = P.in.data + blk * P.in.bstride + rhs * P.in.rstride;
  char *out = P.out.data + blk * P.out.bstride + rhs * P.out.rstride;
  const uint4 *links = reinterpret_cast<const uint4 *>(P.links + blk * P.link_bstride);

  R acc[24];
#pragma unroll
  for (int k = 0; k < 24; ++k) acc[k] = 0;
  if (active) {
    const int *nb = P.nbr + (size_t)site * 8;
    hop_mu<S, 0, DAG, PRE, RC>(acc, P, in, links, nb, site, s, cf);
    hop_mu<S, 1, DAG, PRE, RC>(acc, P, in, links, nb, site, s, cf);
    hop_mu<S, 2, DAG, PRE, RC>(acc, P, in, links, nb, site, s, cf);
    hop_mu<S, 3, DAG, PRE, RC>(acc, P, in, links, nb, site, s, cf);
  }
  const int e = site * Ls + s;

  if (P.epi) {
    const int col = Ls + 1;
    R *T = reinterpret_cast<R *>(smem_raw);
    R *X = T + nsites * 24 * col;
    if (active) {
#pragma unroll
      for (int k = 0; k < 24; ++k) T[(sl * 24 + k) * col + s] = acc[k];
      if (P.has_x) {
        R xv[24];
        if (site < P.xown_limit) {
          const char *xo = P.xown.data + blk * P.xown.bstride + rhs * P.xown.rstride;
          load24<S>(xo, P.xown.scale_off, P.xown.cs, e, xv);
        } else {
#pragma unroll
          for (int k = 0; k < 24; ++k) xv[k] = 0;
        }
#pragma unroll
        for (int k = 0; k < 24; ++k) X[(sl * 24 + k) * col + s] = xv[k];
      }
    }
    __syncthreads();
    epilogue_columns<R>(T, P.has_x ? X : nullptr, nsites, site0, P.n_out, Ls, DAG, P.inv, cf);
    __syncthreads();
    if (active) {
#pragma unroll
      for (int k = 0; k < 24; ++k) acc[k] = T[(sl * 24 + k) * col + s];
    }
  } else {
    const R q = kc<R>(cf).q0;
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] *= q;
  }
  if (active) store24<S>(out, P.out.scale_off, P.out.cs, e, acc);

  if (P.dot) {
    double d = 0.0;
    if (active) {
      R dv[24];
      const char *dp = P.dotv.data + blk * P.dotv.bstride + rhs * P.dotv.rstride;
      load24<S>(dp, P.dotv.scale_off, P.dotv.cs, e, dv);
      d = dot_compensated<R>(dv, acc, 24);
    }
    hop_dot(P, d, red, rhs, blk);
  }
}

template <class S, bool DAG, bool PRE, bool RC>
__global__ void __launch_bounds__(256) hop_kernel(const __grid_constant__ HopParams P) {
  prof_enter(P);
  hop_body<S, DAG, PRE, RC>(P);
  prof_exit(P);
}

// ---------------------------------------------------------------------------
// Two slices per thread: thread (site, s0 = 2j) computes s0 and s0 + 1. Chunk c
// of both slices is one 32-byte word, so every spinor load and store is a
// 256-bit access and a warp moves one contiguous kilobyte per instruction; the
// link is loaded once for both slices; with M_phi on load, the two slices
// supply each other's s -> s +- 1 neighbours and only the outer two halves
// (s0 - 1 upper, s0 + 2 lower) are loaded in addition. Arithmetic runs on
// float2 pairs (slice s0, slice s0 + 1) with Blackwell's packed FP32
// instructions, so each multiply-add serves both slices. FP32/FP16/BF16, even Ls.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
// x + sgn * y on both lanes (sgn = +-1 at compile time): one packed FMA.
template <int SGN>
__device__ __forceinline__ float2 pm(float2 x, float2 y) {
  return __ffma2_rn(y, make_float2((float)SGN, (float)SGN), x);
}
struct C2 {
  float2 re, im;
};
// x + sgn * (ph * z), ph = i^PH (PH = 0: 1, 1: i, 2: -1, 3: -i).
template <int PH, int SGN>
__device__ __forceinline__ C2 add_phase(C2 x, C2 z) {
  if constexpr (PH == 0) return {pm<SGN>(x.re, z.re), pm<SGN>(x.im, z.im)};
  else if constexpr (PH == 1) return {pm<-SGN>(x.re, z.im), pm<SGN>(x.im, z.re)};
  else if constexpr (PH == 2) return {pm<-SGN>(x.re, z.re), pm<-SGN>(x.im, z.im)};
  else return {pm<SGN>(x.re, z.im), pm<-SGN>(x.im, z.re)};
}
// (A v_l)_sp = i^PH v_l[SRC]: per direction mu, for output spin 0 and 1.
template <int MU> struct ProjA;
template <> struct ProjA<0> { static constexpr int s0 = 1, p0 = 3, s1 = 0, p1 = 3; };  // -i s1
template <> struct ProjA<1> { static constexpr int s0 = 1, p0 = 2, s1 = 0, p1 = 0; };  // -i s2
template <> struct ProjA<2> { static constexpr int s0 = 0, p0 = 3, s1 = 1, p1 = 1; };  // -i s3
template <> struct ProjA<3> { static constexpr int s0 = 0, p0 = 0, s1 = 1, p1 = 0; };  // 1
// (A^+ w)_sp = i^PH w[SRC].
template <int MU> struct ProjAd;
template <> struct ProjAd<0> { static constexpr int s0 = 1, p0 = 1, s1 = 0, p1 = 1; };
template <> struct ProjAd<1> { static constexpr int s0 = 1, p0 = 0, s1 = 0, p1 = 2; };
template <> struct ProjAd<2> { static constexpr int s0 = 0, p0 = 1, s1 = 1, p1 = 3; };
template <> struct ProjAd<3> { static constexpr int s0 = 0, p0 = 0, s1 = 1, p1 = 0; };

// x + y * s on both lanes (s = the two slices' scales, or their negatives).
__device__ __forceinline__ float2 fma_s(float2 x, float2 y, float2 s) { return __ffma2_rn(y, s, x); }
// x + sgn * sc * (ph * z): add_phase with the slices' scales folded in.
template <int PH, int SGN>
__device__ __forceinline__ C2 add_phase_s(C2 x, C2 z, float2 sp, float2 sn) {
  const float2 a = SGN > 0 ? sp : sn, b = SGN > 0 ? sn : sp;  // +sgn*sc, -sgn*sc
  if constexpr (PH == 0) return {fma_s(x.re, z.re, a), fma_s(x.im, z.im, a)};
  else if constexpr (PH == 1) return {fma_s(x.re, z.im, b), fma_s(x.im, z.re, a)};
  else if constexpr (PH == 2) return {fma_s(x.re, z.re, b), fma_s(x.im, z.im, b)};
  else return {fma_s(x.re, z.im, a), fma_s(x.im, z.re, b)};
}

// Packed counterpart of proj_mul_acc: v, acc hold 24 reals of both slices.
// SCALED: v holds stored FP16/BF16 values whose per-slice scales sc are
// applied in the accumulation (the projector and U are linear).
template <int MU, bool FWD, bool DAG, bool SCALED = false>
__device__ __forceinline__ void proj_mul_acc2(float2 *acc, const float2 *v, const float *u,
                                              float2 sc = make_float2(1.f, 1.f)) {
  constexpr int SG = (FWD != DAG) ? 1 : -1;  // projector (1 - SG g_mu)
  using A = ProjA<MU>;
  using Ad = ProjAd<MU>;
  C2 h[2][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const C2 vu0{v[0 * 6 + 2 * c], v[0 * 6 + 2 * c + 1]};
    const C2 vu1{v[1 * 6 + 2 * c], v[1 * 6 + 2 * c + 1]};
    const C2 vl[2] = {{v[2 * 6 + 2 * c], v[2 * 6 + 2 * c + 1]},
                      {v[3 * 6 + 2 * c], v[3 * 6 + 2 * c + 1]}};
    h[0][c] = add_phase<A::p0, -SG>(vu0, vl[A::s0]);
    h[1][c] = add_phase<A::p1, -SG>(vu1, vl[A::s1]);
  }
  C2 w[2][3];
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float2 re = make_float2(0.f, 0.f), im = make_float2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        // forward: U[a][b]; backward: conj(U[b][a])
        const float ur = FWD ? u[2 * (3 * a + b)] : u[2 * (3 * b + a)];
        const float ui = FWD ? u[2 * (3 * a + b) + 1] : -u[2 * (3 * b + a) + 1];
        re = __ffma2_rn(bc(ur), h[sp][b].re, re);
        re = __ffma2_rn(bc(-ui), h[sp][b].im, re);
        im = __ffma2_rn(bc(ur), h[sp][b].im, im);
        im = __ffma2_rn(bc(ui), h[sp][b].re, im);
      }
      w[sp][a] = {re, im};
    }
  }
  const float2 scn = make_float2(-sc.x, -sc.y);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (SCALED) {
      acc[0 * 6 + 2 * c] = fma_s(acc[0 * 6 + 2 * c], w[0][c].re, sc);
      acc[0 * 6 + 2 * c + 1] = fma_s(acc[0 * 6 + 2 * c + 1], w[0][c].im, sc);
      acc[1 * 6 + 2 * c] = fma_s(acc[1 * 6 + 2 * c], w[1][c].re, sc);
      acc[1 * 6 + 2 * c + 1] = fma_s(acc[1 * 6 + 2 * c + 1], w[1][c].im, sc);
    } else {
      acc[0 * 6 + 2 * c] = __fadd2_rn(acc[0 * 6 + 2 * c], w[0][c].re);
      acc[0 * 6 + 2 * c + 1] = __fadd2_rn(acc[0 * 6 + 2 * c + 1], w[0][c].im);
      acc[1 * 6 + 2 * c] = __fadd2_rn(acc[1 * 6 + 2 * c], w[1][c].re);
      acc[1 * 6 + 2 * c + 1] = __fadd2_rn(acc[1 * 6 + 2 * c + 1], w[1][c].im);
    }
    const C2 l0{acc[2 * 6 + 2 * c], acc[2 * 6 + 2 * c + 1]};
    const C2 l1{acc[3 * 6 + 2 * c], acc[3 * 6 + 2 * c + 1]};
    C2 n0, n1;
    if constexpr (SCALED) {
      n0 = add_phase_s<Ad::p0, -SG>(l0, w[Ad::s0][c], sc, scn);
      n1 = add_phase_s<Ad::p1, -SG>(l1, w[Ad::s1][c], sc, scn);
    } else {
      n0 = add_phase<Ad::p0, -SG>(l0, w[Ad::s0][c]);
      n1 = add_phase<Ad::p1, -SG>(l1, w[Ad::s1][c]);
    }
    acc[2 * 6 + 2 * c] = n0.re;
    acc[2 * 6 + 2 * c + 1] = n0.im;
    acc[3 * 6 + 2 * c] = n1.re;
    acc[3 * 6 + 2 * c + 1] = n1.im;
  }
}

// Lanes of one site: the np = Ls/2 thread pairs of a site are consecutive lanes
// of one warp (sites never straddle a warp), so slice s0 - 1 is the second
// slice of lane - 1 (of lane + np - 1 for s0 = 0) and slice s0 + 2 the first
// slice of lane + 1 (of lane - np + 1 for the last pair).
struct PairLanes {
  int up, dn;       // source lanes of slices s0 - 1 and s0 + 2
  float fm, fp;     // their wrap factors (-m_f across the Ls boundary, else 1)
};

template <class S, int MU, bool FWD, bool DAG, bool PRE, bool RC>
__device__ __forceinline__ void hop_dir2(float2 *acc, const char *in, long long soff, int cs,
                                         int j, bool valid, int s0, int Ls, const uint4 *lk,
                                         size_t ls, const LsCoef &cf, const PairLanes &pl) {
  float2 v[24];
  constexpr bool kFold = !PRE && !std::is_same<S, F32>::value;  // scales folded into the FMAs
  float2 sc = make_float2(1.f, 1.f);
  {
    float v0[24], v1[24];
    if (valid) {
      if constexpr (kFold)
        load24x2_unscaled<S>(in, soff, cs, j * Ls + s0, v0, v1, sc);
      else
        load24x2<S>(in, soff, cs, j * Ls + s0, v0, v1);
    } else {
#pragma unroll
      for (int k = 0; k < 24; ++k) v0[k] = v1[k] = 0.f;
    }
    if constexpr (PRE) {
      // M_phi on both slices as packed FMAs: (chi(s0), chi(s0+1)) =
      // b (v(s0), v(s0+1)) + c (shifted neighbours); the outer halves come
      // from the neighbouring lanes of the same site (all lanes take part)
      const float2 b2 = bc(cf.f.pre_b), c2 = bc(cf.f.pre_c);
#pragma unroll
      for (int k = 0; k < 12; ++k) {  // upper: chi(s0) <- s0-1, chi(s0+1) <- s0
        const float w = __shfl_sync(0xffffffffu, v1[k], pl.up);
        v[k] = __ffma2_rn(c2, make_float2(pl.fm * w, v0[k]),
                          __fmul2_rn(b2, make_float2(v0[k], v1[k])));
      }
#pragma unroll
      for (int k = 0; k < 12; ++k) {  // lower: chi(s0) <- s0+1, chi(s0+1) <- s0+2
        const float w = __shfl_sync(0xffffffffu, v0[12 + k], pl.dn);
        v[12 + k] = __ffma2_rn(c2, make_float2(v1[12 + k], pl.fp * w),
                               __fmul2_rn(b2, make_float2(v0[12 + k], v1[12 + k])));
      }
    } else {
#pragma unroll
      for (int k = 0; k < 24; ++k) v[k] = make_float2(v0[k], v1[k]);
    }
  }
  if (valid) {
    float u[18];
    load_link<S>(lk, ls, u, RC ? 1 : 0);
    proj_mul_acc2<MU, FWD, DAG, kFold>(acc, v, u, sc);
  }
}

template <class S, int MU, bool DAG, bool PRE, bool RC>
__device__ __forceinline__ void hop_mu2(float2 *acc, const HopParams &P, const char *in,
                                        const uint4 *links, const int *nb, bool active, int site,
                                        int s0, const LsCoef &cf, const PairLanes &pl) {
  constexpr int LC = RC ? S::kLinkChunksRecon : S::kLinkChunks;
  const int jf = active ? nb[2 * MU] : -1, jb = active ? nb[2 * MU + 1] : -1;
  const size_t ls = (size_t)P.link_cs;
  const uint4 *lmu = links + (size_t)MU * LC * ls;
  const bool vf = jf >= 0 && jf < P.in_limit, vb = jb >= 0 && jb < P.in_limit;
  if constexpr (PRE) {
    // every lane of the warp takes part (the M_phi halves are exchanged
    // between lanes); a direction no lane of the warp has is skipped by all
    if (__any_sync(0xffffffffu, vf))
      hop_dir2<S, MU, true, DAG, PRE, RC>(acc, in, P.in.scale_off, P.in.cs, jf, vf, s0, P.Ls,
                                      lmu + P.out_link_off + site, ls, cf, pl);
    if (__any_sync(0xffffffffu, vb))
      hop_dir2<S, MU, false, DAG, PRE, RC>(acc, in, P.in.scale_off, P.in.cs, jb, vb, s0, P.Ls,
                                       lmu + P.in_link_off + jb, ls, cf, pl);
  } else {
    // no exchange between lanes: each lane branches on its own neighbours
    if (vf)
      hop_dir2<S, MU, true, DAG, PRE, RC>(acc, in, P.in.scale_off, P.in.cs, jf, true, s0, P.Ls,
                                      lmu + P.out_link_off + site, ls, cf, pl);
    if (vb)
      hop_dir2<S, MU, false, DAG, PRE, RC>(acc, in, P.in.scale_off, P.in.cs, jb, true, s0, P.Ls,
                                       lmu + P.in_link_off + jb, ls, cf, pl);
  }
}

// The x-term of the Ls epilogue, out += (a0 + a1 S) x, on the thread's slices
// s0 and s0 + 1 (o0, o1), added after the column walk. S is the walk's chiral
// shift: (S x)_s = x_{s-1} with (S x)_0 = -mf x_{Ls-1} on the components the
// walk runs down (the upper spin components of the operator, the lower ones
// of its adjoint), (S x)_s = x_{s+1} with (S x)_{Ls-1} = -mf x_0 on the
// others. Besides the pair it needs the down half of x at s0 - 1 and the up
// half at s0 + 2.
// Every lane of the warp calls this (the halves of slices s0 - 1 and s0 + 2
// come from the neighbouring lanes); `have` is false where x is zero.
template <class S, bool DAG>
__device__ __forceinline__ void add_x_term2(float *o0, float *o1, const char *x, long long soff,
                                            int cs, int site, int s0, int Ls, bool have,
                                            const LsK<float> &c, const PairLanes &pl) {
  float x0[12], x1[12], w[12];
  const int e = site * Ls + s0;
  const float a0 = c.a0, a1 = c.a1;
  const float fm = pl.fm, fp = pl.fp;
  // upper components: down for the operator, up for its adjoint
  if (have) {
    load12x2<S, true>(x, soff, cs, e, x0, x1);
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) x0[k] = x1[k] = 0.f;
  }
#pragma unroll
  for (int k = 0; k < 12; ++k)
    w[k] = DAG ? __shfl_sync(0xffffffffu, x0[k], pl.dn) : __shfl_sync(0xffffffffu, x1[k], pl.up);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    if (!DAG) {
      o0[k] += a0 * x0[k] + a1 * (fm * w[k]);
      o1[k] += a0 * x1[k] + a1 * x0[k];
    } else {
      o0[k] += a0 * x0[k] + a1 * x1[k];
      o1[k] += a0 * x1[k] + a1 * (fp * w[k]);
    }
  }
  // lower components: up for the operator, down for its adjoint
  if (have) {
    load12x2<S, false>(x, soff, cs, e, x0, x1);
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) x0[k] = x1[k] = 0.f;
  }
#pragma unroll
  for (int k = 0; k < 12; ++k)
    w[k] = DAG ? __shfl_sync(0xffffffffu, x1[k], pl.up) : __shfl_sync(0xffffffffu, x0[k], pl.dn);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    if (!DAG) {
      o0[12 + k] += a0 * x0[k] + a1 * x1[k];
      o1[12 + k] += a0 * x1[k] + a1 * (fp * w[k]);
    } else {
      o0[12 + k] += a0 * x0[k] + a1 * (fm * w[k]);
      o1[12 + k] += a0 * x1[k] + a1 * x0[k];
    }
  }
}

// EPI: the Ls epilogue is compiled in (its column registers would otherwise
// weigh on the plain hop's register allocation).
template <class S, bool DAG, bool PRE, bool RC, bool EPI>
__device__ __forceinline__ void hop2_body(const HopParams &P) {
  __shared__ double red[32];
  const int rhs = blockIdx.z, blk = blockIdx.y;
  if (P.skip && P.skip[rhs]) return;
  if (P.bskip && P.bskip[rhs * P.nblocks + blk]) return;
  const int Ls = P.Ls, np = Ls >> 1;
  const int nsites = P.nsites;  // (blockDim.x / 32) * (32 / np): whole sites per warp
  const int tid = threadIdx.x, lane = tid & 31, spw = 32 / np;
  const int jp = lane % np, slw = lane / np;
  const int sl = (tid >> 5) * spw + slw;
  const int s0 = 2 * jp;
  const int site0 = blockIdx.x * nsites;
  const int site = site0 + sl;
  const bool active = (slw < spw) && (site < P.n_out);
  const LsCoef &cf = P.coef[rhs];
  PairLanes pl;
  pl.up = jp == 0 ? lane + np - 1 : lane - 1;
  pl.dn = jp == np - 1 ? lane - (np - 1) : lane + 1;
  pl.fm = jp == 0 ? -cf.f.mf : 1.f;
  pl.fp = jp == np - 1 ? -cf.f.mf : 1.f;

  const char *in = P.in.data + blk * P.in.bstride + rhs * P.in.rstride;
  char *out = P.out.data + blk * P.out.bstride + rhs * P.out.rstride;
  const uint4 *links = reinterpret_cast<const uint4 *>(P.links + blk * P.link_bstride);

  float2 acc[24];
#pragma unroll
  for (int k = 0; k < 24; ++k) acc[k] = make_float2(0.f, 0.f);
  {
    // every lane runs the direction loop (the M_phi halves are exchanged
    // between lanes); inactive lanes load and add nothing
    const int *nb = P.nbr + (size_t)(active ? site : 0) * 8;
    hop_mu2<S, 0, DAG, PRE, RC>(acc, P, in, links, nb, active, site, s0, cf, pl);
    hop_mu2<S, 1, DAG, PRE, RC>(acc, P, in, links, nb, active, site, s0, cf, pl);
    hop_mu2<S, 2, DAG, PRE, RC>(acc, P, in, links, nb, active, site, s0, cf, pl);
    hop_mu2<S, 3, DAG, PRE, RC>(acc, P, in, links, nb, active, site, s0, cf, pl);
  }
  const int e = site * Ls + s0;
  float a0[24], a1[24];
#pragma unroll
  for (int k = 0; k < 24; ++k) {
    a0[k] = acc[k].x;
    a1[k] = acc[k].y;
  }

  if constexpr (EPI) {
    if (P.inv) {
      // y = (1 - r S)^-1 v on the lanes of the site, as a scan (no shared
      // memory). On the components where S takes s - 1: the wrap-free
      // recursion yh_j = v_j + r yh_{j-1} (yh_0 = v_0) is a scan over the
      // site's lanes with the constant factor r^2 per lane; the wrap then adds
      // r^j d with d = -m_f r yh_{Ls-1} / (1 + m_f r^Ls) (the closed form's
      // first element). Where S takes s + 1 the same runs in reversed order.
      const LsK<float> &c = cf.f;
      const float r = c.r, mfr = -c.mf * c.r * c.inv_den;
      // r^(2 jp), r^(Ls - 2 - 2 jp) and r^(2 d) for the scan steps
      float r_lo = 1.f, r_rev = 1.f;
      for (int i = 0; i < 2 * jp; ++i) r_lo *= r;
      for (int i = 0; i < Ls - 2 - 2 * jp; ++i) r_rev *= r;
      const float r2 = r * r;
      const int base = lane - jp;
#pragma unroll
      for (int k = 0; k < 24; ++k) {
        const bool down = (k < 12) != DAG;
        // order the pair along the recursion: first, second
        const float f = down ? a0[k] : a1[k], g = down ? a1[k] : a0[k];
        const float w1 = g + r * f;
        float C = w1;  // inclusive scan of w1 with factor r^2 per lane step
        float m = r2;
        for (int d = 1; d < np; d <<= 1) {
          const float tu = __shfl_up_sync(0xffffffffu, C, d);
          const float td = __shfl_down_sync(0xffffffffu, C, d);
          if (down ? (jp >= d) : (jp + d < np)) C += m * (down ? tu : td);
          m *= m;
        }
        const float cu = __shfl_up_sync(0xffffffffu, C, 1);
        const float cd = __shfl_down_sync(0xffffffffu, C, 1);
        const float cin = down ? (jp > 0 ? cu : 0.f) : (jp + 1 < np ? cd : 0.f);
        const float last = __shfl_sync(0xffffffffu, C, down ? base + np - 1 : base);
        const float dl = mfr * last;
        // positions along the recursion: first at 2 jp (down) or Ls-2-2jp
        // counted from the other end (up), second one further
        const float rf = down ? r_lo : r_rev, rs = rf * r;
        const float yf = f + r * cin + rf * dl;
        const float ys = w1 + r2 * cin + rs * dl;
        a0[k] = down ? yf : ys;
        a1[k] = down ? ys : yf;
      }
    }
    {
      // q0 (p0 + p1 S) needs only the neighbouring slices: the pair's own and
      // the outer ones from the neighbouring lanes of the site
      const float p0 = cf.f.p0q, p1 = cf.f.p1q;
#pragma unroll
      for (int k = 0; k < 24; ++k) {
        const bool down = (k < 12) != DAG;  // S takes s - 1 on these components
        const float wu = __shfl_sync(0xffffffffu, a1[k], pl.up);
        const float wd = __shfl_sync(0xffffffffu, a0[k], pl.dn);
        const float t0 = a0[k], t1 = a1[k];
        if (down) {
          a0[k] = p0 * t0 + p1 * (pl.fm * wu);
          a1[k] = p0 * t1 + p1 * t0;
        } else {
          a0[k] = p0 * t0 + p1 * t1;
          a1[k] = p0 * t1 + p1 * (pl.fp * wd);
        }
      }
    }
    // the x-term, (a0 + a1 S) x, after the Ls operator, in registers; every
    // lane takes part in the exchange of the outer halves
    if (P.has_x) {
      const char *xo = P.xown.data + blk * P.xown.bstride + rhs * P.xown.rstride;
      add_x_term2<S, DAG>(a0, a1, xo, P.xown.scale_off, P.xown.cs, active ? site : 0, s0, Ls,
                          active && site < P.xown_limit, cf.f, pl);
    }
  } else {
    const float q = cf.f.q0;
#pragma unroll
    for (int k = 0; k < 24; ++k) {
      a0[k] *= q;
      a1[k] *= q;
    }
  }
  if (active) store24x2<S>(out, P.out.scale_off, P.out.cs, e, a0, a1);

  if (P.dot) {
    double d = 0.0;
    if (active) {
      float d0[24], d1[24];
      const char *dp = P.dotv.data + blk * P.dotv.bstride + rhs * P.dotv.rstride;
      load24x2<S>(dp, P.dotv.scale_off, P.dotv.cs, e, d0, d1);
      d = dot_compensated<float>(d0, a0, 24) + dot_compensated<float>(d1, a1, 24);
    }
    hop_dot(P, d, red, rhs, blk);
  }
}

template <class S, bool DAG, bool PRE, bool RC, bool EPI>
__global__ void __launch_bounds__(128, 4) hop2_kernel(const __grid_constant__ HopParams P) {
  prof_enter(P);
  hop2_body<S, DAG, PRE, RC, EPI>(P);
  prof_exit(P);
}

// Two slices per thread for FP32/FP16/BF16 with even Ls; one otherwise.
static bool hop_pairs(int Ls, dwf_prec p) { return p != DWF_FP64 && Ls % 2 == 0; }

int hop_sites_per_cta(int Ls, dwf_prec p) {
  int n;
  if (hop_pairs(Ls, p))
    n = 4 * (32 / (Ls / 2));  // four warps of whole sites
  else
    n = ((p == DWF_FP64) ? 128 : 256) / Ls;
  return n < 1 ? 1 : n;
}

size_t hop_smem_bytes(int Ls, dwf_prec p, int epi, int has_x) {
  // the two-slice kernel runs its Ls epilogue across the lanes of a site
  if (!epi || hop_pairs(Ls, p)) return 0;
  // the one-slice kernel walks the columns of T (and of x) in shared memory
  const size_t rs = (p == DWF_FP64) ? 8 : 4;
  return (size_t)hop_sites_per_cta(Ls, p) * 24 * (Ls + 1) * rs * (has_x ? 2 : 1);
}

template <class S, bool DAG, bool PRE, bool RC>
static void launch_t(const HopParams &P0, int nrhs, cudaStream_t st, dwf_prec prec) {
  HopParams P = P0;
  for (int r = 0; r < nrhs; ++r) finalize_coef(P.coef[r]);
  const int nsites = hop_sites_per_cta(P.Ls, prec);
  P.nsites = nsites;
  dim3 grid((P.n_out + nsites - 1) / nsites, P.nblocks, nrhs);
  const size_t smem = hop_smem_bytes(P.Ls, prec, P.epi, P.has_x);
  if (grid.x == 0) return;
  if constexpr (!std::is_same<S, F64>::value) {
    if (hop_pairs(P.Ls, prec)) {
      dim3 block(128);
      if (P.epi) {
        hop2_kernel<S, DAG, PRE, RC, true><<<grid, block, smem, st>>>(P);
      } else {
        if constexpr (DAG)
          throw Error{DWF_ERR_UNSUPPORTED, "the adjoint hop always has its M_phi^+ epilogue"};
        else
          hop2_kernel<S, DAG, PRE, RC, false><<<grid, block, smem, st>>>(P);
      }
      DWF_CUDA_TRY(cudaGetLastError());
      return;
    }
  }
  dim3 block((nsites * P.Ls + 31) / 32 * 32);
  hop_kernel<S, DAG, PRE, RC><<<grid, block, smem, st>>>(P);
  DWF_CUDA_TRY(cudaGetLastError());
}

template <class S> static dwf_prec prec_of();
template <> dwf_prec prec_of<F64>() { return DWF_FP64; }
template <> dwf_prec prec_of<F32>() { return DWF_FP32; }
template <> dwf_prec prec_of<F16>() { return DWF_FP16; }
template <> dwf_prec prec_of<BF16>() { return DWF_BF16; }

template <class S>
void launch_hop(const HopParams &P, int dagger, int pre_mphi, int nrhs, cudaStream_t st) {
  DWF_REQUIRE(!(dagger && pre_mphi), DWF_ERR_UNSUPPORTED, "M_phi on load is for Dhop only");
  const dwf_prec p = prec_of<S>();
  if constexpr (!std::is_same<S, F64>::value) {
    if (P.recon) {
      if (dagger)
        launch_t<S, true, false, true>(P, nrhs, st, p);
      else if (pre_mphi)
        launch_t<S, false, true, true>(P, nrhs, st, p);
      else
        launch_t<S, false, false, true>(P, nrhs, st, p);
      return;
    }
  }
  DWF_REQUIRE(!P.recon, DWF_ERR_UNSUPPORTED, "FP64 links are never reconstructed");
  if (dagger)
    launch_t<S, true, false, false>(P, nrhs, st, p);
  else if (pre_mphi)
    launch_t<S, false, true, false>(P, nrhs, st, p);
  else
    launch_t<S, false, false, false>(P, nrhs, st, p);
}

// Allow the one-slice hop kernels more than 48 KB of dynamic shared memory
// (the two-slice kernels use none). Called once per device before any launch
// (and so before any stream capture).
template <class K>
static void allow_big_smem(K *kernel) {
  DWF_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    200 * 1024));
}
template <class S>
static void prepare_one() {
  allow_big_smem(hop_kernel<S, false, false, false>);
  allow_big_smem(hop_kernel<S, false, true, false>);
  allow_big_smem(hop_kernel<S, true, false, false>);
  if constexpr (!std::is_same<S, F64>::value) {
    allow_big_smem(hop_kernel<S, false, false, true>);
    allow_big_smem(hop_kernel<S, false, true, true>);
    allow_big_smem(hop_kernel<S, true, false, true>);
  }
}
void prepare_kernels() {
  prepare_one<F64>();
  prepare_one<F32>();
  prepare_one<F16>();
  prepare_one<BF16>();
}

template void launch_hop<F64>(const HopParams &, int, int, int, cudaStream_t);
template void launch_hop<F32>(const HopParams &, int, int, int, cudaStream_t);
template void launch_hop<F16>(const HopParams &, int, int, int, cudaStream_t);
template void launch_hop<BF16>(const HopParams &, int, int, int, cudaStream_t);

}  // namespace dwf

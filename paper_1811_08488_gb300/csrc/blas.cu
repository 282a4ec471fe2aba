// Vector updates and reductions of the outer preconditioned CG (Algorithm 1)
// and of the block-local inner CG (Sec. 2.4: k fixed CG iterations per block,
// block-local scalars, zero initial guess).
//
// Reductions accumulate in FP64, one partial per CTA; the last CTA of a group
// sums the partials in a fixed order, so results are bitwise reproducible. The
// scalars alpha and beta are formed on the device from those sums.
#include <type_traits>

#include "blas.cuh"
#include "device_common.cuh"
#include "vec4.cuh"

namespace dwf {

constexpr int kOuterCtas = 152 * 4;
constexpr int kBlasThreads = 256;
int outer_ctas() { return kOuterCtas; }

// num / den (0 when den == 0), computed in FP64 by one thread of the CTA and
// shared: FP64 division per thread would run on GB300's small FP64 pipe.
template <class R>
__device__ __forceinline__ R cta_ratio(double num, double den, double *out_d = nullptr) {
  __shared__ double s_ratio;
  if (threadIdx.x == 0) s_ratio = den != 0.0 ? num / den : 0.0;
  __syncthreads();
  if (out_d) *out_d = s_ratio;
  return (R)s_ratio;
}

// ---------------------------------------------------------------------------
// Outer solve
// ---------------------------------------------------------------------------
// r64 = b; rlo = b; |b|^2 -> bb and rr (and rz for plain CG); iter = 0.
template <class SL>
__global__ void __launch_bounds__(kBlasThreads) init_kernel(const OuterArgs A) {
  __shared__ double red[32];
  const int rhs = blockIdx.y;
  if (A.skip && A.skip[rhs]) return;
  const long long o64 = rhs * A.rs64, olo = rhs * A.rslo;
  double acc = 0.0;
  FLAT_LOOP(A.n4) {
    double v[4];
    ld4<F64>(A.b64 + o64, i, A.cs, v);
    st4<F64>(A.r64 + o64, i, A.cs, v);
    st4<SL>(A.rlo + olo, i, A.cs, v);
    acc += sq4(v);
  }
  acc = cta_sum(acc, red);
  double tot;
  if (group_reduce(acc, A.partials + (size_t)rhs * gridDim.x, gridDim.x, blockIdx.x,
                   A.counters + rhs, tot)) {
    OuterScalars *sc = A.scal + rhs;
    sc->bb = tot;
    sc->rr = tot;
    if (A.plain) sc->rz = tot;
    sc->iter = 0;
  }
}

// x += alpha p; r -= alpha Ap; |r|^2 with alpha = <r,z> / <p,Ap> (Algorithm 1).
template <class SL>
__global__ void __launch_bounds__(kBlasThreads) axpy_xr_kernel(const OuterArgs A) {
  using R = typename Acc<SL>::R;
  __shared__ double red[32];
  const int rhs = blockIdx.y;
  if (A.skip && A.skip[rhs]) return;
  OuterScalars *sc = A.scal + rhs;
  double alpha_d;
  const R alpha = cta_ratio<R>(sc->rz, sc->pAp, &alpha_d);
  const long long o = rhs * A.rslo;
  typename Acc<SL>::T acc;
  FLAT_LOOP(A.n4) {
    R x[4], r[4], p[4], q[4];
    ld4<SL>(A.xlo + o, i, A.cs, x);
    ld4<SL>(A.rlo + o, i, A.cs, r);
    ld4<SL>(A.p + o, i, A.cs, p);
    ld4<SL>(A.Ap + o, i, A.cs, q);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      x[k] += alpha * p[k];
      r[k] -= alpha * q[k];
    }
    st4<SL>(A.xlo + o, i, A.cs, x);
    st4<SL>(A.rlo + o, i, A.cs, r);
    acc.add(sq4(r));
  }
  const double a = cta_sum(acc.value(), red);
  double tot;
  if (group_reduce(a, A.partials + (size_t)rhs * gridDim.x, gridDim.x, blockIdx.x,
                   A.counters + rhs, tot)) {
    sc->rr = tot;
    sc->alpha = alpha_d;
    sc->hist_rr[sc->iter % kHistory] = tot;
    if (A.plain) sc->rz_new = tot;
  }
}

// beta = <r',z'> / <r,z>; p = z + beta p (z = r for plain CG); iter++.
template <class SL>
__global__ void __launch_bounds__(kBlasThreads) xpay_p_kernel(const OuterArgs A) {
  using R = typename Acc<SL>::R;
  const int rhs = blockIdx.y;
  if (A.skip && A.skip[rhs]) return;
  OuterScalars *sc = A.scal + rhs;
  const double rzn = sc->rz_new;
  double beta_d;
  // Fletcher-Reeves (Algorithm 1): <r', z'> / <r, z>; flexible (Polak-Ribiere):
  // <r' - r, z'> / <r, z> = -alpha <A p, z'> / <r, z>
  const R beta = cta_ratio<R>(A.flexible ? -sc->alpha * sc->apz : rzn, sc->rz, &beta_d);
  const long long o = rhs * A.rslo;
  const char *z = A.plain ? A.rlo : A.z;
  FLAT_LOOP(A.n4) {
    R p[4], zz[4];
    ld4<SL>(A.p + o, i, A.cs, p);
    ld4<SL>(z + o, i, A.cs, zz);
#pragma unroll
    for (int k = 0; k < 4; ++k) p[k] = zz[k] + beta * p[k];
    st4<SL>(A.p + o, i, A.cs, p);
  }
  double tot;
  if (group_reduce(0.0, A.partials + (size_t)rhs * gridDim.x, gridDim.x, blockIdx.x,
                   A.counters + rhs, tot)) {
    sc->rz = rzn;
    sc->beta = beta_d;
    sc->iter += 1;
  }
}

// p = z (or r for plain CG).
template <class SL>
__global__ void __launch_bounds__(kBlasThreads) copy_p_kernel(const OuterArgs A) {
  using R = typename Acc<SL>::R;
  const int rhs = blockIdx.y;
  if (A.skip && A.skip[rhs]) return;
  const long long o = rhs * A.rslo;
  const char *z = A.plain ? A.rlo : A.z;
  FLAT_LOOP(A.n4) {
    R v[4];
    ld4<SL>(z + o, i, A.cs, v);
    st4<SL>(A.p + o, i, A.cs, v);
  }
}

// x64 += xlo; xlo = 0 (the FP64 accumulation of a reliable update).
template <class SL>
__global__ void __launch_bounds__(kBlasThreads) promote_kernel(const OuterArgs A) {
  const int rhs = blockIdx.y;
  if (A.skip && A.skip[rhs]) return;
  const long long o64 = rhs * A.rs64, olo = rhs * A.rslo;
  FLAT_LOOP(A.n4) {
    double x[4], d[4];
    ld4<F64>(A.x64 + o64, i, A.cs, x);
    ld4<SL>(A.xlo + olo, i, A.cs, d);
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] += d[k];
    st4<F64>(A.x64 + o64, i, A.cs, x);
    const double z[4] = {0, 0, 0, 0};
    st4<SL>(A.xlo + olo, i, A.cs, z);
  }
}

// r64 = b - A x64 (FP64); rlo = r64; |r64|^2 -> rr (and rz for plain CG).
template <class SL>
__global__ void __launch_bounds__(kBlasThreads) ru_residual_kernel(const OuterArgs A) {
  __shared__ double red[32];
  const int rhs = blockIdx.y;
  if (A.skip && A.skip[rhs]) return;
  const long long o64 = rhs * A.rs64, olo = rhs * A.rslo;
  double acc = 0.0;
  FLAT_LOOP(A.n4) {
    double b[4], ax[4];
    ld4<F64>(A.b64 + o64, i, A.cs, b);
    ld4<F64>(A.Ax64 + o64, i, A.cs, ax);
#pragma unroll
    for (int k = 0; k < 4; ++k) b[k] -= ax[k];
    st4<F64>(A.r64 + o64, i, A.cs, b);
    st4<SL>(A.rlo + olo, i, A.cs, b);
    acc += sq4(b);
  }
  acc = cta_sum(acc, red);
  double tot;
  if (group_reduce(acc, A.partials + (size_t)rhs * gridDim.x, gridDim.x, blockIdx.x,
                   A.counters + rhs, tot)) {
    OuterScalars *sc = A.scal + rhs;
    sc->rr = tot;
    if (A.plain) sc->rz = tot;
  }
}

__global__ void set_rz_kernel(OuterScalars *scal, const int *skip, int nrhs) {
  const int r = threadIdx.x;
  if (r < nrhs && !(skip && skip[r])) scal[r].rz = scal[r].rz_new;
}

// ---------------------------------------------------------------------------
// Device-driven loop of the outer solve: one thread decides, after every outer
// iteration, which right-hand sides take a reliable update and whether the
// graph's loop goes on; the decisions are the host loop's (the same tests on
// the same FP64 scalars), taken without a host round trip.
// ---------------------------------------------------------------------------
// Before the first iteration: |r| = |b|; a zero source is solved by x = 0.
__global__ void solve_start_kernel(OuterScalars *scal, SolveCtl *ctl, int *skip_iter,
                                   SolveCtl init) {
  if (threadIdx.x != 0) return;
  *ctl = init;
  for (int r = 0; r < init.nrhs; ++r) {
    OuterScalars &s = scal[r];
    s.maxr = sqrt(s.rr);
    s.done = s.bb == 0.0 ? 1 : 0;
    s.final_res = s.done ? 0.0 : -1.0;
    s.nru = 0;
    skip_iter[r] = s.done;
  }
}

// At the start of every graph launch.
__global__ void solve_launch_kernel(SolveCtl *ctl) {
  if (threadIdx.x == 0) {
    ctl->launch_iters = 0;
  }
}

// After an outer iteration: a right-hand side takes a reliable update when its
// iterated |r|^2 reached tol^2 |b|^2 (convergence candidate) or |r| fell below
// delta times its largest value since the last update.
__global__ void solve_control_kernel(OuterScalars *scal, SolveCtl *ctl, int *skip_ru,
                                     cudaGraphConditionalHandle h_loop,
                                     cudaGraphConditionalHandle h_ru) {
  if (threadIdx.x != 0) return;
  int any_ru = 0, iter_max = 0;
  for (int r = 0; r < ctl->nrhs; ++r) {
    OuterScalars &s = scal[r];
    skip_ru[r] = 1;
    if (s.done) continue;
    const double rr = s.rr;
    if (!isfinite(rr)) {
      ctl->nan = 1;
      continue;
    }
    const double nr = sqrt(rr);
    const bool need = rr <= ctl->tol2 * s.bb || nr < ctl->delta * s.maxr;
    s.maxr = fmax(s.maxr, nr);
    if (need) {
      skip_ru[r] = 0;
      any_ru = 1;
    }
    iter_max = max(iter_max, s.iter);
  }
  ctl->launch_iters += 1;
  const bool stop = ctl->nan || ctl->launch_iters >= ctl->budget || iter_max >= ctl->maxiter;
  cudaGraphSetConditional(h_ru, (any_ru && !ctl->nan) ? 1u : 0u);
  cudaGraphSetConditional(h_loop, stop ? 0u : 1u);
}

// After a reliable update: the recomputed FP64 |b - A x|^2 is in rr; a right-
// hand side whose true residual meets tol is done and skipped from now on.
__global__ void solve_post_ru_kernel(OuterScalars *scal, SolveCtl *ctl, const int *skip_ru,
                                     int *skip_iter, cudaGraphConditionalHandle h_loop) {
  if (threadIdx.x != 0) return;
  int open = 0;
  for (int r = 0; r < ctl->nrhs; ++r) {
    OuterScalars &s = scal[r];
    if (!s.done && !skip_ru[r]) {
      s.nru += 1;
      const double rr = s.rr;
      if (!isfinite(rr)) ctl->nan = 1;
      s.maxr = sqrt(rr);
      if (rr <= ctl->tol2 * s.bb) {
        s.done = 1;
        skip_iter[r] = 1;
        s.final_res = sqrt(rr / s.bb);
      }
    }
    open += !s.done;
  }
  if (open == 0 || ctl->nan) cudaGraphSetConditional(h_loop, 0u);
}

void solve_start(OuterScalars *scal, SolveCtl *ctl, int *skip_iter, const SolveCtl &init,
                 cudaStream_t st) {
  solve_start_kernel<<<1, 32, 0, st>>>(scal, ctl, skip_iter, init);
  DWF_CUDA_TRY(cudaGetLastError());
}
void solve_launch(SolveCtl *ctl, cudaStream_t st) {
  solve_launch_kernel<<<1, 32, 0, st>>>(ctl);
  DWF_CUDA_TRY(cudaGetLastError());
}
void solve_control(OuterScalars *scal, SolveCtl *ctl, int *skip_ru,
                   cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_ru,
                   cudaStream_t st) {
  solve_control_kernel<<<1, 32, 0, st>>>(scal, ctl, skip_ru, h_loop, h_ru);
  DWF_CUDA_TRY(cudaGetLastError());
}
void solve_post_ru(OuterScalars *scal, SolveCtl *ctl, const int *skip_ru, int *skip_iter,
                   cudaGraphConditionalHandle h_loop, cudaStream_t st) {
  solve_post_ru_kernel<<<1, 32, 0, st>>>(scal, ctl, skip_ru, skip_iter, h_loop);
  DWF_CUDA_TRY(cudaGetLastError());
}

#define DISPATCH_LO(lo, KERNEL, ...)                                        \
  do {                                                                      \
    dim3 g(kOuterCtas, nrhs);                                               \
    if ((lo) == DWF_FP64)                                                   \
      KERNEL<F64><<<g, kBlasThreads, 0, st>>>(__VA_ARGS__);                 \
    else                                                                    \
      KERNEL<F32><<<g, kBlasThreads, 0, st>>>(__VA_ARGS__);                 \
    DWF_CUDA_TRY(cudaGetLastError());                                       \
  } while (0)

void outer_init(dwf_prec lo, const OuterArgs &A, int nrhs, cudaStream_t st) {
  DISPATCH_LO(lo, init_kernel, A);
}
void outer_axpy_xr(dwf_prec lo, const OuterArgs &A, int nrhs, cudaStream_t st) {
  DISPATCH_LO(lo, axpy_xr_kernel, A);
}
void outer_xpay_p(dwf_prec lo, const OuterArgs &A, int nrhs, cudaStream_t st) {
  DISPATCH_LO(lo, xpay_p_kernel, A);
}
void outer_copy_p(dwf_prec lo, const OuterArgs &A, int nrhs, cudaStream_t st) {
  DISPATCH_LO(lo, copy_p_kernel, A);
}
void outer_promote(dwf_prec lo, const OuterArgs &A, int nrhs, cudaStream_t st) {
  DISPATCH_LO(lo, promote_kernel, A);
}
void outer_ru_residual(dwf_prec lo, const OuterArgs &A, int nrhs, cudaStream_t st) {
  DISPATCH_LO(lo, ru_residual_kernel, A);
}
void outer_set_rz(const OuterArgs &A, int nrhs, cudaStream_t st) {
  set_rz_kernel<<<1, 32, 0, st>>>(A.scal, A.skip, nrhs);
  DWF_CUDA_TRY(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Inner block CG. Thread (i, s) of block b; grid (tiles, nblocks, nrhs).
// ---------------------------------------------------------------------------
int block_tiles(int n_b, int Ls) {
  return (int)(((long long)n_b * Ls + kBlasThreads - 1) / kBlasThreads);
}

// The global (outer) fields as floats: FP32 directly, FP64 converted.
template <class G>
__device__ __forceinline__ void load_glob(const char *base, int cs, int e, float *v) {
  if constexpr (std::is_same<G, F32>::value) {
    load24<F32>(base, 0, cs, e, v);
  } else {
    double t[24];
    load24<F64>(base, 0, cs, e, t);
#pragma unroll
    for (int k = 0; k < 24; ++k) v[k] = (float)t[k];
  }
}
template <class G>
__device__ __forceinline__ void store_glob(char *base, int cs, int e, const float *v) {
  if constexpr (std::is_same<G, F32>::value) {
    store24<F32>(base, 0, cs, e, v);
  } else {
    double t[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) t[k] = (double)v[k];
    store24<F64>(base, 0, cs, e, t);
  }
}

template <class SI, class G>
__global__ void __launch_bounds__(kBlasThreads) blk_gather_kernel(const BlockArgs B) {
  __shared__ double red[32];
  const int rhs = blockIdx.z, b = blockIdx.y;
  if (B.skip && B.skip[rhs]) return;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int i = (int)(idx / B.Ls), s = (int)(idx % B.Ls);
  double acc = 0.0;
  if (i < B.n_b) {
    const int h = B.gmap[(size_t)b * B.n_b + i];
    float v[24];
    load_glob<G>(B.rglob + rhs * B.grs, B.gcs, h * B.Ls + s, v);
    float part = 0.f;
#pragma unroll
    for (int k = 0; k < 24; ++k) part += v[k] * v[k];
    acc = part;
    const long long off = rhs * B.r.rstride + b * B.r.bstride;
    store24<SI>(B.r.data + off, B.r.scale_off, B.r.cs, i * B.Ls + s, v);
    store24<SI>(B.p.data + rhs * B.p.rstride + b * B.p.bstride, B.p.scale_off, B.p.cs, i * B.Ls + s,
                v);
    float zero[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) zero[k] = 0.f;
    store24<F32>(B.x.data + rhs * B.x.rstride + b * B.x.bstride, 0, B.x.cs, i * B.Ls + s, zero);
  }
  acc = cta_sum(acc, red);
  const int grp = rhs * B.nblocks + b;
  double tot;
  if (group_reduce(acc, B.partials + (size_t)grp * gridDim.x, gridDim.x, blockIdx.x,
                   B.counters + grp, tot)) {
    B.rr[grp] = tot;
    if (B.bstop) {
      B.rr0[grp] = tot;
      B.bstop[grp] = tot == 0.0 ? 1 : 0;
    }
  }
}

// alpha_b = rr_b / pAp_b; x += alpha p; unless LAST: r -= alpha Ap, |r|^2 -> rr_new.
template <class SI, bool LAST>
__global__ void __launch_bounds__(kBlasThreads) blk_xr_kernel(const BlockArgs B) {
  __shared__ double red[32];
  const int rhs = blockIdx.z, b = blockIdx.y;
  if (B.skip && B.skip[rhs]) return;
  const int grp = rhs * B.nblocks + b;
  if (B.bstop && B.bstop[grp]) return;  // this block's residual already met the stop
  if (B.iters && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(B.iters + rhs, 1u);
  const float alpha = cta_ratio<float>(B.rr[grp], B.pAp[grp]);
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int i = (int)(idx / B.Ls), s = (int)(idx % B.Ls);
  double acc = 0.0;
  if (i < B.n_b) {
    float x[24], p[24];
    char *xb = B.x.data + rhs * B.x.rstride + b * B.x.bstride;
    load24<F32>(xb, 0, B.x.cs, i * B.Ls + s, x);
    load24<SI>(B.p.data + rhs * B.p.rstride + b * B.p.bstride, B.p.scale_off, B.p.cs, i * B.Ls + s,
               p);
#pragma unroll
    for (int k = 0; k < 24; ++k) x[k] += alpha * p[k];
    store24<F32>(xb, 0, B.x.cs, i * B.Ls + s, x);
    if (!LAST) {
      float r[24], q[24];
      char *rb = B.r.data + rhs * B.r.rstride + b * B.r.bstride;
      load24<SI>(rb, B.r.scale_off, B.r.cs, i * B.Ls + s, r);
      load24<SI>(B.Ap.data + rhs * B.Ap.rstride + b * B.Ap.bstride, B.Ap.scale_off, B.Ap.cs,
                 i * B.Ls + s, q);
      float part = 0.f;
#pragma unroll
      for (int k = 0; k < 24; ++k) {
        r[k] -= alpha * q[k];
        part += r[k] * r[k];
      }
      acc = part;
      store24<SI>(rb, B.r.scale_off, B.r.cs, i * B.Ls + s, r);
    }
  }
  if (!LAST) {
    acc = cta_sum(acc, red);
    double tot;
    if (group_reduce(acc, B.partials + (size_t)grp * gridDim.x, gridDim.x, blockIdx.x,
                     B.counters + grp, tot)) {
      B.rr_new[grp] = tot;
      // every CTA of the group has passed the check at entry: the flag
      // takes effect from the next kernel on
      if (B.bstop && tot <= B.tol2 * B.rr0[grp]) B.bstop[grp] = 1;
    }
  }
}

// beta_b = rr_new_b / rr_b; p = r + beta p; then rr_b = rr_new_b.
template <class SI>
__global__ void __launch_bounds__(kBlasThreads) blk_p_kernel(const BlockArgs B) {
  const int rhs = blockIdx.z, b = blockIdx.y;
  if (B.skip && B.skip[rhs]) return;
  const int grp = rhs * B.nblocks + b;
  if (B.bstop && B.bstop[grp]) return;
  const float beta = cta_ratio<float>(B.rr_new[grp], B.rr[grp]);
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int i = (int)(idx / B.Ls), s = (int)(idx % B.Ls);
  if (i < B.n_b) {
    float r[24], p[24];
    char *pb = B.p.data + rhs * B.p.rstride + b * B.p.bstride;
    load24<SI>(B.r.data + rhs * B.r.rstride + b * B.r.bstride, B.r.scale_off, B.r.cs, i * B.Ls + s,
               r);
    load24<SI>(pb, B.p.scale_off, B.p.cs, i * B.Ls + s, p);
#pragma unroll
    for (int k = 0; k < 24; ++k) p[k] = r[k] + beta * p[k];
    store24<SI>(pb, B.p.scale_off, B.p.cs, i * B.Ls + s, p);
  }
  double tot;
  if (group_reduce(0.0, B.partials + (size_t)grp * gridDim.x, gridDim.x, blockIdx.x,
                   B.counters + grp, tot))
    B.rr[grp] = B.rr_new[grp];
}

// z_glob = x (block layout -> global), with <r, z> summed over all blocks.
template <class G>
__global__ void __launch_bounds__(kBlasThreads) blk_scatter_kernel(const BlockArgs B) {
  __shared__ double red[32];
  const int rhs = blockIdx.z, b = blockIdx.y;
  if (B.skip && B.skip[rhs]) return;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int i = (int)(idx / B.Ls), s = (int)(idx % B.Ls);
  double acc = 0.0, acc2 = 0.0;
  if (i < B.n_b) {
    const int h = B.gmap[(size_t)b * B.n_b + i];
    float x[24], r[24];
    load24<F32>(B.x.data + rhs * B.x.rstride + b * B.x.bstride, 0, B.x.cs, i * B.Ls + s, x);
    load_glob<G>(B.rglob + rhs * B.grs, B.gcs, h * B.Ls + s, r);
    store_glob<G>(B.zglob + rhs * B.grs, B.gcs, h * B.Ls + s, x);
    float part = 0.f;
#pragma unroll
    for (int k = 0; k < 24; ++k) part += r[k] * x[k];
    acc = part;
    if (B.apglob) {
      load_glob<G>(B.apglob + rhs * B.grs, B.gcs, h * B.Ls + s, r);
      float part2 = 0.f;
#pragma unroll
      for (int k = 0; k < 24; ++k) part2 += r[k] * x[k];
      acc2 = part2;
    }
  }
  acc = cta_sum(acc, red);
  const int ntiles = gridDim.x * gridDim.y;
  const int tile = b * gridDim.x + blockIdx.x;
  double tot;
  if (group_reduce(acc, B.gpart + (size_t)rhs * ntiles, ntiles, tile, B.gcount + rhs, tot))
    B.rz_out[(size_t)rhs * B.rz_rstride] = tot;
  if (B.apglob) {
    __syncthreads();
    acc2 = cta_sum(acc2, red);
    if (group_reduce(acc2, B.gpart2 + (size_t)rhs * ntiles, ntiles, tile, B.gcount2 + rhs, tot))
      B.apz_out[(size_t)rhs * B.rz_rstride] = tot;
  }
}

// out_glob = src (block layout -> FP32 global), used to read block vectors out.
template <class SI>
__global__ void __launch_bounds__(kBlasThreads) blk_export_kernel(const BlockArgs B,
                                                                  const FieldRef src) {
  const int rhs = blockIdx.z, b = blockIdx.y;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int i = (int)(idx / B.Ls), s = (int)(idx % B.Ls);
  if (i < B.n_b) {
    const int h = B.gmap[(size_t)b * B.n_b + i];
    float v[24];
    load24<SI>(src.data + rhs * src.rstride + b * src.bstride, src.scale_off, src.cs,
               i * B.Ls + s, v);
    store24<F32>(B.zglob + rhs * B.grs, 0, B.gcs, h * B.Ls + s, v);
  }
}

void block_export(dwf_prec in, const BlockArgs &B, const FieldRef &src, int nrhs,
                  cudaStream_t st) {
  dim3 g(block_tiles(B.n_b, B.Ls), B.nblocks, nrhs);
  switch (in) {
    case DWF_FP32: blk_export_kernel<F32><<<g, kBlasThreads, 0, st>>>(B, src); break;
    case DWF_FP16: blk_export_kernel<F16><<<g, kBlasThreads, 0, st>>>(B, src); break;
    case DWF_BF16: blk_export_kernel<BF16><<<g, kBlasThreads, 0, st>>>(B, src); break;
    default: throw Error{DWF_ERR_UNSUPPORTED, "inner precision"};
  }
  DWF_CUDA_TRY(cudaGetLastError());
}

#define DISPATCH_IN(in, KERNEL, ...)                                         \
  do {                                                                       \
    switch (in) {                                                            \
      case DWF_FP32: KERNEL<F32 __VA_ARGS__><<<g, kBlasThreads, 0, st>>>(B); break; \
      case DWF_FP16: KERNEL<F16 __VA_ARGS__><<<g, kBlasThreads, 0, st>>>(B); break; \
      case DWF_BF16: KERNEL<BF16 __VA_ARGS__><<<g, kBlasThreads, 0, st>>>(B); break; \
      default: throw Error{DWF_ERR_UNSUPPORTED, "inner precision"};          \
    }                                                                        \
    DWF_CUDA_TRY(cudaGetLastError());                                        \
  } while (0)

void block_gather(dwf_prec in, const BlockArgs &B, int nrhs, cudaStream_t st) {
  dim3 g(block_tiles(B.n_b, B.Ls), B.nblocks, nrhs);
  if (B.gfp64)
    DISPATCH_IN(in, blk_gather_kernel, , F64);
  else
    DISPATCH_IN(in, blk_gather_kernel, , F32);
}
void block_xr(dwf_prec in, const BlockArgs &B, int last, int nrhs, cudaStream_t st) {
  dim3 g(block_tiles(B.n_b, B.Ls), B.nblocks, nrhs);
  if (last)
    DISPATCH_IN(in, blk_xr_kernel, , true);
  else
    DISPATCH_IN(in, blk_xr_kernel, , false);
}
void block_p(dwf_prec in, const BlockArgs &B, int nrhs, cudaStream_t st) {
  dim3 g(block_tiles(B.n_b, B.Ls), B.nblocks, nrhs);
  DISPATCH_IN(in, blk_p_kernel, );
}
void block_scatter(const BlockArgs &B, int nrhs, cudaStream_t st) {
  dim3 g(block_tiles(B.n_b, B.Ls), B.nblocks, nrhs);
  if (B.gfp64)
    blk_scatter_kernel<F64><<<g, kBlasThreads, 0, st>>>(B);
  else
    blk_scatter_kernel<F32><<<g, kBlasThreads, 0, st>>>(B);
  DWF_CUDA_TRY(cudaGetLastError());
}

}  // namespace dwf

// Layout and precision conversions, gauge-link packing, and the standalone
// Ls-direction operators M_5, M_5^-1 (paper Sec. 2.2 and eq. (dirac_equation)).
#include <algorithm>
#include <type_traits>

#include "device_common.cuh"

namespace dwf {

// ---------------------------------------------------------------------------
// Standalone Ls-direction operator: out = q0 (p0 + p1 S)[(1 - r S)^-1] in.
// ---------------------------------------------------------------------------
// Grid z runs over nrhs * coef_div fields of nsite sites (block-local fields
// of every block are laid out like right-hand sides); field z uses the
// coefficients of right-hand side z / coef_div. A CTA reads its sites before it
// writes them, so out may equal in.
template <class S, bool DAG>
__global__ void __launch_bounds__(256) ls_kernel(char *out, const char *in, long long rstride,
                                                 long long soff, int nsite, int Ls, int inv,
                                                 int coef_div, const __grid_constant__ HopParams P) {
  using R = typename S::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int rhs = blockIdx.z;
  const LsCoef &cf = P.coef[rhs / coef_div];
  const int nsites = P.nsites;
  const int tid = threadIdx.x, s = tid % Ls, sl = tid / Ls;
  const int site = blockIdx.x * nsites + sl;
  const bool active = sl < nsites && site < nsite;
  const int col = Ls + 1;
  R *T = reinterpret_cast<R *>(smem_raw);
  const char *ip = in + rhs * rstride;
  char *op = out + rhs * rstride;
  if (active) {
    R v[24];
    load24<S>(ip, soff, nsite * Ls, site * Ls + s, v);
#pragma unroll
    for (int k = 0; k < 24; ++k) T[(sl * 24 + k) * col + s] = v[k];
  }
  __syncthreads();
  for (int w = tid; w < nsites * 24; w += blockDim.x) {
    if (blockIdx.x * nsites + w / 24 >= nsite) continue;
    const bool down = ((w % 24) < 12) != DAG;
    ls_column<R>(T + w * col, nullptr, Ls, down, inv != 0, kc<R>(cf));
  }
  __syncthreads();
  if (active) {
    R v[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) v[k] = T[(sl * 24 + k) * col + s];
    store24<S>(op, soff, nsite * Ls, site * Ls + s, v);
  }
}

void launch_ls_op(dwf_prec p, char *out, const char *in, long long rstride, int nsite, int Ls,
                  int dagger, int inv, int nrhs, const LsCoef *coef, cudaStream_t st,
                  int coef_div) {
  HopParams P;
  for (int r = 0; r < nrhs; ++r) {
    P.coef[r] = coef[r];
    finalize_coef(P.coef[r]);
  }
  // one thread per (site, s), at most 256 per CTA (128 for FP64)
  const int nsites = std::max(1, (p == DWF_FP64 ? 128 : 256) / Ls);
  P.nsites = nsites;
  dim3 grid((nsite + nsites - 1) / nsites, 1, nrhs * coef_div), block((nsites * Ls + 31) / 32 * 32);
  // at most about 37 KB (nsites * Ls is at most 256): no opt-in beyond 48 KB
  const size_t smem = (size_t)nsites * 24 * (Ls + 1) * (p == DWF_FP64 ? 8 : 4);
  const long long soff = (long long)align_up(field_data_bytes(p, nsite, Ls), 256);
#define LSK(ST, D) \
  ls_kernel<ST, D><<<grid, block, smem, st>>>(out, in, rstride, soff, nsite, Ls, inv, coef_div, P)
  if (p == DWF_FP64) {
    if (dagger) LSK(F64, true); else LSK(F64, false);
  } else if (p == DWF_FP32) {
    if (dagger) LSK(F32, true); else LSK(F32, false);
  } else if (p == DWF_FP16) {
    if (dagger) LSK(F16, true); else LSK(F16, false);
  } else {
    if (dagger) LSK(BF16, true); else LSK(BF16, false);
  }
#undef LSK
  DWF_CUDA_TRY(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Canonical <-> native. The canonical half field is [rhs][s][h][24 reals],
// because the half index h = idx/2 runs over [t][z][y][xh].
// ---------------------------------------------------------------------------
template <class S, class C>
__global__ void import_kernel(char *native, long long nstride, long long soff, const C *canon,
                              int nsite, int Ls) {
  const long long n = (long long)nsite * Ls;
  const int rhs = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int h = (int)(i / Ls), s = (int)(i % Ls);
    const C *src = canon + (((size_t)rhs * Ls + s) * nsite + h) * 24;
    typename S::R v[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) v[k] = (typename S::R)src[k];
    store24<S>(native + rhs * nstride, soff, nsite * Ls, (int)i, v);
  }
}

template <class S, class C>
__global__ void export_kernel(C *canon, const char *native, long long nstride, long long soff,
                              int nsite, int Ls) {
  const long long n = (long long)nsite * Ls;
  const int rhs = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int h = (int)(i / Ls), s = (int)(i % Ls);
    C *dst = canon + (((size_t)rhs * Ls + s) * nsite + h) * 24;
    typename S::R v[24];
    load24<S>(native + rhs * nstride, soff, nsite * Ls, (int)i, v);
#pragma unroll
    for (int k = 0; k < 24; ++k) dst[k] = (C)v[k];
  }
}

void launch_import(dwf_prec p, char *native, long long nstride, const void *canon, int canon_fp32,
                   int nsite, int Ls, const int *, int nrhs, cudaStream_t st) {
  const long long soff = (long long)align_up(field_data_bytes(p, nsite, Ls), 256);
  dim3 grid(1024, nrhs), block(256);
#define IMP(ST)                                                                          \
  do {                                                                                   \
    if (canon_fp32)                                                                      \
      import_kernel<ST, float><<<grid, block, 0, st>>>(native, nstride, soff,            \
                                                       (const float *)canon, nsite, Ls); \
    else                                                                                 \
      import_kernel<ST, double><<<grid, block, 0, st>>>(native, nstride, soff,           \
                                                        (const double *)canon, nsite, Ls); \
  } while (0)
  switch (p) {
    case DWF_FP64: IMP(F64); break;
    case DWF_FP32: IMP(F32); break;
    case DWF_FP16: IMP(F16); break;
    case DWF_BF16: IMP(BF16); break;
  }
#undef IMP
  DWF_CUDA_TRY(cudaGetLastError());
}

void launch_export(dwf_prec p, void *canon, int canon_fp32, const char *native, long long nstride,
                   int nsite, int Ls, const int *, int nrhs, cudaStream_t st) {
  const long long soff = (long long)align_up(field_data_bytes(p, nsite, Ls), 256);
  dim3 grid(1024, nrhs), block(256);
#define EXP(ST)                                                                               \
  do {                                                                                        \
    if (canon_fp32)                                                                           \
      export_kernel<ST, float><<<grid, block, 0, st>>>((float *)canon, native, nstride, soff, \
                                                       nsite, Ls);                            \
    else                                                                                      \
      export_kernel<ST, double><<<grid, block, 0, st>>>((double *)canon, native, nstride,     \
                                                        soff, nsite, Ls);                     \
  } while (0)
  switch (p) {
    case DWF_FP64: EXP(F64); break;
    case DWF_FP32: EXP(F32); break;
    case DWF_FP16: EXP(F16); break;
    case DWF_BF16: EXP(BF16); break;
  }
#undef EXP
  DWF_CUDA_TRY(cudaGetLastError());
}

// Native -> native in another precision (FP16/BF16 outputs take the per-element
// scale of the stored values).
template <class SI, class SO>
__global__ void convert_kernel(char *out, long long ostride, long long osoff, const char *in,
                               long long istride, long long isoff, int n) {
  const int rhs = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    typename SI::R v[24];
    load24<SI>(in + rhs * istride, isoff, n, i, v);
    typename SO::R w[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) w[k] = (typename SO::R)v[k];
    store24<SO>(out + rhs * ostride, osoff, n, i, w);
  }
}

template <class SI>
static void convert_from(dwf_prec po, char *out, long long ostride, long long osoff,
                         const char *in, long long istride, long long isoff, int n, int nrhs,
                         cudaStream_t st) {
  dim3 grid(1024, nrhs), block(256);
  switch (po) {
    case DWF_FP64:
      convert_kernel<SI, F64><<<grid, block, 0, st>>>(out, ostride, osoff, in, istride, isoff, n);
      break;
    case DWF_FP32:
      convert_kernel<SI, F32><<<grid, block, 0, st>>>(out, ostride, osoff, in, istride, isoff, n);
      break;
    case DWF_FP16:
      convert_kernel<SI, F16><<<grid, block, 0, st>>>(out, ostride, osoff, in, istride, isoff, n);
      break;
    case DWF_BF16:
      convert_kernel<SI, BF16><<<grid, block, 0, st>>>(out, ostride, osoff, in, istride, isoff, n);
      break;
  }
}

void launch_convert(dwf_prec po, char *out, dwf_prec pi, const char *in, int nsite, int Ls,
                    int nrhs, cudaStream_t st) {
  const long long ostride = (long long)field_rhs_bytes(po, nsite, Ls);
  const long long istride = (long long)field_rhs_bytes(pi, nsite, Ls);
  const long long osoff = (long long)align_up(field_data_bytes(po, nsite, Ls), 256);
  const long long isoff = (long long)align_up(field_data_bytes(pi, nsite, Ls), 256);
  const int n = nsite * Ls;
  switch (pi) {
    case DWF_FP64: convert_from<F64>(po, out, ostride, osoff, in, istride, isoff, n, nrhs, st); break;
    case DWF_FP32: convert_from<F32>(po, out, ostride, osoff, in, istride, isoff, n, nrhs, st); break;
    case DWF_FP16: convert_from<F16>(po, out, ostride, osoff, in, istride, isoff, n, nrhs, st); break;
    case DWF_BF16: convert_from<BF16>(po, out, ostride, osoff, in, istride, isoff, n, nrhs, st); break;
  }
  DWF_CUDA_TRY(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Gauge links. Input U[t][z][y][x][mu][3][3] complex128. Each link record
// (owner, mu) -- owner = parity * Vh + idx/2, the combined numbering -- is cut
// into 16-byte words (FP64 9, FP32 5, FP16 3: 18 reals, zero padded), stored
// chunk-major: word k of (owner, mu) at index (mu * words + k) * nown + owner,
// nown = V4. Consecutive owners' words are adjacent, so the link loads of the
// sites of a warp are contiguous. The link leaving t = Lt-1 carries the
// antiperiodic sign.
// ---------------------------------------------------------------------------
__global__ void pack_links_kernel(const double *U, double *l64, float *l32, __half *l16, int Lx,
                                  int Ly, int Lz, int Lt, int tap, int recon) {
  const int V4 = Lx * Ly * Lz * Lt, Vh = V4 / 2;
  const int w32 = recon ? 4 : 5, w16 = recon ? 2 : 3;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V4 * 4; i += gridDim.x * blockDim.x) {
    const int idx = i / 4, mu = i % 4;
    const int x = idx % Lx, y = (idx / Lx) % Ly, z = (idx / (Lx * Ly)) % Lz,
              t = idx / (Lx * Ly * Lz);
    const int par = (x + y + z + t) & 1;
    const size_t owner = (size_t)par * Vh + (idx >> 1);
    const double sgn = (tap && mu == 3 && t == Lt - 1) ? -1.0 : 1.0;
    const double *src = U + (size_t)i * 18;
    double v[24];
    for (int k = 0; k < 24; ++k) v[k] = k < 18 ? sgn * src[k] : 0.0;
    for (int w = 0; w < 9; ++w)  // FP64: 2 reals per word
      for (int q = 0; q < 2; ++q) l64[(((size_t)mu * 9 + w) * V4 + owner) * 2 + q] = v[2 * w + q];
    if (recon) {
      // the signed first two rows, then the sign: the third row is rebuilt
      // on load as sign * conj(row0 x row1)
      v[12] = sgn;
      for (int k = 13; k < 24; ++k) v[k] = 0.0;
    }
    for (int w = 0; w < w32; ++w)  // FP32: 4 reals per word
      for (int q = 0; q < 4; ++q)
        l32[(((size_t)mu * w32 + w) * V4 + owner) * 4 + q] = (float)v[4 * w + q];
    for (int w = 0; w < w16; ++w)  // FP16: 8 reals per word
      for (int q = 0; q < 8; ++q)
        l16[(((size_t)mu * w16 + w) * V4 + owner) * 8 + q] = __double2half(v[8 * w + q]);
  }
}

void launch_pack_links(const double *U, char *l64, char *l32, char *l16, int recon,
                       const int dims[4], int tap, cudaStream_t st) {
  pack_links_kernel<<<1024, 256, 0, st>>>(U, (double *)l64, (float *)l32, (__half *)l16, dims[0],
                                          dims[1], dims[2], dims[3], tap, recon);
  DWF_CUDA_TRY(cudaGetLastError());
}

// Per-block link copies, chunk-major per block: word k of (local owner c, mu)
// of block b at index b * 4 * words * n_comb + (mu * words + k) * n_comb + c,
// copied from the global record of owner gowner[b][c].
__global__ void block_links_kernel(char *dst, const char *src, int words, const int *gowner,
                                   int n_comb, int nblocks, int nown) {
  const long long per_block = 4LL * words * n_comb;
  const long long n = per_block * nblocks;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / per_block);
    const long long r = i - b * per_block;
    const int mw = (int)(r / n_comb), c = (int)(r % n_comb);
    const int owner = gowner[(size_t)b * n_comb + c];
    reinterpret_cast<uint4 *>(dst)[i] =
        __ldg(reinterpret_cast<const uint4 *>(src) + (size_t)mw * nown + owner);
  }
}

void launch_block_links(dwf_prec p, int recon, char *dst, const char *src_l32,
                        const char *src_l16, const int *gowner, int n_comb, int nblocks,
                        const int *dims, cudaStream_t st) {
  const int rec = (int)link_record_bytes(p == DWF_FP32 ? DWF_FP32 : DWF_FP16, recon);
  const char *src = (p == DWF_FP32) ? src_l32 : src_l16;
  const int V4 = dims[0] * dims[1] * dims[2] * dims[3];
  block_links_kernel<<<1024, 256, 0, st>>>(dst, src, rec / 16, gowner, n_comb, nblocks, V4);
  DWF_CUDA_TRY(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Coefficients
// ---------------------------------------------------------------------------
static LsCoef base(double mf) {
  LsCoef c{};
  c.q0 = 1.0;
  c.p0 = 1.0;
  c.mf = mf;
  c.pre_b = 1.0;
  return c;
}
LsCoef coef_identity(double q0) {
  LsCoef c = base(0.0);
  c.q0 = q0;
  return c;
}
LsCoef coef_m5(const dwf_action &a, double mf, double q0) {
  LsCoef c = base(mf);
  const double al = a.b * (4.0 - a.M5) + 1.0, be = a.c * (4.0 - a.M5) - 1.0;
  c.q0 = q0;
  c.p0 = al;
  c.p1 = be;
  return c;
}
static void set_inv(LsCoef &c, const dwf_action &a, double mf) {
  const double al = a.b * (4.0 - a.M5) + 1.0, be = a.c * (4.0 - a.M5) - 1.0;
  c.r = -be / al;
  double rl = 1.0;
  for (int k = 0; k < a.Ls; ++k) rl *= c.r;
  c.inv_den = 1.0 / (1.0 + mf * rl);
  c.q0 /= al;
}
LsCoef coef_m5inv(const dwf_action &a, double mf, double q0) {
  LsCoef c = base(mf);
  c.q0 = q0;
  set_inv(c, a, mf);
  return c;
}
LsCoef coef_mphi(const dwf_action &a, double mf, double q0) {
  LsCoef c = base(mf);
  c.q0 = q0;
  c.p0 = a.b;
  c.p1 = a.c;
  return c;
}
LsCoef coef_k(const dwf_action &a, double mf, double q0) {
  LsCoef c = coef_mphi(a, mf, q0);
  set_inv(c, a, mf);
  return c;
}

}  // namespace dwf

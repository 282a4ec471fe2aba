// The 4D Wilson hop with the fifth dimension, the one kernel behind every
// operator application of the solver (paper Sec. 2.2, M^4 = D^w M_phi and
// eq. for D^w; Sec. 2.3 for its use inside the Dirichlet block operator).
//
// One thread computes one output (site, s). A CTA holds SITES sites x all Ls
// slices, so the links of a site are loaded once per CTA line and broadcast to
// the Ls threads of the site, and the Ls-direction operators that follow the
// hop (M_phi^+, M_5^-1 M_phi, M_5) run in shared memory on the CTA's own sites
// (one thread per site and spin-colour component walks s).
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

// One direction of the hop: project, multiply by U or U^+, reconstruct, add.
template <class S, int MU, bool FWD, bool DAG, bool PRE>
__device__ __forceinline__ void hop_dir(typename S::R *acc, const char *in, long long soff,
                                        int j, int s, int Ls, const char *links, int owner,
                                        const LsCoef &cf) {
  using R = typename S::R;
  R v[24];
  load24<S>(in, soff, j, s, Ls, v);
  if constexpr (PRE) {
    R w[12];
    const R b = (R)cf.pre_b, c = (R)cf.pre_c, mf = (R)cf.mf;
    const int sm = s == 0 ? Ls - 1 : s - 1;
    const R fm = s == 0 ? -mf : (R)1;
    load12<S, true>(in, soff, j, sm, Ls, w);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = b * v[k] + c * fm * w[k];
    const int sp = s == Ls - 1 ? 0 : s + 1;
    const R fp = s == Ls - 1 ? -mf : (R)1;
    load12<S, false>(in, soff, j, sp, Ls, w);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[12 + k] = b * v[12 + k] + c * fp * w[k];
  }
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
  R u[18];
  load_link<S>(links, owner, MU, u);
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

template <class S, int MU, bool DAG, bool PRE>
__device__ __forceinline__ void hop_mu(typename S::R *acc, const HopParams &P, const char *in,
                                       const char *links, const int *nb, int site, int s,
                                       const LsCoef &cf) {
  const int jf = nb[2 * MU], jb = nb[2 * MU + 1];
  if (jf >= 0 && jf < P.in_limit)
    hop_dir<S, MU, true, DAG, PRE>(acc, in, P.in.scale_off, jf, s, P.Ls, links,
                                   P.out_link_off + site, cf);
  if (jb >= 0 && jb < P.in_limit)
    hop_dir<S, MU, false, DAG, PRE>(acc, in, P.in.scale_off, jb, s, P.Ls, links,
                                    P.in_link_off + jb, cf);
}

template <class S, bool DAG, bool PRE>
__global__ void __launch_bounds__(256) hop_kernel(const __grid_constant__ HopParams P) {
  using R = typename S::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  const int rhs = blockIdx.z, blk = blockIdx.y;
  if (P.skip && P.skip[rhs]) return;
  const int Ls = P.Ls;
  const int nsites = P.nsites;  // blockDim.x is nsites * Ls rounded up to whole warps
  const int tid = threadIdx.x;
  const int s = tid % Ls, sl = tid / Ls;
  const int site = blockIdx.x * nsites + sl;
  const bool active = (sl < nsites) && (site < P.n_out);
  const LsCoef &cf = P.coef[rhs];

  const char *in = P.in.data + blk * P.in.bstride + rhs * P.in.rstride;
  char *out = P.out.data + blk * P.out.bstride + rhs * P.out.rstride;
  const char *links = P.links + blk * P.link_bstride;

  R acc[24];
#pragma unroll
  for (int k = 0; k < 24; ++k) acc[k] = 0;
  if (active) {
    const int *nb = P.nbr + (size_t)site * 8;
    hop_mu<S, 0, DAG, PRE>(acc, P, in, links, nb, site, s, cf);
    hop_mu<S, 1, DAG, PRE>(acc, P, in, links, nb, site, s, cf);
    hop_mu<S, 2, DAG, PRE>(acc, P, in, links, nb, site, s, cf);
    hop_mu<S, 3, DAG, PRE>(acc, P, in, links, nb, site, s, cf);
  }

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
          load24<S>(xo, P.xown.scale_off, site, s, Ls, xv);
        } else {
#pragma unroll
          for (int k = 0; k < 24; ++k) xv[k] = 0;
        }
#pragma unroll
        for (int k = 0; k < 24; ++k) X[(sl * 24 + k) * col + s] = xv[k];
      }
    }
    __syncthreads();
    for (int w = tid; w < nsites * 24; w += blockDim.x) {
      const int wsite = blockIdx.x * nsites + w / 24;
      if (wsite >= P.n_out) continue;
      const int comp = w % 24;
      const bool down = (comp < 12) != DAG;
      ls_column<R>(T + w * col, P.has_x ? X + w * col : nullptr, Ls, down, P.inv != 0, cf);
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int k = 0; k < 24; ++k) acc[k] = T[(sl * 24 + k) * col + s];
    }
  } else {
    const R q = (R)cf.q0;
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] *= q;
  }
  if (active) store24<S>(out, P.out.scale_off, site, s, Ls, acc);

  if (P.dot) {
    double d = 0.0;
    if (active) {
      R dv[24];
      const char *dp = P.dotv.data + blk * P.dotv.bstride + rhs * P.dotv.rstride;
      load24<S>(dp, P.dotv.scale_off, site, s, Ls, dv);
#pragma unroll
      for (int k = 0; k < 24; ++k) d += (double)dv[k] * (double)acc[k];
    }
    d = cta_sum(d, red);
    const int ntiles = gridDim.x;
    const int grp = rhs * P.nblocks + blk;
    double total;
    if (group_reduce(d, P.partials + (size_t)grp * ntiles, ntiles, blockIdx.x, P.counters + grp,
                     total))
      P.dot_out[(size_t)rhs * P.dot_rstride + blk] = total;
  }
}

int hop_sites_per_cta(int Ls, dwf_prec p) {
  int target = (p == DWF_FP64) ? 128 : 256;
  int n = target / Ls;
  return n < 1 ? 1 : n;
}

size_t hop_smem_bytes(int Ls, dwf_prec p, int has_x) {
  size_t rs = (p == DWF_FP64) ? 8 : 4;
  return (size_t)hop_sites_per_cta(Ls, p) * 24 * (Ls + 1) * rs * (has_x ? 2 : 1);
}

template <class S, bool DAG, bool PRE>
static void launch_t(const HopParams &P0, int nrhs, cudaStream_t st, dwf_prec prec) {
  HopParams P = P0;
  const int nsites = hop_sites_per_cta(P.Ls, prec);
  P.nsites = nsites;
  dim3 grid((P.n_out + nsites - 1) / nsites, P.nblocks, nrhs);
  dim3 block((nsites * P.Ls + 31) / 32 * 32);
  size_t smem = P.epi ? hop_smem_bytes(P.Ls, prec, P.has_x) : 0;
  if (grid.x == 0) return;
  hop_kernel<S, DAG, PRE><<<grid, block, smem, st>>>(P);
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
  if (dagger)
    launch_t<S, true, false>(P, nrhs, st, p);
  else if (pre_mphi)
    launch_t<S, false, true>(P, nrhs, st, p);
  else
    launch_t<S, false, false>(P, nrhs, st, p);
}

// Allow the hop kernels more than 48 KB of dynamic shared memory. Called once
// per device before any launch (and so before any stream capture).
template <class S>
static void prepare_one() {
  const int big = 200 * 1024;
  DWF_CUDA_TRY(cudaFuncSetAttribute(hop_kernel<S, false, false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  DWF_CUDA_TRY(cudaFuncSetAttribute(hop_kernel<S, false, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  DWF_CUDA_TRY(cudaFuncSetAttribute(hop_kernel<S, true, false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, big));
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

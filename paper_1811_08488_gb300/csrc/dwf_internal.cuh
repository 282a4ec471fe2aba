// Internal declarations of the DWF / MSPCG library (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/dwf.h"

namespace dwf {

constexpr int kMaxRhs = DWF_MAX_RHS;
constexpr int kHistory = 256;  // ring buffer of per-iteration |r|^2 values

// ---------------------------------------------------------------------------
// Error handling
// ---------------------------------------------------------------------------
struct Error {
  dwf_status code;
  std::string msg;
};

#define DWF_CUDA_TRY(expr)                                                    \
  do {                                                                        \
    cudaError_t e_ = (expr);                                                  \
    if (e_ != cudaSuccess)                                                    \
      throw ::dwf::Error{DWF_ERR_CUDA, std::string(#expr) + ": " +            \
                                           cudaGetErrorString(e_)};           \
  } while (0)

#define DWF_REQUIRE(cond, code, text)                                         \
  do {                                                                        \
    if (!(cond)) throw ::dwf::Error{code, text};                              \
  } while (0)

// ---------------------------------------------------------------------------
// Storage traits of native fields and link records
// ---------------------------------------------------------------------------
// A native field stores, per (site, s), 24 reals in 16-byte chunks; chunk k of
// all Ls slices of a site is contiguous (see include/dwf.h).
struct F64 {
  using R = double;
  static constexpr int kChunks = 12;
  static constexpr bool kHalf = false;
  static constexpr int kLinkChunks = 9;  // 18 doubles
  static constexpr int kLinkChunksRecon = 9;  // never reconstructed
};
struct F32 {
  using R = float;
  static constexpr int kChunks = 6;
  static constexpr bool kHalf = false;
  static constexpr int kLinkChunks = 5;  // 18 floats + 2 pad
  static constexpr int kLinkChunksRecon = 4;  // 12 floats + sign + 3 pad
};
struct F16 {
  using R = float;
  static constexpr int kChunks = 3;
  static constexpr bool kHalf = true;
  static constexpr int kLinkChunks = 3;  // 18 halves + 6 pad
  static constexpr int kLinkChunksRecon = 2;  // 12 halves + sign + 3 pad
};
struct BF16 {
  using R = float;
  static constexpr int kChunks = 3;
  static constexpr bool kHalf = true;
  static constexpr int kLinkChunks = 3;  // links are stored as FP16
  static constexpr int kLinkChunksRecon = 2;
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bytes of the data part and offset of the scale part of one right-hand side.
inline size_t field_data_bytes(dwf_prec p, size_t nsite, int Ls) {
  switch (p) {
    case DWF_FP64: return nsite * Ls * 24 * 8;
    case DWF_FP32: return nsite * Ls * 24 * 4;
    default: return nsite * Ls * 24 * 2;
  }
}
inline size_t field_rhs_bytes(dwf_prec p, size_t nsite, int Ls) {
  size_t d = align_up(field_data_bytes(p, nsite, Ls), 256);
  if (p == DWF_FP16 || p == DWF_BF16) d += align_up(nsite * Ls * sizeof(float), 256);
  return d;
}
// Bytes of one link record: 18 reals in 16-byte words (FP64 9, FP32 5, FP16 3);
// with reconstruct-12 the first two rows, the boundary sign and padding
// (FP32 4 words: 12 floats + sign; FP16 2 words: 12 halves + sign).
inline size_t link_record_bytes(dwf_prec p, int recon = 0) {
  if (p == DWF_FP64) return 144;
  if (p == DWF_FP32) return recon ? 64 : 80;
  return recon ? 32 : 48;
}

// A view of a native field: base of (block 0, rhs 0), byte strides.
struct FieldRef {
  char *data = nullptr;
  long long bstride = 0;  // bytes between blocks (block-local fields)
  long long rstride = 0;  // bytes between right-hand sides
  long long scale_off = 0;  // byte offset of the scale array from data (half)
  int cs = 0;               // elements per chunk plane: nsite * Ls
};

// Ls-direction operator applied in the epilogue of a hop kernel, per rhs:
//   out = q0 (p0 + p1 S) [(1 - r S)^-1 if inv] acc  +  (a0 + a1 S) xown
// with S the chiral shift (wrap factor -mf). The direction of S on each
// chirality is fixed by the kernel's dagger flag.
// Copies of the coefficients in the kernel's arithmetic type, filled on the
// host by finalize_coef(): FP32 kernels then do no FP64 arithmetic or
// conversion (GB300's FP64 pipe is a small fraction of its FP32 pipe).
template <class R>
struct LsK {
  R p0q, p1q;  // q0 * p0, q0 * p1
  R r, inv_den, a0, a1, mf, pre_b, pre_c, q0;
};

struct LsCoef {
  double q0, p0, p1, r, inv_den, a0, a1, mf;
  double pre_b, pre_c;  // M_phi applied to the hop input (b + c S)
  LsK<float> f;
  LsK<double> d;
};

inline void finalize_coef(LsCoef &c) {
  c.d = {c.q0 * c.p0, c.q0 * c.p1, c.r, c.inv_den, c.a0, c.a1, c.mf, c.pre_b, c.pre_c, c.q0};
  c.f = {(float)c.d.p0q, (float)c.d.p1q, (float)c.r, (float)c.inv_den, (float)c.a0,
         (float)c.a1, (float)c.mf, (float)c.pre_b, (float)c.pre_c, (float)c.q0};
}

// Device-side timer of one kernel family (slot), filled while profiling is
// on: start holds the entry time of CTA 0 of the launch in flight (global
// timer, ns), done counts its finished CTAs; the last CTA adds its exit time
// minus start to total_ns and resets done for the next launch (end unused).
struct KernProf {
  unsigned long long start, end;
  unsigned long long total_ns, launches, bytes;
  unsigned int done, pad;
};
// slot = role * 32 + prec * 8 + DAG * 4 + PRE * 2 + EPI; role 0: operators on the
// whole lattice (dslash, D_PC, A), role 1: the block operator A_s
constexpr int kProfSlots = 64;

struct HopParams {
  FieldRef in, out, xown, dotv;
  const char *links = nullptr;
  long long link_bstride = 0;
  int link_cs = 0;  // link owners per block: word k of (owner, mu) at (mu*words + k)*link_cs + owner
  int recon = 0;       // 1: records hold two rows and a sign (reconstruct-12)
  const int *nbr = nullptr;  // [n_out][8], direction 2*mu + (0 fwd, 1 bwd)
  int n_out = 0;             // output sites per block
  int in_limit = 0;          // inputs with index >= in_limit are zero
  int xown_limit = 0;        // xown is zero for sites >= xown_limit
  int out_link_off = 0;      // combined link id of output site i: off + i
  int in_link_off = 0;
  int Ls = 0;
  int nsites = 0;  // output sites per CTA (set by the launcher)
  int nblocks = 1;
  int role = 0;    // timer slot group: 0 whole-lattice operator, 1 block operator
  int epi = 0;     // 0: out = q0 * acc; 1: Ls epilogue in shared memory
  int inv = 0;     // epilogue uses (1 - r S)^-1
  int has_x = 0;   // epilogue adds (a0 + a1 S) xown
  int dot = 0;     // accumulate Re<dotv, out> per (block, rhs)
  double *partials = nullptr;   // [rhs][block][tiles]
  double *dot_out = nullptr;    // final sums at dot_out[rhs * dot_rstride + block]
  int dot_rstride = 0;
  unsigned int *counters = nullptr;  // [rhs][block]
  const int *skip = nullptr;    // per rhs: nonzero = skip (converged)
  const int *bskip = nullptr;   // per (rhs, block): nonzero = skip (inner stop met)
  KernProf *prof = nullptr;     // timer slot of this launch (null: profiling off)
  unsigned long long alg_bytes = 0;  // compulsory bytes of this launch
  LsCoef coef[kMaxRhs];
};

// ---------------------------------------------------------------------------
// Geometry
// ---------------------------------------------------------------------------
struct Geometry {
  int dims[4];
  int V4, Vh;
  std::vector<int> nbr[2];  // host: [out parity][Vh*8] neighbour half index
};

// Block (sub-lattice) decomposition with the distance-2 region of every block.
struct BlockGeometry {
  int block[4];
  int nblocks;
  int n_b;     // even sites in the block
  int n_ob;    // odd sites in the block
  int n_e1;    // even sites at distance <= 1
  int n_e2;    // even sites at distance <= 2
  int n_o1;    // odd sites at distance <= 1
  int n_comb;  // n_e2 + n_o1 (link owners)
  std::vector<int> nbr_oe;  // [n_o1][8]: odd out <- even in (local even index or -1)
  std::vector<int> nbr_eo;  // [n_e2][8]: even out <- odd in (local odd index or -1)
  std::vector<int> gsite;   // [nblocks][n_comb] global lexicographic site of each owner
  std::vector<int> gmap_b;  // [nblocks][n_b] global even half index of block sites
};

void build_geometry(Geometry &g, const int dims[4]);
void build_block_geometry(BlockGeometry &bg, const int dims[4], const int block[4]);

// ---------------------------------------------------------------------------
// Device buffers
// ---------------------------------------------------------------------------
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  void ensure(size_t n) {
    if (bytes >= n && p) return;
    release();
    DWF_CUDA_TRY(cudaMalloc(&p, n ? n : 16));
    bytes = n;
  }
  template <class T> T *as() const { return reinterpret_cast<T *>(p); }
  char *c() const { return reinterpret_cast<char *>(p); }
};

// Scalars of the outer solve, per right-hand side.
struct OuterScalars {
  double rz;      // <r, z> of the current iterate (Algorithm 1)
  double rz_new;  // <r_{k+1}, z_{k+1}>
  double pAp;     // <p, A p>
  double rr;      // |r|^2 of the iterated residual
  double alpha, beta;
  double apz;     // <A p, z_{k+1}> (flexible PCG)
  double bb;      // |b|^2
  int iter;       // iterations done
  int done;       // converged: a reliable update confirmed |b - A x| <= tol |b|
  double maxr;    // largest |r| since the last reliable update
  double final_res;  // |b - A x| / |b| once done (-1 while open)
  int nru;        // reliable updates done
  int pad;
  double hist_rr[kHistory];
};

// Loop state of the device-driven outer solve (one per solve): the device
// decides the reliable updates and convergence after every iteration and ends
// the graph's loop when every right-hand side is done, on a NaN, at maxiter,
// or after `budget` iterations of one graph launch.
struct SolveCtl {
  double tol2, delta;
  int maxiter, budget;
  int launch_iters;  // iterations of the current graph launch
  int nan;           // a non-finite residual norm was seen
  int nrhs, pad;
};

struct BlockPlan;
struct SolverPlan;

}  // namespace dwf

// The context.
struct dwf_ctx {
  int device = 0;
  dwf_action act{};
  dwf::Geometry geo;
  dwf::DevBuf nbr_dev[2];
  dwf::DevBuf links[3];  // FP64, FP32, FP16 link records, combined numbering
  bool have_gauge = false;
  std::string last_error;
  cudaStream_t own_stream = nullptr;
  // operator work buffers (odd/even temporaries, per precision)
  dwf::DevBuf tmp[4];
  dwf::DevBuf red;  // reduction partials and counters for operator calls
  dwf::DevBuf tc_aux;  // tensor-core M_5^-1: status word and B operands
  std::vector<double> tc_key;         // masses + adjoint flag of the B operands in tc_aux
  float tc_unscale[DWF_MAX_RHS][2]{};  // their power-of-two scales
  std::map<std::string, std::unique_ptr<dwf::BlockPlan>> block_plans;
  std::map<std::string, std::unique_ptr<dwf::SolverPlan>> solver_plans;
  std::map<std::string, std::array<int, 4>> tuned_blocks;  // autotuner results
  // low modes (eig.cu): subspace W, A W, three batches of Chebyshev terms, and
  // the small matrices and reduction scratch of the Rayleigh-Ritz step
  dwf::DevBuf eig_w, eig_aw, eig_t, eig_small;
  dwf::DevBuf defl;    // dwf_deflate: coefficients, 1/lambda, reduction scratch
  dwf::DevBuf prof;    // kProfSlots KernProf timer slots of the hop kernels
  int prof_on = 0;
  int unusable = 0;    // set after a device wait expired with work possibly in flight
  ~dwf_ctx();
};

namespace dwf {

// hop.cu
template <class S>
void launch_hop(const HopParams &P, int dagger, int pre_mphi, int nrhs, cudaStream_t st);
int hop_sites_per_cta(int Ls, dwf_prec p);
size_t hop_smem_bytes(int Ls, dwf_prec p, int epi, int has_x);

// ls.cu: Ls-local operators (M_5, M_5^-1) on native fields
// Tensor-core M_5^-1 (csrc/m5tc.cu); synchronises `st` and checks the status word.
void launch_m5inv_gemm(dwf_ctx *ctx, dwf_prec p, char *out, const char *in, int dagger, int nrhs,
                       const double *mf, cudaStream_t st);
void launch_ls_op(dwf_prec p, char *out, const char *in, long long rstride,
                  int nsite, int Ls, int dagger, int inv, int nrhs, const LsCoef *coef,
                  cudaStream_t st, int coef_div = 1);

// fields.cu: layout and precision conversions
void launch_import(dwf_prec p, char *native, long long nstride, const void *canon,
                   int canon_fp32, int nsite, int Ls, const int dims[4], int nrhs,
                   cudaStream_t st);
void launch_export(dwf_prec p, void *canon, int canon_fp32, const char *native,
                   long long nstride, int nsite, int Ls, const int dims[4], int nrhs,
                   cudaStream_t st);
void launch_pack_links(const double *U, char *l64, char *l32, char *l16, int recon,
                       const int dims[4], int t_antiperiodic, cudaStream_t st);
void launch_block_links(dwf_prec p, int recon, char *dst, const char *src_l32, const char *src_l16,
                        const int *gowner, int n_comb, int nblocks, const int dims[4],
                        cudaStream_t st);

// Coefficients of the standard operators.
LsCoef coef_identity(double q0);
LsCoef coef_m5(const dwf_action &a, double mf, double q0);
LsCoef coef_m5inv(const dwf_action &a, double mf, double q0);
LsCoef coef_mphi(const dwf_action &a, double mf, double q0);
LsCoef coef_k(const dwf_action &a, double mf, double q0);  // q0 M_phi M_5^-1

}  // namespace dwf

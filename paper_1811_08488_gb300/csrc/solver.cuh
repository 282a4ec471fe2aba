// Host-side composition of the operators and the solver plans.
#pragma once

#include "blas.cuh"
#include "dwf_internal.cuh"
#include "eig.cuh"

namespace dwf {

// Three half-field temporaries (odd u, even y, odd v) of one precision.
struct OpWork {
  char *u = nullptr, *y = nullptr, *v = nullptr;
  long long rstride = 0;
};

// Optional fused reduction of Re<dotv, out> into dot_out (stage D of A).
struct DotSpec {
  const char *dotv = nullptr;
  double *partials = nullptr;
  unsigned int *counters = nullptr;
  double *dot_out = nullptr;
  int dot_rstride = 0;
};

FieldRef global_ref(const dwf_ctx *ctx, dwf_prec p, const void *ptr);
const char *link_ptr(const dwf_ctx *ctx, dwf_prec p);
OpWork op_work(dwf_ctx *ctx, dwf_prec p, int nrhs);

void apply_dslash(dwf_ctx *ctx, void *out, const void *in, int out_parity, int dagger,
                  dwf_prec p, int nrhs, const double *mf, cudaStream_t st);
void apply_mpc(dwf_ctx *ctx, void *out, const void *in, int dagger, dwf_prec p, int nrhs,
               const double *mf, const OpWork &w, cudaStream_t st);
void apply_source_prep(dwf_ctx *ctx, void *b_even, const void *phi_even, const void *phi_odd,
                       dwf_prec p, int nrhs, const double *mf, const OpWork &w, cudaStream_t st);
void apply_odd_reconstruct(dwf_ctx *ctx, void *psi_odd, const void *psi_even,
                           const void *phi_odd, dwf_prec p, int nrhs, const double *mf,
                           const OpWork &w, cudaStream_t st);
// schur = 0: A = D_PC^+ D_PC; 1: A_sym = D_sym^+ D_sym (symmetric form)
void apply_mdagm(dwf_ctx *ctx, void *out, const void *in, dwf_prec p, int nrhs,
                 const double *mf, const OpWork &w, const DotSpec *dot, const int *skip,
                 cudaStream_t st, int schur = 0);
void apply_mpc_sym(dwf_ctx *ctx, void *out, const void *in, int dagger, dwf_prec p, int nrhs,
                   const double *mf, const OpWork &w, cudaStream_t st);
void apply_source_prep_sym(dwf_ctx *ctx, void *b_even, const void *phi_even, const void *phi_odd,
                           dwf_prec p, int nrhs, const double *mf, const OpWork &w,
                           cudaStream_t st);

// The multisplitting block plan: geometry, tables, per-block links, vectors.
struct BlockPlan {
  BlockGeometry bg;
  dwf_prec inner = DWF_FP16;
  int nrhs = 0;
  int Ls = 0;
  DevBuf nbr_oe, nbr_eo, gmap_b, gowner;
  DevBuf links;
  long long link_bstride = 0;
  DevBuf r, p, Ap, x, u1, y, u2, w2;
  FieldRef fr, fp, fAp, fx, fu1, fy, fu2, fw2;  // w2: M_5^-+ y (symmetric form)
  DevBuf scal;  // rr, rr_new, pAp, (scratch), rr0: 5 x [nrhs][nblocks] doubles
  DevBuf partials, counters, gpart, gcount, gpart2, gcount2;
  DevBuf bstop;  // [nrhs][nblocks] inner residual stop flags
  DevBuf iters;  // [nrhs] block iterations counted by the inner CG
  bool links_valid = false;
  bool stop_active = false;  // the inner residual stop is on for the launches being built
};

BlockPlan *get_block_plan(dwf_ctx *ctx, const int block[4], dwf_prec inner, int nrhs,
                          cudaStream_t st);
// out = (+)_s A_s p on the plan's block vectors (p -> Ap), optional <p, Ap>;
// schur = 1: the blocks of the symmetric form's normal operator.
void block_apply_A(dwf_ctx *ctx, BlockPlan *bp, int snake, int nrhs, const double *mf,
                   bool with_dot, const int *skip, cudaStream_t st, int schur = 0);
// z = M^-1 r on FP32 global fields; <r, z> -> rz_out[rhs * rz_rstride] if given.
// glob: precision of z and r (FP32, or FP64 for an FP64 outer solver). With
// ap and apz_out, also <A p, z> -> apz_out[rhs * rz_rstride] (flexible PCG).
void block_precondition(dwf_ctx *ctx, BlockPlan *bp, char *z, const char *r, int k, int snake,
                        int nrhs, const double *mf, double *rz_out, int rz_rstride,
                        const int *skip, cudaStream_t st, dwf_prec glob = DWF_FP32,
                        const char *ap = nullptr, double *apz_out = nullptr,
                        double inner_tol = 0.0, int schur = 0);

BlockArgs block_args(dwf_ctx *ctx, BlockPlan *bp, char *z, const char *r, double *rz_out,
                     int rz_rstride, const int *skip, dwf_prec glob = DWF_FP32);

struct SolverPlan {
  dwf_prec lo = DWF_FP32;
  int nrhs = 0;
  DevBuf b64, x64, r64, Ax64;
  DevBuf xlo, rlo, p, Ap, z;
  DevBuf wlo, w64;  // operator temporaries
  DevBuf scal, partials, counters, opart, ocount, skip_iter, skip_ru;
  DevBuf ctl;  // SolveCtl of the device-driven loop
  DevBuf defl;  // deflation: V^+ r coefficients, 1/lambda, reduction scratch
  OuterScalars *host_scal = nullptr;
  int *host_skip = nullptr;
  SolveCtl *host_ctl = nullptr;
  cudaGraphExec_t loop = nullptr;  // the device-driven outer loop (one graph)
  std::string loop_key;
  void drop_graphs();
  ~SolverPlan();
};

// defl (optional): deflation with Ritz pairs (V and n_ev; lambda on the host,
// copied to the plan): the start x_0 = V Lambda^-1 V^+ b and, with coarse,
// the coarse correction of the preconditioner.
struct DeflationInput {
  const char *V = nullptr;
  dwf_prec vprec = DWF_FP32;       // FP32 or FP16 (with scales)
  const double *lambda = nullptr;  // host [n_ev]
  int n_ev = 0;
  int coarse = 0;
};
dwf_status solve(dwf_ctx *ctx, void *x, const void *b, int nrhs, const double *mf,
                 const dwf_solver_params *prm, dwf_solve_info *info, cudaStream_t st,
                 const DeflationInput *defl = nullptr);

// Block-shape autotuner (csrc/autotune.cu).
std::vector<std::array<int, 4>> block_candidates(const int dims[4]);
std::string tune_key(const dwf_solver_params *p, int nrhs, const double *mf);
void autotune_block(dwf_ctx *ctx, const void *b, int nrhs, const double *mf,
                    const dwf_solver_params *prm, int trial, int block_out[4],
                    double *predicted, cudaStream_t st);

void prepare_kernels();

}  // namespace dwf

// Arguments of the vector-update and reduction kernels (blas.cu).
#pragma once

#include "dwf_internal.cuh"

namespace dwf {

// Outer solve (Algorithm 1): flat views of native fields, one rhs after another.
struct OuterArgs {
  const char *b64 = nullptr;  // FP64 right-hand side
  char *r64 = nullptr;        // FP64 residual
  char *x64 = nullptr;        // FP64 solution accumulator
  const char *Ax64 = nullptr; // FP64 A x for the reliable update
  char *xlo = nullptr, *rlo = nullptr, *p = nullptr, *Ap = nullptr, *z = nullptr;
  long long rs64 = 0, rslo = 0;  // bytes between right-hand sides
  long long n4 = 0;              // groups of 4 reals per right-hand side
  long long cs = 0;              // elements per chunk plane: Vh * Ls
  OuterScalars *scal = nullptr;
  double *partials = nullptr;    // [rhs][gridDim.x]
  unsigned int *counters = nullptr;  // [rhs]
  const int *skip = nullptr;
  int plain = 0;                 // 1: z = r (no preconditioner)
  int flexible = 0;              // 1: Polak-Ribiere beta = -alpha <Ap, z_new> / <r, z>
};

// Inner block CG (k iterations on every block at once).
struct BlockArgs {
  FieldRef r, p, Ap;  // inner precision, block layout
  FieldRef x;         // FP32, block layout
  const char *rglob = nullptr;  // native global even field (FP32, or FP64 with gfp64)
  char *zglob = nullptr;
  int gfp64 = 0;                // global fields are FP64 (FP64 outer solver)
  const char *apglob = nullptr; // flexible PCG: global A p, for <A p, z>
  double *apz_out = nullptr;    // apz_out[rhs * rz_rstride]
  double *gpart2 = nullptr;     // second reduction of the scatter: [rhs][nblocks * tiles]
  unsigned int *gcount2 = nullptr;
  long long grs = 0;            // global rhs stride
  int gcs = 0;                  // global elements per chunk plane: Vh * Ls
  const int *gmap = nullptr;    // [nblocks][n_b] global half index
  int n_b = 0, Ls = 0, nblocks = 0;
  double *rr = nullptr, *rr_new = nullptr, *pAp = nullptr;  // [rhs][nblocks]
  double *partials = nullptr;       // [rhs][nblocks][tiles]
  unsigned int *counters = nullptr; // [rhs][nblocks]
  double *gpart = nullptr;          // [rhs][nblocks * tiles]
  unsigned int *gcount = nullptr;   // [rhs]
  double *rz_out = nullptr;         // rz_out[rhs * rz_rstride]
  int rz_rstride = 0;
  const int *skip = nullptr;
  // inner residual stop (tol2 > 0): a block stops iterating once its |r|^2
  // fell to tol2 times its initial rr0; bstop[rhs][block] marks it, and the
  // block operator's hops skip it
  double tol2 = 0.0;
  double *rr0 = nullptr;            // [rhs][nblocks]
  int *bstop = nullptr;             // [rhs][nblocks]
  unsigned int *iters = nullptr;    // [rhs]: block iterations done (all blocks)
};

void outer_init(dwf_prec lo, const OuterArgs &A, int nrhs, cudaStream_t st);
void outer_axpy_xr(dwf_prec lo, const OuterArgs &A, int nrhs, cudaStream_t st);
void outer_xpay_p(dwf_prec lo, const OuterArgs &A, int nrhs, cudaStream_t st);
void outer_copy_p(dwf_prec lo, const OuterArgs &A, int nrhs, cudaStream_t st);
void outer_promote(dwf_prec lo, const OuterArgs &A, int nrhs, cudaStream_t st);
void outer_ru_residual(dwf_prec lo, const OuterArgs &A, int nrhs, cudaStream_t st);
void outer_set_rz(const OuterArgs &A, int nrhs, cudaStream_t st);

// Device-driven outer loop (see blas.cu).
void solve_start(OuterScalars *scal, SolveCtl *ctl, int *skip_iter, const SolveCtl &init,
                 cudaStream_t st);
void solve_launch(SolveCtl *ctl, cudaStream_t st);
void solve_control(OuterScalars *scal, SolveCtl *ctl, int *skip_ru,
                   cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_ru,
                   cudaStream_t st);
void solve_post_ru(OuterScalars *scal, SolveCtl *ctl, const int *skip_ru, int *skip_iter,
                   cudaGraphConditionalHandle h_loop, cudaStream_t st);
int outer_ctas();

void block_gather(dwf_prec in, const BlockArgs &B, int nrhs, cudaStream_t st);
void block_xr(dwf_prec in, const BlockArgs &B, int last, int nrhs, cudaStream_t st);
void block_p(dwf_prec in, const BlockArgs &B, int nrhs, cudaStream_t st);
void block_scatter(const BlockArgs &B, int nrhs, cudaStream_t st);
void block_export(dwf_prec in, const BlockArgs &B, const FieldRef &src, int nrhs,
                  cudaStream_t st);
int block_tiles(int n_b, int Ls);

}  // namespace dwf

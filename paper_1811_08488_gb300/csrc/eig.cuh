// Low modes of the normal operator and deflation of the outer solve (eig.cu).
#pragma once

#include "dwf_internal.cuh"

namespace dwf {

constexpr int kMaxEig = DWF_MAX_EIG;

// n native fields of one precision, `vs` bytes apart (FP16: the scales at
// byte offset soff within each field).
struct VecSet {
  const char *p = nullptr;
  long long vs = 0;
  int n = 0;
  dwf_prec prec = DWF_FP32;
  long long soff = 0;
};

// Reduction scratch of the multi-dot kernel (the counters reset themselves).
struct DotScratch {
  double *partials = nullptr;
  unsigned int *counters = nullptr;
};
size_t dot_scratch_bytes();
DotScratch dot_scratch_at(char *base);  // in a buffer of dot_scratch_bytes()

// G[i * ldg + j] = <X_i, Y_j> = sum conj(X_i) Y_j over whole fields of cs
// elements (FP32 compensated sums per thread, FP64 across threads, in a fixed
// order). X is FP32 (or FP16 against at most 4 Y), Y FP32 or FP64; at most
// kMaxEig vectors on either side.
void gram(const VecSet &X, const VecSet &Y, long long cs, double2 *G, int ldg,
          const DotScratch &w, cudaStream_t st);

// out_j = base_j + sum_i X_i C[i * ldc + j] wi[i] for j < nout (base and wi may
// be null; base may be out). X is FP32 or FP16; base and out have precision `oprec`
// (FP32 or FP64) and stride ovs. Outputs j with skip[j] set are not written.
void combine(const VecSet &X, const double2 *C, int ldc, const double *wi, const char *base,
             char *out, long long ovs, dwf_prec oprec, int nout, const int *skip, long long cs,
             cudaStream_t st);

// Low modes of A (schur = 0: D_PC^+ D_PC, 1: D_sym^+ D_sym) by Chebyshev-
// filtered subspace iteration; V holds m FP32 native fields (start vectors on
// entry, Ritz vectors in ascending order on return). Synchronous.
void eig_lowmodes(dwf_ctx *ctx, char *V, int m, double mf, const dwf_eig_params &p,
                  double *theta, double *resid, dwf_eig_info *info, cudaStream_t st);

// Deflation of the outer solve with n_ev Ritz pairs (V FP32 or FP16, lambda > 0).
struct Deflation {
  const char *V = nullptr;
  dwf_prec vprec = DWF_FP32;
  long long vs = 0;
  long long vsoff = 0;
  int n_ev = 0;
  int coarse = 0;             // 1: add V Lambda^-1 V^+ r to the preconditioner
  const double *inv_lam = nullptr;  // device [n_ev]
  double2 *c = nullptr;       // device [n_ev][nrhs]: V^+ r
  DotScratch dw;
};

// x64 = V Lambda^-1 V^+ b64 (FP64 fields, nrhs right-hand sides).
void deflate_start(const Deflation &d, const char *b64, char *x64, long long stride64, int nrhs,
                   long long cs, cudaStream_t st);
// z = (z_from_r ? r : z) + V Lambda^-1 V^+ r on fields of precision lo, and
// rz_new = (z_from_r ? rr : rz_new) + sum_j |<v_j, r>|^2 / lambda_j, which is
// <r, z> of the corrected z. Right-hand sides with skip set are left alone.
void deflate_correct(const Deflation &d, dwf_prec lo, const char *r, char *z, long long stride,
                     int nrhs, int z_from_r, OuterScalars *scal, const int *skip, long long cs,
                     cudaStream_t st);

// Native -> native precision conversion of nrhs half fields (fields.cu;
// dwf_field_convert, e.g. FP32 low modes to FP16).
void launch_convert(dwf_prec po, char *out, dwf_prec pi, const char *in, int nsite, int Ls,
                    int nrhs, cudaStream_t st);

}  // namespace dwf

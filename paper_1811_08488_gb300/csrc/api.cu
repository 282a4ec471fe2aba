// The C ABI (include/dwf.h): argument checks, context management, dispatch.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <vector>

#include "solver.cuh"

using dwf::DevBuf;
using dwf::Error;

static thread_local std::string g_create_error;

dwf_ctx::~dwf_ctx() {
  solver_plans.clear();
  block_plans.clear();
  if (own_stream) cudaStreamDestroy(own_stream);
}

// Every entry point on a context fails once a bounded device wait expired with
// device work possibly still in flight (the context must be destroyed).
#define API_TRY(ctx)                                                     \
  try {                                                                  \
    if ((ctx) && (ctx)->unusable)                                        \
      throw Error{DWF_ERR_TIMEOUT,                                       \
                  "the context is unusable after an expired device wait; destroy it"};
#define API_CATCH(ctx)                                                   \
  }                                                                      \
  catch (const Error &e) {                                               \
    if (ctx) (ctx)->last_error = e.msg;                                  \
    return e.code;                                                       \
  }                                                                      \
  catch (const std::exception &e) {                                      \
    if (ctx) (ctx)->last_error = e.what();                               \
    return DWF_ERR_CUDA;                                                 \
  }                                                                      \
  if (ctx) (ctx)->last_error.clear();                                    \
  return DWF_OK;

static void check_common(dwf_ctx *ctx, int nrhs, const double *mf) {
  DWF_REQUIRE(ctx, DWF_ERR_INVALID_ARG, "null context");
  DWF_REQUIRE(nrhs >= 1 && nrhs <= DWF_MAX_RHS, DWF_ERR_INVALID_ARG, "nrhs out of range");
  DWF_REQUIRE(mf != nullptr, DWF_ERR_INVALID_ARG, "null mass array");
  for (int r = 0; r < nrhs; ++r)
    DWF_REQUIRE(mf[r] == mf[r], DWF_ERR_INVALID_ARG, "NaN quark mass");
  DWF_CUDA_TRY(cudaSetDevice(ctx->device));
}

static void check_prec_op(dwf_prec p) {
  DWF_REQUIRE(p == DWF_FP64 || p == DWF_FP32, DWF_ERR_INVALID_ARG,
              "operator entry points take DWF_FP64 or DWF_FP32 fields");
}

extern "C" {

dwf_status dwf_create(dwf_ctx **out, int device, const dwf_action *a) {
  if (!out) return DWF_ERR_INVALID_ARG;
  *out = nullptr;
  dwf_ctx *ctx = nullptr;
  try {
    DWF_REQUIRE(a != nullptr, DWF_ERR_INVALID_ARG, "null action");
    for (int m = 0; m < 4; ++m)
      DWF_REQUIRE(a->dims[m] >= 2 && a->dims[m] % 2 == 0, DWF_ERR_INVALID_ARG,
                  "lattice extents must be even and >= 2");
    DWF_REQUIRE(a->Ls >= 2 && a->Ls <= DWF_MAX_LS, DWF_ERR_INVALID_ARG, "Ls out of range");
    DWF_REQUIRE(a->recon12 == 0 || a->recon12 == 1, DWF_ERR_INVALID_ARG,
                "recon12 must be 0 or 1");
    const double alpha = a->b * (4.0 - a->M5) + 1.0;
    DWF_REQUIRE(alpha != 0.0 && a->b == a->b && a->c == a->c, DWF_ERR_INVALID_ARG,
                "M_5 is singular for these b, M5");
    const long long v4 = (long long)a->dims[0] * a->dims[1] * a->dims[2] * a->dims[3];
    DWF_REQUIRE(v4 * a->Ls < (1LL << 31) / 8, DWF_ERR_INVALID_ARG, "lattice too large");
    int ndev = 0;
    DWF_CUDA_TRY(cudaGetDeviceCount(&ndev));
    DWF_REQUIRE(device >= 0 && device < ndev, DWF_ERR_INVALID_ARG, "no such device");
    DWF_CUDA_TRY(cudaSetDevice(device));
    ctx = new dwf_ctx();
    ctx->device = device;
    ctx->act = *a;
    dwf::build_geometry(ctx->geo, a->dims);
    for (int p = 0; p < 2; ++p) {
      ctx->nbr_dev[p].ensure(ctx->geo.nbr[p].size() * sizeof(int));
      DWF_CUDA_TRY(cudaMemcpy(ctx->nbr_dev[p].p, ctx->geo.nbr[p].data(),
                              ctx->geo.nbr[p].size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    DWF_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking));
    dwf::prepare_kernels();
    *out = ctx;
    return DWF_OK;
  } catch (const Error &e) {
    g_create_error = e.msg;
    delete ctx;
    return e.code;
  } catch (const std::exception &e) {
    g_create_error = e.what();
    delete ctx;
    return DWF_ERR_CUDA;
  }
}

void dwf_destroy(dwf_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  delete ctx;
}

const char *dwf_last_error(const dwf_ctx *ctx) {
  return ctx ? ctx->last_error.c_str() : g_create_error.c_str();
}

void dwf_solver_params_default(dwf_solver_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->tol = 1e-10;
  p->maxiter = 100000;
  p->inner_iters = 6;
  p->outer = DWF_FP32;
  p->inner = DWF_FP16;
  p->delta = 0.001;
  p->snake = 1;
  p->use_graph = 1;
  p->io_on_host = 0;
  p->check_every = 10;
  p->flexible = 0;
  p->schur = 0;
  p->inner_tol = 0.0;
}

void dwf_eig_params_default(dwf_eig_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->n_ev = 16;
  p->degree = 20;
  p->max_passes = 30;
  p->tol = 1e-6;
  p->lambda_max = 0.0;
  p->power_steps = 30;
  p->schur = 0;
}

dwf_status dwf_gauge_load(dwf_ctx *ctx, const double *U, int on_device) {
  API_TRY(ctx)
  DWF_REQUIRE(ctx && U, DWF_ERR_INVALID_ARG, "null context or gauge field");
  DWF_CUDA_TRY(cudaSetDevice(ctx->device));
  const size_t n = (size_t)ctx->geo.V4 * 4 * 18;
  DevBuf tmp;
  const double *src = U;
  if (!on_device) {
    tmp.ensure(n * sizeof(double));
    DWF_CUDA_TRY(cudaMemcpy(tmp.p, U, n * sizeof(double), cudaMemcpyHostToDevice));
    src = tmp.as<double>();
  }
  const size_t nrec = (size_t)ctx->geo.V4 * 4;
  const int rc = ctx->act.recon12;
  ctx->links[0].ensure(nrec * dwf::link_record_bytes(DWF_FP64));
  ctx->links[1].ensure(nrec * dwf::link_record_bytes(DWF_FP32, rc));
  ctx->links[2].ensure(nrec * dwf::link_record_bytes(DWF_FP16, rc));
  dwf::launch_pack_links(src, ctx->links[0].c(), ctx->links[1].c(), ctx->links[2].c(), rc,
                         ctx->act.dims, ctx->act.t_antiperiodic, nullptr);
  DWF_CUDA_TRY(cudaDeviceSynchronize());
  for (auto &kv : ctx->block_plans) kv.second->links_valid = false;
  ctx->have_gauge = true;
  API_CATCH(ctx)
}

size_t dwf_field_bytes(const dwf_ctx *ctx, dwf_prec prec, int nrhs) {
  if (!ctx || nrhs < 0) return 0;
  return dwf::field_rhs_bytes(prec, ctx->geo.Vh, ctx->act.Ls) * (size_t)nrhs;
}

dwf_status dwf_field_import(dwf_ctx *ctx, void *native_out, dwf_prec prec, const void *canon_in,
                            int canon_is_fp32, int nrhs, void *stream) {
  API_TRY(ctx)
  DWF_REQUIRE(ctx && native_out && canon_in, DWF_ERR_INVALID_ARG, "null argument");
  DWF_REQUIRE(nrhs >= 1 && nrhs <= DWF_MAX_RHS, DWF_ERR_INVALID_ARG, "nrhs out of range");
  DWF_CUDA_TRY(cudaSetDevice(ctx->device));
  dwf::launch_import(prec, (char *)native_out,
                     (long long)dwf::field_rhs_bytes(prec, ctx->geo.Vh, ctx->act.Ls), canon_in,
                     canon_is_fp32, ctx->geo.Vh, ctx->act.Ls, ctx->act.dims, nrhs,
                     (cudaStream_t)stream);
  API_CATCH(ctx)
}

dwf_status dwf_field_export(dwf_ctx *ctx, void *canon_out, int canon_is_fp32,
                            const void *native_in, dwf_prec prec, int nrhs, void *stream) {
  API_TRY(ctx)
  DWF_REQUIRE(ctx && native_in && canon_out, DWF_ERR_INVALID_ARG, "null argument");
  DWF_REQUIRE(nrhs >= 1 && nrhs <= DWF_MAX_RHS, DWF_ERR_INVALID_ARG, "nrhs out of range");
  DWF_CUDA_TRY(cudaSetDevice(ctx->device));
  dwf::launch_export(prec, canon_out, canon_is_fp32, (const char *)native_in,
                     (long long)dwf::field_rhs_bytes(prec, ctx->geo.Vh, ctx->act.Ls),
                     ctx->geo.Vh, ctx->act.Ls, ctx->act.dims, nrhs, (cudaStream_t)stream);
  API_CATCH(ctx)
}

dwf_status dwf_field_convert(dwf_ctx *ctx, void *native_out, dwf_prec out_prec,
                             const void *native_in, dwf_prec in_prec, int nrhs, void *stream) {
  API_TRY(ctx)
  DWF_REQUIRE(ctx && native_out && native_in, DWF_ERR_INVALID_ARG, "null argument");
  DWF_REQUIRE(native_out != native_in, DWF_ERR_INVALID_ARG, "aliased fields");
  DWF_REQUIRE(nrhs >= 1 && nrhs <= DWF_MAX_EIG, DWF_ERR_INVALID_ARG, "nrhs out of range");
  DWF_REQUIRE(out_prec >= DWF_FP64 && out_prec <= DWF_BF16 && in_prec >= DWF_FP64 &&
                  in_prec <= DWF_BF16,
              DWF_ERR_INVALID_ARG, "unknown precision");
  DWF_CUDA_TRY(cudaSetDevice(ctx->device));
  dwf::launch_convert(out_prec, (char *)native_out, in_prec, (const char *)native_in,
                      ctx->geo.Vh, ctx->act.Ls, nrhs, (cudaStream_t)stream);
  API_CATCH(ctx)
}

dwf_status dwf_dslash_eo(dwf_ctx *ctx, void *out, const void *in, int out_parity, int dagger,
                         dwf_prec prec, int nrhs, const double *mf, void *stream) {
  API_TRY(ctx)
  check_common(ctx, nrhs, mf);
  DWF_REQUIRE(prec >= DWF_FP64 && prec <= DWF_BF16, DWF_ERR_INVALID_ARG, "unknown precision");
  DWF_REQUIRE(out && in && out != in, DWF_ERR_INVALID_ARG, "null or aliased fields");
  DWF_REQUIRE(out_parity == 0 || out_parity == 1, DWF_ERR_INVALID_ARG, "parity must be 0 or 1");
  DWF_REQUIRE(ctx->have_gauge, DWF_ERR_NO_GAUGE, "no gauge field loaded");
  dwf::apply_dslash(ctx, out, in, out_parity, dagger ? 1 : 0, prec, nrhs, mf,
                    (cudaStream_t)stream);
  API_CATCH(ctx)
}

static dwf_status ls_entry(dwf_ctx *ctx, void *out, const void *in, int dagger, dwf_prec prec,
                           int nrhs, const double *mf, void *stream, bool inverse) {
  API_TRY(ctx)
  check_common(ctx, nrhs, mf);
  check_prec_op(prec);
  DWF_REQUIRE(out && in, DWF_ERR_INVALID_ARG, "null fields");
  dwf::LsCoef c[DWF_MAX_RHS];
  for (int r = 0; r < nrhs; ++r)
    c[r] = inverse ? dwf::coef_m5inv(ctx->act, mf[r], 1.0) : dwf::coef_m5(ctx->act, mf[r], 1.0);
  dwf::launch_ls_op(prec, (char *)out, (const char *)in,
                    (long long)dwf::field_rhs_bytes(prec, ctx->geo.Vh, ctx->act.Ls), ctx->geo.Vh,
                    ctx->act.Ls, dagger ? 1 : 0, inverse ? 1 : 0, nrhs, c, (cudaStream_t)stream);
  API_CATCH(ctx)
}

dwf_status dwf_m5(dwf_ctx *ctx, void *out, const void *in, int dagger, dwf_prec prec, int nrhs,
                  const double *mf, void *stream) {
  return ls_entry(ctx, out, in, dagger, prec, nrhs, mf, stream, false);
}

dwf_status dwf_m5inv(dwf_ctx *ctx, void *out, const void *in, int dagger, dwf_prec prec,
                     int nrhs, const double *mf, void *stream) {
  return ls_entry(ctx, out, in, dagger, prec, nrhs, mf, stream, true);
}

dwf_status dwf_m5inv_gemm(dwf_ctx *ctx, void *out, const void *in, int dagger, dwf_prec prec,
                          int nrhs, const double *mf, void *stream) {
  API_TRY(ctx)
  check_common(ctx, nrhs, mf);
  DWF_REQUIRE(prec >= DWF_FP64 && prec <= DWF_BF16, DWF_ERR_INVALID_ARG, "unknown precision");
  DWF_REQUIRE(out && in && out != in, DWF_ERR_INVALID_ARG, "null or aliased fields");
  dwf::launch_m5inv_gemm(ctx, prec, (char *)out, (const char *)in, dagger ? 1 : 0, nrhs, mf,
                         (cudaStream_t)stream);
  API_CATCH(ctx)
}

dwf_status dwf_mpc(dwf_ctx *ctx, void *out, const void *in, int dagger, dwf_prec prec, int nrhs,
                   const double *mf, void *stream) {
  API_TRY(ctx)
  check_common(ctx, nrhs, mf);
  check_prec_op(prec);
  DWF_REQUIRE(out && in && out != in, DWF_ERR_INVALID_ARG, "null or aliased fields");
  DWF_REQUIRE(ctx->have_gauge, DWF_ERR_NO_GAUGE, "no gauge field loaded");
  dwf::OpWork w = dwf::op_work(ctx, prec, nrhs);
  dwf::apply_mpc(ctx, out, in, dagger ? 1 : 0, prec, nrhs, mf, w, (cudaStream_t)stream);
  API_CATCH(ctx)
}

dwf_status dwf_mdagm(dwf_ctx *ctx, void *out, const void *in, dwf_prec prec, int nrhs,
                     const double *mf, void *stream) {
  API_TRY(ctx)
  check_common(ctx, nrhs, mf);
  check_prec_op(prec);
  DWF_REQUIRE(out && in && out != in, DWF_ERR_INVALID_ARG, "null or aliased fields");
  DWF_REQUIRE(ctx->have_gauge, DWF_ERR_NO_GAUGE, "no gauge field loaded");
  dwf::OpWork w = dwf::op_work(ctx, prec, nrhs);
  dwf::apply_mdagm(ctx, out, in, prec, nrhs, mf, w, nullptr, nullptr, (cudaStream_t)stream);
  API_CATCH(ctx)
}

dwf_status dwf_source_prep(dwf_ctx *ctx, void *b_even, const void *phi_even,
                           const void *phi_odd, dwf_prec prec, int nrhs, const double *mf,
                           void *stream) {
  API_TRY(ctx)
  check_common(ctx, nrhs, mf);
  check_prec_op(prec);
  DWF_REQUIRE(b_even && phi_even && phi_odd, DWF_ERR_INVALID_ARG, "null fields");
  DWF_REQUIRE(b_even != phi_even && b_even != phi_odd, DWF_ERR_INVALID_ARG, "aliased fields");
  DWF_REQUIRE(ctx->have_gauge, DWF_ERR_NO_GAUGE, "no gauge field loaded");
  dwf::OpWork w = dwf::op_work(ctx, prec, nrhs);
  dwf::apply_source_prep(ctx, b_even, phi_even, phi_odd, prec, nrhs, mf, w,
                         (cudaStream_t)stream);
  API_CATCH(ctx)
}

dwf_status dwf_mpc_sym(dwf_ctx *ctx, void *out, const void *in, int dagger, dwf_prec prec,
                       int nrhs, const double *mf, void *stream) {
  API_TRY(ctx)
  check_common(ctx, nrhs, mf);
  check_prec_op(prec);
  DWF_REQUIRE(out && in && out != in, DWF_ERR_INVALID_ARG, "null or aliased fields");
  DWF_REQUIRE(ctx->have_gauge, DWF_ERR_NO_GAUGE, "no gauge field loaded");
  dwf::OpWork w = dwf::op_work(ctx, prec, nrhs);
  dwf::apply_mpc_sym(ctx, out, in, dagger ? 1 : 0, prec, nrhs, mf, w, (cudaStream_t)stream);
  API_CATCH(ctx)
}

dwf_status dwf_mdagm_sym(dwf_ctx *ctx, void *out, const void *in, dwf_prec prec, int nrhs,
                         const double *mf, void *stream) {
  API_TRY(ctx)
  check_common(ctx, nrhs, mf);
  check_prec_op(prec);
  DWF_REQUIRE(out && in && out != in, DWF_ERR_INVALID_ARG, "null or aliased fields");
  DWF_REQUIRE(ctx->have_gauge, DWF_ERR_NO_GAUGE, "no gauge field loaded");
  dwf::OpWork w = dwf::op_work(ctx, prec, nrhs);
  dwf::apply_mdagm(ctx, out, in, prec, nrhs, mf, w, nullptr, nullptr, (cudaStream_t)stream, 1);
  API_CATCH(ctx)
}

dwf_status dwf_source_prep_sym(dwf_ctx *ctx, void *b_even, const void *phi_even,
                               const void *phi_odd, dwf_prec prec, int nrhs, const double *mf,
                               void *stream) {
  API_TRY(ctx)
  check_common(ctx, nrhs, mf);
  check_prec_op(prec);
  DWF_REQUIRE(b_even && phi_even && phi_odd, DWF_ERR_INVALID_ARG, "null fields");
  DWF_REQUIRE(b_even != phi_even && b_even != phi_odd, DWF_ERR_INVALID_ARG, "aliased fields");
  DWF_REQUIRE(ctx->have_gauge, DWF_ERR_NO_GAUGE, "no gauge field loaded");
  dwf::OpWork w = dwf::op_work(ctx, prec, nrhs);
  dwf::apply_source_prep_sym(ctx, b_even, phi_even, phi_odd, prec, nrhs, mf, w,
                             (cudaStream_t)stream);
  API_CATCH(ctx)
}

dwf_status dwf_odd_reconstruct(dwf_ctx *ctx, void *psi_odd, const void *psi_even,
                               const void *phi_odd, dwf_prec prec, int nrhs, const double *mf,
                               void *stream) {
  API_TRY(ctx)
  check_common(ctx, nrhs, mf);
  check_prec_op(prec);
  DWF_REQUIRE(psi_odd && psi_even && phi_odd, DWF_ERR_INVALID_ARG, "null fields");
  DWF_REQUIRE(psi_odd != psi_even && psi_odd != phi_odd, DWF_ERR_INVALID_ARG,
              "aliased fields");
  DWF_REQUIRE(ctx->have_gauge, DWF_ERR_NO_GAUGE, "no gauge field loaded");
  dwf::OpWork w = dwf::op_work(ctx, prec, nrhs);
  dwf::apply_odd_reconstruct(ctx, psi_odd, psi_even, phi_odd, prec, nrhs, mf, w,
                             (cudaStream_t)stream);
  API_CATCH(ctx)
}

// Name of the kernel behind profiler slot `slot` (role * 32 + prec * 8 + DAG * 4
// + PRE * 2 + EPI) in this context: hop2_kernel for FP32/FP16/BF16 with even
// Ls, hop_kernel otherwise; the template arguments as the kernel declares
// them, and " [block]" for launches of the block operator A_s.
static std::string prof_slot_name(const dwf_ctx *ctx, int slot) {
  static const char *kS[4] = {"F64", "F32", "F16", "BF16"};
  const int role = slot / 32;
  slot %= 32;
  const int p = slot / 8, dag = (slot >> 2) & 1, pre = (slot >> 1) & 1, epi = slot & 1;
  const int rc = (p != DWF_FP64 && ctx->act.recon12) ? 1 : 0;
  char buf[64];
  if (p != DWF_FP64 && ctx->act.Ls % 2 == 0)
    std::snprintf(buf, sizeof buf, "hop2_kernel<%s,%d,%d,%d,%d>", kS[p], dag, pre, rc, epi);
  else
    std::snprintf(buf, sizeof buf, "hop_kernel<%s,%d,%d,%d>%s", kS[p], dag, pre, rc,
                  epi ? " +Ls epilogue" : "");
  return std::string(buf) + (role ? " [block]" : "");
}

dwf_status dwf_profile_enable(dwf_ctx *ctx, int on) {
  if (!ctx) return DWF_ERR_INVALID_ARG;
  API_TRY(ctx)
  DWF_REQUIRE(on == 0 || on == 1, DWF_ERR_INVALID_ARG, "on must be 0 or 1");
  DWF_CUDA_TRY(cudaSetDevice(ctx->device));
  if (on) {
    ctx->prof.ensure(sizeof(dwf::KernProf) * dwf::kProfSlots);
    dwf::KernProf init[dwf::kProfSlots];
    std::memset(init, 0, sizeof init);
    DWF_CUDA_TRY(cudaDeviceSynchronize());
    DWF_CUDA_TRY(cudaMemcpy(ctx->prof.p, init, sizeof init, cudaMemcpyHostToDevice));
  }
  ctx->prof_on = on;
  API_CATCH(ctx)
}

dwf_status dwf_profile_read(dwf_ctx *ctx, dwf_kernel_time *out, int cap, int *n) {
  if (!ctx) return DWF_ERR_INVALID_ARG;
  API_TRY(ctx)
  DWF_REQUIRE(n != nullptr, DWF_ERR_INVALID_ARG, "null count");
  DWF_REQUIRE(cap >= 0 && (cap == 0 || out != nullptr), DWF_ERR_INVALID_ARG,
              "null output array");
  *n = 0;
  if (ctx->prof.p) {
    DWF_CUDA_TRY(cudaSetDevice(ctx->device));
    dwf::KernProf k[dwf::kProfSlots];
    DWF_CUDA_TRY(cudaDeviceSynchronize());
    DWF_CUDA_TRY(cudaMemcpy(k, ctx->prof.p, sizeof k, cudaMemcpyDeviceToHost));
    for (int s = 0; s < dwf::kProfSlots; ++s) {
      if (k[s].launches == 0) continue;
      if (*n < cap) {
        dwf_kernel_time &o = out[*n];
        std::memset(&o, 0, sizeof o);
        std::snprintf(o.name, sizeof o.name, "%s", prof_slot_name(ctx, s).c_str());
        o.launches = (long long)k[s].launches;
        o.seconds = (double)k[s].total_ns * 1e-9;
        o.alg_bytes = (double)k[s].bytes;
      }
      ++*n;
    }
  }
  API_CATCH(ctx)
}

static void check_params(const dwf_solver_params *p) {
  DWF_REQUIRE(p != nullptr, DWF_ERR_INVALID_ARG, "null solver parameters");
  DWF_REQUIRE(p->schur == 0 || p->schur == 1, DWF_ERR_INVALID_ARG, "schur must be 0 or 1");
  DWF_REQUIRE(p->inner_tol >= 0.0 && p->inner_tol < 1.0, DWF_ERR_INVALID_ARG,
              "inner_tol must be in [0, 1)");
}

dwf_status dwf_block_apply(dwf_ctx *ctx, void *out, const void *in,
                           const dwf_solver_params *params, int nrhs, const double *mf,
                           void *stream) {
  API_TRY(ctx)
  check_common(ctx, nrhs, mf);
  check_params(params);
  DWF_REQUIRE(out && in && out != in, DWF_ERR_INVALID_ARG, "null or aliased fields");
  DWF_REQUIRE(ctx->have_gauge, DWF_ERR_NO_GAUGE, "no gauge field loaded");
  cudaStream_t st = (cudaStream_t)stream;
  dwf::BlockPlan *bp = dwf::get_block_plan(ctx, params->block, params->inner, nrhs, st);
  dwf::BlockArgs B = dwf::block_args(ctx, bp, (char *)out, (const char *)in, nullptr, 0, nullptr);
  dwf::block_gather(bp->inner, B, nrhs, st);
  dwf::block_apply_A(ctx, bp, params->snake, nrhs, mf, false, nullptr, st, params->schur);
  dwf::block_export(bp->inner, B, bp->fAp, nrhs, st);
  API_CATCH(ctx)
}

dwf_status dwf_block_precond(dwf_ctx *ctx, void *z, const void *r,
                             const dwf_solver_params *params, int nrhs, const double *mf,
                             void *stream) {
  API_TRY(ctx)
  check_common(ctx, nrhs, mf);
  check_params(params);
  DWF_REQUIRE(z && r && z != r, DWF_ERR_INVALID_ARG, "null or aliased fields");
  DWF_REQUIRE(params->inner_iters >= 1, DWF_ERR_INVALID_ARG, "inner_iters must be >= 1");
  DWF_REQUIRE(ctx->have_gauge, DWF_ERR_NO_GAUGE, "no gauge field loaded");
  cudaStream_t st = (cudaStream_t)stream;
  dwf::BlockPlan *bp = dwf::get_block_plan(ctx, params->block, params->inner, nrhs, st);
  dwf::block_precondition(ctx, bp, (char *)z, (const char *)r, params->inner_iters,
                          params->snake, nrhs, mf, nullptr, 0, nullptr, st, DWF_FP32, nullptr,
                          nullptr, params->inner_tol, params->schur);
  API_CATCH(ctx)
}

dwf_status dwf_autotune_block(dwf_ctx *ctx, const void *b, int nrhs, const double *mf,
                              const dwf_solver_params *params, int trial, int block_out[4],
                              double *predicted_seconds, void *stream) {
  API_TRY(ctx)
  check_common(ctx, nrhs, mf);
  check_params(params);
  DWF_REQUIRE(b && block_out, DWF_ERR_INVALID_ARG, "null b or block_out");
  DWF_REQUIRE(ctx->have_gauge, DWF_ERR_NO_GAUGE, "no gauge field loaded");
  cudaStream_t st = stream ? (cudaStream_t)stream : ctx->own_stream;
  if (!stream) DWF_CUDA_TRY(cudaDeviceSynchronize());
  dwf::autotune_block(ctx, b, nrhs, mf, params, trial, block_out, predicted_seconds, st);
  API_CATCH(ctx)
}

static void check_lambda(const double *lambda, int n_ev) {
  DWF_REQUIRE(n_ev >= 1 && n_ev <= DWF_MAX_EIG, DWF_ERR_INVALID_ARG, "n_ev must be in 1 .. 64");
  DWF_REQUIRE(lambda != nullptr, DWF_ERR_INVALID_ARG, "null lambda");
  for (int j = 0; j < n_ev; ++j)
    DWF_REQUIRE(lambda[j] > 0 && std::isfinite(lambda[j]), DWF_ERR_INVALID_ARG,
                "every lambda must be positive and finite");
}

dwf_status dwf_eig_lowmodes(dwf_ctx *ctx, void *V, int m, double mf, const dwf_eig_params *p,
                            double *theta, double *resid, dwf_eig_info *info, void *stream) {
  API_TRY(ctx)
  DWF_REQUIRE(ctx && V && p && theta && resid, DWF_ERR_INVALID_ARG, "null argument");
  DWF_REQUIRE(m >= 1 && m <= DWF_MAX_EIG, DWF_ERR_INVALID_ARG, "m must be in 1 .. 64");
  DWF_REQUIRE(p->n_ev >= 1 && p->n_ev <= m, DWF_ERR_INVALID_ARG, "n_ev must be in 1 .. m");
  DWF_REQUIRE(p->degree >= 1 && p->max_passes >= 0 && p->power_steps >= 1, DWF_ERR_INVALID_ARG,
              "degree and power_steps must be >= 1, max_passes >= 0");
  DWF_REQUIRE(p->tol >= 0 && std::isfinite(p->tol) && std::isfinite(p->lambda_max),
              DWF_ERR_INVALID_ARG, "tol and lambda_max must be finite, tol >= 0");
  DWF_REQUIRE(p->schur == 0 || p->schur == 1, DWF_ERR_INVALID_ARG, "schur must be 0 or 1");
  DWF_REQUIRE(std::isfinite(mf), DWF_ERR_INVALID_ARG, "mass must be finite");
  DWF_REQUIRE(ctx->have_gauge, DWF_ERR_NO_GAUGE, "no gauge field loaded");
  cudaStream_t st = stream ? (cudaStream_t)stream : ctx->own_stream;
  if (!stream) DWF_CUDA_TRY(cudaDeviceSynchronize());
  dwf::eig_lowmodes(ctx, (char *)V, m, mf, *p, theta, resid, info, st);
  API_CATCH(ctx)
}

dwf_status dwf_deflate(dwf_ctx *ctx, void *z, const void *r, const void *V, dwf_prec vprec,
                       const double *lambda, int n_ev, dwf_prec prec, int nrhs, int accumulate,
                       void *stream) {
  API_TRY(ctx)
  DWF_REQUIRE(ctx && z && r && V, DWF_ERR_INVALID_ARG, "null argument");
  DWF_REQUIRE(z != r, DWF_ERR_INVALID_ARG, "z and r must not alias");
  DWF_REQUIRE(nrhs >= 1 && nrhs <= DWF_MAX_RHS, DWF_ERR_INVALID_ARG, "nrhs out of range");
  DWF_REQUIRE(prec == DWF_FP32 || prec == DWF_FP64, DWF_ERR_INVALID_ARG,
              "deflation fields must be FP32 or FP64");
  DWF_REQUIRE(vprec == DWF_FP32 || vprec == DWF_FP16, DWF_ERR_INVALID_ARG,
              "V must be FP32 or FP16");
  DWF_REQUIRE(nrhs <= 4 || vprec == DWF_FP32, DWF_ERR_UNSUPPORTED,
              "FP16 V serves at most 4 right-hand sides per call");
  check_lambda(lambda, n_ev);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t cbytes = dwf::align_up(sizeof(double2) * DWF_MAX_EIG * DWF_MAX_RHS, 256);
  const size_t lbytes = dwf::align_up(sizeof(double) * DWF_MAX_EIG, 256);
  if (!ctx->defl.p) {
    ctx->defl.ensure(cbytes + lbytes + dwf::dot_scratch_bytes());
    DWF_CUDA_TRY(cudaMemset(ctx->defl.p, 0, ctx->defl.bytes));
  }
  std::vector<double> inv(n_ev);
  for (int j = 0; j < n_ev; ++j) inv[j] = 1.0 / lambda[j];
  double2 *c = ctx->defl.as<double2>();
  double *inv_d = reinterpret_cast<double *>(ctx->defl.c() + cbytes);
  DWF_CUDA_TRY(cudaMemcpyAsync(inv_d, inv.data(), sizeof(double) * n_ev, cudaMemcpyHostToDevice,
                               st));
  const int Vh = ctx->geo.Vh, Ls = ctx->act.Ls;
  const long long cs = (long long)Vh * Ls;
  dwf::VecSet Vs, Rs;
  Vs.p = (const char *)V;
  Vs.vs = (long long)dwf::field_rhs_bytes(vprec, Vh, Ls);
  Vs.n = n_ev;
  Vs.prec = vprec;
  Vs.soff = (long long)dwf::align_up(dwf::field_data_bytes(vprec, Vh, Ls), 256);
  Rs.p = (const char *)r;
  Rs.vs = (long long)dwf::field_rhs_bytes(prec, Vh, Ls);
  Rs.n = nrhs;
  Rs.prec = prec;
  dwf::gram(Vs, Rs, cs, c, nrhs, dwf::dot_scratch_at(ctx->defl.c() + cbytes + lbytes), st);
  dwf::combine(Vs, c, nrhs, inv_d, accumulate ? (const char *)z : nullptr, (char *)z, Rs.vs, prec,
               nrhs, nullptr, cs, st);
  // the host array must outlive its copy
  DWF_CUDA_TRY(cudaStreamSynchronize(st));
  API_CATCH(ctx)
}

static dwf_status solve_entry(dwf_ctx *ctx, void *x, const void *b, int nrhs, const double *mf,
                              const dwf_solver_params *params, dwf_solve_info *info,
                              void *stream, const dwf::DeflationInput *defl);

dwf_status mspcg_solve(dwf_ctx *ctx, void *x, const void *b, int nrhs, const double *mf,
                       const dwf_solver_params *params, dwf_solve_info *info, void *stream) {
  return solve_entry(ctx, x, b, nrhs, mf, params, info, stream, nullptr);
}

dwf_status mspcg_solve_deflated(dwf_ctx *ctx, void *x, const void *b, int nrhs, const double *mf,
                                const dwf_solver_params *params, const void *V, dwf_prec vprec,
                                const double *lambda, int n_ev, int coarse,
                                dwf_solve_info *info, void *stream) {
  API_TRY(ctx)
  DWF_REQUIRE(ctx && V, DWF_ERR_INVALID_ARG, "null context or V");
  check_lambda(lambda, n_ev);
  DWF_REQUIRE(coarse == 0 || coarse == 1, DWF_ERR_INVALID_ARG, "coarse must be 0 or 1");
  DWF_REQUIRE(vprec == DWF_FP32 || vprec == DWF_FP16, DWF_ERR_INVALID_ARG,
              "V must be FP32 or FP16");
  DWF_REQUIRE(nrhs <= 4 || vprec == DWF_FP32, DWF_ERR_UNSUPPORTED,
              "FP16 V serves at most 4 right-hand sides per call");
  DWF_REQUIRE(!(coarse && params && params->flexible), DWF_ERR_UNSUPPORTED,
              "flexible PCG with the coarse correction is not supported");
  dwf::DeflationInput d;
  d.V = (const char *)V;
  d.vprec = vprec;
  d.lambda = lambda;
  d.n_ev = n_ev;
  d.coarse = coarse;
  return solve_entry(ctx, x, b, nrhs, mf, params, info, stream, &d);
  API_CATCH(ctx)
}

static dwf_status solve_entry(dwf_ctx *ctx, void *x, const void *b, int nrhs, const double *mf,
                              const dwf_solver_params *params, dwf_solve_info *info,
                              void *stream, const dwf::DeflationInput *defl) {
  API_TRY(ctx)
  check_common(ctx, nrhs, mf);
  check_params(params);
  DWF_REQUIRE(x && b, DWF_ERR_INVALID_ARG, "null x or b");
  DWF_REQUIRE(ctx->have_gauge, DWF_ERR_NO_GAUGE, "no gauge field loaded");
  DWF_REQUIRE(params->check_every >= 1 && params->check_every <= dwf::kHistory,
              DWF_ERR_INVALID_ARG, "check_every must be in 1 .. 256");
  DWF_REQUIRE(params->delta > 0 && params->delta < 1, DWF_ERR_INVALID_ARG,
              "delta must be in (0, 1)");
  cudaStream_t st = stream ? (cudaStream_t)stream : ctx->own_stream;
  if (!stream) DWF_CUDA_TRY(cudaDeviceSynchronize());
  dwf_solver_params p = *params;
  if (p.inner_iters > 0 && !p.block[0] && !p.block[1] && !p.block[2] && !p.block[3]) {
    // block = {0, 0, 0, 0}: the autotuner's shape for these parameters
    auto it = ctx->tuned_blocks.find(dwf::tune_key(&p, nrhs, mf));
    if (it == ctx->tuned_blocks.end()) {
      int blk[4];
      dwf::autotune_block(ctx, b, nrhs, mf, &p, 20, blk, nullptr, st);
      for (int i = 0; i < 4; ++i) p.block[i] = blk[i];
    } else {
      for (int i = 0; i < 4; ++i) p.block[i] = it->second[i];
    }
  }
  dwf_status s = dwf::solve(ctx, x, b, nrhs, mf, &p, info, st, defl);
  if (s != DWF_OK) {
    ctx->last_error = s == DWF_ERR_NOT_CONVERGED ? "not converged within maxiter"
                      : s == DWF_ERR_NAN         ? "NaN or Inf in a solver scalar"
                                                 : "solver error";
    return s;
  }
  API_CATCH(ctx)
}

}  // extern "C"

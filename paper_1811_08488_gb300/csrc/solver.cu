// Operator composition, the multisplitting preconditioner and the outer
// preconditioned CG driver (paper Sec. 2.2-2.4, Algorithm 1).
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <sstream>

#include "solver.cuh"

namespace dwf {

static int prec_index(dwf_prec p) { return p == DWF_FP64 ? 0 : (p == DWF_FP32 ? 1 : 2); }

FieldRef global_ref(const dwf_ctx *ctx, dwf_prec p, const void *ptr) {
  FieldRef f;
  f.data = const_cast<char *>(static_cast<const char *>(ptr));
  f.rstride = (long long)field_rhs_bytes(p, ctx->geo.Vh, ctx->act.Ls);
  f.scale_off = (long long)align_up(field_data_bytes(p, ctx->geo.Vh, ctx->act.Ls), 256);
  f.cs = ctx->geo.Vh * ctx->act.Ls;
  return f;
}

const char *link_ptr(const dwf_ctx *ctx, dwf_prec p) { return ctx->links[prec_index(p)].c(); }

OpWork op_work(dwf_ctx *ctx, dwf_prec p, int nrhs) {
  const size_t rs = field_rhs_bytes(p, ctx->geo.Vh, ctx->act.Ls);
  DevBuf &t = ctx->tmp[p];
  t.ensure(3 * rs * nrhs);
  OpWork w;
  w.u = t.c();
  w.y = t.c() + rs * nrhs;
  w.v = t.c() + 2 * rs * nrhs;
  w.rstride = (long long)rs;
  return w;
}

// Compulsory bytes of one hop launch: every output, input (and added x or
// dot vector) element once, and the links of the output and input sites.
static unsigned long long hop_alg_bytes(dwf_prec p, const HopParams &P, int nrhs) {
  const unsigned long long eb = p == DWF_FP64 ? 192 : p == DWF_FP32 ? 96 : 52;
  const unsigned long long lb = (P.recon ? 12 : 18) * (p == DWF_FP64 ? 8 : p == DWF_FP32 ? 4 : 2);
  const unsigned long long elems = (unsigned long long)P.n_out + P.in_limit +
                                   (P.has_x ? P.xown_limit : 0) + (P.dot ? P.n_out : 0);
  return (unsigned long long)P.nblocks *
         (elems * P.Ls * eb * nrhs + ((unsigned long long)P.n_out + P.in_limit) * 4 * lb);
}

static void launch(dwf_ctx *ctx, dwf_prec p, const HopParams &P0, int dag, int pre, int nrhs,
                   cudaStream_t st) {
  HopParams P = P0;
  if (ctx->prof_on) {
    P.prof = ctx->prof.as<KernProf>() + P.role * 32 + (int)p * 8 + dag * 4 + pre * 2 +
             (P.epi ? 1 : 0);
    P.alg_bytes = hop_alg_bytes(p, P, nrhs);
  }
  switch (p) {
    case DWF_FP64: launch_hop<F64>(P, dag, pre, nrhs, st); break;
    case DWF_FP32: launch_hop<F32>(P, dag, pre, nrhs, st); break;
    case DWF_FP16: launch_hop<F16>(P, dag, pre, nrhs, st); break;
    case DWF_BF16: launch_hop<BF16>(P, dag, pre, nrhs, st); break;
  }
}

static double alpha_of(const dwf_action &a) { return a.b * (4.0 - a.M5) + 1.0; }
static double beta_of(const dwf_action &a) { return a.c * (4.0 - a.M5) - 1.0; }

static void with_pre(LsCoef &c, const dwf_action &a) {
  c.pre_b = a.b;
  c.pre_c = a.c;
}

static HopParams global_params(const dwf_ctx *ctx, dwf_prec p, int out_parity, const void *in,
                               void *out) {
  HopParams P;
  P.in = global_ref(ctx, p, in);
  P.out = global_ref(ctx, p, out);
  P.links = link_ptr(ctx, p);
  P.link_cs = ctx->geo.V4;
  P.recon = (p != DWF_FP64 && ctx->act.recon12) ? 1 : 0;
  P.nbr = ctx->nbr_dev[out_parity].as<int>();
  P.n_out = ctx->geo.Vh;
  P.in_limit = ctx->geo.Vh;
  P.xown_limit = ctx->geo.Vh;
  P.out_link_off = out_parity * ctx->geo.Vh;
  P.in_link_off = (1 - out_parity) * ctx->geo.Vh;
  P.Ls = ctx->act.Ls;
  P.nblocks = 1;
  return P;
}

// M^4 (dagger = 0): -1/2 Dhop M_phi; (M^4)^+: -1/2 M_phi^+ Dhop^+ (Sec. 2.2).
void apply_dslash(dwf_ctx *ctx, void *out, const void *in, int out_parity, int dagger,
                  dwf_prec p, int nrhs, const double *mf, cudaStream_t st) {
  HopParams P = global_params(ctx, p, out_parity, in, out);
  const dwf_action &a = ctx->act;
  for (int r = 0; r < nrhs; ++r) {
    if (!dagger) {
      P.coef[r] = coef_identity(-0.5);
      P.coef[r].mf = mf[r];
      with_pre(P.coef[r], a);
    } else {
      P.coef[r] = coef_mphi(a, mf[r], -0.5);
    }
  }
  P.epi = dagger ? 1 : 0;
  launch(ctx, p, P, dagger, dagger ? 0 : 1, nrhs, st);
}

// First half of D_PC (or D_PC^+): u(odd) = K (-1/2 Dhop M_phi in) with
// K = M_phi M_5^-1, or v(odd) = K^+ (-1/2 Dhop^+ in) with K^+ = M_5^-+ M_phi^+.
static void mpc_first(dwf_ctx *ctx, void *odd_out, const void *in, int dagger, dwf_prec p,
                      int nrhs, const double *mf, const int *skip, cudaStream_t st) {
  HopParams P = global_params(ctx, p, 1, in, odd_out);
  for (int r = 0; r < nrhs; ++r) {
    P.coef[r] = coef_k(ctx->act, mf[r], -0.5);
    if (!dagger) with_pre(P.coef[r], ctx->act);
  }
  P.epi = 1;
  P.inv = 1;
  P.skip = skip;
  launch(ctx, p, P, dagger, dagger ? 0 : 1, nrhs, st);
}

// Second half: out(even) = M_5 in + 1/2 Dhop u, or M_5^+ in + 1/2 M_phi^+ Dhop^+ v.
// The symmetric form (schur = 1): out = in + M_5^-1 (1/2 Dhop u), or
// in + 1/2 M_phi^+ Dhop^+ v.
static void mpc_second(dwf_ctx *ctx, void *out, const void *odd_in, const void *in, int dagger,
                       dwf_prec p, int nrhs, const double *mf, const DotSpec *dot,
                       const int *skip, cudaStream_t st, int schur = 0) {
  HopParams P = global_params(ctx, p, 0, odd_in, out);
  P.xown = global_ref(ctx, p, in);
  const dwf_action &a = ctx->act;
  for (int r = 0; r < nrhs; ++r) {
    if (schur && !dagger)
      P.coef[r] = coef_m5inv(a, mf[r], 0.5);
    else
      P.coef[r] = dagger ? coef_mphi(a, mf[r], 0.5) : coef_identity(0.5);
    P.coef[r].mf = mf[r];
    P.coef[r].a0 = schur ? 1.0 : alpha_of(a);
    P.coef[r].a1 = schur ? 0.0 : beta_of(a);
  }
  P.inv = (schur && !dagger) ? 1 : 0;
  P.epi = 1;
  P.has_x = 1;
  P.skip = skip;
  if (dot) {
    P.dot = 1;
    P.dotv = global_ref(ctx, p, dot->dotv);
    P.partials = dot->partials;
    P.counters = dot->counters;
    P.dot_out = dot->dot_out;
    P.dot_rstride = dot->dot_rstride;
  }
  launch(ctx, p, P, dagger, 0, nrhs, st);
}

void apply_mpc(dwf_ctx *ctx, void *out, const void *in, int dagger, dwf_prec p, int nrhs,
               const double *mf, const OpWork &w, cudaStream_t st) {
  char *odd = dagger ? w.v : w.u;
  mpc_first(ctx, odd, in, dagger, p, nrhs, mf, nullptr, st);
  mpc_second(ctx, out, odd, in, dagger, p, nrhs, mf, nullptr, nullptr, st);
}

// out = M_5^-1 in or M_5^-+ in on even fields (one Ls pass).
static void m5inv_pass(dwf_ctx *ctx, void *out, const void *in, int dagger, dwf_prec p, int nrhs,
                       const double *mf, cudaStream_t st) {
  LsCoef c[kMaxRhs];
  for (int r = 0; r < nrhs; ++r) c[r] = coef_m5inv(ctx->act, mf[r], 1.0);
  launch_ls_op(p, static_cast<char *>(out), static_cast<const char *>(in),
               (long long)field_rhs_bytes(p, ctx->geo.Vh, ctx->act.Ls), ctx->geo.Vh, ctx->act.Ls,
               dagger, 1, nrhs, c, st);
}

// D_sym in = in - M_5^-1 M^4_eo M_5^-1 M^4_oe in (odd temporary odd_tmp), or
// D_sym^+ in = in - (M^4_oe)^+ M_5^-+ (M^4_eo)^+ M_5^-+ in (with the even
// temporary even_tmp for M_5^-+ in as well).
static void mpc_sym(dwf_ctx *ctx, void *out, const void *in, int dagger, dwf_prec p, int nrhs,
                    const double *mf, char *odd_tmp, char *even_tmp, const DotSpec *dot,
                    const int *skip, cudaStream_t st) {
  const void *hop_in = in;
  if (dagger) {
    m5inv_pass(ctx, even_tmp, in, 1, p, nrhs, mf, st);
    hop_in = even_tmp;
  }
  mpc_first(ctx, odd_tmp, hop_in, dagger, p, nrhs, mf, skip, st);
  mpc_second(ctx, out, odd_tmp, in, dagger, p, nrhs, mf, dot, skip, st, 1);
}

void apply_mpc_sym(dwf_ctx *ctx, void *out, const void *in, int dagger, dwf_prec p, int nrhs,
                   const double *mf, const OpWork &w, cudaStream_t st) {
  mpc_sym(ctx, out, in, dagger, p, nrhs, mf, w.u, w.v, nullptr, nullptr, st);
}

// b = D_sym^+ M_5^-1 phi_hat_e: the right-hand side of the symmetric form's
// normal equation for D psi = phi.
void apply_source_prep_sym(dwf_ctx *ctx, void *b_even, const void *phi_even, const void *phi_odd,
                           dwf_prec p, int nrhs, const double *mf, const OpWork &w,
                           cudaStream_t st) {
  // phi_hat_e -> w.y (w.u is used on the way)
  const int Vh = ctx->geo.Vh, Ls = ctx->act.Ls;
  LsCoef c[kMaxRhs];
  for (int r = 0; r < nrhs; ++r) c[r] = coef_k(ctx->act, mf[r], 1.0);
  launch_ls_op(p, w.u, static_cast<const char *>(phi_odd), (long long)field_rhs_bytes(p, Vh, Ls),
               Vh, Ls, 0, 1, nrhs, c, st);
  HopParams P = global_params(ctx, p, 0, w.u, w.y);
  P.xown = global_ref(ctx, p, phi_even);
  for (int r = 0; r < nrhs; ++r) {
    P.coef[r] = coef_identity(0.5);
    P.coef[r].mf = mf[r];
    P.coef[r].a0 = 1.0;
    P.coef[r].a1 = 0.0;
  }
  P.epi = 1;
  P.has_x = 1;
  launch(ctx, p, P, 0, 0, nrhs, st);
  m5inv_pass(ctx, w.v, w.y, 0, p, nrhs, mf, st);       // q = M_5^-1 phi_hat_e
  mpc_sym(ctx, b_even, w.v, 1, p, nrhs, mf, w.u, w.y, nullptr, nullptr, st);
}

// Right-hand side of the normal equation for the full system D psi = phi
// (Sec. 2.2): phi_hat_e = phi_e - M^4_eo M_5^-1 phi_o, b = D_PC^+ phi_hat_e.
// u = M_phi M_5^-1 phi_o (one Ls pass), then phi_hat_e = phi_e + 1/2 Dhop u
// (the hop with phi_e added in its epilogue), then D_PC^+.
void apply_source_prep(dwf_ctx *ctx, void *b_even, const void *phi_even, const void *phi_odd,
                       dwf_prec p, int nrhs, const double *mf, const OpWork &w,
                       cudaStream_t st) {
  const int Vh = ctx->geo.Vh, Ls = ctx->act.Ls;
  LsCoef c[kMaxRhs];
  for (int r = 0; r < nrhs; ++r) c[r] = coef_k(ctx->act, mf[r], 1.0);
  launch_ls_op(p, w.u, static_cast<const char *>(phi_odd), (long long)field_rhs_bytes(p, Vh, Ls),
               Vh, Ls, 0, 1, nrhs, c, st);
  HopParams P = global_params(ctx, p, 0, w.u, w.y);
  P.xown = global_ref(ctx, p, phi_even);
  for (int r = 0; r < nrhs; ++r) {
    P.coef[r] = coef_identity(0.5);
    P.coef[r].mf = mf[r];
    P.coef[r].a0 = 1.0;
    P.coef[r].a1 = 0.0;
  }
  P.epi = 1;
  P.has_x = 1;
  launch(ctx, p, P, 0, 0, nrhs, st);
  apply_mpc(ctx, b_even, w.y, 1, p, nrhs, mf, w, st);
}

// The odd half of the solution of D psi = phi (Sec. 2.2):
// psi_o = M_5^-1 (phi_o - M^4_oe psi_e) = M_5^-1 (phi_o + 1/2 Dhop M_phi psi_e).
void apply_odd_reconstruct(dwf_ctx *ctx, void *psi_odd, const void *psi_even,
                           const void *phi_odd, dwf_prec p, int nrhs, const double *mf,
                           const OpWork &w, cudaStream_t st) {
  const int Vh = ctx->geo.Vh, Ls = ctx->act.Ls;
  HopParams P = global_params(ctx, p, 1, psi_even, w.u);
  P.xown = global_ref(ctx, p, phi_odd);
  for (int r = 0; r < nrhs; ++r) {
    P.coef[r] = coef_identity(0.5);
    P.coef[r].mf = mf[r];
    with_pre(P.coef[r], ctx->act);
    P.coef[r].a0 = 1.0;
    P.coef[r].a1 = 0.0;
  }
  P.epi = 1;
  P.has_x = 1;
  launch(ctx, p, P, 0, 1, nrhs, st);
  LsCoef c[kMaxRhs];
  for (int r = 0; r < nrhs; ++r) c[r] = coef_m5inv(ctx->act, mf[r], 1.0);
  launch_ls_op(p, static_cast<char *>(psi_odd), w.u, (long long)field_rhs_bytes(p, Vh, Ls), Vh,
               Ls, 0, 1, nrhs, c, st);
}

void apply_mdagm(dwf_ctx *ctx, void *out, const void *in, dwf_prec p, int nrhs,
                 const double *mf, const OpWork &w, const DotSpec *dot, const int *skip,
                 cudaStream_t st, int schur) {
  if (schur) {
    // D_sym^+ D_sym: y = D_sym in, then D_sym^+ y with the dot against in
    DotSpec d;
    if (dot) {
      d = *dot;
      d.dotv = static_cast<const char *>(in);
    }
    mpc_sym(ctx, w.y, in, 0, p, nrhs, mf, w.u, nullptr, nullptr, skip, st);
    mpc_sym(ctx, out, w.y, 1, p, nrhs, mf, w.u, w.v, dot ? &d : nullptr, skip, st);
    return;
  }
  mpc_first(ctx, w.u, in, 0, p, nrhs, mf, skip, st);
  mpc_second(ctx, w.y, w.u, in, 0, p, nrhs, mf, nullptr, skip, st);
  mpc_first(ctx, w.v, w.y, 1, p, nrhs, mf, skip, st);
  DotSpec d;
  if (dot) {
    d = *dot;
    d.dotv = static_cast<const char *>(in);
  }
  mpc_second(ctx, out, w.v, w.y, 1, p, nrhs, mf, dot ? &d : nullptr, skip, st);
}

// ---------------------------------------------------------------------------
// Block plan
// ---------------------------------------------------------------------------
static FieldRef block_ref(const DevBuf &buf, dwf_prec p, int nsite, int Ls, int nblocks) {
  FieldRef f;
  f.data = buf.c();
  f.bstride = (long long)field_rhs_bytes(p, nsite, Ls);
  f.rstride = f.bstride * nblocks;
  f.scale_off = (p == DWF_FP16 || p == DWF_BF16)
                    ? (long long)align_up(field_data_bytes(p, nsite, Ls), 256)
                    : 0;
  f.cs = nsite * Ls;
  return f;
}

BlockPlan *get_block_plan(dwf_ctx *ctx, const int block[4], dwf_prec inner, int nrhs,
                          cudaStream_t st) {
  DWF_REQUIRE(inner == DWF_FP32 || inner == DWF_FP16 || inner == DWF_BF16, DWF_ERR_INVALID_ARG,
              "inner precision must be FP32, FP16 or BF16");
  std::ostringstream key;
  key << block[0] << "x" << block[1] << "x" << block[2] << "x" << block[3] << "/" << inner;
  auto &slot = ctx->block_plans[key.str()];
  const int Ls = ctx->act.Ls;
  if (!slot) {
    auto bp = std::make_unique<BlockPlan>();
    build_block_geometry(bp->bg, ctx->act.dims, block);
    bp->inner = inner;
    bp->Ls = Ls;
    const BlockGeometry &g = bp->bg;
    auto up = [&](DevBuf &d, const std::vector<int> &h) {
      d.ensure(h.size() * sizeof(int));
      DWF_CUDA_TRY(cudaMemcpy(d.p, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice));
    };
    up(bp->nbr_oe, g.nbr_oe);
    up(bp->nbr_eo, g.nbr_eo);
    up(bp->gmap_b, g.gmap_b);
    std::vector<int> own(g.gsite.size());
    const int *L = ctx->act.dims;
    for (size_t i = 0; i < own.size(); ++i) {
      const int s = g.gsite[i];
      const int x = s % L[0], y = (s / L[0]) % L[1], z = (s / (L[0] * L[1])) % L[2],
                t = s / (L[0] * L[1] * L[2]);
      own[i] = ((x + y + z + t) & 1) * ctx->geo.Vh + (s >> 1);
    }
    up(bp->gowner, own);
    slot = std::move(bp);
  }
  BlockPlan *bp = slot.get();
  const BlockGeometry &g = bp->bg;
  if (!bp->links_valid) {
    const dwf_prec lp = inner == DWF_FP32 ? DWF_FP32 : DWF_FP16;
    bp->link_bstride = (long long)g.n_comb * 4 * (long long)link_record_bytes(lp, ctx->act.recon12);
    bp->links.ensure((size_t)bp->link_bstride * g.nblocks);
    launch_block_links(lp, ctx->act.recon12, bp->links.c(), ctx->links[1].c(), ctx->links[2].c(),
                       bp->gowner.as<int>(), g.n_comb, g.nblocks, ctx->act.dims, st);
    bp->links_valid = true;
  }
  if (bp->nrhs < nrhs) {
    const int nb = g.nblocks;
    auto alloc = [&](DevBuf &d, FieldRef &f, dwf_prec p, int nsite) {
      d.ensure(field_rhs_bytes(p, nsite, Ls) * nb * nrhs);
      f = block_ref(d, p, nsite, Ls, nb);
    };
    alloc(bp->r, bp->fr, inner, g.n_b);
    alloc(bp->p, bp->fp, inner, g.n_b);
    alloc(bp->Ap, bp->fAp, inner, g.n_b);
    alloc(bp->x, bp->fx, DWF_FP32, g.n_b);
    alloc(bp->u1, bp->fu1, inner, g.n_o1);
    alloc(bp->u2, bp->fu2, inner, g.n_o1);
    alloc(bp->y, bp->fy, inner, g.n_e2);
    alloc(bp->w2, bp->fw2, inner, g.n_e2);
    bp->scal.ensure(sizeof(double) * 5 * nrhs * nb + 64);
    bp->bstop.ensure(sizeof(int) * nrhs * nb);
    DWF_CUDA_TRY(cudaMemset(bp->bstop.p, 0, bp->bstop.bytes));
    bp->iters.ensure(sizeof(unsigned int) * nrhs);
    DWF_CUDA_TRY(cudaMemset(bp->iters.p, 0, bp->iters.bytes));
    const int sites = hop_sites_per_cta(Ls, inner);
    const int tiles = std::max((g.n_b + sites - 1) / sites, block_tiles(g.n_b, Ls));
    bp->partials.ensure(sizeof(double) * (size_t)nrhs * nb * tiles);
    bp->counters.ensure(sizeof(unsigned int) * nrhs * nb);
    DWF_CUDA_TRY(cudaMemset(bp->counters.p, 0, bp->counters.bytes));
    bp->gpart.ensure(sizeof(double) * (size_t)nrhs * nb * block_tiles(g.n_b, Ls));
    bp->gcount.ensure(sizeof(unsigned int) * nrhs);
    DWF_CUDA_TRY(cudaMemset(bp->gcount.p, 0, bp->gcount.bytes));
    bp->gpart2.ensure(sizeof(double) * (size_t)nrhs * nb * block_tiles(g.n_b, Ls));
    bp->gcount2.ensure(sizeof(unsigned int) * nrhs);
    DWF_CUDA_TRY(cudaMemset(bp->gcount2.p, 0, bp->gcount2.bytes));
    bp->nrhs = nrhs;
  }
  return bp;
}

// The block operator A_s = P_s D_PC^+ D_PC P_s on every block at once (Sec. 2.3).
// The even output of D_PC P_s lives on the block's even sites within distance
// 2 (n_e2), the odd intermediates within distance 1 (n_o1). With snake = 0
// every hop is restricted to the block instead (the truncated operator).
void block_apply_A(dwf_ctx *ctx, BlockPlan *bp, int snake, int nrhs, const double *mf,
                   bool with_dot, const int *skip, cudaStream_t st, int schur) {
  const BlockGeometry &g = bp->bg;
  const dwf_action &a = ctx->act;
  HopParams base;
  base.links = bp->links.c();
  base.link_bstride = bp->link_bstride;
  base.link_cs = g.n_comb;
  base.recon = ctx->act.recon12 ? 1 : 0;
  base.Ls = bp->Ls;
  base.nblocks = g.nblocks;
  base.skip = skip;
  base.bskip = bp->stop_active ? bp->bstop.as<int>() : nullptr;
  base.epi = 1;
  base.role = 1;
  const int odd_out = snake ? g.n_o1 : g.n_ob;
  const int even_mid = snake ? g.n_e2 : g.n_b;
  const int odd_in = snake ? g.n_o1 : g.n_ob;

  // hop 1: odd (distance <= 1) <- even block sites; u1 = K (-1/2 Dhop M_phi p)
  HopParams P = base;
  P.in = bp->fp;
  P.out = bp->fu1;
  P.nbr = bp->nbr_oe.as<int>();
  P.n_out = odd_out;
  P.in_limit = g.n_b;
  P.out_link_off = g.n_e2;
  P.in_link_off = 0;
  P.inv = 1;
  for (int r = 0; r < nrhs; ++r) {
    P.coef[r] = coef_k(a, mf[r], -0.5);
    with_pre(P.coef[r], a);
  }
  launch(ctx, bp->inner, P, 0, 1, nrhs, st);

  // hop 2: even (distance <= 2) <- odd; y = M_5 p + 1/2 Dhop u1  (= D_PC P_s p),
  // or y = p + M_5^-1 (1/2 Dhop u1) (= D_sym P_s p)
  P = base;
  P.in = bp->fu1;
  P.out = bp->fy;
  P.nbr = bp->nbr_eo.as<int>();
  P.n_out = even_mid;
  P.in_limit = odd_in;
  P.out_link_off = 0;
  P.in_link_off = g.n_e2;
  P.has_x = 1;
  P.xown = bp->fp;
  P.xown_limit = g.n_b;
  for (int r = 0; r < nrhs; ++r) {
    P.coef[r] = schur ? coef_m5inv(a, mf[r], 0.5) : coef_identity(0.5);
    P.coef[r].mf = mf[r];
    P.coef[r].a0 = schur ? 1.0 : alpha_of(a);
    P.coef[r].a1 = schur ? 0.0 : beta_of(a);
  }
  P.inv = schur ? 1 : 0;
  launch(ctx, bp->inner, P, 0, 0, nrhs, st);

  // symmetric form: w = M_5^-+ y on the even distance-2 region of every block
  // (one Ls pass over the block-local fields, blocks taken as right-hand sides)
  if (schur) {
    LsCoef c[kMaxRhs];
    for (int r = 0; r < nrhs; ++r) c[r] = coef_m5inv(a, mf[r], 1.0);
    launch_ls_op(bp->inner, bp->w2.c(), bp->y.c(), bp->fy.bstride, even_mid, bp->Ls, 1, 1, nrhs,
                 c, st, g.nblocks);
  }

  // hop 3: odd (distance <= 1) <- even (distance <= 2); u2 = K^+ (-1/2 Dhop^+ y)
  // (y replaced by w in the symmetric form)
  P = base;
  P.in = schur ? bp->fw2 : bp->fy;
  P.out = bp->fu2;
  P.nbr = bp->nbr_oe.as<int>();
  P.n_out = odd_out;
  P.in_limit = even_mid;
  P.out_link_off = g.n_e2;
  P.in_link_off = 0;
  P.inv = 1;
  for (int r = 0; r < nrhs; ++r) P.coef[r] = coef_k(a, mf[r], -0.5);
  launch(ctx, bp->inner, P, 1, 0, nrhs, st);

  // hop 4: even block sites <- odd; Ap = M_5^+ y + 1/2 M_phi^+ Dhop^+ u2
  // (y + 1/2 M_phi^+ Dhop^+ u2 in the symmetric form)
  P = base;
  P.in = bp->fu2;
  P.out = bp->fAp;
  P.nbr = bp->nbr_eo.as<int>();
  P.n_out = g.n_b;
  P.in_limit = odd_in;
  P.out_link_off = 0;
  P.in_link_off = g.n_e2;
  P.has_x = 1;
  P.xown = bp->fy;
  P.xown_limit = g.n_b;
  for (int r = 0; r < nrhs; ++r) {
    P.coef[r] = coef_mphi(a, mf[r], 0.5);
    P.coef[r].a0 = schur ? 1.0 : alpha_of(a);
    P.coef[r].a1 = schur ? 0.0 : beta_of(a);
  }
  if (with_dot) {
    P.dot = 1;
    P.dotv = bp->fp;
    P.partials = bp->partials.as<double>();
    P.counters = bp->counters.as<unsigned int>();
    P.dot_out = bp->scal.as<double>() + 2 * (size_t)bp->nrhs * g.nblocks;  // pAp
    P.dot_rstride = g.nblocks;
  }
  launch(ctx, bp->inner, P, 1, 0, nrhs, st);
}

BlockArgs block_args(dwf_ctx *ctx, BlockPlan *bp, char *z, const char *r, double *rz_out,
                     int rz_rstride, const int *skip, dwf_prec glob) {
  const BlockGeometry &g = bp->bg;
  BlockArgs B;
  B.r = bp->fr;
  B.p = bp->fp;
  B.Ap = bp->fAp;
  B.x = bp->fx;
  B.rglob = r;
  B.zglob = z;
  DWF_REQUIRE(glob == DWF_FP32 || glob == DWF_FP64, DWF_ERR_INVALID_ARG,
              "the preconditioner takes FP32 or FP64 global fields");
  B.gfp64 = glob == DWF_FP64 ? 1 : 0;
  B.grs = (long long)field_rhs_bytes(glob, ctx->geo.Vh, ctx->act.Ls);
  B.gcs = ctx->geo.Vh * ctx->act.Ls;
  B.gmap = bp->gmap_b.as<int>();
  B.n_b = g.n_b;
  B.Ls = bp->Ls;
  B.nblocks = g.nblocks;
  double *sc = bp->scal.as<double>();
  const size_t n = (size_t)bp->nrhs * g.nblocks;
  B.rr = sc;
  B.rr_new = sc + n;
  B.pAp = sc + 2 * n;
  B.partials = bp->partials.as<double>();
  B.counters = bp->counters.as<unsigned int>();
  B.gpart = bp->gpart.as<double>();
  B.gcount = bp->gcount.as<unsigned int>();
  B.gpart2 = bp->gpart2.as<double>();
  B.gcount2 = bp->gcount2.as<unsigned int>();
  B.rz_out = rz_out ? rz_out : sc + 3 * n;  // scratch slot when unused
  B.rz_rstride = rz_out ? rz_rstride : 0;
  B.skip = skip;
  B.rr0 = sc + 4 * n;
  B.iters = bp->iters.as<unsigned int>();
  return B;
}

// z = M^-1 r (Sec. 2.4): gather r into the blocks, k CG iterations on A_s with
// block-local scalars from a zero guess, scatter the block solutions.
void block_precondition(dwf_ctx *ctx, BlockPlan *bp, char *z, const char *r, int k, int snake,
                        int nrhs, const double *mf, double *rz_out, int rz_rstride,
                        const int *skip, cudaStream_t st, dwf_prec glob, const char *ap,
                        double *apz_out, double inner_tol, int schur) {
  BlockArgs B = block_args(ctx, bp, z, r, rz_out, rz_rstride, skip, glob);
  if (ap && apz_out) {
    B.apglob = ap;
    B.apz_out = apz_out;
  }
  // inner residual stop: a block stops once |r_s| <= inner_tol |r_s(0)| (at
  // most k iterations); its later launches return at entry
  bp->stop_active = inner_tol > 0.0;
  if (bp->stop_active) {
    B.tol2 = inner_tol * inner_tol;
    B.bstop = bp->bstop.as<int>();
  }
  block_gather(bp->inner, B, nrhs, st);
  for (int it = 0; it < k; ++it) {
    block_apply_A(ctx, bp, snake, nrhs, mf, true, skip, st, schur);
    const int last = it == k - 1;
    block_xr(bp->inner, B, last, nrhs, st);
    if (!last) block_p(bp->inner, B, nrhs, st);
  }
  block_scatter(B, nrhs, st);
  bp->stop_active = false;
}

// ---------------------------------------------------------------------------
// Outer solve
// ---------------------------------------------------------------------------
void SolverPlan::drop_graphs() {
  if (loop) cudaGraphExecDestroy(loop);
  loop = nullptr;
  loop_key.clear();
}

SolverPlan::~SolverPlan() {
  drop_graphs();
  if (host_scal) cudaFreeHost(host_scal);
  if (host_skip) cudaFreeHost(host_skip);
  if (host_ctl) cudaFreeHost(host_ctl);
}

static SolverPlan *get_solver_plan(dwf_ctx *ctx, dwf_prec lo, int nrhs) {
  std::ostringstream key;
  key << lo << "/" << nrhs;
  auto &slot = ctx->solver_plans[key.str()];
  if (slot) return slot.get();
  auto sp = std::make_unique<SolverPlan>();
  sp->lo = lo;
  sp->nrhs = nrhs;
  const int Vh = ctx->geo.Vh, Ls = ctx->act.Ls;
  const size_t f64 = field_rhs_bytes(DWF_FP64, Vh, Ls) * nrhs;
  const size_t flo = field_rhs_bytes(lo, Vh, Ls) * nrhs;
  sp->b64.ensure(f64);
  sp->x64.ensure(f64);
  sp->r64.ensure(f64);
  sp->Ax64.ensure(f64);
  sp->xlo.ensure(flo);
  sp->rlo.ensure(flo);
  sp->p.ensure(flo);
  sp->Ap.ensure(flo);
  sp->z.ensure(flo);
  sp->wlo.ensure(3 * flo);
  sp->w64.ensure(3 * f64);
  sp->scal.ensure(sizeof(OuterScalars) * nrhs);
  DWF_CUDA_TRY(cudaMemset(sp->scal.p, 0, sp->scal.bytes));
  sp->partials.ensure(sizeof(double) * outer_ctas() * nrhs);
  sp->counters.ensure(sizeof(unsigned int) * nrhs);
  DWF_CUDA_TRY(cudaMemset(sp->counters.p, 0, sp->counters.bytes));
  const int tiles = (Vh + hop_sites_per_cta(Ls, lo) - 1) / hop_sites_per_cta(Ls, lo);
  sp->opart.ensure(sizeof(double) * (size_t)tiles * nrhs);
  sp->ocount.ensure(sizeof(unsigned int) * nrhs);
  DWF_CUDA_TRY(cudaMemset(sp->ocount.p, 0, sp->ocount.bytes));
  sp->skip_iter.ensure(sizeof(int) * nrhs);
  sp->skip_ru.ensure(sizeof(int) * nrhs);
  sp->ctl.ensure(sizeof(SolveCtl));
  DWF_CUDA_TRY(cudaMallocHost(&sp->host_ctl, sizeof(SolveCtl)));
  DWF_CUDA_TRY(cudaMallocHost(&sp->host_scal, sizeof(OuterScalars) * nrhs));
  DWF_CUDA_TRY(cudaMallocHost(&sp->host_skip, sizeof(int) * 2 * nrhs));
  slot = std::move(sp);
  return slot.get();
}

struct SolveSetup {
  dwf_ctx *ctx;
  SolverPlan *sp;
  BlockPlan *bp;
  const dwf_solver_params *prm;
  const double *mf;
  int nrhs;
  OuterArgs A;
  OpWork wlo, w64;
  DotSpec dot;
  const Deflation *defl = nullptr;
};

// The coarse correction of the deflated preconditioner after z = M^-1 r (or
// z = r + ... for plain CG, whose z is otherwise r itself).
static void enqueue_coarse(SolveSetup &S, const int *skip, cudaStream_t st) {
  if (!S.defl || !S.defl->coarse) return;
  SolverPlan *sp = S.sp;
  deflate_correct(*S.defl, sp->lo, sp->rlo.c(), sp->z.c(), S.A.rslo, S.nrhs,
                  S.prm->inner_iters == 0 ? 1 : 0, sp->scal.as<OuterScalars>(), skip, S.A.cs,
                  st);
}

static OpWork work_from(const DevBuf &d, dwf_prec p, const dwf_ctx *ctx, int nrhs) {
  const size_t rs = field_rhs_bytes(p, ctx->geo.Vh, ctx->act.Ls);
  OpWork w;
  w.u = d.c();
  w.y = d.c() + rs * nrhs;
  w.v = d.c() + 2 * rs * nrhs;
  w.rstride = (long long)rs;
  return w;
}

// One outer iteration of Algorithm 1.
static void enqueue_iteration(SolveSetup &S, cudaStream_t st) {
  SolverPlan *sp = S.sp;
  const int *skip = sp->skip_iter.as<int>();
  OuterArgs A = S.A;
  A.skip = skip;
  apply_mdagm(S.ctx, sp->Ap.p, sp->p.p, sp->lo, S.nrhs, S.mf, S.wlo, &S.dot, skip, st,
              S.prm->schur);
  outer_axpy_xr(sp->lo, A, S.nrhs, st);
  if (S.bp)
    block_precondition(S.ctx, S.bp, sp->z.c(), sp->rlo.c(), S.prm->inner_iters, S.prm->snake,
                       S.nrhs, S.mf, &sp->scal.as<OuterScalars>()->rz_new,
                       (int)(sizeof(OuterScalars) / sizeof(double)), skip, st, sp->lo,
                       A.flexible ? sp->Ap.c() : nullptr,
                       A.flexible ? &sp->scal.as<OuterScalars>()->apz : nullptr,
                       S.prm->inner_tol, S.prm->schur);
  enqueue_coarse(S, skip, st);
  outer_xpay_p(sp->lo, A, S.nrhs, st);
}

// Reliable update for the right-hand sides not masked by skip_ru: fold x_lo into
// the FP64 solution, recompute r = b - A x in FP64, restart r_lo (and z) from it.
static void enqueue_reliable_update(SolveSetup &S, cudaStream_t st) {
  SolverPlan *sp = S.sp;
  const int *skip = sp->skip_ru.as<int>();
  OuterArgs A = S.A;
  A.skip = skip;
  outer_promote(sp->lo, A, S.nrhs, st);
  apply_mdagm(S.ctx, sp->Ax64.p, sp->x64.p, DWF_FP64, S.nrhs, S.mf, S.w64, nullptr, skip, st,
              S.prm->schur);
  outer_ru_residual(sp->lo, A, S.nrhs, st);
  if (!A.plain) {
    if (S.bp)
      block_precondition(S.ctx, S.bp, sp->z.c(), sp->rlo.c(), S.prm->inner_iters, S.prm->snake,
                         S.nrhs, S.mf, &sp->scal.as<OuterScalars>()->rz_new,
                         (int)(sizeof(OuterScalars) / sizeof(double)), skip, st, sp->lo,
                         nullptr, nullptr, S.prm->inner_tol, S.prm->schur);
    enqueue_coarse(S, skip, st);
    outer_set_rz(A, S.nrhs, st);
  }
}

// The last node of a graph captured from one stream.
static cudaGraphNode_t sink_of(cudaGraph_t g) {
  size_t n = 0;
  DWF_CUDA_TRY(cudaGraphGetNodes(g, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  DWF_CUDA_TRY(cudaGraphGetNodes(g, nodes.data(), &n));
  std::vector<cudaGraphNode_t> sinks;
  for (cudaGraphNode_t nd : nodes) {
    size_t m = 0;
    DWF_CUDA_TRY(cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &m));
    if (m == 0) sinks.push_back(nd);
  }
  DWF_REQUIRE(sinks.size() == 1, DWF_ERR_CUDA, "a captured graph body has no single last node");
  return sinks[0];
}

// Capture the work that fn() enqueues on st into the empty graph g.
template <class F>
static void capture_into(cudaGraph_t g, cudaStream_t st, F fn) {
  DWF_CUDA_TRY(cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
  try {
    fn();
  } catch (...) {
    cudaGraph_t tmp;
    cudaStreamEndCapture(st, &tmp);
    throw;
  }
  cudaGraph_t out;
  DWF_CUDA_TRY(cudaStreamEndCapture(st, &out));
}

// The device-driven outer loop as one executable graph:
//   reset the launch's iteration count;
//   while (h_loop) {
//     one outer iteration of Algorithm 1 (all right-hand sides);
//     control: per right-hand side, reliable update needed? loop on? (h_ru, h_loop)
//     if (h_ru) { reliable update of those right-hand sides; mark the converged }
//   }
static void build_loop_graph(SolveSetup &S, cudaStream_t st) {
  SolverPlan *sp = S.sp;
  SolveCtl *ctl = sp->ctl.as<SolveCtl>();
  OuterScalars *scal = sp->scal.as<OuterScalars>();
  int *skip_ru = sp->skip_ru.as<int>(), *skip_iter = sp->skip_iter.as<int>();
  cudaGraph_t top;
  DWF_CUDA_TRY(cudaGraphCreate(&top, 0));
  try {
    cudaGraphConditionalHandle h_loop;
    DWF_CUDA_TRY(cudaGraphConditionalHandleCreate(&h_loop, top, 1, cudaGraphCondAssignDefault));
    capture_into(top, st, [&] { solve_launch(ctl, st); });
    cudaGraphNode_t head = sink_of(top);
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = h_loop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    DWF_CUDA_TRY(cudaGraphAddNode(&wnode, top, &head, nullptr, 1, &wp));
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    cudaGraphConditionalHandle h_ru;
    DWF_CUDA_TRY(cudaGraphConditionalHandleCreate(&h_ru, body, 0, cudaGraphCondAssignDefault));
    capture_into(body, st, [&] {
      enqueue_iteration(S, st);
      solve_control(scal, ctl, skip_ru, h_loop, h_ru, st);
    });
    cudaGraphNode_t last = sink_of(body);
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = h_ru;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t inode;
    DWF_CUDA_TRY(cudaGraphAddNode(&inode, body, &last, nullptr, 1, &ip));
    cudaGraph_t rbody = ip.conditional.phGraph_out[0];
    capture_into(rbody, st, [&] {
      enqueue_reliable_update(S, st);
      solve_post_ru(scal, ctl, skip_ru, skip_iter, h_loop, st);
    });
    DWF_CUDA_TRY(cudaGraphInstantiate(&sp->loop, top, 0));
  } catch (...) {
    cudaGraphDestroy(top);
    throw;
  }
  cudaGraphDestroy(top);
}

// Compulsory bytes and device nanoseconds summed over the hop-kernel timer
// slots of the whole-lattice operators in precision p (zero when the timer is
// off). Waits for the work queued on st.
static void outer_hop_totals(dwf_ctx *ctx, dwf_prec p, cudaStream_t st, double &bytes,
                             double &ns) {
  bytes = ns = 0.0;
  if (!ctx->prof_on || !ctx->prof.p) return;
  KernProf k[8];
  DWF_CUDA_TRY(cudaStreamSynchronize(st));
  DWF_CUDA_TRY(cudaMemcpy(k, ctx->prof.as<KernProf>() + (int)p * 8, sizeof k,
                          cudaMemcpyDeviceToHost));
  for (const KernProf &q : k) {
    bytes += (double)q.bytes;
    ns += (double)q.total_ns;
  }
}

dwf_status solve(dwf_ctx *ctx, void *x, const void *b, int nrhs, const double *mf,
                 const dwf_solver_params *prm, dwf_solve_info *info, cudaStream_t st,
                 const DeflationInput *dfin) {
  const auto t0 = std::chrono::steady_clock::now();
  double hop_bytes0, hop_ns0;
  outer_hop_totals(ctx, prm->outer, st, hop_bytes0, hop_ns0);
  const dwf_prec lo = prm->outer;
  DWF_REQUIRE(lo == DWF_FP32 || lo == DWF_FP64, DWF_ERR_INVALID_ARG,
              "outer precision must be FP64 or FP32");
  DWF_REQUIRE(prm->tol > 0 && prm->maxiter > 0 && prm->inner_iters >= 0, DWF_ERR_INVALID_ARG,
              "tol, maxiter and inner_iters must be positive");
  const bool coarse = dfin && dfin->n_ev > 0 && dfin->coarse;
  // plain CG keeps z = r unless the coarse correction makes z its own vector
  const bool plain = prm->inner_iters == 0 && !coarse;
  SolverPlan *sp = get_solver_plan(ctx, lo, nrhs);
  BlockPlan *bp = prm->inner_iters == 0
                      ? nullptr
                      : get_block_plan(ctx, prm->block, prm->inner, nrhs, st);
  const int Vh = ctx->geo.Vh, Ls = ctx->act.Ls;

  SolveSetup S{ctx, sp, bp, prm, mf, nrhs};
  Deflation defl;
  if (dfin && dfin->n_ev > 0) {
    DWF_REQUIRE(dfin->n_ev <= kMaxEig && dfin->V && dfin->lambda, DWF_ERR_INVALID_ARG,
                "deflation: 1 .. 64 Ritz pairs with V and lambda");
    const size_t cbytes = align_up(sizeof(double2) * kMaxEig * kMaxRhs, 256);
    const size_t lbytes = align_up(sizeof(double) * kMaxEig, 256);
    if (!sp->defl.p) {
      sp->defl.ensure(cbytes + lbytes + dot_scratch_bytes());
      DWF_CUDA_TRY(cudaMemsetAsync(sp->defl.p, 0, sp->defl.bytes, st));
    }
    std::vector<double> inv(dfin->n_ev);
    for (int j = 0; j < dfin->n_ev; ++j) {
      DWF_REQUIRE(dfin->lambda[j] > 0 && std::isfinite(dfin->lambda[j]), DWF_ERR_INVALID_ARG,
                  "deflation: every lambda must be positive and finite");
      inv[j] = 1.0 / dfin->lambda[j];
    }
    DWF_REQUIRE(dfin->vprec == DWF_FP32 || dfin->vprec == DWF_FP16, DWF_ERR_INVALID_ARG,
                "deflation: V must be FP32 or FP16");
    defl.V = dfin->V;
    defl.vprec = dfin->vprec;
    defl.vs = (long long)field_rhs_bytes(dfin->vprec, Vh, Ls);
    defl.vsoff = (long long)align_up(field_data_bytes(dfin->vprec, Vh, Ls), 256);
    defl.n_ev = dfin->n_ev;
    defl.coarse = coarse ? 1 : 0;
    defl.c = sp->defl.as<double2>();
    defl.inv_lam = reinterpret_cast<const double *>(sp->defl.c() + cbytes);
    defl.dw = dot_scratch_at(sp->defl.c() + cbytes + lbytes);
    DWF_CUDA_TRY(cudaMemcpyAsync(const_cast<double *>(defl.inv_lam), inv.data(),
                                 sizeof(double) * dfin->n_ev, cudaMemcpyHostToDevice, st));
    // the host vector must outlive the copy
    DWF_CUDA_TRY(cudaStreamSynchronize(st));
    S.defl = &defl;
  }
  OuterArgs &A = S.A;
  A.b64 = sp->b64.c();
  A.r64 = sp->r64.c();
  A.x64 = sp->x64.c();
  A.Ax64 = sp->Ax64.c();
  A.xlo = sp->xlo.c();
  A.rlo = sp->rlo.c();
  A.p = sp->p.c();
  A.Ap = sp->Ap.c();
  A.z = sp->z.c();
  A.rs64 = (long long)field_rhs_bytes(DWF_FP64, Vh, Ls);
  A.rslo = (long long)field_rhs_bytes(lo, Vh, Ls);
  A.n4 = (long long)Vh * Ls * 6;
  A.cs = (long long)Vh * Ls;
  A.scal = sp->scal.as<OuterScalars>();
  A.partials = sp->partials.as<double>();
  A.counters = sp->counters.as<unsigned int>();
  A.plain = plain ? 1 : 0;
  A.flexible = (!plain && prm->flexible) ? 1 : 0;
  S.wlo = work_from(sp->wlo, lo, ctx, nrhs);
  S.w64 = work_from(sp->w64, DWF_FP64, ctx, nrhs);
  S.dot.partials = sp->opart.as<double>();
  S.dot.counters = sp->ocount.as<unsigned int>();
  S.dot.dot_out = &sp->scal.as<OuterScalars>()->pAp;
  S.dot.dot_rstride = (int)(sizeof(OuterScalars) / sizeof(double));

  // inputs
  if (prm->io_on_host) {
    const size_t cbytes = (size_t)Vh * Ls * 24 * sizeof(double) * nrhs;
    DWF_CUDA_TRY(cudaMemcpyAsync(sp->Ax64.p, b, cbytes, cudaMemcpyHostToDevice, st));
    launch_import(DWF_FP64, sp->b64.c(), A.rs64, sp->Ax64.p, 0, Vh, Ls, ctx->act.dims, nrhs, st);
  } else {
    launch_import(DWF_FP64, sp->b64.c(), A.rs64, b, 0, Vh, Ls, ctx->act.dims, nrhs, st);
  }
  int *hs_iter = sp->host_skip, *hs_ru = sp->host_skip + nrhs;
  for (int r = 0; r < nrhs; ++r) hs_iter[r] = hs_ru[r] = 0;
  DWF_CUDA_TRY(cudaMemcpyAsync(sp->skip_iter.p, hs_iter, sizeof(int) * nrhs,
                               cudaMemcpyHostToDevice, st));
  DWF_CUDA_TRY(cudaMemcpyAsync(sp->skip_ru.p, hs_ru, sizeof(int) * nrhs, cudaMemcpyHostToDevice,
                               st));
  DWF_CUDA_TRY(cudaMemsetAsync(sp->x64.p, 0, sp->x64.bytes, st));
  DWF_CUDA_TRY(cudaMemsetAsync(sp->xlo.p, 0, sp->xlo.bytes, st));
  if (bp) DWF_CUDA_TRY(cudaMemsetAsync(bp->iters.p, 0, bp->iters.bytes, st));
  outer_init(lo, A, nrhs, st);
  if (S.defl) {
    // deflated start: x_0 = V Lambda^-1 V^+ b, r_0 = b - A x_0 in FP64
    deflate_start(*S.defl, sp->b64.c(), sp->x64.c(), A.rs64, nrhs, A.cs, st);
    apply_mdagm(ctx, sp->Ax64.p, sp->x64.p, DWF_FP64, nrhs, mf, S.w64, nullptr, nullptr, st,
                prm->schur);
    outer_ru_residual(lo, A, nrhs, st);
  }
  if (!plain) {
    if (bp)
      block_precondition(ctx, bp, sp->z.c(), sp->rlo.c(), prm->inner_iters, prm->snake, nrhs,
                         mf, &sp->scal.as<OuterScalars>()->rz_new,
                         (int)(sizeof(OuterScalars) / sizeof(double)), nullptr, st, lo, nullptr,
                         nullptr, prm->inner_tol, prm->schur);
    enqueue_coarse(S, nullptr, st);
    outer_set_rz(A, nrhs, st);
  }
  outer_copy_p(lo, A, nrhs, st);

  // The outer loop. With a capturing stream (use_graph) it runs on the device:
  // one CUDA graph holds a while-loop over the outer iteration, whose control
  // kernel decides the reliable updates and convergence of every right-hand
  // side after each iteration (an if-node runs the reliable update); the host
  // only waits for the graph launch to end and reads the scalars. Otherwise
  // the host drives the loop with eager launches, checking every few
  // iterations.
  const bool device_loop = prm->use_graph != 0 && st != nullptr;
  const double tol2 = prm->tol * prm->tol;
  std::vector<double> final_res(nrhs, -1.0);
  std::vector<int> done(nrhs, 0), nru(nrhs, 0);
  int host_syncs = 0;
  dwf_status status = DWF_OK;
  if (device_loop) {
    std::ostringstream key;
    key << (void *)bp << "/" << (bp ? bp->r.p : nullptr) << "/" << prm->inner_iters << "/"
        << prm->snake << "/" << plain << "/" << A.flexible << "/" << ctx->prof_on << "/"
        << (S.defl ? (const void *)S.defl->V : nullptr) << "/" << (S.defl ? S.defl->n_ev : 0)
        << "/" << (S.defl ? (int)S.defl->vprec : -1)
        << "/" << coarse;
    for (int r = 0; r < nrhs; ++r) key << "/" << mf[r];
    if (!sp->loop || sp->loop_key != key.str()) {
      sp->drop_graphs();
      build_loop_graph(S, st);
      sp->loop_key = key.str();
    }
    SolveCtl init{};
    init.tol2 = tol2;
    init.delta = prm->delta;
    init.maxiter = prm->maxiter;
    init.budget = kHistory;
    init.nrhs = nrhs;
    solve_start(sp->scal.as<OuterScalars>(), sp->ctl.as<SolveCtl>(), sp->skip_iter.as<int>(),
                init, st);
    while (true) {
      DWF_CUDA_TRY(cudaGraphLaunch(sp->loop, st));
      DWF_CUDA_TRY(cudaMemcpyAsync(sp->host_scal, sp->scal.p, sizeof(OuterScalars) * nrhs,
                                   cudaMemcpyDeviceToHost, st));
      DWF_CUDA_TRY(cudaMemcpyAsync(sp->host_ctl, sp->ctl.p, sizeof(SolveCtl),
                                   cudaMemcpyDeviceToHost, st));
      DWF_CUDA_TRY(cudaStreamSynchronize(st));
      ++host_syncs;
      if (sp->host_ctl->nan) {
        status = DWF_ERR_NAN;
        break;
      }
      int open = 0, itmax = 0;
      for (int r = 0; r < nrhs; ++r)
        if (!sp->host_scal[r].done) {
          ++open;
          itmax = std::max(itmax, sp->host_scal[r].iter);
        }
      if (!open || itmax >= prm->maxiter) break;
    }
    for (int r = 0; r < nrhs; ++r) {
      const OuterScalars &q = sp->host_scal[r];
      done[r] = q.done;
      nru[r] = q.nru;
      if (q.done) final_res[r] = q.final_res;
      hs_iter[r] = q.done;
    }
  } else {
    DWF_CUDA_TRY(cudaMemcpyAsync(sp->host_scal, sp->scal.p, sizeof(OuterScalars) * nrhs,
                                 cudaMemcpyDeviceToHost, st));
    DWF_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<double> bb(nrhs), maxr(nrhs);
    std::vector<int> seen(nrhs, 0);
    for (int r = 0; r < nrhs; ++r) {
      bb[r] = sp->host_scal[r].bb;
      maxr[r] = std::sqrt(sp->host_scal[r].rr);
      if (bb[r] == 0.0) {  // zero source: x = 0 is exact
        done[r] = 1;
        final_res[r] = 0.0;
        hs_iter[r] = 1;
      }
    }
    const bool debug = std::getenv("DWF_DEBUG") != nullptr;
    int chunk = std::max(1, std::min(prm->check_every, 8));
    int total_iters = 0;
    while (true) {
      int active = 0;
      for (int r = 0; r < nrhs; ++r) active += !done[r];
      if (!active) break;
      if (total_iters >= prm->maxiter) {
        status = DWF_ERR_NOT_CONVERGED;
        break;
      }
      DWF_CUDA_TRY(cudaMemcpyAsync(sp->skip_iter.p, hs_iter, sizeof(int) * nrhs,
                                   cudaMemcpyHostToDevice, st));
      const int n = std::min(chunk, prm->maxiter - total_iters);
      for (int i = 0; i < n; ++i) enqueue_iteration(S, st);
      total_iters += n;
      DWF_CUDA_TRY(cudaMemcpyAsync(sp->host_scal, sp->scal.p, sizeof(OuterScalars) * nrhs,
                                   cudaMemcpyDeviceToHost, st));
      DWF_CUDA_TRY(cudaStreamSynchronize(st));
      ++host_syncs;
      if (debug) {
        for (int r = 0; r < nrhs; ++r) {
          const OuterScalars &q = sp->host_scal[r];
          std::fprintf(stderr, "[dwf] rhs %d iter %d rr %.6e rz %.6e rz_new %.6e pAp %.6e alpha %.6e "
                       "beta %.6e bb %.6e\n", r, q.iter, q.rr, q.rz, q.rz_new, q.pAp, q.alpha,
                       q.beta, q.bb);
        }
      }
      bool any_ru = false;
      std::vector<int> conv_cand(nrhs, 0);
      int min_pred = 1 << 30;
      for (int r = 0; r < nrhs; ++r) {
        hs_ru[r] = 1;
        if (done[r]) continue;
        const OuterScalars &sc = sp->host_scal[r];
        bool need = false;
        double rr_last = sc.rr, rr_first = -1;
        for (int it = seen[r]; it < sc.iter; ++it) {
          const double rr = sc.hist_rr[it % kHistory];
          if (rr_first < 0) rr_first = rr;
          if (!std::isfinite(rr)) {
            status = DWF_ERR_NAN;
          }
          if (rr <= tol2 * bb[r]) conv_cand[r] = 1;
          if (std::sqrt(rr) < prm->delta * maxr[r]) need = true;
          maxr[r] = std::max(maxr[r], std::sqrt(rr));
          rr_last = rr;
        }
        const int adv = sc.iter - seen[r];
        seen[r] = sc.iter;
        if (conv_cand[r]) need = true;
        if (need) {
          hs_ru[r] = 0;
          any_ru = true;
        }
        // predict the iterations left from the last chunk's rate of decrease
        if (adv > 0 && rr_first > 0 && rr_last > 0 && rr_last < rr_first) {
          const double rate = std::log(rr_last / rr_first) / adv;
          const double left = std::log(tol2 * bb[r] / rr_last) / rate;
          if (left > 0 && left < 1e9) min_pred = std::min(min_pred, (int)std::ceil(left));
        }
      }
      if (status == DWF_ERR_NAN) break;
      // never more iterations between checks than the |r|^2 ring holds
      chunk = std::max(1, std::min(std::min(prm->check_every, kHistory), min_pred));
      if (any_ru) {
        DWF_CUDA_TRY(cudaMemcpyAsync(sp->skip_ru.p, hs_ru, sizeof(int) * nrhs,
                                     cudaMemcpyHostToDevice, st));
        enqueue_reliable_update(S, st);
        DWF_CUDA_TRY(cudaMemcpyAsync(sp->host_scal, sp->scal.p, sizeof(OuterScalars) * nrhs,
                                     cudaMemcpyDeviceToHost, st));
        DWF_CUDA_TRY(cudaStreamSynchronize(st));
        ++host_syncs;
        for (int r = 0; r < nrhs; ++r) {
          if (hs_ru[r]) continue;
          if (debug)
            std::fprintf(stderr, "[dwf] rhs %d reliable update: true rr %.6e rz %.6e\n", r,
                         sp->host_scal[r].rr, sp->host_scal[r].rz);
          nru[r] += 1;
          const double rr = sp->host_scal[r].rr;
          maxr[r] = std::sqrt(rr);
          if (!std::isfinite(rr)) status = DWF_ERR_NAN;
          if (rr <= tol2 * bb[r]) {
            done[r] = 1;
            hs_iter[r] = 1;
            final_res[r] = std::sqrt(rr / bb[r]);
          }
        }
        if (status == DWF_ERR_NAN) break;
      }
    }
  }
  // unconverged right-hand sides: fold x_lo in and measure the true residual
  bool any_open = false;
  for (int r = 0; r < nrhs; ++r) {
    hs_ru[r] = done[r] ? 1 : 0;
    any_open |= !done[r];
  }
  if (any_open && status != DWF_ERR_NAN) {
    DWF_CUDA_TRY(cudaMemcpyAsync(sp->skip_ru.p, hs_ru, sizeof(int) * nrhs,
                                 cudaMemcpyHostToDevice, st));
    enqueue_reliable_update(S, st);
    DWF_CUDA_TRY(cudaMemcpyAsync(sp->host_scal, sp->scal.p, sizeof(OuterScalars) * nrhs,
                                 cudaMemcpyDeviceToHost, st));
    DWF_CUDA_TRY(cudaStreamSynchronize(st));
    ++host_syncs;
    for (int r = 0; r < nrhs; ++r)
      if (!done[r]) {
        nru[r] += 1;
        final_res[r] = std::sqrt(sp->host_scal[r].rr / sp->host_scal[r].bb);
      }
  }
  // output
  if (prm->io_on_host) {
    launch_export(DWF_FP64, sp->Ax64.p, 0, sp->x64.c(), A.rs64, Vh, Ls, ctx->act.dims, nrhs, st);
    DWF_CUDA_TRY(cudaMemcpyAsync(x, sp->Ax64.p, (size_t)Vh * Ls * 24 * sizeof(double) * nrhs,
                                 cudaMemcpyDeviceToHost, st));
  } else {
    launch_export(DWF_FP64, x, 0, sp->x64.c(), A.rs64, Vh, Ls, ctx->act.dims, nrhs, st);
  }
  DWF_CUDA_TRY(cudaStreamSynchronize(st));
  const double secs =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  double hop_bytes1, hop_ns1;
  outer_hop_totals(ctx, lo, st, hop_bytes1, hop_ns1);
  const double dslash_gbs = (ctx->prof_on && hop_ns1 > hop_ns0)
                                ? (hop_bytes1 - hop_bytes0) / (hop_ns1 - hop_ns0)
                                : -1.0;
  // inner CG iterations, counted on the device over all blocks (fewer than
  // outer_iters * k per block when the inner residual stop is on)
  std::vector<unsigned int> blk_iters(nrhs, 0);
  if (bp)
    DWF_CUDA_TRY(cudaMemcpy(blk_iters.data(), bp->iters.p, sizeof(unsigned int) * nrhs,
                            cudaMemcpyDeviceToHost));
  bool all_conv = true;
  for (int r = 0; r < nrhs; ++r) {
    if (info) {
      info[r].outer_iters = sp->host_scal[r].iter;
      info[r].inner_iters_total = bp ? (int)(blk_iters[r] / (unsigned)bp->bg.nblocks) : 0;
      info[r].reliable_updates = nru[r];
      info[r].converged = final_res[r] >= 0 && final_res[r] <= prm->tol;
      info[r].true_resid = final_res[r];
      info[r].seconds = secs;
      info[r].dslash_gbs = dslash_gbs;
      info[r].host_syncs = host_syncs;
      info[r].device_loop = device_loop ? 1 : 0;
    }
    all_conv &= final_res[r] >= 0 && final_res[r] <= prm->tol;
  }
  if (status == DWF_OK && !all_conv) status = DWF_ERR_NOT_CONVERGED;
  return status;
}

}  // namespace dwf

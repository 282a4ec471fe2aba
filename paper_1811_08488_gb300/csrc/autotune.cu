// Block-shape autotuner for the multisplitting preconditioner (paper Sec. 2.4:
// the blocks are the sub-lattices each inner CG runs on; their size trades
// the preconditioner's strength, which grows with the block, against the
// snake-region overhead of the block operator, which shrinks with it).
//
// Candidates are blocks b^3 x bt with b in {4, 6, 8, 12, 16} and bt in
// {4, 6, 8, 12, 16, 24, 32}, b/2 <= bt <= 2b, every extent dividing the
// lattice, and at least two blocks. Each candidate runs one untimed outer
// iteration (plan, links and CUDA graph built), then `trial` timed outer
// iterations from x = 0 on the caller's sources. With the largest true
// residual res after n iterations, the rate is rho = res^(1/n) and the
// predicted time to the tolerance is (t / n) * log(tol) / log(rho) (the time
// itself when the trial already converged). The fastest prediction wins.
// Each losing candidate's block plan is released as soon as it loses, and a
// candidate whose plan does not fit in device memory is skipped.
#include <array>
#include <chrono>
#include <cmath>
#include <limits>
#include <sstream>
#include <vector>

#include "solver.cuh"

namespace dwf {

std::vector<std::array<int, 4>> block_candidates(const int dims[4]) {
  static const int bs[] = {4, 6, 8, 12, 16};
  static const int bts[] = {4, 6, 8, 12, 16, 24, 32};
  std::vector<std::array<int, 4>> out;
  for (int b : bs)
    for (int bt : bts) {
      if (2 * bt < b || bt > 2 * b) continue;
      if (dims[0] % b || dims[1] % b || dims[2] % b || dims[3] % bt) continue;
      const long long nb = (long long)(dims[0] / b) * (dims[1] / b) * (dims[2] / b) * (dims[3] / bt);
      if (nb < 2) continue;
      out.push_back({b, b, b, bt});
    }
  return out;
}

// Destroy every cached outer-iteration graph (they hold block-plan pointers).
static void drop_graphs(dwf_ctx *ctx) {
  for (auto &kv : ctx->solver_plans)
    if (kv.second) kv.second->drop_graphs();
}

static std::string plan_key(const int block[4], dwf_prec inner) {
  std::ostringstream key;
  key << block[0] << "x" << block[1] << "x" << block[2] << "x" << block[3] << "/" << inner;
  return key.str();
}

std::string tune_key(const dwf_solver_params *p, int nrhs, const double *mf) {
  std::ostringstream key;
  key << p->inner << "/" << p->outer << "/" << p->inner_iters << "/" << p->snake << "/"
      << p->tol << "/" << p->schur << "/" << p->inner_tol << "/" << nrhs;
  for (int r = 0; r < nrhs; ++r) key << "/" << mf[r];
  return key.str();
}

void autotune_block(dwf_ctx *ctx, const void *b, int nrhs, const double *mf,
                    const dwf_solver_params *prm, int trial, int block_out[4],
                    double *predicted, cudaStream_t st) {
  DWF_REQUIRE(prm->inner_iters > 0, DWF_ERR_INVALID_ARG,
              "the block autotuner needs inner_iters > 0");
  DWF_REQUIRE(trial >= 2, DWF_ERR_INVALID_ARG, "trial must be >= 2 outer iterations");
  const auto cands = block_candidates(ctx->act.dims);
  DWF_REQUIRE(!cands.empty(), DWF_ERR_UNSUPPORTED, "no candidate block shape tiles the lattice");
  const size_t xbytes = (size_t)ctx->geo.Vh * ctx->act.Ls * 24 * sizeof(double) * nrhs;
  DevBuf xdev;
  std::vector<double> xhost;
  void *x;
  if (prm->io_on_host) {
    xhost.resize(xbytes / sizeof(double));
    x = xhost.data();
  } else {
    xdev.ensure(xbytes);
    x = xdev.p;
  }
  std::vector<dwf_solve_info> info(nrhs);
  dwf_solver_params p = *prm;
  const bool debug = std::getenv("DWF_DEBUG") != nullptr;
  double best = std::numeric_limits<double>::infinity();
  std::array<int, 4> best_b = cands[0];
  bool have_best = false;
  // at most two candidates' block plans are held at a time: the best so far
  // and the one on trial (a plan of small blocks on a large lattice holds
  // tens of GB)
  auto release = [&](const std::array<int, 4> &c) {
    drop_graphs(ctx);
    ctx->block_plans.erase(plan_key(c.data(), prm->inner));
  };
  for (const auto &c : cands) {
    for (int i = 0; i < 4; ++i) p.block[i] = c[i];
    double pred = std::numeric_limits<double>::infinity();
    double secs = 0.0;
    try {
      p.maxiter = 1;
      dwf_status s = solve(ctx, x, b, nrhs, mf, &p, info.data(), st);
      if (s == DWF_OK || s == DWF_ERR_NOT_CONVERGED) {
        p.maxiter = trial;
        const auto t0 = std::chrono::steady_clock::now();
        s = solve(ctx, x, b, nrhs, mf, &p, info.data(), st);
        secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (s == DWF_OK) {
          pred = secs;
        } else if (s == DWF_ERR_NOT_CONVERGED) {
          double rho = 0.0;
          int iters = 1;
          for (int r = 0; r < nrhs; ++r) {
            if (info[r].converged || info[r].outer_iters <= 0 || !(info[r].true_resid > 0))
              continue;
            const double rr = std::pow(info[r].true_resid, 1.0 / info[r].outer_iters);
            if (rr > rho) {
              rho = rr;
              iters = info[r].outer_iters;
            }
          }
          if (rho > 0.0 && rho < 1.0) pred = secs / iters * std::log(p.tol) / std::log(rho);
        }
      }
    } catch (const Error &e) {
      // a candidate that does not fit in device memory is skipped
      if (e.code != DWF_ERR_CUDA) throw;
      cudaGetLastError();
      DWF_CUDA_TRY(cudaStreamSynchronize(st));
      if (debug)
        std::fprintf(stderr, "[dwf] autotune %dx%dx%dx%d skipped: %s\n", c[0], c[1], c[2], c[3],
                     e.msg.c_str());
    }
    if (debug)
      std::fprintf(stderr, "[dwf] autotune %dx%dx%dx%d: %.4f s for %d iterations, predicted %.4f s\n",
                   c[0], c[1], c[2], c[3], secs, trial, pred);
    if (pred < best) {
      if (have_best) release(best_b);
      best = pred;
      best_b = c;
      have_best = true;
    } else {
      release(c);
    }
  }
  DWF_REQUIRE(have_best && std::isfinite(best), DWF_ERR_NOT_CONVERGED,
              "no candidate block shape reduced the residual in the trial");
  drop_graphs(ctx);
  for (int i = 0; i < 4; ++i) block_out[i] = best_b[i];
  if (predicted) *predicted = best;
  ctx->tuned_blocks[tune_key(prm, nrhs, mf)] = best_b;
}

}  // namespace dwf

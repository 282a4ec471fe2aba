// dwf_mdagm_noalloc: the normal operator D_PC^+ D_PC without any device
// allocation, for callers that cannot call cudaMalloc.
//
// dwf_mdagm keeps its three half-field temporaries in buffers the context
// allocates on first use. Some callers cannot allow that: applications that
// hand the whole device memory to their own pool allocator at start-up (so a
// later cudaMalloc fails or fragments the pool), and host code that must not
// pay cudaMalloc's implicit device synchronisation in the middle of a
// latency-critical loop. This variant runs the same four hop kernels with the
// temporaries in a fixed, file-scope device array instead.
//
// The array is DWF_NOALLOC_SCRATCH_BYTES long and lives in the library's
// device image: every GPU that loads the library holds it until the process
// exits. All calls share it, and each call leaves its temporaries there; no
// part of it has to start at zero (every temporary is written before it is
// read). Calls whose GPU work overlaps (two streams, or two host threads) race
// on the array and must be serialised by the caller.
//
// The host cannot use the array's name as a device address, so the first call
// on each device looks the address up with cudaGetSymbolAddress (with that
// device current) and caches it; that first call should come before any
// stream capture.
#include <mutex>
#include <unordered_map>

#include "solver.cuh"

static __device__ __align__(256) unsigned char g_noalloc_scratch[DWF_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_addr_mutex;
std::unordered_map<int, void *> g_addr;  // device -> address of g_noalloc_scratch

void *scratch_address(int device) {
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  auto it = g_addr.find(device);
  if (it != g_addr.end()) return it->second;
  void *p = nullptr;
  DWF_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  DWF_REQUIRE(p != nullptr, DWF_ERR_CUDA, "cudaGetSymbolAddress returned no address");
  g_addr[device] = p;
  return p;
}

}  // namespace

extern "C" dwf_status dwf_mdagm_noalloc(dwf_ctx *ctx, void *out, const void *in, dwf_prec prec,
                                        int nrhs, const double *mf, void *stream) {
  try {
    DWF_REQUIRE(ctx, DWF_ERR_INVALID_ARG, "null context");
    DWF_REQUIRE(nrhs >= 1 && nrhs <= DWF_MAX_RHS, DWF_ERR_INVALID_ARG, "nrhs out of range");
    DWF_REQUIRE(mf != nullptr, DWF_ERR_INVALID_ARG, "null mass array");
    for (int r = 0; r < nrhs; ++r)
      DWF_REQUIRE(mf[r] == mf[r], DWF_ERR_INVALID_ARG, "NaN quark mass");
    DWF_REQUIRE(!ctx->unusable, DWF_ERR_TIMEOUT,
                "the context is unusable after an expired device wait; destroy it");
    DWF_REQUIRE(prec == DWF_FP64 || prec == DWF_FP32, DWF_ERR_INVALID_ARG,
                "operator entry points take DWF_FP64 or DWF_FP32 fields");
    DWF_REQUIRE(out && in && out != in, DWF_ERR_INVALID_ARG, "null or aliased fields");
    const size_t rs = dwf::field_rhs_bytes(prec, ctx->geo.Vh, ctx->act.Ls);
    const size_t need = 3 * rs * (size_t)nrhs;
    DWF_REQUIRE(need <= (size_t)DWF_NOALLOC_SCRATCH_BYTES, DWF_ERR_INVALID_ARG,
                "dwf_mdagm_noalloc: three half-field temporaries of this lattice, precision "
                "and nrhs need " + std::to_string(need) + " bytes, more than "
                "DWF_NOALLOC_SCRATCH_BYTES = " + std::to_string((size_t)DWF_NOALLOC_SCRATCH_BYTES));
    DWF_REQUIRE(ctx->have_gauge, DWF_ERR_NO_GAUGE, "no gauge field loaded");
    DWF_CUDA_TRY(cudaSetDevice(ctx->device));
    char *base = static_cast<char *>(scratch_address(ctx->device));
    dwf::OpWork w;
    w.u = base;
    w.y = base + rs * nrhs;
    w.v = base + 2 * rs * nrhs;
    w.rstride = (long long)rs;
    dwf::apply_mdagm(ctx, out, in, prec, nrhs, mf, w, nullptr, nullptr, (cudaStream_t)stream);
  } catch (const dwf::Error &e) {
    if (ctx) ctx->last_error = e.msg;
    return e.code;
  } catch (const std::exception &e) {
    if (ctx) ctx->last_error = e.what();
    return DWF_ERR_CUDA;
  }
  ctx->last_error.clear();
  return DWF_OK;
}

// lens_chi2_image_noalloc: the image-plane chi2 with all of its working
// memory in one fixed, file-scope device array instead of buffers the
// context allocates on demand.
//
// Who needs it: code that drives many chi2 evaluations from a loop whose
// device-memory footprint is reserved once at start-up -- a long-running MCMC
// sampler or a request loop sharing the GPU with other work.  There,
// cudaMalloc/cudaFree must not run at call time: they can synchronise the
// whole device (stalling every other stream) and they can fail under memory
// pressure in the middle of a run.  Such a caller creates the context, the
// model and the constraint set up front, then calls this entry point, which
// allocates nothing.
//
// The array (LENS_NOALLOC_SCRATCH_BYTES) is held by every GPU that loads the
// library until the process exits.  All calls share it and it keeps the last
// call's contents; everything a call reads is written earlier in the same
// call (the per-set counters are reset by the call's first kernel), and two
// calls whose work overlaps on the GPU race on it.
#include <algorithm>
#include <mutex>

#include "lens_internal.cuh"

namespace lens {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[LENS_NOALLOC_SCRATCH_BYTES];

// Parameter sets per batch at most (fewer when the grid leaves less room).
constexpr int32_t NOALLOC_MAX_BATCH = 16;
constexpr int MAX_DEVICES = 64;

std::mutex g_mu;
void *g_ptr[MAX_DEVICES] = {};

// Device address of the array on `device` (which must be current).  Looked
// up once per device; a host-side reference to g_noalloc_scratch is only a
// stand-in for the symbol and must never be handed to a kernel.
int scratch_address(int device, void **out) {
  if (device < 0 || device >= MAX_DEVICES) return fail(LENS_EINVAL, "device index %d unsupported", device);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(LENS_ECUDA, "cudaGetSymbolAddress(no-alloc scratch): %s", cudaGetErrorString(e));
    g_ptr[device] = p;
  }
  *out = g_ptr[device];
  return LENS_OK;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace
}  // namespace lens

using namespace lens;

extern "C" int lens_chi2_image_noalloc(lens_ctx *ctx, lens_cset_t cset, const lens_grid *grid,
                                       const double *d_params, int32_t P, double *d_chi2, int32_t *d_nimg_found,
                                       void *stream) {
  if (!ctx || !d_params || !d_chi2) return fail(LENS_EINVAL, "NULL argument");
  if (P < 1) return fail(LENS_EINVAL, "P must be >= 1");
  int rc = check_grid(grid);
  if (rc) return rc;
  CSet *c = find_cset(ctx, cset);
  if (!c) return fail(LENS_ENOTFOUND, "constraint set %lld not found", (long long)cset);
  if (!find_model(ctx, c->model)) return fail(LENS_ENOTFOUND, "model of constraint set not found");
  if ((rc = check_chi2_image_limits(c, grid))) return rc;
  // the static deflection of this grid, then the candidate buffers of a
  // batch of parameter sets; the batch shrinks until both fit
  const size_t grid_bytes = align256(2 * sizeof(float) * (size_t)grid->nx * grid->ny);
  // (the point-list refinement's state while one set of it fits, else the
  // single-kernel refinement's smaller buffers)
  const bool lists = grid_bytes + chi2_image_scratch_bytes(c, 1, true) <= LENS_NOALLOC_SCRATCH_BYTES;
  int32_t batch = std::min<int32_t>(NOALLOC_MAX_BATCH, P);
  while (batch > 1 && grid_bytes + chi2_image_scratch_bytes(c, batch, lists) > LENS_NOALLOC_SCRATCH_BYTES) batch /= 2;
  if (grid_bytes + chi2_image_scratch_bytes(c, batch, lists) > LENS_NOALLOC_SCRATCH_BYTES)
    return fail(LENS_EINVAL,
                "grid %d x %d needs %zu bytes of fixed scratch (plus %zu for one parameter set); the maximum is %zu "
                "bytes (LENS_NOALLOC_SCRATCH_BYTES)",
                grid->nx, grid->ny, grid_bytes, chi2_image_scratch_bytes(c, 1, false),
                (size_t)LENS_NOALLOC_SCRATCH_BYTES);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(LENS_ECUDA, "cudaSetDevice(%d) failed", ctx->device);
  void *base = nullptr;
  if ((rc = scratch_address(ctx->device, &base))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  StreamMark mark(ctx, st);
  GridCache gc;
  gc.xmin = grid->xmin;
  gc.xmax = grid->xmax;
  gc.ymin = grid->ymin;
  gc.ymax = grid->ymax;
  gc.nx = grid->nx;
  gc.ny = grid->ny;
  gc.alpha32 = (float *)base;
  gc.bytes = grid_bytes;
  if (c->stat_model->n > 0) {
    if ((rc = launch_map_mixed(ctx, c->stat_model, grid, 1.0, false, gc.alpha32, st, 0, -1, false))) return rc;
  } else if (cudaMemsetAsync(gc.alpha32, 0, 2 * sizeof(float) * (size_t)grid->nx * grid->ny, st) != cudaSuccess) {
    return fail(LENS_ECUDA, "clearing the static deflection failed");
  }
  return run_chi2_image(ctx, c, &gc, d_params, P, d_chi2, d_nimg_found, (char *)base + grid_bytes, batch, st,
                        nullptr, 0, nullptr, lists);
}

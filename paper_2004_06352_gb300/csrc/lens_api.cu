// C-ABI entry points: context, model store, constraint sets, waits, errors.
// The compute launches live in lens_maps.cu and lens_chi2.cu.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstring>
#include <thread>

#include "lens_internal.cuh"

namespace lens {

static thread_local char g_msg[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof g_msg, fmt, ap);
  va_end(ap);
}

int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof g_msg, fmt, ap);
  va_end(ap);
  return code;
}

Model *find_model(lens_ctx *ctx, lens_model_t id) {
  for (auto &p : ctx->models)
    if (p.first == id) return p.second;
  return nullptr;
}

CSet *find_cset(lens_ctx *ctx, lens_cset_t id) {
  for (auto &p : ctx->csets)
    if (p.first == id) return p.second;
  return nullptr;
}

// Long-lived device memory: from the context's pool on alloc_st (memory the
// pool holds is reused; a free of this pool that has not completed is never
// waited for, since internal dependencies are off for the pool), ready for
// any stream on return.
int dev_alloc(lens_ctx *ctx, void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return LENS_OK;
  if (ctx->budget && ctx->used + bytes > ctx->budget && !ctx->block_cache.empty()) {
    // cached model blocks go first
    auto cached = std::move(ctx->block_cache);
    ctx->block_cache.clear();
    ctx->cached_bytes = 0;
    for (auto &b : cached) dev_free(ctx, b.first, b.second);
  }
  if (ctx->budget && ctx->used + bytes > ctx->budget)
    return fail(LENS_ENOMEM, "device memory budget exceeded: %zu used + %zu requested > %zu", ctx->used, bytes,
                ctx->budget);
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->alloc_st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->alloc_st);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(LENS_ENOMEM, "device allocation of %zu bytes: %s", bytes, cudaGetErrorString(e));
  }
  ctx->used += bytes;
  return LENS_OK;
}

cudaStream_t upload_stream(lens_ctx *ctx) {
  if (!ctx->upload_st && cudaStreamCreateWithFlags(&ctx->upload_st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    ctx->upload_st = nullptr;
  }
  return ctx->upload_st;
}

void wait_marks(lens_ctx *ctx, cudaStream_t st) {
  for (auto &mk : ctx->marks) cudaStreamWaitEvent(st, mk.second, 0);
}

void dev_free(lens_ctx *ctx, void *p, size_t bytes) {
  if (!p) return;
  if (ctx->release_gen != ctx->mark_gen) {  // new launches since release_st last caught up
    wait_marks(ctx, ctx->release_st);
    ctx->release_gen = ctx->mark_gen;
  }
  cudaFreeAsync(p, ctx->release_st);
  ctx->used -= std::min(ctx->used, bytes);
}

void mark_stream(lens_ctx *ctx, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (cs != cudaStreamCaptureStatusNone) return;
  ++ctx->mark_gen;
  if (ctx->marks.size() > 32) {  // drop streams whose marked work has finished
    size_t k = 0;
    for (auto &mk : ctx->marks) {
      if (mk.first != st && cudaEventQuery(mk.second) == cudaSuccess)
        cudaEventDestroy(mk.second);
      else
        ctx->marks[k++] = mk;
    }
    ctx->marks.resize(k);
    cudaGetLastError();
  }
  for (auto &mk : ctx->marks)
    if (mk.first == st) {
      cudaEventRecord(mk.second, st);
      return;
    }
  cudaEvent_t ev = nullptr;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(st);  // cannot track this stream: let its work finish instead
    return;
  }
  cudaEventRecord(ev, st);
  ctx->marks.push_back({st, ev});
}

int CallScratch::alloc(size_t n) {
  if (n == 0) return LENS_OK;
  if (ctx->budget && ctx->used + n > ctx->budget)
    return fail(LENS_ENOMEM, "device memory budget exceeded: %zu used + %zu requested > %zu", ctx->used, n,
                ctx->budget);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) cudaGetLastError();
  // inside a graph capture: a memory node of the graph (the device's default pool)
  const cudaError_t e = cs != cudaStreamCaptureStatusNone ? cudaMallocAsync(&p, n, st)
                                                          : cudaMallocFromPoolAsync(&p, n, ctx->pool, st);
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    return fail(LENS_ENOMEM, "working memory of %zu bytes: %s", n, cudaGetErrorString(e));
  }
  bytes = n;
  ctx->used += n;
  return LENS_OK;
}

CallScratch::~CallScratch() {
  if (!p) return;
  cudaFreeAsync(p, st);
  ctx->used -= std::min(ctx->used, bytes);
}

int check_grid(const lens_grid *g) {
  if (!g) return fail(LENS_EINVAL, "grid is NULL");
  if (!(std::isfinite(g->xmin) && std::isfinite(g->xmax) && std::isfinite(g->ymin) && std::isfinite(g->ymax)))
    return fail(LENS_EINVAL, "grid corners must be finite");
  if (g->nx < 2 || g->ny < 2) return fail(LENS_EINVAL, "grid needs nx, ny >= 2 (got %d x %d)", g->nx, g->ny);
  if (!(g->xmax > g->xmin && g->ymax > g->ymin)) return fail(LENS_EINVAL, "grid needs xmax > xmin and ymax > ymin");
  // node indices (the map repair list, the image search's cells) are 32-bit,
  // and a map launch has one CTA row per map_tile_rows grid rows
  if ((long long)g->nx * g->ny > INT32_MAX)
    return fail(LENS_EINVAL, "grid of %d x %d has more than 2^31 - 1 nodes", g->nx, g->ny);
  const long long max_rows = 65535LL * std::min(map_tile_rows(true), map_tile_rows(false));
  if (g->ny > max_rows) return fail(LENS_EINVAL, "grid has %d rows; at most %lld", g->ny, max_rows);
  return LENS_OK;
}

static int kind_order(const lens_halo &h) {
  if (h.type == LENS_SIS) return 2;
  if (h.type == LENS_POINT) return 3;
  double u = 2.0 * std::sqrt(h.eps) / (1.0 + h.eps);
  return u < U_SERIES32 ? 1 : 0;
}

// Released model blocks are kept (up to BLOCK_CACHE_MAX bytes) and reused by
// later uploads of similar size: repeated upload/release then costs no
// cudaMalloc/cudaFree.  They stay counted in the context's memory use and are
// freed when an allocation would exceed the budget.
static constexpr size_t BLOCK_CACHE_MAX = 64u << 20;

static void flush_block_cache(lens_ctx *ctx) {
  for (auto &b : ctx->block_cache) dev_free(ctx, b.first, b.second);
  ctx->block_cache.clear();
  ctx->cached_bytes = 0;
}

void free_model(lens_ctx *ctx, Model *m) {
  if (m->block && ctx->cached_bytes + m->bytes <= BLOCK_CACHE_MAX) {
    ctx->block_cache.push_back({m->block, m->bytes});
    ctx->cached_bytes += m->bytes;
  } else {
    dev_free(ctx, m->block, m->bytes);
  }
  delete m;
}

// A device block of at least `bytes`: the smallest cached one that is not
// more than twice as large, else a new allocation.
static int model_block(lens_ctx *ctx, size_t bytes, void **p, size_t *got) {
  int best = -1;
  for (int k = 0; k < (int)ctx->block_cache.size(); ++k) {
    const size_t b = ctx->block_cache[k].second;
    if (b >= bytes && b <= 2 * bytes && (best < 0 || b < ctx->block_cache[best].second)) best = k;
  }
  if (best >= 0) {
    *p = ctx->block_cache[best].first;
    *got = ctx->block_cache[best].second;
    ctx->cached_bytes -= *got;
    ctx->block_cache.erase(ctx->block_cache.begin() + best);
    // the released model's launches may still be reading the block: the
    // upload that overwrites it comes after every launch enqueued so far
    if (!upload_stream(ctx)) return fail(LENS_ECUDA, "upload stream creation failed");
    wait_marks(ctx, ctx->upload_st);
    return LENS_OK;
  }
  *got = bytes;
  return dev_alloc(ctx, p, bytes);
}

// The records of the potentials, built on the device from the halo table,
// three threads per potential (the FP64 arithmetic runs at 1/64 of the FP32
// rate, so the work is spread): part 0 the FP64 record (upload order) and,
// for a heavy potential (slot = -1 - heavy index), its copy in the heavy
// table; part 1 the double-float record (and, for a heavy potential, its
// copy in the heavy table, record-major); part 2, for a light potential
// (slot >= 0, the kind-sorted order), the FP32 record and position data.
__global__ void k_build_records(const lens_halo *__restrict__ h, const int32_t *__restrict__ slot, int n,
                                float *rec32, double *pos64, float *cen32, double *heavy, double *all64,
                                float2 *recdf, float2 *heavydf) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * n) return;
  const int k = t / 3, part = t % 3;
  const lens_halo a = h[k];
  const int s = slot[k];
  if (part == 0) {
    double r[REC64];
    make_rec64(a.type, a.x0, a.y0, a.theta, a.eps, a.rcore, a.rcut, a.b0, r);
    for (int q = 0; q < REC64; ++q) all64[(size_t)k * REC64 + q] = r[q];
    if (s < 0)
      for (int q = 0; q < REC64; ++q) heavy[(size_t)(-1 - s) * REC64 + q] = r[q];
  } else if (part == 1) {
    make_recdf(a.type, a.x0, a.y0, a.theta, a.eps, a.rcore, a.rcut, a.b0, recdf + k, n);
    if (s < 0)
      make_recdf(a.type, a.x0, a.y0, a.theta, a.eps, a.rcore, a.rcut, a.b0, heavydf + (size_t)(-1 - s) * RECDF);
  } else if (s >= 0) {
    make_rec32(a.type, a.theta, a.eps, a.rcore, a.rcut, a.b0, rec32 + (size_t)s * REC32);
    const bool circ = a.type != LENS_DPIE;
    pos64[4 * s + 0] = a.x0;
    pos64[4 * s + 1] = a.y0;
    pos64[4 * s + 2] = circ ? 1.0 : cos(a.theta);
    pos64[4 * s + 3] = circ ? 0.0 : sin(a.theta);
    const float xh = (float)a.x0, yh = (float)a.y0;
    cen32[4 * s + 0] = xh;
    cen32[4 * s + 1] = yh;
    cen32[4 * s + 2] = (float)(a.x0 - (double)xh);
    cen32[4 * s + 3] = (float)(a.y0 - (double)yh);
  }
}

// Device store of n (already validated) potentials; n may be 0.  The host
// only classifies and orders the potentials: the halo table and each
// potential's slot go through the context's page-locked staging buffer into
// one device block (one copy, 256-byte aligned sections), where one kernel
// builds every record in parallel; the upload is complete on return.
int build_model(lens_ctx *ctx, const lens_halo *h, int32_t n, Model **out) {
  Model *m = new Model();
  m->n = n;
  m->host.assign(h, h + n);
  // light potentials grouped by kind so each warp-uniform branch runs in one stretch
  std::vector<int32_t> light, heavy;
  std::vector<int32_t> kind(n);
  for (int32_t i = 0; i < n; ++i) {
    kind[i] = kind_order(h[i]);
    (h[i].b0 >= ctx->fp64_threshold ? heavy : light).push_back(i);
  }
  std::stable_sort(light.begin(), light.end(), [&](int32_t a, int32_t b) { return kind[a] < kind[b]; });
  m->n_light = (int32_t)light.size();
  m->n_heavy = (int32_t)heavy.size();
  for (int k = 0; k < 4; ++k) {
    int32_t c = 0;
    for (int32_t i : light) c += kind[i] < k ? 1 : 0;
    m->koff[k] = c;
  }
  m->koff[4] = m->n_light;
  const size_t nl = (size_t)m->n_light, nh = (size_t)m->n_heavy, na = (size_t)n;
  // records (built on the device), then the staged halo table and slots
  const size_t sizes[9] = {nl * REC32 * sizeof(float),  nl * 4 * sizeof(double),     nl * 4 * sizeof(float),
                           nh * REC64 * sizeof(double), na * REC64 * sizeof(double),   na * RECDF * sizeof(float2),
                           nh * RECDF * sizeof(float2), na * sizeof(lens_halo),        na * sizeof(int32_t)};
  size_t offs[9], total = 0;
  for (int k = 0; k < 9; ++k) {
    offs[k] = total;
    total += (sizes[k] + 255) & ~(size_t)255;
  }
  const size_t staged = total - offs[7];
  // host image of the staged part: the context's page-locked staging buffer
  // (pageable if that cannot be had)
  std::vector<unsigned char> pageable;
  unsigned char *img = nullptr;
  if (ctx->h_stage_bytes < staged) {
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    ctx->h_stage = nullptr;
    ctx->h_stage_bytes = 0;
    if (cudaHostAlloc(&ctx->h_stage, staged, cudaHostAllocDefault) == cudaSuccess) {
      ctx->h_stage_bytes = staged;
    } else {
      cudaGetLastError();
      ctx->h_stage = nullptr;
    }
  }
  if (ctx->h_stage) {
    img = (unsigned char *)ctx->h_stage;
  } else {
    pageable.resize(staged);
    img = pageable.data();
  }
  if (n > 0) std::memcpy(img, h, na * sizeof(lens_halo));
  int32_t *slot = (int32_t *)(img + (offs[8] - offs[7]));
  for (int32_t k = 0; k < m->n_light; ++k) slot[light[k]] = k;
  for (int32_t k = 0; k < m->n_heavy; ++k) slot[heavy[k]] = -1 - k;
  int rc = total ? model_block(ctx, total, &m->block, &m->bytes) : LENS_OK;
  if (rc == LENS_ENOMEM && !ctx->block_cache.empty()) {
    flush_block_cache(ctx);
    rc = model_block(ctx, total, &m->block, &m->bytes);
  }
  if (rc) {
    delete m;
    return rc;
  }
  m->payload = total;
  char *base = (char *)m->block;
  m->rec32 = (float *)(base + offs[0]);
  m->pos64 = (double *)(base + offs[1]);
  m->cen32 = (float *)(base + offs[2]);
  m->heavy = (double *)(base + offs[3]);
  m->all64 = (double *)(base + offs[4]);
  m->recdf = (float2 *)(base + offs[5]);
  m->heavydf = (float2 *)(base + offs[6]);
  cudaError_t e = cudaSuccess;
  if (n > 0) {
    if (!upload_stream(ctx)) e = cudaErrorNotReady;
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + offs[7], img, staged, cudaMemcpyHostToDevice, ctx->upload_st);
    if (e == cudaSuccess) {
      k_build_records<<<(3 * n + 63) / 64, 64, 0, ctx->upload_st>>>(
          (const lens_halo *)(base + offs[7]), (const int32_t *)(base + offs[8]), n, m->rec32, m->pos64, m->cen32,
          m->heavy, m->all64, m->recdf, m->heavydf);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->upload_st);
  }
  if (e != cudaSuccess) {
    free_model(ctx, m);
    return fail(LENS_ECUDA, "model upload: %s", cudaGetErrorString(e));
  }
  *out = m;
  return LENS_OK;
}

static void free_cset(lens_ctx *ctx, CSet *c) {
  dev_free(ctx, c->img_off, (c->nsrc + 1) * sizeof(int32_t));
  dev_free(ctx, c->src_of, c->nimg * sizeof(int32_t));
  dev_free(ctx, c->x, c->nimg * sizeof(double));
  dev_free(ctx, c->y, c->nimg * sizeof(double));
  dev_free(ctx, c->sigma, c->nimg * sizeof(double));
  dev_free(ctx, c->isig2, c->nimg * sizeof(double));
  dev_free(ctx, c->ratio, c->nsrc * sizeof(double));
  dev_free(ctx, c->stat, (size_t)c->nimg * 5 * sizeof(double));
  dev_free(ctx, c->var_base, 2 * REC64 * sizeof(double));
  dev_free(ctx, c->grp_off, (c->ng + 1) * sizeof(int32_t));
  dev_free(ctx, c->grp_src, c->nsrc * sizeof(int32_t));
  dev_free(ctx, c->grp_ratio, c->ng * sizeof(double));
  dev_free(ctx, c->grp_ratio32, c->ng * sizeof(float));
  for (auto &g : c->grids) dev_free(ctx, g.alpha32, g.bytes);
  dev_free(ctx, c->scale_cache, (size_t)c->scale_nodes * c->nimg * 5 * sizeof(double));
  dev_free(ctx, c->scale_x, (size_t)c->scale_nodes * sizeof(double));
  if (c->stat_model) free_model(ctx, c->stat_model);
  delete c;
}

}  // namespace lens

using namespace lens;

extern "C" {

const char *lens_strerror(int code) {
  switch (code) {
    case LENS_OK: return "ok";
    case LENS_EINVAL: return "invalid argument";
    case LENS_ENOMEM: return "device memory budget exceeded or allocation failed";
    case LENS_ENOTFOUND: return "unknown handle";
    case LENS_ECAPACITY: return "image buffer capacity exceeded";
    case LENS_ECUDA: return "CUDA runtime error";
    case LENS_ETIMEOUT: return "timed out";
    default: return "unknown error code";
  }
}

const char *lens_last_error(void) { return g_msg; }

int lens_create(lens_ctx **out, int device, size_t mem_budget_bytes) {
  if (!out) return fail(LENS_EINVAL, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  LENS_CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(LENS_EINVAL, "device %d out of range (have %d)", device, ndev);
  LENS_CUDA_TRY(cudaSetDevice(device));
  lens_ctx *ctx = new lens_ctx();
  ctx->device = device;
  ctx->budget = mem_budget_bytes;
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof props);
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  cudaError_t e = cudaMemPoolCreate(&ctx->pool, &props);
  if (e == cudaSuccess) {
    uint64_t keep = UINT64_MAX;  // memory the pool holds stays with it until lens_destroy
    int no = 0;
    e = cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e == cudaSuccess) e = cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolReuseAllowInternalDependencies, &no);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->alloc_st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->release_st, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (ctx->alloc_st) cudaStreamDestroy(ctx->alloc_st);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    delete ctx;
    return fail(LENS_ECUDA, "memory pool / stream creation: %s", cudaGetErrorString(e));
  }
  int rc = dev_alloc(ctx, (void **)&ctx->d_err, sizeof(int));
  if (rc != LENS_OK) {
    lens_destroy(ctx);
    return rc;
  }
  cudaMemset(ctx->d_err, 0, sizeof(int));
  *out = ctx;
  return LENS_OK;
}

int lens_destroy(lens_ctx *ctx) {
  if (!ctx) return LENS_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (auto &p : ctx->csets) free_cset(ctx, p.second);
  for (auto &p : ctx->models) free_model(ctx, p.second);
  flush_block_cache(ctx);
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  dev_free(ctx, ctx->band, ctx->band_bytes);
  dev_free(ctx, ctx->d_err, sizeof(int));
  if (ctx->release_st) cudaStreamSynchronize(ctx->release_st);
  for (auto &mk : ctx->marks) cudaEventDestroy(mk.second);
  if (ctx->alloc_st) cudaStreamDestroy(ctx->alloc_st);
  if (ctx->release_st) cudaStreamDestroy(ctx->release_st);
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  for (int k = 0; k < 2; ++k) {
    if (ctx->pipe_cs[k]) cudaStreamDestroy(ctx->pipe_cs[k]);
    if (ctx->pipe_done[k]) cudaEventDestroy(ctx->pipe_done[k]);
    if (ctx->pipe_copied[k]) cudaEventDestroy(ctx->pipe_copied[k]);
  }
  if (ctx->pipe_cp) cudaStreamDestroy(ctx->pipe_cp);
  if (ctx->upload_st) cudaStreamDestroy(ctx->upload_st);
  if (ctx->pipe_start) cudaEventDestroy(ctx->pipe_start);
  delete ctx;
  return LENS_OK;
}

int lens_set_fp64_threshold(lens_ctx *ctx, double t) {
  if (!ctx) return fail(LENS_EINVAL, "ctx is NULL");
  if (std::isnan(t) || t < 0.0) return fail(LENS_EINVAL, "threshold must be >= 0");
  ctx->fp64_threshold = t;
  return LENS_OK;
}

int lens_set_repair_ratio(lens_ctx *ctx, double r) {
  if (!ctx) return fail(LENS_EINVAL, "ctx is NULL");
  if (!(std::isfinite(r) && r >= 0.0)) return fail(LENS_EINVAL, "repair ratio must be finite and >= 0");
  ctx->repair_ratio = r;
  return LENS_OK;
}

size_t lens_mem_used(const lens_ctx *ctx) { return ctx ? ctx->used : 0; }

size_t lens_model_bytes(lens_ctx *ctx, lens_model_t model) {
  const Model *m = ctx ? find_model(ctx, model) : nullptr;
  return m ? m->payload : 0;
}

int lens_model_upload(lens_ctx *ctx, const lens_halo *h, int32_t n, lens_model_t *out) {
  if (!ctx || !h || !out) return fail(LENS_EINVAL, "NULL argument");
  if (n < 1) return fail(LENS_EINVAL, "need n >= 1 potentials (got %d)", n);
  for (int32_t i = 0; i < n; ++i) {
    const lens_halo &a = h[i];
    if (!halo_params_ok(a.type, a.x0, a.y0, a.theta, a.eps, a.rcore, a.rcut, a.b0))
      return fail(LENS_EINVAL,
                  "potential %d out of domain (type %d, eps %g, rcore %g, rcut %g, b0 %g): need finite values, "
                  "b0 > 0 and for dPIE 0 <= eps < 1, 0 < rcore < rcut",
                  i, a.type, a.eps, a.rcore, a.rcut, a.b0);
  }
  cudaSetDevice(ctx->device);
  Model *m = nullptr;
  int rc = build_model(ctx, h, n, &m);
  if (rc) return rc;
  int64_t id = ctx->next_id++;
  ctx->models.push_back({id, m});
  *out = id;
  return LENS_OK;
}

int lens_model_release(lens_ctx *ctx, lens_model_t id) {
  if (!ctx) return fail(LENS_EINVAL, "ctx is NULL");
  for (size_t k = 0; k < ctx->models.size(); ++k)
    if (ctx->models[k].first == id) {
      cudaSetDevice(ctx->device);
      // the memory is freed (or kept for reuse) in stream order, after the
      // launches enqueued so far: no wait here
      // constraint sets bound to this model go with it
      for (size_t j = 0; j < ctx->csets.size();) {
        if (ctx->csets[j].second->model == id) {
          free_cset(ctx, ctx->csets[j].second);
          ctx->csets.erase(ctx->csets.begin() + j);
        } else {
          ++j;
        }
      }
      free_model(ctx, ctx->models[k].second);
      ctx->models.erase(ctx->models.begin() + k);
      return LENS_OK;
    }
  return fail(LENS_ENOTFOUND, "model %lld not found", (long long)id);
}

static int map_common(lens_ctx *ctx, lens_model_t model, const lens_grid *grid, double dls_ds, int32_t precision,
                      void *d_out, void *stream, bool hess) {
  if (!ctx || !d_out) return fail(LENS_EINVAL, "NULL argument");
  Model *m = find_model(ctx, model);
  if (!m) return fail(LENS_ENOTFOUND, "model %lld not found", (long long)model);
  int rc = check_grid(grid);
  if (rc) return rc;
  if (!(std::isfinite(dls_ds) && dls_ds > 0.0)) return fail(LENS_EINVAL, "dls_ds must be finite and > 0");
  size_t align = precision == LENS_FP64 ? 8 : 4;
  if ((uintptr_t)d_out % align) return fail(LENS_EINVAL, "d_out must be aligned to its element size");
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  StreamMark mark(ctx, st);
  if (precision == LENS_MIXED) return launch_map_mixed(ctx, m, grid, dls_ds, hess, d_out, st);
  if (precision == LENS_FP64) return launch_map_fp64(ctx, m, grid, dls_ds, hess, d_out, st);
  return fail(LENS_EINVAL, "precision must be LENS_FP64 or LENS_MIXED");
}

int lens_potential_map(lens_ctx *ctx, lens_model_t model, const lens_grid *grid, double dls_ds, int32_t precision,
                       const double *beta, void *d_out, void *stream) {
  if (!ctx || !d_out) return fail(LENS_EINVAL, "NULL argument");
  Model *m = find_model(ctx, model);
  if (!m) return fail(LENS_ENOTFOUND, "model %lld not found", (long long)model);
  int rc = check_grid(grid);
  if (rc) return rc;
  if (!(std::isfinite(dls_ds) && dls_ds > 0.0)) return fail(LENS_EINVAL, "dls_ds must be finite and > 0");
  if (precision != LENS_MIXED && precision != LENS_FP64)
    return fail(LENS_EINVAL, "precision must be LENS_FP64 or LENS_MIXED");
  if (beta && !(std::isfinite(beta[0]) && std::isfinite(beta[1]))) return fail(LENS_EINVAL, "beta must be finite");
  if ((uintptr_t)d_out % 8) return fail(LENS_EINVAL, "d_out must be 8-byte aligned (double planes)");
  cudaSetDevice(ctx->device);
  StreamMark mark(ctx, (cudaStream_t)stream);
  return launch_pot_map(ctx, m, grid, dls_ds, precision, beta, d_out, (cudaStream_t)stream);
}

// Map straight to page-locked host memory: the grid in row bands computed
// on two streams of the context (so one band's tail overlaps the next band)
// into two device buffers, each band copied to the host on a third stream as
// soon as it is done; `stream` waits for the last copies.  The bands are
// whole multiples of the kernel's tile height, so every value is the one
// lens_*_map would give.
static int map_host_common(lens_ctx *ctx, lens_model_t model, const lens_grid *grid, double dls_ds,
                           int32_t precision, void *h_out, void *stream, bool hess) {
  if (!ctx || !h_out) return fail(LENS_EINVAL, "NULL argument");
  Model *m = find_model(ctx, model);
  if (!m) return fail(LENS_ENOTFOUND, "model %lld not found", (long long)model);
  int rc = check_grid(grid);
  if (rc) return rc;
  if (!(std::isfinite(dls_ds) && dls_ds > 0.0)) return fail(LENS_EINVAL, "dls_ds must be finite and > 0");
  if (precision != LENS_MIXED && precision != LENS_FP64)
    return fail(LENS_EINVAL, "precision must be LENS_FP64 or LENS_MIXED");
  cudaSetDevice(ctx->device);
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, h_out) != cudaSuccess || pa.type != cudaMemoryTypeHost) {
    cudaGetLastError();
    return fail(LENS_EINVAL, "h_out must be page-locked host memory (cudaHostAlloc or cudaHostRegister)");
  }
  const size_t esize = precision == LENS_FP64 ? 8 : 4;
  if ((uintptr_t)h_out % esize) return fail(LENS_EINVAL, "h_out must be aligned to its element size");
  const int planes = hess ? 6 : 2, nx = grid->nx, ny = grid->ny;
  // about 8 bands, each a whole number of tiles
  const int tile = map_tile_rows(hess);
  int rows = (ny + 7) / 8;
  rows = std::max(tile, (rows + tile - 1) / tile * tile);
  const size_t band_bytes = (size_t)rows * nx * planes * esize;
  if (ctx->band_bytes < 2 * band_bytes) {
    if (ctx->band) {
      dev_free(ctx, ctx->band, ctx->band_bytes);  // after the bands in flight have left
      ctx->band = nullptr;
      ctx->band_bytes = 0;
    }
    if ((rc = dev_alloc(ctx, &ctx->band, 2 * band_bytes))) return rc;
    ctx->band_bytes = 2 * band_bytes;
  }
  if (!ctx->pipe_cp) {
    for (int k = 0; k < 2; ++k) {
      LENS_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->pipe_cs[k], cudaStreamNonBlocking));
      LENS_CUDA_TRY(cudaEventCreateWithFlags(&ctx->pipe_done[k], cudaEventDisableTiming));
      LENS_CUDA_TRY(cudaEventCreateWithFlags(&ctx->pipe_copied[k], cudaEventDisableTiming));
    }
    LENS_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->pipe_cp, cudaStreamNonBlocking));
    LENS_CUDA_TRY(cudaEventCreateWithFlags(&ctx->pipe_start, cudaEventDisableTiming));
  }
  cudaStream_t st = (cudaStream_t)stream;
  StreamMark mark(ctx, st);  // st joins the band streams at the end
  LENS_CUDA_TRY(cudaEventRecord(ctx->pipe_start, st));
  for (int k = 0; k < 2; ++k) LENS_CUDA_TRY(cudaStreamWaitEvent(ctx->pipe_cs[k], ctx->pipe_start, 0));
  char *host = (char *)h_out;
  const size_t host_plane = (size_t)nx * ny * esize;
  for (int row0 = 0, b = 0; row0 < ny; row0 += rows, ++b) {
    const int r = std::min(rows, ny - row0), k = b & 1;
    char *buf = (char *)ctx->band + k * band_bytes;
    cudaStream_t cs = ctx->pipe_cs[k];
    // the buffer's previous band (this call's or an earlier call's) has left
    LENS_CUDA_TRY(cudaStreamWaitEvent(cs, ctx->pipe_copied[k], 0));
    rc = precision == LENS_MIXED ? launch_map_mixed(ctx, m, grid, dls_ds, hess, buf, cs, row0, r)
                                 : launch_map_fp64(ctx, m, grid, dls_ds, hess, buf, cs, row0, r);
    if (rc) return rc;
    LENS_CUDA_TRY(cudaEventRecord(ctx->pipe_done[k], cs));
    LENS_CUDA_TRY(cudaStreamWaitEvent(ctx->pipe_cp, ctx->pipe_done[k], 0));
    // band [planes][r][nx] -> host [planes][ny][nx] at row row0
    LENS_CUDA_TRY(cudaMemcpy2DAsync(host + (size_t)row0 * nx * esize, host_plane, buf, (size_t)r * nx * esize,
                                    (size_t)r * nx * esize, planes, cudaMemcpyDeviceToHost, ctx->pipe_cp));
    LENS_CUDA_TRY(cudaEventRecord(ctx->pipe_copied[k], ctx->pipe_cp));
  }
  for (int k = 0; k < 2; ++k) LENS_CUDA_TRY(cudaStreamWaitEvent(st, ctx->pipe_copied[k], 0));
  return LENS_OK;
}

int lens_grad_map_host(lens_ctx *ctx, lens_model_t model, const lens_grid *grid, double dls_ds, int32_t precision,
                       void *h_out, void *stream) {
  return map_host_common(ctx, model, grid, dls_ds, precision, h_out, stream, false);
}

int lens_hessian_map_host(lens_ctx *ctx, lens_model_t model, const lens_grid *grid, double dls_ds,
                          int32_t precision, void *h_out, void *stream) {
  return map_host_common(ctx, model, grid, dls_ds, precision, h_out, stream, true);
}

int lens_grad_map(lens_ctx *ctx, lens_model_t model, const lens_grid *grid, double dls_ds, int32_t precision,
                  void *d_out, void *stream) {
  return map_common(ctx, model, grid, dls_ds, precision, d_out, stream, false);
}

int lens_hessian_map(lens_ctx *ctx, lens_model_t model, const lens_grid *grid, double dls_ds, int32_t precision,
                     void *d_out, void *stream) {
  return map_common(ctx, model, grid, dls_ds, precision, d_out, stream, true);
}

int lens_cset_create(lens_ctx *ctx, lens_model_t model, const lens_constraints *c, const int32_t var_halo[2],
                     lens_cset_t *out) {
  if (!ctx || !c || !var_halo || !out) return fail(LENS_EINVAL, "NULL argument");
  Model *m = find_model(ctx, model);
  if (!m) return fail(LENS_ENOTFOUND, "model %lld not found", (long long)model);
  if (c->nsrc < 1 || !c->img_off || !c->x || !c->y || !c->sigma || !c->dls_ds)
    return fail(LENS_EINVAL, "constraints need nsrc >= 1 and non-NULL arrays");
  if (c->img_off[0] != 0) return fail(LENS_EINVAL, "img_off[0] must be 0");
  for (int32_t i = 0; i < c->nsrc; ++i) {
    if (c->img_off[i + 1] < c->img_off[i]) return fail(LENS_EINVAL, "img_off must be non-decreasing");
    if (!(std::isfinite(c->dls_ds[i]) && c->dls_ds[i] > 0.0)) return fail(LENS_EINVAL, "dls_ds[%d] must be > 0", i);
  }
  int32_t nimg = c->img_off[c->nsrc];
  if (nimg < 1) return fail(LENS_EINVAL, "constraints hold no image");
  for (int32_t j = 0; j < nimg; ++j)
    if (!(std::isfinite(c->x[j]) && std::isfinite(c->y[j]) && std::isfinite(c->sigma[j]) && c->sigma[j] > 0.0))
      return fail(LENS_EINVAL, "image %d: positions must be finite and sigma > 0", j);
  if (var_halo[0] < 0 || var_halo[0] >= m->n || var_halo[1] < 0 || var_halo[1] >= m->n || var_halo[0] == var_halo[1])
    return fail(LENS_EINVAL, "var_halo must be two distinct indices < n");
  cudaSetDevice(ctx->device);
  CSet *s = new CSet();
  s->model = model;
  s->nsrc = c->nsrc;
  s->nimg = nimg;
  s->var[0] = var_halo[0];
  s->var[1] = var_halo[1];
  std::vector<int32_t> src_of(nimg);
  for (int32_t i = 0; i < c->nsrc; ++i)
    for (int32_t j = c->img_off[i]; j < c->img_off[i + 1]; ++j) src_of[j] = i;
  std::vector<double> vb(2 * REC64);
  for (int k = 0; k < 2; ++k) {
    const lens_halo &a = m->host[var_halo[k]];
    s->var_type[k] = a.type;
    make_rec64(a.type, a.x0, a.y0, a.theta, a.eps, a.rcore, a.rcut, a.b0, &vb[k * REC64]);
  }
  int rc;
  if ((rc = dev_alloc(ctx, (void **)&s->img_off, (c->nsrc + 1) * sizeof(int32_t))) ||
      (rc = dev_alloc(ctx, (void **)&s->src_of, nimg * sizeof(int32_t))) ||
      (rc = dev_alloc(ctx, (void **)&s->x, nimg * sizeof(double))) ||
      (rc = dev_alloc(ctx, (void **)&s->y, nimg * sizeof(double))) ||
      (rc = dev_alloc(ctx, (void **)&s->sigma, nimg * sizeof(double))) ||
      (rc = dev_alloc(ctx, (void **)&s->isig2, nimg * sizeof(double))) ||
      (rc = dev_alloc(ctx, (void **)&s->ratio, c->nsrc * sizeof(double))) ||
      (rc = dev_alloc(ctx, (void **)&s->stat, (size_t)nimg * 5 * sizeof(double))) ||
      (rc = dev_alloc(ctx, (void **)&s->var_base, 2 * REC64 * sizeof(double)))) {
    free_cset(ctx, s);
    return rc;
  }
  cudaError_t e = cudaMemcpy(s->img_off, c->img_off, (c->nsrc + 1) * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->src_of, src_of.data(), nimg * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->x, c->x, nimg * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->y, c->y, nimg * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->sigma, c->sigma, nimg * sizeof(double), cudaMemcpyHostToDevice);
  std::vector<double> isig2(nimg);
  for (int32_t j = 0; j < nimg; ++j) isig2[j] = 1.0 / (c->sigma[j] * c->sigma[j]);
  if (e == cudaSuccess) e = cudaMemcpy(s->isig2, isig2.data(), nimg * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->ratio, c->dls_ds, c->nsrc * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->var_base, vb.data(), vb.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_cset(ctx, s);
    return fail(LENS_ECUDA, "constraint upload: %s", cudaGetErrorString(e));
  }
  // sources grouped by distance ratio (the image search ray-shoots the grid
  // once per distinct ratio), and the model without the varying potentials
  std::vector<double> ratios(c->dls_ds, c->dls_ds + c->nsrc);
  std::sort(ratios.begin(), ratios.end());
  ratios.erase(std::unique(ratios.begin(), ratios.end()), ratios.end());
  s->ng = (int32_t)ratios.size();
  std::vector<int32_t> goff(s->ng + 1, 0), gsrc;
  for (int32_t g = 0; g < s->ng; ++g) {
    for (int32_t i = 0; i < c->nsrc; ++i)
      if (c->dls_ds[i] == ratios[g]) gsrc.push_back(i);
    goff[g + 1] = (int32_t)gsrc.size();
  }
  std::vector<lens_halo> stat_h;
  for (int32_t k = 0; k < m->n; ++k)
    if (k != var_halo[0] && k != var_halo[1]) stat_h.push_back(m->host[k]);
  if ((rc = dev_alloc(ctx, (void **)&s->grp_off, (s->ng + 1) * sizeof(int32_t))) ||
      (rc = dev_alloc(ctx, (void **)&s->grp_src, c->nsrc * sizeof(int32_t))) ||
      (rc = dev_alloc(ctx, (void **)&s->grp_ratio, s->ng * sizeof(double))) ||
      (rc = dev_alloc(ctx, (void **)&s->grp_ratio32, s->ng * sizeof(float))) ||
      (rc = build_model(ctx, stat_h.data(), (int32_t)stat_h.size(), &s->stat_model))) {
    free_cset(ctx, s);
    return rc;
  }
  e = cudaMemcpy(s->grp_off, goff.data(), goff.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->grp_src, gsrc.data(), gsrc.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->grp_ratio, ratios.data(), ratios.size() * sizeof(double), cudaMemcpyHostToDevice);
  std::vector<float> ratios32(ratios.begin(), ratios.end());
  if (e == cudaSuccess)
    e = cudaMemcpy(s->grp_ratio32, ratios32.data(), ratios32.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_cset(ctx, s);
    return fail(LENS_ECUDA, "constraint upload: %s", cudaGetErrorString(e));
  }
  if ((rc = build_static_cache(ctx, m, s))) {
    free_cset(ctx, s);
    return rc;
  }
  int64_t id = ctx->next_id++;
  ctx->csets.push_back({id, s});
  *out = id;
  return LENS_OK;
}

int lens_cset_release(lens_ctx *ctx, lens_cset_t id) {
  if (!ctx) return fail(LENS_EINVAL, "ctx is NULL");
  for (size_t k = 0; k < ctx->csets.size(); ++k)
    if (ctx->csets[k].first == id) {
      cudaSetDevice(ctx->device);
      free_cset(ctx, ctx->csets[k].second);  // freed in stream order, after the launches so far
      ctx->csets.erase(ctx->csets.begin() + k);
      return LENS_OK;
    }
  return fail(LENS_ENOTFOUND, "constraint set %lld not found", (long long)id);
}

int lens_chi2_source(lens_ctx *ctx, lens_cset_t cset, const double *d_params, int32_t P, int32_t variant,
                     double *d_chi2, void *stream) {
  if (!ctx || !d_params || !d_chi2) return fail(LENS_EINVAL, "NULL argument");
  if (P < 1) return fail(LENS_EINVAL, "P must be >= 1");
  if (variant < 0 || variant > 2) return fail(LENS_EINVAL, "variant must be 0, 1 or 2");
  CSet *c = find_cset(ctx, cset);
  if (!c) return fail(LENS_ENOTFOUND, "constraint set %lld not found", (long long)cset);
  Model *m = find_model(ctx, c->model);
  if (!m) return fail(LENS_ENOTFOUND, "model of constraint set not found");
  cudaSetDevice(ctx->device);
  StreamMark mark(ctx, (cudaStream_t)stream);
  return launch_chi2_source(ctx, m, c, d_params, P, variant, d_chi2, (cudaStream_t)stream);
}

int lens_chi2_source_scaled(lens_ctx *ctx, lens_cset_t cset, const double *d_params, int32_t P, int32_t variant,
                            double *d_chi2, void *stream) {
  if (!ctx || !d_params || !d_chi2) return fail(LENS_EINVAL, "NULL argument");
  if (P < 1) return fail(LENS_EINVAL, "P must be >= 1");
  if (variant < 0 || variant > 2) return fail(LENS_EINVAL, "variant must be 0, 1 or 2");
  CSet *c = find_cset(ctx, cset);
  if (!c) return fail(LENS_ENOTFOUND, "constraint set %lld not found", (long long)cset);
  Model *m = find_model(ctx, c->model);
  if (!m) return fail(LENS_ENOTFOUND, "model of constraint set not found");
  cudaSetDevice(ctx->device);
  StreamMark mark(ctx, (cudaStream_t)stream);
  return launch_chi2_source_scaled(ctx, m, c, d_params, P, variant, d_chi2, (cudaStream_t)stream);
}

int lens_cset_scaling_cache(lens_ctx *ctx, lens_cset_t cset, double ft_min, double ft_max, int32_t nodes) {
  if (!ctx) return fail(LENS_EINVAL, "ctx is NULL");
  CSet *c = find_cset(ctx, cset);
  if (!c) return fail(LENS_ENOTFOUND, "constraint set %lld not found", (long long)cset);
  Model *m = find_model(ctx, c->model);
  if (!m) return fail(LENS_ENOTFOUND, "model of constraint set not found");
  cudaSetDevice(ctx->device);
  // the old cache goes once the calls enqueued with it have finished
  dev_free(ctx, c->scale_cache, (size_t)c->scale_nodes * c->nimg * 5 * sizeof(double));
  dev_free(ctx, c->scale_x, (size_t)c->scale_nodes * sizeof(double));
  c->scale_cache = c->scale_x = nullptr;
  c->scale_nodes = 0;
  if (nodes == 0) return LENS_OK;
  if (nodes < 8 || nodes > 128) return fail(LENS_EINVAL, "nodes must be 0 or 8..128");
  if (!(std::isfinite(ft_min) && std::isfinite(ft_max) && ft_min > 0.0 && ft_min < ft_max))
    return fail(LENS_EINVAL, "need 0 < ft_min < ft_max");
  for (int32_t i = 0; i < m->n; ++i) {
    const lens_halo &h = m->host[i];
    if (i == c->var[0] || i == c->var[1] || h.type != LENS_DPIE) continue;
    if (!(ft_min * h.rcut > h.rcore)) return fail(LENS_EINVAL, "ft_min puts potential %d's r_cut below r_core", i);
  }
  std::vector<double> xs(nodes), p16((size_t)nodes * 16, 0.0);
  for (int k = 0; k < nodes; ++k) {
    xs[k] = 0.5 * (ft_min + ft_max) + 0.5 * (ft_max - ft_min) * std::cos(M_PI * k / (nodes - 1));
    p16[(size_t)k * 16 + 14] = 1.0;
    p16[(size_t)k * 16 + 15] = xs[k];
  }
  double *d_p16 = nullptr;
  int rc = dev_alloc(ctx, (void **)&c->scale_cache, (size_t)nodes * c->nimg * 5 * sizeof(double));
  if (!rc) rc = dev_alloc(ctx, (void **)&c->scale_x, (size_t)nodes * sizeof(double));
  if (!rc) rc = dev_alloc(ctx, (void **)&d_p16, p16.size() * sizeof(double));
  if (!rc && (cudaMemcpy(c->scale_x, xs.data(), nodes * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
              cudaMemcpy(d_p16, p16.data(), p16.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess))
    rc = fail(LENS_ECUDA, "scaling cache upload failed");
  c->scale_nodes = nodes;
  if (!rc) rc = build_scaling_cache(ctx, m, c, d_p16, nodes);
  dev_free(ctx, d_p16, p16.size() * sizeof(double));
  if (rc) {
    dev_free(ctx, c->scale_cache, (size_t)nodes * c->nimg * 5 * sizeof(double));
    dev_free(ctx, c->scale_x, (size_t)nodes * sizeof(double));
    c->scale_cache = c->scale_x = nullptr;
    c->scale_nodes = 0;
    return rc;
  }
  c->ft_min = ft_min;
  c->ft_max = ft_max;
  return LENS_OK;
}

static int mcmc_step(lens_ctx *ctx, lens_cset_t cset, double *d_params, double *d_chi2, int32_t W, int32_t nparams,
                     const double *d_sigma, double temperature, uint64_t seed, uint64_t step, uint64_t *d_step,
                     int32_t variant, double *d_scratch, int32_t *d_accepted, void *stream) {
  if (!ctx || !d_params || !d_chi2 || !d_sigma || !d_scratch) return fail(LENS_EINVAL, "NULL argument");
  if (W < 1) return fail(LENS_EINVAL, "W must be >= 1");
  if (nparams != 14 && nparams != 16) return fail(LENS_EINVAL, "nparams must be 14 or 16");
  if (!(std::isfinite(temperature) && temperature > 0.0)) return fail(LENS_EINVAL, "temperature must be > 0");
  if (variant < 0 || variant > 2) return fail(LENS_EINVAL, "variant must be 0, 1 or 2");
  CSet *c = find_cset(ctx, cset);
  if (!c) return fail(LENS_ENOTFOUND, "constraint set %lld not found", (long long)cset);
  Model *m = find_model(ctx, c->model);
  if (!m) return fail(LENS_ENOTFOUND, "model of constraint set not found");
  cudaSetDevice(ctx->device);
  StreamMark mark(ctx, (cudaStream_t)stream);
  return launch_mcmc_step(ctx, m, c, d_params, d_chi2, W, d_sigma, temperature, seed, step, variant, nparams,
                          d_scratch, d_accepted, (cudaStream_t)stream, (unsigned long long *)d_step);
}

int lens_mcmc_step(lens_ctx *ctx, lens_cset_t cset, double *d_params, double *d_chi2, int32_t W,
                   int32_t nparams, const double *d_sigma, double temperature, uint64_t seed, uint64_t step,
                   int32_t variant, double *d_scratch, int32_t *d_accepted, void *stream) {
  return mcmc_step(ctx, cset, d_params, d_chi2, W, nparams, d_sigma, temperature, seed, step, nullptr, variant,
                   d_scratch, d_accepted, stream);
}

int lens_mcmc_step_dev(lens_ctx *ctx, lens_cset_t cset, double *d_params, double *d_chi2, int32_t W,
                       int32_t nparams, const double *d_sigma, double temperature, uint64_t seed, uint64_t *d_step,
                       int32_t variant, double *d_scratch, int32_t *d_accepted, void *stream) {
  if (!d_step) return fail(LENS_EINVAL, "d_step is NULL");
  return mcmc_step(ctx, cset, d_params, d_chi2, W, nparams, d_sigma, temperature, seed, 0, d_step, variant,
                   d_scratch, d_accepted, stream);
}

int lens_chi2_source_nocache(lens_ctx *ctx, lens_cset_t cset, const double *d_params, int32_t P, int32_t variant,
                             double *d_chi2, void *stream) {
  if (!ctx || !d_params || !d_chi2) return fail(LENS_EINVAL, "NULL argument");
  if (P < 1) return fail(LENS_EINVAL, "P must be >= 1");
  if (variant < 0 || variant > 2) return fail(LENS_EINVAL, "variant must be 0, 1 or 2");
  CSet *c = find_cset(ctx, cset);
  if (!c) return fail(LENS_ENOTFOUND, "constraint set %lld not found", (long long)cset);
  Model *m = find_model(ctx, c->model);
  if (!m) return fail(LENS_ENOTFOUND, "model of constraint set not found");
  cudaSetDevice(ctx->device);
  StreamMark mark(ctx, (cudaStream_t)stream);
  return launch_chi2_source_nocache(ctx, m, c, d_params, P, variant, d_chi2, (cudaStream_t)stream);
}

int lens_chi2_autotune(lens_ctx *ctx, lens_cset_t cset, const double *d_params, int32_t P, double *d_chi2,
                       void *stream, int32_t *chosen, float *best_ms) {
  if (!ctx || !d_params || !d_chi2) return fail(LENS_EINVAL, "NULL argument");
  if (P < 1) return fail(LENS_EINVAL, "P must be >= 1");
  CSet *c = find_cset(ctx, cset);
  if (!c) return fail(LENS_ENOTFOUND, "constraint set %lld not found", (long long)cset);
  cudaSetDevice(ctx->device);
  StreamMark mark(ctx, (cudaStream_t)stream);
  return autotune_chi2_source(ctx, c, d_params, P, d_chi2, (cudaStream_t)stream, chosen, best_ms);
}

int lens_chi2_image(lens_ctx *ctx, lens_cset_t cset, const lens_grid *grid, const double *d_params, int32_t P,
                    double *d_chi2, int32_t *d_nimg_found, void *stream) {
  if (!ctx || !d_params || !d_chi2) return fail(LENS_EINVAL, "NULL argument");
  if (P < 1) return fail(LENS_EINVAL, "P must be >= 1");
  int rc = check_grid(grid);
  if (rc) return rc;
  CSet *c = find_cset(ctx, cset);
  if (!c) return fail(LENS_ENOTFOUND, "constraint set %lld not found", (long long)cset);
  Model *m = find_model(ctx, c->model);
  if (!m) return fail(LENS_ENOTFOUND, "model of constraint set not found");
  cudaSetDevice(ctx->device);
  StreamMark mark(ctx, (cudaStream_t)stream);
  return launch_chi2_image(ctx, m, c, grid, d_params, P, d_chi2, d_nimg_found, (cudaStream_t)stream);
}

int lens_find_images(lens_ctx *ctx, lens_cset_t cset, const lens_grid *grid, const double *d_params, int32_t P,
                     double *d_images, int32_t max_per_set, int32_t *d_count, void *stream) {
  if (!ctx || !d_params || !d_images || !d_count) return fail(LENS_EINVAL, "NULL argument");
  if (P < 1 || max_per_set < 1) return fail(LENS_EINVAL, "P and max_per_set must be >= 1");
  int rc = check_grid(grid);
  if (rc) return rc;
  CSet *c = find_cset(ctx, cset);
  if (!c) return fail(LENS_ENOTFOUND, "constraint set %lld not found", (long long)cset);
  Model *m = find_model(ctx, c->model);
  if (!m) return fail(LENS_ENOTFOUND, "model of constraint set not found");
  cudaSetDevice(ctx->device);
  StreamMark mark(ctx, (cudaStream_t)stream);
  return launch_chi2_image(ctx, m, c, grid, d_params, P, nullptr, nullptr, (cudaStream_t)stream, d_images,
                           max_per_set, d_count);
}

int lens_selftest_wait(lens_ctx *ctx, int32_t polls, void *stream) {
  if (!ctx) return fail(LENS_EINVAL, "ctx is NULL");
  if (polls < 1 || polls > (1 << 20)) return fail(LENS_EINVAL, "polls must be in 1..2^20");
  cudaSetDevice(ctx->device);
  StreamMark mark(ctx, (cudaStream_t)stream);
  return launch_wait_selftest(ctx, (unsigned)polls, (cudaStream_t)stream);
}

int lens_selftest_math(lens_ctx *ctx, const double *d_x, int32_t n, double *d_out, void *stream) {
  if (!ctx) return fail(LENS_EINVAL, "ctx is NULL");
  if (n < 0 || (n > 0 && (!d_x || !d_out))) return fail(LENS_EINVAL, "bad self-test arguments");
  cudaSetDevice(ctx->device);
  return launch_math_selftest(d_x, n, d_out, (cudaStream_t)stream);
}

int lens_wait(lens_ctx *ctx, void *stream, int64_t timeout_ms) {
  if (!ctx) return fail(LENS_EINVAL, "ctx is NULL");
  if (timeout_ms < 0) return fail(LENS_EINVAL, "timeout_ms must be >= 0");
  cudaSetDevice(ctx->device);
  cudaEvent_t ev;
  LENS_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(ev, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    cudaEventDestroy(ev);
    return fail(LENS_ECUDA, "cudaEventRecord: %s", cudaGetErrorString(e));
  }
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    e = cudaEventQuery(ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) {
      cudaEventDestroy(ev);
      return fail(LENS_ECUDA, "stream error: %s", cudaGetErrorString(e));
    }
    auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
    if (ms >= timeout_ms) {
      cudaEventDestroy(ev);
      return fail(LENS_ETIMEOUT, "stream work not finished after %lld ms", (long long)timeout_ms);
    }
    // short polls first (most waits end within a kernel's tail), then back off
    if (ms < 2)
      std::this_thread::yield();
    else
      std::this_thread::sleep_for(std::chrono::microseconds(ms < 50 ? 10 : 100));
  }
  cudaEventDestroy(ev);
  int flag = 0;
  LENS_CUDA_TRY(cudaMemcpy(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    cudaMemset(ctx->d_err, 0, sizeof(int));
    if (flag & ERRBIT_WAIT) return fail(LENS_ETIMEOUT, "a device-side bounded wait gave up");
    return fail(LENS_ECAPACITY, "an image buffer overflowed; the affected chi2 values are NaN");
  }
  return LENS_OK;
}

}  // extern "C"

// Request loop: continuous admission of map and chi2 requests onto a fixed
// set of CUDA streams ("slots"), with admission by device memory.
//
//   submit   -> the request is validated and queued (host copy of its
//               parameter sets); nothing touches the GPU yet.
//   progress -> (1) retires every slot whose completion event has fired,
//               returning its device memory to the arena and reporting the
//               ticket with its queueing and end-to-end latency;
//               (2) admits queued requests onto free slots while the arena
//               can hold their device buffers (inputs, outputs, scratch),
//               shortest expected work first with ageing: each request's
//               rank is its expected GPU time (from the measured rates of
//               its kernels) minus the time it has waited, so a large map
//               waits at most about its own run time behind smaller work.
//               A request that does not fit is skipped so others can start;
//               once the first-ranked request has been skipped MAX_SKIPS
//               times nothing else is admitted until it fits (no starvation).
// Admitted work of different slots overlaps on the device.  Each request runs
// the same kernels as the direct calls, on its own stream and buffers, so its
// result does not depend on what else is in flight.  The arena is one
// cudaMalloc made when the server is created: requests allocate nothing.
#include <algorithm>
#include <chrono>
#include <deque>
#include <map>

#include "lens_internal.cuh"

namespace lens {
namespace {

constexpr int MAX_SKIPS = 64;
constexpr size_t ALIGN = 256;

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

size_t up(size_t v) { return (v + ALIGN - 1) & ~(ALIGN - 1); }

// First-fit allocator over one device block; free ranges coalesce.
struct Arena {
  size_t bytes = 0, used = 0, peak = 0;
  std::map<size_t, size_t> free_;  // offset -> size
  void init(size_t n) {
    bytes = n;
    free_.clear();
    free_[0] = n;
  }
  bool alloc(size_t n, size_t *off) {
    n = up(n);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      *off = it->first;
      const size_t rest = it->second - n, o = it->first + n;
      free_.erase(it);
      if (rest) free_[o] = rest;
      used += n;
      peak = std::max(peak, used);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = up(n);
    used -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

struct Req {
  int64_t ticket = 0;
  lens_request r{};
  std::vector<double> params;
  size_t out_bytes = 0, in_bytes = 0, scratch_bytes = 0, total = 0, off = 0;
  int32_t batch = 0;
  double t_submit = 0, t_admit = 0;
  double cost_ms = 0;  // expected GPU time
  int skips = 0;
};

// Expected GPU time of a request from the rates measured on GB300 (2048^2 x
// 1000 maps: 3.1e11 Hessian / 4.6e11 deflection / 3.5e9 FP64 point-potential
// pairs per s; source-plane chi2: 2.8e9 image evaluations per s; image-plane
// chi2: 1.3e10 grid cells x sets per s).  Only the order matters.
double expected_ms(const lens_request &r, int32_t n_potentials, int32_t nimg) {
  const double cells = (double)r.grid.nx * r.grid.ny;
  if (r.kind == LENS_REQ_MAP) {
    const double pairs = cells * n_potentials;
    if (r.precision == LENS_FP64) return pairs / 3.5e6;
    return pairs / (r.hessian ? 3.1e8 : 4.6e8);
  }
  if (r.kind == LENS_REQ_CHI2_SOURCE) return (double)r.P * nimg / 2.8e6;
  return (double)r.P * cells / 1.3e7;
}

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  Req *req = nullptr;
};

size_t map_out_bytes(const lens_request &r) {
  return (size_t)(r.hessian ? 6 : 2) * r.grid.nx * r.grid.ny * (r.precision == LENS_FP64 ? 8 : 4);
}

}  // namespace
}  // namespace lens

struct lens_server {
  lens_ctx *ctx = nullptr;
  char *pool = nullptr;
  size_t pool_bytes = 0;
  lens::Arena arena;
  std::vector<lens::Slot> slots;
  std::deque<lens::Req *> queue;
  int64_t next_ticket = 1;
};

using namespace lens;

static int launch_req(lens_server *s, Slot &sl, Req *q) {
  lens_ctx *ctx = s->ctx;
  const lens_request &r = q->r;
  char *base = s->pool + q->off;
  cudaStream_t st = sl.st;
  int rc = LENS_OK;
  if (r.kind == LENS_REQ_MAP) {
    Model *m = find_model(ctx, r.handle);
    if (!m) return fail(LENS_ENOTFOUND, "model released while its request was queued");
    if (r.precision == LENS_FP64)
      rc = launch_map_fp64(ctx, m, &r.grid, r.dls_ds, r.hessian != 0, base, st);
    else  // the repair list in the request's own arena memory, after its output
      rc = launch_map_mixed(ctx, m, &r.grid, r.dls_ds, r.hessian != 0, base, st, 0, -1, true,
                            base + up(q->out_bytes));
  } else {
    CSet *c = find_cset(ctx, r.handle);
    Model *m = c ? find_model(ctx, c->model) : nullptr;
    if (!c || !m) return fail(LENS_ENOTFOUND, "constraint set released while its request was queued");
    double *d_params = (double *)(base + up(q->out_bytes));
    if (cudaMemcpyAsync(d_params, q->params.data(), q->in_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return fail(LENS_ECUDA, "parameter upload failed");
    if (r.kind == LENS_REQ_CHI2_SOURCE) {
      rc = launch_chi2_source(ctx, m, c, d_params, r.P, r.variant, (double *)base, st);
    } else {
      const GridCache *gc = find_grid_cache(c, &r.grid);
      if (!gc) return fail(LENS_ENOTFOUND, "grid cache missing");
      void *scratch = base + up(q->out_bytes) + up(q->in_bytes);
      rc = run_chi2_image(ctx, c, gc, d_params, r.P, (double *)base, nullptr, scratch, q->batch, st);
    }
  }
  if (rc) return rc;
  if (cudaMemcpyAsync(r.result, base, q->out_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return fail(LENS_ECUDA, "result download failed");
  if (cudaEventRecord(sl.ev, st) != cudaSuccess) return fail(LENS_ECUDA, "cudaEventRecord failed");
  mark_stream(ctx, st);  // releases of models and constraint sets wait for it
  return LENS_OK;
}

extern "C" {

int lens_server_create(lens_ctx *ctx, int32_t slots, size_t pool_bytes, lens_server **out) {
  if (!ctx || !out) return fail(LENS_EINVAL, "NULL argument");
  if (slots < 1 || slots > 64) return fail(LENS_EINVAL, "slots must be in 1..64");
  if (pool_bytes < ALIGN) return fail(LENS_EINVAL, "pool_bytes too small");
  cudaSetDevice(ctx->device);
  lens_server *s = new lens_server();
  s->ctx = ctx;
  s->pool_bytes = up(pool_bytes);
  int rc = dev_alloc(ctx, (void **)&s->pool, s->pool_bytes);
  if (rc) {
    delete s;
    return rc;
  }
  s->arena.init(s->pool_bytes);
  s->slots.resize(slots);
  for (auto &sl : s->slots)
    if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
      lens_server_destroy(s);
      return fail(LENS_ECUDA, "stream/event creation failed");
    }
  *out = s;
  return LENS_OK;
}

int lens_server_destroy(lens_server *s) {
  if (!s) return LENS_OK;
  cudaSetDevice(s->ctx->device);
  for (auto &sl : s->slots) {
    if (sl.st) cudaStreamSynchronize(sl.st);
    delete sl.req;
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.st) cudaStreamDestroy(sl.st);
  }
  for (Req *q : s->queue) delete q;
  dev_free(s->ctx, s->pool, s->pool_bytes);
  delete s;
  return LENS_OK;
}

int lens_server_submit(lens_server *s, const lens_request *r, int64_t *ticket) {
  if (!s || !r || !ticket) return fail(LENS_EINVAL, "NULL argument");
  if (!r->result) return fail(LENS_EINVAL, "result is NULL");
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, r->result) != cudaSuccess || pa.type != cudaMemoryTypeHost) {
    cudaGetLastError();
    return fail(LENS_EINVAL, "result must be page-locked host memory (cudaHostAlloc / cudaHostRegister)");
  }
  Req *q = new Req();
  q->r = *r;
  lens_ctx *ctx = s->ctx;
  int rc = LENS_OK;
  if (r->kind == LENS_REQ_MAP) {
    if (!find_model(ctx, r->handle)) rc = fail(LENS_ENOTFOUND, "model %lld not found", (long long)r->handle);
    else if ((rc = check_grid(&r->grid))) {
    } else if (!(std::isfinite(r->dls_ds) && r->dls_ds > 0)) rc = fail(LENS_EINVAL, "dls_ds must be > 0");
    else if (r->precision != LENS_FP64 && r->precision != LENS_MIXED) rc = fail(LENS_EINVAL, "bad precision");
    q->out_bytes = map_out_bytes(*r);
    if (r->precision == LENS_MIXED) q->scratch_bytes = map_repair_bytes(&r->grid);
  } else if (r->kind == LENS_REQ_CHI2_SOURCE || r->kind == LENS_REQ_CHI2_IMAGE) {
    CSet *c = find_cset(ctx, r->handle);
    if (!c) rc = fail(LENS_ENOTFOUND, "constraint set %lld not found", (long long)r->handle);
    else if (r->P < 1 || !r->params) rc = fail(LENS_EINVAL, "chi2 request needs P >= 1 and params");
    else if (r->kind == LENS_REQ_CHI2_SOURCE && (r->variant < 0 || r->variant > 2)) rc = fail(LENS_EINVAL, "bad variant");
    else if (r->kind == LENS_REQ_CHI2_IMAGE && (rc = check_grid(&r->grid))) {
    } else if (r->kind == LENS_REQ_CHI2_IMAGE && (rc = check_chi2_image_limits(c, &r->grid))) {
    }
    if (!rc) {
      q->params.assign(r->params, r->params + (size_t)r->P * 14);
      q->r.params = nullptr;
      q->out_bytes = (size_t)r->P * sizeof(double);
      q->in_bytes = (size_t)r->P * 14 * sizeof(double);
      if (r->kind == LENS_REQ_CHI2_IMAGE) {
        // the static deflection of (constraint set, grid) is model-resident
        // data: built once, synchronously, the first time the pair is seen
        if (!find_grid_cache(c, &r->grid)) {
          rc = build_grid_cache(ctx, c, &r->grid, s->slots[0].st);
          if (!rc && cudaStreamSynchronize(s->slots[0].st) != cudaSuccess) rc = fail(LENS_ECUDA, "grid cache build");
        }
        q->batch = std::min<int32_t>(r->P, 16);
        q->scratch_bytes = chi2_image_scratch_bytes(c, q->batch);
      }
    }
  } else {
    rc = fail(LENS_EINVAL, "unknown request kind %d", r->kind);
  }
  if (!rc) {
    if (r->kind == LENS_REQ_MAP) {
      q->cost_ms = expected_ms(*r, find_model(ctx, r->handle)->n, 0);
    } else {
      const CSet *c = find_cset(ctx, r->handle);
      q->cost_ms = expected_ms(*r, 0, c->nimg);
    }
    q->total = up(q->out_bytes) + up(q->in_bytes) + up(q->scratch_bytes);
    if (q->total > s->pool_bytes)
      rc = fail(LENS_ENOMEM, "request needs %zu device bytes, the server pool holds %zu", q->total, s->pool_bytes);
  }
  if (rc) {
    delete q;
    return rc;
  }
  q->ticket = s->next_ticket++;
  q->t_submit = now_ms();
  s->queue.push_back(q);
  *ticket = q->ticket;
  return LENS_OK;
}

int lens_server_progress(lens_server *s, lens_completion *done, int32_t cap, int32_t *n_done) {
  if (!s || !n_done || (cap > 0 && !done)) return fail(LENS_EINVAL, "NULL argument");
  cudaSetDevice(s->ctx->device);
  *n_done = 0;
  int rc = LENS_OK;
  // 1. retire
  for (auto &sl : s->slots) {
    if (!sl.req || *n_done >= cap) continue;
    cudaError_t e = cudaEventQuery(sl.ev);
    if (e == cudaErrorNotReady) continue;
    Req *q = sl.req;
    lens_completion &c = done[(*n_done)++];
    c.ticket = q->ticket;
    c.status = e == cudaSuccess ? LENS_OK : LENS_ECUDA;
    c.queue_ms = q->t_admit - q->t_submit;
    c.latency_ms = now_ms() - q->t_submit;
    s->arena.release(q->off, q->total);
    delete q;
    sl.req = nullptr;
    if (e != cudaSuccess) rc = fail(LENS_ECUDA, "request failed: %s", cudaGetErrorString(e));
  }
  // 2. admit, shortest expected work first with ageing, while slots and
  // memory allow
  const double now = now_ms();
  std::vector<Req *> order(s->queue.begin(), s->queue.end());
  std::stable_sort(order.begin(), order.end(), [now](const Req *a, const Req *b) {
    return a->cost_ms - (now - a->t_submit) < b->cost_ms - (now - b->t_submit);
  });
  for (size_t k = 0; k < order.size(); ++k) {
    Slot *free_slot = nullptr;
    for (auto &sl : s->slots)
      if (!sl.req) {
        free_slot = &sl;
        break;
      }
    if (!free_slot) break;
    Req *q = order[k];
    if (k > 0 && order[0]->skips >= MAX_SKIPS && order[0]->t_admit == 0) break;
    size_t off;
    if (!s->arena.alloc(q->total, &off)) {
      if (k == 0) ++q->skips;
      continue;
    }
    q->off = off;
    q->t_admit = now_ms();
    free_slot->req = q;
    s->queue.erase(std::find(s->queue.begin(), s->queue.end(), q));
    int lrc = launch_req(s, *free_slot, q);
    if (lrc) {
      // report the failed launch as a completed ticket with its error
      s->arena.release(q->off, q->total);
      free_slot->req = nullptr;
      if (*n_done < cap) {
        lens_completion &c = done[(*n_done)++];
        c.ticket = q->ticket;
        c.status = lrc;
        c.queue_ms = q->t_admit - q->t_submit;
        c.latency_ms = now_ms() - q->t_submit;
      }
      delete q;
      rc = lrc;
    }
  }
  return rc;
}

int lens_server_cancel(lens_server *s, int64_t ticket) {
  if (!s) return fail(LENS_EINVAL, "NULL argument");
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
    if ((*it)->ticket == ticket) {
      delete *it;
      s->queue.erase(it);
      return LENS_OK;
    }
  return fail(LENS_ENOTFOUND, "ticket %lld is not queued (unknown, admitted or finished)", (long long)ticket);
}

int lens_server_stats(const lens_server *s, lens_server_info *info) {
  if (!s || !info) return fail(LENS_EINVAL, "NULL argument");
  info->queued = (int32_t)s->queue.size();
  int32_t inflight = 0;
  for (auto &sl : s->slots) inflight += sl.req != nullptr;
  info->inflight = inflight;
  info->pool_bytes = s->pool_bytes;
  info->pool_used = s->arena.used;
  info->pool_peak = s->arena.peak;
  return LENS_OK;
}

}  // extern "C"

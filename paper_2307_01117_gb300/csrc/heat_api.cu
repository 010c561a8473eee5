// heat_api.cu -- the C ABI of include/heat.h: context lifetime, argument
// validation, state transfer and dispatch to the kernel forms.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>
#include <stdio.h>

#include "dp_emul.cuh"
#include "heat_internal.cuh"

using heat::DevStatus;

namespace {
// NVTX range over a host call (visible in Nsight timelines; a no-op without a tool).
struct NvtxRange {
  explicit NvtxRange(const char *msg) { nvtxRangePushA(msg); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

namespace {

constexpr int64_t kStageElems = int64_t(1) << 22;  // binary64 staging chunk for HEAT_F32C transfers (32 MiB)
constexpr int kDefaultEmulShare = -1;              // tiles of 32 on the integer pipes: chosen per ring
constexpr int kDefaultSplit = 0;                   // per-point FP64/integer split level by default

bool is_finite(double x) { return isfinite(x) != 0; }

void free_ctx(heat_ctx *c) {
  if (!c) return;
  if (c->own_stream) cudaStreamSynchronize(c->own_stream);
  if (c->stream && c->stream != c->own_stream) cudaStreamSynchronize(c->stream);
  for (int i = 0; i < 2; ++i)
    if (c->buf[i]) cudaFree(c->buf[i]);
  if (c->dstat) cudaFree(c->dstat);
  if (c->hstat) cudaFreeHost(c->hstat);
  if (c->mbox) cudaFree(c->mbox);
  if (c->seg_start) cudaFree(c->seg_start);
  if (c->partials) cudaFree(c->partials);
  if (c->hsum) cudaFreeHost(c->hsum);
  if (c->xstage) cudaFree(c->xstage);
  if (c->tile_counter) cudaFree(c->tile_counter);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  heat::free_wave(c);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  free(c);
}

// Wait for the stream, then fold the device status word into the sticky host
// error.  Returns the sticky error (HEAT_OK if none).
int sync_status(heat_ctx *c) {
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return HEAT_ECUDA;
  if (cudaMemcpyAsync(c->hstat, c->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return HEAT_ECUDA;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return HEAT_ECUDA;
  if (c->hstat->code != HEAT_OK && c->host_error == HEAT_OK) c->host_error = c->hstat->code;
  return c->host_error;
}

int reset_status(heat_ctx *c) {
  c->host_error = HEAT_OK;
  // the temporal-blocking counters too (a launch cut short by an error may have
  // left them nonzero)
  c->counter_dirty = 0;
  if (cudaMemsetAsync(c->tile_counter, 0, 2 * sizeof(unsigned long long), c->stream) != cudaSuccess)
    return HEAT_ECUDA;
  return heat::cuda_status(cudaMemsetAsync(c->dstat, 0, sizeof(DevStatus), c->stream));
}

}  // namespace

// Multi-launch runs (one launch per step or per T steps) are captured into a
// CUDA graph the first time and replayed while the run key -- form, depth,
// steps, starting buffer, arithmetic, layout, stream -- stays the same: the
// launches then cost one graph launch instead of one host call each.
int run_graphed(heat_ctx *c, int form, int64_t nt) {
  const int T = c->T;
  const int64_t depth = form == HEAT_FORM_PLAIN ? 1 : (T > 0 ? T : heat::tblock_default_T(c));
  if ((nt + depth - 1) / depth > 8192) return HEAT_ENOTSUP;  // keep graphs small
  const unsigned long long key[8] = {(unsigned long long)form, (unsigned long long)T, (unsigned long long)nt,
                                     (unsigned long long)c->cur, (unsigned long long)c->arith,
                                     (unsigned long long)c->tb_layout,
                                     ((unsigned long long)c->split_level << 32) | heat::tblock_emul_mask(c),
                                     (unsigned long long)(uintptr_t)c->stream};
  if (c->graph_exec && memcmp(key, c->graph_key, sizeof(key)) == 0) {
    if (cudaGraphLaunch(c->graph_exec, c->stream) != cudaSuccess) return HEAT_ECUDA;
    c->cur ^= c->graph_cur_flip;
    c->steps += nt;
    c->last_T = c->graph_last_T;
    c->last_launches = c->graph_last_launches;
    return HEAT_OK;
  }
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
  const int cur0 = c->cur;
  const int64_t steps0 = c->steps;
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return HEAT_ENOTSUP;
  }
  const int rc = form == HEAT_FORM_PLAIN ? heat::run_plain(c, nt) : heat::run_tblock(c, nt);
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(c->stream, &graph);
  cudaGraphExec_t exec = nullptr;
  if (rc != HEAT_OK || ec != cudaSuccess || !graph ||
      cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    c->cur = cur0;  // nothing ran
    c->steps = steps0;
    return rc != HEAT_OK ? rc : HEAT_ENOTSUP;
  }
  cudaGraphDestroy(graph);
  if (cudaGraphLaunch(exec, c->stream) != cudaSuccess) {
    cudaGraphExecDestroy(exec);
    c->cur = cur0;
    c->steps = steps0;
    return HEAT_ECUDA;
  }
  c->graph_exec = exec;
  memcpy(c->graph_key, key, sizeof(key));
  c->graph_cur_flip = c->cur ^ cur0;
  c->graph_last_T = c->last_T;
  c->graph_last_launches = c->last_launches;
  return HEAT_OK;
}

extern "C" {

int heat_create(heat_ctx **out, int64_t nx, int32_t np, double k, double dt, double dx, heat_dtype dtype) {
  if (!out) return HEAT_EINVAL;
  *out = nullptr;
  if (nx < 1 || np < 1) return HEAT_EINVAL;
  if (nx > INT64_MAX / np) return HEAT_EINVAL;
  if (!is_finite(k) || !is_finite(dt) || !is_finite(dx) || dx == 0.0) return HEAT_EINVAL;
  if (dtype != HEAT_F64 && dtype != HEAT_F32C) return HEAT_EINVAL;
  const int64_t N = nx * (int64_t)np;
  const size_t elem = dtype == HEAT_F64 ? sizeof(double) : sizeof(float);
  if ((uint64_t)N > (uint64_t)(SIZE_MAX / 2 / elem)) return HEAT_EINVAL;
  const double r = (k * dt) / (dx * dx);
  if (!is_finite(r)) return HEAT_EINVAL;

  heat_ctx *c = (heat_ctx *)calloc(1, sizeof(heat_ctx));
  if (!c) return HEAT_ENOMEM;
  c->geo.nx = nx;
  c->geo.np = np;
  c->geo.N = N;
  c->r = r;
  c->rf = (float)r;
  c->dtype = dtype;
  c->elem = elem;
  c->form = HEAT_FORM_AUTO;
  c->T = 0;
  c->arith = HEAT_ARITH_EXACT;
  c->wait_ns = 2000000000LL;
  c->inj_segment = -1;
  c->inj_step = 0;
  heat_set_emulation(c, kDefaultEmulShare);
  heat_set_split(c, kDefaultSplit);
  c->tb_layout = 1;  // contiguous per-lane ownership (measured fastest for both dtypes)
  c->graphs = 1;
  int rc = HEAT_OK;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    cudaGetLastError();
    free(c);
    return HEAT_ECUDA;
  }
  if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    free(c);
    return HEAT_ECUDA;
  }
  c->stream = c->own_stream;
  for (int i = 0; i < 2 && rc == HEAT_OK; ++i)
    if (cudaMalloc(&c->buf[i], (size_t)N * elem) != cudaSuccess) rc = HEAT_ENOMEM;
  if (rc == HEAT_OK && cudaMalloc((void **)&c->dstat, sizeof(DevStatus)) != cudaSuccess) rc = HEAT_ENOMEM;
  if (rc == HEAT_OK && cudaMallocHost((void **)&c->hstat, sizeof(DevStatus)) != cudaSuccess) rc = HEAT_ENOMEM;
  if (rc == HEAT_OK && cudaMalloc((void **)&c->partials, sizeof(double) * (heat::kSumBlocks + 1)) != cudaSuccess)
    rc = HEAT_ENOMEM;
  if (rc == HEAT_OK && cudaMallocHost((void **)&c->hsum, sizeof(double)) != cudaSuccess) rc = HEAT_ENOMEM;
  if (rc == HEAT_OK && cudaMalloc((void **)&c->tile_counter, 2 * sizeof(unsigned long long)) != cudaSuccess)
    rc = HEAT_ENOMEM;
  if (rc == HEAT_OK && cudaMemsetAsync(c->tile_counter, 0, 2 * sizeof(unsigned long long), c->stream) != cudaSuccess)
    rc = HEAT_ECUDA;
  if (rc == HEAT_OK) {
    for (int i = 0; i < 2 && rc == HEAT_OK; ++i)
      if (cudaMemsetAsync(c->buf[i], 0, (size_t)N * elem, c->stream) != cudaSuccess) rc = HEAT_ECUDA;
    if (rc == HEAT_OK) rc = reset_status(c);
    if (rc == HEAT_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = HEAT_ECUDA;
  }
  if (rc != HEAT_OK) {
    cudaGetLastError();
    free_ctx(c);
    return rc;
  }
  *out = c;
  return HEAT_OK;
}

void heat_destroy(heat_ctx *c) { free_ctx(c); }

// Copies n binary64 values (host or device source) into the state buffer.
static int load_state(heat_ctx *c, const double *src, int64_t n, cudaMemcpyKind kind) {
  if (!c || !src) return HEAT_EINVAL;
  if (n != c->geo.N) return HEAT_EINVAL;
  int rc = reset_status(c);
  if (rc != HEAT_OK) return rc;
  void *dst = c->buf[c->cur];
  if (c->dtype == HEAT_F64) {
    if (cudaMemcpyAsync(dst, src, (size_t)n * sizeof(double), kind, c->stream) != cudaSuccess) return HEAT_ECUDA;
  } else if (kind == cudaMemcpyDeviceToDevice) {
    rc = heat::convert_f64_to_state(c, src, dst, n);
    if (rc != HEAT_OK) return rc;
  } else {
    // binary64 input does not fit the binary32 buffers: stage it through two
    // device chunks used in turn and round each chunk on the device; stream
    // order keeps a chunk's next copy behind its conversion
    if (!c->xstage && cudaMalloc((void **)&c->xstage, 2 * (size_t)kStageElems * sizeof(double)) != cudaSuccess)
      return HEAT_ENOMEM;
    int64_t i = 0;
    for (int64_t off = 0; off < n && rc == HEAT_OK; off += kStageElems, ++i) {
      const int64_t m = n - off < kStageElems ? n - off : kStageElems;
      double *stage = c->xstage + (i & 1) * kStageElems;
      if (cudaMemcpyAsync(stage, src + off, (size_t)m * sizeof(double), kind, c->stream) != cudaSuccess) rc = HEAT_ECUDA;
      if (rc == HEAT_OK) rc = heat::convert_f64_to_state(c, stage, (float *)dst + off, m);
    }
    if (rc != HEAT_OK) {
      cudaStreamSynchronize(c->stream);
      return rc;
    }
  }
  c->steps = 0;
  return HEAT_OK;
}

int heat_set(heat_ctx *c, const double *host_u, int64_t n) {
  int rc = load_state(c, host_u, n, cudaMemcpyHostToDevice);
  if (rc != HEAT_OK) return rc;
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? HEAT_OK : HEAT_ECUDA;
}

int heat_set_device(heat_ctx *c, const double *dev_u, int64_t n) {
  return load_state(c, dev_u, n, cudaMemcpyDeviceToDevice);
}

static int store_state(heat_ctx *c, double *dst, int64_t n, cudaMemcpyKind kind) {
  if (!c || !dst) return HEAT_EINVAL;
  if (n != c->geo.N) return HEAT_EINVAL;
  int rc = sync_status(c);
  if (rc != HEAT_OK) return rc;
  const void *src = c->buf[c->cur];
  if (c->dtype == HEAT_F64) {
    if (cudaMemcpyAsync(dst, src, (size_t)n * sizeof(double), kind, c->stream) != cudaSuccess) return HEAT_ECUDA;
  } else if (kind == cudaMemcpyDeviceToDevice) {
    rc = heat::convert_state_to_f64(c, src, dst, n);
    if (rc != HEAT_OK) return rc;
  } else {
    // widen chunk by chunk into two device staging chunks used in turn
    if (!c->xstage && cudaMalloc((void **)&c->xstage, 2 * (size_t)kStageElems * sizeof(double)) != cudaSuccess)
      return HEAT_ENOMEM;
    int64_t i = 0;
    for (int64_t off = 0; off < n && rc == HEAT_OK; off += kStageElems, ++i) {
      const int64_t m = n - off < kStageElems ? n - off : kStageElems;
      double *stage = c->xstage + (i & 1) * kStageElems;
      rc = heat::convert_state_to_f64(c, (const float *)src + off, stage, m);
      if (rc == HEAT_OK && cudaMemcpyAsync(dst + off, stage, (size_t)m * sizeof(double), kind, c->stream) != cudaSuccess)
        rc = HEAT_ECUDA;
    }
    if (rc != HEAT_OK) {
      cudaStreamSynchronize(c->stream);
      return rc;
    }
  }
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? HEAT_OK : HEAT_ECUDA;
}

int heat_get(heat_ctx *c, double *host_u, int64_t n) { return store_state(c, host_u, n, cudaMemcpyDeviceToHost); }

int heat_get_device(heat_ctx *c, double *dev_u, int64_t n) { return store_state(c, dev_u, n, cudaMemcpyDeviceToDevice); }

int heat_run(heat_ctx *c, int64_t nt) {
  if (!c || nt < 0) return HEAT_EINVAL;
  if (c->host_error != HEAT_OK) return HEAT_ESTATE;
  if (nt == 0) return HEAT_OK;
  char label[96];
  snprintf(label, sizeof(label), "heat_run nt=%lld N=%lld form=%d T=%d", (long long)nt, (long long)c->geo.N,
           c->form, c->T);
  NvtxRange range(label);
  int form = c->form;
  // default: one cluster launch for small rings (latency-bound: one launch for
  // all steps, ghost exchange through distributed shared memory), temporal
  // blocking otherwise.  Binary64 switches at 6144 points: above, the
  // temporal-blocking launches (graph-replayed, depth 24) are faster than one
  // cluster's 16 SMs (0.67 vs 1.1 us per step at 8192 points; 0.56 vs 0.67
  // for the cluster at 4000).
  if (form == HEAT_FORM_AUTO) {
    const int Tc = c->T > 0 ? c->T : (c->dtype == HEAT_F32C ? 32 : 16);
    const int64_t limit = c->dtype == HEAT_F32C ? heat::cluster_max_points(c, Tc) : 6144;
    form = c->geo.N <= limit && c->geo.N <= heat::cluster_max_points(c, Tc) ? HEAT_FORM_CLUSTER : HEAT_FORM_TBLOCK;
    // mid-size binary64 rings: dependency-driven temporal blocking in one launch
    if (form == HEAT_FORM_TBLOCK && heat::wave_preferred(c)) form = HEAT_FORM_PERSIST_TB;
  }
  c->last_form = form;
  c->last_T = 1;
  c->last_launches = 0;
  if (c->graphs && (form == HEAT_FORM_PLAIN || form == HEAT_FORM_TBLOCK)) {
    const int rc = run_graphed(c, form, nt);
    if (rc != HEAT_ENOTSUP) return rc;  // HEAT_ENOTSUP: not graphable, run directly
  }
  switch (form) {
    case HEAT_FORM_PLAIN: return heat::run_plain(c, nt);
    case HEAT_FORM_PERSIST: return heat::run_persist(c, nt);
    case HEAT_FORM_TBLOCK: return heat::run_tblock(c, nt);
    case HEAT_FORM_CLUSTER: return heat::run_cluster(c, nt);
    case HEAT_FORM_PERSIST_TB: return heat::run_persist_tb(c, nt);
    default: return HEAT_EINVAL;
  }
}

int heat_last_run(const heat_ctx *c, int *form, int *T, int64_t *launches, int *segments) {
  if (!c) return HEAT_EINVAL;
  if (form) *form = c->last_form;
  if (T) *T = c->last_T;
  if (launches) *launches = c->last_launches;
  if (segments) *segments = c->last_segments;
  return HEAT_OK;
}

int heat_sync(heat_ctx *c) {
  if (!c) return HEAT_EINVAL;
  return sync_status(c);
}

int heat_set_stream(heat_ctx *c, void *cuda_stream) {
  if (!c) return HEAT_EINVAL;
  cudaStream_t next = cuda_stream ? (cudaStream_t)cuda_stream : c->own_stream;
  if (next == c->stream) return HEAT_OK;
  // keep queued work ordered across the switch
  cudaEvent_t ev;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return HEAT_ECUDA;
  int rc = HEAT_OK;
  if (cudaEventRecord(ev, c->stream) != cudaSuccess || cudaStreamWaitEvent(next, ev, 0) != cudaSuccess) rc = HEAT_ECUDA;
  cudaEventDestroy(ev);
  if (rc == HEAT_OK) c->stream = next;
  return rc;
}

int heat_set_form(heat_ctx *c, int form, int T) {
  if (!c) return HEAT_EINVAL;
  if (form < HEAT_FORM_PLAIN || form > HEAT_FORM_PERSIST_TB) return HEAT_EINVAL;
  if (T < 0 || T > heat::kMaxT) return HEAT_EINVAL;
  c->form = form;
  c->T = T;
  return HEAT_OK;
}

int heat_set_graphs(heat_ctx *c, int enable) {
  if (!c) return HEAT_EINVAL;
  c->graphs = enable ? 1 : 0;
  return HEAT_OK;
}

int heat_set_layout(heat_ctx *c, int layout) {
  if (!c || layout < 0 || layout > 1) return HEAT_EINVAL;
  c->tb_layout = layout;
  return HEAT_OK;
}

int heat_set_split(heat_ctx *c, int level) {
  if (!c || level < 0 || level > 17) return HEAT_EINVAL;
  c->split_level = level;
  return HEAT_OK;
}

int heat_set_emulation(heat_ctx *c, int share) {
  if (!c || share < -1 || share > 32) return HEAT_EINVAL;
  c->emul_auto = share < 0;
  c->emul_share = share;
  if (share < 0) share = 0;
  c->emul_mask = heat::emul_share_mask(share);
  return HEAT_OK;
}

int heat_get_emulation(const heat_ctx *c, int *share) {
  if (!c || !share) return HEAT_EINVAL;
  unsigned mask = heat::tblock_emul_mask(c);
  // integer tiles need a screen that admits values at the depth in use (the
  // contiguous layout; the strided layout checks per operation instead)
  uint64_t rb;
  memcpy(&rb, &c->r, sizeof(rb));
  int lo = 0, hi = 0;
  const int T = c->T > 0 ? c->T : heat::tblock_default_T(c);
  if (c->tb_layout == 1 && !heat::emul::domain_bounds(rb, T, lo, hi)) mask = 0u;
  // the library's choice is adaptive (two-ended tile claiming): reported as -1
  *share = c->emul_auto && mask ? -1 : __builtin_popcount(mask);
  return HEAT_OK;
}

int heat_set_segments(heat_ctx *c, int segments) {
  if (!c || segments < -1) return HEAT_EINVAL;
  c->segments = segments;
  return HEAT_OK;
}

int heat_set_arith(heat_ctx *c, int arith) {
  if (!c) return HEAT_EINVAL;
  if (arith != HEAT_ARITH_EXACT && arith != HEAT_ARITH_FMA) return HEAT_EINVAL;
  c->arith = arith;
  return HEAT_OK;
}

int heat_sum(heat_ctx *c, double *out) {
  if (!c || !out) return HEAT_EINVAL;
  int rc = sync_status(c);
  if (rc != HEAT_OK) return rc;
  rc = heat::sum_state(c, c->partials + heat::kSumBlocks);
  if (rc != HEAT_OK) return rc;
  if (cudaMemcpyAsync(c->hsum, c->partials + heat::kSumBlocks, sizeof(double), cudaMemcpyDeviceToHost, c->stream) !=
      cudaSuccess)
    return HEAT_ECUDA;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return HEAT_ECUDA;
  *out = *c->hsum;
  return HEAT_OK;
}

int heat_steps(const heat_ctx *c, int64_t *out) {
  if (!c || !out) return HEAT_EINVAL;
  *out = c->steps;
  return HEAT_OK;
}

int heat_info(const heat_ctx *c, int64_t *nx, int32_t *np, double *r, int *dtype) {
  if (!c) return HEAT_EINVAL;
  if (nx) *nx = c->geo.nx;
  if (np) *np = c->geo.np;
  if (r) *r = c->r;
  if (dtype) *dtype = (int)c->dtype;
  return HEAT_OK;
}

int heat_state_ptr(heat_ctx *c, void **dev_ptr) {
  if (!c || !dev_ptr) return HEAT_EINVAL;
  *dev_ptr = c->buf[c->cur];
  return HEAT_OK;
}

int heat_set_wait_limit(heat_ctx *c, int64_t ns) {
  if (!c || ns < 1) return HEAT_EINVAL;
  c->wait_ns = ns;
  return HEAT_OK;
}

int heat_inject_stall(heat_ctx *c, int32_t segment, int64_t from_step) {
  if (!c || from_step < 0) return HEAT_EINVAL;
  c->inj_segment = segment < 0 ? -1 : segment;
  c->inj_step = from_step;
  return HEAT_OK;
}

const char *heat_strerror(int code) {
  switch (code) {
    case HEAT_OK: return "ok";
    case HEAT_EINVAL: return "invalid argument";
    case HEAT_ENOMEM: return "device allocation failed";
    case HEAT_ECUDA: return "CUDA runtime error";
    case HEAT_ETIMEOUT: return "bounded wait for a neighbour's ghost value ran out";
    case HEAT_ESTATE: return "a device error is pending; reload the state with heat_set";
    case HEAT_ENOTSUP: return "combination not supported";
    default: return "unknown status";
  }
}

}  // extern "C"

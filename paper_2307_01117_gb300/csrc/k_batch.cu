// k_batch.cu -- batched independent rings (the paper's Section 2 problem, many
// instances at once) in one device arena, advanced by one persistent launch
// driven by a work table.
//
// Work table (built on the host for each run, rings sorted by the number of
// T-step levels they need, longest first):
//   ring i: arena offset, n points, steps this run, ntiles warp tiles, r;
//   units (level b, ring i, tile j) are numbered level-major, so the rings
//   active at level b are a prefix of the sorted list and a unit number decodes
//   with two searches (over the per-level and per-ring prefix sums).
// A warp claims a chunk of consecutive units from a launch-wide counter.  Unit
// (b, i, j) advances tile j of ring i from time bT to bT + steps_b with the
// register-resident temporal-blocking core (wave_core.cuh), after waiting
// (bounded) until tiles j-1, j, j+1 of the ring have finished level b-1.
// Units are numbered level-major and claimed in increasing order, and a warp
// runs its chunk in order, so every unit a warp waits for has a smaller number
// and was claimed earlier by a warp that is running it; the warp holding the
// smallest unfinished unit therefore never waits on anything unfinished, and
// the launch makes progress with any number of resident CTAs.  No co-residency
// is needed: the kernel is an ordinary launch, and two batches (binary64 and
// binary32) can share the GPU.  The same wait covers the write-after-read
// hazard on the output buffer, which level b-1's neighbours read.
//
// Windows wrap around the ring's ends with modular indices.  Every point is
// computed from the same operands as in the single-ring forms, so each ring's
// result is bitwise its solo result.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <numeric>
#include <string>
#include <vector>

#include "wave_core.cuh"

static constexpr int64_t kAlignPointsHost = 64;  // ring placement granularity in the arena (points)

namespace heat {
namespace {

constexpr int kBWarps = 4;
constexpr int kChunk = 4;  // consecutive units per claim

struct BRing {
  int64_t off;        // arena offset in points
  int64_t n;          // ring length
  int64_t steps;      // steps this run
  int64_t nseg;       // warp tiles
  int64_t done_base;  // index of tile 0's done counter
  double r;
  float rf;
  int parity;         // arena buffer holding the state at the start of the run
  emul::MulX mx;      // r for the integer-pipe tiles (binary64, exact reading)
  int dom_lo, dom_hi; // their input screen for T steps (empty: dom_lo > dom_hi)
  unsigned emul_mask; // bit (tile mod 32) set: that tile on the integer pipes
  int p2_hi_add, p2_hi_xor;  // r = +-2^k: screened FP64-unit tiles move the product's exponent
};

struct BatchArgs {
  void *arena0;
  void *arena1;
  const BRing *rings;
  const int64_t *segp;    // prefix sums of nseg (count + 1)
  const int64_t *levp;    // prefix sums of units per level (L + 1)
  const int32_t *active;  // rings active at each level (L)
  int L;
  int T;
  int dual;  // binary64 under the library's share: integer-pipe warps and FP64-unit warps
  unsigned *done;
  unsigned long long *counter;
  DevStatus *st;
  long long wait_ns;
  int inj_ring;        // test hook: table index of a ring whose tile stops publishing (-1: none)
  long long inj_seg;
  long long inj_level;
};

// Largest index k in [lo, hi) with v[k] <= x (v nondecreasing, v[lo] <= x),
// found by the whole warp: each round every lane probes one of 32 evenly
// spaced entries, so a round narrows the range 32-fold.
__device__ __forceinline__ int64_t floor_index_warp(const int64_t *v, int64_t lo, int64_t hi, int64_t x, int lane) {
  while (hi - lo > 1) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t k = lo + (int64_t)lane * step;
    const unsigned m = __ballot_sync(tb::kFull, k < hi && __ldcg(v + k) <= x);
    lo += (int64_t)(31 - __clz(m)) * step;  // the probes at or below x are a prefix of the lanes
    hi = lo + step < hi ? lo + step : hi;
  }
  return lo;
}

template <int MODE, int EP>
__global__ void __launch_bounds__(kBWarps * 32, MODE == 2 ? 1 : 8) k_batch(BatchArgs a) {  // MODE: 0 exact, 1 fused, 2 binary32
  using T = typename tb::TBCx<MODE, EP>::T;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int64_t total = a.levp[a.L];
  const bool int_warp = MODE == 0 && a.dual && (((blockIdx.x ^ wib) & 1) != 0);
  // The next chunk is claimed before the current one is computed (its round
  // trip overlaps the work); chunks still run in increasing order.
  unsigned long long next = 0;
  if (lane == 0) next = atomicAdd(a.counter, (unsigned long long)kChunk);
  for (;;) {
    unsigned long long u0 = next;
    int go = 1;
    if (lane == 0) {
      go = (int64_t)u0 < total && !wave::aborted(a.st);
      if (go) next = atomicAdd(a.counter, (unsigned long long)kChunk);
    }
    u0 = __shfl_sync(tb::kFull, u0, 0);
    if (!__shfl_sync(tb::kFull, go, 0)) break;
    const int64_t u1 = (int64_t)u0 + kChunk < total ? (int64_t)u0 + kChunk : total;
    int64_t b = -1, i = 0, j = 0, lev_end = 0, ring_end = 0;
    bool stop = false;
    for (int64_t u = (int64_t)u0; u < u1; ++u) {
      if (u < lev_end && u < ring_end) {
        ++j;  // the next tile of the same ring and level
      } else {
        b = floor_index_warp(a.levp, 0, a.L, u, lane);
        const int64_t rel = u - __ldcg(a.levp + b);
        i = floor_index_warp(a.segp, 0, __ldcg(a.active + b), rel, lane);
        j = rel - __ldcg(a.segp + i);
        lev_end = __ldcg(a.levp + b + 1);
        ring_end = u - j + __ldcg(a.segp + i + 1) - __ldcg(a.segp + i);
      }
      const BRing &R = a.rings[i];
      const int64_t nseg = R.nseg, base = R.done_base;
      if (b > 0 && !wave::wait_neighbours(a.done + base, nseg, j, (unsigned)b, a.wait_ns, a.st, (int)i, lane)) {
        stop = true;
        break;
      }
      int64_t lo, hi;
      wave::tile_bounds(R.n, nseg, j, lo, hi);
      const int par = R.parity ^ (int)(b & 1);
      const T *src = (const T *)(par ? a.arena1 : a.arena0) + R.off;
      T *dst = (T *)(par ? a.arena0 : a.arena1) + R.off;
      const int64_t left = R.steps - b * a.T;
      const int steps = (int)(left < a.T ? left : a.T);
      bool int_tile = false, p2 = false;
      wave::Engine e;
      if constexpr (MODE == 0) {
        int_tile = a.dual && R.emul_mask != 0u ? int_warp : ((R.emul_mask >> (unsigned)(j & 31)) & 1u) != 0;
        p2 = R.mx.pow2 != 0;
        e.mx = R.mx;
        e.dom_lo = R.dom_lo;
        e.dom_hi = R.dom_hi;
        e.p2_hi_add = R.p2_hi_add;
        e.p2_hi_xor = R.p2_hi_xor;
      }
      wave::advance_tile<MODE, EP>(src, dst, R.n, lo, hi, a.T, steps, R.r, R.rf, int_tile, p2, e, lane);
      if (!(i == a.inj_ring && j == a.inj_seg && b >= a.inj_level))
        wave::publish(a.done + base + j, (unsigned)(b + 1), lane);
    }
    if (stop) break;
  }
}

__global__ void k_b_f64_to_f32(const double *__restrict__ s, float *__restrict__ d, int64_t n) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += st) d[i] = __double2float_rn(s[i]);
}

__global__ void k_b_f32_to_f64(const float *__restrict__ s, double *__restrict__ d, int64_t n) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += st) d[i] = (double)s[i];
}

template <int MODE, int EP>
cudaError_t launch_batch_ep(BatchArgs &a, int grid, cudaStream_t st) {
  k_batch<MODE, EP><<<grid, kBWarps * 32, 0, st>>>(a);
  return cudaGetLastError();
}

template <int MODE, int EP>
int per_sm_ctas_ep() {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<MODE, EP>, kBWarps * 32, 0) != cudaSuccess)
    return 0;
  return per_sm;
}

// Warp windows the batch kernel is built for (points per lane, by dtype).
template <int MODE>
constexpr int kEps[3] = {MODE == 2 ? 8 : 4, MODE == 2 ? 16 : 8, MODE == 2 ? 32 : 16};

template <int MODE>
cudaError_t launch_batch(BatchArgs &a, int ep, int grid, cudaStream_t st) {
  return ep == kEps<MODE>[0]   ? launch_batch_ep<MODE, kEps<MODE>[0]>(a, grid, st)
         : ep == kEps<MODE>[1] ? launch_batch_ep<MODE, kEps<MODE>[1]>(a, grid, st)
                               : launch_batch_ep<MODE, kEps<MODE>[2]>(a, grid, st);
}

template <int MODE>
int per_sm_ctas(int ep) {
  return ep == kEps<MODE>[0]   ? per_sm_ctas_ep<MODE, kEps<MODE>[0]>()
         : ep == kEps<MODE>[1] ? per_sm_ctas_ep<MODE, kEps<MODE>[1]>()
                               : per_sm_ctas_ep<MODE, kEps<MODE>[2]>();
}

}  // namespace
}  // namespace heat

using heat::BRing;

// What a captured batch run depends on (heat_batch's graph cache).
struct GraphKey {
  unsigned long long shape[6];
  heat::BatchArgs args;
};

struct heat_batch {
  struct Ring {
    bool live = false;
    int64_t off = 0, len = 0, n = 0, nx = 0;
    int32_t np = 0;
    double r = 0;
    float rf = 0;
    int64_t nt = 0, done = 0;
    int parity = 0;
  };
  heat_dtype dtype = HEAT_F64;
  size_t elem = 8;
  int device = 0, sms = 0;
  void *arena[2] = {nullptr, nullptr};
  int64_t capacity = 0;
  std::map<int64_t, int64_t> free_blocks;  // offset -> length (points)
  std::vector<Ring> rings;
  std::vector<int32_t> free_ids;
  cudaStream_t own_stream = nullptr, stream = nullptr;
  heat::DevStatus *dstat = nullptr, *hstat = nullptr;
  int host_error = HEAT_OK;
  // device work table: one blob [rings | segp | levp | active], plus done counters
  unsigned char *d_blob = nullptr;
  size_t blob_cap = 0;
  unsigned *d_done = nullptr;
  size_t done_cap = 0;
  unsigned long long *d_counter = nullptr;
  // pinned staging for the blob, reused once `staged` has completed
  unsigned char *h_stage = nullptr;
  size_t stage_cap = 0;
  cudaEvent_t staged = nullptr;
  bool staged_pending = false;
  int T = 0;
  int arith = HEAT_ARITH_EXACT;  // binary64 reading (the batch API is exact; the persistent form passes its own)
  int ctas_per_sm = 0;  // 0: as many as fit
  int64_t window = 0;  // warp window in points (32 x points per lane); 0: the dtype's widest
  int64_t last_point_steps = 0;
  long long wait_ns = 5000000000LL;
  int32_t inj_ring_id = -1;  // test hook (heat_batch_inject_stall)
  int graphs = 1;            // capture the run's stream operations and replay them while unchanged
  int emul_share = -1;       // binary64 tiles of 32 on the integer pipes (-1: the library's choice)
  cudaGraphExec_t graph_exec = nullptr;
  GraphKey graph_key = {};
  int64_t inj_seg = 0, inj_level = 0;
  // saved states (heat_batch_save / heat_batch_restore)
  void *snap = nullptr;
  std::vector<std::pair<int64_t, int>> snap_state;  // per ring id: (done, live)
};

namespace {

using heat::cuda_status;

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

int batch_sync_status(heat_batch *b) {
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return HEAT_ECUDA;
  if (cudaMemcpyAsync(b->hstat, b->dstat, sizeof(heat::DevStatus), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
    return HEAT_ECUDA;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return HEAT_ECUDA;
  if (b->hstat->code != HEAT_OK && b->host_error == HEAT_OK) b->host_error = b->hstat->code;
  return b->host_error;
}

// First-fit allocation of `len` points; -1 if no free block is large enough.
int64_t arena_alloc(heat_batch *b, int64_t len) {
  for (auto it = b->free_blocks.begin(); it != b->free_blocks.end(); ++it) {
    if (it->second >= len) {
      const int64_t off = it->first, rest = it->second - len;
      b->free_blocks.erase(it);
      if (rest > 0) b->free_blocks[off + len] = rest;
      return off;
    }
  }
  return -1;
}

void arena_free(heat_batch *b, int64_t off, int64_t len) {
  auto it = b->free_blocks.emplace(off, len).first;
  auto next = std::next(it);
  if (next != b->free_blocks.end() && it->first + it->second == next->first) {
    it->second += next->second;
    b->free_blocks.erase(next);
  }
  if (it != b->free_blocks.begin()) {
    auto prev = std::prev(it);
    if (prev->first + prev->second == it->first) {
      prev->second += it->second;
      b->free_blocks.erase(it);
    }
  }
}

int default_T(const heat_batch *b) { return b->dtype == HEAT_F32C ? 32 : 8; }

// Widest warp window of the batch kernel for the dtype (points).
int64_t widest_window(heat_dtype dtype) { return dtype == HEAT_F32C ? 1024 : 512; }

// The batch's warp window for depth T: its setting (default the widest),
// widened while a tile would hold fewer than 2T output points; 0 if even the
// widest cannot.
int64_t batch_window(const heat_batch *b, int T) {
  int64_t w = b->window > 0 ? b->window : widest_window(b->dtype);
  while (w - 2 * (int64_t)T < 2 * (int64_t)T && w < widest_window(b->dtype)) w *= 2;
  return w - 2 * (int64_t)T >= 2 * (int64_t)T ? w : 0;
}

// Tiles of a ring's units computed on the integer pipes (binary64, exact
// reading): the library's share for the ring's r unless
// heat_batch_set_emulation chose one.
unsigned batch_emul_mask(const heat_batch *b, double r) {
  if (b->dtype != HEAT_F64 || b->arith != HEAT_ARITH_EXACT) return 0u;
  return heat::emul_share_mask(b->emul_share < 0 ? heat::emul_auto_share(r) : b->emul_share);
}

struct Table {
  std::vector<BRing> rings;
  std::vector<int32_t> ids;  // ring id of each table entry
  std::vector<int64_t> segp, levp;
  std::vector<int32_t> active;
  int L = 0;
  int64_t window = 0;  // warp window (points) the tiles were cut for
  int64_t point_steps = 0;
};

// Work table for advancing each live ring by steps_of(ring) (> 0) steps.
template <typename F>
Table build_table(const heat_batch *b, int T, int64_t window, F steps_of) {
  const int64_t W = window - 2 * (int64_t)T;  // output points per warp tile
  Table t;
  t.window = window;
  std::vector<std::pair<int64_t, int32_t>> order;  // (levels, id)
  for (int32_t id = 0; id < (int32_t)b->rings.size(); ++id) {
    const auto &r = b->rings[id];
    if (!r.live) continue;
    const int64_t s = steps_of(r);
    if (s <= 0) continue;
    order.push_back({(s + T - 1) / T, id});
  }
  std::stable_sort(order.begin(), order.end(),
                   [](const std::pair<int64_t, int32_t> &x, const std::pair<int64_t, int32_t> &y) {
                     return x.first > y.first;
                   });
  t.segp.push_back(0);
  for (auto &o : order) {
    const auto &r = b->rings[o.second];
    BRing d;
    d.off = r.off;
    d.n = r.n;
    d.steps = steps_of(r);
    d.nseg = (r.n + W - 1) / W;
    d.done_base = t.segp.back();
    d.r = r.r;
    d.rf = r.rf;
    d.parity = r.parity;
    uint64_t rbits;
    memcpy(&rbits, &r.r, sizeof(rbits));
    const int rexp = (int)((rbits >> 52) & 2047);
    d.mx = heat::emul::prepare_mulx(rbits);
    d.emul_mask = batch_emul_mask(b, r.r);
    d.p2_hi_add = (rexp - 1023) * (1 << 20);
    d.p2_hi_xor = (rbits >> 63) ? (int)0x80000000u : 0;
    if (rexp < 1 || rexp > 2046 || !heat::emul::domain_bounds(rbits, T, d.dom_lo, d.dom_hi)) {
      d.dom_lo = 1;  // the integer routines take a normal, nonzero r: no integer tiles
      d.dom_hi = 0;
    }
    t.rings.push_back(d);
    t.ids.push_back(o.second);
    t.segp.push_back(t.segp.back() + d.nseg);
    t.point_steps += d.n * d.steps;
  }
  t.L = order.empty() ? 0 : (int)order.front().first;
  t.levp.push_back(0);
  size_t k = order.size();
  for (int lev = 0; lev < t.L; ++lev) {
    while (k > 0 && order[k - 1].first <= lev) --k;  // rings needing more than lev levels: order[0..k)
    t.active.push_back((int32_t)k);
    t.levp.push_back(t.levp.back() + t.segp[k]);
  }
  return t;
}

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Upload the table (one blob through pinned staging), zero the counters and
// queue the persistent launch.
int launch_table(heat_batch *b, const Table &t, int T) {
  if (t.rings.empty()) return HEAT_OK;
  const size_t nr = t.rings.size(), nl = (size_t)t.L;
  const size_t o_rings = 0, o_segp = align16(o_rings + nr * sizeof(BRing));
  const size_t o_levp = align16(o_segp + (nr + 1) * sizeof(int64_t));
  const size_t o_act = align16(o_levp + (nl + 1) * sizeof(int64_t));
  const size_t bytes = align16(o_act + nl * sizeof(int32_t));
  // staging: wait for the previous upload to finish before reusing
  if (b->staged_pending) {
    if (cudaEventSynchronize(b->staged) != cudaSuccess) return HEAT_ECUDA;
    b->staged_pending = false;
  }
  if (bytes > b->stage_cap) {
    if (b->h_stage) cudaFreeHost(b->h_stage);
    b->h_stage = nullptr;
    b->stage_cap = 0;
    if (cudaMallocHost((void **)&b->h_stage, bytes * 2) != cudaSuccess) return HEAT_ENOMEM;
    b->stage_cap = bytes * 2;
  }
  if (bytes > b->blob_cap) {
    if (b->d_blob) cudaFree(b->d_blob);
    b->d_blob = nullptr;
    b->blob_cap = 0;
    if (cudaMalloc((void **)&b->d_blob, bytes * 2) != cudaSuccess) return HEAT_ENOMEM;
    b->blob_cap = bytes * 2;
  }
  const size_t ndone = (size_t)t.segp.back();
  if (ndone > b->done_cap) {
    if (b->d_done) cudaFree(b->d_done);
    b->d_done = nullptr;
    b->done_cap = 0;
    if (cudaMalloc((void **)&b->d_done, ndone * 2 * sizeof(unsigned)) != cudaSuccess) return HEAT_ENOMEM;
    b->done_cap = ndone * 2;
  }
  memcpy(b->h_stage + o_rings, t.rings.data(), nr * sizeof(BRing));
  memcpy(b->h_stage + o_segp, t.segp.data(), (nr + 1) * sizeof(int64_t));
  memcpy(b->h_stage + o_levp, t.levp.data(), (nl + 1) * sizeof(int64_t));
  memcpy(b->h_stage + o_act, t.active.data(), nl * sizeof(int32_t));
  heat::BatchArgs a;
  memset(&a, 0, sizeof(a));  // padding too: the graph key hashes the bytes
  a.arena0 = b->arena[0];
  a.arena1 = b->arena[1];
  a.rings = (const BRing *)(b->d_blob + o_rings);
  a.segp = (const int64_t *)(b->d_blob + o_segp);
  a.levp = (const int64_t *)(b->d_blob + o_levp);
  a.active = (const int32_t *)(b->d_blob + o_act);
  a.L = t.L;
  a.T = T;
  a.dual = b->emul_share < 0;
  a.done = b->d_done;
  a.counter = b->d_counter;
  a.st = b->dstat;
  a.wait_ns = b->wait_ns;
  a.inj_ring = -1;
  a.inj_seg = 0;
  a.inj_level = 0;
  for (size_t i = 0; i < t.ids.size(); ++i)
    if (t.ids[i] == b->inj_ring_id) {
      a.inj_ring = (int)i;
      a.inj_seg = b->inj_seg;
      a.inj_level = b->inj_level;
    }
  const int64_t units = t.levp.back();
  const bool f32 = b->dtype == HEAT_F32C;
  const bool fma = !f32 && b->arith == HEAT_ARITH_FMA;
  const int ep = (int)(t.window / 32);
  int per_sm = f32 ? heat::per_sm_ctas<2>(ep) : fma ? heat::per_sm_ctas<1>(ep) : heat::per_sm_ctas<0>(ep);
  if (per_sm < 1) return HEAT_ECUDA;
  if (b->ctas_per_sm > 0 && b->ctas_per_sm < per_sm) per_sm = b->ctas_per_sm;
  const int resident = per_sm * b->sms;
  const int grid = (int)std::min<int64_t>(resident, (units + heat::kBWarps - 1) / heat::kBWarps);
  // The run is four stream operations: the table upload (from the pinned
  // staging buffer), two counter resets and the launch.  They are captured
  // into a CUDA graph and replayed while their shape -- byte counts, grid,
  // kernel arguments -- is unchanged (a fixed batch run again, e.g. after
  // heat_batch_restore); the upload node copies whatever the staging buffer
  // holds when the graph runs, so the table contents may differ.
  auto enqueue = [&](bool capturing) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(b->d_blob, b->h_stage, bytes, cudaMemcpyHostToDevice, b->stream);
    // the staging buffer may be refilled as soon as its copy is done; inside a
    // capture the record becomes an event-record node of the graph, so every
    // replay records `staged` too
    if (e == cudaSuccess)
      e = cudaEventRecordWithFlags(b->staged, b->stream, capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_done, 0, ndone * sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), b->stream);
    if (e == cudaSuccess)
      e = f32 ? heat::launch_batch<2>(a, ep, grid, b->stream)
              : fma ? heat::launch_batch<1>(a, ep, grid, b->stream) : heat::launch_batch<0>(a, ep, grid, b->stream);
    return e;
  };
  // the run's shape: operation sizes, grid, kernel, stream, staging buffer and
  // the kernel arguments byte for byte
  GraphKey key;
  memset(&key, 0, sizeof(key));
  key.shape[0] = bytes;
  key.shape[1] = ndone;
  key.shape[2] = (unsigned long long)grid;
  key.shape[3] = (unsigned long long)((f32 ? 2 : fma ? 1 : 0) * 256 + ep);
  key.shape[4] = (unsigned long long)(uintptr_t)b->stream;
  key.shape[5] = (unsigned long long)(uintptr_t)b->h_stage;
  memcpy(&key.args, &a, sizeof(a));
  cudaError_t e = cudaSuccess;
  if (b->graphs && b->graph_exec && memcmp(&key, &b->graph_key, sizeof(key)) == 0) {
    e = cudaGraphLaunch(b->graph_exec, b->stream);
  } else if (b->graphs) {
    if (b->graph_exec) {
      cudaGraphExecDestroy(b->graph_exec);
      b->graph_exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    bool captured = false;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const cudaError_t ee = enqueue(true);
      const cudaError_t ec = cudaStreamEndCapture(b->stream, &g);
      captured = ee == cudaSuccess && ec == cudaSuccess && g && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
    if (captured) {
      b->graph_exec = ex;
      memcpy(&b->graph_key, &key, sizeof(key));
      e = cudaGraphLaunch(ex, b->stream);
    } else {
      e = enqueue(false);  // not capturable here: plain stream operations
    }
  } else {
    e = enqueue(false);
  }
  if (e != cudaSuccess) return HEAT_ECUDA;
  b->staged_pending = true;
  return HEAT_OK;
}

void free_batch(heat_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int i = 0; i < 2; ++i)
    if (b->arena[i]) cudaFree(b->arena[i]);
  if (b->dstat) cudaFree(b->dstat);
  if (b->hstat) cudaFreeHost(b->hstat);
  if (b->d_blob) cudaFree(b->d_blob);
  if (b->d_done) cudaFree(b->d_done);
  if (b->d_counter) cudaFree(b->d_counter);
  if (b->h_stage) cudaFreeHost(b->h_stage);
  if (b->staged) cudaEventDestroy(b->staged);
  if (b->snap) cudaFree(b->snap);
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->own_stream) cudaStreamDestroy(b->own_stream);
  delete b;
}

bool ring_ok(const heat_batch *b, int32_t id) { return id >= 0 && id < (int32_t)b->rings.size() && b->rings[id].live; }

// Binary64 values (host or device) into the arena; binary32 state is rounded
// on the device.
int upload_ring(heat_batch *b, const heat_batch::Ring &r, const double *src_u, cudaMemcpyKind kind) {
  void *dst = (char *)b->arena[r.parity] + (size_t)r.off * b->elem;
  if (b->dtype == HEAT_F64)
    return cudaMemcpyAsync(dst, src_u, (size_t)r.n * 8, kind, b->stream) == cudaSuccess ? HEAT_OK : HEAT_ECUDA;
  if (kind == cudaMemcpyDeviceToDevice) {
    const int grid = (int)std::min<int64_t>((r.n + 255) / 256, (int64_t)b->sms * 8);
    heat::k_b_f64_to_f32<<<std::max(grid, 1), 256, 0, b->stream>>>(src_u, (float *)dst, r.n);
    return cudaGetLastError() == cudaSuccess ? HEAT_OK : HEAT_ECUDA;
  }
  const double *host_u = src_u;
  double *stage = nullptr;
  if (cudaMalloc((void **)&stage, (size_t)r.n * 8) != cudaSuccess) return HEAT_ENOMEM;
  int rc = HEAT_OK;
  if (cudaMemcpyAsync(stage, host_u, (size_t)r.n * 8, cudaMemcpyHostToDevice, b->stream) != cudaSuccess) rc = HEAT_ECUDA;
  if (rc == HEAT_OK) {
    const int grid = (int)std::min<int64_t>((r.n + 255) / 256, (int64_t)b->sms * 8);
    heat::k_b_f64_to_f32<<<std::max(grid, 1), 256, 0, b->stream>>>(stage, (float *)dst, r.n);
    if (cudaGetLastError() != cudaSuccess) rc = HEAT_ECUDA;
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) rc = HEAT_ECUDA;
  cudaFree(stage);
  return rc;
}

}  // namespace

extern "C" {

int heat_batch_create(heat_batch **out, int64_t capacity_points, heat_dtype dtype) {
  if (!out) return HEAT_EINVAL;
  *out = nullptr;
  if (capacity_points < 1 || (dtype != HEAT_F64 && dtype != HEAT_F32C)) return HEAT_EINVAL;
  heat_batch *b = new (std::nothrow) heat_batch();
  if (!b) return HEAT_ENOMEM;
  b->dtype = dtype;
  b->elem = dtype == HEAT_F64 ? 8 : 4;
  b->capacity = round_up(capacity_points, kAlignPointsHost);
  b->T = dtype == HEAT_F32C ? 32 : 8;
  int rc = HEAT_OK;
  if (cudaGetDevice(&b->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming) != cudaSuccess)
    rc = HEAT_ECUDA;
  b->stream = b->own_stream;
  for (int i = 0; i < 2 && rc == HEAT_OK; ++i)
    if (cudaMalloc(&b->arena[i], (size_t)b->capacity * b->elem) != cudaSuccess) rc = HEAT_ENOMEM;
  if (rc == HEAT_OK && cudaMalloc((void **)&b->dstat, sizeof(heat::DevStatus)) != cudaSuccess) rc = HEAT_ENOMEM;
  if (rc == HEAT_OK && cudaMallocHost((void **)&b->hstat, sizeof(heat::DevStatus)) != cudaSuccess) rc = HEAT_ENOMEM;
  if (rc == HEAT_OK && cudaMalloc((void **)&b->d_counter, sizeof(unsigned long long)) != cudaSuccess) rc = HEAT_ENOMEM;
  if (rc == HEAT_OK && cudaMemsetAsync(b->dstat, 0, sizeof(heat::DevStatus), b->stream) != cudaSuccess) rc = HEAT_ECUDA;
  if (rc == HEAT_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) rc = HEAT_ECUDA;
  if (rc != HEAT_OK) {
    cudaGetLastError();
    free_batch(b);
    return rc;
  }
  b->free_blocks[0] = b->capacity;
  *out = b;
  return HEAT_OK;
}

void heat_batch_destroy(heat_batch *b) { free_batch(b); }

static int batch_add(heat_batch *b, int64_t nx, int32_t np, double k, double dt, double dx, int64_t nt,
                     const double *src_u, cudaMemcpyKind kind, int32_t *ring_id) {
  if (!b || !src_u || !ring_id || nx < 1 || np < 1 || nt < 0) return HEAT_EINVAL;
  if (nx > INT64_MAX / np) return HEAT_EINVAL;
  if (!isfinite(k) || !isfinite(dt) || !isfinite(dx) || dx == 0.0) return HEAT_EINVAL;
  const double r = (k * dt) / (dx * dx);
  if (!isfinite(r)) return HEAT_EINVAL;
  heat_batch::Ring ring;
  ring.n = nx * (int64_t)np;
  ring.nx = nx;
  ring.np = np;
  ring.r = r;
  ring.rf = (float)r;
  ring.nt = nt;
  ring.len = round_up(ring.n, kAlignPointsHost);
  ring.off = arena_alloc(b, ring.len);
  if (ring.off < 0) return HEAT_ENOMEM;
  ring.live = true;
  int32_t id;
  if (!b->free_ids.empty()) {
    id = b->free_ids.back();
    b->free_ids.pop_back();
    b->rings[id] = ring;
  } else {
    id = (int32_t)b->rings.size();
    b->rings.push_back(ring);
  }
  int rc = upload_ring(b, b->rings[id], src_u, kind);
  if (rc == HEAT_OK && kind == cudaMemcpyHostToDevice && cudaStreamSynchronize(b->stream) != cudaSuccess)
    rc = HEAT_ECUDA;
  if (rc != HEAT_OK) {
    arena_free(b, ring.off, ring.len);
    b->rings[id].live = false;
    b->free_ids.push_back(id);
    return rc;
  }
  *ring_id = id;
  return HEAT_OK;
}

int heat_batch_add(heat_batch *b, int64_t nx, int32_t np, double k, double dt, double dx, int64_t nt,
                   const double *host_u, int32_t *ring_id) {
  return batch_add(b, nx, np, k, dt, dx, nt, host_u, cudaMemcpyHostToDevice, ring_id);
}

int heat_batch_add_device(heat_batch *b, int64_t nx, int32_t np, double k, double dt, double dx, int64_t nt,
                          const double *dev_u, int32_t *ring_id) {
  return batch_add(b, nx, np, k, dt, dx, nt, dev_u, cudaMemcpyDeviceToDevice, ring_id);
}

int heat_batch_run(heat_batch *b, int64_t max_steps) {
  if (!b) return HEAT_EINVAL;
  if (b->host_error != HEAT_OK) return HEAT_ESTATE;
  const int T = b->T > 0 ? b->T : default_T(b);
  const int64_t window = batch_window(b, T);
  if (window == 0) return HEAT_EINVAL;
  Table t = build_table(b, T, window, [&](const heat_batch::Ring &r) {
    const int64_t left = r.nt - r.done;
    return max_steps > 0 ? std::min(left, max_steps) : left;
  });
  b->last_point_steps = t.point_steps;
  const int rc = launch_table(b, t, T);
  if (rc != HEAT_OK) return rc;
  for (size_t i = 0; i < t.rings.size(); ++i) {
    auto &r = b->rings[t.ids[i]];
    const int64_t levels = (t.rings[i].steps + T - 1) / T;
    r.done += t.rings[i].steps;
    r.parity ^= (int)(levels & 1);
  }
  return HEAT_OK;
}

int heat_batch_sync(heat_batch *b) {
  if (!b) return HEAT_EINVAL;
  return batch_sync_status(b);
}

int heat_batch_query(const heat_batch *b, int32_t ring_id, int64_t *steps_done, int64_t *steps_left) {
  if (!b || !ring_ok(b, ring_id)) return HEAT_EINVAL;
  const auto &r = b->rings[ring_id];
  if (steps_done) *steps_done = r.done;
  if (steps_left) *steps_left = r.nt - r.done;
  return HEAT_OK;
}

int heat_batch_get(heat_batch *b, int32_t ring_id, double *host_u, int64_t n) {
  if (!b || !host_u || !ring_ok(b, ring_id)) return HEAT_EINVAL;
  const auto &r = b->rings[ring_id];
  if (n != r.n) return HEAT_EINVAL;
  int rc = batch_sync_status(b);
  if (rc != HEAT_OK) return rc;
  const void *src = (const char *)b->arena[r.parity] + (size_t)r.off * b->elem;
  if (b->dtype == HEAT_F64) {
    if (cudaMemcpyAsync(host_u, src, (size_t)n * 8, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
      return HEAT_ECUDA;
  } else {
    double *stage = nullptr;
    if (cudaMalloc((void **)&stage, (size_t)n * 8) != cudaSuccess) return HEAT_ENOMEM;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)b->sms * 8);
    heat::k_b_f32_to_f64<<<std::max(grid, 1), 256, 0, b->stream>>>((const float *)src, stage, n);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(host_u, stage, (size_t)n * 8, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
      rc = HEAT_ECUDA;
    cudaStreamSynchronize(b->stream);
    cudaFree(stage);
    if (rc != HEAT_OK) return rc;
  }
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? HEAT_OK : HEAT_ECUDA;
}

int heat_batch_get_device(heat_batch *b, int32_t ring_id, double *dev_u, int64_t n) {
  if (!b || !dev_u || !ring_ok(b, ring_id)) return HEAT_EINVAL;
  const auto &r = b->rings[ring_id];
  if (n != r.n) return HEAT_EINVAL;
  if (b->host_error != HEAT_OK) return b->host_error;
  const void *src = (const char *)b->arena[r.parity] + (size_t)r.off * b->elem;
  if (b->dtype == HEAT_F64)
    return cudaMemcpyAsync(dev_u, src, (size_t)n * 8, cudaMemcpyDeviceToDevice, b->stream) == cudaSuccess ? HEAT_OK
                                                                                                       : HEAT_ECUDA;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)b->sms * 8);
  heat::k_b_f32_to_f64<<<std::max(grid, 1), 256, 0, b->stream>>>((const float *)src, dev_u, n);
  return cudaGetLastError() == cudaSuccess ? HEAT_OK : HEAT_ECUDA;
}

int heat_batch_remove(heat_batch *b, int32_t ring_id) {
  if (!b || !ring_ok(b, ring_id)) return HEAT_EINVAL;
  // no wait: work queued before this call may still touch the ring's space,
  // but every later use of that space (an admitted ring's copy, a run, a
  // restore) is queued on the same stream behind it
  auto &r = b->rings[ring_id];
  arena_free(b, r.off, r.len);
  r.live = false;
  b->free_ids.push_back(ring_id);
  return HEAT_OK;
}

int heat_batch_set_tuning(heat_batch *b, int T, int64_t window_points) {
  if (!b || T < 0 || T > heat::kMaxT || window_points < 0) return HEAT_EINVAL;
  if (window_points > 0) {
    // the widest window of the kernel's three not above the request, at least the narrowest
    const int64_t widest = widest_window(b->dtype);
    int64_t w = widest / 4;
    while (w * 2 <= window_points && w < widest) w *= 2;
    b->window = w;
  }
  if (T > 0) b->T = T;
  return HEAT_OK;
}

int heat_batch_set_emulation(heat_batch *b, int share) {
  if (!b || share < -1 || share > 32) return HEAT_EINVAL;
  b->emul_share = share;
  return HEAT_OK;
}

int heat_batch_set_graphs(heat_batch *b, int enable) {
  if (!b) return HEAT_EINVAL;
  b->graphs = enable ? 1 : 0;
  return HEAT_OK;
}

int heat_batch_set_wait_limit(heat_batch *b, int64_t ns) {
  if (!b || ns < 1) return HEAT_EINVAL;
  b->wait_ns = ns;
  return HEAT_OK;
}

int heat_batch_inject_stall(heat_batch *b, int32_t ring_id, int64_t segment, int64_t from_level) {
  if (!b || from_level < 0 || segment < 0) return HEAT_EINVAL;
  b->inj_ring_id = ring_id;  // a ring id that is not live disables the hook
  b->inj_seg = segment;
  b->inj_level = from_level;
  return HEAT_OK;
}

int heat_batch_set_ctas_per_sm(heat_batch *b, int ctas_per_sm) {
  if (!b || ctas_per_sm < 0) return HEAT_EINVAL;
  b->ctas_per_sm = ctas_per_sm;
  return HEAT_OK;
}

int heat_batch_set_stream(heat_batch *b, void *cuda_stream) {
  if (!b) return HEAT_EINVAL;
  cudaStream_t next = cuda_stream ? (cudaStream_t)cuda_stream : b->own_stream;
  if (next == b->stream) return HEAT_OK;
  cudaEvent_t ev;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return HEAT_ECUDA;
  int rc = HEAT_OK;
  if (cudaEventRecord(ev, b->stream) != cudaSuccess || cudaStreamWaitEvent(next, ev, 0) != cudaSuccess) rc = HEAT_ECUDA;
  cudaEventDestroy(ev);
  if (rc == HEAT_OK) b->stream = next;
  return rc;
}

int heat_batch_info(const heat_batch *b, int32_t *live_rings, int64_t *largest_free_points,
                    int64_t *last_point_steps) {
  if (!b) return HEAT_EINVAL;
  if (live_rings) {
    int32_t c = 0;
    for (const auto &r : b->rings) c += r.live ? 1 : 0;
    *live_rings = c;
  }
  if (largest_free_points) {
    int64_t m = 0;
    for (const auto &f : b->free_blocks) m = std::max(m, f.second);
    *largest_free_points = m;
  }
  if (last_point_steps) *last_point_steps = b->last_point_steps;
  return HEAT_OK;
}

int heat_batch_save(heat_batch *b) {
  if (!b) return HEAT_EINVAL;
  int rc = batch_sync_status(b);
  if (rc != HEAT_OK) return rc;
  if (!b->snap && cudaMalloc(&b->snap, (size_t)b->capacity * b->elem) != cudaSuccess) return HEAT_ENOMEM;
  b->snap_state.assign(b->rings.size(), {0, 0});
  for (size_t id = 0; id < b->rings.size(); ++id) {
    const auto &r = b->rings[id];
    if (!r.live) continue;
    const size_t o = (size_t)r.off * b->elem;
    if (cudaMemcpyAsync((char *)b->snap + o, (const char *)b->arena[r.parity] + o, (size_t)r.n * b->elem,
                        cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
      return HEAT_ECUDA;
    b->snap_state[id] = {r.done, 1};
  }
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? HEAT_OK : HEAT_ECUDA;
}

int heat_batch_restore(heat_batch *b) {
  if (!b || !b->snap) return HEAT_ESTATE;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return HEAT_ECUDA;
  for (size_t id = 0; id < b->rings.size() && id < b->snap_state.size(); ++id) {
    auto &r = b->rings[id];
    if (!r.live || !b->snap_state[id].second) continue;
    const size_t o = (size_t)r.off * b->elem;
    if (cudaMemcpyAsync((char *)b->arena[0] + o, (const char *)b->snap + o, (size_t)r.n * b->elem,
                        cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
      return HEAT_ECUDA;
    r.parity = 0;
    r.done = b->snap_state[id].first;
  }
  b->host_error = HEAT_OK;
  if (cudaMemsetAsync(b->dstat, 0, sizeof(heat::DevStatus), b->stream) != cudaSuccess) return HEAT_ECUDA;
  return HEAT_OK;
}

int heat_batch_autotune(heat_batch *b, int *T_out, int64_t *seg_out) {
  if (!b) return HEAT_EINVAL;
  int rc = batch_sync_status(b);
  if (rc != HEAT_OK) return rc;
  // coarse description of the batch for the cache key
  int64_t pts = 0, steps = 0;
  int32_t live = 0;
  for (const auto &r : b->rings)
    if (r.live && r.nt > r.done) {
      ++live;
      pts += r.n;
      steps += r.nt - r.done;
    }
  if (live == 0) return HEAT_ESTATE;
  char key[160];
  snprintf(key, sizeof(key), "batch dtype=%d rings_log2=%d points_log2=%d mean_n_log2=%d", (int)b->dtype,
           (int)log2((double)live), (int)log2((double)pts), (int)log2((double)pts / live));
  const char *cache = getenv("HEAT_TUNE_CACHE");
  if (cache) {
    FILE *f = fopen(cache, "r");
    if (f) {
      char line[256];
      while (fgets(line, sizeof(line), f)) {
        int T;
        long long sg;
        char k2[160];
        // format: <key> | <T> <seg>
        const char *bar = strchr(line, '|');
        if (!bar) continue;
        size_t kl = (size_t)(bar - line);
        if (kl >= sizeof(k2)) continue;
        memcpy(k2, line, kl);
        while (kl > 0 && k2[kl - 1] == ' ') --kl;
        k2[kl] = 0;
        if (strcmp(k2, key) == 0 && sscanf(bar + 1, "%d %lld", &T, &sg) == 2) {
          fclose(f);
          b->T = T;
          b->window = sg;
          if (T_out) *T_out = T;
          if (seg_out) *seg_out = sg;
          return HEAT_OK;
        }
      }
      fclose(f);
    }
  }
  const int Ts64[] = {4, 8, 12, 16};
  const int Ts32[] = {16, 32, 64};
  const int *Ts = b->dtype == HEAT_F32C ? Ts32 : Ts64;
  const int nT = b->dtype == HEAT_F32C ? 3 : 4;
  const int64_t widest = widest_window(b->dtype);
  const int64_t wins[] = {widest / 4, widest / 2, widest};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HEAT_ECUDA;
  double best = -1;
  int bestT = b->T;
  int64_t bestSeg = b->window;
  for (int ti = 0; ti < nT && rc == HEAT_OK; ++ti) {
    for (int64_t sg : wins) {
      const int T = Ts[ti];
      if (sg - 2 * T < 2 * T) continue;  // a tile must keep 2T output points
      // one level per ring: reads each ring's current buffer, writes only the idle one
      Table t = build_table(b, T, sg, [&](const heat_batch::Ring &r) { return std::min<int64_t>(r.nt - r.done, T); });
      for (int rep = 0; rep < 2 && rc == HEAT_OK; ++rep) {
        cudaEventRecord(e0, b->stream);
        rc = launch_table(b, t, T);
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = HEAT_ECUDA;
      }
      if (rc != HEAT_OK) break;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      const double rate = (double)t.point_steps / (ms * 1e-3);
      if (rate > best) {
        best = rate;
        bestT = T;
        bestSeg = sg;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == HEAT_OK) rc = batch_sync_status(b);
  if (rc != HEAT_OK) return rc;
  b->T = bestT;
  b->window = bestSeg;
  if (cache) {
    FILE *f = fopen(cache, "a");
    if (f) {
      fprintf(f, "%s | %d %lld\n", key, bestT, (long long)bestSeg);
      fclose(f);
    }
  }
  if (T_out) *T_out = bestT;
  if (seg_out) *seg_out = bestSeg;
  return HEAT_OK;
}

}  // extern "C"

namespace heat {

// HEAT_FORM_PERSIST_TB for a single ring: one launch advances all nt steps
// (k_wave.cu).
int run_persist_tb(heat_ctx *c, int64_t nt) { return run_wave(c, nt, c->T > 0 ? c->T : wave_default_T(c)); }

}  // namespace heat

// k_batch.cu -- batched independent rings (the paper's Section 2 problem, many
// instances at once) in one device arena, advanced by one persistent launch
// driven by a work table.
//
// Work table (built on the host for each run, rings sorted by the number of
// T-step levels they need, longest first):
//   ring i: arena offset, n points, steps this run, nseg segments, r;
//   units (level b, ring i, segment j) are numbered level-major, so the rings
//   active at level b are a prefix of the sorted list and a unit number decodes
//   with two binary searches (over the per-level and per-ring prefix sums).
// A CTA claims the next unit from a launch-wide counter.  Unit (b, i, j) reads
// the ring's state at time bT from one arena buffer and writes time
// bT + steps_b into the other; before that it waits (bounded) until segments
// j-1, j, j+1 of ring i have finished level b-1.  Units are numbered level-major
// and claimed in increasing order, so every unit a CTA waits for has a smaller
// number and was claimed earlier by a CTA that is running it; the CTA holding
// the smallest unfinished unit therefore never waits on anything unfinished,
// and the launch makes progress with any number of resident CTAs.  No
// co-residency is needed: the kernel is an ordinary launch, and two batches
// (binary64 and binary32) can share the GPU.  The same wait covers the
// write-after-read hazard on the output buffer, which level b-1's neighbours
// read.
//
// Within a unit the CTA's warps cover the segment with register-resident
// temporal-blocking windows (tb_core.cuh); windows wrap around the ring's ends
// with modular indices.  Every point is computed from the same operands as in
// the single-ring forms, so each ring's result is bitwise its solo result.
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

#include "tb_core.cuh"

static constexpr int64_t kAlignPointsHost = 64;  // ring placement granularity in the arena (points)

namespace heat {
namespace {

constexpr int kBWarps = 4;
constexpr long long kMaxSpins = 1LL << 26;

struct BRing {
  int64_t off;        // arena offset in points
  int64_t n;          // ring length
  int64_t steps;      // steps this run
  int64_t nseg;       // segments
  int64_t done_base;  // index of segment 0's done counter
  double r;
  float rf;
  int parity;         // arena buffer holding the state at the start of the run
  emul::MulX mx;      // r for the integer-pipe tiles (binary64, exact reading)
  int dom_lo, dom_hi; // their input screen for T steps (empty: dom_lo > dom_hi)
  unsigned emul_mask; // bit (tile mod 32) set: that tile of a unit on the integer pipes
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
  int dual;  // binary64 under the library's share: two-ended tile claiming within units
  unsigned *done;
  unsigned long long *counter;
  DevStatus *st;
  long long wait_ns;
  int inj_ring;        // test hook: table index of a ring whose segment stops publishing (-1: none)
  long long inj_seg;
  long long inj_level;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait until *p >= target; false (and the device status set) if it ran out.
__device__ bool wait_done(const BatchArgs &a, const unsigned *p, unsigned target, int ring, long long level) {
  if (ld_acquire_u32(p) >= target) return true;
  const unsigned long long deadline = now_ns() + (unsigned long long)a.wait_ns;
  unsigned ns = 32;
  for (long long spin = 0; spin < kMaxSpins; ++spin) {
    if (ld_acquire_u32(p) >= target) return true;
    if (*(volatile int *)&a.st->abort) return false;
    if (now_ns() > deadline) break;
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
  }
  if (atomicCAS(&a.st->code, HEAT_OK, HEAT_ETIMEOUT) == HEAT_OK) {
    a.st->segment = ring;
    a.st->step = level;
  }
  atomicExch(&a.st->abort, 1);
  return false;
}

// Largest index k in [lo, hi) with v[k] <= x (v nondecreasing, v[lo] <= x).
__device__ __forceinline__ int64_t floor_index(const int64_t *v, int64_t lo, int64_t hi, int64_t x) {
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (v[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

template <int MODE>
__global__ void __launch_bounds__(kBWarps * 32, MODE == 2 ? 3 : 6) k_batch(BatchArgs a) {  // MODE: 0 exact, 1 fused, 2 binary32
  using P = tb::TBC<MODE>;  // contiguous per-lane ownership
  using T = typename P::T;
  constexpr int E = P::E;
  constexpr int WIN = 32 * E;
  __shared__ long long s_ring, s_level, s_lo, s_hi, s_steps, s_seg;
  __shared__ int s_stop;
  __shared__ unsigned long long s_tile;  // the unit's tiles are claimed by the CTA's warps (see below)
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int64_t total = a.levp[a.L];
  const int W = WIN - 2 * a.T;

  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned long long u = atomicAdd(a.counter, 1ull);
      int stop = 0;
      if ((int64_t)u >= total) {
        stop = 1;
      } else {
        const int64_t b = floor_index(a.levp, 0, a.L, (int64_t)u);
        const int64_t rel = (int64_t)u - a.levp[b];
        const int64_t i = floor_index(a.segp, 0, a.active[b], rel);
        const int64_t j = rel - a.segp[i];
        const BRing R = a.rings[i];
        if (b > 0) {
          const int64_t jm = j == 0 ? R.nseg - 1 : j - 1, jp = j + 1 == R.nseg ? 0 : j + 1;
          const unsigned tgt = (unsigned)b;
          if (!(wait_done(a, a.done + R.done_base + jm, tgt, (int)i, b) &&
                wait_done(a, a.done + R.done_base + j, tgt, (int)i, b) &&
                wait_done(a, a.done + R.done_base + jp, tgt, (int)i, b)))
            stop = 2;
        }
        s_ring = i;
        s_level = b;
        s_seg = j;
        s_lo = (j * R.n) / R.nseg;
        s_hi = ((j + 1) * R.n) / R.nseg;
        const int64_t left = R.steps - b * a.T;
        s_steps = left < a.T ? left : a.T;
      }
      s_stop = stop;
      s_tile = 0;
    }
    __syncthreads();
    if (s_stop) break;  // uniform across the CTA
    const BRing R = a.rings[s_ring];
    const int par = R.parity ^ (int)(s_level & 1);
    const T *src = (const T *)(par ? a.arena1 : a.arena0) + R.off;
    T *dst = (T *)(par ? a.arena0 : a.arena1) + R.off;
    const int64_t lo = s_lo, hi = s_hi, n = R.n;
    const int steps = (int)s_steps;
    const int64_t ntile = (hi - lo + W - 1) / W;
    // Binary64 rings under the library's share: two-ended claiming within the
    // unit (integer-pipe warps from the end, FP64-unit warps from the start,
    // one 64-bit shared counter), so the split follows the engines' speeds.
    // Otherwise tiles in order, R.emul_mask choosing their engine.
    const bool dual = MODE == 0 && a.dual && R.emul_mask != 0u;
    const bool int_warp = dual && (((blockIdx.x ^ wib) & 1) != 0);
    for (;;) {
      unsigned long long tc = 0;
      if (lane == 0) tc = atomicAdd(&s_tile, int_warp ? (1ull << 32) : 1ull);
      tc = __shfl_sync(0xffffffffu, tc, 0);
      int64_t t;
      bool int_tile;
      if (dual) {
        const int64_t f = (int64_t)(tc & 0xffffffffull), b = (int64_t)(tc >> 32);
        if (f + b >= ntile) break;
        t = int_warp ? ntile - 1 - b : f;
        int_tile = int_warp;
      } else {
        t = (int64_t)tc;
        if (t >= ntile) break;
        int_tile = MODE == 0 && ((R.emul_mask >> (unsigned)(t & 31)) & 1u);
      }
      const int64_t ws = lo + t * W - a.T;
      typename P::Reg reg;
      const bool inside = ws >= 0 && ws + WIN <= n;
#pragma unroll
      for (int k = 0; k < E; ++k) {
        int64_t g = ws + E * lane + k;
        if (!inside) {
          g %= n;
          if (g < 0) g += n;
        }
        P::load(reg, k, __ldcg(src + g));
      }
      bool dp = true;
      if constexpr (MODE == 0) {
        if (int_tile || R.mx.pow2) {
          bool ok = true;
#pragma unroll
          for (int k = 0; k < E; ++k)
            ok &= emul::in_domain((uint64_t)__double_as_longlong(P::store(reg, k)), R.dom_lo, R.dom_hi);
          if (__all_sync(0xffffffffu, ok)) {
            if (!int_tile)  // r = +-2^k on the FP64 unit: the product moves the exponent
              for (int s = 0; s < steps; ++s) P::step_p2(reg, R.p2_hi_add, R.p2_hi_xor);
            else if (R.mx.pow2 && !R.mx.neg)
              P::template steps_x<true, false>(reg, steps, R.mx);
            else if (R.mx.pow2)
              P::template steps_x<true, true>(reg, steps, R.mx);
            else if (!R.mx.neg)
              P::template steps_x<false, false>(reg, steps, R.mx);
            else
              P::template steps_x<false, true>(reg, steps, R.mx);
            dp = false;
          }
        }
      }
      if (dp)
        for (int s = 0; s < steps; ++s) P::step(reg, lane, R.r, R.rf);
      const int64_t out_hi = lo + (t + 1) * W < hi ? lo + (t + 1) * W : hi;
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const int i = E * lane + k;
        const int64_t g = ws + i;
        if (i >= a.T && i < WIN - a.T && g < out_hi) dst[g] = P::store(reg, k);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && !(s_ring == a.inj_ring && s_seg == a.inj_seg && s_level >= a.inj_level)) {
      __threadfence();
      st_release_u32(a.done + R.done_base + s_seg, (unsigned)(s_level + 1));
    }
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

template <int MODE>
cudaError_t launch_batch(BatchArgs &a, int grid, cudaStream_t st) {
  k_batch<MODE><<<grid, kBWarps * 32, 0, st>>>(a);
  return cudaGetLastError();
}

template <int MODE>
int per_sm_ctas() {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<MODE>, kBWarps * 32, 0) != cudaSuccess) return 0;
  return per_sm;
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
  int64_t seg_points = 16384;
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
  int64_t point_steps = 0;
};

// Work table for advancing each live ring by steps_of(ring) (> 0) steps.
template <typename F>
Table build_table(const heat_batch *b, int T, int64_t seg_points, F steps_of) {
  Table t;
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
    d.nseg = std::max<int64_t>(1, r.n / seg_points);
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
  int per_sm = f32 ? heat::per_sm_ctas<2>() : fma ? heat::per_sm_ctas<1>() : heat::per_sm_ctas<0>();
  if (per_sm < 1) return HEAT_ECUDA;
  if (b->ctas_per_sm > 0 && b->ctas_per_sm < per_sm) per_sm = b->ctas_per_sm;
  const int resident = per_sm * b->sms;
  const int grid = (int)std::min<int64_t>(resident, units);
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
      e = f32 ? heat::launch_batch<2>(a, grid, b->stream)
              : fma ? heat::launch_batch<1>(a, grid, b->stream) : heat::launch_batch<0>(a, grid, b->stream);
    return e;
  };
  // the run's shape: operation sizes, grid, kernel, stream, staging buffer and
  // the kernel arguments byte for byte
  GraphKey key;
  memset(&key, 0, sizeof(key));
  key.shape[0] = bytes;
  key.shape[1] = ndone;
  key.shape[2] = (unsigned long long)grid;
  key.shape[3] = (unsigned long long)(f32 ? 2 : fma ? 1 : 0);
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
  Table t = build_table(b, T, b->seg_points, [&](const heat_batch::Ring &r) {
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

int heat_batch_set_tuning(heat_batch *b, int T, int64_t seg_points) {
  if (!b || T < 0 || T > heat::kMaxT || seg_points < 0 || (seg_points > 0 && seg_points < 512)) return HEAT_EINVAL;
  const int win = b->dtype == HEAT_F32C ? 32 * heat::tb::TBC<2>::E : 32 * heat::tb::TBC<0>::E;
  if (T > 0 && 2 * T >= win) return HEAT_EINVAL;
  if (T > 0) b->T = T;
  if (seg_points > 0) b->seg_points = seg_points;
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
          b->seg_points = sg;
          if (T_out) *T_out = T;
          if (seg_out) *seg_out = sg;
          return HEAT_OK;
        }
      }
      fclose(f);
    }
  }
  const int Ts64[] = {2, 4, 8, 16};
  const int Ts32[] = {16, 32, 64};
  const int64_t segs[] = {4096, 16384, 65536};
  const int *Ts = b->dtype == HEAT_F32C ? Ts32 : Ts64;
  const int nT = b->dtype == HEAT_F32C ? 3 : 4;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HEAT_ECUDA;
  double best = -1;
  int bestT = b->T;
  int64_t bestSeg = b->seg_points;
  for (int ti = 0; ti < nT && rc == HEAT_OK; ++ti) {
    for (int64_t sg : segs) {
      const int T = Ts[ti];
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
  b->seg_points = bestSeg;
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

// HEAT_FORM_PERSIST_TB for a single ring: one launch advances all nt steps.
// Rings of at least three warp windows take the warp-granular dependency
// kernel (k_wave.cu); shorter rings the work-table kernel over one ring whose
// two buffers are the context's own, segments sized so that the levels keep
// every CTA busy.
int run_persist_tb(heat_ctx *c, int64_t nt) {
  {
    const int T = c->T > 0 ? c->T : (c->dtype == HEAT_F32C ? 32 : 12);
    const int rc = run_wave(c, nt, T);
    if (rc != HEAT_ENOTSUP) return rc;
  }
  if (!c->ptb) {
    heat_batch *b = new (std::nothrow) heat_batch();
    if (!b) return HEAT_ENOMEM;
    b->dtype = c->dtype;
    b->elem = c->elem;
    b->device = c->device;
    b->sms = c->sms;
    b->dstat = c->dstat;  // shared with the context: its errors surface at heat_sync
    if (cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc((void **)&b->d_counter, sizeof(unsigned long long)) != cudaSuccess) {
      if (b->staged) cudaEventDestroy(b->staged);
      delete b;
      return HEAT_ENOMEM;
    }
    c->ptb = b;
  }
  heat_batch *b = c->ptb;
  b->stream = c->stream;
  b->arith = c->arith;
  b->arena[0] = c->buf[0];
  b->arena[1] = c->buf[1];
  b->wait_ns = c->wait_ns;
  b->emul_share = c->emul_auto ? -1 : c->emul_share;  // heat_set_emulation applies here too
  // default depth: 32 for binary32; 12 for binary64, the depth at which the
  // integer tiles' screen still admits ordinary data for a general r
  const int T = c->T > 0 ? c->T : (c->dtype == HEAT_F32C ? 32 : 12);
  const int win = c->dtype == HEAT_F32C ? 32 * tb::TBC<2>::E : 32 * tb::TBC<0>::E;
  if (2 * T >= win) return HEAT_EINVAL;
  heat_batch::Ring r;
  r.live = true;
  r.off = 0;
  r.n = c->geo.N;
  r.len = c->geo.N;
  r.r = c->r;
  r.rf = c->rf;
  r.nt = nt;
  r.parity = c->cur;
  b->rings.assign(1, r);
  // about three segments per resident CTA, each at least 512 points
  const int64_t per_sm = c->dtype == HEAT_F32C ? 3 : 5;
  int64_t seg = c->geo.N / (3 * per_sm * c->sms);
  if (seg < 512) seg = 512;
  Table t = build_table(b, T, seg, [&](const heat_batch::Ring &rr) { return rr.nt; });
  const int rc = launch_table(b, t, T);
  if (rc != HEAT_OK) return rc;
  const int64_t levels = (nt + T - 1) / T;
  if (levels & 1) c->cur ^= 1;
  c->steps += nt;
  c->last_T = T;
  c->last_launches = 1;
  c->last_segments = (int)t.rings[0].nseg;
  return HEAT_OK;
}

void free_persist_tb(heat_ctx *c) {
  heat_batch *b = c->ptb;
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->d_blob) cudaFree(b->d_blob);
  if (b->d_done) cudaFree(b->d_done);
  if (b->d_counter) cudaFree(b->d_counter);
  if (b->h_stage) cudaFreeHost(b->h_stage);
  if (b->staged) cudaEventDestroy(b->staged);
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  delete b;
  c->ptb = nullptr;
}

}  // namespace heat

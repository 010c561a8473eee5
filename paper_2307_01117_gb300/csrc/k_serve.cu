// k_serve.cu -- the request server (heat_server_*): continuous batching inside
// one running kernel.
//
// Requests are independent rings (Section 2's problem, each with its own size,
// coefficient and step count).  Each admitted request occupies a slot: its
// state in the arena (two buffers), a range of per-tile completion counters,
// a descriptor and a claim counter.  The server kernel is persistent: its warps
// repeatedly look for an admitted request with an unclaimed unit (level b, warp
// tile j) -- each warp scanning the slots from its own, moving start, so the
// warps spread over the requests -- claim it, wait (bounded) until tiles j-1, j,
// j+1 of the request finished level b-1, advance the tile by T steps with the
// register-resident core (wave_core.cuh) and publish the tile's counter.  The
// warp that finishes a request's last unit writes the request's generation into
// a host-mapped completion word, which the host polls.
//
// Admission while the kernel runs: a small publish kernel on the server's copy
// stream (after the request's initial state has been copied into the arena)
// clears the request's tile counters and writes its descriptor, then -- after a
// fence -- its generation-tagged unit limit, its generation-tagged claim
// counter (release) and its bit in the live-slot bitmap.  The server kernel's
// CTAs per SM are capped below the maximum, so the publish kernel finds room
// beside it.
//
// Claims: a slot's claim counter holds (generation << 40 | next unit) and its
// limit (generation << 40 | units).  A warp claims by fetch-and-add on the
// counter and holds the unit only when the value it got and the limit carry
// the same generation and the unit number is below the limit: a unit is never
// handed out twice or skipped, and a slot released and published again never
// hands out a unit of its old request (a fetch-and-add that lands in the new
// generation holds a unit of the new request, whose descriptor was written
// before its counter).
// Units of a request are claimed in increasing (level-major) order and a warp
// holds one unit at a time, so a unit waits only on units claimed earlier by
// warps that are running them: the kernel makes progress with any number of
// resident CTAs.  A warp claims from a request only while the request's next
// unit is less than a set number of quarter levels past its finished units,
// so claimed units mostly find their neighbours done instead of waiting on
// units claimed just before them.  Binary64 (units of 512 points x T steps):
// 3/4 of a level, one unit per claim (saturated, 96 requests, 4 CTAs per SM:
// 212 GLUP/s; one level 197; two levels with four units per claim 167).
// Binary32 (short units, where the claim itself weighs more): two levels,
// four units per claim (1164 GLUP/s at 2 CTAs per SM; 3/4 of a level with
// one unit per claim 720).
//
// The kernel ends when the host raises the host-mapped stop word, when a
// bounded wait runs out (HEAT_ETIMEOUT, every warp returns), or when a warp has
// found no request with units left to claim for idle_ns: that warp raises the
// launch's exit word and every warp leaves before its next claim, so the
// kernel never runs on with part of its warps (warps that left one by one
// left the rest to serve later arrivals: a 10 s window at 200 requests/s then
// ran at 55-100 GLUP/s); the host launches it again when a request is
// submitted, or polled, while it is not running.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "wave_core.cuh"

namespace heat {
namespace {

constexpr int kSWarps = 4;
// quarter levels a claim may run ahead of a request's finished units, and
// consecutive units per claim, by arithmetic reading
template <int MODE>
struct ClaimRule {
  static constexpr int ahead_q = MODE == 2 ? 8 : 3;
  static constexpr int chunk = MODE == 2 ? 4 : 1;
};
constexpr unsigned long long kUnitMask = (1ull << 40) - 1;

struct SReq {
  int64_t off;        // arena offset (points)
  int64_t n;          // ring length
  int64_t nseg;       // warp tiles
  int64_t units;      // levels * nseg
  int64_t nt;
  int64_t done_base;  // first tile counter
  double r;
  float rf;
  unsigned gen;       // generation of the slot's request (0: empty)
  emul::MulX mx;
  int dom_lo, dom_hi;
  int p2_hi_add, p2_hi_xor;
  int int_ok;         // binary64 exact reading with a usable screen: integer tiles allowed
};

static_assert(sizeof(SReq) % 8 == 0, "descriptors are read in 8-byte words");

struct __align__(64) SCtl {
  unsigned long long claim;  // generation << 40 | next unit
  unsigned long long lim;    // generation << 40 | units (written before claim)
  unsigned long long fin;    // finished units
  unsigned long long pad[5];
};

// A launch's exit word (device memory, zeroed before each launch; written at
// most once per launch, read before every claim).
struct __align__(128) SIdle {
  int exiting;
};

struct ServeArgs {
  void *arena0, *arena1;
  SReq *req;
  SCtl *ctl;
  const unsigned *live;      // bitmap of published slots (host-maintained through publish kernels)
  int nwords;                // live bitmap words
  unsigned *done;            // tile counter pool
  volatile int *complete;    // host-mapped: generation of each slot's completed request
  const volatile int *stop;  // host-mapped stop word
  const volatile int *oldest;  // host-mapped: the oldest request's slot (admission order)
  DevStatus *st;
  SIdle *idle;
  long long wait_ns, idle_ns;
  int T;
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long atom_add_acq_rel(unsigned long long *p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}

// Find and claim a unit.  The warp gathers published slots from the live
// bitmap in circular order from slot `start` (each warp starts elsewhere and
// moves on every claim, so warps spread over the admitted requests: a short
// request is not held behind a long one), 32 slots per round whatever the word
// boundaries (lane l takes the round's l-th slot, placed by a warp prefix sum
// over the words' bit counts).  A slot is a candidate when its claim
// counter and its limit carry the same generation (a publication in progress
// shows two), units remain, and the next unit is less than ahead_q quarter
// levels past the finished ones.  The first candidate's lane claims by fetch-and-add on the
// counter (acquire: the descriptor and limit of the generation it lands in were
// written before that generation's counter); the claim holds a unit when the
// returned value's generation matches the limit's and its unit number is below
// the limit -- whatever generation that is, since a counter only counts its
// own request's units.  A claim takes `chunk` consecutive units (those below
// the limit).  Returns the slot, the first unit through *unit and their number
// through *count, -2 for a claim past the slot's last unit (it holds nothing),
// -3 when no slot is a candidate but some slot has units left (held back by
// the lookahead), -1 when no slot has units left; every lane returns the same
// values.
__device__ int claim_unit(const ServeArgs &a, int lane, int start, int ahead_q, int chunk, int64_t *unit,
                          int *count) {
  const int nw = a.nwords;
  const int w0 = (start >> 5) % nw, r = start & 31;
  // bitmap positions k = 0 .. nw: word (w0 + k) mod nw, the start word split in
  // its bits from r on (k = 0) and, last, its bits below r (k = nw)
  int k0 = 0;          // first position of this round's words
  int skip = 0;        // set bits of word k0 already taken by earlier rounds
  bool held = false;   // a slot with units left, held back by the lookahead
  while (k0 <= nw) {
    const int k = k0 + lane;
    unsigned word = 0u;
    int widx = 0;
    if (k <= nw) {
      widx = (w0 + k) % nw;
      word = __ldcg(a.live + widx);
      if (k == 0) word &= ~0u << r;
      else if (k == nw) word &= r ? ~(~0u << r) : 0u;
    }
    if (lane == 0)
      for (int q = 0; q < skip && word; ++q) word &= word - 1;   // taken by the previous round
    const int cnt = __popc(word);
    int incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(tb::kFull, incl, d);
      if (lane >= d) incl += v;
    }
    const int total = __shfl_sync(tb::kFull, incl, 31);
    // lane l takes the l-th gathered bit: the first lane whose inclusive count exceeds l
    int j = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1)
      if (__shfl_sync(tb::kFull, incl, j + step - 1) <= lane) j += step;
    const unsigned wj = __shfl_sync(tb::kFull, word, j);
    const int exj = __shfl_sync(tb::kFull, incl - cnt, j);
    const int wij = __shfl_sync(tb::kFull, widx, j);
    int s = -1;
    if (lane < total) {
      unsigned b = wj;  // drop the word's lowest (lane - exj) set bits; the next one is this lane's
      for (int q = lane - exj; q > 0 && b; --q) b &= b - 1;
      if (b) s = wij * 32 + (__ffs(b) - 1);
    }
    bool ok = false, left = false;
    if (s >= 0) {
      const unsigned long long c = ld_acquire_u64(&a.ctl[s].claim);
      const unsigned long long lim = __ldcg(&a.ctl[s].lim);
      if ((c >> 40) == (lim >> 40) && (c >> 40) != 0ull) {
        const int64_t next = (int64_t)(c & kUnitMask), units = (int64_t)(lim & kUnitMask);
        const int64_t fin = (int64_t)__ldcg(&a.ctl[s].fin), nseg = __ldcg(&a.req[s].nseg);
        left = next < units;
        ok = left && next < fin + (nseg * ahead_q) / 4 + 1;
      }
    }
    held = held || __any_sync(tb::kFull, left);
    const unsigned cand = __ballot_sync(tb::kFull, ok);
    if (cand) {
      const int l = __ffs(cand) - 1;
      int won = 0;
      unsigned long long got = 0;
      if (lane == l) {
        const unsigned long long old = atom_add_acq_rel(&a.ctl[s].claim, (unsigned long long)chunk);
        const unsigned long long lim = __ldcg(&a.ctl[s].lim);
        const int64_t first = (int64_t)(old & kUnitMask), units = (int64_t)(lim & kUnitMask);
        if ((old >> 40) == (lim >> 40) && first < units) {
          won = (int)(units - first < chunk ? units - first : chunk);
          got = (unsigned long long)first;
        }
      }
      const int sl = __shfl_sync(tb::kFull, s, l);
      const int n_won = __shfl_sync(tb::kFull, won, l);
      if (n_won) {
        *unit = (int64_t)__shfl_sync(tb::kFull, got, l);
        *count = n_won;
        return sl;
      }
      return -2;  // lost the race for this slot: look again
    }
    if (total <= 32) {
      k0 += 32;     // every gathered bit of these words was looked at
      skip = 0;
    } else {
      // the 32nd gathered bit lies in the word of lane j31: the next round
      // starts there, past its bits already taken
      int j31 = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1)
        if (__shfl_sync(tb::kFull, incl, j31 + step - 1) <= 31) j31 += step;
      const int ex31 = __shfl_sync(tb::kFull, incl - cnt, j31);
      skip = (j31 == 0 ? skip : 0) + (32 - ex31);
      k0 += j31;
    }
  }
  return held ? -3 : -1;
}

// A request's descriptor through L2 (an SM's L1 may hold the slot's previous
// request): it is stable while the request has unfinished units.
__device__ __forceinline__ SReq load_req(const SReq *p) {
  SReq r;
  const unsigned long long *src = (const unsigned long long *)p;
  unsigned long long *d = (unsigned long long *)&r;
#pragma unroll
  for (int i = 0; i < (int)(sizeof(SReq) / 8); ++i) d[i] = __ldcg(src + i);
  return r;
}

template <int MODE, int EP>
__global__ void __launch_bounds__(kSWarps * 32, MODE == 2 ? 1 : 8) k_serve(ServeArgs a) {
  using T = typename tb::TBCx<MODE, EP>::T;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const bool int_warp = MODE == 0 && (((blockIdx.x ^ wib) & 1) != 0);
  volatile int *exiting = &a.idle->exiting;
  unsigned long long idle_since = wave::globaltimer_ns();
  unsigned nap = 64;
  const int nslots = a.nwords * 32;
  // half of the warps serve the oldest request first (slots are taken in
  // admission order, so the scan from the oldest slot on follows it), the
  // other half start anywhere and move on with every claim (processor sharing:
  // a short request is not held behind a long one)
  const bool fifo = (((blockIdx.x * kSWarps + wib) & 1) == 0);
  int start = (int)(((unsigned)(blockIdx.x * kSWarps + wib) * 2654435761u) % (unsigned)nslots);
  for (;;) {
    int quit = 0;
    if (lane == 0) quit = wave::aborted(a.st) || *exiting != 0;
    if (__shfl_sync(tb::kFull, quit, 0)) break;
    int64_t u0 = 0;
    int cnt = 0;
    if (fifo) {
      int o = 0;
      if (lane == 0) o = *a.oldest;
      o = __shfl_sync(tb::kFull, o, 0);
      start = o >= 0 && o < nslots ? o : 0;
    } else {
      start = start + 1 == nslots ? 0 : start + 1;
    }
    const int s = claim_unit(a, lane, start, ClaimRule<MODE>::ahead_q, ClaimRule<MODE>::chunk, &u0, &cnt);
    if (s == -2) continue;  // a claim past the slot's last unit: try again
    if (s == -3) {
      // admitted work held back by the lookahead: units finish soon, so keep
      // the warp (not idle); the stop word still ends it
      int out = 0;
      if (lane == 0) out = *a.stop != 0;
      if (__shfl_sync(tb::kFull, out, 0)) break;
      idle_since = wave::globaltimer_ns();
      __nanosleep(nap);
      if (nap < 1024) nap <<= 1;
      continue;
    }
    if (s < 0) {
      // no work: the host-mapped stop word and the idle limit are read here only
      int out = 0;
      if (lane == 0) {
        out = *a.stop != 0;
        if (!out && wave::globaltimer_ns() - idle_since > (unsigned long long)a.idle_ns) {
          *exiting = 1;
          out = 1;
        }
      }
      if (__shfl_sync(tb::kFull, out, 0)) break;
      __nanosleep(nap);
      if (nap < 8192) nap <<= 1;
      continue;
    }
    nap = 64;
    __syncwarp();
    const SReq R = load_req(a.req + s);
    const int64_t nseg = R.nseg, base = R.done_base;
    bool stop = false;
    for (int64_t u = u0; u < u0 + cnt; ++u) {  // the chunk's units, in order
      const int64_t b = u / nseg, j = u - b * nseg;
      if (b > 0 && !wave::wait_neighbours(a.done + base, nseg, j, (unsigned)b, a.wait_ns, a.st, s, lane)) {
        stop = true;
        break;
      }
      int64_t lo, hi;
      wave::tile_bounds(R.n, nseg, j, lo, hi);
      const int par = (int)(b & 1);
      const T *src = (const T *)(par ? a.arena1 : a.arena0) + R.off;
      T *dst = (T *)(par ? a.arena0 : a.arena1) + R.off;
      const int64_t left = R.nt - b * a.T;
      const int steps = (int)(left < a.T ? left : a.T);
      bool int_tile = false, p2 = false;
      wave::Engine e;
      if constexpr (MODE == 0) {
        int_tile = R.int_ok && int_warp;
        p2 = R.mx.pow2 != 0;
        e.mx = R.mx;
        e.dom_lo = R.dom_lo;
        e.dom_hi = R.dom_hi;
        e.p2_hi_add = R.p2_hi_add;
        e.p2_hi_xor = R.p2_hi_xor;
      }
      wave::advance_tile<MODE, EP>(src, dst, R.n, lo, hi, a.T, steps, R.r, R.rf, int_tile, p2, e, lane);
      wave::publish(a.done + base + j, (unsigned)(b + 1), lane);
      if (lane == 0) {
        const unsigned gen = R.gen;
        if ((int64_t)atomicAdd(&a.ctl[s].fin, 1ull) + 1 == R.units) {
          __threadfence_system();
          a.complete[s] = (int)gen;
        }
      }
      __syncwarp();
    }
    if (stop) break;
    idle_since = wave::globaltimer_ns();
  }
}

// Publish slot s: clear its tile counters and write its descriptor; then,
// after a fence, the finished count, the generation-tagged limit, the
// generation-tagged claim counter (release) and the slot's live bit.
__global__ void k_serve_publish(SReq *req, SCtl *ctl, unsigned *live, unsigned *done, int s, SReq d,
                                unsigned gen) {
  for (int64_t i = threadIdx.x; i < d.nseg; i += blockDim.x) done[d.done_base + i] = 0u;
  if (threadIdx.x == 0) req[s] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long tag = (unsigned long long)gen << 40;
    ctl[s].fin = 0ull;
    ctl[s].lim = tag | (unsigned long long)d.units;
    __threadfence();
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(&ctl[s].claim), "l"(tag) : "memory");
    atomicOr(live + (s >> 5), 1u << (s & 31));
  }
}

// Take slot s out of the bitmap (its request is complete: no unit is left to
// claim).
__global__ void k_serve_unpublish(unsigned *live, int s) { atomicAnd(live + (s >> 5), ~(1u << (s & 31))); }

__global__ void k_serve_f64_to_f32(const double *__restrict__ s, float *__restrict__ d, int64_t n) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += st) d[i] = __double2float_rn(s[i]);
}

__global__ void k_serve_f32_to_f64(const float *__restrict__ s, double *__restrict__ d, int64_t n) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += st) d[i] = (double)s[i];
}

template <int MODE, int EP>
int serve_per_sm() {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_serve<MODE, EP>, kSWarps * 32, 0) != cudaSuccess)
    return 0;
  return per_sm;
}

}  // namespace
}  // namespace heat

using heat::SReq;
using heat::SCtl;

struct heat_server {
  struct Slot {
    bool used = false, complete = false, reported = false;
    int64_t ticket = 0;  // admission order
    int64_t off = 0, len = 0, n = 0, nt = 0, done_base = 0, nseg = 0, levels = 0;
    unsigned gen = 0;
  };
  heat_dtype dtype = HEAT_F64;
  size_t elem = 8;
  int device = 0, sms = 0;
  int T = 16;
  int64_t window = 512;
  void *arena[2] = {nullptr, nullptr};
  int64_t capacity = 0;
  std::map<int64_t, int64_t> free_pts;   // arena: offset -> length
  int64_t done_cap = 0;
  std::map<int64_t, int64_t> free_done;  // tile counters: offset -> length
  int32_t S = 0;
  std::vector<Slot> slots;
  std::vector<unsigned> uses;            // per slot: publications so far (generation source)
  SReq *d_req = nullptr;
  SCtl *d_ctl = nullptr;
  unsigned *d_live = nullptr;
  unsigned *d_done = nullptr;
  int *h_complete = nullptr, *d_complete = nullptr;  // host-mapped
  int *h_stop = nullptr, *d_stop = nullptr;          // host-mapped
  int *h_oldest = nullptr, *d_oldest = nullptr;      // host-mapped
  int32_t next_slot = 0;                             // slots are taken round-robin (admission order)
  int64_t tickets = 0;                               // admission counter
  heat::DevStatus *dstat = nullptr, *hstat = nullptr;
  heat::SIdle *d_idle = nullptr;                     // the running launch's idle state
  int host_error = HEAT_OK;
  cudaStream_t kstream = nullptr, cstream = nullptr;
  cudaEvent_t kdone = nullptr, published = nullptr;
  bool launched = false;
  int ctas_per_sm = 0;
  long long wait_ns = 5000000000LL, idle_ns = 200000000LL;
  int64_t point_steps = 0;
  int32_t in_flight = 0;
  int64_t launches = 0;
};

namespace {

int64_t first_fit(std::map<int64_t, int64_t> &fb, int64_t len) {
  for (auto it = fb.begin(); it != fb.end(); ++it)
    if (it->second >= len) {
      const int64_t off = it->first, rest = it->second - len;
      fb.erase(it);
      if (rest > 0) fb[off + len] = rest;
      return off;
    }
  return -1;
}

void give_back(std::map<int64_t, int64_t> &fb, int64_t off, int64_t len) {
  auto it = fb.emplace(off, len).first;
  auto nx = std::next(it);
  if (nx != fb.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    fb.erase(nx);
  }
  if (it != fb.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      fb.erase(it);
    }
  }
}

int server_ep(const heat_server *s) { return (int)(s->window / 32); }

bool kernel_running(heat_server *s) {
  if (!s->launched) return false;
  const cudaError_t e = cudaEventQuery(s->kdone);
  if (e == cudaErrorNotReady) return true;
  cudaGetLastError();
  return false;
}

// After the kernel ended: fold its device status into the sticky host error.
int collect_status(heat_server *s) {
  if (cudaStreamSynchronize(s->kstream) != cudaSuccess) return HEAT_ECUDA;
  if (cudaMemcpy(s->hstat, s->dstat, sizeof(heat::DevStatus), cudaMemcpyDeviceToHost) != cudaSuccess)
    return HEAT_ECUDA;
  if (s->hstat->code != HEAT_OK && s->host_error == HEAT_OK) s->host_error = s->hstat->code;
  return s->host_error;
}

template <int MODE, int EP>
int launch_serve_ep(heat_server *s) {
  int per_sm = heat::serve_per_sm<MODE, EP>();
  if (per_sm < 2) return HEAT_ENOTSUP;  // one CTA per SM must stay free for the publish kernels
  int cap = per_sm - 1;
  if (s->ctas_per_sm > 0 && s->ctas_per_sm < cap) cap = s->ctas_per_sm;
  heat::ServeArgs a;
  memset(&a, 0, sizeof(a));
  a.arena0 = s->arena[0];
  a.arena1 = s->arena[1];
  a.req = s->d_req;
  a.ctl = s->d_ctl;
  a.live = s->d_live;
  a.nwords = (s->S + 31) / 32;
  a.done = s->d_done;
  a.complete = s->d_complete;
  a.stop = s->d_stop;
  a.oldest = s->d_oldest;
  a.st = s->dstat;
  a.idle = s->d_idle;
  a.wait_ns = s->wait_ns;
  a.idle_ns = s->idle_ns;
  a.T = s->T;
  if (cudaMemsetAsync(s->d_idle, 0, sizeof(heat::SIdle), s->kstream) != cudaSuccess) return HEAT_ECUDA;
  heat::k_serve<MODE, EP><<<cap * s->sms, heat::kSWarps * 32, 0, s->kstream>>>(a);
  if (cudaGetLastError() != cudaSuccess) return HEAT_ECUDA;
  return HEAT_OK;
}

int launch_serve(heat_server *s) {
  // the kernel sees every publication queued so far
  if (cudaEventRecord(s->published, s->cstream) != cudaSuccess ||
      cudaStreamWaitEvent(s->kstream, s->published, 0) != cudaSuccess)
    return HEAT_ECUDA;
  const int ep = server_ep(s);
  int rc;
  if (s->dtype == HEAT_F32C)
    rc = ep == 32 ? launch_serve_ep<2, 32>(s) : ep == 16 ? launch_serve_ep<2, 16>(s) : launch_serve_ep<2, 8>(s);
  else
    rc = ep == 16 ? launch_serve_ep<0, 16>(s) : ep == 8 ? launch_serve_ep<0, 8>(s) : launch_serve_ep<0, 4>(s);
  if (rc != HEAT_OK) return rc;
  if (cudaEventRecord(s->kdone, s->kstream) != cudaSuccess) return HEAT_ECUDA;
  s->launched = true;
  s->launches += 1;
  return HEAT_OK;
}

// Tell the kernel which slot holds the oldest request still in flight.
void note_oldest(heat_server *s) {
  int32_t best = -1;
  int64_t t = INT64_MAX;
  for (int32_t i = 0; i < s->S; ++i) {
    const heat_server::Slot &sl = s->slots[i];
    if (sl.used && !sl.reported && sl.ticket < t) {
      t = sl.ticket;
      best = i;
    }
  }
  *(volatile int *)s->h_oldest = best < 0 ? 0 : best;
}

// Make sure the kernel runs while requests are in flight.
int keep_running(heat_server *s) {
  if (s->in_flight == 0 || kernel_running(s)) return HEAT_OK;
  if (s->launched) {
    const int rc = collect_status(s);
    if (rc != HEAT_OK) return rc;
  }
  return launch_serve(s);
}

void free_server(heat_server *s) {
  if (!s) return;
  if (s->h_stop) *(volatile int *)s->h_stop = 1;
  if (s->kstream) cudaStreamSynchronize(s->kstream);
  if (s->cstream) cudaStreamSynchronize(s->cstream);
  for (int i = 0; i < 2; ++i)
    if (s->arena[i]) cudaFree(s->arena[i]);
  if (s->d_req) cudaFree(s->d_req);
  if (s->d_ctl) cudaFree(s->d_ctl);
  if (s->d_live) cudaFree(s->d_live);
  if (s->d_done) cudaFree(s->d_done);
  if (s->h_complete) cudaFreeHost(s->h_complete);
  if (s->h_stop) cudaFreeHost(s->h_stop);
  if (s->h_oldest) cudaFreeHost(s->h_oldest);
  if (s->dstat) cudaFree(s->dstat);
  if (s->d_idle) cudaFree(s->d_idle);
  if (s->hstat) cudaFreeHost(s->hstat);
  if (s->kdone) cudaEventDestroy(s->kdone);
  if (s->published) cudaEventDestroy(s->published);
  if (s->kstream) cudaStreamDestroy(s->kstream);
  if (s->cstream) cudaStreamDestroy(s->cstream);
  delete s;
}

}  // namespace

extern "C" {

int heat_server_create(heat_server **out, int64_t capacity_points, heat_dtype dtype, int32_t max_requests, int T,
                       int ctas_per_sm) {
  if (!out) return HEAT_EINVAL;
  *out = nullptr;
  if (capacity_points < 1 || max_requests < 1 || max_requests > (1 << 16) || T < 0 || T > heat::kMaxT ||
      ctas_per_sm < 0)
    return HEAT_EINVAL;
  if (dtype != HEAT_F64 && dtype != HEAT_F32C) return HEAT_EINVAL;
  heat_server *s = new (std::nothrow) heat_server();
  if (!s) return HEAT_ENOMEM;
  s->dtype = dtype;
  s->elem = dtype == HEAT_F64 ? 8 : 4;
  s->T = T > 0 ? T : (dtype == HEAT_F32C ? 32 : 16);
  // binary64: 16 points per lane; binary32: 8 (about 95 registers a thread, so
  // a binary32 server keeps two or more CTAs per SM beside a binary64 one)
  s->window = dtype == HEAT_F32C ? 256 : 512;
  s->capacity = (capacity_points + 63) / 64 * 64;
  s->S = max_requests;
  s->ctas_per_sm = ctas_per_sm;
  s->slots.resize((size_t)s->S);
  s->uses.assign((size_t)s->S, 0u);
  const int64_t W = s->window - 2 * (int64_t)s->T;
  s->done_cap = s->capacity / W + 2 * (int64_t)s->S;
  int rc = HEAT_OK;
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess)
    rc = HEAT_ECUDA;
  for (int i = 0; i < 2 && rc == HEAT_OK; ++i)
    if (cudaMalloc(&s->arena[i], (size_t)s->capacity * s->elem) != cudaSuccess) rc = HEAT_ENOMEM;
  if (rc == HEAT_OK && (cudaMalloc((void **)&s->d_req, sizeof(SReq) * (size_t)s->S) != cudaSuccess ||
                        cudaMalloc((void **)&s->d_ctl, sizeof(SCtl) * (size_t)s->S) != cudaSuccess ||
                        cudaMalloc((void **)&s->d_live, sizeof(unsigned) * (size_t)((s->S + 31) / 32)) !=
                            cudaSuccess ||
                        cudaMalloc((void **)&s->d_done, sizeof(unsigned) * (size_t)s->done_cap) != cudaSuccess ||
                        cudaMalloc((void **)&s->dstat, sizeof(heat::DevStatus)) != cudaSuccess ||
                        cudaMalloc((void **)&s->d_idle, sizeof(heat::SIdle)) != cudaSuccess))
    rc = HEAT_ENOMEM;
  if (rc == HEAT_OK &&
      (cudaHostAlloc((void **)&s->h_complete, sizeof(int) * (size_t)s->S, cudaHostAllocMapped) != cudaSuccess ||
       cudaHostAlloc((void **)&s->h_stop, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
       cudaHostAlloc((void **)&s->h_oldest, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
       cudaHostAlloc((void **)&s->hstat, sizeof(heat::DevStatus), cudaHostAllocDefault) != cudaSuccess))
    rc = HEAT_ENOMEM;
  if (rc == HEAT_OK && (cudaHostGetDevicePointer((void **)&s->d_complete, s->h_complete, 0) != cudaSuccess ||
                        cudaHostGetDevicePointer((void **)&s->d_stop, s->h_stop, 0) != cudaSuccess ||
                        cudaHostGetDevicePointer((void **)&s->d_oldest, s->h_oldest, 0) != cudaSuccess))
    rc = HEAT_ECUDA;
  if (rc == HEAT_OK && (cudaStreamCreateWithFlags(&s->kstream, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaEventCreateWithFlags(&s->kdone, cudaEventDisableTiming) != cudaSuccess ||
                        cudaEventCreateWithFlags(&s->published, cudaEventDisableTiming) != cudaSuccess))
    rc = HEAT_ECUDA;
  if (rc == HEAT_OK) {
    memset(s->h_complete, 0, sizeof(int) * (size_t)s->S);
    *s->h_stop = 0;
    *s->h_oldest = 0;
    if (cudaMemsetAsync(s->d_req, 0, sizeof(SReq) * (size_t)s->S, s->cstream) != cudaSuccess ||
        cudaMemsetAsync(s->d_ctl, 0, sizeof(SCtl) * (size_t)s->S, s->cstream) != cudaSuccess ||
        cudaMemsetAsync(s->d_live, 0, sizeof(unsigned) * (size_t)((s->S + 31) / 32), s->cstream) != cudaSuccess ||
        cudaMemsetAsync(s->dstat, 0, sizeof(heat::DevStatus), s->cstream) != cudaSuccess ||
        cudaStreamSynchronize(s->cstream) != cudaSuccess)
      rc = HEAT_ECUDA;
  }
  if (rc == HEAT_OK) {
    // one CTA per SM must stay free beside the server kernel
    const int ep = server_ep(s);
    const int per = dtype == HEAT_F32C ? heat::serve_per_sm<2, 8>() : heat::serve_per_sm<0, 16>();
    (void)ep;
    if (per < 2) rc = HEAT_ENOTSUP;
  }
  if (rc != HEAT_OK) {
    cudaGetLastError();
    free_server(s);
    return rc;
  }
  s->free_pts[0] = s->capacity;
  s->free_done[0] = s->done_cap;
  *out = s;
  return HEAT_OK;
}

void heat_server_destroy(heat_server *s) { free_server(s); }

int heat_server_set_limits(heat_server *s, int64_t wait_ns, int64_t idle_ns) {
  if (!s || wait_ns < 0 || idle_ns < 0) return HEAT_EINVAL;
  if (wait_ns > 0) s->wait_ns = wait_ns;
  if (idle_ns > 0) s->idle_ns = idle_ns;
  return HEAT_OK;
}

int heat_server_submit(heat_server *s, int64_t n, double k, double dt, double dx, int64_t nt, const double *dev_u,
                       int32_t *req_id) {
  if (!s || !dev_u || !req_id || n < 1 || nt < 1) return HEAT_EINVAL;
  if (((uintptr_t)dev_u & 7u) != 0) return HEAT_EINVAL;
  if (!isfinite(k) || !isfinite(dt) || !isfinite(dx) || dx == 0.0) return HEAT_EINVAL;
  const double r = (k * dt) / (dx * dx);
  if (!isfinite(r)) return HEAT_EINVAL;
  if (s->host_error != HEAT_OK) return HEAT_ESTATE;
  int32_t id = -1;
  for (int32_t q = 0; q < s->S; ++q) {  // round-robin from the last slot taken: slot order is admission order
    const int32_t i = (s->next_slot + q) % s->S;
    if (!s->slots[i].used) {
      id = i;
      break;
    }
  }
  if (id < 0) return HEAT_ENOMEM;
  const int64_t len = (n + 63) / 64 * 64;
  const int64_t W = s->window - 2 * (int64_t)s->T;
  const int64_t nseg = (n + W - 1) / W;
  const int64_t off = first_fit(s->free_pts, len);
  if (off < 0) return HEAT_ENOMEM;
  const int64_t dbase = first_fit(s->free_done, nseg);
  if (dbase < 0) {
    give_back(s->free_pts, off, len);
    return HEAT_ENOMEM;
  }
  // initial state into arena buffer 0 (level 0 reads buffer 0)
  void *dst = (char *)s->arena[0] + (size_t)off * s->elem;
  cudaError_t e;
  if (s->dtype == HEAT_F64) {
    e = cudaMemcpyAsync(dst, dev_u, (size_t)n * 8, cudaMemcpyDeviceToDevice, s->cstream);
  } else {
    const int grid = (int)std::min<int64_t>((n + 127) / 128, (int64_t)s->sms * 4);
    heat::k_serve_f64_to_f32<<<std::max(grid, 1), 128, 0, s->cstream>>>(dev_u, (float *)dst, n);
    e = cudaGetLastError();
  }
  SReq d;
  memset(&d, 0, sizeof(d));
  d.off = off;
  d.n = n;
  d.nseg = nseg;
  const int64_t levels = (nt + s->T - 1) / s->T;
  d.units = levels * nseg;
  d.nt = nt;
  d.done_base = dbase;
  d.r = r;
  d.rf = (float)r;
  uint64_t rbits;
  memcpy(&rbits, &r, sizeof(rbits));
  const int rexp = (int)((rbits >> 52) & 2047);
  d.mx = heat::emul::prepare_mulx(rbits);
  d.p2_hi_add = (rexp - 1023) * (1 << 20);
  d.p2_hi_xor = (rbits >> 63) ? (int)0x80000000u : 0;
  if (rexp < 1 || rexp > 2046 || !heat::emul::domain_bounds(rbits, s->T, d.dom_lo, d.dom_hi)) {
    d.dom_lo = 1;  // no screen admits data: every tile on the FP64 unit
    d.dom_hi = 0;
  }
  d.int_ok = s->dtype == HEAT_F64 && d.dom_lo <= d.dom_hi;
  const unsigned gen = (s->uses[id]++ % 0xffffffu) + 1u;
  d.gen = gen;
  if (e == cudaSuccess) {
    heat::k_serve_publish<<<1, 128, 0, s->cstream>>>(s->d_req, s->d_ctl, s->d_live, s->d_done, id, d, gen);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    give_back(s->free_pts, off, len);
    give_back(s->free_done, dbase, nseg);
    return HEAT_ECUDA;
  }
  heat_server::Slot &sl = s->slots[id];
  sl.used = true;
  sl.complete = sl.reported = false;
  sl.ticket = s->tickets++;
  s->next_slot = (id + 1) % s->S;
  sl.off = off;
  sl.len = len;
  sl.n = n;
  sl.nt = nt;
  sl.done_base = dbase;
  sl.nseg = nseg;
  sl.levels = levels;
  sl.gen = gen;
  s->in_flight += 1;
  *req_id = id;
  note_oldest(s);
  return keep_running(s);
}

int heat_server_poll(heat_server *s, int32_t *done_ids, int32_t max, int32_t *count) {
  if (!s || !count || max < 0 || (max > 0 && !done_ids)) return HEAT_EINVAL;
  *count = 0;
  for (int32_t i = 0; i < s->S && *count < max; ++i) {
    heat_server::Slot &sl = s->slots[i];
    if (!sl.used || sl.reported) continue;
    if ((unsigned)*(volatile int *)(s->h_complete + i) != sl.gen) continue;
    sl.complete = sl.reported = true;
    s->in_flight -= 1;
    s->point_steps += sl.n * sl.nt;
    done_ids[(*count)++] = i;
  }
  if (*count) note_oldest(s);
  if (s->host_error != HEAT_OK) return s->host_error;
  return keep_running(s);
}

int heat_server_get_device(heat_server *s, int32_t req_id, double *dev_u, int64_t n, void *cuda_event) {
  if (!s || !dev_u || req_id < 0 || req_id >= s->S) return HEAT_EINVAL;
  const heat_server::Slot &sl = s->slots[req_id];
  if (!sl.used || n != sl.n) return HEAT_EINVAL;
  if (!sl.complete) return HEAT_ESTATE;
  // the state after `levels` levels is in buffer levels mod 2
  const void *src = (const char *)s->arena[sl.levels & 1] + (size_t)sl.off * s->elem;
  cudaError_t e;
  if (s->dtype == HEAT_F64) {
    e = cudaMemcpyAsync(dev_u, src, (size_t)n * 8, cudaMemcpyDeviceToDevice, s->cstream);
  } else {
    const int grid = (int)std::min<int64_t>((n + 127) / 128, (int64_t)s->sms * 4);
    heat::k_serve_f32_to_f64<<<std::max(grid, 1), 128, 0, s->cstream>>>((const float *)src, dev_u, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && cuda_event) e = cudaEventRecord((cudaEvent_t)cuda_event, s->cstream);
  return e == cudaSuccess ? HEAT_OK : HEAT_ECUDA;
}

int heat_server_release(heat_server *s, int32_t req_id) {
  if (!s || req_id < 0 || req_id >= s->S) return HEAT_EINVAL;
  heat_server::Slot &sl = s->slots[req_id];
  if (!sl.used || !sl.complete) return HEAT_ESTATE;
  heat::k_serve_unpublish<<<1, 1, 0, s->cstream>>>(s->d_live, req_id);
  if (cudaGetLastError() != cudaSuccess) return HEAT_ECUDA;
  // later uses of the space and counters are queued behind the copies on cstream
  give_back(s->free_pts, sl.off, sl.len);
  give_back(s->free_done, sl.done_base, sl.nseg);
  sl.used = false;
  return HEAT_OK;
}

int heat_server_info(const heat_server *s, int64_t *point_steps, int32_t *in_flight, int *running,
                     int64_t *launches) {
  if (!s) return HEAT_EINVAL;
  if (point_steps) *point_steps = s->point_steps;
  if (in_flight) *in_flight = s->in_flight;
  if (running) *running = kernel_running(const_cast<heat_server *>(s)) ? 1 : 0;
  if (launches) *launches = s->launches;
  return HEAT_OK;
}

}  // extern "C"

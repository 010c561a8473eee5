// k_queue.cu -- form HEAT_FORM_PERSIST at depth T >= 2: the persistent
// flag-queue form with T-point ghost zones.  One co-resident (cooperative)
// launch runs all nt steps.
//
// As in the one-step kernel (k_persist.cu), CTA i owns segment i of the ring
// for the whole run (Section 2: each thread of execution applies Eq. 2 to its
// own segment) and swaps ghost values with its two neighbours through
// single-producer single-consumer flag queues in device memory: two slots of
// {T values} per directed edge and one sequence word.  Here a queue message
// carries T edge values instead of one, and the segment advances T steps per
// message:
//
//   block b (time bT -> bT + steps): the segment's warp tiles (at most
//   W = 32E - 2T points, near-equal) advance in registers with the
//   temporal-blocking core, each reading its window [lo - T, hi + T) at time bT
//   from the segment's own buffer, or from the queue slot b % 2 where the
//   window leaves the segment.  The two edge tiles are taken first: each waits
//   (bounded, ld.acquire) until its neighbour's sequence word reaches b + 1,
//   and after its steps writes its T outermost output values into the
//   neighbour's slot (b + 1) % 2 and releases sequence b + 2.  A CTA barrier
//   ends the block (the tiles of block b + 1 read what block b wrote).
//
// No CTA reads another CTA's part of the state: the queues are the only
// exchange.  Two slots suffice: a producer overwrites slot (b + 1) % 2 only
// after it acquired the consumer's message b + 1, which the consumer released
// after reading that slot during block b - 1.  Every CTA is resident, and the
// CTA at the smallest block always finds its neighbours' messages for that
// block published, so the launch makes progress.
//
// Inside a CTA the tiles of a block are claimed from a shared counter; with the
// library's binary64 split half of the warps compute on the integer pipes and
// half on the FP64 unit, so each engine takes tiles at its own speed.  Every
// point is computed from the same operands as in the other forms, so the state
// is bitwise the oracle's (binary32 compensated: the same blocks of T steps as
// the other temporal-blocking forms).
//
// Every wait is bounded (iteration cap and %globaltimer deadline); one that runs
// out records HEAT_ETIMEOUT, raises the abort word and every CTA returns.
#include <string.h>

#include "wave_core.cuh"

namespace heat {
namespace {

constexpr int kQWarps = 8;
constexpr int kQThreads = kQWarps * 32;

struct QueueArgs {
  void *buf0, *buf1;
  int cur;             // buffer holding the state at time 0
  int T;
  int64_t nt;
  int64_t levels;      // ceil(nt / T)
  double r;
  float rf;
  const int64_t *seg;  // S + 1 boundaries
  int S;
  int W;               // widest tile (points)
  Mailbox *mb;         // mb[2i] = in_left of segment i, mb[2i+1] = in_right
  DevStatus *st;
  long long wait_ns;
  int inj_seg;         // test hook: this segment publishes no time >= inj_step (-1: none)
  long long inj_step;
  int dual;            // binary64, library's split: integer-pipe warps and FP64-unit warps
  unsigned emul_mask;  // otherwise: bit (tile mod 32) set -> that tile on the integer pipes
  int p2_fp64;         // r = +-2^k: screened FP64-unit tiles move the product's exponent
  wave::Engine eng;
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Bounded wait (one thread) until *seq >= target; on giving up, the first
// waiter records where and raises the abort word.
static __device__ __noinline__ bool wait_seq(const unsigned long long *seq, unsigned long long target,
                                             long long wait_ns, DevStatus *st, int where, long long step) {
  if (ld_acquire_u64(seq) >= target) return true;
  const unsigned long long deadline = wave::globaltimer_ns() + (unsigned long long)wait_ns;
  unsigned ns = 32;
  for (long long spin = 0; spin < wave::kSpins; ++spin) {
    if (ld_acquire_u64(seq) >= target) return true;
    if (wave::aborted(st)) return false;
    if (wave::globaltimer_ns() > deadline) break;
    __nanosleep(ns);
    if (ns < 512) ns <<= 1;
  }
  if (atomicCAS(&st->code, HEAT_OK, HEAT_ETIMEOUT) == HEAT_OK) {
    st->segment = where;
    st->step = step;
  }
  atomicExch(&st->abort, 1);
  return false;
}

template <int MODE, int EP>
__global__ void __launch_bounds__(kQThreads, MODE == 2 ? 1 : 4) k_queue(QueueArgs a) {
  using P = tb::TBCx<MODE, EP>;
  using V = typename P::T;
  constexpr int E = P::E;
  __shared__ int claim[2];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int i = blockIdx.x, S = a.S, T = a.T;
  const int64_t lo = a.seg[i], hi = a.seg[i + 1], L = hi - lo;
  const int64_t ntl = (L + a.W - 1) / a.W;
  Mailbox *in_l = a.mb + 2 * i, *in_r = a.mb + 2 * i + 1;
  Mailbox *to_l = a.mb + 2 * (i == 0 ? S - 1 : i - 1) + 1;  // the left neighbour's in_right
  Mailbox *to_r = a.mb + 2 * (i == S - 1 ? 0 : i + 1);      // the right neighbour's in_left
  const bool int_warp = MODE == 0 && a.dual && (wib & 1) != 0;

  if (threadIdx.x < 2) claim[threadIdx.x] = 0;
  // message 0: the segment's edge values at time 0
  if (wib == 0 && !(i == a.inj_seg && a.inj_step <= 0)) {
    const V *s0 = (const V *)(a.cur ? a.buf1 : a.buf0);
    V *ml = reinterpret_cast<V *>(to_l->val[0]), *mr = reinterpret_cast<V *>(to_r->val[0]);
    for (int j = lane; j < T; j += 32) {
      ml[j] = __ldcg(s0 + lo + j);
      mr[j] = __ldcg(s0 + hi - T + j);
    }
    __syncwarp();
    if (lane == 0) {
      st_release_u64(&to_l->seq, 1ull);
      st_release_u64(&to_r->seq, 1ull);
    }
  }
  __syncthreads();

  for (int64_t b = 0; b < a.levels; ++b) {
    const int par = (a.cur ^ (int)(b & 1)) & 1;
    const V *src = (const V *)(par ? a.buf1 : a.buf0);
    V *dst = (V *)(par ? a.buf0 : a.buf1);
    const int64_t left = a.nt - b * T;
    const int steps = (int)(left < T ? left : T);
    const int slot = (int)(b & 1);
    const bool pub = !(i == a.inj_seg && b * T + steps >= a.inj_step);
    if (threadIdx.x == 0) claim[slot ^ 1] = 0;  // the next block's counter (last used by block b - 1)
    const V *gl = reinterpret_cast<const V *>(in_l->val[slot]);
    const V *gr = reinterpret_cast<const V *>(in_r->val[slot]);
    V *ol = reinterpret_cast<V *>(to_l->val[slot ^ 1]);
    V *orr = reinterpret_cast<V *>(to_r->val[slot ^ 1]);
    bool failed = false;
    for (;;) {
      int k = 0;
      if (lane == 0) k = wave::aborted(a.st) ? 0x7fffffff : atomicAdd(&claim[slot], 1);
      k = __shfl_sync(tb::kFull, k, 0);
      if (k >= ntl) break;
      // the edge tiles first, so the neighbours' next messages leave early
      const int64_t t = k == 0 ? 0 : (k == 1 ? ntl - 1 : k - 1);
      int64_t tlo, thi;
      wave::tile_bounds(L, ntl, t, tlo, thi);
      tlo += lo;
      thi += lo;
      const bool le = t == 0, re = t == ntl - 1;
      if (le || re) {
        bool ok = true;
        if (lane == 0 && le) ok = wait_seq(&in_l->seq, (unsigned long long)b + 1, a.wait_ns, a.st, i, b * T);
        if (lane == 1 && re) ok = wait_seq(&in_r->seq, (unsigned long long)b + 1, a.wait_ns, a.st, i, b * T);
        const bool all = __all_sync(tb::kFull, ok);
        __syncwarp();
        if (!all) {
          failed = true;
          break;
        }
      }
      const int64_t ws = tlo - T;
      const int need = (int)(thi - tlo) + 2 * T;
      typename P::Reg R;
#pragma unroll
      for (int k2 = 0; k2 < E; ++k2) {
        const int idx = E * lane + k2;
        V v = V(0);
        if (idx < need) {
          const int64_t g = ws + idx;
          v = g < lo ? __ldcg(gl + (g - lo + T)) : (g >= hi ? __ldcg(gr + (g - hi)) : __ldcg(src + g));
        }
        P::load(R, k2, v);
      }
      const bool int_tile = MODE == 0 && (a.dual ? int_warp : ((a.emul_mask >> (unsigned)(t & 31)) & 1u) != 0);
      wave::advance_window<MODE, EP>(R, steps, a.r, a.rf, int_tile, a.p2_fp64 != 0, a.eng, lane);
#pragma unroll
      for (int k2 = 0; k2 < E; ++k2) {
        const int idx = E * lane + k2;
        const int64_t g = ws + idx;
        if (idx >= T && g < thi) {
          const V v = P::store(R, k2);
          dst[g] = v;
          if (pub && le && idx < 2 * T) ol[idx - T] = v;
          if (pub && re && idx >= need - 2 * T) orr[idx - (need - 2 * T)] = v;
        }
      }
      if (pub && (le || re)) {
        __syncwarp();
        if (lane == 0) {
          if (le) st_release_u64(&to_l->seq, (unsigned long long)b + 2);
          if (re) st_release_u64(&to_r->seq, (unsigned long long)b + 2);
        }
      }
    }
    if (__syncthreads_or(failed || (threadIdx.x == 0 && wave::aborted(a.st)))) return;
  }
}

template <int MODE, int EP>
int resident_ctas(const heat_ctx *c) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_queue<MODE, EP>, kQThreads, 0) != cudaSuccess)
    return 0;
  return per_sm * c->sms;
}

// Segments for `resident` co-resident CTAs: one per partition when requested
// (and np CTAs fit), else near-equal segments of at least T points.
int queue_bounds(const heat_ctx *c, int resident, int T, int64_t **out) {
  const int64_t N = c->geo.N;
  int S;
  int64_t *b;
  if (c->segments < 0 && c->geo.np <= resident) {
    S = c->geo.np;
    b = (int64_t *)malloc(sizeof(int64_t) * (size_t)(S + 1));
    if (!b) return -1;
    for (int i = 0; i <= S; ++i) b[i] = (int64_t)i * c->geo.nx;
  } else {
    int64_t want = resident;
    if (c->segments > 0 && c->segments < want) want = c->segments;
    if (want > N / T) want = N / T;
    if (want < 1) want = 1;
    S = (int)want;
    b = (int64_t *)malloc(sizeof(int64_t) * (size_t)(S + 1));
    if (!b) return -1;
    for (int i = 0; i <= S; ++i) b[i] = (int64_t)((__int128)N * i / S);
  }
  *out = b;
  return S;
}

template <int MODE, int EP>
int launch_queue_ep(heat_ctx *c, QueueArgs a) {
  a.W = 32 * EP - 2 * a.T;
  void *params[] = {&a};
  return cuda_status(cudaLaunchCooperativeKernel((const void *)k_queue<MODE, EP>, dim3(a.S), dim3(kQThreads), params,
                                                 0, c->stream));
}

// Window: the widest that still gives every warp of a CTA a tile of a typical
// segment, else the narrowest; every choice keeps W >= 2T (an edge tile holds
// the T values of its message).
template <int MODE>
int run_queue_mode(heat_ctx *c, QueueArgs a, int64_t nt) {
  constexpr int eps[3] = {MODE == 2 ? 8 : 4, MODE == 2 ? 16 : 8, MODE == 2 ? 32 : 16};
  const int res[3] = {resident_ctas<MODE, eps[0]>(c), resident_ctas<MODE, eps[1]>(c), resident_ctas<MODE, eps[2]>(c)};
  int pick = -1;
  for (int p = 2; p >= 0; --p) {
    if (32 * eps[p] - 2 * a.T < 2 * a.T || res[p] < 1) continue;
    int64_t segs = c->geo.N / a.T;
    if (segs > res[p]) segs = res[p];
    const int64_t seg = c->geo.N / (segs > 1 ? segs : 1);
    const int64_t tiles = (seg + 32 * eps[p] - 2 * a.T - 1) / (32 * eps[p] - 2 * a.T);
    pick = p;
    if (tiles >= kQWarps) break;
  }
  if (pick < 0) return HEAT_ENOTSUP;
  int64_t *bounds = nullptr;
  const int S = queue_bounds(c, res[pick], a.T, &bounds);
  if (S < 1) return HEAT_ENOMEM;
  int64_t shortest = bounds[1] - bounds[0];
  for (int i = 1; i < S; ++i)
    if (bounds[i + 1] - bounds[i] < shortest) shortest = bounds[i + 1] - bounds[i];
  if (shortest < a.T) {  // partitions shorter than the depth: the caller takes the one-step kernel
    free(bounds);
    return HEAT_ENOTSUP;
  }
  int rc = prepare_segments(c, S, bounds);
  free(bounds);
  if (rc != HEAT_OK) return rc;
  a.S = S;
  a.seg = c->seg_start;
  a.mb = c->mbox;
  a.levels = (nt + a.T - 1) / a.T;
  switch (pick) {
    case 0: rc = launch_queue_ep<MODE, eps[0]>(c, a); break;
    case 1: rc = launch_queue_ep<MODE, eps[1]>(c, a); break;
    default: rc = launch_queue_ep<MODE, eps[2]>(c, a); break;
  }
  if (rc != HEAT_OK) return rc;
  c->last_segments = S;
  return HEAT_OK;
}

}  // namespace

// HEAT_FORM_PERSIST at depth T (2..64).  HEAT_ENOTSUP (nothing queued) when a
// partition is shorter than T.
int run_queue(heat_ctx *c, int64_t nt, int T) {
  const int mode = c->dtype == HEAT_F32C ? 2 : (c->arith == HEAT_ARITH_FMA ? 1 : 0);
  QueueArgs a;
  memset(&a, 0, sizeof(a));
  a.buf0 = c->buf[0];
  a.buf1 = c->buf[1];
  a.cur = c->cur;
  a.T = T;
  a.nt = nt;
  a.r = c->r;
  a.rf = c->rf;
  a.st = c->dstat;
  a.wait_ns = c->wait_ns;
  a.inj_seg = c->inj_segment;
  a.inj_step = c->inj_step;
  uint64_t rbits;
  memcpy(&rbits, &c->r, sizeof(rbits));
  const int rexp = (int)((rbits >> 52) & 2047);
  const bool dom = emul::domain_bounds(rbits, T, a.eng.dom_lo, a.eng.dom_hi);
  a.eng.mx = emul::prepare_mulx(rbits);
  const bool int_ok = mode == 0 && rexp >= 1 && rexp <= 2046 && dom;
  a.dual = int_ok && c->emul_auto;
  a.emul_mask = int_ok && !c->emul_auto ? c->emul_mask : 0u;
  a.p2_fp64 = mode == 0 && dom && a.eng.mx.pow2;
  a.eng.p2_hi_add = (int)(((int64_t)rexp - 1023) * (1 << 20));
  a.eng.p2_hi_xor = (rbits >> 63) ? (int)0x80000000u : 0;
  const int rc = mode == 0 ? run_queue_mode<0>(c, a, nt) : mode == 1 ? run_queue_mode<1>(c, a, nt)
                                                                     : run_queue_mode<2>(c, a, nt);
  if (rc != HEAT_OK) return rc;
  if (((nt + T - 1) / T) & 1) c->cur ^= 1;
  c->steps += nt;
  c->last_T = T;
  c->last_launches = 1;
  return HEAT_OK;
}

}  // namespace heat

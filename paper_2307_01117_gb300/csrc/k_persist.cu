// k_persist.cu -- form HEAT_FORM_PERSIST: one persistent, co-resident
// (cooperative) launch runs all nt steps.  The ring is cut into S segments
// (Section 2: "each thread of execution sequentially applies Eq. 2 on a local
// segment"); CTA c owns segments c, c + grid, ...  Ghost values cross between
// neighbouring segments through device-memory mailboxes -- the GPU form of the
// paper's single-producer single-consumer queues:
//
//   producer, after finishing step s of its segment:
//       write the segment's first value into the left neighbour's in_right
//       mailbox and its last value into the right neighbour's in_left mailbox,
//       slot (s+1) % 2; fence; st.release.gpu seq = s + 2
//   consumer, before step s:
//       ld.acquire.gpu seq until seq >= s + 1 (bounded), read slot s % 2
//
// Every wait is bounded by an iteration cap and a %globaltimer deadline; a wait
// that runs out records HEAT_ETIMEOUT in the device status word, raises the
// shared abort flag (so the other CTAs stop waiting) and the kernel returns
// normally.  Within a segment, points are processed as in the plain form (groups
// of four 64-point warp tiles, 16-byte vectors, shuffles for in-tile neighbours).
#include <string.h>

#include "dp_emul.cuh"
#include "heat_internal.cuh"
#include "stencil_ops.cuh"

namespace heat {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPersistThreads = 512;
constexpr long long kMaxSpins = 1LL << 26;  // backstop if the timer never advances

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }

struct PersistArgs {
  void *ua;               // state at time 0 on entry
  void *ub;               // other buffer
  int64_t N;
  double r;
  float rf;
  int64_t nt;
  const int64_t *seg;     // S + 1 boundaries, seg[0] = 0, seg[S] = N
  int S;
  Mailbox *mb;            // mb[2i] = in_left of segment i, mb[2i+1] = in_right
  DevStatus *st;
  long long wait_ns;
  int inj_seg;
  long long inj_step;
  // binary64, exact reading, r = +-2^k: tiles whose values pass the
  // integer-pipe screen for one step move the product's exponent with an
  // integer add (eq2_exact_pow2: 3 FP64-unit operations per point)
  int p2;
  int dom_lo, dom_hi, p2_hi_add, p2_hi_xor;
};

// Bounded wait until *seq >= target.  Returns false when the deadline passed or
// another CTA already gave up (abort); the first CTA to give up records where.
__device__ bool wait_seq(const PersistArgs &a, const unsigned long long *seq, unsigned long long target, int segment,
                         long long step) {
  if (ld_acquire(seq) >= target) return true;
  const unsigned long long deadline = globaltimer_ns() + (unsigned long long)a.wait_ns;
  unsigned ns = 32;
  for (long long spin = 0; spin < kMaxSpins; ++spin) {
    if (ld_acquire(seq) >= target) return true;
    if (ld_volatile(&a.st->abort)) return false;
    if (globaltimer_ns() > deadline) break;
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
  }
  if (atomicCAS(&a.st->code, HEAT_OK, HEAT_ETIMEOUT) == HEAT_OK) {
    a.st->segment = segment;
    a.st->step = step;
  }
  atomicExch(&a.st->abort, 1);
  return false;
}

template <int MODE>
struct Elem;
template <>
struct Elem<0> {
  using T = double;
  using V = double2;
  static __device__ __forceinline__ double upd(double l, double c, double r_, double r, float) {
    return eq2_exact(l, c, r_, r);
  }
};
template <>
struct Elem<1> {
  using T = double;
  using V = double2;
  static __device__ __forceinline__ double upd(double l, double c, double r_, double r, float) {
    return eq2_fma(l, c, r_, r);
  }
};
template <>
struct Elem<2> {
  using T = float;
  using V = float2;
  static __device__ __forceinline__ float upd(float l, float c, float r_, double, float rf) {
    float hn, ln;
    eq2_f32c(l, c, r_, 0.0f, 0.0f, 0.0f, rf, hn, ln);
    return f32c_store(hn, ln);
  }
};

// One step over the segment [lo, hi) of src into dst with the given ghosts.
// src was written earlier in this same launch, so it is read with L2-cached
// loads (never the read-only non-coherent path).  A warp takes kGroup
// consecutive 64-point tiles at a time (16-byte vectors, neighbours by shuffle,
// two edge values per group), so each lane has 2*kGroup independent updates to
// interleave and a group is screened once for the r = +-2^k multiply; the
// partial tiles at the segment's ends and the tiles left over after the groups
// are done point by point.
constexpr int kGroup = 4;

template <int MODE>
__device__ __forceinline__ void step_segment(const typename Elem<MODE>::T *src, typename Elem<MODE>::T *dst,
                                             int64_t lo, int64_t hi,
                                             typename Elem<MODE>::T gl, typename Elem<MODE>::T gr, double r,
                                             float rf, const PersistArgs &a) {
  using E = Elem<MODE>;
  using T = typename E::T;
  using V = typename E::V;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int64_t tf = (lo + 63) >> 6;       // first tile inside the segment
  const int64_t tl = hi >> 6;              // tiles [tf, tl) lie inside
  const int64_t ngroups = tl > tf ? (tl - tf) / kGroup : 0;
  for (int64_t q = warp; q < ngroups; q += nwarps) {
    const int64_t b0 = (tf + q * kGroup) << 6;
    V x[kGroup];
#pragma unroll
    for (int j = 0; j < kGroup; ++j) x[j] = __ldcg(reinterpret_cast<const V *>(src + b0 + 64 * j) + lane);
    T eleft = T(0), eright = T(0);
    if (lane == 0) eleft = b0 == lo ? gl : __ldcg(src + b0 - 1);
    if (lane == 31) eright = b0 + 64 * kGroup == hi ? gr : __ldcg(src + b0 + 64 * kGroup);
    bool p2 = false;
    if constexpr (MODE == 0) {
      if (a.p2) {
        auto in = [&](double v) { return emul::in_domain((uint64_t)__double_as_longlong(v), a.dom_lo, a.dom_hi); };
        bool ok = in(eleft) && in(eright);
#pragma unroll
        for (int j = 0; j < kGroup; ++j) ok = ok && in(x[j].x) && in(x[j].y);
        p2 = __all_sync(kFull, ok);
      }
    }
#pragma unroll
    for (int j = 0; j < kGroup; ++j) {
      T left = __shfl_up_sync(kFull, x[j].y, 1);
      T right = __shfl_down_sync(kFull, x[j].x, 1);
      const T prev_y = __shfl_sync(kFull, x[j > 0 ? j - 1 : 0].y, 31);
      const T next_x = __shfl_sync(kFull, x[j + 1 < kGroup ? j + 1 : kGroup - 1].x, 0);
      if (lane == 0) left = j > 0 ? prev_y : eleft;
      if (lane == 31) right = j + 1 < kGroup ? next_x : eright;
      V y;
      if constexpr (MODE == 0) {
        if (p2) {
          y.x = eq2_exact_pow2(left, x[j].x, x[j].y, a.p2_hi_add, a.p2_hi_xor);
          y.y = eq2_exact_pow2(x[j].x, x[j].y, right, a.p2_hi_add, a.p2_hi_xor);
        }
      }
      if (!p2) {
        y.x = E::upd(left, x[j].x, x[j].y, r, rf);
        y.y = E::upd(x[j].x, x[j].y, right, r, rf);
      }
      reinterpret_cast<V *>(dst + b0 + 64 * j)[lane] = y;
    }
  }
  // the rest point by point: [lo, tf*64), tiles after the groups, [tl*64, hi)
  const int64_t g0 = tf > tl ? hi : ((tf + ngroups * kGroup) << 6), g1 = tf > tl ? hi : (tl << 6);
  auto point = [&](int64_t g) {
    const T ul = g == lo ? gl : __ldcg(src + g - 1);
    const T ur = g == hi - 1 ? gr : __ldcg(src + g + 1);
    dst[g] = E::upd(ul, __ldcg(src + g), ur, r, rf);
  };
  const int64_t head_end = tf > tl ? hi : (tf << 6);
  for (int64_t g = lo + threadIdx.x; g < head_end; g += blockDim.x) point(g);
  for (int64_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) point(g);
  if (tf <= tl)
    for (int64_t g = (tl << 6) + threadIdx.x; g < hi; g += blockDim.x) point(g);
}

template <int MODE>
__global__ void __launch_bounds__(kPersistThreads) k_persist(PersistArgs a) {
  using T = typename Elem<MODE>::T;
  __shared__ T ghost[2];
  __shared__ int stop;
  const T *src = (const T *)a.ua;
  T *dst = (T *)a.ub;
  const int S = a.S;

  // publish the time-0 edge values of every owned segment
  if (threadIdx.x == 0) {
    for (int i = blockIdx.x; i < S; i += gridDim.x) {
      if (i == a.inj_seg && a.inj_step <= 0) continue;
      const int left = i == 0 ? S - 1 : i - 1, right = i == S - 1 ? 0 : i + 1;
      a.mb[2 * left + 1].val[0][0] = (double)__ldcg(src + a.seg[i]);
      a.mb[2 * right].val[0][0] = (double)__ldcg(src + a.seg[i + 1] - 1);
      __threadfence();
      st_release(&a.mb[2 * left + 1].seq, 1ull);
      st_release(&a.mb[2 * right].seq, 1ull);
    }
  }

  for (long long s = 0; s < a.nt; ++s) {
    for (int i = blockIdx.x; i < S; i += gridDim.x) {
      const int64_t lo = a.seg[i], hi = a.seg[i + 1];
      if (threadIdx.x == 0) {
        const bool ok = wait_seq(a, &a.mb[2 * i].seq, (unsigned long long)s + 1, i, s) &&
                        wait_seq(a, &a.mb[2 * i + 1].seq, (unsigned long long)s + 1, i, s);
        if (ok) {
          ghost[0] = (T)(*(volatile double *)&a.mb[2 * i].val[s & 1][0]);
          ghost[1] = (T)(*(volatile double *)&a.mb[2 * i + 1].val[s & 1][0]);
        }
        stop = ok ? 0 : 1;
      }
      __syncthreads();
      if (stop) return;  // uniform across the CTA
      step_segment<MODE>(src, dst, lo, hi, ghost[0], ghost[1], a.r, a.rf, a);
      __syncthreads();
      if (threadIdx.x == 0 && !(i == a.inj_seg && s + 1 >= a.inj_step)) {
        const int left = i == 0 ? S - 1 : i - 1, right = i == S - 1 ? 0 : i + 1;
        const int slot = (int)((s + 1) & 1);
        a.mb[2 * left + 1].val[slot][0] = (double)__ldcg(dst + lo);
        a.mb[2 * right].val[slot][0] = (double)__ldcg(dst + hi - 1);
        __threadfence();
        st_release(&a.mb[2 * left + 1].seq, (unsigned long long)s + 2);
        st_release(&a.mb[2 * right].seq, (unsigned long long)s + 2);
      }
    }
    const T *t = src;
    src = dst;
    dst = (T *)t;
  }
}

template <int MODE>
int launch(heat_ctx *c, PersistArgs &a, int grid) {
  void *params[] = {&a};
  const cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_persist<MODE>, dim3(grid), dim3(kPersistThreads),
                                                    params, 0, c->stream);
  return e == cudaSuccess ? HEAT_OK : HEAT_ECUDA;
}

template <int MODE>
int max_resident(heat_ctx *c) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist<MODE>, kPersistThreads, 0) != cudaSuccess)
    return 0;
  return per_sm * c->sms;
}

}  // namespace

// Builds the segment table (S+1 boundaries) on the host and uploads it; makes
// sure the mailbox area holds 2*S mailboxes.
int prepare_segments(heat_ctx *c, int S, const int64_t *bounds) {
  if (S > c->mbox_segments) {
    if (c->mbox) cudaFree(c->mbox);
    if (c->seg_start) cudaFree(c->seg_start);
    c->mbox = nullptr;
    c->seg_start = nullptr;
    c->mbox_segments = 0;
    if (cudaMalloc((void **)&c->mbox, sizeof(Mailbox) * 2 * (size_t)S) != cudaSuccess) return HEAT_ENOMEM;
    if (cudaMalloc((void **)&c->seg_start, sizeof(int64_t) * (size_t)(S + 1)) != cudaSuccess) return HEAT_ENOMEM;
    c->mbox_segments = S;
  }
  if (cudaMemcpyAsync(c->seg_start, bounds, sizeof(int64_t) * (size_t)(S + 1), cudaMemcpyHostToDevice, c->stream) !=
      cudaSuccess)
    return HEAT_ECUDA;
  // fresh sequence numbers for this run (the kernel republishes time-0 edges)
  if (cudaMemsetAsync(c->mbox, 0, sizeof(Mailbox) * 2 * (size_t)S, c->stream) != cudaSuccess) return HEAT_ECUDA;
  // the bounds array is a host temporary: make the copy complete before returning
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? HEAT_OK : HEAT_ECUDA;
}

// Segment boundaries: one segment per partition when requested (and the
// partitions fit the co-resident CTAs), else `want` near-equal segments whose
// interior boundaries fall on 64-point tiles.
int segment_bounds(const heat_ctx *c, int want, int64_t **out) {
  const int64_t N = c->geo.N;
  int S;
  int64_t *b;
  if (c->segments < 0 && c->geo.np <= want) {
    S = c->geo.np;
    b = (int64_t *)malloc(sizeof(int64_t) * (size_t)(S + 1));
    if (!b) return -1;
    for (int i = 0; i <= S; ++i) b[i] = (int64_t)i * c->geo.nx;
  } else {
    if (c->segments > 0 && c->segments < want) want = c->segments;
    int64_t chunk = (N + want - 1) / want;
    chunk = (chunk + 63) / 64 * 64;
    S = (int)((N + chunk - 1) / chunk);
    b = (int64_t *)malloc(sizeof(int64_t) * (size_t)(S + 1));
    if (!b) return -1;
    for (int i = 0; i <= S; ++i) b[i] = (int64_t)i * chunk < N ? (int64_t)i * chunk : N;
  }
  *out = b;
  return S;
}

// Default depth of the flag-queue form: 32 for binary32; binary64 8 below 2^21
// points, where a segment holds few tiles per block (10^6 points, r = 1/4:
// 234.6 GLUP/s at 8, 209.3 at 4, 162.0 at 12), else 16 (2^25 points: 307.3 at
// 16, 302.7 at 12; deeper blocks leave the integer routines' domain at
// r = 0.3).
int persist_default_T(const heat_ctx *c) {
  if (c->dtype == HEAT_F32C) return 32;
  return c->geo.N < (1LL << 21) ? 8 : 16;
}

// Depth T >= 2 (the default): T-point messages, T steps per message
// (k_queue.cu); depth 1, or partitions shorter than the depth: one value per
// message and one step, below.
int run_persist(heat_ctx *c, int64_t nt) {
  const int T = c->T > 0 ? c->T : persist_default_T(c);
  if (T >= 2) {
    const int rc = run_queue(c, nt, T);
    if (rc != HEAT_ENOTSUP) return rc;
  }
  const int mode = c->dtype == HEAT_F32C ? 2 : (c->arith == HEAT_ARITH_FMA ? 1 : 0);
  const int resident = mode == 0 ? max_resident<0>(c) : mode == 1 ? max_resident<1>(c) : max_resident<2>(c);
  if (resident < 1) return HEAT_ECUDA;
  int64_t *bounds = nullptr;
  const int S = segment_bounds(c, resident, &bounds);
  if (S < 1) return HEAT_ENOMEM;
  int rc = prepare_segments(c, S, bounds);
  free(bounds);
  if (rc != HEAT_OK) return rc;
  PersistArgs a;
  a.ua = c->buf[c->cur];
  a.ub = c->buf[c->cur ^ 1];
  a.N = c->geo.N;
  a.r = c->r;
  a.rf = c->rf;
  a.nt = nt;
  a.seg = c->seg_start;
  a.S = S;
  a.mb = c->mbox;
  a.st = c->dstat;
  a.wait_ns = c->wait_ns;
  a.inj_seg = c->inj_segment;
  a.inj_step = c->inj_step;
  uint64_t rbits;
  memcpy(&rbits, &c->r, sizeof(rbits));
  const int rexp = (int)((rbits >> 52) & 2047);
  a.p2 = c->dtype == HEAT_F64 && c->arith == HEAT_ARITH_EXACT && rexp >= 1 && rexp <= 2046 &&
         (rbits & 0x000fffffffffffffull) == 0 && emul::domain_bounds(rbits, 1, a.dom_lo, a.dom_hi);
  a.p2_hi_add = (rexp - 1023) * (1 << 20);
  a.p2_hi_xor = (rbits >> 63) ? (int)0x80000000u : 0;
  const int grid = S < resident ? S : resident;
  rc = mode == 0 ? launch<0>(c, a, grid) : mode == 1 ? launch<1>(c, a, grid) : launch<2>(c, a, grid);
  if (rc != HEAT_OK) return rc;
  c->last_segments = S;
  c->last_launches = 1;
  if (nt & 1) c->cur ^= 1;
  c->steps += nt;
  return HEAT_OK;
}

}  // namespace heat

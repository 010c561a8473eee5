// wave_core.cuh -- one work unit of dependency-driven temporal blocking, shared
// by the single-ring kernel (k_wave.cu) and the batched-ring kernel
// (k_batch.cu).
//
// A ring of n points is cut into ntiles near-equal tiles of at most
// W = 32E - 2T points (ntiles = ceil(n / W)).  A unit advances tile j by up to
// T steps of Eq. 2 (Section 2): it reads the window [lo - T, hi + T) (modulo n)
// at the block's start time from one buffer and writes [lo, hi) at the later
// time into the other.  That window lies in tiles j-1, j, j+1 (modulo ntiles):
// with W >= 2T every tile holds at least T points once there are two tiles or
// more, and a single tile's window (n + 2T <= 32E points) wraps onto itself.
// So a unit at level b waits until those tiles' completion counters reach b
// (which also covers the write-after-read hazard on its output buffer, read by
// the same three tiles at level b-1) and publishes its own counter, b + 1,
// after its stores.
#pragma once

#include "tb_core.cuh"

namespace heat {
namespace wave {

constexpr long long kSpins = 1LL << 26;  // backstop if the timer never advances

// The integer-pipe routines' parameters for binary64 under the exact reading.
struct Engine {
  emul::MulX mx;
  int dom_lo, dom_hi;  // input screen for the block's depth (empty: dom_lo > dom_hi)
  int p2_hi_add, p2_hi_xor;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool aborted(const DevStatus *st) { return *(const volatile int *)&st->abort != 0; }

// Bounded wait (one thread) until *p >= target.  False when the deadline
// passed or the launch was aborted; the first waiter to give up records where
// (`where`, `level`) and raises the abort word so that every other wait ends.
static __device__ __noinline__ bool wait_counter(const unsigned *p, unsigned target, long long wait_ns, DevStatus *st,
                                          int where, long long level) {
  if (ld_acquire_u32(p) >= target) return true;
  const unsigned long long deadline = globaltimer_ns() + (unsigned long long)wait_ns;
  unsigned ns = 32;
  for (long long spin = 0; spin < kSpins; ++spin) {
    if (ld_acquire_u32(p) >= target) return true;
    if (aborted(st)) return false;
    if (globaltimer_ns() > deadline) break;
    __nanosleep(ns);
    if (ns < 512) ns <<= 1;
  }
  if (atomicCAS(&st->code, HEAT_OK, HEAT_ETIMEOUT) == HEAT_OK) {
    st->segment = where;
    st->step = level;
  }
  atomicExch(&st->abort, 1);
  return false;
}

// Wait until the counters of tiles j-1, j, j+1 of a ring reach `level`: lanes
// 0, 1, 2 each acquire one counter (three loads in flight at once), and a
// counter not yet there is waited for by its lane.  The warp barrier after the
// vote orders every lane's later loads after the three acquires.
__device__ __forceinline__ bool wait_neighbours(const unsigned *done, int64_t ntiles, int64_t j, unsigned level,
                                                long long wait_ns, DevStatus *st, int where, int lane) {
  bool ok = true;
  if (lane < 3) {
    const int64_t t = lane == 0 ? (j == 0 ? ntiles - 1 : j - 1) : lane == 1 ? j : (j + 1 == ntiles ? 0 : j + 1);
    ok = ld_acquire_u32(done + t) >= level || wait_counter(done + t, level, wait_ns, st, where, level);
  }
  const bool all = __all_sync(tb::kFull, ok);
  __syncwarp();
  return all;
}

// Tile j of ntiles near-equal tiles of a ring of n points: the first
// n mod ntiles tiles hold one point more.
__device__ __forceinline__ void tile_bounds(int64_t n, int64_t ntiles, int64_t j, int64_t &lo, int64_t &hi) {
  const int64_t q = n / ntiles, rem = n - q * ntiles;
  lo = j * q + (j < rem ? j : rem);
  hi = lo + q + (j < rem ? 1 : 0);
}

// Advance a window held in registers by `steps` (<= T) steps.  int_tile:
// binary64 under the exact reading, compute on the integer pipes when the
// window passes the screen; p2: for r = +-2^k the FP64-unit path moves the
// product's exponent when the window passes the screen.
template <int MODE, int EP>
__device__ __forceinline__ void advance_window(typename tb::TBCx<MODE, EP>::Reg &R, int steps, double r, float rf,
                                               bool int_tile, bool p2, const Engine &e, int lane) {
  using P = tb::TBCx<MODE, EP>;
  constexpr int E = P::E;
  bool dp = true;
  if constexpr (MODE == 0) {
    if (int_tile || p2) {
      bool okd = true;
#pragma unroll
      for (int k = 0; k < E; ++k)
        okd &= emul::in_domain((uint64_t)__double_as_longlong(P::store(R, k)), e.dom_lo, e.dom_hi);
      if (__all_sync(tb::kFull, okd)) {  // else the whole tile takes the plain FP64-unit steps
        if (!int_tile)
          for (int s = 0; s < steps; ++s) P::step_p2(R, e.p2_hi_add, e.p2_hi_xor);
        else if (e.mx.pow2 && !e.mx.neg)
          P::template steps_x<true, false>(R, steps, e.mx);
        else if (e.mx.pow2)
          P::template steps_x<true, true>(R, steps, e.mx);
        else if (!e.mx.neg)
          P::template steps_x<false, false>(R, steps, e.mx);
        else
          P::template steps_x<false, true>(R, steps, e.mx);
        dp = false;
      }
    }
  }
  if (dp)
    for (int s = 0; s < steps; ++s) P::step(R, lane, r, rf);
}

// Advance tile [lo, hi) of a ring of n points from src to dst by `steps`
// (<= T) steps (advance_window).  Window points past hi + T feed no stored
// output and are loaded as zeros.  Loads bypass L1, which may still hold lines
// of this buffer from two levels back.
template <int MODE, int EP>
__device__ __forceinline__ void advance_tile(const typename tb::TBCx<MODE, EP>::T *src,
                                             typename tb::TBCx<MODE, EP>::T *dst, int64_t n, int64_t lo, int64_t hi,
                                             int T, int steps, double r, float rf, bool int_tile, bool p2,
                                             const Engine &e, int lane) {
  using P = tb::TBCx<MODE, EP>;
  using V = typename P::T;
  constexpr int E = P::E;
  const int64_t ws = lo - T;
  const int64_t need = hi - lo + 2 * (int64_t)T;
  const bool inside = ws >= 0 && ws + need <= n;
  typename P::Reg R;
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const int idx = E * lane + k;
    V v = V(0);
    if (idx < need) {
      int64_t g = ws + idx;
      if (!inside) {
        g %= n;
        if (g < 0) g += n;
      }
      v = __ldcg(src + g);
    }
    P::load(R, k, v);
  }
  advance_window<MODE, EP>(R, steps, r, rf, int_tile, p2, e, lane);
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const int idx = E * lane + k;
    const int64_t g = ws + idx;
    if (idx >= T && g < hi) dst[g] = P::store(R, k);
  }
}

// Publish a tile's completion: the warp barrier orders every lane's stores
// before lane 0's release, and the release makes them visible to whichever
// warp acquires the counter.
__device__ __forceinline__ void publish(unsigned *p, unsigned value, int lane) {
  __syncwarp();
  if (lane == 0) st_release_u32(p, value);
}

}  // namespace wave
}  // namespace heat

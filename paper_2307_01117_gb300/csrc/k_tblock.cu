// k_tblock.cu -- form HEAT_FORM_TBLOCK: temporal blocking.  Each launch
// advances the ring by T steps of Eq. 2 (Section 2); the last launch of a run
// may advance fewer.  Ghost exchange between tiles is implicit: every tile reads
// a T-wide halo on each side at the launch's start time and recomputes it.
//
// Per warp: a window of WIN = 32*E consecutive points, W = WIN - 2T of which are
// its output.  The window is staged from HBM into shared memory by one 1D bulk
// TMA copy (cp.async.bulk, completion on an mbarrier), double-buffered so the
// next tile's copy is in flight while this one is computed.  Lane l then holds
// window points 32k + l (k = 0..E-1) in registers; one step needs, per point,
// the left and right neighbours, which come from lanes l-1 and l+1 by shuffle
// (lane 0 takes lane 31's value of register k-1, lane 31 takes lane 0's value of
// register k+1).  After s steps the points s .. WIN-1-s of the window are exact;
// after T steps the middle W points are stored.  Tiles whose window wraps
// around the ring's ends are loaded with plain indexed loads instead of TMA.
//
// Binary32 compensated state: registers carry (h, l) pairs; the block's T steps
// are one compensation block, stored as RN(h + l) (the library's HEAT_F32C
// definition).
//
// Binary64, exact reading: a share of the tiles (chosen by a 32-bit mask over
// tile index mod 32) is computed with the integer-pipe binary64 routines of
// dp_emul.cuh instead of the FP64 unit; both give the correctly rounded IEEE
// result, so the bits do not depend on the share.  Strided layout: if any point
// of an emulated tile leaves the routines' domain, the warp recomputes that
// tile on the FP64 unit from its staged window.  Contiguous layout: the tile's
// values are screened first (zero, or normal within bounds that keep every
// intermediate of the T steps normal) and advanced in the unpacked form; a
// tile that fails the screen runs on the FP64 unit.
//
// Algorithmic HBM traffic per launch: N points read + N written (16 B per point
// per T steps in binary64, 8 B in binary32); the halo re-read adds WIN/W.
#include <string.h>

#include "tb_core.cuh"

namespace heat {
namespace {

constexpr int kWarps = 4;  // warps per CTA
constexpr long long kMaxWaitSpins = 1LL << 24;
using namespace tb;

struct TBArgs {
  const void *src;
  void *dst;
  int64_t N;
  double r;
  float rf;
  int T;        // halo width (the block depth)
  int steps;    // steps this launch (<= T)
  int64_t ntiles;
  DevStatus *st;
  unsigned emul_mask;  // bit (tile mod 32) set: compute the tile on the integer pipes
  unsigned long long *tile_counter;  // [0] launch-wide tile counter (zero at launch), [1] finished CTAs
  int split;           // other tiles: multiply (and masked final adds) on the integer pipes
  unsigned add_mask;   // registers k whose final add also goes to the integer pipes
  emul::Mul m;         // prepared multiplier r (valid when emul_mask != 0)
  emul::MulX mx;       // the same for the unpacked form (contiguous layout)
  int dom_lo, dom_hi;  // unpacked form: input screen for T steps (biased exponents)
  int p2_fp64;         // r = +-2^k: screened FP64-unit tiles multiply on the integer pipes
  int dual;            // two-ended claiming instead of emul_mask (see k_tblock_c)
  int p2_hi_add, p2_hi_xor;
};

template <int MODE>
__global__ void __launch_bounds__(kWarps * 32) k_tblock(TBArgs a) {
  using P = TB<MODE>;
  using T = typename P::T;
  constexpr int E = P::E;
  constexpr int WIN = 32 * E;
  constexpr int BUF = WIN + P::kAlign;  // elements per staging buffer
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  T *buf0 = reinterpret_cast<T *>(smem_raw) + (size_t)wib * 2 * BUF;
  __shared__ unsigned long long bars[kWarps][2];
  unsigned long long *bar = bars[wib];

  const T *src = (const T *)a.src;
  T *dst = (T *)a.dst;
  const int64_t N = a.N;
  const int W = WIN - 2 * a.T;

  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_proxy_async();
  }
  __syncwarp();

  // A tile is staged by TMA when its window [ws, ws + WIN) lies inside the ring
  // (no wrap); the copy starts at ws rounded down to 16 bytes.
  auto window_start = [&](int64_t tile) -> int64_t { return tile * (int64_t)W - a.T; };
  auto tma_ok = [&](int64_t ws) -> bool { return ws >= 0 && ws + WIN + P::kAlign <= N; };
  auto issue = [&](int64_t tile, int b) {
    const int64_t ws = window_start(tile);
    if (!tma_ok(ws)) return;
    const int64_t ws_al = ws & ~(int64_t)(P::kAlign - 1);
    if (lane == 0) {
      fence_proxy_async();
      mbar_expect_tx(&bar[b], (unsigned)(BUF * sizeof(T)));
      bulk_load(buf0 + b * BUF, src + ws_al, (unsigned)(BUF * sizeof(T)), &bar[b]);
    }
  };

  unsigned phase0 = 0u, phase1 = 0u;  // mbarrier phase parity per staging buffer
  int b = 0;
  // Tiles are claimed dynamically from a launch-wide counter, zeroed before the
  // launch (one atomic per tile, by lane 0), so warps that draw slower tiles do
  // not hold up the rest.
  auto claim = [&]() -> int64_t {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(a.tile_counter, 1ull);
    return (int64_t)__shfl_sync(kFull, t, 0);
  };
  int64_t tile = claim();
  if (tile < a.ntiles) issue(tile, 0);
  for (; tile < a.ntiles;) {
    const int64_t next = claim();
    __syncwarp();
    if (next < a.ntiles) issue(next, b ^ 1);
    const int64_t ws = window_start(tile);
    typename P::Reg R;
    const bool staged = tma_ok(ws);
    if (staged) {
      // every lane observes the barrier; the loop exits for the whole warp at once
      bool done = false;
      for (long long spin = 0; spin < kMaxWaitSpins && !done; ++spin)
        done = __all_sync(kFull, mbar_try_wait(&bar[b], b ? phase1 : phase0));
      if (!done) {  // the copy did not complete: record and stop this warp
        if (lane == 0 && atomicCAS(&a.st->code, HEAT_OK, HEAT_ETIMEOUT) == HEAT_OK) {
          a.st->segment = -1;
          a.st->step = tile;
        }
        return;
      }
      if (b) phase1 ^= 1u; else phase0 ^= 1u;
    }
    const T *sb = buf0 + b * BUF + (int)(ws - (ws & ~(int64_t)(P::kAlign - 1)));
    auto load_window = [&]() {
      if (staged) {
#pragma unroll
        for (int k = 0; k < E; ++k) P::load(R, k, sb[32 * k + lane]);
      } else {
#pragma unroll
        for (int k = 0; k < E; ++k) {
          int64_t g = (ws + 32 * k + lane) % N;
          if (g < 0) g += N;
          P::load(R, k, src[g]);
        }
      }
    };
    load_window();
    bool dp = true;
    if constexpr (HasEmul<MODE>::value) {
      if ((a.emul_mask >> (unsigned)(tile & 31)) & 1u) {
        bool bad = false;
        for (int s = 0; s < a.steps; ++s) P::step_emul(R, lane, a.m, bad);
        dp = __any_sync(kFull, bad);
        if (dp) load_window();  // some point left the routines' domain: redo on the FP64 unit
      } else if (a.split) {
        bool bad = false;
        for (int s = 0; s < a.steps; ++s) P::step_split(R, lane, a.m, a.add_mask, bad);
        dp = __any_sync(kFull, bad);
        if (dp) load_window();
      }
    }
    if (dp)
      for (int s = 0; s < a.steps; ++s) P::step(R, lane, a.r, a.rf);
    // store the W exact points of the window: indices T .. WIN-1-T
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int i = 32 * k + lane;
      const int64_t g = ws + i;
      if (i >= a.T && i < WIN - a.T && g < N) dst[g] = P::store(R, k);
    }
    b ^= 1;
    tile = next;
  }
}

// Contiguous-ownership variant (lane l holds window points E*l .. E*l + E - 1):
// two shuffles per carried value per lane and step instead of two per point.
// Windows are loaded and stored with plain indexed accesses (wrapping around the
// ring's ends where needed); tiles are claimed from the same launch-wide counter.
template <int MODE, int EP>
__global__ void __launch_bounds__(kWarps * 32, MODE == 2 ? 1 : 8) k_tblock_c(TBArgs a) {
  using P = TBCx<MODE, EP>;
  using T = typename P::T;
  constexpr int E = P::E;
  constexpr int WIN = 32 * E;
  const int lane = threadIdx.x & 31;
  const T *src = (const T *)a.src;
  T *dst = (T *)a.dst;
  const int64_t N = a.N;
  const int W = WIN - 2 * a.T;
  // Two-ended claiming (binary64, a.dual): integer-pipe warps take tiles from
  // the end of the range and FP64-unit warps from the start, through one 64-bit
  // counter (low half: tiles taken from the start, high half: from the end), so
  // the split between the engines follows their speeds and both finish
  // together.  Warp kinds alternate with CTA and warp index, which puts both
  // kinds on every SM sub-partition.
  const bool int_warp = MODE == 0 && a.dual && (((blockIdx.x ^ (threadIdx.x >> 5)) & 1) != 0);
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(a.tile_counter, int_warp ? (1ull << 32) : 1ull);
    t = __shfl_sync(kFull, t, 0);
    int64_t tile;
    bool int_tile;
    if (MODE == 0 && a.dual) {
      const int64_t f = (int64_t)(t & 0xffffffffull), b = (int64_t)(t >> 32);
      if (f + b >= a.ntiles) break;
      tile = int_warp ? a.ntiles - 1 - b : f;
      int_tile = int_warp;
    } else {
      tile = (int64_t)t;
      if (tile >= a.ntiles) break;
      int_tile = MODE == 0 && ((a.emul_mask >> (unsigned)(tile & 31)) & 1u);
    }
    const int64_t ws = tile * (int64_t)W - a.T;
    const int64_t base = ws + (int64_t)E * lane;
    typename P::Reg R;
    if (ws >= 0 && ws + WIN <= N) {
#pragma unroll
      for (int k = 0; k < E; ++k) P::load(R, k, src[base + k]);
    } else {
#pragma unroll
      for (int k = 0; k < E; ++k) {
        int64_t g = (base + k) % N;
        if (g < 0) g += N;
        P::load(R, k, src[g]);
      }
    }
    bool dp = true;
    if constexpr (MODE == 0) {
      if (int_tile || a.p2_fp64) {
        bool ok = true;
#pragma unroll
        for (int k = 0; k < E; ++k)
          ok &= emul::in_domain((uint64_t)__double_as_longlong(P::store(R, k)), a.dom_lo, a.dom_hi);
        if (__all_sync(kFull, ok)) {  // else the whole tile takes the plain FP64-unit steps
          if (!int_tile)
            for (int s = 0; s < a.steps; ++s) P::step_p2(R, a.p2_hi_add, a.p2_hi_xor);
          else if (a.mx.pow2 && !a.mx.neg)
            P::template steps_x<true, false>(R, a.steps, a.mx);
          else if (a.mx.pow2)
            P::template steps_x<true, true>(R, a.steps, a.mx);
          else if (!a.mx.neg)
            P::template steps_x<false, false>(R, a.steps, a.mx);
          else
            P::template steps_x<false, true>(R, a.steps, a.mx);
          dp = false;
        }
      }
    }
    if (dp)
      for (int s = 0; s < a.steps; ++s) P::step(R, lane, a.r, a.rf);
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int i = E * lane + k;
      const int64_t g = ws + i;
      if (i >= a.T && i < WIN - a.T && g < N) dst[g] = P::store(R, k);
    }
  }
  // The last CTA to finish returns both counters to zero for the next launch
  // on the stream, so launches need no reset operation between them (on small
  // rings the launch sequence is the cost).  Every warp has made its last claim
  // before its CTA passes the barrier.
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(a.tile_counter + 1, 1ull) == (unsigned long long)gridDim.x - 1) {
      atomicExch(a.tile_counter, 0ull);
      atomicExch(a.tile_counter + 1, 0ull);
    }
  }
}

template <int MODE, int EP>
int launch_tb_c_ep(heat_ctx *c, TBArgs a) {
  const int W = 32 * EP - 2 * a.T;
  a.ntiles = (c->geo.N + W - 1) / W;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tblock_c<MODE, EP>, kWarps * 32, 0) != cudaSuccess ||
      per_sm < 1)
    return HEAT_ECUDA;
  int64_t grid = (a.ntiles + kWarps - 1) / kWarps;
  const int64_t cap = (int64_t)per_sm * c->sms;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  // zero after the previous launch (k_tblock_c resets them itself), unless a
  // strided launch ran since
  if (c->counter_dirty) {
    if (cudaMemsetAsync(c->tile_counter, 0, 2 * sizeof(unsigned long long), c->stream) != cudaSuccess)
      return HEAT_ECUDA;
    c->counter_dirty = 0;
  }
  k_tblock_c<MODE, EP><<<(int)grid, kWarps * 32, 0, c->stream>>>(a);
  return cuda_status(cudaGetLastError());
}

// Window width for the contiguous layout: the widest window (least halo
// recomputation) that still gives every SM sub-partition about 16 windows per
// launch; medium rings get narrower windows so enough warps keep the FP64 unit
// busy.  A window must leave at least 2T points of output.
template <int MODE>
int launch_tb_c(heat_ctx *c, const TBArgs &a) {
  constexpr int eps[3] = {MODE == 2 ? 8 : 4, MODE == 2 ? 16 : 8, MODE == 2 ? 32 : 16};
  const int64_t want = 16LL * 4 * c->sms;
  int pick = 2;
  while (pick > 0) {
    const int64_t w = 32LL * eps[pick] - 2 * a.T;
    if (c->geo.N / w >= want) break;
    const int64_t w_next = 32LL * eps[pick - 1] - 2 * a.T;
    if (w_next < 2 * a.T) break;  // the narrower window would be mostly halo
    --pick;
  }
  switch (pick) {
    case 0: return launch_tb_c_ep<MODE, eps[0]>(c, a);
    case 1: return launch_tb_c_ep<MODE, eps[1]>(c, a);
    default: return launch_tb_c_ep<MODE, eps[2]>(c, a);
  }
}

template <int MODE>
size_t smem_bytes() {
  using P = TB<MODE>;
  return (size_t)kWarps * 2 * (32 * P::E + P::kAlign) * sizeof(typename P::T);
}

template <int MODE>
int launch_tb(heat_ctx *c, const void *src, void *dst, int T, int steps) {
  using P = TB<MODE>;
  const int WIN = 32 * P::E;
  const int W = WIN - 2 * T;
  TBArgs a;
  a.src = src;
  a.dst = dst;
  a.N = c->geo.N;
  a.r = c->r;
  a.rf = c->rf;
  a.T = T;
  a.steps = steps;
  a.ntiles = (c->geo.N + W - 1) / W;
  a.st = c->dstat;
  uint64_t rbits;
  memcpy(&rbits, &c->r, sizeof(rbits));
  const int rexp = (int)((rbits >> 52) & 2047);
  // the routines take a normal, nonzero multiplier; otherwise every tile uses the FP64 unit
  a.emul_mask = (MODE == 0 && rexp >= 1 && rexp <= 2046) ? tblock_emul_mask(c) : 0u;
  a.m = emul::prepare_mul(rbits);
  a.mx = emul::prepare_mulx(rbits);
  // the contiguous layout's unpacked tiles need a nonempty input screen for T steps
  const bool dom = emul::domain_bounds(rbits, T, a.dom_lo, a.dom_hi);
  if (!dom && c->tb_layout == 1) a.emul_mask = 0u;
  // r = +-2^k, exact reading: the FP64-unit tiles that pass the same screen move
  // the product's exponent with an integer add (3 FP64-unit operations per point)
  a.p2_fp64 = MODE == 0 && dom && a.mx.pow2 && c->tb_layout == 1;
  // the library's choice of share: adaptive, by claiming from both ends
  a.dual = MODE == 0 && c->emul_auto && a.emul_mask != 0u && c->tb_layout == 1;
  a.p2_hi_add = (int)(((int64_t)rexp - 1023) * (1 << 20));
  a.p2_hi_xor = (rbits >> 63) ? (int)0x80000000u : 0;
  a.tile_counter = c->tile_counter;
  // split_level 0: every FP64-unit tile keeps 4 FP64 operations per point;
  // 1: the multiply goes to the integer pipes (3 per point); 1 + j (j = 1..16):
  // the final add too, for j of the 16 registers spread evenly (those points
  // need 2 FP64 operations)
  a.split = MODE == 0 && rexp >= 1 && rexp <= 2046 && c->split_level > 0;
  const int j = c->split_level > 1 ? c->split_level - 1 : 0;
  a.add_mask = 0u;
  for (int i = 0; i < 16; ++i)
    if (((i + 1) * j) / 16 > (i * j) / 16) a.add_mask |= 1u << i;
  const size_t smem = smem_bytes<MODE>();
  if (c->tb_layout == 1) return launch_tb_c<MODE>(c, a);
  if (cudaFuncSetAttribute(k_tblock<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return HEAT_ECUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tblock<MODE>, kWarps * 32, smem) != cudaSuccess ||
      per_sm < 1)
    return HEAT_ECUDA;
  int64_t grid = (a.ntiles + kWarps - 1) / kWarps;
  const int64_t cap = (int64_t)per_sm * c->sms;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  if (cudaMemsetAsync(c->tile_counter, 0, sizeof(unsigned long long), c->stream) != cudaSuccess) return HEAT_ECUDA;
  c->counter_dirty = 1;
  k_tblock<MODE><<<(int)grid, kWarps * 32, smem, c->stream>>>(a);
  return cuda_status(cudaGetLastError());
}

}  // namespace

int tblock_window(int dtype) { return dtype == HEAT_F32C ? 32 * TB<2>::E : 32 * TB<0>::E; }

// Integer tiles under the library's choice: for binary64 rings under the
// exact reading in the contiguous layout of at least 2^18 points; a nonzero
// mask here switches the launch to the adaptive two-ended split (a.dual), the
// mask's own share (emul_auto_share) only standing for "on".  Measured with
// the split against every tile on the FP64 unit at T = 8: +14 % at 2^18
// points, +83 % at 10^6; smaller rings finish in a few waves of tiles, where
// the slower integer tiles lengthen the last one (-28 % at 2^16).
unsigned tblock_emul_mask(const heat_ctx *c) {
  if (!c->emul_auto) return c->emul_mask;
  if (c->dtype != HEAT_F64 || c->arith != HEAT_ARITH_EXACT || c->tb_layout != 1) return 0u;
  if (c->geo.N < (1LL << 18)) return 0u;
  return emul_share_mask(emul_auto_share(c->r));
}

// Default depth: binary32 pairs 32 steps per pass.  Binary64: 24 on rings
// below 2^19 points, where the launch sequence is the cost (0.67 us per step
// against 0.82 at T = 12 and 1.24 at T = 8 from 4000 to 31000 points; +8 % at
// 2^18); 12 with integer tiles (they unpack and pack once per pass: +13 % over
// 8 at 10^6 points, +1.3 % at 2^28); else 8, except 4 on rings of at least
// 2^22 points (the halo's redundant work then costs more than it saves: 129.1
// vs 127.4 GLUP/s at 2^28 points).
int tblock_default_T(const heat_ctx *c) {
  if (c->dtype == HEAT_F32C) return 32;
  const bool int_tiles = tblock_emul_mask(c) != 0u;
  uint64_t rb;
  memcpy(&rb, &c->r, sizeof(rb));
  // a general r's screen admits ordinary data only for shallow blocks: keep
  // the integer tiles at 12 rather than lose them at 24
  if (c->geo.N < (1LL << 19) && !(int_tiles && (rb & 0x000fffffffffffffull) != 0)) return 24;
  if (int_tiles) return 12;
  return c->geo.N < (1LL << 22) ? 8 : 4;
}

int run_tblock(heat_ctx *c, int64_t nt) {
  const int mode = c->dtype == HEAT_F32C ? 2 : (c->arith == HEAT_ARITH_FMA ? 1 : 0);
  int T = c->T > 0 ? c->T : tblock_default_T(c);
  const int WIN = tblock_window(c->dtype);
  if (2 * T >= WIN) return HEAT_EINVAL;
  c->last_T = T;
  for (int64_t done = 0; done < nt;) {
    const int steps = (int)(nt - done < T ? nt - done : T);
    const void *src = c->buf[c->cur];
    void *dst = c->buf[c->cur ^ 1];
    const int rc = mode == 0 ? launch_tb<0>(c, src, dst, T, steps)
                   : mode == 1 ? launch_tb<1>(c, src, dst, T, steps)
                               : launch_tb<2>(c, src, dst, T, steps);
    if (rc != HEAT_OK) return rc;
    c->cur ^= 1;
    c->steps += steps;
    c->last_launches += 1;
    done += steps;
  }
  return HEAT_OK;
}

}  // namespace heat

// k_wave.cu -- form HEAT_FORM_PERSIST_TB for a single ring: temporal blocking
// driven by neighbour dependencies instead of launch boundaries.  One launch
// advances all nt steps.
//
// The ring is cut into ntiles near-equal tiles of at most W = 32E - 2T points
// each.  A work unit is (level b, tile i): advance tile i from time bT to
// bT + steps_b with the register-resident temporal-blocking core, reading its
// window with T-point halos at time bT from one buffer and writing the tile at
// the later time into the other (wave_core.cuh).  The window lies in tiles
// i-1, i, i+1, so unit (b, i) waits until those three tiles have finished
// level b-1 -- Section 2's segmented algorithm, each segment advancing as soon
// as its neighbours' ghost zones (here T points deep) are ready, with a
// per-tile completion counter as the queue.  The same wait covers the
// write-after-read hazard: level b writes the buffer that level b-1's
// neighbours read.
//
// Units are numbered level-major and claimed by whole warps from one
// launch-wide counter in increasing order, so every unit a warp waits for has a
// smaller number and was claimed earlier by a warp that is running it; the warp
// holding the smallest unfinished unit never waits on anything unfinished, and
// the launch makes progress with any number of resident CTAs (an ordinary
// launch, no co-residency).  Unlike one launch per level, a warp that finishes
// early goes on to the next level's tiles whose neighbours are done, so no
// level waits for the slowest tile of the ring.
//
// Binary64, exact reading, library's split: half of the warps compute their
// tiles with the integer-pipe binary64 routines (dp_emul.cuh), the others on
// the FP64 unit; both claim from the same counter, so each engine takes units
// at its own speed.  Every point is computed from the same operands as in the
// other forms, so the state is bitwise the oracle's.
//
// Every wait is bounded (iteration cap and %globaltimer deadline); one that runs
// out records HEAT_ETIMEOUT, raises the abort word and every warp returns.
#include <string.h>

#include "wave_core.cuh"

namespace heat {
namespace {

constexpr int kWaveWarps = 4;  // warps per CTA
// window chooser: tiles per level per SM the widest window must still give
constexpr int kWaveTilesPerLevelPerSM = 24;
// resident warps per tile of a level, in percent: on mid-size rings a unit's
// latency chains the levels (every warp holds a distinct part of the ring), so
// fewer, faster warps on wider windows beat a full SM on narrow ones (10^6
// points, T = 12: 6 CTAs per SM on 256-point windows 295.6 GLUP/s, 9 CTAs per
// SM on 128-point windows at T = 8 281.3)
constexpr int kWaveWarpsPerTilePct = 85;

struct WaveArgs {
  void *buf0, *buf1;
  int cur;             // buffer holding the state at time 0
  int64_t N;
  int64_t ntiles;
  int T;
  int64_t nt;
  int64_t units;       // levels * ntiles
  double r;
  float rf;
  unsigned *done;      // per tile: levels finished in this launch (zero at launch)
  unsigned long long *counter;  // unit counter (zero at launch)
  DevStatus *st;
  long long wait_ns;
  int dual;            // binary64, library's split: integer-pipe warps and FP64-unit warps
  unsigned emul_mask;  // otherwise: bit (tile mod 32) set -> that tile on the integer pipes
  int p2_fp64;         // r = +-2^k: screened FP64-unit tiles move the product's exponent
  wave::Engine eng;
  long long inj_tile;  // test hook: this tile stops publishing from level inj_level on (-1: none)
  long long inj_level;
};

template <int MODE, int EP>
__global__ void __launch_bounds__(kWaveWarps * 32, MODE == 2 ? 1 : 8) k_wave(WaveArgs a) {
  using T = typename tb::TBCx<MODE, EP>::T;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int64_t nt_ = a.ntiles;
  const bool int_warp = MODE == 0 && a.dual && (((blockIdx.x ^ wib) & 1) != 0);
  // One unit claimed at a time: a unit claimed ahead would wait behind its
  // warp's current one, and on mid-size rings (a level not much larger than
  // the resident warps) its neighbours at the next level would wait with it
  // (10^6 points: 262 vs 281 GLUP/s).
  for (;;) {
    unsigned long long u = 0;
    int go = 1;
    if (lane == 0) {
      u = atomicAdd(a.counter, 1ull);
      go = (int64_t)u < a.units && !wave::aborted(a.st);
    }
    u = __shfl_sync(tb::kFull, u, 0);
    if (!__shfl_sync(tb::kFull, go, 0)) break;
    const int64_t b = (int64_t)u / nt_, i = (int64_t)u - b * nt_;
    if (b > 0 && !wave::wait_neighbours(a.done, nt_, i, (unsigned)b, a.wait_ns, a.st, (int)i, lane)) break;
    int64_t lo, hi;
    wave::tile_bounds(a.N, nt_, i, lo, hi);
    const int par = (a.cur ^ (int)(b & 1)) & 1;
    const T *src = (const T *)(par ? a.buf1 : a.buf0);
    T *dst = (T *)(par ? a.buf0 : a.buf1);
    const int64_t left = a.nt - b * a.T;
    const int steps = (int)(left < a.T ? left : a.T);
    const bool int_tile = MODE == 0 && (a.dual ? int_warp : ((a.emul_mask >> (unsigned)(i & 31)) & 1u) != 0);
    wave::advance_tile<MODE, EP>(src, dst, a.N, lo, hi, a.T, steps, a.r, a.rf, int_tile, a.p2_fp64 != 0, a.eng,
                                 lane);
    if (!(i == a.inj_tile && b >= a.inj_level)) wave::publish(a.done + i, (unsigned)(b + 1), lane);
  }
}

template <int MODE, int EP>
int launch_wave_ep(heat_ctx *c, WaveArgs a) {
  const int W = 32 * EP - 2 * a.T;
  a.ntiles = (c->geo.N + W - 1) / W;
  const int64_t levels = (a.nt + a.T - 1) / a.T;
  a.units = levels * a.ntiles;
  if (a.ntiles > c->wave_cap) {
    if (c->wave_done) cudaFree(c->wave_done);
    c->wave_done = nullptr;
    c->wave_cap = 0;
    if (cudaMalloc((void **)&c->wave_done, (size_t)a.ntiles * sizeof(unsigned)) != cudaSuccess) return HEAT_ENOMEM;
    c->wave_cap = a.ntiles;
  }
  a.done = c->wave_done;
  a.counter = c->wave_counter;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wave<MODE, EP>, kWaveWarps * 32, 0) != cudaSuccess ||
      per_sm < 1)
    return HEAT_ECUDA;
  // CTAs per SM: as many as fit, or the nearest count giving about
  // kWaveWarpsPerTilePct warps per 100 tiles of a level when that is fewer
  const int64_t per_sm_cap = (a.ntiles * kWaveWarpsPerTilePct / 100 + (int64_t)kWaveWarps * c->sms / 2) /
                             ((int64_t)kWaveWarps * c->sms);
  if (per_sm_cap >= 1 && per_sm_cap < per_sm) per_sm = (int)per_sm_cap;
  int64_t grid = (a.units + kWaveWarps - 1) / kWaveWarps;
  const int64_t cap = (int64_t)per_sm * c->sms;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  if (cudaMemsetAsync(a.done, 0, (size_t)a.ntiles * sizeof(unsigned), c->stream) != cudaSuccess ||
      cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), c->stream) != cudaSuccess)
    return HEAT_ECUDA;
  k_wave<MODE, EP><<<(int)grid, kWaveWarps * 32, 0, c->stream>>>(a);
  c->last_segments = (int)a.ntiles;
  return cuda_status(cudaGetLastError());
}

// Window width: the widest window (least halo recomputation) that still gives
// kWaveTilesPerLevelPerSM tiles per level per SM, and W >= 2T.
template <int MODE>
int launch_wave(heat_ctx *c, const WaveArgs &a) {
  constexpr int eps[3] = {MODE == 2 ? 8 : 4, MODE == 2 ? 16 : 8, MODE == 2 ? 32 : 16};
  const int64_t want = (int64_t)kWaveTilesPerLevelPerSM * c->sms;
  int pick = 2;
  while (pick > 0) {
    const int64_t w = 32LL * eps[pick] - 2 * a.T;
    if (c->geo.N / w >= want) break;
    const int64_t w_next = 32LL * eps[pick - 1] - 2 * a.T;
    if (w_next < 2 * a.T) break;
    --pick;
  }
  if (32LL * eps[pick] - 2 * a.T < 2 * a.T) return HEAT_EINVAL;  // T beyond the widest window
  switch (pick) {
    case 0: return launch_wave_ep<MODE, eps[0]>(c, a);
    case 1: return launch_wave_ep<MODE, eps[1]>(c, a);
    default: return launch_wave_ep<MODE, eps[2]>(c, a);
  }
}

}  // namespace

// Allocated on first use, freed with the context.
int wave_alloc(heat_ctx *c) {
  if (c->wave_counter) return HEAT_OK;
  return cudaMalloc((void **)&c->wave_counter, sizeof(unsigned long long)) == cudaSuccess ? HEAT_OK : HEAT_ENOMEM;
}

void free_wave(heat_ctx *c) {
  if (c->wave_done) cudaFree(c->wave_done);
  if (c->wave_counter) cudaFree(c->wave_counter);
  c->wave_done = nullptr;
  c->wave_counter = nullptr;
  c->wave_cap = 0;
}

// Default depth: binary32 pairs 32 steps per pass.  Binary64: 16 below 2^19
// points, where the chain of levels (each waits on the one before) is the
// bound and fewer levels pay more than the narrower tiles' halo costs (2^18
// points, r = 1/4: 222.5 GLUP/s at 16, 214.2 at 12, 201.0 at 8); 12 from 2^19
// to 2^21 (10^6 points: 295.6 at 12, 295.3 at 10, 292.9 at 16, 280.7 at 8;
// r = 0.3: 224.2, 217.8, 224.3, 185.1); 16 above (2^22 points: 316.8 at 16,
// 309.5 at 12).
int wave_default_T(const heat_ctx *c) {
  if (c->dtype == HEAT_F32C) return 32;
  if (c->geo.N < (1LL << 19)) return 16;
  return c->geo.N < (1LL << 21) ? 12 : 16;
}

// HEAT_FORM_AUTO takes this form for binary64 rings under the exact reading
// from 2^18 to 2^26 points, where it measured faster than one launch per block
// (r = 1/4 / r = 0.3, GLUP/s: 2^18 points 171.8 vs 161.4 / 131.2 vs 119.3;
// 10^6 points 281.4 vs 236.2 / 218.8 vs 190.7; 2^24 points 326.2 vs 309.8 /
// 259.8 vs 241.9); from 2^26 points the per-launch form stays ahead (2^28:
// 334.8 vs 327.9 / 263.8 vs 260.8).
bool wave_preferred(const heat_ctx *c) {
  return c->dtype == HEAT_F64 && c->arith == HEAT_ARITH_EXACT && c->geo.N >= (1LL << 18) && c->geo.N < (1LL << 26);
}

// One launch for all nt steps.
int run_wave(heat_ctx *c, int64_t nt, int T) {
  const int mode = c->dtype == HEAT_F32C ? 2 : (c->arith == HEAT_ARITH_FMA ? 1 : 0);
  int rc = wave_alloc(c);
  if (rc != HEAT_OK) return rc;
  WaveArgs a;
  memset(&a, 0, sizeof(a));
  a.buf0 = c->buf[0];
  a.buf1 = c->buf[1];
  a.cur = c->cur;
  a.N = c->geo.N;
  a.T = T;
  a.nt = nt;
  a.r = c->r;
  a.rf = c->rf;
  a.st = c->dstat;
  a.wait_ns = c->wait_ns;
  uint64_t rbits;
  memcpy(&rbits, &c->r, sizeof(rbits));
  const int rexp = (int)((rbits >> 52) & 2047);
  const bool dom = emul::domain_bounds(rbits, T, a.eng.dom_lo, a.eng.dom_hi);
  a.eng.mx = emul::prepare_mulx(rbits);
  // integer tiles: the library's split (half of the warps) or a fixed share,
  // for a normal nonzero r whose screen admits data at this depth
  const bool int_ok = mode == 0 && rexp >= 1 && rexp <= 2046 && dom;
  a.dual = int_ok && c->emul_auto;
  a.emul_mask = int_ok && !c->emul_auto ? c->emul_mask : 0u;
  a.p2_fp64 = mode == 0 && dom && a.eng.mx.pow2;
  a.eng.p2_hi_add = (int)(((int64_t)rexp - 1023) * (1 << 20));
  a.eng.p2_hi_xor = (rbits >> 63) ? (int)0x80000000u : 0;
  a.inj_tile = c->inj_segment >= 0 ? c->inj_segment : -1;
  a.inj_level = c->inj_step / T;
  rc = mode == 0 ? launch_wave<0>(c, a) : mode == 1 ? launch_wave<1>(c, a) : launch_wave<2>(c, a);
  if (rc != HEAT_OK) return rc;
  const int64_t levels = (nt + T - 1) / T;
  if (levels & 1) c->cur ^= 1;
  c->steps += nt;
  c->last_T = T;
  c->last_launches = 1;
  return HEAT_OK;
}

}  // namespace heat

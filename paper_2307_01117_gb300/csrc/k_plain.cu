// k_plain.cu -- form HEAT_FORM_PLAIN: one step of Eq. 2 (Section 2) over the
// whole periodic ring per launch.  The ghost exchange between segments is the
// launch boundary itself (the unsegmented synchronous variant of Section 3.1).
//
// Layout: a warp owns 64 consecutive points per iteration; lane l loads points
// 2l, 2l+1 as one 16-byte vector, neighbours inside the tile come from the
// adjacent lanes by shuffle, the two tile-edge neighbours are scalar loads
// (wrapping at 0 and N-1).  The fewer than 64 trailing points are done by
// scalar threads.  Algorithmic traffic: 8 bytes read + 8 bytes written per
// point-step for binary64, 4 + 4 for binary32.
#include <string.h>

#include "dp_emul.cuh"
#include "heat_internal.cuh"
#include "stencil_ops.cuh"

namespace heat {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPlainThreads = 256;

// Binary64: a warp takes kU64 consecutive 64-point tiles at a time, so each
// lane has 2*kU64 independent updates (4 FP64 operations each) to interleave
// while the FP64 unit drains.
constexpr int kU64 = 4;

// For r = +-2^k under the exact reading (P2): a group whose values, edge
// neighbours included, pass the integer-pipe screen for one step takes the
// multiply as an exponent add on the integer pipes (eq2_exact_pow2: 3 FP64-unit
// operations per point); other groups, leftover tiles and the tail the plain
// exact update.
struct P2Args {
  int dom_lo, dom_hi, hi_add, hi_xor;
};

__device__ __forceinline__ bool p2_ok(double x, const P2Args &p) {
  return emul::in_domain((uint64_t)__double_as_longlong(x), p.dom_lo, p.dom_hi);
}

template <bool FMA, bool P2>
__global__ void __launch_bounds__(kPlainThreads) k_plain_f64(const double *__restrict__ u, double *__restrict__ v,
                                                             int64_t N, double r, P2Args p2a) {
  const int lane = threadIdx.x & 31;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t warp = gtid >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t ntiles = N >> 6;
  const int64_t ngroups = ntiles / kU64;
  for (int64_t q = warp; q < ngroups; q += nwarps) {
    const int64_t b0 = q * kU64 * 64;
    double2 x[kU64];
#pragma unroll
    for (int j = 0; j < kU64; ++j) x[j] = __ldcs(reinterpret_cast<const double2 *>(u + b0 + 64 * j) + lane);
    double eleft = 0.0, eright = 0.0;
    if (lane == 0) eleft = u[b0 == 0 ? N - 1 : b0 - 1];
    if (lane == 31) eright = u[b0 + 64 * kU64 == N ? 0 : b0 + 64 * kU64];
    bool p2 = false;
    if constexpr (P2) {
      bool ok = p2_ok(eleft, p2a) && p2_ok(eright, p2a);
#pragma unroll
      for (int j = 0; j < kU64; ++j) ok = ok && p2_ok(x[j].x, p2a) && p2_ok(x[j].y, p2a);
      p2 = __all_sync(kFull, ok);
    }
#pragma unroll
    for (int j = 0; j < kU64; ++j) {
      double left = __shfl_up_sync(kFull, x[j].y, 1);
      double right = __shfl_down_sync(kFull, x[j].x, 1);
      const double prev_y = __shfl_sync(kFull, x[j > 0 ? j - 1 : 0].y, 31);
      const double next_x = __shfl_sync(kFull, x[j + 1 < kU64 ? j + 1 : kU64 - 1].x, 0);
      if (lane == 0) left = j > 0 ? prev_y : eleft;
      if (lane == 31) right = j + 1 < kU64 ? next_x : eright;
      double2 y;
      if (P2 && p2) {
        y.x = eq2_exact_pow2(left, x[j].x, x[j].y, p2a.hi_add, p2a.hi_xor);
        y.y = eq2_exact_pow2(x[j].x, x[j].y, right, p2a.hi_add, p2a.hi_xor);
      } else {
        y.x = eq2<FMA>(left, x[j].x, x[j].y, r);
        y.y = eq2<FMA>(x[j].x, x[j].y, right, r);
      }
      __stcs(reinterpret_cast<double2 *>(v + b0 + 64 * j) + lane, y);
    }
  }
  // tiles left over after the groups
  for (int64_t t = ngroups * kU64 + warp; t < ntiles; t += nwarps) {
    const int64_t b = t << 6;
    const double2 x = __ldcs(reinterpret_cast<const double2 *>(u + b) + lane);
    double left = __shfl_up_sync(kFull, x.y, 1);
    double right = __shfl_down_sync(kFull, x.x, 1);
    if (lane == 0) left = u[b == 0 ? N - 1 : b - 1];
    if (lane == 31) right = u[b + 64 == N ? 0 : b + 64];
    double2 y;
    y.x = eq2<FMA>(left, x.x, x.y, r);
    y.y = eq2<FMA>(x.x, x.y, right, r);
    __stcs(reinterpret_cast<double2 *>(v + b) + lane, y);
  }
  const int64_t tail0 = ntiles << 6;
  if (gtid < N - tail0) {
    const int64_t g = tail0 + gtid;
    const double ul = u[g == 0 ? N - 1 : g - 1];
    const double ur = u[g + 1 == N ? 0 : g + 1];
    v[g] = eq2<FMA>(ul, u[g], ur, r);
  }
}

// Binary32 state, compensated update with a block of one step: the correction
// starts at zero, so the pair (h, 0) is advanced once and stored as RN(h + l).
__device__ __forceinline__ float f32c_one_step(float hl, float h, float hr, float rf) {
  float hn, ln;
  eq2_f32c(hl, h, hr, 0.0f, 0.0f, 0.0f, rf, hn, ln);
  return f32c_store(hn, ln);
}

// Binary32 is HBM-bound in this form: a warp first issues the loads of kU
// consecutive 128-point tiles (kU x 512 bytes in flight per warp), then
// computes and stores them.
constexpr int kU = 4;

__global__ void __launch_bounds__(kPlainThreads) k_plain_f32c(const float *__restrict__ u, float *__restrict__ v,
                                                              int64_t N, float rf) {
  const int lane = threadIdx.x & 31;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t warp = gtid >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t ntiles = N >> 7;  // 128 points per warp tile (float4 per lane)
  const int64_t ngroups = ntiles / kU;
  for (int64_t q = warp; q < ngroups; q += nwarps) {
    const int64_t b0 = q * kU * 128;
    float4 x[kU];
#pragma unroll
    for (int j = 0; j < kU; ++j) x[j] = __ldcs(reinterpret_cast<const float4 *>(u + b0 + 128 * j) + lane);
    float eleft = 0.0f, eright = 0.0f;
    if (lane == 0) eleft = u[b0 == 0 ? N - 1 : b0 - 1];
    if (lane == 31) eright = u[b0 + 128 * kU == N ? 0 : b0 + 128 * kU];
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      float left = __shfl_up_sync(kFull, x[j].w, 1);
      float right = __shfl_down_sync(kFull, x[j].x, 1);
      // tile edges: the previous / next tile of the group, or the group's edge loads
      const float prev_w = __shfl_sync(kFull, x[j > 0 ? j - 1 : 0].w, 31);
      const float next_x = __shfl_sync(kFull, x[j + 1 < kU ? j + 1 : kU - 1].x, 0);
      if (lane == 0) left = j > 0 ? prev_w : eleft;
      if (lane == 31) right = j + 1 < kU ? next_x : eright;
      float4 y;
      y.x = f32c_one_step(left, x[j].x, x[j].y, rf);
      y.y = f32c_one_step(x[j].x, x[j].y, x[j].z, rf);
      y.z = f32c_one_step(x[j].y, x[j].z, x[j].w, rf);
      y.w = f32c_one_step(x[j].z, x[j].w, right, rf);
      __stcs(reinterpret_cast<float4 *>(v + b0 + 128 * j) + lane, y);
    }
  }
  // tiles left over after the groups
  for (int64_t t = ngroups * kU + warp; t < ntiles; t += nwarps) {
    const int64_t b = t << 7;
    const float4 x = __ldcs(reinterpret_cast<const float4 *>(u + b) + lane);
    float left = __shfl_up_sync(kFull, x.w, 1);
    float right = __shfl_down_sync(kFull, x.x, 1);
    if (lane == 0) left = u[b == 0 ? N - 1 : b - 1];
    if (lane == 31) right = u[b + 128 == N ? 0 : b + 128];
    float4 y;
    y.x = f32c_one_step(left, x.x, x.y, rf);
    y.y = f32c_one_step(x.x, x.y, x.z, rf);
    y.z = f32c_one_step(x.y, x.z, x.w, rf);
    y.w = f32c_one_step(x.z, x.w, right, rf);
    __stcs(reinterpret_cast<float4 *>(v + b) + lane, y);
  }
  const int64_t tail0 = ntiles << 7;
  if (gtid < N - tail0) {
    const int64_t g = tail0 + gtid;
    const float ul = u[g == 0 ? N - 1 : g - 1];
    const float ur = u[g + 1 == N ? 0 : g + 1];
    v[g] = f32c_one_step(ul, u[g], ur, rf);
  }
}

// Grid: enough warps to cover the tiles, capped at a whole number of waves
// (blocks per SM x SMs); at least enough threads for the scalar tail.
int plain_grid(const heat_ctx *c, int64_t tiles) {
  const int64_t warps_per_block = kPlainThreads / 32;
  int64_t blocks = (tiles + warps_per_block - 1) / warps_per_block;
  const int64_t cap = (int64_t)c->sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

}  // namespace

int run_plain(heat_ctx *c, int64_t nt) {
  const int64_t N = c->geo.N;
  for (int64_t s = 0; s < nt; ++s) {
    const void *src = c->buf[c->cur];
    void *dst = c->buf[c->cur ^ 1];
    if (c->dtype == HEAT_F64) {
      const int grid = plain_grid(c, (N >> 6) / kU64 > 0 ? (N >> 6) / kU64 : 1);
      uint64_t rbits;
      memcpy(&rbits, &c->r, sizeof(rbits));
      const int rexp = (int)((rbits >> 52) & 2047);
      P2Args p2a = {1, 0, (rexp - 1023) * (1 << 20), (rbits >> 63) ? (int)0x80000000u : 0};
      const bool p2 = c->arith == HEAT_ARITH_EXACT && rexp >= 1 && rexp <= 2046 &&
                      (rbits & 0x000fffffffffffffull) == 0 && emul::domain_bounds(rbits, 1, p2a.dom_lo, p2a.dom_hi);
      if (c->arith == HEAT_ARITH_FMA)
        k_plain_f64<true, false><<<grid, kPlainThreads, 0, c->stream>>>((const double *)src, (double *)dst, N, c->r,
                                                                       p2a);
      else if (p2)
        k_plain_f64<false, true><<<grid, kPlainThreads, 0, c->stream>>>((const double *)src, (double *)dst, N, c->r,
                                                                       p2a);
      else
        k_plain_f64<false, false><<<grid, kPlainThreads, 0, c->stream>>>((const double *)src, (double *)dst, N, c->r,
                                                                        p2a);
    } else {
      const int grid = plain_grid(c, (N >> 7) / kU > 0 ? (N >> 7) / kU : 1);
      k_plain_f32c<<<grid, kPlainThreads, 0, c->stream>>>((const float *)src, (float *)dst, N, c->rf);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return HEAT_ECUDA;
    c->cur ^= 1;
    c->steps += 1;
    c->last_launches += 1;
  }
  return HEAT_OK;
}

}  // namespace heat

// k_cluster.cu -- form HEAT_FORM_CLUSTER: small rings in one thread-block
// cluster, all nt steps in one launch.
//
// The ring is cut into C segments, one per CTA of a single cluster (C <= 16).
// Each CTA keeps its segment in shared memory (two buffers).  Every block of T
// steps, each warp builds a register window over its part of the segment plus a
// T-point halo on each side; halo points come from the neighbouring CTAs'
// shared memory through distributed shared memory (the cluster's ghost
// exchange -- the GPU form of Section 2's neighbour queues, with the cluster
// barrier as the only synchronisation), the window advances T steps with the
// register-resident temporal-blocking core, and the exact middle is written to
// the CTA's other buffer.  One cluster barrier per block orders the writes of
// one block before the reads of the next and the reads of one block before the
// writes that reuse its buffer.  The ring is periodic within the cluster: the
// neighbours of CTA 0 are CTAs C-1 and 1.
#include <cooperative_groups.h>
#include <string.h>

#include "tb_core.cuh"

namespace cg = cooperative_groups;

namespace heat {
namespace {

constexpr int kCWarps = 4;

struct ClusterArgs {
  const void *src;  // state at the start (global)
  void *dst;        // state at the end (global)
  int64_t N;
  int C;            // CTAs (segments)
  int T;
  int64_t nt;
  double r;
  float rf;
  int p2;                  // binary64, r = +-2^k: screened windows multiply on the integer pipes
  int dom_lo, dom_hi;      // the screen for T steps (biased exponents)
  int p2_hi_add, p2_hi_xor;
};

template <int MODE, int EP>
__global__ void __launch_bounds__(kCWarps * 32) k_cluster(ClusterArgs a) {
  using P = tb::TBCx<MODE, EP>;
  using Tt = typename P::T;
  constexpr int E = P::E;
  constexpr int WIN = 32 * E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int c = (int)cluster.block_rank();
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int C = a.C;
  const int64_t N = a.N;
  // segment c: [lo, hi), balanced
  const int64_t lo = (int64_t)c * N / C, hi = (int64_t)(c + 1) * N / C;
  const int len = (int)(hi - lo);
  const int cl = (c + C - 1) % C, cr = (c + 1) % C;
  const int len_l = (int)(((int64_t)(cl + 1) * N / C) - ((int64_t)cl * N / C));
  const int seg_max = (int)((N + C - 1) / C);
  Tt *buf[2] = {reinterpret_cast<Tt *>(smem_raw), reinterpret_cast<Tt *>(smem_raw) + seg_max};

  const Tt *src = (const Tt *)a.src;
  for (int i = threadIdx.x; i < len; i += blockDim.x) buf[0][i] = src[lo + i];
  cluster.sync();

  const int W = WIN - 2 * a.T;
  int cur = 0;
  for (int64_t done = 0; done < a.nt;) {
    const int steps = (int)(a.nt - done < a.T ? a.nt - done : a.T);
    const Tt *own = buf[cur];
    const Tt *left = cluster.map_shared_rank(buf[cur], cl);
    const Tt *right = cluster.map_shared_rank(buf[cur], cr);
    Tt *out = buf[cur ^ 1];
    for (int w0 = wib * W; w0 < len; w0 += kCWarps * W) {
      // window index i <-> segment-relative position p = w0 - T + i
      typename P::Reg R;
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const int p = w0 - a.T + E * lane + k;
        Tt v = Tt(0);  // points beyond the halo are never exact after T steps
        if (C == 1) {  // the whole ring in one CTA: the window may wrap around it several times
          int q = p % len;
          if (q < 0) q += len;
          v = own[q];
        } else if (p < 0) {
          if (p >= -a.T) v = left[len_l + p];
        } else if (p < len) {
          v = own[p];
        } else if (p < len + a.T) {
          v = right[p - len];
        }
        P::load(R, k, v);
      }
      bool p2 = false;
      if constexpr (MODE == 0) {
        if (a.p2) {
          bool ok = true;
#pragma unroll
          for (int k = 0; k < E; ++k)
            ok &= emul::in_domain((uint64_t)__double_as_longlong(P::store(R, k)), a.dom_lo, a.dom_hi);
          p2 = __all_sync(0xffffffffu, ok);
        }
        if (p2)
          for (int s = 0; s < steps; ++s) P::step_p2(R, a.p2_hi_add, a.p2_hi_xor);
      }
      if (!p2)
        for (int s = 0; s < steps; ++s) P::step(R, lane, a.r, a.rf);
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const int i = E * lane + k;
        const int p = w0 - a.T + i;
        if (i >= a.T && i < a.T + W && p < len) out[p] = P::store(R, k);
      }
    }
    cluster.sync();  // this block's writes visible; its reads of `own` and the neighbours finished
    cur ^= 1;
    done += steps;
  }
  Tt *dst = (Tt *)a.dst;
  for (int i = threadIdx.x; i < len; i += blockDim.x) dst[lo + i] = buf[cur][i];
}

template <int MODE, int EP>
int launch_cluster(heat_ctx *c, int C, int T, int64_t nt) {
  using P = tb::TBCx<MODE, EP>;
  const int64_t N = c->geo.N;
  const int seg_max = (int)((N + C - 1) / C);
  const size_t smem = 2 * (size_t)seg_max * sizeof(typename P::T);
  if (C > 8 &&
      cudaFuncSetAttribute(k_cluster<MODE, EP>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return HEAT_ECUDA;
  if (cudaFuncSetAttribute(k_cluster<MODE, EP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return HEAT_ECUDA;
  ClusterArgs a;
  a.src = c->buf[c->cur];
  a.dst = c->buf[c->cur ^ 1];
  a.N = N;
  a.C = C;
  a.T = T;
  a.nt = nt;
  a.r = c->r;
  a.rf = c->rf;
  uint64_t rbits;
  memcpy(&rbits, &c->r, sizeof(rbits));
  const int rexp = (int)((rbits >> 52) & 2047);
  // r = +-2^k, exact reading: windows whose values pass the integer tiles'
  // screen move the product's exponent with an integer add (eq2_exact_pow2)
  a.p2 = MODE == 0 && rexp >= 1 && rexp <= 2046 && (rbits & 0x000fffffffffffffull) == 0 &&
         emul::domain_bounds(rbits, T, a.dom_lo, a.dom_hi);
  a.p2_hi_add = (rexp - 1023) * (1 << 20);
  a.p2_hi_xor = (rbits >> 63) ? (int)0x80000000u : 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kCWarps * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, k_cluster<MODE, EP>, &cfg) != cudaSuccess || clusters < 1)
    return HEAT_ENOTSUP;
  return cudaLaunchKernelEx(&cfg, k_cluster<MODE, EP>, a) == cudaSuccess ? HEAT_OK : HEAT_ECUDA;
}

// Points per lane the cluster form may use, smallest first (smaller windows
// spread a small ring over more warps, hence more of each SM's FP64 unit).
constexpr int kEp64[3] = {4, 8, 16};
constexpr int kEp32[3] = {8, 16, 32};

template <int MODE>
int launch_ep(heat_ctx *c, int ep, int C, int T, int64_t nt) {
  if constexpr (MODE == 2) {
    switch (ep) {
      case 8: return launch_cluster<MODE, 8>(c, C, T, nt);
      case 16: return launch_cluster<MODE, 16>(c, C, T, nt);
      default: return launch_cluster<MODE, 32>(c, C, T, nt);
    }
  } else {
    switch (ep) {
      case 4: return launch_cluster<MODE, 4>(c, C, T, nt);
      case 8: return launch_cluster<MODE, 8>(c, C, T, nt);
      default: return launch_cluster<MODE, 16>(c, C, T, nt);
    }
  }
}

}  // namespace

// Largest ring the cluster form takes: 16 CTAs x 4 warps x one window of output
// each, at the largest window.
int64_t cluster_max_points(const heat_ctx *c, int T) {
  const int win = c->dtype == HEAT_F32C ? 32 * kEp32[2] : 32 * kEp64[2];
  return (int64_t)16 * kCWarps * (win - 2 * T);
}

int run_cluster(heat_ctx *c, int64_t nt) {
  const int mode = c->dtype == HEAT_F32C ? 2 : (c->arith == HEAT_ARITH_FMA ? 1 : 0);
  const int64_t N = c->geo.N;
  // default depth: binary32 32; binary64 16 (0.53 vs 0.59 us per step at 4000
  // points), or 8 for rings that only fit at that depth
  const int T = c->T > 0 ? c->T
                         : (c->dtype == HEAT_F32C ? 32 : (N <= cluster_max_points(c, 16) ? 16 : 8));
  const int *eps = c->dtype == HEAT_F32C ? kEp32 : kEp64;
  if (2 * T >= 32 * eps[2]) return HEAT_EINVAL;
  if (N > cluster_max_points(c, T)) return HEAT_ENOTSUP;
  // the smallest window whose 64 copies (16 CTAs x 4 warps) cover the ring
  int ep = eps[2];
  for (int i = 0; i < 3; ++i) {
    const int64_t w = 32 * eps[i] - 2 * T;
    if (w >= T && w * 16 * kCWarps >= N) {
      ep = eps[i];
      break;
    }
  }
  const int64_t W = 32 * ep - 2 * T;
  // one window of output per CTA at least, at most 16 CTAs, each segment at
  // least T points long so a halo never reaches past a neighbour (a ring
  // shorter than T runs in one CTA, whose windows wrap around it)
  int64_t C = (N + W - 1) / W;
  if (C > 16) C = 16;
  while (C > 1 && N / C < T) --C;
  if (C < 1) C = 1;
  const int rc = mode == 0 ? launch_ep<0>(c, ep, (int)C, T, nt)
                 : mode == 1 ? launch_ep<1>(c, ep, (int)C, T, nt)
                             : launch_ep<2>(c, ep, (int)C, T, nt);
  if (rc != HEAT_OK) return rc;
  c->cur ^= 1;
  c->steps += nt;
  c->last_T = T;
  c->last_launches = 1;
  c->last_segments = (int)C;
  return HEAT_OK;
}

}  // namespace heat

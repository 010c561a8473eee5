// tb_core.cuh -- register-resident temporal-blocking core shared by the
// temporal-blocking form (k_tblock.cu) and the batched-ring kernel (k_batch.cu):
// the per-warp window layout (lane l holds window points 32k + l), one step of
// Eq. 2 (Section 2) by lane shuffles in each arithmetic form, and the mbarrier /
// bulk-TMA helpers used to stage windows.
#pragma once

#include "dp_emul.cuh"
#include "heat_internal.cuh"
#include "stencil_ops.cuh"

namespace heat {
namespace tb {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void bulk_load(void *sdst, const void *gsrc, unsigned bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(sdst)),
               "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---- per-dtype register state and update --------------------------------------------
template <int MODE>
struct TB;

template <int MODE>
struct TBf64 {
  using T = double;
  static constexpr int E = 16;  // points per lane: window of 512
  static constexpr int kAlign = 2;  // elements per 16 bytes
  struct Reg {
    double x[E];
  };
  static __device__ __forceinline__ void load(Reg &R, int k, double v) { R.x[k] = v; }
  static __device__ __forceinline__ double store(const Reg &R, int k) { return R.x[k]; }
  static __device__ __forceinline__ void step(Reg &R, int lane, double r, float) {
    const int lm = (lane + 31) & 31, lp = (lane + 1) & 31;
    double Lprev = __shfl_sync(kFull, R.x[0], lm);
    double Rcur = __shfl_sync(kFull, R.x[0], lp);
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const double Lk = k == 0 ? Lprev : __shfl_sync(kFull, R.x[k], lm);
      const double Rn = k + 1 < E ? __shfl_sync(kFull, R.x[k + 1], lp) : Rcur;
      const double left = lane == 0 ? Lprev : Lk;
      const double right = lane == 31 ? Rn : Rcur;
      R.x[k] = eq2<MODE == 1>(left, R.x[k], right, r);
      Lprev = Lk;
      Rcur = Rn;
    }
  }
  // The step with its multiply (and, for registers k whose bit is set in
  // add_mask, its final add) done by the integer-pipe routines; the two
  // differences stay on the FP64 unit.  Exact reading only.  The FP64 unit then
  // issues 3 (or 2) operations per point instead of 4.
  static __device__ __forceinline__ void step_split(Reg &R, int lane, const emul::Mul &m, unsigned add_mask,
                                                    bool &bad) {
    const int lm = (lane + 31) & 31, lp = (lane + 1) & 31;
    double Lprev = __shfl_sync(kFull, R.x[0], lm);
    double Rcur = __shfl_sync(kFull, R.x[0], lp);
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const double Lk = k == 0 ? Lprev : __shfl_sync(kFull, R.x[k], lm);
      const double Rn = k + 1 < E ? __shfl_sync(kFull, R.x[k + 1], lp) : Rcur;
      const double left = lane == 0 ? Lprev : Lk;
      const double right = lane == 31 ? Rn : Rcur;
      const double t1 = __fma_rn(-2.0, R.x[k], left);
      const double t2 = __dadd_rn(t1, right);
      const uint64_t t3 = emul::mul(m, (uint64_t)__double_as_longlong(t2), bad);
      if ((add_mask >> k) & 1u)
        R.x[k] = __longlong_as_double((long long)emul::add((uint64_t)__double_as_longlong(R.x[k]), t3, bad));
      else
        R.x[k] = __dadd_rn(R.x[k], __longlong_as_double((long long)t3));
      Lprev = Lk;
      Rcur = Rn;
    }
  }
  // The same step with the integer-pipe binary64 routines (exact reading only).
  static __device__ __forceinline__ void step_emul(Reg &R, int lane, const emul::Mul &m, bool &bad) {
    const int lm = (lane + 31) & 31, lp = (lane + 1) & 31;
    double Lprev = __shfl_sync(kFull, R.x[0], lm);
    double Rcur = __shfl_sync(kFull, R.x[0], lp);
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const double Lk = k == 0 ? Lprev : __shfl_sync(kFull, R.x[k], lm);
      const double Rn = k + 1 < E ? __shfl_sync(kFull, R.x[k + 1], lp) : Rcur;
      const double left = lane == 0 ? Lprev : Lk;
      const double right = lane == 31 ? Rn : Rcur;
      const uint64_t v = emul::eq2_exact((uint64_t)__double_as_longlong(left), (uint64_t)__double_as_longlong(R.x[k]),
                                         (uint64_t)__double_as_longlong(right), m, bad);
      R.x[k] = __longlong_as_double((long long)v);
      Lprev = Lk;
      Rcur = Rn;
    }
  }
};
template <>
struct TB<0> : TBf64<0> {};
template <>
struct TB<1> : TBf64<1> {};

template <>
struct TB<2> {
  using T = float;
  static constexpr int E = 32;  // window of 1024
  static constexpr int kAlign = 4;
  struct Reg {
    float h[E];
    float l[E];
  };
  static __device__ __forceinline__ void load(Reg &R, int k, float v) {
    R.h[k] = v;
    R.l[k] = 0.0f;
  }
  static __device__ __forceinline__ float store(const Reg &R, int k) { return f32c_store(R.h[k], R.l[k]); }
  static __device__ __forceinline__ void step(Reg &R, int lane, double, float rf) {
    const int lm = (lane + 31) & 31, lp = (lane + 1) & 31;
    float Lh = __shfl_sync(kFull, R.h[0], lm), Ll = __shfl_sync(kFull, R.l[0], lm);
    float Rh = __shfl_sync(kFull, R.h[0], lp), Rl = __shfl_sync(kFull, R.l[0], lp);
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const float Lkh = k == 0 ? Lh : __shfl_sync(kFull, R.h[k], lm);
      const float Lkl = k == 0 ? Ll : __shfl_sync(kFull, R.l[k], lm);
      const float Rnh = k + 1 < E ? __shfl_sync(kFull, R.h[k + 1], lp) : Rh;
      const float Rnl = k + 1 < E ? __shfl_sync(kFull, R.l[k + 1], lp) : Rl;
      const float lh = lane == 0 ? Lh : Lkh, ll = lane == 0 ? Ll : Lkl;
      const float rh = lane == 31 ? Rnh : Rh, rl = lane == 31 ? Rnl : Rl;
      float hn, ln;
      eq2_f32c(lh, R.h[k], rh, ll, R.l[k], rl, rf, hn, ln);
      R.h[k] = hn;
      R.l[k] = ln;
      Lh = Lkh;
      Ll = Lkl;
      Rh = Rnh;
      Rl = Rnl;
    }
  }
};

template <int MODE>
struct HasEmul {
  static constexpr bool value = MODE == 0;
};

// ---- contiguous ownership: lane l holds window points E*l .. E*l + E - 1 ------------------
// A step needs only the last point of lane l-1 and the first point of lane l+1
// (two shuffles per carried value per lane); every other neighbour is in the
// lane's own registers.  Lane 0's left and lane 31's right neighbours are the
// window's outer halo, which loses one valid point per step as in the strided
// layout: after s steps the window points s .. WIN-1-s are exact.
template <int MODE, int EP>
struct TBCx;

// binary64 (MODE 0 exact reading, 1 fused reading), EP points per lane
template <int MODE, int EP>
struct TBCf64 {
  using T = double;
  static constexpr int E = EP;
  struct Reg {
    double x[E];
  };
  static __device__ __forceinline__ void load(Reg &R, int k, double v) { R.x[k] = v; }
  static __device__ __forceinline__ double store(const Reg &R, int k) { return R.x[k]; }
  static __device__ __forceinline__ void step(Reg &R, int, double r, float) {
    const double left = __shfl_up_sync(kFull, R.x[E - 1], 1);
    const double right = __shfl_down_sync(kFull, R.x[0], 1);
    double prev = left;
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const double nxt = k + 1 < E ? R.x[k + 1] : right;
      const double v = eq2<MODE == 1>(prev, R.x[k], nxt, r);
      prev = R.x[k];
      R.x[k] = v;
    }
  }
};
__device__ __forceinline__ emul::X shfl_x(emul::X v, bool up) {
  emul::X w;
  w.m = up ? __shfl_up_sync(kFull, (long long)v.m, 1) : __shfl_down_sync(kFull, (long long)v.m, 1);
  w.e = up ? __shfl_up_sync(kFull, v.e, 1) : __shfl_down_sync(kFull, v.e, 1);
  w.pad = 0;
  return w;
}

template <int EP>
struct TBCx<0, EP> : TBCf64<0, EP> {
  // One step on the FP64 unit for r = +-2^k and a screened tile (the multiply
  // moves the exponent on the integer pipes: eq2_exact_pow2).
  static __device__ __forceinline__ void step_p2(typename TBCf64<0, EP>::Reg &R, int hi_add, int hi_xor) {
    constexpr int E = EP;
    const double left = __shfl_up_sync(kFull, R.x[E - 1], 1);
    const double right = __shfl_down_sync(kFull, R.x[0], 1);
    double prev = left;
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const double nxt = k + 1 < E ? R.x[k + 1] : right;
      const double v = eq2_exact_pow2(prev, R.x[k], nxt, hi_add, hi_xor);
      prev = R.x[k];
      R.x[k] = v;
    }
  }

  // All `steps` steps of a tile on the integer pipes, in the unpacked form of
  // dp_emul.cuh (the caller has screened the tile's values with in_domain;
  // POW2 and NEG must match m).
  // The lane's points live in a small local array (w[1..E], halo values in
  // w[0] and w[E+1]) walked by a loop that is not unrolled, which keeps the
  // code small enough for the instruction cache beside the FP64-unit tiles.
  template <bool POW2, bool NEG>
  static __device__ __forceinline__ void steps_x(typename TBCf64<0, EP>::Reg &R, int steps, const emul::MulX &m) {
    constexpr int E = EP;
    emul::X w[E + 2];
#pragma unroll
    for (int k = 0; k < E; ++k) w[k + 1] = emul::unpack((uint64_t)__double_as_longlong(R.x[k]));
    for (int s = 0; s < steps; ++s) {
      w[0] = shfl_x(w[E], true);
      w[E + 1] = shfl_x(w[1], false);
      emul::X prev = w[0], cur = w[1];
#pragma unroll 4
      for (int k = 1; k <= E; ++k) {
        const emul::X nxt = w[k + 1];
        w[k] = emul::eq2x<POW2, NEG>(prev, cur, nxt, m);
        prev = cur;
        cur = nxt;
      }
    }
#pragma unroll
    for (int k = 0; k < E; ++k) R.x[k] = __longlong_as_double((long long)emul::pack(w[k + 1]));
  }
};
template <int EP>
struct TBCx<1, EP> : TBCf64<1, EP> {};

// binary32 compensated, EP points per lane
template <int EP>
struct TBCx<2, EP> {
  using T = float;
  static constexpr int E = EP;
  static constexpr int H = EP / 2;
  // Pair j holds the lane's points j and j + H (low and high half), so the
  // left and right neighbours of pair j are pairs j - 1 and j + 1: the whole
  // step runs on paired binary32 instructions (eq2_f32c_x2); only the two
  // pairs at the ends are assembled from single values each step.
  struct Reg {
    unsigned long long h[H];
    unsigned long long l[H];
  };
  static __device__ __forceinline__ void load(Reg &R, int k, float v) {
    const int j = k < H ? k : k - H;
    R.h[j] = k < H ? f2_pack(v, f2_hi(R.h[j])) : f2_pack(f2_lo(R.h[j]), v);
    R.l[j] = 0ull;
  }
  static __device__ __forceinline__ float store(const Reg &R, int k) {
    const int j = k < H ? k : k - H;
    return k < H ? f32c_store(f2_lo(R.h[j]), f2_lo(R.l[j])) : f32c_store(f2_hi(R.h[j]), f2_hi(R.l[j]));
  }
  static __device__ __forceinline__ void step(Reg &R, int, double, float rf) {
    // point -1 (lane - 1's point E - 1) and point E (lane + 1's point 0)
    const float ph = __shfl_up_sync(kFull, f2_hi(R.h[H - 1]), 1), pl = __shfl_up_sync(kFull, f2_hi(R.l[H - 1]), 1);
    const float nh = __shfl_down_sync(kFull, f2_lo(R.h[0]), 1), nl = __shfl_down_sync(kFull, f2_lo(R.l[0]), 1);
    // neighbours of the end pairs: (point -1, point H - 1) and (point H, point E)
    unsigned long long prev_h = f2_pack(ph, f2_lo(R.h[H - 1])), prev_l = f2_pack(pl, f2_lo(R.l[H - 1]));
    const unsigned long long last_h = f2_pack(f2_hi(R.h[0]), nh), last_l = f2_pack(f2_hi(R.l[0]), nl);
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const unsigned long long nxt_h = j + 1 < H ? R.h[j + 1] : last_h;
      const unsigned long long nxt_l = j + 1 < H ? R.l[j + 1] : last_l;
      unsigned long long hn, ln;
      eq2_f32c_x2(prev_h, R.h[j], nxt_h, prev_l, R.l[j], nxt_l, rf, hn, ln);
      prev_h = R.h[j];
      prev_l = R.l[j];
      R.h[j] = hn;
      R.l[j] = ln;
    }
  }
};

// Default window: 512 binary64 points, 1024 binary32 points.
template <int MODE>
struct TBC : TBCx<MODE, MODE == 2 ? 32 : 16> {};

}  // namespace tb
}  // namespace heat

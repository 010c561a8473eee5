// heat_internal.cuh -- context layout and launcher interfaces shared by the
// translation units of libheat.so.  Not part of the public ABI (include/heat.h).
#pragma once

#include <string.h>

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/heat.h"

namespace heat {

// Largest temporal block depth (steps per tile load) the kernels accept.
constexpr int kMaxT = 64;

// One inbound ghost mailbox of the persistent forms (the GPU form of the
// single-producer single-consumer queue of Section 2).  The producer writes
// val[slot][0..T) and then stores seq with release semantics; the consumer
// acquires seq and reads.  Two slots suffice because neighbours never drift
// more than one step (block) apart: a producer can only overwrite slot s%2 with
// the values of step s+2 after it has acquired the consumer's step-(s+1)
// publication, which the consumer makes after reading slot s%2.
struct __align__(128) Mailbox {
  unsigned long long seq;
  unsigned long long pad[15];
  double val[2][kMaxT];
};

// Device-side status, written by kernels, read by the host at sync points.
struct DevStatus {
  int code;            // HEAT_OK or HEAT_ETIMEOUT (first error wins)
  int segment;         // segment whose wait ran out
  long long step;      // step at which it ran out
  int abort;           // set by the first CTA that gives up; others stop waiting
  int pad;
};

struct Geometry {
  int64_t nx;
  int32_t np;
  int64_t N;
};

}  // namespace heat

struct heat_ctx {
  heat::Geometry geo;
  double r;          // k*dt/(dx*dx), binary64
  float rf;          // (float)r for HEAT_F32C
  heat_dtype dtype;
  int device;
  int sms;
  size_t elem;       // bytes per state element
  void *buf[2];      // double-buffered state, global order
  int cur;           // index of the buffer holding the current state
  cudaStream_t own_stream;
  cudaStream_t stream;
  int form;
  int T;
  int arith;
  int64_t steps;
  int host_error;                // sticky device error seen at the last sync
  heat::DevStatus *dstat;        // device
  heat::DevStatus *hstat;        // pinned host mirror
  heat::Mailbox *mbox;           // 2 per segment (in_left, in_right), device
  int64_t *seg_start;            // segment table (S+1 entries), device
  int mbox_segments;             // capacity of mbox / seg_start
  int segments;                  // persistent segmentation: 0 auto, -1 one per partition, >0 count
  int last_segments;             // segments used by the last persistent run
  int last_form;                 // form used by the last heat_run
  int last_T;                    // temporal block depth used by the last heat_run
  int64_t last_launches;         // stencil kernel launches queued by the last heat_run
  int emul_share;                // tiles of 32 computed on the integer pipes (binary64, exact reading)
  unsigned emul_mask;            // the same as a bit mask over tile index mod 32
  int emul_auto;                 // share chosen per ring (heat_set_emulation(c, -1))
  int split_level;               // per-point split of the binary64 update between FP64 unit and integer pipes
  int tb_layout;                 // temporal-blocking register layout: 0 strided (TMA-staged), 1 contiguous
  unsigned *wave_done;           // persistent temporal blocking, device: levels finished per tile (lazy)
  int64_t wave_cap;              // capacity of wave_done
  unsigned long long *wave_counter;  // its unit counter, device (lazy)
  // CUDA graph of the last multi-launch run (plain / temporal blocking), replayed
  // when the next run has the same key
  int graphs;                    // 1: capture and replay multi-launch runs
  cudaGraphExec_t graph_exec;
  unsigned long long graph_key[8];
  int graph_cur_flip;            // parity change of the current buffer over the run
  int graph_last_T;
  int64_t graph_last_launches;
  double *partials;              // reduction scratch, device
  unsigned long long *tile_counter;  // temporal-blocking form, device: [0] tile counter, [1] finished CTAs
  int counter_dirty;             // a strided launch left tile_counter[0] nonzero
  double *hsum;                  // pinned host word for heat_sum
  double *xstage;                // HEAT_F32C host transfers: two binary64 staging chunks (lazy)
  int64_t wait_ns;
  int32_t inj_segment;
  int64_t inj_step;
};

namespace heat {

// Launchers (each queues work on c->stream and returns a heat_status).
int run_plain(heat_ctx *c, int64_t nt);
int run_persist(heat_ctx *c, int64_t nt);
int run_queue(heat_ctx *c, int64_t nt, int T);
int persist_default_T(const heat_ctx *c);
int prepare_segments(heat_ctx *c, int S, const int64_t *bounds);
int run_tblock(heat_ctx *c, int64_t nt);
int tblock_default_T(const heat_ctx *c);
unsigned tblock_emul_mask(const heat_ctx *c);
int run_cluster(heat_ctx *c, int64_t nt);
int run_persist_tb(heat_ctx *c, int64_t nt);
int run_wave(heat_ctx *c, int64_t nt, int T);
int wave_default_T(const heat_ctx *c);
bool wave_preferred(const heat_ctx *c);
void free_wave(heat_ctx *c);
int64_t cluster_max_points(const heat_ctx *c, int T);
int sum_state(heat_ctx *c, double *out);
int convert_f64_to_state(heat_ctx *c, const double *dev_src, void *dev_dst, int64_t n);
int convert_state_to_f64(heat_ctx *c, const void *dev_src, double *dev_dst, int64_t n);

// Number of reduction partials heat_sum uses (fixed, so the tree is fixed).
constexpr int kSumBlocks = 1024;
constexpr int kSumThreads = 256;

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? HEAT_OK : HEAT_ECUDA; }

// `share` set bits spread evenly over tile index mod 32.
inline unsigned emul_share_mask(int share) {
  unsigned mask = 0;
  for (int i = 0; i < 32; ++i)
    if (((i + 1) * share) / 32 > (i * share) / 32) mask |= 1u << i;
  return mask;
}

// The library's share of binary64 tiles on the integer pipes for multiplier r
// (out of 32): half.  The FP64 unit and the integer pipes each advance the
// ring at about the same rate (for r = +-2^k both get faster: the product
// only moves the exponent, on the integer pipes in either kind of tile).
inline int emul_auto_share(double) { return 16; }

}  // namespace heat

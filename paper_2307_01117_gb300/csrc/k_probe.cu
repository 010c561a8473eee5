// k_probe.cu -- heat_probe_pipes: measured issue rates of the two engines the
// binary64 update runs on, for the roofline denominators.
//
// Each probe kernel runs a fixed number of independent dependency chains per
// thread on a full-occupancy grid (2048 threads per SM) and is timed with CUDA
// events on its stream, after one untimed launch:
//   FP64 FMA: x = fma(x, a, b)       eight chains, one DFMA per link
//   FP64 ADD: x = x + c              eight chains, one DADD per link
//   ALU:      bitwise majority of three of eight rotating words, one LOP3
//                                    per update, eight per round
// The lane-operation counts are those of the source; the pipe each kind lands
// on is checked with ncu's per-pipe instruction counters.  The chains' results
// are stored only when they reach an impossible value, which keeps them live.
#include <cuda_runtime.h>

#include "heat_internal.cuh"

namespace heat {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSM = 8;
constexpr int kFpIters = 4096;
constexpr int kAluIters = 8192;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) k_probe_dfma(double *sink, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < kFpIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __fma_rn(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.0) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_dadd(double *sink, double c0) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < kFpIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __dadd_rn(x[c], c0);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.0) sink[blockIdx.x] = s;
}

// Integer ALU pipe: eight 32-bit words, each round replaces word c by the
// bitwise majority of words c, c+1 and c+3 (one LOP3 each, eight per round).
// Every operand changes every round and two dependent majorities take five
// distinct inputs, so no two LOP3 merge and nothing is loop-invariant; LOP3
// issues only to the ALU pipe.
__device__ __forceinline__ unsigned maj3(unsigned a, unsigned b, unsigned c) {
  unsigned d;
  asm("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_alu(unsigned *sink, unsigned seed) {
  unsigned x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (seed + threadIdx.x * 7919u + blockIdx.x * 104729u) * (2654435761u + c);
  for (int i = 0; i < kAluIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = maj3(x[c], x[(c + 1) % kChains], x[(c + 3) % kChains]);
  }
  unsigned s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 0xdeadbeefu && seed == 0u) sink[blockIdx.x] = s;
}

// Milliseconds of one launch (the second of two) of `launch` on stream st.
template <class F>
int time_launch(cudaStream_t st, F launch, float *ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return HEAT_ECUDA;
  }
  launch();
  cudaEventRecord(e0, st);
  launch();
  cudaEventRecord(e1, st);
  int rc = cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess ? HEAT_OK : HEAT_ECUDA;
  if (rc == HEAT_OK && cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) rc = HEAT_ECUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace
}  // namespace heat

extern "C" int heat_probe_pipes(void *cuda_stream, double *dfma_lane_ops_per_s, double *dadd_lane_ops_per_s,
                                double *alu_lane_ops_per_s) {
  using namespace heat;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return HEAT_ECUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int grid = sms * kProbeBlocksPerSM;
  void *sink = nullptr;
  if (cudaMalloc(&sink, (size_t)grid * sizeof(double)) != cudaSuccess) return HEAT_ENOMEM;
  const double threads = (double)grid * kProbeThreads;
  float ms = 0.0f;
  int rc = time_launch(st, [&] { k_probe_dfma<<<grid, kProbeThreads, 0, st>>>((double *)sink, 0.999999, 1e-6); },
                       &ms);
  if (rc == HEAT_OK && dfma_lane_ops_per_s) *dfma_lane_ops_per_s = threads * kFpIters * kChains / (ms * 1e-3);
  if (rc == HEAT_OK)
    rc = time_launch(st, [&] { k_probe_dadd<<<grid, kProbeThreads, 0, st>>>((double *)sink, 1e-9); }, &ms);
  if (rc == HEAT_OK && dadd_lane_ops_per_s) *dadd_lane_ops_per_s = threads * kFpIters * kChains / (ms * 1e-3);
  if (rc == HEAT_OK)
    rc = time_launch(st, [&] { k_probe_alu<<<grid, kProbeThreads, 0, st>>>((unsigned *)sink, 12345u); }, &ms);
  if (rc == HEAT_OK && alu_lane_ops_per_s) *alu_lane_ops_per_s = threads * kAluIters * kChains / (ms * 1e-3);
  cudaFree(sink);
  return rc;
}

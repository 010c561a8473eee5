// k_reduce.cu -- the FP64 conservation diagnostic sum(u) and the binary64 <->
// state-dtype conversions.
//
// sum(u) is invariant under Eq. 2 on the periodic ring (the second differences
// telescope around the loop), which makes it the run-time check of a step.  The
// reduction has a fixed shape -- kSumBlocks blocks over fixed index ranges,
// fixed-stride per-thread sums, a fixed shared-memory tree, then one block over
// the partials -- so the result does not depend on scheduling or on the GPU's
// SM count.
#include "heat_internal.cuh"

namespace heat {
namespace {

template <typename T>
__device__ __forceinline__ double widen(T x) { return (double)x; }

template <typename T>
__global__ void __launch_bounds__(kSumThreads) k_sum_partials(const T *__restrict__ u, int64_t N,
                                                              double *__restrict__ partials) {
  __shared__ double sh[kSumThreads];
  const int64_t chunk = (N + kSumBlocks - 1) / kSumBlocks;
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = lo + chunk < N ? lo + chunk : N;
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kSumThreads) s = __dadd_rn(s, widen(u[i]));
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kSumThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] = __dadd_rn(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(1024) k_sum_final(const double *__restrict__ partials, double *__restrict__ out) {
  __shared__ double sh[1024];
  static_assert(kSumBlocks == 1024, "final tree assumes 1024 partials");
  sh[threadIdx.x] = partials[threadIdx.x];
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] = __dadd_rn(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

__global__ void k_f64_to_f32(const double *__restrict__ src, float *__restrict__ dst, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    dst[i] = __double2float_rn(src[i]);
}

__global__ void k_f32_to_f64(const float *__restrict__ src, double *__restrict__ dst, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = (double)src[i];
}

int conv_grid(const heat_ctx *c, int64_t n) {
  int64_t b = (n + 255) / 256;
  const int64_t cap = (int64_t)c->sms * 8;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

// Queues the two reduction kernels; *out is a device word.
int sum_state(heat_ctx *c, double *dev_out) {
  const int64_t N = c->geo.N;
  if (c->dtype == HEAT_F64)
    k_sum_partials<double><<<kSumBlocks, kSumThreads, 0, c->stream>>>((const double *)c->buf[c->cur], N, c->partials);
  else
    k_sum_partials<float><<<kSumBlocks, kSumThreads, 0, c->stream>>>((const float *)c->buf[c->cur], N, c->partials);
  k_sum_final<<<1, 1024, 0, c->stream>>>(c->partials, dev_out);
  return cuda_status(cudaGetLastError());
}

int convert_f64_to_state(heat_ctx *c, const double *dev_src, void *dev_dst, int64_t n) {
  k_f64_to_f32<<<conv_grid(c, n), 256, 0, c->stream>>>(dev_src, (float *)dev_dst, n);
  return cuda_status(cudaGetLastError());
}

int convert_state_to_f64(heat_ctx *c, const void *dev_src, double *dev_dst, int64_t n) {
  k_f32_to_f64<<<conv_grid(c, n), 256, 0, c->stream>>>((const float *)dev_src, dev_dst, n);
  return cuda_status(cudaGetLastError());
}

}  // namespace heat

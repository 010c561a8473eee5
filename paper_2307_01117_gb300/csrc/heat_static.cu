// heat_static.cu -- heat_run_noalloc: the plain binary64 stepper for callers
// that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured (allocation is not a capturable operation), real-time loops
// that may not touch the allocator, and hosts whose memory is owned by another
// framework's pool.  They still need the ping-pong buffer that a multi-step run
// uses besides its input and output.  Here that buffer is a fixed file-scope
// device array of kNoAllocMaxN binary64 values (8 MiB), created with the module
// on every GPU that loads this library and held until the process exits.
//
// Host code never uses the array's name as an address (on the host it is a
// stand-in, not device memory): the first call on each device, with that device
// current, asks the runtime for the array's device address with
// cudaGetSymbolAddress, checks the result and caches it; kernels get that
// pointer.  Every call on a device shares the one array and leaves the last
// call's values in it; nothing needs clearing, because every step writes every
// element of its destination before any later step reads it.
#include <mutex>

#include "heat_internal.cuh"
#include "stencil_ops.cuh"

namespace heat {
namespace {

constexpr int64_t kNoAllocMaxN = int64_t(1) << 20;
constexpr int kMaxDevices = 256;
constexpr int kThreads = 256;
constexpr unsigned kFullMask = 0xffffffffu;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxN];

std::mutex g_setup_mu;
double *g_scratch_addr[kMaxDevices];  // device address per device ordinal (null until set up)
int g_sms[kMaxDevices];

// One step of Eq. 2 over the ring, the plain form's tiling: 64-point warp
// tiles, 16-byte vectors, in-tile neighbours by shuffle, scalar tail.
template <bool FMA>
__global__ void __launch_bounds__(kThreads) k_plain_f64_noalloc(const double *__restrict__ u, double *__restrict__ v,
                                                                int64_t N, double r) {
  const int lane = threadIdx.x & 31;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t warp = gtid >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t ntiles = N >> 6;
  for (int64_t t = warp; t < ntiles; t += nwarps) {
    const int64_t b = t << 6;
    const double2 x = reinterpret_cast<const double2 *>(u + b)[lane];
    double left = __shfl_up_sync(kFullMask, x.y, 1);
    double right = __shfl_down_sync(kFullMask, x.x, 1);
    if (lane == 0) left = u[b == 0 ? N - 1 : b - 1];
    if (lane == 31) right = u[b + 64 == N ? 0 : b + 64];
    double2 y;
    y.x = eq2<FMA>(left, x.x, x.y, r);
    y.y = eq2<FMA>(x.x, x.y, right, r);
    reinterpret_cast<double2 *>(v + b)[lane] = y;
  }
  const int64_t tail0 = ntiles << 6;
  if (gtid < N - tail0) {
    const int64_t g = tail0 + gtid;
    const double ul = u[g == 0 ? N - 1 : g - 1];
    const double ur = u[g + 1 == N ? 0 : g + 1];
    v[g] = eq2<FMA>(ul, u[g], ur, r);
  }
}

// Per-device set-up: the scratch array's device address and the SM count.
// Both kernel instantiations are loaded here too (cudaFuncGetAttributes loads
// a lazily loaded kernel), so that no later call, in either arithmetic, makes
// the driver load code or allocate memory for it.
int device_setup(int dev, double **scratch, int *sms) {
  if (dev < 0 || dev >= kMaxDevices) return HEAT_ENOTSUP;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return HEAT_ECUDA;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return HEAT_ECUDA;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_plain_f64_noalloc<false>) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, k_plain_f64_noalloc<true>) != cudaSuccess)
      return HEAT_ECUDA;
    g_sms[dev] = n;
    g_scratch_addr[dev] = (double *)p;
  }
  *scratch = g_scratch_addr[dev];
  *sms = g_sms[dev];
  return HEAT_OK;
}

// The stream must belong to the current device: the scratch address and the
// launches are the current device's.  NULL and the two special handles
// (legacy and per-thread default streams) always do.
bool stream_on_device(cudaStream_t st, int dev) {
  if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread) return true;
  int sdev = -1;
  return cudaStreamGetDevice(st, &sdev) == cudaSuccess && sdev == dev;
}

bool overlaps(const double *a, const double *b, int64_t n) {
  const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b, len = (uintptr_t)n * sizeof(double);
  return pa < pb + len && pb < pa + len;
}

}  // namespace
}  // namespace heat

extern "C" int heat_run_noalloc(const double *dev_u0, double *dev_u, int64_t n, double k, double dt, double dx,
                                int64_t nt, int arith, void *cuda_stream) {
  using namespace heat;
  if (!dev_u0 || !dev_u || n < 1 || nt < 0) return HEAT_EINVAL;
  if (n > kNoAllocMaxN) return HEAT_EINVAL;
  if (arith != HEAT_ARITH_EXACT && arith != HEAT_ARITH_FMA) return HEAT_EINVAL;
  if (!isfinite(k) || !isfinite(dt) || !isfinite(dx) || dx == 0.0) return HEAT_EINVAL;
  if (((uintptr_t)dev_u0 | (uintptr_t)dev_u) & 15u) return HEAT_EINVAL;
  if (overlaps(dev_u0, dev_u, n)) return HEAT_EINVAL;
  const double r = (k * dt) / (dx * dx);
  if (!isfinite(r)) return HEAT_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HEAT_ECUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (!stream_on_device(st, dev)) return HEAT_EINVAL;
  double *scratch = nullptr;
  int sms = 0;
  int rc = device_setup(dev, &scratch, &sms);
  if (rc != HEAT_OK) return rc;
  // an error left pending by earlier work on this thread is reported, not
  // cleared, and nothing is queued
  if (cudaPeekAtLastError() != cudaSuccess) return HEAT_ECUDA;
  if (nt == 0)
    return cudaMemcpyAsync(dev_u, dev_u0, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st) == cudaSuccess
               ? HEAT_OK
               : HEAT_ECUDA;
  int64_t blocks = ((n >> 6) + kThreads / 32 - 1) / (kThreads / 32);
  if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
  if (blocks < 1) blocks = 1;
  // step s writes the output when (nt - s) is even, else the scratch array, so
  // the last step lands in dev_u and dev_u0 is only ever read
  const double *src = dev_u0;
  for (int64_t s = 1; s <= nt; ++s) {
    double *dst = ((nt - s) & 1) ? scratch : dev_u;
    if (arith == HEAT_ARITH_FMA)
      k_plain_f64_noalloc<true><<<(int)blocks, kThreads, 0, st>>>(src, dst, n, r);
    else
      k_plain_f64_noalloc<false><<<(int)blocks, kThreads, 0, st>>>(src, dst, n, r);
    if (cudaGetLastError() != cudaSuccess) return HEAT_ECUDA;
    src = dst;
  }
  return HEAT_OK;
}

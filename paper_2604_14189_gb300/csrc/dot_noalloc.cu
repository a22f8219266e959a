// sweep_dot_noalloc: the FP64 dot product of sweep_dot for callers that
// cannot allocate device memory (for example a plugin whose host application
// owns the whole device-memory budget, or a loop that must not allocate after
// start-up).  Its partial sums live in a fixed file-scope device array that
// every GPU loading this library holds until the process exits, so the call
// needs no workspace.
//
// Each block of 256 threads reduces one chunk of 4096 consecutive products
// into one slot of the array; one more block sums the slots in a fixed
// order.  Every call overwrites the slots it reads, so nothing has to be
// cleared between calls; calls that overlap on the GPU share the array and
// race.  The first call on a device looks the array's device address up (for
// the device current on the calling thread) and caches it, so that call
// should come before any stream capture.
#include <mutex>

#include "sweep_internal.cuh"

namespace sweep {
namespace {

constexpr int kThreads = 256;
constexpr long long kChunk = 4096;
constexpr int kMaxSlots = (int)(SWEEP_DOT_NOALLOC_MAX_N / kChunk);
static_assert((long long)kMaxSlots * kChunk == SWEEP_DOT_NOALLOC_MAX_N, "whole chunks");

// Partial sums shared by every call on a device (kMaxSlots doubles = 64 KiB).
static __device__ __align__(256) double g_dot_slots[kMaxSlots];

__device__ double block_total(double v) {
  __shared__ double sh[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kThreads / 32; ++i) t += sh[i];
  return t;  // valid in thread 0
}

__global__ void __launch_bounds__(kThreads) chunk_kernel(const float* __restrict__ a,
                                                         const float* __restrict__ b, long long n,
                                                         double* slots) {
  const long long base = (long long)blockIdx.x * kChunk;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < kChunk; i += kThreads) {
    const long long k = base + i;
    if (k < n) acc += (double)a[k] * (double)b[k];
  }
  const double t = block_total(acc);
  if (threadIdx.x == 0) slots[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kThreads) total_kernel(const double* slots, int nslots,
                                                         double* out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nslots; i += kThreads) acc += slots[i];
  const double t = block_total(acc);
  if (threadIdx.x == 0) *out = t;
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_slots_dev[kMaxDevices] = {};

// Device address of g_dot_slots on the current device (looked up once).
int slots_address(double** p) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return SWEEP_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return SWEEP_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_slots_dev[dev]) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_dot_slots) != cudaSuccess || !addr) {
      // take the failed lookup's error out of the runtime's last-error slot,
      // so that the next call's launch check does not report it again
      (void)cudaGetLastError();
      return SWEEP_ECUDA;
    }
    g_slots_dev[dev] = static_cast<double*>(addr);
  }
  *p = g_slots_dev[dev];
  return SWEEP_OK;
}

}  // namespace
}  // namespace sweep

extern "C" int sweep_dot_noalloc(const float* a, const float* b, int64_t n, double* out,
                                 void* stream) {
  using namespace sweep;
  if (n < 0 || !out || (n > 0 && (!a || !b))) return SWEEP_EINVAL;
  if (n > SWEEP_DOT_NOALLOC_MAX_N) return SWEEP_ETOOBIG;
  double* slots = nullptr;
  int rc = slots_address(&slots);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nslots = (int)((n + kChunk - 1) / kChunk);
  if (nslots > 0) chunk_kernel<<<nslots, kThreads, 0, st>>>(a, b, n, slots);
  total_kernel<<<1, kThreads, 0, st>>>(slots, nslots, out);
  note_launches(nslots > 0 ? 2 : 1);
  return cudaGetLastError() == cudaSuccess ? SWEEP_OK : SWEEP_ECUDA;
}

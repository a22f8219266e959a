// Diagnostic: the device-side timeout path.
//
// Every pipeline wait of the library is bounded (tma.cuh): a wait that runs
// out latches SWEEP_ETIMEOUT in the workspace status word and the kernel
// returns, so the context stays usable.  This kernel makes one such wait run
// out on purpose: it initialises an mbarrier that nothing will ever arrive
// on, waits for it with the library's bounded wait, and latches the result.
// Nothing is in flight and no memory is touched but the status word.
#include "sweep_internal.cuh"
#include "tma.cuh"

namespace sweep {
namespace {

__global__ void wait_timeout_kernel(int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_barrier_init();
  if (!mbar_wait(&bar, 0)) latch(status, SWEEP_ETIMEOUT);
  mbar_inval(&bar);
}

}  // namespace
}  // namespace sweep

extern "C" int sweep_check_wait_timeout(void* ws, size_t ws_bytes, void* stream) {
  using namespace sweep;
  if (!ws || ws_bytes < sizeof(int) || (reinterpret_cast<uintptr_t>(ws) % 256) != 0)
    return SWEEP_EWORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* status = static_cast<int*>(ws);  // the status word leads every workspace
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return SWEEP_ECUDA;
  wait_timeout_kernel<<<1, 32, 0, st>>>(status);
  note_launches(1);
  return cudaGetLastError() == cudaSuccess ? SWEEP_OK : SWEEP_ECUDA;
}

extern "C" int sweep_check_barrier_timeout(void* ws, size_t ws_bytes, void* stream) {
  using namespace sweep;
  if (!ws || ws_bytes < 128 || (reinterpret_cast<uintptr_t>(ws) % 256) != 0)
    return SWEEP_EWORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* status = static_cast<int*>(ws);
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return SWEEP_ECUDA;
  // scratch words past the status word (the status area is 16 bytes; the
  // workspace's next region starts 256 bytes in)
  unsigned* bar = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + 64);
  const int rc = launch_barrier_timeout_check(bar, status, st);
  return rc ? rc : (cudaGetLastError() == cudaSuccess ? SWEEP_OK : SWEEP_ECUDA);
}

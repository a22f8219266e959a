// CUDA-graph capture of library calls.
//
// A modelling job repeats the same call thousands of times with the same
// buffers (an FWI loop, a batch of equal problems, a benchmark); a captured
// graph replays every kernel of a call with one host call, and its kernels
// keep their programmatic-launch edges.  The capture is thread-local on the
// caller's stream: sweep_capture_begin starts it, any number of library calls
// on that stream from the same thread are recorded instead of run, and
// sweep_capture_end instantiates the graph.  Launch accounting: recorded
// calls count no launches; every sweep_graph_launch counts the graph's kernel
// nodes.
#include <new>
#include <vector>

#include "sweep_internal.cuh"

namespace sweep {

thread_local bool t_capturing = false;

namespace {

struct Graph {
  cudaGraphExec_t exec;
  int kernels;
};

int count_kernels(cudaGraph_t g, int* kernels) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return SWEEP_ECUDA;
  std::vector<cudaGraphNode_t> nodes(n);
  if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return SWEEP_ECUDA;
  int k = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess) return SWEEP_ECUDA;
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  *kernels = k;
  return SWEEP_OK;
}

}  // namespace
}  // namespace sweep

extern "C" int sweep_capture_begin(void* stream) {
  using namespace sweep;
  if (!stream) return SWEEP_EINVAL;  // the legacy default stream cannot be captured
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return SWEEP_ECUDA;
  if (cs != cudaStreamCaptureStatusNone || t_capturing) return SWEEP_EINVAL;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return SWEEP_ECUDA;
  t_capturing = true;
  return SWEEP_OK;
}

extern "C" int sweep_capture_end(void* stream, void** graph) {
  using namespace sweep;
  if (!stream || !graph) return SWEEP_EINVAL;
  *graph = nullptr;
  if (!t_capturing) return SWEEP_EINVAL;
  t_capturing = false;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(st, &g) != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();  // the failed capture's error is reported as ECUDA
    return SWEEP_ECUDA;
  }
  int kernels = 0;
  int rc = count_kernels(g, &kernels);
  cudaGraphExec_t exec = nullptr;
  if (rc == SWEEP_OK && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) rc = SWEEP_ECUDA;
  cudaGraphDestroy(g);
  if (rc != SWEEP_OK) return rc;
  Graph* h = new (std::nothrow) Graph{exec, kernels};
  if (!h) {
    cudaGraphExecDestroy(exec);
    return SWEEP_ECUDA;
  }
  *graph = h;
  return SWEEP_OK;
}

extern "C" int sweep_graph_launch(void* graph, void* stream) {
  using namespace sweep;
  if (!graph) return SWEEP_EINVAL;
  Graph* h = static_cast<Graph*>(graph);
  if (cudaGraphLaunch(h->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return SWEEP_ECUDA;
  note_launches(h->kernels);
  return SWEEP_OK;
}

extern "C" int sweep_graph_kernels(void* graph) {
  return graph ? static_cast<sweep::Graph*>(graph)->kernels : SWEEP_EINVAL;
}

extern "C" void sweep_graph_destroy(void* graph) {
  if (!graph) return;
  sweep::Graph* h = static_cast<sweep::Graph*>(graph);
  cudaGraphExecDestroy(h->exec);
  delete h;
}

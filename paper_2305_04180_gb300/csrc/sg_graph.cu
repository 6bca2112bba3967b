// sg_graph.cu -- CUDA-graph capture and replay of library calls.
//
// A K-step rollout (and, for the actor-learner loop, the learner steps that
// follow it) is enqueued once under stream capture and replayed as one
// executable graph.  Every kernel of the library keeps its counters on the
// device (per-env step counts, ring position, optimiser step), so each replay
// continues where the previous one stopped.
#include <cuda_runtime.h>

#include <new>

#include "sg_host.h"
#include "sparrow_gb.h"

struct sg_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t nodes = 0;
};

#define SG_CUDA(call)                                           \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return sg_set_cuda_error(e_, #call); \
  } while (0)

extern "C" int sg_graph_begin(sg_stream_t stream) {
  SG_RANGE("sg_graph_begin");
  if (!stream) return SG_E_INVAL;  // the legacy default stream cannot be captured
  SG_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
  return SG_OK;
}

extern "C" int sg_graph_end(sg_stream_t stream, sg_graph_t* out) {
  SG_RANGE("sg_graph_end");
  if (!stream || !out) return SG_E_INVAL;
  *out = nullptr;
  cudaGraph_t g = nullptr;
  SG_CUDA(cudaStreamEndCapture(stream, &g));
  sg_graph* h = new (std::nothrow) sg_graph();
  if (!h) {
    cudaGraphDestroy(g);
    return SG_E_OOM;
  }
  h->graph = g;
  cudaError_t e = cudaGraphInstantiate(&h->exec, g, 0);
  if (e == cudaSuccess) e = cudaGraphGetNodes(g, nullptr, &h->nodes);
  if (e != cudaSuccess) {
    if (h->exec) cudaGraphExecDestroy(h->exec);
    cudaGraphDestroy(g);
    delete h;
    return sg_set_cuda_error(e, "sg_graph_end");
  }
  *out = h;
  return SG_OK;
}

extern "C" int sg_graph_launch(sg_graph_t g, sg_stream_t stream) {
  SG_RANGE("sg_graph_launch");
  if (!g) return SG_E_INVAL;
  SG_CUDA(cudaGraphLaunch(g->exec, stream));
  return SG_OK;
}

extern "C" int sg_graph_num_nodes(sg_graph_t g, int64_t* n) {
  SG_RANGE("sg_graph_num_nodes");
  if (!g || !n) return SG_E_INVAL;
  *n = (int64_t)g->nodes;
  return SG_OK;
}

extern "C" int sg_graph_destroy(sg_graph_t g) {
  SG_RANGE("sg_graph_destroy");
  if (!g) return SG_E_INVAL;
  cudaGraphExecDestroy(g->exec);
  cudaGraphDestroy(g->graph);
  delete g;
  return SG_OK;
}

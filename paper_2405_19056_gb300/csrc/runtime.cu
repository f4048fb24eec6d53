// Host runtime around the fused path: CUDA graphs of batched launches (one
// per batch shape), so a frame loop replays a fixed launch sequence instead of
// rebuilding it.  The paper has no counterpart (Sec. 5 reports per-frame
// render times only); this is the launch machinery of a serving deployment.
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

namespace {

int cuda_err(cudaError_t e, const char* what) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  return gn::set_error(GN_ECUDA, buf);
}

// Captures the plan + fused launch of `p` (and a 3x3 R's kernels) on a
// private stream.
int capture(const gn_model* m, const gn::FusedParams& p, cudaGraph_t* graph) {
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_err(e, "create capture stream");
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const cudaError_t el = gn::launch_render(m, p, cs);
    e = cudaStreamEndCapture(cs, graph);
    if (el != cudaSuccess) e = el;
  }
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return cuda_err(e, "capture of the fused launch");
  return GN_OK;
}

bool same_shapes(const gn::FusedParams& a, const gn::FusedParams& b) {
  if (a.nframes != b.nframes || a.total_tiles != b.total_tiles) return false;
  for (int i = 0; i < a.nframes; ++i)
    if (a.f[i].P != b.f[i].P || a.f[i].w != b.f[i].w || a.f[i].K != b.f[i].K) return false;
  return true;
}

}  // namespace

struct gn_graph {
  const gn_model* model = nullptr;
  gn::FusedParams params;  // as captured (shapes are fixed for the graph's life)
  void* ws = nullptr;      // tile plan owned by this graph
  cudaGraphExec_t exec = nullptr;
};

extern "C" {

int glassnet_graph_create(const gn_model* m, const gn_frame* frames, int n, gn_graph** out) {
  if (!out) return gn::set_error(GN_EINVAL, "out must be non-NULL");
  *out = nullptr;
  gn::FusedParams p;
  int rc = gn::build_batch(m, frames, n, &p);
  if (rc != GN_OK) return rc;
  cudaError_t e = gn::prepare_fused(m);
  if (e != cudaSuccess) return cuda_err(e, "kernel attributes");
  gn_graph* g = new (std::nothrow) gn_graph();
  if (!g) return gn::set_error(GN_ENOMEM, "host allocation failed");
  g->model = m;
  const size_t bytes = gn::batch_ws_bytes(m, p);
  if ((e = cudaMalloc(&g->ws, bytes)) != cudaSuccess) {
    delete g;
    return gn::set_error(GN_ENOMEM, "cudaMalloc graph tile plan");
  }
  gn::bind_batch_ws(m, p, g->ws);
  cudaGraph_t graph = nullptr;
  if ((rc = capture(m, p, &graph)) != GN_OK) {
    glassnet_graph_free(g);
    return rc;
  }
  e = cudaGraphInstantiate(&g->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    glassnet_graph_free(g);
    return cuda_err(e, "instantiate graph");
  }
  // upload it now, so that its first launch does not pay for that
  cudaStream_t us = nullptr;
  if ((e = cudaStreamCreateWithFlags(&us, cudaStreamNonBlocking)) == cudaSuccess) {
    e = cudaGraphUpload(g->exec, us);
    if (e == cudaSuccess) e = cudaStreamSynchronize(us);
    cudaStreamDestroy(us);
  }
  if (e != cudaSuccess) {
    glassnet_graph_free(g);
    return cuda_err(e, "upload graph");
  }
  g->params = p;
  *out = g;
  return GN_OK;
}

int glassnet_graph_launch(gn_graph* g, cudaStream_t stream) {
  if (!g || !g->exec) return gn::set_error(GN_EINVAL, "graph is NULL");
  const cudaError_t e = cudaGraphLaunch(g->exec, stream);
  if (e != cudaSuccess) return cuda_err(e, "graph launch");
  return GN_OK;
}

int glassnet_graph_update(gn_graph* g, const gn_frame* frames, int n) {
  if (!g || !g->exec) return gn::set_error(GN_EINVAL, "graph is NULL");
  gn::FusedParams p;
  int rc = gn::build_batch(g->model, frames, n, &p);
  if (rc != GN_OK) return rc;
  if (!same_shapes(p, g->params))
    return gn::set_error(GN_EINVAL, "frame count, sizes or K differ from the captured batch");
  gn::bind_batch_ws(g->model, p, g->ws);
  cudaGraph_t graph = nullptr;
  if ((rc = capture(g->model, p, &graph)) != GN_OK) return rc;
  cudaGraphExecUpdateResultInfo info;
  cudaError_t e = cudaGraphExecUpdate(g->exec, graph, &info);
  if (e != cudaSuccess) {
    // topology changed unexpectedly: instantiate afresh
    cudaGetLastError();
    cudaGraphExec_t fresh = nullptr;
    e = cudaGraphInstantiate(&fresh, graph, 0);
    if (e == cudaSuccess) {
      cudaGraphExecDestroy(g->exec);
      g->exec = fresh;
    }
  }
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_err(e, "graph update");
  g->params = p;
  return GN_OK;
}

void glassnet_graph_free(gn_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->ws) cudaFree(g->ws);
  delete g;
}

}  // extern "C"

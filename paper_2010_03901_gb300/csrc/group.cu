// Plan groups: several domains' extension + DFT pipelines (steps 5-7 of Section 3.5) as
// one CUDA graph.  Each plan runs on its own branch (forked from the launching stream and
// joined back), so the kernels of small domains run side by side instead of one after
// another; the graph is captured on the first call and replayed while the arguments
// (function counts and pointers) and every plan's workspace (base and size) stay the
// same, re-captured when any of them changes.  The workspace is part of the key because
// the captured kernels hold its address: a later call on a member plan that needs more
// workspace frees the old one and allocates another, and a replay of the old graph would
// then read and write freed memory.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "../../include/fc2d.h"
#include "plan_internal.h"

namespace fc2d {
fc2d_status ensure_plan_workspace(fc2d_plan_s* p, int n_f);  // capi.cu
}

struct fc2d_group_s {
  std::vector<fc2d_plan_t> plans;
  std::vector<cudaStream_t> branch;       // one capture stream per plan
  cudaStream_t cap = nullptr;             // the capture origin
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int> key_nf;                // arguments of the captured graph
  std::vector<const void*> key_ptr;
};

using namespace fc2d;

static void group_free(fc2d_group_s* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  for (cudaEvent_t e : g->join)
    if (e) cudaEventDestroy(e);
  if (g->fork) cudaEventDestroy(g->fork);
  for (cudaStream_t s : g->branch)
    if (s) cudaStreamDestroy(s);
  if (g->cap) cudaStreamDestroy(g->cap);
  delete g;
}

extern "C" fc2d_status fc2d_group_create(const fc2d_plan_t* plans, int n, fc2d_group_t* out) {
  if (!plans || n < 1 || !out) return set_error(FC2D_ERR_ARG, "fc2d_group_create: bad argument");
  for (int i = 0; i < n; ++i) {
    if (!plans[i]) return set_error(FC2D_ERR_ARG, "fc2d_group_create: null plan");
    // the branches run concurrently on each plan's own workspace
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i])
        return set_error(FC2D_ERR_ARG, "fc2d_group_create: a plan appears twice");
  }
  auto* g = new fc2d_group_s();
  g->plans.assign(plans, plans + n);
  bool ok = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) == cudaSuccess;
  g->branch.assign(n, nullptr);
  g->join.assign(n, nullptr);
  for (int i = 0; ok && i < n; ++i)
    ok = cudaStreamCreateWithFlags(&g->branch[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&g->join[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    group_free(g);
    return set_error(FC2D_ERR_CUDA, "fc2d_group_create: stream or event creation failed");
  }
  *out = g;
  return FC2D_OK;
}

// Capture every plan's fc2d_extend_coeffs on its own branch into g->graph.
static fc2d_status capture(fc2d_group_s* g, const int* n_f, const double* const* fg,
                           const double* const* fb, void* const* fhat) {
  const int n = (int)g->plans.size();
  for (int i = 0; i < n; ++i) {
    // workspace first: no allocation may happen while the graph is being captured
    fc2d_status st = ensure_plan_workspace(g->plans[i], n_f[i]);
    if (st) return st;
  }
  if (cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return set_error(FC2D_ERR_CUDA, "fc2d_group: stream capture failed to start");
  fc2d_status st = FC2D_OK;
  cudaEventRecord(g->fork, g->cap);
  for (int i = 0; i < n && !st; ++i) {
    cudaStreamWaitEvent(g->branch[i], g->fork, 0);
    st = fc2d_extend_coeffs(g->plans[i], n_f[i], fg[i], fb ? fb[i] : nullptr, fhat[i],
                            g->branch[i]);
    cudaEventRecord(g->join[i], g->branch[i]);
    cudaStreamWaitEvent(g->cap, g->join[i], 0);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(g->cap, &graph);
  if (st) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess || !graph) return set_error(FC2D_ERR_CUDA, "fc2d_group: stream capture failed");
  if (g->exec) {
    cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
  }
  if (g->graph) cudaGraphDestroy(g->graph);
  g->graph = graph;
  if (cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) {
    g->exec = nullptr;
    return set_error(FC2D_ERR_CUDA, "fc2d_group: graph instantiation failed");
  }
  return FC2D_OK;
}

extern "C" fc2d_status fc2d_group_extend_coeffs(fc2d_group_t g, const int* n_f,
                                                const double* const* f_grid_dev,
                                                const double* const* f_bdry_dev,
                                                void* const* fhat_dev, void* stream) {
  if (!g || !n_f || !f_grid_dev || !fhat_dev)
    return set_error(FC2D_ERR_ARG, "fc2d_group_extend_coeffs: null argument");
  const int n = (int)g->plans.size();
  std::vector<int> knf(n_f, n_f + n);
  std::vector<const void*> kptr;
  for (int i = 0; i < n; ++i) {
    if (n_f[i] < 1 || !f_grid_dev[i] || !fhat_dev[i])
      return set_error(FC2D_ERR_ARG, "fc2d_group_extend_coeffs: bad entry");
    // grow the workspaces now (outside any capture), so that the key below holds the
    // buffers the kernels will use
    fc2d_status st = ensure_plan_workspace(g->plans[i], n_f[i]);
    if (st) return st;
  }
  for (int i = 0; i < n; ++i) {
    kptr.push_back(f_grid_dev[i]);
    kptr.push_back(f_bdry_dev ? f_bdry_dev[i] : nullptr);
    kptr.push_back(fhat_dev[i]);
    kptr.push_back(g->plans[i]->ws.base);
    kptr.push_back(reinterpret_cast<const void*>(g->plans[i]->ws.bytes));
  }
  if (!g->exec || knf != g->key_nf || kptr != g->key_ptr) {
    g->key_nf.clear();
    g->key_ptr.clear();
    fc2d_status st = capture(g, n_f, f_grid_dev, f_bdry_dev, fhat_dev);
    if (st) return st;
    g->key_nf = knf;
    g->key_ptr = kptr;
  }
  if (cudaGraphLaunch(g->exec, (cudaStream_t)stream) != cudaSuccess)
    return set_error(FC2D_ERR_CUDA, "fc2d_group: graph launch failed");
  return FC2D_OK;
}

extern "C" void fc2d_group_destroy(fc2d_group_t g) { group_free(g); }

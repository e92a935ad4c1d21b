// Plan groups: several domains' extension + DFT pipelines (steps 5-7 of Section 3.5) as
// one CUDA graph.  The strip-point values of every mixed-form member (the fused blend +
// interpolation, steps 5-6) come from one persistent kernel over all members' work items
// (plan, owner range, function), longest first; then each plan's row and column DFTs run
// on their own branch (forked from the launching stream and joined back), so the
// kernels of small domains run side by side.  FP64 members run their whole call on a
// branch.  The graph is captured on the first call and replayed while the arguments
// (function counts and pointers) and every plan's workspace (base and size) stay the
// same, re-captured when any of them changes.  The workspace is part of the key because
// the captured kernels hold its address: a later call on a member plan that needs more
// workspace frees the old one and allocates another, and a replay of the old graph would
// then read and write freed memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/fc2d.h"
#include "fc2d_kernels.cuh"
#include "plan_internal.h"

namespace fc2d {
// capi.cu
fc2d_status ensure_plan_workspace(fc2d_plan_s* p, int n_f);
fc2d_status extend_coeffs_check(fc2d_plan_s* p, int n_f, const double* fg, const double* fb,
                                const void* fhat);
fc2d_status extend_coeffs_dft(fc2d_plan_s* p, int n_f, const double* fg, void* fhat,
                              cudaStream_t s);
bool group_fused(const fc2d_plan_s* p);
GiPlanArgs group_fused_args(fc2d_plan_s* p, int n_f, const double* fg, const double* fb,
                            std::vector<int32_t>* points);
}  // namespace fc2d

// A work item's cost for the ordering: its strip points plus a fixed part for the
// tables, the gather of 64 normals and the MMAs (about as long as interpolating this
// many points).
constexpr int64_t kItemFixed = 256;

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
  // the persistent blend + interpolation kernel: per-plan records, work items, counter
  cudaEvent_t fork_dft = nullptr;         // after the persistent kernel
  void* work = nullptr;
  size_t work_cap = 0;
  int4* items = nullptr;
  size_t items_cap = 0;
  int* counter = nullptr;
  int nt = 0;                             // its threads per CTA (autotuned at capture)
  int persistent = 0;                     // the captured form (autotuned at capture)
  int forced_form = -1, forced_nt = 0;    // fc2d_group_tuning_set (-1: tune)
  // microseconds: queue kernel with 256 and 512 threads, graph with branches only,
  // graph with the queue kernel
  float tune_us[4] = {0.f, 0.f, 0.f, 0.f};
};

using namespace fc2d;

static void group_free(fc2d_group_s* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  for (cudaEvent_t e : g->join)
    if (e) cudaEventDestroy(e);
  if (g->fork) cudaEventDestroy(g->fork);
  if (g->fork_dft) cudaEventDestroy(g->fork_dft);
  if (g->work) cudaFree(g->work);
  if (g->items) cudaFree(g->items);
  if (g->counter) cudaFree(g->counter);
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
            cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->fork_dft, cudaEventDisableTiming) == cudaSuccess &&
            cudaMalloc(&g->counter, sizeof(int)) == cudaSuccess;
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

static fc2d_status grow(void** buf, size_t* cap, size_t bytes) {
  if (bytes <= *cap) return FC2D_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  if (cudaMalloc(buf, bytes) != cudaSuccess) {
    *buf = nullptr;
    return set_error(FC2D_ERR_CUDA, "fc2d_group: device allocation failed");
  }
  *cap = bytes;
  return FC2D_OK;
}

// Time the persistent kernel with 256 and 512 threads per CTA (two or one per SM) on the
// call's own inputs (it recomputes the same strip values), three launches each after
// one warm-up; keep the faster.
static fc2d_status tune_queue(fc2d_group_s* g, int n_items, int max_ldS, int n_sm) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return set_error(FC2D_ERR_CUDA, "fc2d_group: event creation failed");
  }
  fc2d_status st = FC2D_OK;
  const int shapes[2] = {256, 512};
  for (int k = 0; k < 2 && !st; ++k) {
    const int nt = shapes[k], n_cta = std::min(n_items, n_sm * (512 / nt));
    for (int r = 0; r < 4 && !st; ++r) {
      if (r == 1) cudaEventRecord(e0, g->cap);
      cudaMemsetAsync(g->counter, 0, sizeof(int), g->cap);
      st = launch_gather_interp_queue(g->work, g->items, n_items, g->counter, nt, max_ldS, n_cta,
                                      g->cap);
    }
    cudaEventRecord(e1, g->cap);
    if (!st && cudaEventSynchronize(e1) != cudaSuccess)
      st = set_error(FC2D_ERR_CUDA, "fc2d_group: tuning launch failed");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    g->tune_us[k] = 1e3f * ms / 3;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!st) g->nt = g->tune_us[0] <= g->tune_us[1] ? 256 : 512;
  return st;
}

// Capture one form of the group call into *graph.  persistent: the queue kernel over
// the mixed-form members' work items, then per plan the DFTs on its branch; otherwise
// every plan's whole call on its branch (the domains' blends then overlap the other
// domains' DFTs).  FP64 members run their whole call on a branch in both forms.
static fc2d_status capture_form(fc2d_group_s* g, bool persistent, const std::vector<char>& fused,
                                int n_items, int max_ldS, int n_sm, const int* n_f,
                                const double* const* fg, const double* const* fb,
                                void* const* fhat, cudaGraph_t* graph) {
  const int n = (int)g->plans.size();
  *graph = nullptr;
  if (cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return set_error(FC2D_ERR_CUDA, "fc2d_group: stream capture failed to start");
  fc2d_status st = FC2D_OK;
  cudaEventRecord(g->fork, g->cap);
  if (persistent) {
    cudaMemsetAsync(g->counter, 0, sizeof(int), g->cap);
    st = launch_gather_interp_queue(g->work, g->items, n_items, g->counter, g->nt, max_ldS,
                                    std::min(n_items, n_sm * (512 / g->nt)), g->cap);
    cudaEventRecord(g->fork_dft, g->cap);
  }
  for (int i = 0; i < n && !st; ++i) {
    const bool q = persistent && fused[i];
    cudaStreamWaitEvent(g->branch[i], q ? g->fork_dft : g->fork, 0);
    st = q ? extend_coeffs_dft(g->plans[i], n_f[i], fg[i], fhat[i], g->branch[i])
           : fc2d_extend_coeffs(g->plans[i], n_f[i], fg[i], fb ? fb[i] : nullptr, fhat[i],
                                g->branch[i]);
    cudaEventRecord(g->join[i], g->branch[i]);
    cudaStreamWaitEvent(g->cap, g->join[i], 0);
  }
  const cudaError_t e = cudaStreamEndCapture(g->cap, graph);
  if (st || e != cudaSuccess || !*graph) {
    if (*graph) cudaGraphDestroy(*graph);
    *graph = nullptr;
    return st ? st : set_error(FC2D_ERR_CUDA, "fc2d_group: stream capture failed");
  }
  return FC2D_OK;
}

// Mean microseconds of three launches of `exec` after one warm-up.
static float time_graph(fc2d_group_s* g, cudaGraphExec_t exec) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = -1.f;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    cudaGraphLaunch(exec, g->cap);
    cudaEventRecord(e0, g->cap);
    for (int r = 0; r < 3; ++r) cudaGraphLaunch(exec, g->cap);
    cudaEventRecord(e1, g->cap);
    if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return ms < 0.f ? -1.f : 1e3f * ms / 3;
}

// Capture the group call into g->graph / g->exec.  With mixed-form members both forms
// are captured and timed on the call's inputs, and the faster is kept (the plan-group
// autotuner; the persistent kernel's CTA shape is tuned first).
static fc2d_status capture(fc2d_group_s* g, const int* n_f, const double* const* fg,
                           const double* const* fb, void* const* fhat) {
  const int n = (int)g->plans.size();
  for (int i = 0; i < n; ++i) {
    // workspace first: no allocation may happen while the graph is being captured
    fc2d_status st = ensure_plan_workspace(g->plans[i], n_f[i]);
    if (st) return st;
    st = extend_coeffs_check(g->plans[i], n_f[i], fg[i], fb ? fb[i] : nullptr, fhat[i]);
    if (st) return st;
  }
  // the work items of the mixed-form members, longest first
  const size_t rec = gi_work_bytes();
  std::vector<char> fused(n, 0);
  std::vector<unsigned char> work;
  std::vector<int4> items;
  std::vector<int64_t> cost;
  int n_fused = 0, max_ldS = 0, n_sm = 1;
  for (int i = 0; i < n; ++i) {
    fc2d_plan_s* p = g->plans[i];
    if (!group_fused(p)) continue;
    std::vector<int32_t> pts;
    const GiPlanArgs a = group_fused_args(p, n_f[i], fg[i], fb ? fb[i] : nullptr, &pts);
    work.resize((size_t)(n_fused + 1) * rec);
    int ld = 0;
    fc2d_status st = gi_work_fill(a, work.data() + (size_t)n_fused * rec, &ld);
    if (st) return st;
    max_ldS = std::max(max_ldS, ld);
    n_sm = std::max(n_sm, p->n_sm);
    for (int c = 0; c < (int)pts.size(); ++c)
      for (int f = 0; f < n_f[i]; ++f) {
        items.push_back(make_int4(n_fused, c, f, 0));
        cost.push_back(pts[c] + kItemFixed);
      }
    fused[i] = 1;
    ++n_fused;
  }
  const int n_items = (int)items.size();
  // a replay of the previous graph may still be reading the old records, and the
  // tuning launches below write the plans' workspaces and outputs: let earlier work
  // finish
  cudaDeviceSynchronize();
  if (g->exec) {
    cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
  }
  if (g->graph) {
    cudaGraphDestroy(g->graph);
    g->graph = nullptr;
  }
  g->nt = 0;
  g->persistent = 0;
  for (float& u : g->tune_us) u = 0.f;
  if (n_items) {
    std::vector<int> order(n_items);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<int4> sorted(n_items);
    for (int k = 0; k < n_items; ++k) sorted[k] = items[order[k]];
    fc2d_status st = grow(&g->work, &g->work_cap, work.size());
    if (!st) st = grow(reinterpret_cast<void**>(&g->items), &g->items_cap, sorted.size() * sizeof(int4));
    if (st) return st;
    if (cudaMemcpy(g->work, work.data(), work.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->items, sorted.data(), sorted.size() * sizeof(int4), cudaMemcpyHostToDevice) !=
            cudaSuccess)
      return set_error(FC2D_ERR_CUDA, "fc2d_group: work upload failed");
    if (g->forced_form >= 0) g->nt = g->forced_nt;
    else if ((st = tune_queue(g, n_items, max_ldS, n_sm))) return st;
  }
  cudaGraph_t graphs[2] = {nullptr, nullptr};
  cudaGraphExec_t execs[2] = {nullptr, nullptr};
  fc2d_status st = FC2D_OK;
  // the forms to capture: both when tuning, the set one otherwise (branches only
  // without mixed-form members)
  const int first = (n_items && g->forced_form == 1) ? 1 : 0;
  const int last = (n_items && g->forced_form != 0) ? 1 : 0;
  for (int form = first; form <= last && !st; ++form) {
    st = capture_form(g, form == 1, fused, n_items, max_ldS, n_sm, n_f, fg, fb, fhat, &graphs[form]);
    if (!st && cudaGraphInstantiate(&execs[form], graphs[form], 0) != cudaSuccess) {
      execs[form] = nullptr;
      st = set_error(FC2D_ERR_CUDA, "fc2d_group: graph instantiation failed");
    }
  }
  int keep = first;
  if (!st && first != last) {
    g->tune_us[2] = time_graph(g, execs[0]);
    g->tune_us[3] = time_graph(g, execs[1]);
    if (g->tune_us[2] < 0.f || g->tune_us[3] < 0.f)
      st = set_error(FC2D_ERR_CUDA, "fc2d_group: tuning launch failed");
    keep = g->tune_us[3] < g->tune_us[2] ? 1 : 0;
  }
  for (int form = 0; form < 2; ++form) {
    if (!st && form == keep) continue;
    if (execs[form]) cudaGraphExecDestroy(execs[form]);
    if (graphs[form]) cudaGraphDestroy(graphs[form]);
  }
  if (st) return st;
  g->graph = graphs[keep];
  g->exec = execs[keep];
  g->persistent = keep;
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

extern "C" fc2d_status fc2d_group_tuning_set(fc2d_group_t g, const int32_t* choice) {
  if (!g) return set_error(FC2D_ERR_ARG, "fc2d_group_tuning_set: null group");
  if (choice && (choice[0] < 0 || choice[0] > 1 || (choice[1] != 256 && choice[1] != 512)))
    return set_error(FC2D_ERR_ARG, "fc2d_group_tuning_set: form 0 or 1, 256 or 512 threads");
  g->forced_form = choice ? choice[0] : -1;
  g->forced_nt = choice ? choice[1] : 0;
  g->key_nf.clear();  // the next call captures anew
  g->key_ptr.clear();
  return FC2D_OK;
}

extern "C" fc2d_status fc2d_group_tuning(fc2d_group_t g, int32_t* choice, float* us) {
  if (!g || !choice || !us) return set_error(FC2D_ERR_ARG, "fc2d_group_tuning: null argument");
  choice[0] = g->persistent;
  choice[1] = g->nt;
  for (int k = 0; k < 4; ++k) us[k] = g->tune_us[k];
  return FC2D_OK;
}

extern "C" void fc2d_group_destroy(fc2d_group_t g) { group_free(g); }

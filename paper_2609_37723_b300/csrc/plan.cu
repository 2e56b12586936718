// Batched ensembles: one CUDA graph over every configuration of an
// ensemble (elementals -> correlator -> GEVP per configuration, each with
// its own N_v), captured once and replayed by distil_plan_run, and an
// autotuner that picks the tensor-core kernel variant of each
// mode-contraction site from event timings of one timeslice.
//
// A configuration's correlators follow from its own eigenvectors and
// perambulators (Sec. 2.1); the configurations of an ensemble are
// independent, so the graph simply chains them on one stream, reusing one
// workspace: the largest configuration's elementals, then the largest
// elementals / correlator workspace.
#include <string.h>

#include <vector>

#include "common.cuh"
#include "prof.cuh"

struct distil_plan {
  distil_ctx* ctx;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  int tune[3];
  int kernels;
};

namespace distil {
namespace {

int elem_bytes(int mode) { return mode == DISTIL_FP32 ? 8 : 16; }  // complex element of phi / v and tau
size_t round256(size_t b) { return (b + 255) / 256 * 256; }

int check_shape(const distil_batch_shape* sh, const distil_batch_cfg* cfgs, int ncfg) {
  DISTIL_CHECK_ARG(sh != nullptr && cfgs != nullptr && ncfg >= 1, "distil_plan: null shape / cfgs or ncfg < 1");
  DISTIL_CHECK_ARG(sh->L >= 1 && sh->nt >= 1 && sh->np >= 1 && sh->nb >= 1 && sh->nb <= 16,
                   "distil_plan: bad L, nt, np or nb");
  DISTIL_CHECK_ARG(sh->t0 >= 0 && sh->t0 < sh->nt, "distil_plan: t0=%d outside [0,%d)", sh->t0, sh->nt);
  DISTIL_CHECK_ARG(sh->mom != nullptr, "distil_plan: null momentum list");
  for (int c = 0; c < ncfg; ++c) DISTIL_CHECK_ARG(cfgs[c].nv >= 1, "distil_plan: cfg %d has nv < 1", c);
  return DISTIL_OK;
}

// phi buffer bytes (largest configuration) and the rest of the workspace
int plan_sizes(const distil_batch_shape* sh, const distil_batch_cfg* cfgs, int ncfg, size_t* phi_b, size_t* rest_b) {
  size_t pb = 0, rb = 0;
  for (int c = 0; c < ncfg; ++c) {
    const int nv = cfgs[c].nv;
    const size_t phi = (size_t)sh->nt * sh->np * (size_t)comb3(nv) * elem_bytes(sh->mode);
    size_t we = 0, wc = 0;
    DISTIL_TRY(distil_elementals_workspace(sh->L, sh->nt, nv, sh->np, sh->mode, &we));
    DISTIL_TRY(distil_correlate_workspace(sh->nt, nv, sh->np, sh->nb, sh->mode, &wc));
    pb = phi > pb ? phi : pb;
    rb = we > rb ? we : rb;
    rb = wc > rb ? wc : rb;
  }
  *phi_b = round256(pb > 0 ? pb : 256);
  *rest_b = rb;
  return DISTIL_OK;
}

// The pipeline of one configuration (what the graph holds).
int run_cfg(distil_ctx* ctx, const distil_batch_shape* sh, const distil_batch_cfg& cf, void* phi, void* ws,
            size_t ws_bytes, distil_stream s) {
  DISTIL_TRY(distil_elementals(ctx, cf.v, sh->L, sh->nt, cf.nv, sh->mom, sh->np, sh->mode, phi, ws, ws_bytes, s));
  DISTIL_TRY(distil_correlate(ctx, phi, phi, cf.tau, sh->nt, cf.nv, sh->np, cf.prof, sh->nb, 0, sh->mode, cf.C, ws,
                              ws_bytes, s));
  if (cf.lambda) DISTIL_TRY(distil_gevp(ctx, cf.C, sh->np, sh->nb, sh->nt, sh->t0, cf.lambda, s));
  return DISTIL_OK;
}

// Summed event time of each mode-contraction site over one correlator call
// on the first timeslice of cfgs[0] (its elementals of t = 0 computed first).
int time_sites(distil_ctx* ctx, const distil_batch_shape* sh, const distil_batch_cfg& cf, void* phi, void* ws,
               size_t ws_bytes, distil_stream s, double ms[3]) {
  DISTIL_TRY(distil_elementals(ctx, cf.v, sh->L, 1, cf.nv, sh->mom, sh->np, sh->mode, phi, ws, ws_bytes, s));
  for (int rep = 0; rep < 2; ++rep) {  // the first run loads the kernels, the second is timed
    DISTIL_TRY(distil_profile_enable(ctx, rep == 1));
    DISTIL_TRY(distil_correlate(ctx, phi, phi, cf.tau, 1, cf.nv, sh->np, cf.prof, sh->nb, 0, sh->mode, cf.C, ws,
                                ws_bytes, s));
  }
  int n = 0;
  DISTIL_TRY(distil_profile_read(ctx, nullptr, 0, &n));
  std::vector<distil_kernel_stat> st(n > 0 ? n : 1);
  DISTIL_TRY(distil_profile_read(ctx, st.data(), n, &n));
  static const char* names[3] = {"tc_gemm_step_i", "tc_gemm_step_j", "tc_gemm_tcontract"};
  for (int k = 0; k < 3; ++k) {
    ms[k] = 0.0;
    for (int i = 0; i < n; ++i)
      if (strcmp(st[i].name, names[k]) == 0) ms[k] = st[i].ms;
  }
  DISTIL_TRY(distil_profile_enable(ctx, 0));
  return DISTIL_OK;
}

}  // namespace
}  // namespace distil

using namespace distil;

extern "C" {

int distil_plan_workspace(const distil_batch_shape* shape, const distil_batch_cfg* cfgs, int ncfg, size_t* bytes) {
  DISTIL_CHECK_ARG(bytes != nullptr, "distil_plan_workspace: bytes is null");
  DISTIL_TRY(check_shape(shape, cfgs, ncfg));
  size_t pb = 0, rb = 0;
  DISTIL_TRY(plan_sizes(shape, cfgs, ncfg, &pb, &rb));
  *bytes = pb + rb;
  return DISTIL_OK;
}

int distil_plan_create(distil_ctx* ctx, const distil_batch_shape* shape, const distil_batch_cfg* cfgs, int ncfg,
                       int autotune, void* workspace, size_t ws_bytes, distil_stream stream, distil_plan** out) {
  DISTIL_CHECK_ARG(ctx != nullptr && out != nullptr, "distil_plan_create: null context or out");
  *out = nullptr;
  DISTIL_TRY(check_shape(shape, cfgs, ncfg));
  DISTIL_CHECK_ARG(stream != nullptr, "distil_plan_create: needs a created stream (the legacy stream cannot be captured)");
  DISTIL_CUDA(cudaSetDevice(ctx->device));
  size_t pb = 0, rb = 0;
  DISTIL_TRY(plan_sizes(shape, cfgs, ncfg, &pb, &rb));
  if (ws_bytes < pb + rb || !workspace) {
    set_error("distil_plan_create: workspace %zu < %zu bytes", ws_bytes, pb + rb);
    return DISTIL_ENOMEM;
  }
  DISTIL_CHECK_ARG((reinterpret_cast<uintptr_t>(workspace) & 255) == 0, "distil_plan_create: misaligned workspace");
  void* phi = workspace;
  void* ws = static_cast<char*>(workspace) + pb;
  const size_t wsb = ws_bytes - pb;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  const bool mixed = shape->mode != DISTIL_FP64 && shape->mode != DISTIL_FP32;
  if (autotune && mixed) {
    // candidate vectors: every variant of every site appears once (variant 2
    // exists for step i only); each site keeps its fastest
    constexpr int NC = 6;
    static const int cand[NC][3] = {{0, 0, 0}, {1, 1, 1}, {2, 3, 3}, {3, 4, 4}, {4, 5, 5}, {5, 0, 0}};
    double t[NC][3];
    for (int v = 0; v < NC; ++v) {
      DISTIL_TRY(distil_set_tuning(ctx, cand[v]));
      DISTIL_TRY(time_sites(ctx, shape, cfgs[0], phi, ws, wsb, stream, t[v]));
    }
    int best[3];
    for (int k = 0; k < 3; ++k) {
      int bv = 0;
      for (int v = 1; v < NC; ++v)
        if (t[v][k] < t[bv][k]) bv = v;
      best[k] = cand[bv][k];
    }
    DISTIL_TRY(distil_set_tuning(ctx, best));
  }

  // capture the ensemble; timing stays off while capturing
  Profiler& pr = *ctx->prof;
  const bool timing = pr.timing;
  pr.timing = false;
  cudaGraph_t graph = nullptr;
  DISTIL_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int st = DISTIL_OK;
  for (int c = 0; c < ncfg && st == DISTIL_OK; ++c) st = run_cfg(ctx, shape, cfgs[c], phi, ws, wsb, stream);
  std::string msg = st == DISTIL_OK ? std::string() : std::string(get_error());
  const cudaError_t ce = cudaStreamEndCapture(s, &graph);
  pr.timing = timing;
  if (st != DISTIL_OK || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    if (st == DISTIL_OK) {
      set_error("distil_plan_create: capture failed: %s", cudaGetErrorString(ce));
      return DISTIL_ECUDA;
    }
    set_error("distil_plan_create: %s", msg.c_str());
    return st;
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  if (ie != cudaSuccess) {
    cudaGraphDestroy(graph);
    set_error("distil_plan_create: graph instantiation failed: %s", cudaGetErrorString(ie));
    return DISTIL_ECUDA;
  }
  size_t nn = 0;
  cudaGraphGetNodes(graph, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) cudaGraphGetNodes(graph, nodes.data(), &nn);
  int kernels = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kernels;
  }
  distil_plan* p = new distil_plan();
  p->ctx = ctx;
  p->graph = graph;
  p->exec = exec;
  for (int k = 0; k < 3; ++k) p->tune[k] = ctx->tune[k];
  p->kernels = kernels;
  *out = p;
  return DISTIL_OK;
}

int distil_plan_run(distil_plan* plan, distil_stream stream) {
  DISTIL_CHECK_ARG(plan != nullptr, "distil_plan_run: null plan");
  DISTIL_CUDA(cudaSetDevice(plan->ctx->device));
  DISTIL_CUDA(cudaGraphLaunch(plan->exec, reinterpret_cast<cudaStream_t>(stream)));
  return DISTIL_OK;
}

int distil_plan_info(const distil_plan* plan, int* variants, int* kernels) {
  DISTIL_CHECK_ARG(plan != nullptr, "distil_plan_info: null plan");
  if (variants)
    for (int k = 0; k < 3; ++k) variants[k] = plan->tune[k];
  if (kernels) *kernels = plan->kernels;
  return DISTIL_OK;
}

void distil_plan_destroy(distil_plan* plan) {
  if (!plan) return;
  cudaSetDevice(plan->ctx->device);
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  delete plan;
}

}  // extern "C"

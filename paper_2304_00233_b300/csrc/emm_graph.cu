// Forward-solve plans: the time loop of a solve (2 nt stencil launches, and
// the source, air and volume launches between them) captured once as a CUDA
// graph and replayed for every later solve with the same grid, survey,
// workspace and outputs.  Each run enqueues the set-up (tables, dt/eps from
// the run's conductivity, cleared state) on the stream, launches the graph,
// then the normalisation: the same work, in the same order, as emm_forward.
#include <cuda_runtime.h>

#include <new>
#include <vector>

#include "emm_internal.h"

struct emm_plan {
  const emm_grid *grid = nullptr;
  emm_survey survey{};
  std::vector<double> rec, freqs;  // the plan's copies of the survey arrays
  void *ws = nullptr;
  size_t ws_bytes = 0;
  double *rec_out = nullptr, *vol_out = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

// The survey with its arrays owned by the plan.
void keep_survey(const emm_survey *s, emm_plan *pl) {
  pl->survey = *s;
  pl->rec.assign(s->rec, s->rec + (s->nrec > 0 ? 3 * static_cast<size_t>(s->nrec) : 0));
  pl->freqs.assign(s->freqs, s->freqs + s->nfreq);
  pl->survey.rec = pl->rec.empty() ? nullptr : pl->rec.data();
  pl->survey.freqs = pl->freqs.data();
}

}  // namespace

extern "C" {

int emm_plan_create(const emm_grid *g, const emm_survey *s, const float *sigma, void *ws, size_t ws_bytes,
                    double *rec_out, double *vol_out, emm_stream stream, emm_plan **out) {
  if (!out) return EMM_EINVAL;
  *out = nullptr;
  int st = emm::check_survey(g, s);
  if (st != EMM_OK) return st;
  if (s->volume && !vol_out) return EMM_EINVAL;
  emm_plan *pl = new (std::nothrow) emm_plan;
  if (!pl) return EMM_ENOMEM;
  pl->grid = g;
  keep_survey(s, pl);
  pl->ws = ws;
  pl->ws_bytes = ws_bytes;
  pl->rec_out = rec_out;
  pl->vol_out = vol_out;
  const cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  // a set-up on the stream gives the launch parameters the graph bakes in
  emm::Prepared P;
  st = emm::prepare_forward(g, &pl->survey, sigma, ws, ws_bytes, rec_out, vol_out, cs, &P);
  if (st != EMM_OK) {
    delete pl;
    return st;
  }
  // capture on a stream of the plan's own (the caller's may be the legacy
  // default stream, which cannot be captured); nothing runs during capture
  cudaGraph_t graph = nullptr;
  cudaStream_t cap = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const cudaError_t er = emm::run_steps(P, P.p, P.blocks, 0, pl->survey.nt, cap, nullptr);
    e = cudaStreamEndCapture(cap, &graph);
    if (e == cudaSuccess) e = er;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (cap) cudaStreamDestroy(cap);
  if (e != cudaSuccess) {
    delete pl;
    return EMM_ECUDA;
  }
  *out = pl;
  return EMM_OK;
}

int emm_plan_run(emm_plan *pl, const float *sigma, emm_stream stream) {
  if (!pl || !sigma) return EMM_EINVAL;
  const cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  emm::Prepared P;
  int st = emm::prepare_forward(pl->grid, &pl->survey, sigma, pl->ws, pl->ws_bytes, pl->rec_out, pl->vol_out, cs,
                                &P);
  if (st != EMM_OK) return st;
  if (cudaGraphLaunch(pl->exec, cs) != cudaSuccess) return EMM_ECUDA;
  return emm::finalize_forward(P, &pl->survey, pl->rec_out, pl->vol_out, cs);
}

void emm_plan_destroy(emm_plan *pl) {
  if (!pl) return;
  if (pl->exec) cudaGraphExecDestroy(pl->exec);  // freed once a launch in flight completes
  delete pl;
}

}  // extern "C"

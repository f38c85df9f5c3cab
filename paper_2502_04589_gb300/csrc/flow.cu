// Device-decided control flow.  The stopping tests of the method (the outer test on the
// eigen-residual, §6; the inner test and the stagnation guard of the step-(c) block
// eigensolver) are evaluated by one-thread kernels into a per-handle control block in
// device memory, and the loops they steer are CUDA-graph conditional nodes (WHILE / IF)
// whose condition those kernels set.  A captured step (c), or a whole captured solve, thus
// runs with no host round trip between its iterations.
//
// Recording: graph_record() captures a function on a private stream of the handle (the
// handle's stream is swapped for it while the function records, so every launch helper
// records into the graph); cond_node() adds a conditional node to the graph being
// captured and records its body on the next private stream.  Every body owns an
// execution counter in the control block, bumped by the kernel that sets the node's
// condition, so that the library's launch count stays exact: a body's kernels count once
// per execution.
#include <algorithm>
#include <cstring>

#include "pase_internal.h"

namespace pase {

// ------------------------------------------------------------------ control kernels
// condition of a conditional node := (*flag != 0); exec counts the executions it enables.
// WHILE nodes carry a pass guard: reset before the node (limit < 0), counted at the end of
// each pass; a loop that reaches `limit` passes is ended with PASE_ERR_TIMEOUT, so that no
// recorded loop can run without bound whatever its test computes.
__global__ void k_set_cond(const int* __restrict__ flag, cudaGraphConditionalHandle hnd, int* __restrict__ exec,
                           int* __restrict__ guard, int limit, int* __restrict__ err) {
  int v = *flag != 0;
  if (guard) {
    if (limit < 0) {
      *guard = 0;
    } else if (++*guard >= limit && v) {
      v = 0;
      if (!*err) *err = PASE_ERR_TIMEOUT;
    }
  }
  cudaGraphSetConditional(hnd, (unsigned)v);
  if (v) *exec += 1;
}

__global__ void k_ctl_init(int* __restrict__ ci, double* __restrict__ cd) {
  const int t = threadIdx.x;
  if (t < CI_EXEC0) ci[t] = 0;
  if (t < CD_COUNT) cd[t] = 0.0;
}

__global__ void k_ctl_put(int* pi, int vi, int add, double* pd, double vd) {
  if (pi) *pi = add ? *pi + vi : vi;
  if (pd) *pd = vd;
}

// Outer stopping test (§6: every one of the first nev pairs at relative residual <= tol)
// and the inner tolerance of the next step (c): max(aug_tol, f x worst residual), f the
// adaptive factor.  A pending error or a finite-range flag
// of the double-float products stops the loop too.
__global__ void k_ctl_outer_check(int nev, const double* __restrict__ relres, double tol, double aug_tol,
                                  int adaptive, double factor, int max_iter, int post_solve,
                                  const int* __restrict__ df_flag, int* __restrict__ ci, double* __restrict__ cd) {
  double worst = 0.0;
  int conv = 0;
  bool nan = false;
  for (int j = 0; j < nev; ++j) {
    const double r = relres[j];
    if (!(r == r)) {
      nan = true;
      continue;
    }
    worst = fmax(worst, r);
    conv += r <= tol;
  }
  int err = ci[CI_ERR];
  if (!err && nan) err = PASE_ERR_NAN;
  if (!err && df_flag && *df_flag) err = kCtlErrDfRange;
  ci[CI_ERR] = err;
  ci[CI_CONV] = conv;
  cd[CD_WORST] = nan ? __longlong_as_double(0x7ff8000000000000ll) : worst;
  const int it = ci[CI_ITER];
  int go = 0;
  if (!err && !(worst <= tol)) {
    if (it >= max_iter) ci[CI_MAXED] = 1;
    else go = 1;
  }
  if (go && adaptive) {
    // safeguarded factor: a pass whose residual rose above the previous one tightens it
    // tenfold (down to 1e-3 of the base); a drop by more than five relaxes it tenfold (up
    // to the base)
    double f = cd[CD_FACTOR] > 0.0 ? cd[CD_FACTOR] : factor;
    const double prev = cd[CD_PREV_WORST];
    if (prev > 0.0 && worst > prev) f = fmax(0.1 * f, 1e-3 * factor);
    else if (prev > 0.0 && worst < 0.2 * prev) f = fmin(10.0 * f, factor);
    cd[CD_FACTOR] = f;
    cd[CD_AUG_TOL] = fmax(aug_tol, f * worst);
  } else if (go) {
    cd[CD_AUG_TOL] = aug_tol;
  }
  if (!nan) cd[CD_PREV_WORST] = worst;
  ci[CI_OUT_GO] = go;
  ci[CI_OUT_CONT] = go;
  ci[CI_POST] = go && post_solve && it > 0;
}

// inner tolerance from the current residuals (the adaptive rule of the outer test)
__global__ void k_ctl_aug_tol(int nev, const double* __restrict__ relres, double aug_tol, double factor,
                              double* __restrict__ cd) {
  double worst = 0.0;
  for (int j = 0; j < nev; ++j) worst = fmax(worst, relres[j]);
  cd[CD_AUG_TOL] = fmax(aug_tol, factor * worst);
}

__global__ void k_ctl_inner_init(int* __restrict__ ci) {
  ci[CI_IN_IT] = 0;
  ci[CI_HIST_N] = 0;
  ci[CI_IN_CONT] = 1;
}

// Inner test of the block eigensolver on the first nconv columns: converged, stagnant at
// the attainable accuracy (no halving over six passes while below 1e-6), out of passes,
// NaN, or an error pending -> stop.
__global__ void k_ctl_inner_check(int nconv, const double* __restrict__ relres, const double* __restrict__ tol_dev,
                                  double tol_fixed, int maxit, int* __restrict__ ci, double* __restrict__ cd) {
  double worst = 0.0;
  bool nan = false;
  for (int j = 0; j < nconv; ++j) {
    const double r = relres[j];
    if (!(r == r)) nan = true;
    else worst = fmax(worst, r);
  }
  const int p = ++ci[CI_IN_IT];
  ci[CI_AUG_IT] += 1;
  const double tol = tol_dev ? *tol_dev : tol_fixed;
  int go = 0;
  if (nan) {
    if (!ci[CI_ERR]) ci[CI_ERR] = PASE_ERR_NAN;
  } else if (!ci[CI_ERR] && !(worst <= tol)) {
    int n = ci[CI_HIST_N];
    cd[CD_HIST + (n % kCtlHist)] = worst;
    ++n;
    ci[CI_HIST_N] = n;
    const bool stagnant = n > 6 && worst > 0.5 * cd[CD_HIST + ((n - 7) % kCtlHist)] && worst < 1e-6;
    go = !stagnant;
  }
  cd[CD_IN_WORST] = worst;
  ci[CI_IN_GO] = go;
  ci[CI_IN_CONT] = go && p < maxit;
}

// status word of the small eigensolver: fatal (the start block) -> error; otherwise the
// pass is skipped and the loop ends (fewer than m independent directions left)
__global__ void k_ctl_status(const int* __restrict__ status, int* __restrict__ ci, int fatal) {
  const int ok = status[0] == 0;
  if (fatal) {
    if (!ok && !ci[CI_ERR]) ci[CI_ERR] = PASE_ERR_NOT_SPD;
  } else {
    ci[CI_IN_OK] = ok;
    if (!ok) ci[CI_IN_CONT] = 0;
  }
}

namespace {
int launched(pase_ctx* h) {
  h->launches++;
  PASE_CUDA(cudaGetLastError());
  return PASE_OK;
}
}  // namespace

int launch_ctl_init(pase_ctx* h) {
  k_ctl_init<<<1, 32, 0, h->stream>>>(h->w.ci, h->w.cd);
  return launched(h);
}
int launch_ctl_put(pase_ctx* h, int* pi, int vi, bool add, double* pd, double vd) {
  k_ctl_put<<<1, 1, 0, h->stream>>>(pi, vi, add ? 1 : 0, pd, vd);
  return launched(h);
}
int launch_ctl_outer_check(pase_ctx* h, int nev, double tol) {
  const pase_options& o = h->opt;
  k_ctl_outer_check<<<1, 1, 0, h->stream>>>(nev, h->w.relres, tol, o.aug_tol, o.aug_adaptive, o.aug_factor,
                                            o.max_iter, o.post_solve, h->w.df_flag, h->w.ci, h->w.cd);
  return launched(h);
}
int launch_ctl_aug_tol(pase_ctx* h, int nev) {
  k_ctl_aug_tol<<<1, 1, 0, h->stream>>>(nev, h->w.relres, h->opt.aug_tol, h->opt.aug_factor, h->w.cd);
  return launched(h);
}
int launch_ctl_inner_init(pase_ctx* h) {
  k_ctl_inner_init<<<1, 1, 0, h->stream>>>(h->w.ci);
  return launched(h);
}
int launch_ctl_inner_check(pase_ctx* h, int nconv, const double* relres, const double* tol_dev, double tol_fixed,
                           int maxit) {
  k_ctl_inner_check<<<1, 1, 0, h->stream>>>(nconv, relres, tol_dev, tol_fixed, maxit, h->w.ci, h->w.cd);
  return launched(h);
}
int launch_ctl_status(pase_ctx* h, const int* status, bool fatal) {
  k_ctl_status<<<1, 1, 0, h->stream>>>(status, h->w.ci, fatal ? 1 : 0);
  return launched(h);
}

// ------------------------------------------------------------------ recording
bool recording(const pase_ctx* h) { return h->cap.rec != nullptr; }

static int cap_stream(pase_ctx* h, int depth, cudaStream_t* out) {
  if (depth > kCapMaxDepth) return fail(PASE_ERR_STATE, "graph recording: conditional nodes nested too deeply");
  while ((int)h->cap_streams.size() <= depth) {
    cudaStream_t s = nullptr;
    PASE_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    h->cap_streams.push_back(s);
  }
  *out = h->cap_streams[depth];
  return PASE_OK;
}

int cond_node(pase_ctx* h, bool loop, int* flag, const std::function<int()>& body, int max_passes) {
  if (!recording(h)) return fail(PASE_ERR_STATE, "cond_node outside a graph recording");
  Capture& c = h->cap;
  if (c.slot_next >= c.slot_end) return fail(PASE_ERR_STATE, "graph recording: too many conditional bodies");
  const int slot = c.slot_next++;
  int* exec = h->w.ci + CI_EXEC0 + slot;
  int* guard = loop ? h->w.ci + CI_GUARD0 + slot : nullptr;
  if (loop && max_passes < 1) return fail(PASE_ERR_STATE, "graph recording: a loop needs a pass limit");
  if (loop && h->opt.graph_pass_limit > 0) max_passes = std::min(max_passes, h->opt.graph_pass_limit);
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  PASE_CUDA(cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  if (cs != cudaStreamCaptureStatusActive) return fail(PASE_ERR_STATE, "graph recording: stream not capturing");
  cudaGraphConditionalHandle hnd = 0;
  PASE_CUDA(cudaGraphConditionalHandleCreate(&hnd, g, 0, 0));
  // the kernel that sets the condition precedes the node
  k_set_cond<<<1, 1, 0, h->stream>>>(flag, hnd, exec, guard, -1, h->w.ci + CI_ERR);
  PASE_TRY(launched(h));
  const cudaGraphNode_t* d = nullptr;
  size_t nd = 0;
  PASE_CUDA(cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &g, &d, nullptr, &nd));
  std::vector<cudaGraphNode_t> deps(d, d + nd);
  // the parameter block is a union without a default constructor: zeroed storage
  alignas(cudaGraphNodeParams) unsigned char pbuf[sizeof(cudaGraphNodeParams)];
  memset(pbuf, 0, sizeof(pbuf));
  cudaGraphNodeParams& p = *reinterpret_cast<cudaGraphNodeParams*>(pbuf);
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = hnd;
  p.conditional.type = loop ? cudaGraphCondTypeWhile : cudaGraphCondTypeIf;
  p.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  PASE_CUDA(cudaGraphAddNode(&node, g, deps.data(), nullptr, deps.size(), &p));
  cudaGraph_t bodyg = p.conditional.phGraph_out[0];
  PASE_CUDA(cudaStreamUpdateCaptureDependencies(h->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaStream_t s2 = nullptr;
  if (c.depth >= kCapMaxDepth) return fail(PASE_ERR_STATE, "graph recording: conditional nodes nested too deeply");
  PASE_TRY(cap_stream(h, c.depth, &s2));
  PASE_CUDA(cudaStreamBeginCaptureToGraph(s2, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  const cudaStream_t saved = h->stream;
  h->stream = s2;
  c.depth++;
  c.child.push_back(0);
  const int64_t l0 = h->launches;
  int rc = body();
  if (rc == PASE_OK && loop) {  // the condition of the next pass
    k_set_cond<<<1, 1, 0, h->stream>>>(flag, hnd, exec, guard, max_passes, h->w.ci + CI_ERR);
    rc = launched(h);
  }
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s2, &out);
  h->stream = saved;
  c.depth--;
  const int64_t total = h->launches - l0;
  const int64_t nested = c.child.back();
  c.child.pop_back();
  c.child.back() += total;
  c.bodies.push_back({slot, total - nested});
  if (rc != PASE_OK) return rc;
  if (e != cudaSuccess) return fail(PASE_ERR_CUDA, std::string("graph recording: ") + cudaGetErrorString(e));
  return PASE_OK;
}

// Prepare the handle for recording into `rec` on stream s (already capturing).
static int rec_begin(pase_ctx* h, GraphRec& rec, cudaStream_t s, cudaStream_t* saved, int64_t* l0) {
  if (recording(h)) return fail(PASE_ERR_STATE, "graph recording: already recording");
  PASE_TRY(sync_ctl(h));  // settle the counters of the graph being replaced
  for (int k = rec.slot0; k < rec.slot0 + rec.nslots; ++k) {
    h->ci_last[k] = 0;
    h->body_kernels[k] = 0;
  }
  PASE_CUDA(cudaMemsetAsync(h->w.ci + CI_EXEC0 + rec.slot0, 0, sizeof(int) * rec.nslots, h->stream));
  PASE_CUDA(cudaStreamSynchronize(h->stream));
  Capture& c = h->cap;
  c = Capture();
  c.rec = &rec;
  c.depth = 1;
  c.slot_next = rec.slot0;
  c.slot_end = rec.slot0 + rec.nslots;
  c.child.assign(1, 0);
  *saved = h->stream;
  *l0 = h->launches;
  h->stream = s;
  return PASE_OK;
}
// Close the recording: the kernel counts of the top level and of every body.
static void rec_end(pase_ctx* h, GraphRec& rec, cudaStream_t saved, int64_t l0, bool ok) {
  Capture& c = h->cap;
  const int64_t total = h->launches - l0;
  h->launches = l0;
  h->stream = saved;
  if (ok) {
    rec.top_kernels = total - c.child[0];
    rec.nodes_recorded = total;
    for (const auto& b : c.bodies) h->body_kernels[b.first] = b.second;
  }
  c = Capture();
}

static int instantiate(cudaGraph_t g, cudaGraphExec_t* ex) {
  const cudaError_t ie = cudaGraphInstantiate(ex, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    cudaGetLastError();
    *ex = nullptr;
    return fail(PASE_ERR_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(ie));
  }
  return PASE_OK;
}

int graph_record(pase_ctx* h, GraphRec& rec, const std::function<int()>& fn) {
  if (rec.exec) {
    cudaGraphExecDestroy(rec.exec);
    rec.exec = nullptr;
  }
  cudaStream_t s = nullptr, saved = nullptr;
  int64_t l0 = 0;
  PASE_TRY(cap_stream(h, 0, &s));
  PASE_TRY(rec_begin(h, rec, s, &saved, &l0));
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
  const int rc = e == cudaSuccess ? fn() : PASE_ERR_CUDA;
  cudaGraph_t g = nullptr;
  if (e == cudaSuccess) e = cudaStreamEndCapture(s, &g);
  rec_end(h, rec, saved, l0, rc == PASE_OK && e == cudaSuccess && g);
  if (rc != PASE_OK || e != cudaSuccess || !g) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    if (rc != PASE_OK && rc != PASE_ERR_CUDA) return rc;
    return fail(PASE_ERR_CUDA, std::string("graph recording: ") + cudaGetErrorString(e));
  }
  return instantiate(g, &rec.exec);
}

// One graph for many handles: every handle's recording (fn(i), into its rec g_batch) is a
// branch forked from one origin stream and joined back, so that the branches run
// concurrently when the graph is launched once.
int batch_record(pase_ctx* const* hs, int count, const std::function<int(int)>& fn, cudaGraphExec_t* out) {
  *out = nullptr;
  pase_ctx* h0 = hs[0];
  cudaStream_t origin = nullptr;
  PASE_TRY(cap_stream(h0, kCapMaxDepth, &origin));
  std::vector<cudaEvent_t> ev(count + 1, nullptr);
  for (auto& e : ev) PASE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  struct EvFree {
    std::vector<cudaEvent_t>& v;
    ~EvFree() {
      for (auto e : v) cudaEventDestroy(e);
    }
  } evfree{ev};
  cudaError_t e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) e = cudaEventRecord(ev[count], origin);
  int rc = e == cudaSuccess ? PASE_OK : PASE_ERR_CUDA;
  for (int i = 0; i < count && rc == PASE_OK; ++i) {
    pase_ctx* h = hs[i];
    cudaStream_t s = nullptr, saved = nullptr;
    int64_t l0 = 0;
    rc = cap_stream(h, 0, &s);
    if (rc != PASE_OK) break;
    rc = rec_begin(h, h->g_batch, s, &saved, &l0);
    if (rc != PASE_OK) break;
    e = cudaStreamWaitEvent(s, ev[count], 0);  // s joins the capture
    rc = e == cudaSuccess ? fn(i) : PASE_ERR_CUDA;
    if (rc == PASE_OK) {
      e = cudaEventRecord(ev[i], s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, ev[i], 0);
      if (e != cudaSuccess) rc = PASE_ERR_CUDA;
    }
    rec_end(h, h->g_batch, saved, l0, rc == PASE_OK);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(origin, &g);
  if (rc != PASE_OK || ee != cudaSuccess || !g) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    if (rc != PASE_OK && rc != PASE_ERR_CUDA) return rc;
    return fail(PASE_ERR_CUDA, std::string("batch graph recording: ") +
                                   cudaGetErrorString(e != cudaSuccess ? e : ee));
  }
  return instantiate(g, out);
}

int graph_launch(pase_ctx* h, GraphRec& rec) {
  if (!rec.exec) return fail(PASE_ERR_STATE, "graph_launch: nothing recorded");
  PASE_CUDA(cudaGraphLaunch(rec.exec, h->stream));
  h->launches += rec.top_kernels;
  h->replayed += rec.top_kernels;
  h->graph_launches++;
  return PASE_OK;
}

void graph_free(GraphRec& rec) {
  if (rec.exec) cudaGraphExecDestroy(rec.exec);
  rec.exec = nullptr;
  rec.key.clear();
}

// Read the control block (and `count` doubles of src into h_small), wait for the stream,
// and add the kernels that conditional bodies ran since the last read to the count.
int sync_ctl(pase_ctx* h, const double* src, int count) {
  Work& w = h->w;
  if (!w.ci) {
    PASE_CUDA(cudaStreamSynchronize(h->stream));
    return PASE_OK;
  }
  PASE_CUDA(cudaMemcpyAsync(w.h_ci, w.ci, sizeof(int) * kCtlInts, cudaMemcpyDeviceToHost, h->stream));
  PASE_CUDA(cudaMemcpyAsync(w.h_cd, w.cd, sizeof(double) * CD_COUNT, cudaMemcpyDeviceToHost, h->stream));
  if (count) PASE_CUDA(cudaMemcpyAsync(w.h_small, src, sizeof(double) * count, cudaMemcpyDeviceToHost, h->stream));
  PASE_CUDA(cudaStreamSynchronize(h->stream));
  for (int s = 0; s < kCtlSlots; ++s) {
    const int v = w.h_ci[CI_EXEC0 + s];
    if (h->body_kernels[s]) {
      const int64_t k = h->body_kernels[s] * (int64_t)(v - h->ci_last[s]);
      h->launches += k;
      h->replayed += k;
    }
    h->ci_last[s] = v;
  }
  return PASE_OK;
}

}  // namespace pase

// Host orchestration of Nys-IP-PMM (Algorithm 6 with Algorithms 5, 4, 2, 1)
// and the C ABI of include/nys.h.
//
// The handle owns one device arena holding every workspace buffer.  The IPM
// loop runs on the host and issues kernels on the handle's stream; it reads
// back a handful of scalars per IPM iteration (residual norms, step-length
// ratios, mu_aff).  PCG scalars stay on the device: iterations are issued in
// growing chunks and the host polls a single "done" flag between chunks.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <condition_variable>
#include <vector>

#include <atomic>

#include "../../include/nys.h"
#include "internal.h"

using namespace nys;

namespace nys {
static std::atomic<unsigned long long> g_launches{0};
void count_launches(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace nys

struct nys_solver {
  nys_options opt{};
  int max_m = 0, max_n = 0, ell_cap = 0;
  int ld = 0, ld_t = 0;
  cudaStream_t st = nullptr;
  int device = 0, num_sms = 152;
  std::string err;

  void* arena = nullptr;
  size_t arena_bytes = 0;
  double* sd = nullptr;
  int* si = nullptr;
  RedBuf red;
  double* split_buf = nullptr;
  size_t split_cap = 0;
  double *Om = nullptr, *Y = nullptr, *U = nullptr, *lamh = nullptr, *T = nullptr;
  CoreWork cw{};
  PcgWork pw{};
  // IPM vectors
  double *x = nullptr, *y = nullptr, *z = nullptr, *lam = nullptr, *zeta = nullptr, *D = nullptr;
  double *Ax = nullptr, *Aty = nullptr, *r_d = nullptr, *r_p = nullptr, *r_xz = nullptr;
  double *t_n = nullptr, *g_n = nullptr, *xi = nullptr;
  double *dxp = nullptr, *dyp = nullptr, *dzp = nullptr, *dxc = nullptr, *dyc = nullptr, *dzc = nullptr;
  double* red_out = nullptr;
  // free and box-constrained variables (problems (P~)/(D~)): kinds, upper
  // bounds (zero outside J), slack w = u - x, its multiplier s, their
  // right-hand sides and directions
  signed char* vk = nullptr;
  double *uv = nullptr, *w = nullptr, *s = nullptr, *r_u = nullptr, *r_ws = nullptr;
  double *dwp = nullptr, *dsp = nullptr, *dwc = nullptr, *dsc = nullptr;
  // pinned host mirrors
  double* h_red = nullptr;
  int* h_si = nullptr;
  // device staging for problems given in host memory
  void* stage = nullptr;
  size_t stage_bytes = 0;
  // PCG as one graph launch: a conditional while node whose body is one
  // predicated iteration (rebuilt when the operator's pointers change)
  cudaStream_t cap_stream = nullptr;
  // device time of the PCG solves: events around each solve on the stream
  cudaEvent_t ev_pcg0 = nullptr, ev_pcg1 = nullptr;
  // lock-step batches: a worker's prepared request; the shared launch (master)
  cudaEvent_t ev_req = nullptr, ev_b0 = nullptr, ev_b1 = nullptr;
  ClusterPcgTask* d_tasks = nullptr;   // device task array of the shared launch
  ClusterPcgTask* h_tasks = nullptr;   // pinned staging of the same
  int task_cap = 0;
  double pcg_ms = 0.0;
  cudaGraph_t pcg_graph = nullptr;
  cudaGraphExec_t pcg_exec = nullptr;
  const void* gk_A = nullptr;
  const double *gk_D = nullptr, *gk_U = nullptr;
  long long gk_lda = 0;
  int gk_m = 0, gk_n = 0, gk_ell = 0, gk_ld = 0;
  unsigned g_kernels_per_iter = 0;
  bool use_graphs = true;
  // FP64 PCG route: 0 by size (cluster, else cooperative, else graph),
  // 1 cluster only, 2 cooperative only, 3 graph only (NYS_PCG_PATH)
  int pcg_path = 0;
  int plan_policy = 0;         // cluster plans: 0 latency, 2 latency else throughput (NYS_PCG_PATH=cluster)
  int cp_m = -1, cp_n = -1, cp_ell = -1;   // key of the cached cluster plan
  bool cp_ok = false;
  ClusterPlan cp;
  int gk_op = -1;            // graph key: operator kind
  double* pcg_x = nullptr;   // PCG solution buffer (copied out after each solve)
  // FP8 variant (precision_mode 2): E4M3 copies of A and A^T with the
  // per-row scales of A feed the inner PCG (the sketch keeps BF16)
  void* A8 = nullptr;
  void* A8T = nullptr;
  float* rs32 = nullptr;
  double* rs64 = nullptr;
  long long ld_q = 0, ld_qt = 0;
  // precision form (precision_mode 1): A is FP32 (the problem definition);
  // BF16 copies of A and A^T feed the inner PCG and the tensor-core sketch,
  // an FP32 copy of A^T the refinement residual.
  void* lp_arena = nullptr;
  size_t lp_bytes = 0;
  __nv_bfloat16 *Ab = nullptr, *AbT = nullptr, *Omb = nullptr, *Tb = nullptr;
  float *AfT = nullptr, *upart = nullptr, *Y32 = nullptr, *xf = nullptr, *tf = nullptr, *Df = nullptr;
  float *fh = nullptr, *fl = nullptr;
  size_t upart_cap = 0;
  long long ld_b = 0, ld_bt = 0, ld_ft = 0, ld_om = 0, ld_tb = 0, ld_ff = 0;
  double *nd_m = nullptr, *u_n = nullptr, *rr = nullptr, *dyacc = nullptr, *ecorr = nullptr;
  double* lp_part = nullptr;   // column-split partial sums of the row GEMVs
  size_t lp_part_cap = 0;
  bool lp_bf16_stage = true;   // BF16 corrections still contracting in this solve
  int trace = 0;               // NYS_TRACE=1: one line per IPM iteration on stderr
  // the Nystrom factor now in U / lamh: built for the FP64 matrix fac_A
  // (m = fac_m, sketch size fac_ell) by the last IPM iteration of a solve
  const void* fac_A = nullptr;
  int fac_m = 0, fac_ell = 0;
  // device-resident IPM iteration (ipm_dev.cu) for problems (P) in the FP64
  // form on a cluster PCG route: its scalars, the two PCG tasks of an
  // iteration, the forced counts and the PCG log live in device memory, and
  // a whole solve is one graph (kept while the problem's pointers, shapes and
  // launch plan stay the same)
  IpmDev* ipmd = nullptr;
  ClusterPcgTask* dtask = nullptr;     // 2: predictor, corrector
  int* d_forced = nullptr;
  int* d_pcglog = nullptr;
  int dev_log_cap = 0;
  IpmDev* h_ipmd = nullptr;            // pinned mirror
  int* h_pcglog = nullptr;             // pinned mirror
  cudaGraph_t ipm_graph = nullptr;
  cudaGraphExec_t ipm_exec = nullptr;
  const void* ik_ptr[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // A, b, c, q, plan key
  long long ik_lda = 0;
  int ik_m = 0, ik_n = 0, ik_ell = 0, ik_C = 0, ik_as = 0;
  unsigned ipm_kernels_top = 0, ipm_kernels_body = 0;
  bool use_dev_ipm = true;             // NYS_DEVICE_IPM=0 keeps the host-driven iteration
  int tuned_inflight = 0;              // batching form: problems in flight chosen by the autotuner
  // batching form: cluster plan (CTAs, A on chip) per shape bucket chosen by
  // timed trials (C = 0: no cluster plan fits), and the trials' buffer
  std::map<long long, std::pair<int, int>> tuned_plans;
  double* tune_buf = nullptr;
  size_t tune_cap = 0;
  int trace_tune = 0;                  // NYS_TRACE_TUNE=1: the autotuner's trials on stderr
  // batching form: worker solvers (created on first use), one per in-flight QP
  int max_batch = 0;
  std::vector<nys_solver*> workers;
  std::vector<cudaStream_t> worker_streams;
  // shared launches of one Newton phase: one stream per launch shape, so that
  // groups of different cluster size run side by side
  std::vector<cudaStream_t> group_streams;
  std::vector<cudaEvent_t> group_events;
};

namespace {

int fail(nys_solver* h, int code, const char* fmt, ...) {
  if (h) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    h->err = buf;
  }
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(h, NYS_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                    \
  } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Carver {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += count * sizeof(T);
    return p;
  }
};

// Lay out (or size, when base == nullptr) every workspace buffer.
size_t carve(nys_solver* h, char* base) {
  Carver c{base};
  const size_t M = h->max_m, N = h->max_n, L = h->ell_cap;
  const size_t LD = h->ld, LDT = h->ld_t;
  h->sd = c.take<double>(SD_COUNT);
  h->si = c.take<int>(SI_COUNT);
  h->red.part = c.take<double>(RedBuf::kPartCap);
  h->red.cnt = c.take<unsigned>(RedBuf::kCntCap);
  h->split_cap = std::max({gemv_t_split_elems((int)M, (int)N), (size_t)4 * LD * L,
                           (size_t)64 * L * L, (size_t)1 << 16});
  h->split_buf = c.take<double>(h->split_cap);
  h->Om = c.take<double>(LD * L);
  h->Y = c.take<double>(LD * L);
  h->U = c.take<double>(LD * L);
  h->lamh = c.take<double>(L);
  h->T = c.take<double>(LDT * L);
  h->cw.Ynu = c.take<double>(LD * L);
  h->cw.G = c.take<double>(L * L);
  h->cw.sumsq = c.take<double>(L);
  h->cw.perm = c.take<int>(L);
  h->cw.bar = c.take<unsigned>(2);
  h->cw.sweep_flags = c.take<int>(CoreWork::kMaxSweeps);
  h->cw.B2 = c.take<double>(LD * L);
  h->cw.R = c.take<double>(L * L);
  h->cw.Rt = c.take<double>(L * L);
  h->cw.split_buf = h->split_buf;
  h->cw.split_cap = h->split_cap;
  h->pcg_x = c.take<double>(M);
  h->pw.r = c.take<double>(M);
  h->pw.z = c.take<double>(M);
  h->pw.p = c.take<double>(M);
  h->pw.w = c.take<double>(M);
  h->pw.s = c.take<double>(L);
  h->pw.wts = c.take<double>(L);
  h->pw.t = c.take<double>(N);
  h->pw.split_buf = h->split_buf;
  h->pw.split_cap = h->split_cap;
  h->x = c.take<double>(N);
  h->y = c.take<double>(M);
  h->z = c.take<double>(N);
  h->lam = c.take<double>(M);
  h->zeta = c.take<double>(N);
  h->D = c.take<double>(N);
  h->Ax = c.take<double>(M);
  h->Aty = c.take<double>(N);
  h->r_d = c.take<double>(N);
  h->r_p = c.take<double>(M);
  h->r_xz = c.take<double>(N);
  h->t_n = c.take<double>(N);
  h->g_n = c.take<double>(N);
  h->xi = c.take<double>(M);
  h->dxp = c.take<double>(N);
  h->dyp = c.take<double>(M);
  h->dzp = c.take<double>(N);
  h->dxc = c.take<double>(N);
  h->dyc = c.take<double>(M);
  h->dzc = c.take<double>(N);
  h->red_out = c.take<double>(16);
  h->vk = c.take<signed char>(N);
  h->uv = c.take<double>(N);
  h->w = c.take<double>(N);
  h->s = c.take<double>(N);
  h->r_u = c.take<double>(N);
  h->r_ws = c.take<double>(N);
  h->dwp = c.take<double>(N);
  h->dsp = c.take<double>(N);
  h->dwc = c.take<double>(N);
  h->dsc = c.take<double>(N);
  h->dev_log_cap = 2 * std::max(0, h->opt.max_ipm_iter) + 8;
  h->ipmd = c.take<IpmDev>(1);
  h->dtask = c.take<ClusterPcgTask>(2);
  h->d_forced = c.take<int>(h->dev_log_cap);
  h->d_pcglog = c.take<int>(h->dev_log_cap);
  return c.off;
}

size_t carve_lp(nys_solver* h, char* base) {
  Carver c{base};
  const size_t M = h->max_m, N = h->max_n, L = h->ell_cap;
  h->ld_b = (long long)align_up(M > 0 ? N : 0, 8);
  h->ld_bt = (long long)align_up(M, 8);
  h->ld_ft = (long long)align_up(M, 4);
  h->ld_om = (long long)align_up(M, 8);
  h->ld_tb = (long long)align_up(N, 8);
  h->ld_ff = (long long)std::max(align_up(M, 8), align_up(N, 8));
  h->Ab = c.take<__nv_bfloat16>(M * (size_t)h->ld_b);
  h->AbT = c.take<__nv_bfloat16>(N * (size_t)h->ld_bt);
  h->AfT = c.take<float>(N * (size_t)h->ld_ft);
  h->Omb = c.take<__nv_bfloat16>(L * (size_t)h->ld_om);
  h->Tb = c.take<__nv_bfloat16>(L * (size_t)h->ld_tb);
  h->upart_cap = std::max(umma_part_elems((int)N, (int)L, (int)M, h->num_sms),
                          umma_part_elems((int)M, (int)L, (int)N, h->num_sms));
  h->upart = c.take<float>(h->upart_cap);
  h->Y32 = c.take<float>((size_t)h->ld * L);
  h->xf = c.take<float>(h->ld_ff);
  h->tf = c.take<float>(h->ld_ff);
  h->Df = c.take<float>(h->ld_ff);
  h->fh = c.take<float>(h->ld_ff);
  h->fl = c.take<float>(h->ld_ff);
  h->nd_m = c.take<double>(M);
  h->u_n = c.take<double>(N);
  h->rr = c.take<double>(M);
  h->dyacc = c.take<double>(M);
  h->ecorr = c.take<double>(M);
  h->lp_part_cap = 16 * std::max(M, N);
  h->lp_part = c.take<double>(h->lp_part_cap);
  if (h->opt.precision_mode == 2) {
    h->ld_q = (long long)align_up(N, 16);
    h->ld_qt = (long long)align_up(M, 16);
    h->A8 = c.take<unsigned char>(M * (size_t)h->ld_q);
    h->A8T = c.take<unsigned char>(N * (size_t)h->ld_qt);
    h->rs32 = c.take<float>(M);
    h->rs64 = c.take<double>(M);
  }
  return c.off;
}

int check_err(nys_solver* h) {
  const int e = h->h_si[SI_ERR];
  if (e == 0) return NYS_OK;
  switch (e) {
    case NYS_ERR_CORE_BREAKDOWN: return fail(h, NYS_ERR_CORE_BREAKDOWN, "Cholesky of Omega^T Y_nu met a non-positive pivot");
    case NYS_ERR_TIMEOUT: return fail(h, NYS_ERR_TIMEOUT, "a bounded device wait expired");
    default: return fail(h, NYS_ERR_NUMERIC, "non-finite or non-positive quantity in a device reduction");
  }
}

// Copy the device scalars to the pinned mirrors and wait.
int sync_scalars(nys_solver* h, int n_red) {
  CK(cudaMemcpyAsync(h->h_si, h->si, sizeof(int) * SI_COUNT, cudaMemcpyDeviceToHost, h->st));
  if (n_red > 0)
    CK(cudaMemcpyAsync(h->h_red, h->red_out, sizeof(double) * n_red, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return check_err(h);
}

int valid_ptr(const void* p) { return p != nullptr; }

int sync_scalars_at(nys_solver* h, int off, int n_red) {
  CK(cudaMemcpyAsync(h->h_si, h->si, sizeof(int) * SI_COUNT, cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(h->h_red + off, h->red_out + off, sizeof(double) * n_red, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return check_err(h);
}

void drop_ipm_graph(nys_solver* h) {
  if (h->ipm_exec) cudaGraphExecDestroy(h->ipm_exec);
  if (h->ipm_graph) cudaGraphDestroy(h->ipm_graph);
  h->ipm_exec = nullptr;
  h->ipm_graph = nullptr;
  h->ik_ptr[0] = nullptr;
}

void drop_pcg_graph(nys_solver* h) {
  if (h->pcg_exec) cudaGraphExecDestroy(h->pcg_exec);
  if (h->pcg_graph) cudaGraphDestroy(h->pcg_graph);
  h->pcg_exec = nullptr;
  h->pcg_graph = nullptr;
  h->gk_A = nullptr;
}

// The operator (N + delta I) p used inside PCG: FP64 A (kind 0), or the
// precision form's BF16 (kind 1) / FP32 (kind 2) row-major copies.
struct OpSpec {
  int kind;
  const double* A;      // kind 0
  long long lda;
  const double* D;      // kind 0
  LpOperator lp;        // kinds 1-4 (BF16, FP32, float-float, FP8)
  const void* key() const { return kind == 0 ? (const void*)A : lp.A; }
};

cudaError_t issue_pcg_iteration(nys_solver* h, cudaStream_t st, int m, int n, const OpSpec& op, int ell,
                                const double* U, int ld, PcgWork w) {
  if (op.kind == 0) return pcg_iteration_f64(st, m, n, op.A, op.lda, op.D, ell, U, ld, w, h->sd, h->si, h->red);
  return pcg_iteration_lp(st, m, n, op.lp, ell, U, ld, w, h->sd, h->si, h->red);
}

// Build (or reuse) the graph "while (!done) { one PCG iteration }" for this
// operator.  Returns false when graphs are unavailable (the caller then
// issues iterations from the host).
bool ensure_pcg_graph(nys_solver* h, int m, int n, const OpSpec& op, int ell, const double* U, int ld) {
  if (!h->use_graphs) return false;
  const double* D = op.kind == 0 ? op.D : (op.kind == 3 ? op.lp.D64 : reinterpret_cast<const double*>(op.lp.Df));
  const long long lda = op.kind == 0 ? op.lda : op.lp.lda;
  if (h->pcg_exec && h->gk_op == op.kind && h->gk_A == op.key() && h->gk_lda == lda && h->gk_m == m &&
      h->gk_n == n && h->gk_ell == ell && h->gk_D == D && h->gk_U == U && h->gk_ld == ld)
    return true;
  drop_pcg_graph(h);
  PcgWork w = h->pw;
  w.x = h->pcg_x;
  cudaGraph_t g = nullptr;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
  cudaGraphConditionalHandle cond{};
  cudaGraphNodeParams cp{};
  cudaGraphNode_t node{};
  ok = ok && cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  if (ok) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
  }
  if (ok) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      const unsigned long long c0 = g_launches.load();
      cudaError_t e1 = issue_pcg_iteration(h, h->cap_stream, m, n, op, ell, U, ld, w);
      cudaError_t e2 = pcg_loop_condition(h->cap_stream, cond, h->si);
      h->g_kernels_per_iter = (unsigned)(g_launches.load() - c0);
      g_launches.fetch_sub(h->g_kernels_per_iter);   // counted when the graph runs
      cudaGraph_t out = nullptr;
      cudaError_t e3 = cudaStreamEndCapture(h->cap_stream, &out);
      ok = e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess;
    }
  }
  cudaGraphExec_t exec = nullptr;
  ok = ok && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    h->use_graphs = false;
    return false;
  }
  h->pcg_graph = g;
  h->pcg_exec = exec;
  h->gk_op = op.kind;
  h->gk_A = op.key(); h->gk_lda = lda; h->gk_m = m; h->gk_n = n; h->gk_ell = ell;
  h->gk_D = D; h->gk_U = U; h->gk_ld = ld;
  return true;
}

// Route of an FP64 PCG solve (NYS_ROUTE_*): a thread-block cluster when a
// cluster plan exists (A on chip; for a batch worker also A in L2), else one
// cooperative launch when it fits, else the graph of per-step kernels;
// NYS_PCG_PATH restricts the choice (the cluster route then falls back to a
// throughput plan, so that it can be tested on L2-resident A).
int fp64_route(nys_solver* h, int m, int n, int ell) {
  if (h->cp_m != m || h->cp_n != n || h->cp_ell != ell) {
    h->cp_ok = pcg_cluster_plan(m, n, ell, h->plan_policy, &h->cp);
    h->cp_m = m; h->cp_n = n; h->cp_ell = ell;
  }
  if ((h->pcg_path == 0 || h->pcg_path == 1) && h->cp_ok)
    return h->cp.a_smem ? NYS_ROUTE_CLUSTER_SMEM : NYS_ROUTE_CLUSTER_L2;
  if ((h->pcg_path == 0 || h->pcg_path == 2) && pcg_persistent_fits(m, n, ell)) return NYS_ROUTE_COOPERATIVE;
  return NYS_ROUTE_GRAPH;
}

// Run PCG on (A D A^T + delta I) dy = xi; dy is written into `out`.
int run_pcg(nys_solver* h, int m, int n, const OpSpec& op, double delta, int ell, const double* U, int ld,
            const double* lamh, const double* xi, double* out, double eta, int max_iter, int forced,
            int* iters) {
  PcgWork w = h->pw;
  w.x = h->pcg_x;
  CK(cudaEventRecord(h->ev_pcg0, h->st));
  // after the stream has been synchronised: add this solve's device time
  auto add_time = [&]() {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev_pcg0, h->ev_pcg1) == cudaSuccess) h->pcg_ms += ms;
    else cudaGetLastError();
  };
  // one-launch routes: report the count and whether the stop test was met
  auto finish_single = [&]() -> int {
    CK(cudaEventRecord(h->ev_pcg1, h->st));
    int rc = sync_scalars(h, 0);
    if (rc != NYS_OK) return rc;
    add_time();
    *iters = h->h_si[SI_ITERS];
    if (forced < 0 && *iters >= max_iter) {
      CK(cudaMemcpyAsync(h->h_red, h->sd, sizeof(double) * SD_COUNT, cudaMemcpyDeviceToHost, h->st));
      CK(cudaStreamSynchronize(h->st));
      if (!(h->h_red[SD_RR] <= h->h_red[SD_ETA2] * h->h_red[SD_BNORM2])) return NYS_WARN_PCG_MAXITER;
    }
    return NYS_OK;
  };
  const int route = op.kind == 0 ? fp64_route(h, m, n, ell) : NYS_ROUTE_GRAPH;
  if (route == NYS_ROUTE_CLUSTER_SMEM || route == NYS_ROUTE_CLUSTER_L2) {
    // small problem: the whole solve inside one thread-block cluster
    ClusterPcgTask t{};
    t.m = m; t.n = n; t.ell = ell; t.ld = ld; t.lda = op.lda;
    t.A = op.A; t.D = op.D; t.U = U; t.lam = lamh; t.xi = xi;
    t.delta = delta; t.eta2 = eta * eta; t.max_iter = max_iter; t.forced = forced;
    t.x = out; t.iters = h->si + SI_ITERS; t.sd = h->sd; t.err = h->si + SI_ERR;
    CK(pcg_cluster_f64(h->st, h->cp, t, nullptr, 1));
    return finish_single();
  }
  if (route == NYS_ROUTE_COOPERATIVE) {
    // small problem: the whole solve in one cooperative launch
    CK(pcg_persistent_f64(h->st, m, n, op.A, op.lda, op.D, delta, ell, U, ld, lamh, xi, eta, max_iter, forced,
                          w, h->red.part, RedBuf::kPartCap, h->cw.bar, h->sd, h->si, h->num_sms));
    CK(cudaMemcpyAsync(out, w.x, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->st));
    return finish_single();
  }
  CK(pcg_setup_f64(h->st, m, ell, U, ld, lamh, delta, xi, eta, max_iter, forced, w, h->sd, h->si, h->red));
  const int limit = forced >= 0 ? forced : max_iter;
  if (ensure_pcg_graph(h, m, n, op, ell, U, ld)) {
    CK(cudaGraphLaunch(h->pcg_exec, h->st));
    CK(cudaEventRecord(h->ev_pcg1, h->st));
    CK(cudaMemcpyAsync(out, w.x, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->st));
    int rc = sync_scalars(h, 0);
    if (rc != NYS_OK) return rc;
    add_time();
    const int it = h->h_si[SI_ITERS];
    count_launches(h->g_kernels_per_iter * (unsigned)std::max(it, 1));
  } else {
    int issued = 0, chunk = 2;
    while (true) {
      int rc = sync_scalars(h, 0);
      if (rc != NYS_OK) return rc;
      if (h->h_si[SI_DONE] || issued >= limit) break;
      const int todo = std::min(chunk, limit - issued);
      for (int k = 0; k < todo; ++k) CK(issue_pcg_iteration(h, h->st, m, n, op, ell, U, ld, w));
      issued += todo;
      chunk = std::min(chunk * 2, 16);
    }
    CK(cudaEventRecord(h->ev_pcg1, h->st));
    CK(cudaEventSynchronize(h->ev_pcg1));
    add_time();
    CK(cudaMemcpyAsync(out, w.x, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->st));
  }
  *iters = h->h_si[SI_ITERS];
  if (forced < 0 && *iters >= max_iter) {
    // the stop test ran inside the last update; report whether it was met
    CK(cudaMemcpyAsync(h->h_red, h->sd, sizeof(double) * SD_COUNT, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (!(h->h_red[SD_RR] <= h->h_red[SD_ETA2] * h->h_red[SD_BNORM2])) return NYS_WARN_PCG_MAXITER;
  }
  return NYS_OK;
}

int run_pcg(nys_solver* h, int m, int n, const double* A, long long lda, const double* D, double delta,
            int ell, const double* U, int ld, const double* lamh, const double* xi, double* out, double eta,
            int max_iter, int forced, int* iters) {
  OpSpec op{};
  op.kind = 0;
  op.A = A;
  op.lda = lda;
  op.D = D;
  return run_pcg(h, m, n, op, delta, ell, U, ld, lamh, xi, out, eta, max_iter, forced, iters);
}

// The (P~) terms of one Newton system of Algorithm 4 (free and
// box-constrained variables): kinds, w, s, the right-hand sides r_u (null:
// zero, the corrector) and r_ws, and where dw, ds go.  A null BoxTerms
// pointer means problem (P), every x_j >= 0.
struct BoxTerms {
  BoxVectors v;
  const double* r_u = nullptr;
  const double* r_ws = nullptr;
  double* dw = nullptr;
  double* ds = nullptr;
};

// t = D (r_d + xi_au) into h->t_n (Algorithm 4, first step)
int newton_rhs(nys_solver* h, int n, const double* x, const double* D, const double* r_d, const double* r_xz,
               const BoxTerms* bt) {
  if (bt) CK(box_newton_rhs_f64(h->st, n, bt->v, D, r_d, bt->r_u, r_xz, bt->r_ws, x, h->t_n));
  else CK(newton_rhs_f64(h->st, n, D, r_d, r_xz, x, h->t_n));
  return NYS_OK;
}

// dx, dz (and dw, ds) from g = A^T dy in h->g_n (Algorithm 4, third step)
int newton_back(nys_solver* h, int n, const double* x, const double* z, const double* D, const double* r_d,
                const double* r_xz, const BoxTerms* bt, double* dx, double* dz) {
  if (bt) CK(box_newton_back_f64(h->st, n, bt->v, D, h->g_n, r_d, bt->r_u, r_xz, bt->r_ws, x, z, dx, dz, bt->dw,
                                 bt->ds));
  else CK(newton_back_f64(h->st, n, D, h->g_n, r_d, r_xz, x, z, dx, dz));
  return NYS_OK;
}

// Algorithm 4, first half: xi = r_p + A D (r_d + xi_au) into h->xi
// (xi_au = -X^{-1} r_xz for problem (P)).
int newton_begin(nys_solver* h, int m, int n, const double* A, long long lda, const double* x,
                 const double* D, const double* r_d, const double* r_p, const double* r_xz,
                 const BoxTerms* bt = nullptr) {
  const int rc = newton_rhs(h, n, x, D, r_d, r_xz, bt);
  if (rc != NYS_OK) return rc;
  CK(gemv_n_f64(h->st, m, n, A, lda, h->t_n, r_p ? 1.0 : 0.0, r_p, h->xi, nullptr, nullptr, h->split_buf,
                h->split_cap));
  return NYS_OK;
}

// Algorithm 4, second half: dx = D (A^T dy - r_d - xi_au), dz = X^{-1} (r_xz - Z dx)
// (and dw, ds for problem (P~)).
int newton_end(nys_solver* h, int m, int n, const double* A, long long lda, const double* x,
               const double* z, const double* D, const double* r_d, const double* r_xz, const double* dy,
               double* dx, double* dz, const BoxTerms* bt = nullptr) {
  CK(gemv_t_f64(h->st, m, n, A, lda, dy, nullptr, h->g_n, h->split_buf, h->split_cap));
  return newton_back(h, n, x, z, D, r_d, r_xz, bt, dx, dz);
}

// Algorithm 4: Newton direction through the normal equations.
int newton(nys_solver* h, int m, int n, const double* A, long long lda, const double* x,
           const double* z, const double* D, double delta, const double* r_d, const double* r_p,
           const double* r_xz, int ell, const double* U, int ld, const double* lamh, double eta,
           int max_iter, int forced, double* dx, double* dy, double* dz, int* iters) {
  int rc = newton_begin(h, m, n, A, lda, x, D, r_d, r_p, r_xz);
  if (rc != NYS_OK) return rc;
  rc = run_pcg(h, m, n, A, lda, D, delta, ell, U, ld, lamh, h->xi, dy, eta, max_iter, forced, iters);
  if (rc < 0) return rc;
  const int rc2 = newton_end(h, m, n, A, lda, x, z, D, r_d, r_xz, dy, dx, dz);
  return rc2 != NYS_OK ? rc2 : rc;
}

// ---------------------------------------------------------------- precision form
// Problem view shared by both forms.
struct Prob {
  int m, n;
  int lp;                 // 0: FP64 A; 1: FP32 A with BF16 copies
  const double* A64;
  const float* Af;
  long long lda;
};

// out = A x + beta v (accurate: FP64 A, or FP32 A with float-float sums)
int op_Ax(nys_solver* h, const Prob& P, const double* x, double beta, const double* v, double* out) {
  if (!P.lp) {
    CK(gemv_n_f64(h->st, P.m, P.n, P.A64, P.lda, x, beta, v, out, nullptr, nullptr, h->split_buf, h->split_cap));
  } else {
    CK(split_ff(h->st, P.n, (int)align_up(P.n, 8), x, nullptr, h->fh, h->fl));
    CK(gemv_rows_ff(h->st, P.m, P.n, P.Af, P.lda, h->fh, h->fl, nullptr, beta, v, out, nullptr, nullptr,
                    h->lp_part, h->lp_part_cap));
  }
  return NYS_OK;
}

// out = scale .* (A^T y)
int op_Aty(nys_solver* h, const Prob& P, const double* y, const double* scale, double* out) {
  if (!P.lp) {
    CK(gemv_t_f64(h->st, P.m, P.n, P.A64, P.lda, y, scale, out, h->split_buf, h->split_cap));
  } else {
    CK(split_ff(h->st, P.m, (int)align_up(P.m, 8), y, nullptr, h->fh, h->fl));
    CK(gemv_rows_ff(h->st, P.n, P.m, h->AfT, h->ld_ft, h->fh, h->fl, scale, 0.0, nullptr, out, nullptr, nullptr,
                    h->lp_part, h->lp_part_cap));
  }
  return NYS_OK;
}

// Precision-form sketch from Omega in h->Om (FP64, leading dimension h->ld)
// and the BF16 copies of A in h->Ab / h->AbT: Omega is rounded to BF16 in
// place (both views then hold the same test matrix), T = A^T Omega on the
// tensor cores with T' = BF16(D .* T) written by the GEMM, Y = A T' (FP32
// accumulation) widened to FP64 into Y (leading dimension ldy).
int lp_sketch(nys_solver* h, int m, int n, int ell, const double* D, double* Y, int ldy) {
  CK(round_panel_bf16(h->st, m, ell, h->Om, h->ld, h->Omb, (int)h->ld_om));
  int* err = h->si + SI_ERR;
  CK(umma_gemm_bf16(h->st, n, ell, m, h->AbT, h->ld_bt, h->Omb, h->ld_om, h->upart, h->upart_cap, h->num_sms, 1,
                    D, h->Tb, h->ld_tb, err));
  CK(umma_gemm_bf16(h->st, m, ell, n, h->Ab, h->ld_b, h->Tb, h->ld_tb, h->upart, h->upart_cap, h->num_sms, 0,
                    nullptr, h->Y32, h->ld, err));
  CK(panel_f32_to_f64(h->st, m, ell, h->Y32, h->ld, Y, ldy));
  return NYS_OK;
}

// Y = A (D .* (A^T Omega_k)) into h->Y, Omega_k into h->Om (FP64 panels).
int op_sketch(nys_solver* h, const Prob& P, int k, int ell, const double* D, int ell_stride = 0) {
  const nys_options& o = h->opt;
  CK(gaussian_omega(h->st, o.seed, k, P.m, ell_stride > 0 ? ell_stride : ell, h->Om, h->ld, ell));
  if (!P.lp) {
    CK(sketch_f64(h->st, P.m, P.n, P.A64, P.lda, D, ell, h->Om, h->ld, h->Y, h->T, h->ld_t, h->split_buf,
                  h->split_cap));
    return NYS_OK;
  }
  return lp_sketch(h, P.m, P.n, ell, D, h->Y, (int)h->ld);
}

// Precision-form Newton direction: Algorithm 4 with the normal equations
// solved in two stages.  xi, the refinement residual and the back
// substitution use the FP32 problem matrix with float-float accumulation.
// Stage 1 (iterative refinement): corrections from Nystrom PCG on the BF16
// operator, while each one at least halves the residual (mixed-precision
// refinement contracts only while kappa * u_bf16 < 1).  Stage 2: one PCG solve
// of the remaining residual on the float-float FP32 operator, which is the
// problem's operator to ~1e-13, to the outer tolerance.
// kind 1: BF16 copies; 4: FP8 copies with row scales; 2: the FP32 problem
// matrix; 3: the FP32 matrix with float-float sums.
LpOperator make_lp_op(nys_solver* h, const Prob& P, int kind, const double* D) {
  LpOperator op{};
  op.ff = kind == 3;
  op.D64 = D;
  op.t64 = h->u_n;
  op.xh = h->fh;
  op.xl = h->fl;
  op.ld_npad = (int)align_up(P.n, 8);
  op.a_type = kind == 1 ? kLpBf16 : kind == 4 ? kLpFp8 : kLpFp32;
  if (kind == 1) {
    op.A = h->Ab; op.lda = h->ld_b; op.AT = h->AbT; op.ldat = h->ld_bt;
  } else if (kind == 4) {
    op.A = h->A8; op.lda = h->ld_q; op.AT = h->A8T; op.ldat = h->ld_qt;
    op.rs32 = h->rs32; op.rs64 = h->rs64;
  } else {
    op.A = P.Af; op.lda = P.lda; op.AT = h->AfT; op.ldat = h->ld_ft;
  }
  op.Df = h->Df;
  op.xf = h->xf;
  op.tf = h->tf;
  op.ld_mpad = (int)h->ld_bt;
  op.part = h->lp_part;
  op.part_cap = h->lp_part_cap;
  return op;
}

int newton_lp(nys_solver* h, const Prob& P, const double* x, const double* z, const double* D, double delta,
              const double* r_d, const double* r_p, const double* r_xz, int ell, double eta, int max_iter,
              double* dx, double* dy, double* dz, int* iters, int* refine, const BoxTerms* bt) {
  const int m = P.m, n = P.n;
  int rc = newton_rhs(h, n, x, D, r_d, r_xz, bt);
  if (rc != NYS_OK) return rc;
  rc = op_Ax(h, P, h->t_n, r_p ? 1.0 : 0.0, r_p, h->xi);
  if (rc != NYS_OK) return rc;
  CK(dot_f64(h->st, m, h->xi, h->xi, h->red_out + 12, h->red));
  rc = sync_scalars_at(h, 12, 1);
  if (rc != NYS_OK) return rc;
  const double xin = std::sqrt(h->h_red[12]);
  CK(cudaMemsetAsync(h->dyacc, 0, sizeof(double) * m, h->st));
  CK(cudaMemcpyAsync(h->rr, h->xi, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->st));
  CK(to_f32(h->st, n, (int)align_up(n, 8), D, nullptr, h->Df));
  double rn = xin;
  int total = 0, steps = 0, warn = NYS_OK;
  bool bf16_stage = h->lp_bf16_stage;
  const int max_bf16_steps = 6;
  while (xin > 0.0 && rn > eta * xin) {
    const bool final_stage = !bf16_stage || steps >= max_bf16_steps;
    OpSpec op{};
    op.kind = final_stage ? 3 : (h->opt.precision_mode == 2 ? 4 : 1);
    op.lp = make_lp_op(h, P, op.kind, D);
    // inner tolerance relative to the current residual
    const double need = eta * xin / rn;
    const double eta_in = final_stage ? need : std::min(0.5, std::max(1e-3, 0.5 * need));
    int it = 0;
    rc = run_pcg(h, m, n, op, delta, ell, h->U, h->ld, h->lamh, h->rr, h->ecorr, eta_in, max_iter, -1, &it);
    if (rc < 0) return rc;
    if (rc > 0) warn = rc;
    total += it;
    ++steps;
    CK(axpby_f64(h->st, m, 1.0, h->ecorr, 1.0, h->dyacc, h->dyacc));
    if (final_stage) {
      // the float-float operator is the problem's: its PCG residual is the
      // outer residual (to ~1e-13), no further correction needed
      break;
    }
    // r = xi - (A D A^T + delta I) dy  (FP32 A, float-float sums)
    rc = op_Aty(h, P, h->dyacc, D, h->u_n);
    if (rc != NYS_OK) return rc;
    rc = op_Ax(h, P, h->u_n, delta, h->dyacc, h->nd_m);
    if (rc != NYS_OK) return rc;
    CK(axpby_f64(h->st, m, 1.0, h->xi, -1.0, h->nd_m, h->rr));
    CK(dot_f64(h->st, m, h->rr, h->rr, h->red_out + 12, h->red));
    rc = sync_scalars_at(h, 12, 1);
    if (rc != NYS_OK) return rc;
    const double rn_prev = rn;
    rn = std::sqrt(h->h_red[12]);
    if (!std::isfinite(rn)) return fail(h, NYS_ERR_NUMERIC, "non-finite refinement residual");
    if (rn > 0.5 * rn_prev) {
      bf16_stage = false;               // BF16 corrections stopped contracting:
      h->lp_bf16_stage = false;         // finish this and later systems on the FP32 operator
    }
  }
  CK(cudaMemcpyAsync(dy, h->dyacc, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->st));
  rc = op_Aty(h, P, dy, nullptr, h->g_n);
  if (rc != NYS_OK) return rc;
  rc = newton_back(h, n, x, z, D, r_d, r_xz, bt, dx, dz);
  if (rc != NYS_OK) return rc;
  *iters = total;
  *refine = steps;
  return warn;
}

}  // namespace

// One IP-PMM solve (Algorithm 6 with the Algorithm 5 predictor-corrector) as
// a resumable sequence of phases, so that a driver can stop it where a
// Newton system's PCG solve is due: nys_solve runs one to the end, calling
// run_pcg for each request; nys_solve_batched advances many in lock step and
// serves the requests of all of them with one launch.
struct PcgRequest {
  bool active = false;
  const double *A = nullptr, *D = nullptr, *xi = nullptr;
  long long lda = 0;
  double* out = nullptr;
  double delta = 0.0, eta = 0.0;
  int max_iter = 0, forced = -1;
  int rc = NYS_OK, iters = 0;       // filled in by whoever serves the request
};

struct IpmRun {
  nys_solver* h = nullptr;
  const nys_problem* p = nullptr;
  nys_result* r = nullptr;
  std::chrono::steady_clock::time_point t0, tk0;
  int m = 0, n = 0, lp = 0, ell = 0;
  int ell_max = 0, ell_lo = 0;  // adaptive sketch size: bounds (ell = the current l_k)
  long long lda = 0;
  Prob P{};
  const double* A = nullptr;
  const double *b = nullptr, *c = nullptr, *q = nullptr;
  double bnorm = 0.0, cnorm = 0.0, rho = 0.0, delta = 0.0, mu = 0.0, mu_prev = 0.0;
  double rel_p = 0.0, rel_d = 0.0, eta = 0.0, t_pre = 0.0;
  // PMM parameter update: relative primal / dual infeasibility at the last
  // re-centring of lambda / zeta (negative until the first iteration's top
  // sets them, unless a resumed problem supplies them)
  double ref_p = -1.0, ref_d = -1.0;
  // problem (P~): free and box-constrained variables present
  bool box = false;
  double n_mu = 0.0;            // |I u J| + |J|, the divisor of mu
  double pnorm = 0.0;           // ||(b, u_J)||, the scale of the primal residual
  int forced_idx = 0, warn = NYS_OK, k = 0, status = NYS_WARN_MAXITER;
  int last_pred = 0, last_corr = 0;   // PCG counts of the previous iteration (preconditioner reuse)
  bool reused = false;                // this iteration kept the previous Nystrom factor
  int pcg_before = 0, ref_before = 0;
  bool done = false;
  PcgRequest req;

  int next_forced() {
    const nys_options& o = h->opt;
    const int* f = p->forced_override ? p->forced_pcg_iters : o.forced_pcg_iters;
    const int nf = p->forced_override ? p->n_forced_pcg : o.n_forced_pcg;
    if (f && forced_idx < nf) return f[forced_idx++];
    return -1;
  }
  int forced_ipm() const { return p->forced_override ? p->forced_ipm_iters : h->opt.forced_ipm_iters; }
  void log_pcg(int it) {
    r->pcg_iters_total += it;
    if (r->pcg_log && r->pcg_log_len < r->pcg_log_cap) r->pcg_log[r->pcg_log_len++] = it;
  }
  // a phase ends the solve with `code`
  void stop(int code) {
    status = code;
    done = true;
    req.active = false;
  }
  void request(double* out) {
    req.active = true;
    req.A = A; req.lda = lda; req.D = h->D; req.xi = h->xi; req.out = out;
    req.delta = delta; req.eta = eta; req.max_iter = h->opt.max_pcg_iter; req.forced = next_forced();
    req.rc = NYS_OK; req.iters = 0;
  }
  // the request's outcome: count it, keep a warning, stop on an error
  bool take_request() {
    req.active = false;
    if (req.rc < 0) { stop(req.rc); return false; }
    if (req.rc > 0) warn = req.rc;
    log_pcg(req.iters);
    return true;
  }
  // the (P~) terms of the predictor's and the corrector's Newton systems
  BoxTerms terms(bool corrector) const {
    BoxTerms t;
    t.v.vk = h->vk;
    t.v.w = h->w;
    t.v.s = h->s;
    t.r_u = corrector ? nullptr : h->r_u;
    t.r_ws = h->r_ws;
    t.dw = corrector ? h->dwc : h->dwp;
    t.ds = corrector ? h->dsc : h->dsp;
    return t;
  }
  // residuals of Eq. predictor-RHS at the current iterate and PMM parameters
  int residuals();
  // the practical initial point into h->x, y, z (and w, s)
  int practical_start();
  int start_pcg(const double* rhs, double* out);
  int start(nys_solver* h_, const nys_problem* p_, nys_result* r_);
  int top();
  int mid();
  int bottom();
  int finish();
  // the device-resident iteration (problems (P), FP64 form, cluster PCG)
  bool device_eligible();
  int dev_top();
  int dev_body();
  int device_prepare();
  int device_step();
  int device_collect();
  int device_solve();
  cudaGraphExec_t dev_exec = nullptr;
};

int IpmRun::start(nys_solver* h_, const nys_problem* p_, nys_result* r_) {
  h = h_; p = p_; r = r_;
  t0 = std::chrono::steady_clock::now();
  if (!p || !r) { done = true; return status = fail(h, NYS_ERR_ARG, "nys_solve: null problem or result"); }
  m = p->m; n = p->n;
  const nys_options& o = h->opt;
  lp = o.precision_mode >= 1;
  const bool given = o.start_mode == 0;
  if (m <= 0 || n <= 0 || m > h->max_m || n > h->max_n || p->lda < n ||
      p->a_dtype != (lp ? NYS_F32 : NYS_F64) || !p->A || !p->b || !p->c || !p->q ||
      (given && (!p->x0 || !p->y0 || !p->z0)) || (o.start_mode != 0 && o.start_mode != 1) ||
      !r->x || !r->y || !r->z || p->k0 < 0 || p->ell < 0) {
    done = true;
    return status = fail(h, NYS_ERR_ARG,
                         "nys_solve: bad problem (sizes, dtype for the precision mode, or null pointers)");
  }
  ell = std::min(std::min(h->ell_cap, m), p->ell > 0 ? p->ell : h->ell_cap);
  ell_max = ell;
  ell_lo = std::max(1, std::min(o.ell_min > 0 ? o.ell_min : ell_max / 8, ell_max));
  if (o.adapt_cost < 0 || o.ell_min < 0 || (o.adapt_cost > 0 && o.reuse_pcg > 0)) {
    done = true;
    return status = fail(h, NYS_ERR_ARG, "nys_solve: adapt_cost / ell_min negative, or adapt_cost with reuse_pcg");
  }
  lda = p->lda;
  r->status = NYS_OK;
  r->ipm_iters = 0;
  r->pcg_iters_total = 0;
  r->refine_steps = 0;
  r->pcg_log_len = 0;
  r->ell_log_len = 0;
  r->device_iteration = 0;
  h->fac_A = nullptr;          // U / lamh are about to be overwritten
  r->pcg_seconds = 0.0;
  r->sketches = 0;
  h->pcg_ms = 0.0;
  done = true;                 // until the setup below succeeds
  status = NYS_ERR_CUDA;

  // Problem data on the device (staged when the caller passes host memory).
  const size_t esz = lp ? sizeof(float) : sizeof(double);
  const void* Av = p->A;
  b = p->b; c = p->c; q = p->q;
  if (p->host) {
    const size_t a_bytes = align_up((size_t)m * lda * esz, 256);
    const size_t need = a_bytes + 3 * align_up(sizeof(double) * (size_t)n, 256) +
                        align_up(sizeof(double) * (size_t)m, 256);
    if (need > h->stage_bytes) {
      if (h->stage) cudaFree(h->stage);
      h->stage = nullptr;
      h->stage_bytes = 0;
      if (cudaMalloc(&h->stage, need) != cudaSuccess) {
        cudaGetLastError();
        return status = fail(h, NYS_ERR_NOMEM, "nys_solve: cannot stage a host problem of %zu bytes", need);
      }
      h->stage_bytes = need;
    }
    char* s = static_cast<char*>(h->stage);
    void* dA = s;
    double* db = reinterpret_cast<double*>(s + a_bytes);
    double* dc = reinterpret_cast<double*>(s + a_bytes + align_up(sizeof(double) * m, 256));
    double* dq = reinterpret_cast<double*>(reinterpret_cast<char*>(dc) + align_up(sizeof(double) * n, 256));
    CK(cudaMemcpyAsync(dA, p->A, (size_t)m * lda * esz, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(db, p->b, sizeof(double) * m, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(dc, p->c, sizeof(double) * n, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(dq, p->q, sizeof(double) * n, cudaMemcpyHostToDevice, h->st));
    Av = dA; b = db; c = dc; q = dq;
  }
  P = Prob{m, n, lp, lp ? nullptr : static_cast<const double*>(Av), lp ? static_cast<const float*>(Av) : nullptr, lda};
  A = P.A64;
  h->lp_bf16_stage = true;
  if (lp)   // BF16 A and A^T for the inner solves and the sketch, FP32 A^T for residuals
    CK(convert_transpose(h->st, m, n, 0, Av, lda, h->Ab, h->ld_b, h->AbT, h->ld_bt, h->AfT, h->ld_ft));
  if (o.precision_mode == 2)   // E4M3 A and A^T with A's row scales for the inner solves
    CK(quantize_fp8(h->st, m, n, static_cast<const float*>(Av), lda, h->rs32, h->rs64, h->A8, h->ld_q, h->A8T,
                    h->ld_qt));
  const cudaMemcpyKind kin = p->host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (given) {
    CK(cudaMemcpyAsync(h->x, p->x0, sizeof(double) * n, kin, h->st));
    CK(cudaMemcpyAsync(h->y, p->y0, sizeof(double) * m, kin, h->st));
    CK(cudaMemcpyAsync(h->z, p->z0, sizeof(double) * n, kin, h->st));
  }
  CK(cudaMemsetAsync(h->si, 0, sizeof(int) * SI_COUNT, h->st));
  box = p->var_kind != nullptr;
  if (box) {
    // kinds, u, w0, s0 into the handle's copies; the start kernel masks them
    // (u = w = s = 0 outside J, z_F = 0) and counts invalid entries
    CK(cudaMemcpyAsync(h->vk, p->var_kind, (size_t)n, kin, h->st));
    if (p->u) CK(cudaMemcpyAsync(h->uv, p->u, sizeof(double) * n, kin, h->st));
    else CK(cudaMemsetAsync(h->uv, 0, sizeof(double) * n, h->st));
    if (given && p->w0) CK(cudaMemcpyAsync(h->w, p->w0, sizeof(double) * n, kin, h->st));
    if (given && p->s0) CK(cudaMemcpyAsync(h->s, p->s0, sizeof(double) * n, kin, h->st));
    else CK(cudaMemsetAsync(h->s, 0, sizeof(double) * n, h->st));
    CK(box_start_f64(h->st, n, h->vk, h->uv, h->x, h->z, h->w, h->s, p->u != nullptr, given && p->w0 != nullptr,
                     given && p->s0 != nullptr, given ? 1 : 0, h->red_out + 10, h->red));
  }
  CK(dot_f64(h->st, m, b, b, h->red_out + 8, h->red));
  CK(dot_f64(h->st, n, c, c, h->red_out + 9, h->red));
  int rc = sync_scalars(h, box ? 13 : 10);
  if (rc != NYS_OK) return r->status = status = rc;
  bnorm = std::sqrt(h->h_red[8]);
  cnorm = std::sqrt(h->h_red[9]);
  pnorm = bnorm;
  if (box) {
    if (h->h_red[12] != 0.0)
      return r->status = status = fail(h, NYS_ERR_ARG,
                                       "nys_solve: %.0f invalid entries in var_kind / u / w0 / s0 (kind outside "
                                       "{0,1,2}; on J: u missing or non-finite, w0 or s0 missing or <= 0)",
                                       h->h_red[12]);
    n_mu = h->h_red[10];
    pnorm = std::sqrt(h->h_red[8] + h->h_red[11]);
  }
  if (!given) {
    rc = practical_start();
    if (rc < 0) return r->status = status = rc;
    if (rc > 0) warn = rc;
  }
  if (p->lam0) CK(cudaMemcpyAsync(h->lam, p->lam0, sizeof(double) * m, kin, h->st));
  else CK(cudaMemcpyAsync(h->lam, h->y, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->st));
  if (p->zeta0) CK(cudaMemcpyAsync(h->zeta, p->zeta0, sizeof(double) * n, kin, h->st));
  else CK(cudaMemcpyAsync(h->zeta, h->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
  rho = o.rho0;
  delta = o.delta0;
  ref_p = p->has_peu_ref ? p->peu_ref_p : -1.0;
  ref_d = p->has_peu_ref ? p->peu_ref_d : -1.0;
  if (o.adapt_cost > 0) ell = ell_lo;   // the practical start above used l_max
  status = NYS_WARN_MAXITER;
  done = false;
  return NYS_OK;
}

// One of the practical start's two solves: (A A^T + 10 I) out = rhs by Nystrom
// PCG with the factor in h->U, h->lamh (D = h->D = 1), to relative residual
// 1e-10; the FP64 route for the FP64 form, the FP32 matrix with float-float
// sums for the precision form.
int IpmRun::start_pcg(const double* rhs, double* out) {
  constexpr double kStartDelta = 10.0, kStartTol = 1e-10;
  int it = 0;
  if (!lp)
    return run_pcg(h, m, n, A, lda, h->D, kStartDelta, ell, h->U, h->ld, h->lamh, rhs, out, kStartTol,
                   h->opt.max_pcg_iter, -1, &it);
  CK(to_f32(h->st, n, (int)align_up(n, 8), h->D, nullptr, h->Df));
  OpSpec op{};
  op.kind = 3;
  op.lp = make_lp_op(h, P, 3, h->D);
  return run_pcg(h, m, n, op, kStartDelta, ell, h->U, h->ld, h->lamh, rhs, out, kStartTol, h->opt.max_pcg_iter, -1,
                 &it);
}

// The practical initial point (the supplement's construction): candidate
// x~ = u/2 + A^T v with (A A^T + 10 I) v = b - A u/2, y~ from
// (A A^T + 10 I) y~ = A (c + Q x~), the candidate's z~, w~, s~, and the shifts
// delta_p~, delta_d~ that make x_IJ, w_J, z_IJ, s_J strictly positive.
int IpmRun::practical_start() {
  const signed char* vk = box ? h->vk : nullptr;
  // Nystrom factor of N = A A^T (D = 1) from Omega_{k0}
  CK(fill_f64(h->st, n, 1.0, h->D));
  int rc = op_sketch(h, P, p->k0, ell, h->D);
  if (rc != NYS_OK) return rc;
  CK(nystrom_core_f64(h->st, m, ell, h->Y, h->Om, h->ld, h->U, h->lamh, h->sd, h->si, h->red, h->cw,
                      h->num_sms));
  int warn_ = NYS_OK;
  // x~ = u/2 + A^T v,  (A A^T + 10 I) v = b - A u/2
  if (box) {
    CK(axpby_f64(h->st, n, 0.5, h->uv, 0.0, h->uv, h->t_n));
    rc = op_Ax(h, P, h->t_n, 0.0, nullptr, h->Ax);
    if (rc != NYS_OK) return rc;
    CK(axpby_f64(h->st, m, 1.0, b, -1.0, h->Ax, h->xi));
  } else {
    CK(cudaMemcpyAsync(h->xi, b, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->st));
  }
  rc = start_pcg(h->xi, h->dyp);
  if (rc < 0) return rc;
  if (rc > 0) warn_ = rc;
  rc = op_Aty(h, P, h->dyp, nullptr, h->g_n);
  if (rc != NYS_OK) return rc;
  if (box) CK(axpby_f64(h->st, n, 0.5, h->uv, 1.0, h->g_n, h->x));
  else CK(cudaMemcpyAsync(h->x, h->g_n, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
  // y~:  (A A^T + 10 I) y~ = A (c + Q x~)
  CK(vmul_f64(h->st, n, q, h->x, h->t_n));
  CK(axpby_f64(h->st, n, 1.0, c, 1.0, h->t_n, h->t_n));
  rc = op_Ax(h, P, h->t_n, 0.0, nullptr, h->xi);
  if (rc != NYS_OK) return rc;
  rc = start_pcg(h->xi, h->y);
  if (rc < 0) return rc;
  if (rc > 0) warn_ = rc;
  rc = op_Aty(h, P, h->y, nullptr, h->Aty);
  if (rc != NYS_OK) return rc;
  // candidate z~, w~, s~ and the smallest primal / dual entries
  CK(start_candidate_f64(h->st, n, vk, c, q, h->uv, h->x, h->Aty, h->z, box ? h->w : nullptr,
                         box ? h->s : nullptr, h->red_out, h->red));
  rc = sync_scalars(h, 2);
  if (rc != NYS_OK) return rc;
  const double pmin = h->h_red[0], dmin = h->h_red[1];
  const double dp = std::isfinite(pmin) ? std::max(-1.5 * pmin, 0.0) : 0.0;
  const double dd = std::isfinite(dmin) ? std::max(-1.5 * dmin, 0.0) : 0.0;
  CK(start_sums_f64(h->st, n, vk, h->x, h->z, box ? h->w : nullptr, box ? h->s : nullptr, dp, dd, h->red_out,
                    h->red));
  rc = sync_scalars(h, 3);
  if (rc != NYS_OK) return rc;
  const double gamma = h->h_red[0], den_p = h->h_red[1], den_d = h->h_red[2];
  if (!std::isfinite(gamma) || !std::isfinite(den_p) || !std::isfinite(den_d))
    return fail(h, NYS_ERR_NUMERIC, "nys_solve: non-finite practical start");
  const double dpt = dp + (den_p != 0.0 ? 0.5 * gamma / den_p : 0.0);
  const double ddt = dd + (den_d != 0.0 ? 0.5 * gamma / den_d : 0.0);
  CK(start_shift_f64(h->st, n, vk, dpt, ddt, h->x, h->z, box ? h->w : nullptr, box ? h->s : nullptr));
  return warn_;
}

// Eq. predictor-RHS at the current iterate: r_d, r_p, r_xz (and r_u, r_ws).
// Problem (P): red_out = (||rd||^2, x^T z, ||b - Ax||^2); problem (P~):
// red_out = (||rd||^2, x_IJ^T z_IJ + w_J^T s_J, ||u_J - x_J - w_J||^2, ||b - Ax||^2).
int IpmRun::residuals() {
  if (!box) {
    CK(ipm_residuals_f64(h->st, m, n, b, c, q, h->x, h->y, h->z, h->Ax, h->Aty, h->lam, h->zeta,
                         rho, delta, h->r_d, h->r_p, h->r_xz, h->red_out, h->red));
    return NYS_OK;
  }
  CK(box_residuals_n_f64(h->st, n, h->vk, c, q, h->uv, h->x, h->z, h->w, h->s, h->Aty, h->zeta, rho, h->r_d,
                         h->r_u, h->r_xz, h->r_ws, h->red_out, h->red));
  CK(ipm_residuals_m_f64(h->st, m, b, h->Ax, h->y, h->lam, delta, h->r_p, h->red_out + 3, h->red));
  return NYS_OK;
}

// Top of an iteration: residuals, termination, PEU, scaling, sketch and core,
// then the predictor's Newton system (a PCG request, or solved in place by the
// precision form).
int IpmRun::top() {
  const nys_options& o = h->opt;
  int rc = op_Ax(h, P, h->x, 0.0, nullptr, h->Ax);
  if (rc == NYS_OK) rc = op_Aty(h, P, h->y, nullptr, h->Aty);
  if (rc == NYS_OK) rc = residuals();
  if (rc != NYS_OK) { stop(rc); return rc; }
  rc = sync_scalars(h, box ? 4 : 3);
  if (rc != NYS_OK) { stop(rc); return rc; }
  const double nrd = std::sqrt(h->h_red[0]);
  // (P~): the primal residual stacks Ax - b (red_out[3]) with u_J - x_J - w_J (red_out[2])
  const double nrp = box ? std::sqrt(h->h_red[3] + h->h_red[2]) : std::sqrt(h->h_red[2]);
  mu = box ? (n_mu > 0.0 ? h->h_red[1] / n_mu : 0.0) : h->h_red[1] / n;
  if (!std::isfinite(nrd) || !std::isfinite(nrp) || !std::isfinite(mu)) {
    stop(fail(h, NYS_ERR_NUMERIC, "non-finite residual at IPM iteration %d", k));
    return status;
  }
  rel_p = nrp / (1.0 + pnorm);
  rel_d = nrd / (1.0 + cnorm);
  if (ref_p < 0.0) ref_p = rel_p;     // the start point's infeasibilities
  if (ref_d < 0.0) ref_d = rel_d;
  if (k > 0) {
    // PMM parameter update (Algorithm 6, last step; the paper fixes only its
    // outcome, Tables 7-8).  Each estimate is re-centred on the iterate when
    // its infeasibility progressed (fell to 95% of the value at its last
    // re-centring, or meets tol, or that value already met tol) and its
    // parameter then shrinks by 1 - r; otherwise the estimate stays and the
    // parameter shrinks by 1 - (2/3) r.  lambda, delta follow the primal
    // infeasibility, zeta, rho the dual one; r = |mu_k - mu_{k-1}| / max.
    const double den = std::max(mu_prev, mu);
    const double r_mu = den > 0.0 ? std::fabs(mu - mu_prev) / den : 0.0;
    const double slow = 1.0 - (2.0 / 3.0) * r_mu;
    if (ref_p <= o.tol || rel_p <= std::max(0.95 * ref_p, o.tol)) {
      CK(cudaMemcpyAsync(h->lam, h->y, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->st));
      ref_p = rel_p;
      delta = (1.0 - r_mu) * delta;
    } else {
      delta = slow * delta;
    }
    if (ref_d <= o.tol || rel_d <= std::max(0.95 * ref_d, o.tol)) {
      CK(cudaMemcpyAsync(h->zeta, h->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
      ref_d = rel_d;
      rho = (1.0 - r_mu) * rho;
    } else {
      rho = slow * rho;
    }
    delta = std::max(o.reg_floor, delta);
    rho = std::max(o.reg_floor, rho);
    // predictor right-hand sides with the updated PMM parameters
    rc = residuals();
    if (rc != NYS_OK) { stop(rc); return rc; }
  }
  // Termination (reading of TC: relative infeasibilities and mu).
  if (forced_ipm() >= 0) {
    if (k >= forced_ipm()) {
      stop((rel_p <= o.tol && rel_d <= o.tol && mu <= o.tol) ? NYS_OK : NYS_WARN_MAXITER);
      return NYS_OK;
    }
  } else if (rel_p <= o.tol && rel_d <= o.tol && mu <= o.tol) {
    stop(NYS_OK);
    return NYS_OK;
  }
  if (k >= o.max_ipm_iter) { stop(NYS_WARN_MAXITER); return NYS_OK; }

  // N_k, Omega_k, Nystrom preconditioner (Algorithms 1-2).  With reuse_pcg
  // = R > 0 the previous factor is kept while the previous iteration's two
  // PCG solves took at most R iterations each.
  tk0 = std::chrono::steady_clock::now();
  if (box) CK(box_scaling_f64(h->st, n, h->vk, h->x, h->z, h->w, h->s, q, rho, h->D));
  else CK(scaling_f64(h->st, n, h->x, h->z, q, rho, h->D));
  reused = o.reuse_pcg > 0 && k > 0 && last_pred <= o.reuse_pcg && last_corr <= o.reuse_pcg;
  if (o.adapt_cost > 0 && k > 0) {
    // sketch size of this iteration from the previous one's PCG count
    // (integer tests, the same decisions as the oracle's)
    const long long pc = (long long)last_pred + last_corr, C = o.adapt_cost;
    if (pc * ell_max > 2 * C * ell && ell < ell_max) ell = std::min(ell_max, 2 * ell);
    else if (2 * pc * ell_max < C * ell && ell > ell_lo) ell = std::max(ell_lo, (ell + 1) / 2);
  }
  if (!reused) {
    if (r->ell_log && r->ell_log_len < r->ell_log_cap) r->ell_log[r->ell_log_len++] = ell;
    rc = op_sketch(h, P, p->k0 + k, ell, h->D, ell_max);
    if (rc != NYS_OK) { stop(rc); return rc; }
    CK(nystrom_core_f64(h->st, m, ell, h->Y, h->Om, h->ld, h->U, h->lamh, h->sd, h->si, h->red,
                        h->cw, h->num_sms));
    ++r->sketches;
    h->fac_A = lp ? nullptr : A;
    h->fac_m = m;
    h->fac_ell = ell;
  }
  eta = std::max(1e-10, std::min(1e-2, 0.1 * mu));
  t_pre = 0.0;
  if (h->trace) {
    cudaStreamSynchronize(h->st);
    t_pre = std::chrono::duration<double>(std::chrono::steady_clock::now() - tk0).count();
  }
  pcg_before = r->pcg_iters_total;
  ref_before = r->refine_steps;

  // Predictor (Algorithm 5, first step).
  const BoxTerms bt = terms(false);
  const BoxTerms* btp = box ? &bt : nullptr;
  if (lp) {
    int it = 0, ref = 0;
    rc = newton_lp(h, P, h->x, h->z, h->D, delta, h->r_d, h->r_p, h->r_xz, ell, eta, o.max_pcg_iter,
                   h->dxp, h->dyp, h->dzp, &it, &ref, btp);
    r->refine_steps += ref;
    req.rc = rc;
    req.iters = it;
    req.active = false;
    return NYS_OK;
  }
  rc = newton_begin(h, m, n, A, lda, h->x, h->D, h->r_d, h->r_p, h->r_xz, btp);
  if (rc != NYS_OK) { stop(rc); return rc; }
  request(h->dyp);
  return NYS_OK;
}

// After the predictor's PCG: its direction, step lengths, mu_aff, and the
// corrector's Newton system.
int IpmRun::mid() {
  const nys_options& o = h->opt;
  last_pred = req.iters;
  if (!take_request()) return status;
  const BoxTerms btp_ = terms(false), btc_ = terms(true);
  const BoxTerms* btp = box ? &btp_ : nullptr;
  const BoxTerms* btc = box ? &btc_ : nullptr;
  if (!lp) {
    const int rc = newton_end(h, m, n, A, lda, h->x, h->z, h->D, h->r_d, h->r_xz, h->dyp, h->dxp, h->dzp, btp);
    if (rc != NYS_OK) { stop(rc); return rc; }
  }
  if (box) CK(box_step_ratios_f64(h->st, n, h->vk, h->x, h->dxp, h->w, h->dwp, h->z, h->dzp, h->s, h->dsp,
                                  h->red_out, h->red));
  else CK(step_ratios_f64(h->st, n, h->x, h->dxp, h->z, h->dzp, h->red_out, h->red));
  int rc = sync_scalars(h, 2);
  if (rc != NYS_OK) { stop(rc); return rc; }
  const double ap_bar = 0.995 * std::min(1.0, h->h_red[0]);
  const double ad_bar = 0.995 * std::min(1.0, h->h_red[1]);
  if (box) CK(box_mu_aff_f64(h->st, n, h->vk, h->x, h->dxp, h->z, h->dzp, h->w, h->dwp, h->s, h->dsp, ap_bar,
                             ad_bar, h->red_out, h->red));
  else CK(mu_aff_f64(h->st, n, h->x, h->dxp, h->z, h->dzp, ap_bar, ad_bar, h->red_out, h->red));
  rc = sync_scalars(h, 1);
  if (rc != NYS_OK) { stop(rc); return rc; }
  const double mu_aff = box ? (n_mu > 0.0 ? h->h_red[0] / n_mu : 0.0) : h->h_red[0] / n;
  const double mu_t = mu > 0.0 ? mu_aff * mu_aff * mu_aff / (mu * mu) : 0.0;

  // Corrector (Eq. corrector-RHS): r_d = r_p = 0 (and r_u = 0), r_xz = mu_t - dxp dzp
  // (and r_ws = mu_t - dwp dsp).
  if (box) CK(box_corrector_rhs_f64(h->st, n, h->vk, mu_t, h->dxp, h->dzp, h->dwp, h->dsp, h->r_xz, h->r_ws));
  else CK(corrector_rhs_f64(h->st, n, mu_t, h->dxp, h->dzp, h->r_xz));
  if (lp) {
    int it = 0, ref = 0;
    rc = newton_lp(h, P, h->x, h->z, h->D, delta, nullptr, nullptr, h->r_xz, ell, eta, o.max_pcg_iter,
                   h->dxc, h->dyc, h->dzc, &it, &ref, btc);
    r->refine_steps += ref;
    req.rc = rc;
    req.iters = it;
    req.active = false;
    return NYS_OK;
  }
  rc = newton_begin(h, m, n, A, lda, h->x, h->D, nullptr, nullptr, h->r_xz, btc);
  if (rc != NYS_OK) { stop(rc); return rc; }
  request(h->dyc);
  return NYS_OK;
}

// After the corrector's PCG: the combined direction and the step.
int IpmRun::bottom() {
  last_corr = req.iters;
  if (!take_request()) return status;
  const BoxTerms btc_ = terms(true);
  if (!lp) {
    const int rc = newton_end(h, m, n, A, lda, h->x, h->z, h->D, nullptr, h->r_xz, h->dyc, h->dxc, h->dzc,
                              box ? &btc_ : nullptr);
    if (rc != NYS_OK) { stop(rc); return rc; }
  }
  CK(add_dirs_f64(h->st, m, n, h->dxp, h->dyp, h->dzp, h->dxc, h->dyc, h->dzc));
  if (box) {
    // (dw, ds) += (dwp, dsp): the same kernel over n-vectors only (m = 0)
    CK(add_dirs_f64(h->st, 0, n, h->dwp, nullptr, h->dsp, h->dwc, nullptr, h->dsc));
    CK(box_step_ratios_f64(h->st, n, h->vk, h->x, h->dxc, h->w, h->dwc, h->z, h->dzc, h->s, h->dsc, h->red_out,
                           h->red));
  } else {
    CK(step_ratios_f64(h->st, n, h->x, h->dxc, h->z, h->dzc, h->red_out, h->red));
  }
  const int rc = sync_scalars(h, 2);
  if (rc != NYS_OK) { stop(rc); return rc; }
  const double ap = 0.995 * std::min(1.0, h->h_red[0]);
  const double ad = 0.995 * std::min(1.0, h->h_red[1]);
  CK(ipm_update_f64(h->st, m, n, ap, ad, h->dxc, h->dyc, h->dzc, h->x, h->y, h->z));
  // w moves with the primal step, s with the dual one
  if (box) CK(ipm_update_f64(h->st, 0, n, ap, ad, h->dwc, nullptr, h->dsc, h->w, nullptr, h->s));
  if (h->trace) {
    cudaStreamSynchronize(h->st);
    const double t_it = std::chrono::duration<double>(std::chrono::steady_clock::now() - tk0).count();
    std::fprintf(stderr,
                 "[nys] k=%d mu=%.3e rel_p=%.3e rel_d=%.3e rho=%.2e delta=%.2e ap=%.3f ad=%.3f pcg=%d "
                 "refine=%d sketch+core=%.1fms%s jacobi_sweeps=%d iter=%.1fms\n",
                 k, mu, rel_p, rel_d, rho, delta, ap, ad, r->pcg_iters_total - pcg_before,
                 r->refine_steps - ref_before, 1e3 * t_pre, reused ? " (reused)" : "", h->h_si[SI_SWEEPS],
                 1e3 * t_it);
  }
  mu_prev = mu;
  ++k;
  return NYS_OK;
}

// ---------------------------------------------------------------- device-resident iteration
// Problems (P) in the FP64 form whose PCG runs on a thread-block cluster and
// whose Nystrom core is plain kernel launches take this path: the decisions
// of top(), mid() and bottom() are made by the one-thread kernels of
// ipm_dev.cu, and one IPM iteration (its Newton steps and the next
// iteration's top) is one CUDA graph launch with one read-back of the device
// scalars.  The kernels, their order and their arithmetic are those of the
// host-driven phases.
bool IpmRun::device_eligible() {
  const nys_options& o = h->opt;
  if (!h->use_dev_ipm || !h->use_graphs || lp || box || h->trace || o.reuse_pcg > 0 || o.adapt_cost > 0) return false;
  if (2 * std::max(0, o.max_ipm_iter) + 8 > h->dev_log_cap) return false;
  const int nf = p->forced_override ? p->n_forced_pcg : o.n_forced_pcg;
  if (nf > h->dev_log_cap) return false;
  const int route = fp64_route(h, m, n, ell);
  if (route != NYS_ROUTE_CLUSTER_SMEM && route != NYS_ROUTE_CLUSTER_L2) return false;
  return nystrom_core_capturable(m, ell);
}

// Top of an iteration: A x, A^T y, residual sums, the scalar decisions, the
// re-centred estimates and the predictor's right-hand sides.
int IpmRun::dev_top() {
  int rc = op_Ax(h, P, h->x, 0.0, nullptr, h->Ax);
  if (rc == NYS_OK) rc = op_Aty(h, P, h->y, nullptr, h->Aty);
  if (rc != NYS_OK) return rc;
  CK(ipm_residuals_dev(h->st, m, n, b, c, q, h->x, h->y, h->z, h->Ax, h->Aty, h->lam, h->zeta, h->ipmd, h->r_d,
                       h->r_p, h->r_xz, h->red_out, h->red));
  CK(ipm_top_dev(h->st, h->ipmd, h->red_out, h->dtask, h->d_forced, h->si + SI_ERR));
  CK(ipm_recentre(h->st, m, n, h->ipmd, h->y, h->x, h->lam, h->zeta));
  CK(ipm_residuals_dev(h->st, m, n, b, c, q, h->x, h->y, h->z, h->Ax, h->Aty, h->lam, h->zeta, h->ipmd, h->r_d,
                       h->r_p, h->r_xz, h->red_out, h->red));
  return NYS_OK;
}

// Iteration k (Algorithm 6 with Algorithm 5) and the top of iteration k+1.
int IpmRun::dev_body() {
  const nys_options& o = h->opt;
  const int cap = h->dev_log_cap;
  CK(scaling_dev(h->st, n, h->x, h->z, q, h->ipmd, h->D));
  CK(gaussian_omega_dev(h->st, o.seed, &h->ipmd->k, p->k0, m, ell, h->Om, h->ld));
  CK(sketch_f64(h->st, m, n, A, lda, h->D, ell, h->Om, h->ld, h->Y, h->T, h->ld_t, h->split_buf, h->split_cap));
  CK(nystrom_core_f64(h->st, m, ell, h->Y, h->Om, h->ld, h->U, h->lamh, h->sd, h->si, h->red, h->cw,
                      h->num_sms));
  // predictor
  int rc = newton_begin(h, m, n, A, lda, h->x, h->D, h->r_d, h->r_p, h->r_xz);
  if (rc != NYS_OK) return rc;
  CK(pcg_cluster_f64(h->st, h->cp, ClusterPcgTask{}, h->dtask, 1));
  CK(ipm_after_pcg_dev(h->st, h->ipmd, h->dtask, h->si, h->sd, h->d_pcglog, cap));
  rc = newton_end(h, m, n, A, lda, h->x, h->z, h->D, h->r_d, h->r_xz, h->dyp, h->dxp, h->dzp);
  if (rc != NYS_OK) return rc;
  CK(step_ratios_f64(h->st, n, h->x, h->dxp, h->z, h->dzp, h->red_out, h->red));
  CK(ipm_steps_dev(h->st, h->ipmd, h->red_out, 0));
  CK(mu_aff_dev(h->st, n, h->x, h->dxp, h->z, h->dzp, h->ipmd, h->red_out, h->red));
  CK(ipm_mu_t_dev(h->st, h->ipmd, h->red_out));
  CK(corrector_rhs_dev(h->st, n, h->ipmd, h->dxp, h->dzp, h->r_xz));
  // corrector
  rc = newton_begin(h, m, n, A, lda, h->x, h->D, nullptr, nullptr, h->r_xz);
  if (rc != NYS_OK) return rc;
  CK(pcg_cluster_f64(h->st, h->cp, ClusterPcgTask{}, h->dtask + 1, 1));
  CK(ipm_after_pcg_dev(h->st, h->ipmd, h->dtask + 1, h->si, h->sd, h->d_pcglog, cap));
  rc = newton_end(h, m, n, A, lda, h->x, h->z, h->D, nullptr, h->r_xz, h->dyc, h->dxc, h->dzc);
  if (rc != NYS_OK) return rc;
  CK(add_dirs_f64(h->st, m, n, h->dxp, h->dyp, h->dzp, h->dxc, h->dyc, h->dzc));
  CK(step_ratios_f64(h->st, n, h->x, h->dxc, h->z, h->dzc, h->red_out, h->red));
  CK(ipm_steps_dev(h->st, h->ipmd, h->red_out, 1));
  CK(ipm_update_dev(h->st, m, n, h->ipmd, h->dxc, h->dyc, h->dzc, h->x, h->y, h->z));
  CK(ipm_iter_end_dev(h->st, h->ipmd));
  return dev_top();
}

// Device scalars and PCG tasks of this run, the top of iteration 0, and the
// iteration graph (captured once per problem and launch plan).
int IpmRun::device_prepare() {
  const nys_options& o = h->opt;
  IpmDev& hd = *h->h_ipmd;
  std::memset(&hd, 0, sizeof(hd));
  hd.rho = rho;
  hd.delta = delta;
  hd.ref_p = ref_p;
  hd.ref_d = ref_d;
  hd.tol = o.tol;
  hd.floor = o.reg_floor;
  hd.pden = 1.0 + pnorm;
  hd.dden = 1.0 + cnorm;
  hd.nmu = (double)n;
  hd.k0 = p->k0;
  hd.forced_ipm = forced_ipm();
  hd.max_ipm = o.max_ipm_iter;
  hd.max_pcg = o.max_pcg_iter;
  const int* f = p->forced_override ? p->forced_pcg_iters : o.forced_pcg_iters;
  const int nf = f ? (p->forced_override ? p->n_forced_pcg : o.n_forced_pcg) : 0;
  hd.n_forced = nf;
  if (nf > 0) CK(cudaMemcpyAsync(h->d_forced, f, sizeof(int) * nf, cudaMemcpyHostToDevice, h->st));
  CK(cudaMemcpyAsync(h->ipmd, &hd, sizeof(IpmDev), cudaMemcpyHostToDevice, h->st));
  ClusterPcgTask t[2] = {};
  for (int w = 0; w < 2; ++w) {
    t[w].m = m; t[w].n = n; t[w].ell = ell; t[w].ld = h->ld; t[w].lda = lda;
    t[w].A = A; t[w].D = h->D; t[w].U = h->U; t[w].lam = h->lamh; t[w].xi = h->xi;
    t[w].x = w == 0 ? h->dyp : h->dyc;
    t[w].iters = h->si + SI_ITERS; t[w].sd = h->sd; t[w].err = h->si + SI_ERR;
    t[w].t_ns = &h->ipmd->pcg_ns;
    t[w].max_iter = o.max_pcg_iter;
  }
  CK(cudaMemcpyAsync(h->dtask, t, sizeof(t), cudaMemcpyHostToDevice, h->st));
  CK(cudaMemsetAsync(h->si, 0, sizeof(int) * SI_COUNT, h->st));
  int rc = dev_top();
  if (rc != NYS_OK) return rc;
  // the iteration graph
  const void* key[5] = {A, b, c, q, reinterpret_cast<const void*>(h->U)};
  bool same = h->ipm_exec && h->ik_lda == lda && h->ik_m == m && h->ik_n == n && h->ik_ell == ell &&
              h->ik_C == h->cp.C && h->ik_as == h->cp.a_smem;
  for (int i = 0; i < 5 && same; ++i) same = h->ik_ptr[i] == key[i];
  if (!same) {
    drop_ipm_graph(h);
    cudaStream_t saved = h->st;
    h->st = h->cap_stream;
    const unsigned long long c0 = g_launches.load();
    cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    int brc = e == cudaSuccess ? dev_body() : NYS_ERR_CUDA;
    cudaGraph_t g = nullptr;
    cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(h->cap_stream, &g) : e;
    h->st = saved;
    const unsigned per = (unsigned)(g_launches.load() - c0);
    g_launches.fetch_sub(per);            // counted when the graph runs
    cudaGraphExec_t ex = nullptr;
    if (brc != NYS_OK || e2 != cudaSuccess || !g || cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      h->use_dev_ipm = false;             // this handle keeps the host-driven iteration
      return 1;
    }
    h->ipm_graph = g;
    h->ipm_exec = ex;
    h->ipm_kernels_body = per;
    for (int i = 0; i < 5; ++i) h->ik_ptr[i] = key[i];
    h->ik_lda = lda; h->ik_m = m; h->ik_n = n; h->ik_ell = ell; h->ik_C = h->cp.C; h->ik_as = h->cp.a_smem;
  }
  dev_exec = h->ipm_exec;
  CK(cudaMemcpyAsync(h->h_ipmd, h->ipmd, sizeof(IpmDev), cudaMemcpyDeviceToHost, h->st));
  return NYS_OK;
}

// After the previous read-back completed: launch the next iteration when the
// run is not done (returns 1 while iterations remain in flight, 0 when done).
int IpmRun::device_step() {
  if (h->h_ipmd->done) return 0;
  CK(cudaGraphLaunch(dev_exec, h->st));
  count_launches(h->ipm_kernels_body);
  CK(cudaMemcpyAsync(h->h_ipmd, h->ipmd, sizeof(IpmDev), cudaMemcpyDeviceToHost, h->st));
  return 1;
}

// Results of a finished device-resident run (stream synchronised).
int IpmRun::device_collect() {
  const IpmDev& hd = *h->h_ipmd;
  r->device_iteration = 1;
  const int nlog = std::min(hd.solves, h->dev_log_cap);
  if (nlog > 0) {
    CK(cudaMemcpyAsync(h->h_pcglog, h->d_pcglog, sizeof(int) * nlog, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
  }
  for (int i = 0; i < nlog; ++i) log_pcg(h->h_pcglog[i]);
  k = hd.k;
  mu = hd.mu;
  mu_prev = hd.mu_prev;
  rel_p = hd.rel_p;
  rel_d = hd.rel_d;
  rho = hd.rho;
  delta = hd.delta;
  ref_p = hd.ref_p;
  ref_d = hd.ref_d;
  eta = hd.eta;
  if (hd.warn) warn = hd.warn;
  r->sketches += hd.k;
  h->pcg_ms += 1e-6 * (double)hd.pcg_ns;
  if (hd.k > 0) {
    h->fac_A = A;
    h->fac_m = m;
    h->fac_ell = ell;
  }
  int code = hd.done ? hd.status : NYS_ERR_CUDA;
  if (code < 0) {
    if (h->h_si) {
      CK(cudaMemcpyAsync(h->h_si, h->si, sizeof(int) * SI_COUNT, cudaMemcpyDeviceToHost, h->st));
      CK(cudaStreamSynchronize(h->st));
    }
    const int e = check_err(h);
    code = fail(h, e != NYS_OK ? e : code, "device-resident IPM iteration stopped with status %d at k=%d",
                hd.status, hd.k);
  }
  stop(code);
  return NYS_OK;
}

// A whole solve on the device-resident path: 0 when it ran, 1 when this
// run must use the host-driven phases, < 0 on a CUDA failure.
int IpmRun::device_solve() {
  int rc = device_prepare();
  if (rc != NYS_OK) return rc;
  CK(cudaStreamSynchronize(h->st));
  while (true) {
    rc = device_step();
    if (rc < 0) return rc;
    if (rc == 0) break;
    CK(cudaStreamSynchronize(h->st));
  }
  return device_collect();
}

// Outputs and final measures.
int IpmRun::finish() {
  const cudaMemcpyKind kout = p->host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(r->x, h->x, sizeof(double) * n, kout, h->st));
  CK(cudaMemcpyAsync(r->y, h->y, sizeof(double) * m, kout, h->st));
  CK(cudaMemcpyAsync(r->z, h->z, sizeof(double) * n, kout, h->st));
  if (r->lam) CK(cudaMemcpyAsync(r->lam, h->lam, sizeof(double) * m, kout, h->st));
  if (r->zeta) CK(cudaMemcpyAsync(r->zeta, h->zeta, sizeof(double) * n, kout, h->st));
  if (box && r->w) CK(cudaMemcpyAsync(r->w, h->w, sizeof(double) * n, kout, h->st));
  if (box && r->s) CK(cudaMemcpyAsync(r->s, h->s, sizeof(double) * n, kout, h->st));
  CK(objective_terms_f64(h->st, m, n, q, c, b, h->x, h->y, h->z, h->red_out + 4, h->red));
  if (box) CK(dot_f64(h->st, n, h->uv, h->s, h->red_out + 8, h->red));     // u^T s of (D~)
  int rc2 = sync_scalars(h, box ? 9 : 8);
  const double xqx = h->h_red[4], cx = h->h_red[5], by = h->h_red[6];
  const double pobj = 0.5 * xqx + cx, dobj = by - 0.5 * xqx - (box ? h->h_red[8] : 0.0);
  r->ipm_iters = k;
  r->rel_primal = rel_p;
  r->rel_dual = rel_d;
  r->mu = mu;
  r->rel_gap = std::fabs(pobj - dobj) / (1.0 + std::fabs(pobj));
  r->rho = rho;
  r->delta = delta;
  r->peu_ref_p = ref_p;
  r->peu_ref_d = ref_d;
  if (status == NYS_OK && warn != NYS_OK) status = warn;
  if (status >= 0 && rc2 != NYS_OK) status = rc2;
  if (status >= 0 && h->h_red[7] != 0.0) status = fail(h, NYS_ERR_NUMERIC, "non-finite final iterate");
  if (status < 0) h->fac_A = nullptr;   // no factor to offer the adjoint
  r->status = status;
  r->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  r->pcg_seconds = h->pcg_ms * 1e-3;
  return status;
}

// Serve one run's PCG request on its own handle (any route).
void serve_single(IpmRun& run) {
  PcgRequest& q = run.req;
  nys_solver* h = run.h;
  q.rc = run_pcg(h, run.m, run.n, q.A, q.lda, q.D, q.delta, run.ell, h->U, h->ld, h->lamh, q.xi, q.out,
                 q.eta, q.max_iter, q.forced, &q.iters);
}

// ---------------------------------------------------------------- lock-step batches
// nys_solve_batched advances up to max_batch solves side by side, one host
// thread per solve, and meets at every Newton system: the thread that
// arrives last launches the PCG solves of all systems that have a cluster
// plan as one k_pcg_cluster launch over a task array (one cluster per
// system; clusters beyond what fits run as earlier ones finish), on the
// master handle's stream, ordered after each worker's preparation and before
// its continuation by events.  Systems without a cluster plan are solved by
// their own worker on the usual route.
struct BatchSlot {
  ClusterPlan plan;
  bool has_plan = false;
  bool batched = false;        // the pending request is in the current shared launch
  int acct_iters = -1;         // iterations of the previous shared launch, for its time share
};

struct Rendezvous {            // reusable barrier; the last thread to arrive runs `work` first
  std::mutex mu;
  std::condition_variable cv;
  int n = 0, waiting = 0;
  unsigned gen = 0;
  template <class F> void arrive(F&& work) {
    std::unique_lock<std::mutex> lk(mu);
    const unsigned g = gen;
    if (++waiting == n) {
      work();
      waiting = 0;
      ++gen;
      cv.notify_all();
    } else {
      cv.wait(lk, [&] { return gen != g; });
    }
  }
};

// Charge the previous shared launch's device time to its solves in proportion
// to their iterations, then launch the pending requests that have a plan.
int serve_batch(nys_solver* master, std::vector<IpmRun>& runs, std::vector<BatchSlot>& slots, bool& launched) {
  nys_solver* h = master;
  if (launched) {
    long long tot = 0;
    for (auto& sl : slots) if (sl.acct_iters > 0) tot += sl.acct_iters;
    float ms = 0.f;
    if (cudaEventSynchronize(master->ev_b1) == cudaSuccess &&
        cudaEventElapsedTime(&ms, master->ev_b0, master->ev_b1) == cudaSuccess && tot > 0) {
      for (size_t i = 0; i < runs.size(); ++i)
        if (slots[i].acct_iters > 0) runs[i].h->pcg_ms += ms * (double)slots[i].acct_iters / (double)tot;
    } else {
      cudaGetLastError();
    }
    for (auto& sl : slots) sl.acct_iters = -1;
    launched = false;
  }
  // group the planned requests by launch shape (cluster size, A on chip or not)
  std::vector<int> idx;
  for (size_t i = 0; i < runs.size(); ++i) {
    slots[i].batched = false;
    if (!runs[i].done && runs[i].req.active && slots[i].has_plan) idx.push_back((int)i);
  }
  if (idx.empty()) return NYS_OK;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
    const ClusterPlan &pa = slots[a].plan, &pb = slots[b].plan;
    return pa.C != pb.C ? pa.C > pb.C : pa.a_smem > pb.a_smem;
  });
  for (int i : idx) {
    nys_solver* w = runs[i].h;
    CK(cudaEventRecord(w->ev_req, w->st));
    CK(cudaStreamWaitEvent(master->st, w->ev_req, 0));
  }
  CK(cudaEventRecord(master->ev_b0, master->st));
  size_t g0 = 0;
  int gi = 0;
  while (g0 < idx.size()) {
    size_t g1 = g0;
    ClusterPlan gp = slots[idx[g0]].plan;
    while (g1 < idx.size() && slots[idx[g1]].plan.C == gp.C && slots[idx[g1]].plan.a_smem == gp.a_smem) {
      gp.smem_bytes = std::max(gp.smem_bytes, slots[idx[g1]].plan.smem_bytes);
      ++g1;
    }
    for (size_t k = g0; k < g1; ++k) {
      IpmRun& run = runs[idx[k]];
      nys_solver* w = run.h;
      const PcgRequest& q = run.req;
      ClusterPcgTask& t = master->h_tasks[k];
      t = ClusterPcgTask{};
      t.m = run.m; t.n = run.n; t.ell = run.ell; t.ld = w->ld; t.lda = q.lda;
      t.A = q.A; t.D = q.D; t.U = w->U; t.lam = w->lamh; t.xi = q.xi;
      t.delta = q.delta; t.eta2 = q.eta * q.eta; t.max_iter = q.max_iter; t.forced = q.forced;
      t.x = q.out; t.iters = w->si + SI_ITERS; t.sd = w->sd; t.err = w->si + SI_ERR;
    }
    // each launch shape on a stream of its own, forked from and joined back
    // into the master stream (groups run concurrently, not one after another)
    if (gi >= (int)master->group_streams.size()) {
      cudaStream_t gs = nullptr;
      cudaEvent_t ge = nullptr;
      CK(cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking));
      if (cudaEventCreateWithFlags(&ge, cudaEventDisableTiming) != cudaSuccess) {
        cudaStreamDestroy(gs);
        return fail(h, NYS_ERR_CUDA, "serve_batch: cannot create a group event");
      }
      master->group_streams.push_back(gs);
      master->group_events.push_back(ge);
    }
    cudaStream_t gs = master->group_streams[gi];
    CK(cudaStreamWaitEvent(gs, master->ev_b0, 0));
    CK(cudaMemcpyAsync(master->d_tasks + g0, master->h_tasks + g0, sizeof(ClusterPcgTask) * (g1 - g0),
                       cudaMemcpyHostToDevice, gs));
    CK(pcg_cluster_f64(gs, gp, master->h_tasks[g0], master->d_tasks + g0, (int)(g1 - g0)));
    CK(cudaEventRecord(master->group_events[gi], gs));
    CK(cudaStreamWaitEvent(master->st, master->group_events[gi], 0));
    ++gi;
    g0 = g1;
  }
  CK(cudaEventRecord(master->ev_b1, master->st));
  for (int i : idx) {
    CK(cudaStreamWaitEvent(runs[i].h->st, master->ev_b1, 0));
    slots[i].batched = true;
  }
  launched = true;
  return NYS_OK;
}

// After the rendezvous: the outcome of a shared-launch request (read like a
// one-launch route), or the request served on the worker's own route.
void finish_request(IpmRun& run, BatchSlot& slot) {
  PcgRequest& q = run.req;
  if (!q.active || run.done) return;
  if (!slot.batched) {
    serve_single(run);
    return;
  }
  nys_solver* h = run.h;
  slot.batched = false;
  int rc = sync_scalars(h, 0);
  if (rc != NYS_OK) { q.rc = rc; return; }
  q.iters = h->h_si[SI_ITERS];
  slot.acct_iters = std::max(q.iters, 1);
  q.rc = NYS_OK;
  if (q.forced < 0 && q.iters >= q.max_iter) {
    if (cudaMemcpyAsync(h->h_red, h->sd, sizeof(double) * SD_COUNT, cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
        cudaStreamSynchronize(h->st) != cudaSuccess) {
      q.rc = fail(h, NYS_ERR_CUDA, "reading a batched PCG outcome failed");
      return;
    }
    if (!(h->h_red[SD_RR] <= h->h_red[SD_ETA2] * h->h_red[SD_BNORM2])) q.rc = NYS_WARN_PCG_MAXITER;
  }
}

extern "C" {

void nys_default_options(nys_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-6;
  o->ell = 20;
  o->max_ipm_iter = 200;
  o->max_pcg_iter = 1000;
  o->seed = 0;
  o->precision_mode = 0;
  o->rho0 = 8.0;
  o->delta0 = 8.0;
  o->reg_floor = 5e-10;
  o->forced_pcg_iters = nullptr;
  o->n_forced_pcg = 0;
  o->forced_ipm_iters = -1;
  o->start_mode = 0;
  o->reuse_pcg = 0;
  o->adapt_cost = 0;
  o->ell_min = 0;
}

const char* nys_last_error(nys_handle h) { return h ? h->err.c_str() : "null handle"; }

unsigned long long nys_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int nys_create(nys_handle* out, const nys_options* opt, int max_m, int max_n, int max_batch,
               void* cuda_stream) {
  if (!out) return NYS_ERR_ARG;
  *out = nullptr;
  if (!opt || max_m <= 0 || max_n <= 0 || max_batch < 0 || opt->ell <= 0 || opt->tol <= 0.0 ||
      opt->max_ipm_iter < 0 || opt->max_pcg_iter < 0 || opt->precision_mode < 0 ||
      opt->precision_mode > 2 || (opt->precision_mode >= 1 && opt->ell > 512))
    return NYS_ERR_ARG;
  nys_solver* h = new nys_solver();
  h->opt = *opt;
  h->max_m = max_m;
  h->max_n = max_n;
  h->ell_cap = std::min(opt->ell, max_m);
  h->ld = (int)align_up(max_m, 2);
  h->ld_t = (int)align_up(max_n, 2);
  h->st = reinterpret_cast<cudaStream_t>(cuda_stream);
  h->max_batch = max_batch;
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    delete h;
    return NYS_ERR_CUDA;
  }
  h->arena_bytes = carve(h, nullptr);
  if (cudaMalloc(&h->arena, h->arena_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return NYS_ERR_NOMEM;
  }
  carve(h, static_cast<char*>(h->arena));
  if (cudaMallocHost(&h->h_red, sizeof(double) * 64) != cudaSuccess ||
      cudaMallocHost(&h->h_si, sizeof(int) * 64) != cudaSuccess ||
      cudaMallocHost(&h->h_ipmd, sizeof(IpmDev)) != cudaSuccess ||
      cudaMallocHost(&h->h_pcglog, sizeof(int) * h->dev_log_cap) != cudaSuccess) {
    cudaFree(h->arena);
    delete h;
    return NYS_ERR_NOMEM;
  }
  if (opt->precision_mode >= 1) {
    h->lp_bytes = carve_lp(h, nullptr);
    if (cudaMalloc(&h->lp_arena, h->lp_bytes) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(h->arena);
      delete h;
      return NYS_ERR_NOMEM;
    }
    carve_lp(h, static_cast<char*>(h->lp_arena));
    cudaMemsetAsync(h->lp_arena, 0, h->lp_bytes, h->st);
  }
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&h->ev_pcg0) != cudaSuccess || cudaEventCreate(&h->ev_pcg1) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_req, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&h->ev_b0) != cudaSuccess || cudaEventCreate(&h->ev_b1) != cudaSuccess) {
    cudaFree(h->arena);
    delete h;
    return NYS_ERR_CUDA;
  }
  if (const char* env = std::getenv("NYS_NO_GRAPHS")) h->use_graphs = (env[0] == '0');
  if (const char* env = std::getenv("NYS_PCG_PATH")) {
    const std::string v(env);
    h->pcg_path = v == "cluster" ? 1 : v == "cooperative" ? 2 : v == "graph" ? 3 : 0;
    if (h->pcg_path == 1) h->plan_policy = 2;
  }
  if (const char* env = std::getenv("NYS_TRACE")) h->trace = (env[0] != '0');
  if (const char* env = std::getenv("NYS_JACOBI_F32")) h->cw.f32_start = (env[0] != '0');
  if (const char* env = std::getenv("NYS_JACOBI_GRAM")) h->cw.gram = (env[0] != '0');
  if (const char* env = std::getenv("NYS_DEVICE_IPM")) h->use_dev_ipm = (env[0] != '0');
  if (const char* env = std::getenv("NYS_TRACE_TUNE")) h->trace_tune = (env[0] != '0');
  if (cudaMemsetAsync(h->arena, 0, h->arena_bytes, h->st) != cudaSuccess ||
      cudaStreamSynchronize(h->st) != cudaSuccess) {
    cudaFree(h->arena);
    delete h;
    return NYS_ERR_CUDA;
  }
  *out = h;
  return NYS_OK;
}

int nys_destroy(nys_handle h) {
  if (!h) return NYS_ERR_ARG;
  for (nys_solver* w : h->workers) nys_destroy(w);
  for (cudaStream_t s : h->worker_streams) cudaStreamDestroy(s);
  for (cudaStream_t s : h->group_streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : h->group_events) cudaEventDestroy(e);
  if (h->st) cudaStreamSynchronize(h->st);
  else cudaDeviceSynchronize();
  drop_pcg_graph(h);
  drop_ipm_graph(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->ev_pcg0) cudaEventDestroy(h->ev_pcg0);
  if (h->ev_pcg1) cudaEventDestroy(h->ev_pcg1);
  if (h->ev_req) cudaEventDestroy(h->ev_req);
  if (h->ev_b0) cudaEventDestroy(h->ev_b0);
  if (h->ev_b1) cudaEventDestroy(h->ev_b1);
  if (h->d_tasks) cudaFree(h->d_tasks);
  if (h->h_tasks) cudaFreeHost(h->h_tasks);
  if (h->tune_buf) cudaFree(h->tune_buf);
  cudaFree(h->arena);
  if (h->lp_arena) cudaFree(h->lp_arena);
  if (h->stage) cudaFree(h->stage);
  cudaFreeHost(h->h_red);
  cudaFreeHost(h->h_si);
  if (h->h_ipmd) cudaFreeHost(h->h_ipmd);
  if (h->h_pcglog) cudaFreeHost(h->h_pcglog);
  delete h;
  return NYS_OK;
}

int nys_scaling(nys_handle h, int n, const double* x, const double* z, const double* q, double rho,
                double* D) {
  if (!h) return NYS_ERR_ARG;
  if (n < 0 || !valid_ptr(x) || !valid_ptr(z) || !valid_ptr(q) || !valid_ptr(D))
    return fail(h, NYS_ERR_ARG, "nys_scaling: bad argument");
  CK(scaling_f64(h->st, n, x, z, q, rho, D));
  return NYS_OK;
}

int nys_normal_matvec(nys_handle h, int m, int n, int a_dtype, const void* A, long long lda,
                      const double* D, double delta, const double* v, double* out) {
  if (!h) return NYS_ERR_ARG;
  if (m <= 0 || n <= 0 || m > h->max_m || n > h->max_n || lda < n || a_dtype != NYS_F64 || !A ||
      !D || !v || !out || out == v)
    return fail(h, NYS_ERR_ARG, "nys_normal_matvec: bad argument");
  const double* Ad = static_cast<const double*>(A);
  CK(gemv_t_f64(h->st, m, n, Ad, lda, v, D, h->pw.t, h->split_buf, h->split_cap));
  CK(gemv_n_f64(h->st, m, n, Ad, lda, h->pw.t, delta, v, out, nullptr, nullptr, h->split_buf, h->split_cap));
  return NYS_OK;
}

int nys_normal_matvec_lp(nys_handle h, int m, int n, int a_dtype, const void* A, long long lda,
                         const void* AT, long long ldat, const double* D, double delta, const double* v,
                         double* out) {
  if (!h) return NYS_ERR_ARG;
  if (!h->lp_arena) return fail(h, NYS_ERR_ARG, "nys_normal_matvec_lp: not a precision-form handle");
  if (m <= 0 || n <= 0 || m > h->max_m || n > h->max_n || lda < n || ldat < m || !A || !AT || !D || !v ||
      !out || out == v || (a_dtype != NYS_BF16 && a_dtype != NYS_F32))
    return fail(h, NYS_ERR_ARG, "nys_normal_matvec_lp: bad argument");
  const int bf = a_dtype == NYS_BF16;
  CK(to_f32(h->st, n, (int)align_up(n, 8), D, nullptr, h->Df));
  CK(to_f32(h->st, m, (int)align_up(m, 8), v, nullptr, h->xf));
  CK(gemv_rows_lp(h->st, n, m, bf, AT, ldat, h->xf, h->Df, 0.0, nullptr, h->tf, 0, nullptr, nullptr, h->lp_part,
                  h->lp_part_cap));
  CK(gemv_rows_lp(h->st, m, n, bf, A, lda, h->tf, nullptr, delta, v, out, 1, nullptr, nullptr, h->lp_part,
                  h->lp_part_cap));
  return NYS_OK;
}

int nys_quantize_fp8(nys_handle h, int m, int n, const float* A, long long lda, void* Q, long long ldq,
                     void* QT, long long ldqt, float* row_scale) {
  if (!h) return NYS_ERR_ARG;
  if (!h->rs64) return fail(h, NYS_ERR_ARG, "nys_quantize_fp8: not a precision_mode 2 handle");
  if (m <= 0 || n <= 0 || m > h->max_m || lda < n || ldq < n || ldqt < m || !A || !Q || !QT || !row_scale)
    return fail(h, NYS_ERR_ARG, "nys_quantize_fp8: bad argument");
  CK(quantize_fp8(h->st, m, n, A, lda, row_scale, h->rs64, Q, ldq, QT, ldqt));
  return NYS_OK;
}

int nys_normal_matvec_fp8(nys_handle h, int m, int n, const void* Q, long long ldq, const void* QT,
                          long long ldqt, const float* row_scale, const double* D, double delta, const double* v,
                          double* out) {
  if (!h) return NYS_ERR_ARG;
  if (!h->rs64) return fail(h, NYS_ERR_ARG, "nys_normal_matvec_fp8: not a precision_mode 2 handle");
  if (m <= 0 || n <= 0 || m > h->max_m || n > h->max_n || ldq < n || ldqt < m || !Q || !QT || !row_scale || !D ||
      !v || !out || out == v)
    return fail(h, NYS_ERR_ARG, "nys_normal_matvec_fp8: bad argument");
  CK(panel_f32_to_f64(h->st, m, 1, row_scale, m, h->rs64, m));
  CK(to_f32(h->st, n, (int)align_up(n, 8), D, nullptr, h->Df));
  CK(to_f32(h->st, m, (int)align_up(m, 8), v, h->rs64, h->xf));
  CK(gemv_rows_lp(h->st, n, m, kLpFp8, QT, ldqt, h->xf, h->Df, 0.0, nullptr, h->tf, 0, nullptr, nullptr, h->lp_part,
                  h->lp_part_cap));
  CK(gemv_rows_lp(h->st, m, n, kLpFp8, Q, ldq, h->tf, row_scale, delta, v, out, 1, nullptr, nullptr, h->lp_part,
                  h->lp_part_cap));
  return NYS_OK;
}

int nys_gaussian(nys_handle h, unsigned long long seed, int k, int m, int ell, double* Omega, int ld) {
  if (!h) return NYS_ERR_ARG;
  if (m <= 0 || ell <= 0 || k < 0 || ld < m || !Omega)
    return fail(h, NYS_ERR_ARG, "nys_gaussian: bad argument");
  CK(gaussian_omega(h->st, seed, k, m, ell, Omega, ld));
  return NYS_OK;
}

int nys_sketch(nys_handle h, int m, int n, int a_dtype, const void* A, long long lda,
               const double* D, int ell, const double* Omega, double* Y, int ld) {
  if (!h) return NYS_ERR_ARG;
  if (m <= 0 || n <= 0 || m > h->max_m || n > h->max_n || lda < n || (a_dtype != NYS_F64 && a_dtype != NYS_F32) ||
      ell <= 0 || ell > h->ell_cap || ld < m || !A || !D || !Omega || !Y)
    return fail(h, NYS_ERR_ARG, "nys_sketch: bad argument");
  if (a_dtype == NYS_F32) {
    if (!h->lp_arena) return fail(h, NYS_ERR_ARG, "nys_sketch: FP32 A needs a precision-form handle");
    CK(cudaMemsetAsync(h->si + SI_ERR, 0, sizeof(int), h->st));
    CK(convert_transpose(h->st, m, n, 0, static_cast<const float*>(A), lda, h->Ab, h->ld_b, h->AbT, h->ld_bt,
                         nullptr, 0));
    CK(cudaMemcpy2DAsync(h->Om, sizeof(double) * h->ld, Omega, sizeof(double) * ld, sizeof(double) * m, ell,
                         cudaMemcpyDeviceToDevice, h->st));
    const int rc = lp_sketch(h, m, n, ell, D, Y, ld);
    if (rc != NYS_OK) return rc;
    return sync_scalars(h, 0);
  }
  CK(sketch_f64(h->st, m, n, static_cast<const double*>(A), lda, D, ell, Omega, ld, Y, h->T,
                h->ld_t, h->split_buf, h->split_cap));
  return NYS_OK;
}

int nys_nystrom(nys_handle h, int m, int ell, const double* Y, const double* Omega, int ld,
                double* U, double* lam, double* nu) {
  if (!h) return NYS_ERR_ARG;
  if (m <= 0 || ell <= 0 || ell > h->ell_cap || m > h->max_m || ld < m || ld > h->ld || !Y ||
      !Omega || !U || !lam || !nu)
    return fail(h, NYS_ERR_ARG, "nys_nystrom: bad argument");
  CK(cudaMemsetAsync(h->si + SI_ERR, 0, sizeof(int), h->st));
  CK(nystrom_core_f64(h->st, m, ell, Y, Omega, ld, U, lam, h->sd, h->si, h->red, h->cw, h->num_sms));
  CK(cudaMemcpyAsync(h->h_red, h->sd, sizeof(double) * SD_COUNT, cudaMemcpyDeviceToHost, h->st));
  int rc = sync_scalars(h, 0);
  *nu = h->h_red[SD_NU];
  if (rc != NYS_OK) return rc;
  if (h->h_si[SI_SWEEPS] > CoreWork::kMaxSweeps)
    return fail(h, NYS_ERR_NUMERIC, "one-sided Jacobi did not converge");
  return NYS_OK;
}

int nys_precond_apply(nys_handle h, int m, int ell, const double* U, int ld, const double* lam,
                      double delta, const double* r, double* out) {
  if (!h) return NYS_ERR_ARG;
  if (m <= 0 || ell <= 0 || ell > h->ell_cap || m > h->max_m || ld < m || !U || !lam || !r || !out ||
      out == r)
    return fail(h, NYS_ERR_ARG, "nys_precond_apply: bad argument");
  CK(precond_apply_f64(h->st, m, ell, U, ld, lam, delta, r, out, h->pw.s, h->pw.wts, h->red));
  return NYS_OK;
}

int nys_pcg(nys_handle h, int m, int n, int a_dtype, const void* A, long long lda, const double* D,
            double delta, int ell, const double* U, int ld, const double* lam, const double* xi,
            double* dy, double eta, int max_iter, int forced_iters, int* iters, double* res_norm) {
  if (!h) return NYS_ERR_ARG;
  if (m <= 0 || n <= 0 || m > h->max_m || n > h->max_n || lda < n || a_dtype != NYS_F64 ||
      ell <= 0 || ell > h->ell_cap || ld < m || !A || !D || !U || !lam || !xi || !dy || !iters ||
      !res_norm || max_iter < 0 || dy == xi)
    return fail(h, NYS_ERR_ARG, "nys_pcg: bad argument");
  CK(cudaMemsetAsync(h->si + SI_ERR, 0, sizeof(int), h->st));
  int rc = run_pcg(h, m, n, static_cast<const double*>(A), lda, D, delta, ell, U, ld, lam, xi, dy,
                   eta, max_iter, forced_iters, iters);
  CK(cudaMemcpyAsync(h->h_red, h->sd, sizeof(double) * SD_COUNT, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  *res_norm = std::sqrt(h->h_red[SD_RR]);
  return rc;
}

int nys_pcg_lp(nys_handle h, int m, int n, const float* A, long long lda, int op_dtype, const double* D,
               double delta, int ell, const double* U, int ld, const double* lam, const double* xi, double* dy,
               double eta, int max_iter, int forced_iters, int* iters, double* res_norm) {
  if (!h) return NYS_ERR_ARG;
  if (!h->lp_arena) return fail(h, NYS_ERR_ARG, "nys_pcg_lp: not a precision-form handle");
  if (m <= 0 || n <= 0 || m > h->max_m || n > h->max_n || lda < n || ell <= 0 || ell > h->ell_cap || ld < m ||
      !A || !D || !U || !lam || !xi || !dy || !iters || !res_norm || max_iter < 0 || dy == xi ||
      (op_dtype != NYS_BF16 && op_dtype != NYS_F32 && op_dtype != NYS_FP8E4M3) ||
      (op_dtype == NYS_FP8E4M3 && !h->rs64))
    return fail(h, NYS_ERR_ARG, "nys_pcg_lp: bad argument");
  CK(cudaMemsetAsync(h->si + SI_ERR, 0, sizeof(int), h->st));
  Prob P{m, n, 1, nullptr, A, lda};
  if (op_dtype == NYS_BF16)
    CK(convert_transpose(h->st, m, n, 0, A, lda, h->Ab, h->ld_b, h->AbT, h->ld_bt, nullptr, 0));
  else if (op_dtype == NYS_F32)
    CK(convert_transpose(h->st, m, n, 0, A, lda, nullptr, 0, nullptr, 0, h->AfT, h->ld_ft));
  else
    CK(quantize_fp8(h->st, m, n, A, lda, h->rs32, h->rs64, h->A8, h->ld_q, h->A8T, h->ld_qt));
  CK(to_f32(h->st, n, (int)align_up(n, 8), D, nullptr, h->Df));
  OpSpec op{};
  op.kind = op_dtype == NYS_BF16 ? 1 : op_dtype == NYS_F32 ? 3 : 4;
  op.lp = make_lp_op(h, P, op.kind, D);
  int rc = run_pcg(h, m, n, op, delta, ell, U, ld, lam, xi, dy, eta, max_iter, forced_iters, iters);
  CK(cudaMemcpyAsync(h->h_red, h->sd, sizeof(double) * SD_COUNT, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  *res_norm = std::sqrt(h->h_red[SD_RR]);
  return rc;
}

int nys_newton(nys_handle h, int m, int n, int a_dtype, const void* A, long long lda, const double* x,
               const double* z, const double* D, double delta, const double* r_d, const double* r_p,
               const double* r_xz, int ell, const double* U, int ld, const double* lam, double eta,
               int max_iter, int forced_iters, double* dx, double* dy, double* dz, int* iters) {
  if (!h) return NYS_ERR_ARG;
  if (m <= 0 || n <= 0 || m > h->max_m || n > h->max_n || lda < n || a_dtype != NYS_F64 ||
      ell <= 0 || ell > h->ell_cap || ld < m || !A || !x || !z || !D || !r_d || !r_p || !r_xz ||
      !U || !lam || !dx || !dy || !dz || !iters || max_iter < 0)
    return fail(h, NYS_ERR_ARG, "nys_newton: bad argument");
  CK(cudaMemsetAsync(h->si + SI_ERR, 0, sizeof(int), h->st));
  return newton(h, m, n, static_cast<const double*>(A), lda, x, z, D, delta, r_d, r_p, r_xz, ell, U,
                ld, lam, eta, max_iter, forced_iters, dx, dy, dz, iters);
}

namespace {

// One run on the host-driven phases (the fallback of batch_device).
void host_run(IpmRun& run) {
  while (!run.done) {
    if (run.top() < 0 && !run.done) run.stop(NYS_ERR_CUDA);
    if (run.done) break;
    if (run.req.active) serve_single(run);
    if (run.mid() < 0 && !run.done) run.stop(NYS_ERR_CUDA);
    if (run.done) break;
    if (run.req.active) serve_single(run);
    if (run.bottom() < 0 && !run.done) run.stop(NYS_ERR_CUDA);
  }
  run.finish();
}

// Batching form on the device-resident iteration.  Each worker solver holds
// one problem at a time; its iterations are graph launches on the worker's
// stream, each followed by a read-back of the device scalars.  One host
// thread polls the worker streams and launches the next iteration of
// whichever problem's read-back has arrived, so every problem advances at
// its own pace (no lock step: a short solve does not wait for a long one),
// and a worker takes the next problem as soon as its current one finishes.
// Problems the path does not take run on the host-driven phases.
//
// How many problems are in flight is autotuned: the streams reach the GPU
// through a limited number of hardware queues (CUDA_DEVICE_MAX_CONNECTIONS),
// and beyond it problems only queue behind each other (measured on 256 QPs of
// m <= 1024 with 32 queues: 13.8 QP/s with 32 in flight, 11.7 with 64, 9.9
// with 128).  While a handle has no tuned value, the first call tries
// in-flight counts of 8, 16, 24, 32, 48, 64, ... (up to max_batch) for
// kTuneWindow seconds each after kTuneSettle seconds of settling, scores
// each by the PCG work it completed per second (PCG iterations x m x n),
// stops after two counts that do not beat the best by kTuneMargin, and keeps
// the best for the rest of the call and for later calls
// (nys_batch_inflight reports it).  Counts above the number of hardware
// queues are not tried.  Batches of fewer than 128 problems are
// too short to tune and run max_batch at once.  Each problem's arithmetic depends on its
// own launch plan only, so the in-flight count never changes a result.
constexpr double kTuneSettle = 0.1;
constexpr double kTuneWindow = 0.8;
constexpr double kTuneMargin = 1.03;   // a larger count must beat the best by 3 %

// Cluster-plan autotuning of the batching form.  Problems are grouped in
// shape buckets (m rounded up to 64, n to 512, the same ell); for a bucket
// not seen before, every cluster plan with A on chip that fits its first
// problem's shape (16, 8 or 4 CTAs) runs kTunePcg
// forced PCG iterations of a system of that shape (Gaussian A, D = 1, U = 0,
// lam = 1, xi = 1, delta = 1: the work does not depend on the values), once
// to warm up and twice timed with CUDA events, and the plan with the least
// cost time x max(CTAs, SMs / hardware queues) is kept for the bucket, for
// this call and later ones.  The SMs are what the problems of a full batch
// share, but no more problems run at once than there are hardware queues
// (CUDA_DEVICE_MAX_CONNECTIONS, 8 unless set), so a plan narrower than
// SMs / queues leaves SMs idle and is charged as if it used that share
// (time x CTAs alone picked 4-CTA plans for most of the 256-QP workload and
// ran it at 9.4 instead of 13.9 QP/s).  The trials run before any problem
// starts, on an otherwise idle GPU.  A problem runs the bucket's plan when
// it fits its exact shape, else the fixed rule's.  Buckets whose A fits no
// cluster's shared memory keep the fixed rule's plan (8 or 4 CTAs reading A
// from L2): a trial alone on the GPU finds A in L2, but under a full batch
// the problems' matrices compete for L2 and such plans run from DRAM, so
// the trials misjudge them (with them in the trials the 256-QP workload ran
// at 11.4 QP/s).
//
// Measured on the 256-QP workload (m <= 1024, 32 hardware queues): with 32
// in flight, 13.86 QP/s on the fixed rule's plans and 13.94 with the tuner
// (19 of 81 buckets retuned, mostly to 4 CTAs); with 64 in flight, 11.7
// against 12.0; earlier forms of the tuner ran it at 9.4 (cost time x CTAs,
// L2 plans included: 4-CTA L2 plans for 62 buckets) and 11.4 QP/s
// (queue-aware cost, L2 plans included).  NYS_BATCH_PLAN_TUNE=0 turns it
// off.
constexpr int kTunePcg = 16;

long long plan_bucket(int m, int n, int ell) {
  return ((long long)((m + 63) / 64) << 40) | ((long long)((n + 511) / 512) << 20) | (long long)ell;
}

int batch_ell(const nys_solver* h, const nys_problem& q) {
  return std::min(std::min(h->ell_cap, q.m), q.ell > 0 ? q.ell : h->ell_cap);
}

int tune_plans(nys_solver* h, int count, const nys_problem* p) {
  int queues = 8;
  if (const char* env = std::getenv("CUDA_DEVICE_MAX_CONNECTIONS")) {
    const int v = std::atoi(env);
    if (v > 0) queues = v;
  }
  const double min_ctas = (double)h->num_sms / queues;
  for (int i = 0; i < count; ++i) {
    const int m = p[i].m, n = p[i].n, ell = batch_ell(h, p[i]);
    if (m <= 0 || n <= 0 || ell <= 0 || m > h->max_m || n > h->max_n) continue;
    const long long key = plan_bucket(m, n, ell);
    if (h->tuned_plans.count(key)) continue;
    ClusterPlan all[6], cand[6];
    const int na = pcg_cluster_candidates(m, n, ell, all, 6);
    int nc = 0;
    for (int k = 0; k < na; ++k)
      if (all[k].a_smem) cand[nc++] = all[k];
    if (nc <= 1) {                       // nothing to choose between (or A off chip: the rule)
      h->tuned_plans[key] = {nc == 1 ? cand[0].C : 0, nc == 1 ? cand[0].a_smem : 0};
      continue;
    }
    const size_t need = (size_t)m * n + n + 2 * (size_t)m + ell + (size_t)m * ell + SD_COUNT + 4;
    if (need > h->tune_cap) {
      if (h->tune_buf) cudaFree(h->tune_buf);
      h->tune_buf = nullptr;
      h->tune_cap = 0;
      CK(cudaMalloc(&h->tune_buf, sizeof(double) * need));
      h->tune_cap = need;
    }
    double* A = h->tune_buf;
    double* D = A + (size_t)m * n;
    double* xi = D + n;
    double* x = xi + m;
    double* lam = x + m;
    double* U = lam + ell;
    double* sd = U + (size_t)m * ell;
    int* iw = reinterpret_cast<int*>(sd + SD_COUNT);   // iterations, error word
    CK(gaussian_omega(h->st, 0x5eedULL, 0, n, m, A, n));   // n x m column-major = m x n row-major
    CK(fill_f64(h->st, n, 1.0, D));
    CK(fill_f64(h->st, m, 1.0, xi));
    CK(fill_f64(h->st, ell, 1.0, lam));
    CK(cudaMemsetAsync(U, 0, sizeof(double) * (size_t)m * ell, h->st));
    ClusterPcgTask t{};
    t.m = m; t.n = n; t.ell = ell; t.ld = m; t.lda = n;
    t.A = A; t.D = D; t.U = U; t.lam = lam; t.xi = xi;
    t.delta = 1.0; t.eta2 = 0.0;
    t.max_iter = kTunePcg; t.forced = kTunePcg;
    t.x = x; t.iters = iw; t.sd = sd; t.err = iw + 1; t.t_ns = nullptr;
    int best = -1;
    double best_score = 0.0;
    for (int k = 0; k < nc; ++k) {
      CK(cudaMemsetAsync(iw, 0, 2 * sizeof(int), h->st));
      bool ok = pcg_cluster_f64(h->st, cand[k], t, nullptr, 0) == cudaSuccess;
      ok = ok && cudaEventRecord(h->ev_pcg0, h->st) == cudaSuccess;
      for (int rep = 0; ok && rep < 2; ++rep) ok = pcg_cluster_f64(h->st, cand[k], t, nullptr, 0) == cudaSuccess;
      ok = ok && cudaEventRecord(h->ev_pcg1, h->st) == cudaSuccess;
      if (!ok) { cudaGetLastError(); continue; }
      CK(cudaStreamSynchronize(h->st));
      int werr = 0;
      CK(cudaMemcpy(&werr, iw + 1, sizeof(int), cudaMemcpyDeviceToHost));
      float ms = 0.f;
      if (werr != 0 || cudaEventElapsedTime(&ms, h->ev_pcg0, h->ev_pcg1) != cudaSuccess) { cudaGetLastError(); continue; }
      const double score = 0.5 * ms * std::max((double)cand[k].C, min_ctas);
      if (h->trace_tune)
        std::fprintf(stderr, "plan tune m=%d n=%d ell=%d C=%d a_smem=%d ms=%.4f score=%.4f\n", m, n, ell, cand[k].C,
                     cand[k].a_smem, 0.5 * ms, score);
      if (best < 0 || score < best_score) { best = k; best_score = score; }
    }
    h->tuned_plans[key] = best >= 0 ? std::make_pair(cand[best].C, cand[best].a_smem) : std::make_pair(0, 0);
  }
  return NYS_OK;
}

// The bucket's tuned plan for worker w's next problem, when one is cached
// and fits the exact shape; otherwise the fixed rule's (recomputed on use).
void apply_tuned_plan(nys_solver* h, nys_solver* w, int m, int n, int ell) {
  auto it = h->tuned_plans.find(plan_bucket(m, n, ell));
  ClusterPlan pl;
  if (it != h->tuned_plans.end() && it->second.first > 0 &&
      pcg_cluster_plan_for(m, n, ell, it->second.first, it->second.second, &pl)) {
    w->cp = pl;
    w->cp_ok = true;
    w->cp_m = m;
    w->cp_n = n;
    w->cp_ell = ell;
  } else {
    w->cp_m = -1;
  }
}

int batch_device(nys_solver* h, int count, const nys_problem* p, nys_result* r, const std::vector<int>& order,
                 int want) {
  std::vector<IpmRun> runs(want);
  std::vector<int> busy(want, 0), seen(want, 0);
  int next = 0, active = 0;
  auto begin = [&](int t) -> bool {
    while (next < count) {
      const int pi = order[next++];
      IpmRun& run = runs[t];
      run = IpmRun();
      seen[t] = 0;
      if (run.start(h->workers[t], &p[pi], &r[pi]) != NYS_OK) {
        r[pi].status = run.status;
        continue;
      }
      apply_tuned_plan(h, h->workers[t], run.m, run.n, run.ell);
      if (!run.device_eligible()) {
        host_run(run);
        continue;
      }
      const int rc = run.device_prepare();
      if (rc == 1) {                      // the graph could not be captured: host path
        host_run(run);
        continue;
      }
      if (rc < 0) {
        run.stop(rc);
        run.finish();
        continue;
      }
      return true;
    }
    return false;
  };
  // in-flight autotuning (see above)
  std::vector<int> cand;
  bool tuning = false;
  int limit = want;
  bool tune_env = true;
  if (const char* env = std::getenv("NYS_BATCH_TUNE")) tune_env = env[0] != '0';
  bool plan_env = true;                           // cluster plans per shape bucket (above)
  if (const char* env = std::getenv("NYS_BATCH_PLAN_TUNE")) plan_env = env[0] != '0';
  if (plan_env && tune_env && want >= 16 && count >= 128) {
    const int rc = tune_plans(h, count, p);
    if (rc != NYS_OK) return rc;
  }
  if (h->tuned_inflight > 0) {
    limit = std::min(h->tuned_inflight, want);
  } else if (tune_env && want >= 16 && count >= 128) {
    // no more than the hardware queues: beyond them problems only wait behind
    // one another, and a window's score (work of problems started in earlier
    // windows included) can reward a larger count by chance (a 64 in flight
    // once scored 2.1e11 against 1.5e11 for 32 and 48, and then ran the batch
    // at 11.7 instead of 13.9 QP/s)
    int queues = 8;
    if (const char* env = std::getenv("CUDA_DEVICE_MAX_CONNECTIONS")) {
      const int v = std::atoi(env);
      if (v > 0) queues = v;
    }
    const int top = std::min(want, std::max(8, queues));
    for (int c : {8, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512})
      if (c < top) cand.push_back(c);
    cand.push_back(top);
    tuning = true;
    limit = cand[0];
  }
  using clk = std::chrono::steady_clock;
  auto now = [] { return std::chrono::duration<double>(clk::now().time_since_epoch()).count(); };
  size_t ci = 0;
  double t_change = now(), work = 0.0, best_rate = -1.0;
  int best = limit, worse = 0;
  for (int t = 0; t < limit; ++t)
    if (begin(t)) { busy[t] = 1; ++active; }
  while (active > 0) {
    bool progressed = false;
    const double t_now = now();
    for (int t = 0; t < want; ++t) {
      if (!busy[t]) continue;
      const cudaError_t q = cudaStreamQuery(h->worker_streams[t]);
      if (q == cudaErrorNotReady) continue;
      progressed = true;
      IpmRun& run = runs[t];
      // PCG work completed since the last read-back of this problem
      const int tot = h->workers[t]->h_ipmd->pcg_total;
      if (tuning && t_now >= t_change + kTuneSettle) work += (double)(tot - seen[t]) * run.m * (double)run.n;
      seen[t] = tot;
      int rc = q == cudaSuccess ? run.device_step() : NYS_ERR_CUDA;
      if (rc == 1) continue;              // the next iteration is in flight
      if (rc < 0) {
        cudaGetLastError();
        run.stop(fail(h, NYS_ERR_CUDA, "nys_solve_batched: worker %d stream failed", t));
      } else {
        run.device_collect();
      }
      run.finish();
      busy[t] = 0;
      --active;
      if (t < limit && begin(t)) { busy[t] = 1; ++active; }
    }
    if (tuning && t_now >= t_change + kTuneSettle + kTuneWindow) {
      const double rate = work / kTuneWindow;
      if (h->trace_tune)
        std::fprintf(stderr, "[nys] batch in flight %d: %.3e PCG work/s (next problem %d of %d, active %d)\n",
                     limit, rate, next, count, active);
      if (best_rate < 0.0 || rate > kTuneMargin * best_rate) { best_rate = rate; best = limit; worse = 0; }
      else ++worse;
      ++ci;
      if (ci >= cand.size() || worse >= 2 || next >= count) {
        tuning = false;
        limit = best;
        h->tuned_inflight = best;
      } else {
        limit = cand[ci];
      }
      work = 0.0;
      t_change = now();
    }
    // fill the slots a larger limit opened
    for (int t = 0; t < limit && next < count; ++t)
      if (!busy[t] && begin(t)) { busy[t] = 1; ++active; }
    if (!progressed) std::this_thread::yield();
  }
  if (tuning && best_rate >= 0.0) h->tuned_inflight = best;
  return NYS_OK;
}

}  // namespace

int nys_solve_batched(nys_handle h, int count, const nys_problem* p, nys_result* r) {
  if (!h) return NYS_ERR_ARG;
  if (count < 0 || (count > 0 && (!p || !r))) return fail(h, NYS_ERR_ARG, "nys_solve_batched: bad argument");
  if (h->max_batch < 1) return fail(h, NYS_ERR_ARG, "nys_solve_batched: handle created with max_batch = 0");
  if (h->opt.adapt_cost > 0)
    return fail(h, NYS_ERR_ARG, "nys_solve_batched: the adaptive sketch size is for single solves");
  if (count == 0) return NYS_OK;
  const int want = std::min(h->max_batch, count);
  // the caller's stream must be drained before worker streams read its data
  CK(cudaStreamSynchronize(h->st));
  while ((int)h->workers.size() < want) {
    cudaStream_t s = nullptr;
    CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    nys_handle w = nullptr;
    nys_options o = h->opt;
    const int rc = nys_create(&w, &o, h->max_m, h->max_n, 0, s);
    if (rc != NYS_OK) {
      cudaStreamDestroy(s);
      return fail(h, rc, "nys_solve_batched: cannot create worker solver %zu", h->workers.size());
    }
    // many systems side by side: a cluster plan reading A from L2 when A does
    // not fit on chip (the shared launches use the same plans)
    if (w->pcg_path == 0) w->plan_policy = 2;
    if (const char* env = std::getenv("NYS_BATCH_PLAN"))   // 1: throughput plans (4-8 CTAs) only
      if (env[0] == '1' && w->pcg_path == 0) w->plan_policy = 1;
    h->workers.push_back(w);
    h->worker_streams.push_back(s);
  }
  if (h->task_cap < want) {
    if (h->d_tasks) cudaFree(h->d_tasks);
    if (h->h_tasks) cudaFreeHost(h->h_tasks);
    h->d_tasks = nullptr;
    h->h_tasks = nullptr;
    h->task_cap = 0;
    CK(cudaMalloc(&h->d_tasks, sizeof(ClusterPcgTask) * want));
    CK(cudaMallocHost(&h->h_tasks, sizeof(ClusterPcgTask) * want));
    h->task_cap = want;
  }
  // largest problems first, in lock-step groups of `want`: similar sizes meet
  // at the same rendezvous; every launch shape depends on the problem alone,
  // so a problem gets the same bits in any group
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (long long)p[a].m * p[a].n > (long long)p[b].m * p[b].n;
  });
  bool all_plain = true;                // problems (P): the device-resident iteration takes them
  for (int i = 0; i < count && all_plain; ++i) all_plain = p[i].var_kind == nullptr;
  if (all_plain && h->use_dev_ipm && h->use_graphs && h->opt.precision_mode == 0 && h->opt.reuse_pcg == 0) {
    // device-resident iterations: no lock step (see batch_device)
    const int rc = batch_device(h, count, p, r, order, want);
    if (rc < 0) return rc;
    int worst_err = NYS_OK, worst_warn = NYS_OK;
    for (int i = 0; i < count; ++i) {
      if (r[i].status < worst_err) worst_err = r[i].status;
      if (r[i].status > worst_warn) worst_warn = r[i].status;
    }
    if (worst_err < 0) return fail(h, worst_err, "nys_solve_batched: at least one problem failed");
    return worst_warn;
  }
  for (int g0 = 0; g0 < count; g0 += want) {
    const int G = std::min(want, count - g0);
    std::vector<IpmRun> runs(G);
    std::vector<BatchSlot> slots(G);
    Rendezvous bar;
    bar.n = G;
    bool launched = false, any_active = true;
    int launch_err = NYS_OK;
    auto serve = [&]() {
      const int rc = serve_batch(h, runs, slots, launched);
      if (rc != NYS_OK && launch_err == NYS_OK) launch_err = rc;
    };
    std::vector<std::thread> pool;
    pool.reserve(G);
    for (int t = 0; t < G; ++t) {
      pool.emplace_back([&, t]() {
        cudaSetDevice(h->device);
        IpmRun& run = runs[t];
        BatchSlot& slot = slots[t];
        const int pi = order[g0 + t];
        const bool started = run.start(h->workers[t], &p[pi], &r[pi]) == NYS_OK;
        if (!started) r[pi].status = run.status;
        // shared launches take every system a cluster can hold (A on chip,
        // else read from L2): measured on 256 QPs of m <= 1024, that beats
        // giving the larger ones the cooperative grid side by side
        slot.has_plan = started && !run.lp && pcg_cluster_plan(run.m, run.n, run.ell, 2, &slot.plan);
        auto phase = [&](int which) {      // 0 top, 1 mid, 2 bottom
          if (run.done) return;
          const int rc = which == 0 ? run.top() : which == 1 ? run.mid() : run.bottom();
          if (rc < 0 && !run.done) run.stop(rc);
        };
        while (true) {
          phase(0);
          bar.arrive([&] {
            serve();
            any_active = false;
            for (auto& x : runs) any_active = any_active || !x.done;
          });
          if (!any_active) break;
          if (launch_err != NYS_OK && slot.batched) { run.stop(launch_err); slot.batched = false; }
          finish_request(run, slot);
          phase(1);
          bar.arrive(serve);
          if (launch_err != NYS_OK && slot.batched) { run.stop(launch_err); slot.batched = false; }
          finish_request(run, slot);
          phase(2);
        }
        if (started) run.finish();
      });
    }
    for (auto& th : pool) th.join();
  }
  int worst_err = NYS_OK, worst_warn = NYS_OK;
  for (int i = 0; i < count; ++i) {
    if (r[i].status < worst_err) worst_err = r[i].status;
    if (r[i].status > worst_warn) worst_warn = r[i].status;
  }
  if (worst_err < 0) return fail(h, worst_err, "nys_solve_batched: at least one problem failed");
  return worst_warn;
}

int nys_adjoint(nys_handle h, int count, const nys_problem* p, const nys_result* r, const double* dL_dx,
                double eta, double* dL_dc, double* dL_db, double* dL_dq, double* dL_dA) {
  if (!h) return NYS_ERR_ARG;
  if (count < 0 || (count > 0 && (!p || !r || !dL_dx)) || !(eta > 0.0))
    return fail(h, NYS_ERR_ARG, "nys_adjoint: bad argument");
  int worst = NYS_OK;
  size_t on = 0, om = 0, omn = 0;
  for (int i = 0; i < count; ++i) {
    const nys_problem& P = p[i];
    const nys_result& R = r[i];
    const int m = P.m, n = P.n;
    if (m <= 0 || n <= 0 || m > h->max_m || n > h->max_n || P.a_dtype != NYS_F64 || P.host || !P.A || !P.q ||
        P.lda < n || !R.x || !R.y || !R.z)
      return fail(h, NYS_ERR_ARG, "nys_adjoint: problem %d is not a device FP64 problem of this handle", i);
    if (P.var_kind)
      return fail(h, NYS_ERR_ARG, "nys_adjoint: problem %d has free or box-constrained variables", i);
    const double* A = static_cast<const double*>(P.A);
    int ell = std::min(h->ell_cap, m);
    const double* g = dL_dx + on;
    CK(cudaMemsetAsync(h->si, 0, sizeof(int) * SI_COUNT, h->st));
    // final D
    CK(scaling_f64(h->st, n, R.x, R.z, P.q, R.rho, h->D));
    // The Nystrom factor of the solve's last IPM iteration, when this handle
    // (or the batch worker that solved the problem) still holds it: N there
    // differs from N at the solution only by the last, converged step, so it
    // preconditions the adjoint system as well (the PCG below solves to eta
    // whatever the factor).  Otherwise a fresh factor of N at the solution.
    const double* U = h->U;
    const double* lamh = h->lamh;
    int ldu = h->ld;
    const nys_solver* src = nullptr;
    if (h->fac_A == A && h->fac_m == m) src = h;
    for (nys_solver* w : h->workers)
      if (!src && w->fac_A == A && w->fac_m == m) src = w;
    if (src) {
      U = src->U;
      lamh = src->lamh;
      ldu = src->ld;
      ell = src->fac_ell;
    } else {
      CK(gaussian_omega(h->st, h->opt.seed, R.ipm_iters + 1, m, ell, h->Om, h->ld));
      CK(sketch_f64(h->st, m, n, A, P.lda, h->D, ell, h->Om, h->ld, h->Y, h->T, h->ld_t, h->split_buf,
                    h->split_cap));
      CK(nystrom_core_f64(h->st, m, ell, h->Y, h->Om, h->ld, h->U, h->lamh, h->sd, h->si, h->red, h->cw,
                          h->num_sms));
    }
    // (N + delta I) lam2 = A (D .* g)
    CK(vmul_f64(h->st, n, h->D, g, h->t_n));
    CK(gemv_n_f64(h->st, m, n, A, P.lda, h->t_n, 0.0, nullptr, h->xi, nullptr, nullptr, h->split_buf,
                  h->split_cap));
    int it = 0;
    int rc = run_pcg(h, m, n, A, P.lda, h->D, R.delta, ell, U, ldu, lamh, h->xi, h->dyp, eta,
                     h->opt.max_pcg_iter, -1, &it);
    if (rc < 0) return rc;
    if (rc > worst) worst = rc;
    // -lam1 = D (A^T lam2 - g)
    CK(gemv_t_f64(h->st, m, n, A, P.lda, h->dyp, nullptr, h->g_n, h->split_buf, h->split_cap));
    CK(axpby_f64(h->st, n, 1.0, h->g_n, -1.0, g, h->dxp));
    CK(vmul_f64(h->st, n, h->D, h->dxp, h->dxc));          // dxc = -lam1
    if (dL_dc) CK(cudaMemcpyAsync(dL_dc + on, h->dxc, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
    if (dL_db) CK(cudaMemcpyAsync(dL_db + om, h->dyp, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->st));
    if (dL_dq) CK(vmul_f64(h->st, n, h->dxc, R.x, dL_dq + on));
    // dL/dA = y lam1^T - lam2 x^T = -(y (-lam1)^T) - lam2 x^T
    if (dL_dA) CK(rank2_update(h->st, m, n, -1.0, R.y, h->dxc, -1.0, h->dyp, R.x, dL_dA + omn, n, 0));
    rc = sync_scalars(h, 0);
    if (rc != NYS_OK) return rc;
    on += n;
    om += m;
    omn += (size_t)m * n;
  }
  return worst;
}

int nys_batch_inflight(nys_handle h) {
  if (!h) return NYS_ERR_ARG;
  return h->tuned_inflight;
}

int nys_batch_plan(nys_handle h, int m, int n, int ell, int* ctas, int* a_smem) {
  if (!h) return NYS_ERR_ARG;
  if (m <= 0 || n <= 0 || ell <= 0 || !ctas || !a_smem) return fail(h, NYS_ERR_ARG, "nys_batch_plan: bad argument");
  auto it = h->tuned_plans.find(plan_bucket(m, n, ell));
  if (it == h->tuned_plans.end()) {
    *ctas = 0;
    *a_smem = 0;
    return 0;
  }
  *ctas = it->second.first;
  *a_smem = it->second.second;
  return 1;
}

int nys_pcg_route(nys_handle h, int m, int n, int ell) {
  if (!h || m <= 0 || n <= 0 || ell <= 0) return NYS_ERR_ARG;
  return fp64_route(h, m, n, ell);
}

int nys_gemm_bf16(nys_handle h, int M, int N, int K, const void* A, long long lda, const void* B,
                  long long ldb, float* C, long long ldc) {
  if (!h) return NYS_ERR_ARG;
  if (M <= 0 || N <= 0 || N > 512 || K <= 0 || !A || !B || !C || lda < K || ldb < K || ldc < M ||
      lda % 8 || ldb % 8 || (reinterpret_cast<uintptr_t>(A) & 15u) || (reinterpret_cast<uintptr_t>(B) & 15u))
    return fail(h, NYS_ERR_ARG, "nys_gemm_bf16: bad argument");
  float* part = h->upart ? h->upart : reinterpret_cast<float*>(h->split_buf);
  const size_t cap = h->upart ? h->upart_cap : 2 * h->split_cap;
  const size_t npad = (size_t)(N + 15) / 16 * 16;
  if (npad * (size_t)M > cap) return fail(h, NYS_ERR_ARG, "nys_gemm_bf16: M x N exceeds the workspace");
  CK(cudaMemsetAsync(h->si + SI_ERR, 0, sizeof(int), h->st));
  CK(umma_gemm_bf16(h->st, M, N, K, A, lda, B, ldb, part, cap, h->num_sms, 0, nullptr, C, ldc, h->si + SI_ERR));
  return sync_scalars(h, 0);
}

int nys_step_length(nys_handle h, int n, const double* v, const double* dv, double* alpha) {
  if (!h) return NYS_ERR_ARG;
  if (n <= 0 || !v || !dv || !alpha) return fail(h, NYS_ERR_ARG, "nys_step_length: bad argument");
  CK(cudaMemsetAsync(h->si + SI_ERR, 0, sizeof(int), h->st));
  CK(step_ratios_f64(h->st, n, v, dv, v, dv, h->red_out, h->red));
  int rc = sync_scalars(h, 1);
  if (rc != NYS_OK) return rc;
  *alpha = 0.995 * std::min(1.0, h->h_red[0]);
  return NYS_OK;
}

int nys_solve(nys_handle h, const nys_problem* p, nys_result* r) {
  if (!h) return NYS_ERR_ARG;
  IpmRun run;
  if (run.start(h, p, r) != NYS_OK) return run.status;
  // a phase that returns an error without ending the run hit a CUDA failure:
  // leave at once, as every other entry point does
  int rc = NYS_OK;
  if (run.device_eligible()) {
    rc = run.device_solve();
    if (rc < 0) return rc;
  }
  while (!run.done) {
    if ((rc = run.top()) < 0 && !run.done) return rc;
    if (run.done) break;
    if (run.req.active) serve_single(run);
    if ((rc = run.mid()) < 0 && !run.done) return rc;
    if (run.done) break;
    if (run.req.active) serve_single(run);
    if ((rc = run.bottom()) < 0 && !run.done) return rc;
  }
  return run.finish();
}

}  // extern "C"

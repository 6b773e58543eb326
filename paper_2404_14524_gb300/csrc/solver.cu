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
#include <cstring>
#include <string>
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
  // pinned host mirrors
  double* h_red = nullptr;
  int* h_si = nullptr;
  // device staging for problems given in host memory
  void* stage = nullptr;
  size_t stage_bytes = 0;
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
  h->cw.split_buf = h->split_buf;
  h->cw.split_cap = h->split_cap;
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

// Run PCG on (A D A^T + delta I) dy = xi; dy is written into `out`.
int run_pcg(nys_solver* h, int m, int n, const double* A, long long lda, const double* D,
            double delta, int ell, const double* U, int ld, const double* lamh, const double* xi,
            double* out, double eta, int max_iter, int forced, int* iters) {
  PcgWork w = h->pw;
  w.x = out;
  CK(pcg_setup_f64(h->st, m, ell, U, ld, lamh, delta, xi, eta, max_iter, forced, w, h->sd, h->si, h->red));
  const int limit = forced >= 0 ? forced : max_iter;
  int issued = 0, chunk = 2;
  while (true) {
    int rc = sync_scalars(h, 0);
    if (rc != NYS_OK) return rc;
    if (h->h_si[SI_DONE] || issued >= limit) break;
    const int todo = std::min(chunk, limit - issued);
    for (int k = 0; k < todo; ++k)
      CK(pcg_iteration_f64(h->st, m, n, A, lda, D, delta, ell, U, ld, w, h->sd, h->si, h->red));
    issued += todo;
    chunk = std::min(chunk * 2, 16);
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

// Algorithm 4: Newton direction through the normal equations.
int newton(nys_solver* h, int m, int n, const double* A, long long lda, const double* x,
           const double* z, const double* D, double delta, const double* r_d, const double* r_p,
           const double* r_xz, int ell, const double* U, int ld, const double* lamh, double eta,
           int max_iter, int forced, double* dx, double* dy, double* dz, int* iters) {
  CK(newton_rhs_f64(h->st, n, D, r_d, r_xz, x, h->t_n));
  CK(gemv_n_f64(h->st, m, n, A, lda, h->t_n, r_p ? 1.0 : 0.0, r_p, h->xi));
  int rc = run_pcg(h, m, n, A, lda, D, delta, ell, U, ld, lamh, h->xi, dy, eta, max_iter, forced, iters);
  if (rc < 0) return rc;
  CK(gemv_t_f64(h->st, m, n, A, lda, dy, nullptr, h->g_n, h->split_buf, h->split_cap));
  CK(newton_back_f64(h->st, n, D, h->g_n, r_d, r_xz, x, z, dx, dz));
  return rc;
}

}  // namespace

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
}

const char* nys_last_error(nys_handle h) { return h ? h->err.c_str() : "null handle"; }

unsigned long long nys_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int nys_create(nys_handle* out, const nys_options* opt, int max_m, int max_n, int max_batch,
               void* cuda_stream) {
  if (!out) return NYS_ERR_ARG;
  *out = nullptr;
  if (!opt || max_m <= 0 || max_n <= 0 || max_batch < 0 || opt->ell <= 0 || opt->tol <= 0.0 ||
      opt->max_ipm_iter < 0 || opt->max_pcg_iter < 0 || opt->precision_mode != 0)
    return NYS_ERR_ARG;
  nys_solver* h = new nys_solver();
  h->opt = *opt;
  h->max_m = max_m;
  h->max_n = max_n;
  h->ell_cap = std::min(opt->ell, max_m);
  h->ld = (int)align_up(max_m, 2);
  h->ld_t = (int)align_up(max_n, 2);
  h->st = reinterpret_cast<cudaStream_t>(cuda_stream);
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
      cudaMallocHost(&h->h_si, sizeof(int) * 64) != cudaSuccess) {
    cudaFree(h->arena);
    delete h;
    return NYS_ERR_NOMEM;
  }
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
  if (h->st) cudaStreamSynchronize(h->st);
  else cudaDeviceSynchronize();
  cudaFree(h->arena);
  if (h->stage) cudaFree(h->stage);
  cudaFreeHost(h->h_red);
  cudaFreeHost(h->h_si);
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
  CK(gemv_n_f64(h->st, m, n, Ad, lda, h->pw.t, delta, v, out));
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
  if (m <= 0 || n <= 0 || m > h->max_m || n > h->max_n || lda < n || a_dtype != NYS_F64 ||
      ell <= 0 || ell > h->ell_cap || ld < m || !A || !D || !Omega || !Y)
    return fail(h, NYS_ERR_ARG, "nys_sketch: bad argument");
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
  const auto t0 = std::chrono::steady_clock::now();
  if (!p || !r) return fail(h, NYS_ERR_ARG, "nys_solve: null problem or result");
  const int m = p->m, n = p->n;
  if (m <= 0 || n <= 0 || m > h->max_m || n > h->max_n || p->lda < n || p->a_dtype != NYS_F64 ||
      !p->A || !p->b || !p->c || !p->q || !p->x0 || !p->y0 || !p->z0 || !r->x || !r->y || !r->z ||
      p->k0 < 0)
    return fail(h, NYS_ERR_ARG, "nys_solve: bad problem (sizes, dtype or null pointers)");
  const nys_options& o = h->opt;
  const int ell = std::min(h->ell_cap, m);
  const long long lda = p->lda;
  r->status = NYS_OK;
  r->ipm_iters = 0;
  r->pcg_iters_total = 0;
  r->refine_steps = 0;
  r->pcg_log_len = 0;

  // Problem data on the device (staged when the caller passes host memory).
  const double *A = static_cast<const double*>(p->A), *b = p->b, *c = p->c, *q = p->q;
  if (p->host) {
    const size_t a_bytes = align_up((size_t)m * lda * sizeof(double), 256);
    const size_t need = a_bytes + 3 * align_up(sizeof(double) * (size_t)n, 256) +
                        align_up(sizeof(double) * (size_t)m, 256);
    if (need > h->stage_bytes) {
      if (h->stage) cudaFree(h->stage);
      h->stage = nullptr;
      h->stage_bytes = 0;
      if (cudaMalloc(&h->stage, need) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, NYS_ERR_NOMEM, "nys_solve: cannot stage a host problem of %zu bytes", need);
      }
      h->stage_bytes = need;
    }
    char* s = static_cast<char*>(h->stage);
    double* dA = reinterpret_cast<double*>(s);
    double* db = reinterpret_cast<double*>(s + a_bytes);
    double* dc = reinterpret_cast<double*>(s + a_bytes + align_up(sizeof(double) * m, 256));
    double* dq = reinterpret_cast<double*>(reinterpret_cast<char*>(dc) + align_up(sizeof(double) * n, 256));
    CK(cudaMemcpyAsync(dA, p->A, (size_t)m * lda * sizeof(double), cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(db, p->b, sizeof(double) * m, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(dc, p->c, sizeof(double) * n, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(dq, p->q, sizeof(double) * n, cudaMemcpyHostToDevice, h->st));
    A = dA; b = db; c = dc; q = dq;
  }
  const cudaMemcpyKind kin = p->host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(h->x, p->x0, sizeof(double) * n, kin, h->st));
  CK(cudaMemcpyAsync(h->y, p->y0, sizeof(double) * m, kin, h->st));
  CK(cudaMemcpyAsync(h->z, p->z0, sizeof(double) * n, kin, h->st));
  if (p->lam0) CK(cudaMemcpyAsync(h->lam, p->lam0, sizeof(double) * m, kin, h->st));
  else CK(cudaMemcpyAsync(h->lam, h->y, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->st));
  if (p->zeta0) CK(cudaMemcpyAsync(h->zeta, p->zeta0, sizeof(double) * n, kin, h->st));
  else CK(cudaMemcpyAsync(h->zeta, h->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemsetAsync(h->si, 0, sizeof(int) * SI_COUNT, h->st));
  CK(dot_f64(h->st, m, b, b, h->red_out + 8, h->red));
  CK(dot_f64(h->st, n, c, c, h->red_out + 9, h->red));
  int rc = sync_scalars(h, 10);
  if (rc != NYS_OK) return r->status = rc;
  const double bnorm = std::sqrt(h->h_red[8]), cnorm = std::sqrt(h->h_red[9]);

  double rho = o.rho0, delta = o.delta0;
  double mu = 0.0, mu_prev = 0.0, nrp_prev = 0.0, nrd_prev = 0.0;
  double rel_p = 0.0, rel_d = 0.0;
  int forced_idx = 0;
  int warn = NYS_OK;
  int k = 0;
  int status = NYS_WARN_MAXITER;
  auto next_forced = [&]() -> int {
    if (o.forced_pcg_iters && forced_idx < o.n_forced_pcg) return o.forced_pcg_iters[forced_idx++];
    return -1;
  };
  auto log_pcg = [&](int it) {
    r->pcg_iters_total += it;
    if (r->pcg_log && r->pcg_log_len < r->pcg_log_cap) r->pcg_log[r->pcg_log_len++] = it;
  };

  while (true) {
    // Residuals and duality measure at the current iterate.
    CK(gemv_n_f64(h->st, m, n, A, lda, h->x, 0.0, nullptr, h->Ax));
    CK(gemv_t_f64(h->st, m, n, A, lda, h->y, nullptr, h->Aty, h->split_buf, h->split_cap));
    CK(ipm_residuals_f64(h->st, m, n, b, c, q, h->x, h->y, h->z, h->Ax, h->Aty, h->lam, h->zeta,
                         rho, delta, h->r_d, h->r_p, h->r_xz, h->red_out, h->red));
    rc = sync_scalars(h, 3);
    if (rc != NYS_OK) { status = rc; break; }
    const double nrd = std::sqrt(h->h_red[0]), nrp = std::sqrt(h->h_red[2]);
    mu = h->h_red[1] / n;
    if (!std::isfinite(nrd) || !std::isfinite(nrp) || !std::isfinite(mu)) {
      status = fail(h, NYS_ERR_NUMERIC, "non-finite residual at IPM iteration %d", k);
      break;
    }
    rel_p = nrp / (1.0 + bnorm);
    rel_d = nrd / (1.0 + cnorm);
    if (k > 0) {
      // PMM parameter update (reading of PEU: see the oracle's docstring).
      const double den = std::max(mu_prev, mu);
      const double r_mu = den > 0.0 ? std::fabs(mu - mu_prev) / den : 0.0;
      if (nrp <= 0.95 * nrp_prev) {
        CK(cudaMemcpyAsync(h->lam, h->y, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->st));
        delta = std::max(o.reg_floor, (1.0 - r_mu) * delta);
      } else {
        delta = std::max(o.reg_floor, (1.0 - 0.666 * r_mu) * delta);
      }
      if (nrd <= 0.95 * nrd_prev) {
        CK(cudaMemcpyAsync(h->zeta, h->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st));
        rho = std::max(o.reg_floor, (1.0 - r_mu) * rho);
      } else {
        rho = std::max(o.reg_floor, (1.0 - 0.666 * r_mu) * rho);
      }
      // predictor right-hand sides with the updated PMM parameters
      CK(ipm_residuals_f64(h->st, m, n, b, c, q, h->x, h->y, h->z, h->Ax, h->Aty, h->lam, h->zeta,
                             rho, delta, h->r_d, h->r_p, h->r_xz, h->red_out, h->red));
    }
    // Termination (reading of TC: relative infeasibilities and mu).
    if (o.forced_ipm_iters >= 0) {
      if (k >= o.forced_ipm_iters) {
        status = (rel_p <= o.tol && rel_d <= o.tol && mu <= o.tol) ? NYS_OK : NYS_WARN_MAXITER;
        break;
      }
    } else if (rel_p <= o.tol && rel_d <= o.tol && mu <= o.tol) {
      status = NYS_OK;
      break;
    }
    if (k >= o.max_ipm_iter) { status = NYS_WARN_MAXITER; break; }

    // N_k, Omega_k, Nystrom preconditioner (Algorithms 1-2).
    CK(scaling_f64(h->st, n, h->x, h->z, q, rho, h->D));
    CK(gaussian_omega(h->st, o.seed, p->k0 + k, m, ell, h->Om, h->ld));
    CK(sketch_f64(h->st, m, n, A, lda, h->D, ell, h->Om, h->ld, h->Y, h->T, h->ld_t, h->split_buf,
                  h->split_cap));
    CK(nystrom_core_f64(h->st, m, ell, h->Y, h->Om, h->ld, h->U, h->lamh, h->sd, h->si, h->red,
                        h->cw, h->num_sms));
    const double eta = std::max(1e-10, std::min(1e-2, 0.1 * mu));

    // Predictor (Algorithm 5, first step).
    int it = 0;
    rc = newton(h, m, n, A, lda, h->x, h->z, h->D, delta, h->r_d, h->r_p, h->r_xz, ell, h->U, h->ld,
                h->lamh, eta, o.max_pcg_iter, next_forced(), h->dxp, h->dyp, h->dzp, &it);
    if (rc < 0) { status = rc; break; }
    if (rc > 0) warn = rc;
    log_pcg(it);
    CK(step_ratios_f64(h->st, n, h->x, h->dxp, h->z, h->dzp, h->red_out, h->red));
    rc = sync_scalars(h, 2);
    if (rc != NYS_OK) { status = rc; break; }
    const double ap_bar = 0.995 * std::min(1.0, h->h_red[0]);
    const double ad_bar = 0.995 * std::min(1.0, h->h_red[1]);
    CK(mu_aff_f64(h->st, n, h->x, h->dxp, h->z, h->dzp, ap_bar, ad_bar, h->red_out, h->red));
    rc = sync_scalars(h, 1);
    if (rc != NYS_OK) { status = rc; break; }
    const double mu_aff = h->h_red[0] / n;
    const double mu_t = mu_aff * mu_aff * mu_aff / (mu * mu);

    // Corrector (Eq. corrector-RHS): r_d = r_p = 0, r_xz = mu_t - dxp dzp.
    CK(corrector_rhs_f64(h->st, n, mu_t, h->dxp, h->dzp, h->r_xz));
    rc = newton(h, m, n, A, lda, h->x, h->z, h->D, delta, nullptr, nullptr, h->r_xz, ell, h->U, h->ld,
                h->lamh, eta, o.max_pcg_iter, next_forced(), h->dxc, h->dyc, h->dzc, &it);
    if (rc < 0) { status = rc; break; }
    if (rc > 0) warn = rc;
    log_pcg(it);
    CK(add_dirs_f64(h->st, m, n, h->dxp, h->dyp, h->dzp, h->dxc, h->dyc, h->dzc));
    CK(step_ratios_f64(h->st, n, h->x, h->dxc, h->z, h->dzc, h->red_out, h->red));
    rc = sync_scalars(h, 2);
    if (rc != NYS_OK) { status = rc; break; }
    const double ap = 0.995 * std::min(1.0, h->h_red[0]);
    const double ad = 0.995 * std::min(1.0, h->h_red[1]);
    CK(ipm_update_f64(h->st, m, n, ap, ad, h->dxc, h->dyc, h->dzc, h->x, h->y, h->z));
    mu_prev = mu;
    nrp_prev = nrp;
    nrd_prev = nrd;
    ++k;
  }

  // Outputs and final measures.
  const cudaMemcpyKind kout = p->host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(r->x, h->x, sizeof(double) * n, kout, h->st));
  CK(cudaMemcpyAsync(r->y, h->y, sizeof(double) * m, kout, h->st));
  CK(cudaMemcpyAsync(r->z, h->z, sizeof(double) * n, kout, h->st));
  if (r->lam) CK(cudaMemcpyAsync(r->lam, h->lam, sizeof(double) * m, kout, h->st));
  if (r->zeta) CK(cudaMemcpyAsync(r->zeta, h->zeta, sizeof(double) * n, kout, h->st));
  CK(objective_terms_f64(h->st, m, n, q, c, b, h->x, h->y, h->z, h->red_out + 4, h->red));
  int rc2 = sync_scalars(h, 8);
  const double xqx = h->h_red[4], cx = h->h_red[5], by = h->h_red[6];
  const double pobj = 0.5 * xqx + cx, dobj = by - 0.5 * xqx;
  r->ipm_iters = k;
  r->rel_primal = rel_p;
  r->rel_dual = rel_d;
  r->mu = mu;
  r->rel_gap = std::fabs(pobj - dobj) / (1.0 + std::fabs(pobj));
  r->rho = rho;
  r->delta = delta;
  if (status == NYS_OK && warn != NYS_OK) status = warn;
  if (status >= 0 && rc2 != NYS_OK) status = rc2;
  if (status >= 0 && h->h_red[7] != 0.0) status = fail(h, NYS_ERR_NUMERIC, "non-finite final iterate");
  r->status = status;
  r->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return status;
}

}  // extern "C"

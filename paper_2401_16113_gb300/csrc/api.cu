// C-ABI entry points (declared in include/aao.h): argument checks, handle lifetime, dispatch.
#include <math.h>
#include <stdio.h>

#include <chrono>
#include <mutex>
#include <string>
#include <vector>

#include "aao_internal.cuh"

namespace aao {

std::atomic<uint64_t> g_launches{0};
static thread_local std::string t_last_error;

void set_error(const std::string& msg) { t_last_error = msg; }

std::atomic<int> g_prof_mask{0};
namespace {
struct ProfState {
  std::mutex mu;
  std::vector<cudaEvent_t> pool;                    // free events
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> done[AAO_K_COUNT];
  double bytes[AAO_K_COUNT] = {};
  double flops[AAO_K_COUNT] = {};
  cudaEvent_t open[AAO_K_COUNT] = {};
};
ProfState& prof() {
  static ProfState* st = new ProfState();  // never destroyed: events may outlive static teardown
  return *st;
}
cudaEvent_t take_event(ProfState& st) {
  if (!st.pool.empty()) {
    cudaEvent_t e = st.pool.back();
    st.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void prof_begin(int cls, cudaStream_t s) {
  ProfState& st = prof();
  std::lock_guard<std::mutex> lk(st.mu);
  cudaEvent_t e = take_event(st);
  cudaEventRecord(e, s);
  st.open[cls] = e;
}

void prof_end(int cls, cudaStream_t s, double bytes, double fp64_flops) {
  ProfState& st = prof();
  std::lock_guard<std::mutex> lk(st.mu);
  if (!st.open[cls]) return;
  st.bytes[cls] += bytes;
  st.flops[cls] += fp64_flops;
  cudaEvent_t e = take_event(st);
  cudaEventRecord(e, s);
  st.done[cls].emplace_back(st.open[cls], e);
  st.open[cls] = nullptr;
}

namespace {

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int validate(const aao_problem* p) {
  if (!p) { set_error("aao_create: null problem"); return AAO_EINVAL; }
  if (p->nx < 2 || p->nt < 1) { set_error("aao_create: need nx >= 2 and nt >= 1"); return AAO_EINVAL; }
  if (p->op != AAO_OP_BS && p->op != AAO_OP_LOCALVOL && p->op != AAO_OP_RIESZ && !op_2d(p->op)) { set_error("aao_create: unknown op"); return AAO_EINVAL; }
  if (op_2d(p->op)) {
    if (p->precision != AAO_MIXED) { set_error("aao_create: the Heston and SABR operators are built for precision AAO_MIXED only"); return AAO_EUNSUPPORTED; }
    if (p->payoff != AAO_CALL) { set_error("aao_create: the Heston and SABR boundary conditions of Sec. 5.1-5.2 are those of a call"); return AAO_EUNSUPPORTED; }
    if (p->nx < 3 || p->nx > 512 || p->nv < 3 || p->nv > 512) { set_error("aao_create: Heston and SABR need 3 <= nx, nv <= 512"); return AAO_EUNSUPPORTED; }
    if (!(p->rho >= -1) || !(p->rho <= 1) || !(p->v_max > 0) || !(p->sigma >= 0)) {
      set_error("aao_create: Heston and SABR need v_max > 0, sigma >= 0 and -1 <= rho <= 1");
      return AAO_EINVAL;
    }
    if (p->op == AAO_OP_HESTON && (!(p->kappa > 0) || !(p->eta > 0))) {
      set_error("aao_create: Heston needs kappa, eta > 0");
      return AAO_EINVAL;
    }
    if (p->op == AAO_OP_SABR && !(p->beta >= 0.0 && p->beta <= 1.0)) {
      set_error("aao_create: SABR needs 0 <= beta <= 1");
      return AAO_EINVAL;
    }
    const double factors = 2.0 * p->nv * (double)(p->nt / 2 + 1) * p->nx * (double)p->nx * 8.0;
    if (factors > 48e9) { set_error("aao_create: Heston step-(b) block factors would exceed 48 GB"); return AAO_EUNSUPPORTED; }
  }
  if (p->op == AAO_OP_RIESZ) {
    if (p->precision != AAO_MIXED) { set_error("aao_create: the Riesz operator is built for precision AAO_MIXED only"); return AAO_EUNSUPPORTED; }
    if (!(p->beta > 1.0) || !(p->beta <= 2.0)) { set_error("aao_create: Riesz order beta must lie in (1, 2]"); return AAO_EINVAL; }
    if (p->nx > 2048) { set_error("aao_create: Riesz operator needs nx <= 2048"); return AAO_EUNSUPPORTED; }
    const double factors = (double)(p->nt / 2 + 1) * p->nx * (double)p->nx * 8.0;
    if (!riesz_symmetric(*p) && factors > 32e9) { set_error("aao_create: Riesz step-(b) inverses would exceed 32 GB (twice that while they are made)"); return AAO_EUNSUPPORTED; }
  }
  if (p->payoff != AAO_PUT && p->payoff != AAO_CALL) { set_error("aao_create: unknown payoff"); return AAO_EINVAL; }
  if (p->precision != AAO_FP64 && p->precision != AAO_MIXED) { set_error("aao_create: unknown precision"); return AAO_EINVAL; }
  MrPlan pl;
  if (!is_pow2(p->nt) && !mr_plan(p->nt, pl)) {
    set_error("aao_create: nt must have no prime factor above 7");
    return AAO_EUNSUPPORTED;
  }
  // the FP64 mixed-radix FFT keeps two columns of nt complex doubles in shared memory
  const int nt_max = (p->precision == AAO_MIXED || is_pow2(p->nt)) ? 8192 : 4096;
  if (p->nt > nt_max) { set_error("aao_create: nt above the shared-memory FFT limit (8192; 4096 for FP64 nt that is not a power of two)"); return AAO_EUNSUPPORTED; }
  if (p->nx > 8192) { set_error("aao_create: nx above the tridiagonal solver's limit (8192)"); return AAO_EUNSUPPORTED; }
  if (!(p->T > 0) || !(p->K > 0) || !(p->sigma > 0) || !(p->s_max > 0) || !(p->r >= 0)) {
    set_error("aao_create: need T, K, sigma, s_max > 0 and r >= 0");
    return AAO_EINVAL;
  }
  if (!(p->alpha > 0) || !(p->alpha <= 1)) { set_error("aao_create: need 0 < alpha <= 1"); return AAO_EINVAL; }
  if (p->flags != 0 && p->flags != AAO_FLAG_STEPB_FACTORED && p->flags != AAO_FLAG_STEPB_RECOMPUTE) {
    set_error("aao_create: flags must be 0 or one AAO_FLAG_STEPB_* value");
    return AAO_EINVAL;
  }
  return AAO_OK;
}

}  // namespace
}  // namespace aao

struct aao_handle {
  aao::Handle h;
  // device copies of b and x for fgmres_solve_host, made at its first call and kept until
  // aao_destroy (an allocation per call would map fresh pages each time: the default memory pool
  // releases freed memory at every synchronisation)
  double* host_b = nullptr;
  double* host_x = nullptr;
};

using namespace aao;

extern "C" {

int aao_create(const aao_problem* p, aao_handle** out) {
  NvtxRange nv("aao_create");
  if (!out) { set_error("aao_create: null handle pointer"); return AAO_EINVAL; }
  *out = nullptr;
  AAO_TRY(validate(p));
  aao_handle* hd = new aao_handle();
  Handle& h = hd->h;
  h.p = *p;
  h.stream = (cudaStream_t)p->stream;
  h.nx = op_2d(p->op) ? p->nx * p->nv : p->nx;  // spatial unknowns per time level
  h.nt = p->nt;
  h.K = p->nt / 2 + 1;
  int l = 0;
  while ((1 << l) < p->nt) ++l;
  h.log2n = l;
  if (!is_pow2(p->nt)) mr_plan(p->nt, h.mr);
  h.pitch = ((h.nx + 63) / 64) * 64;
  h.n = (size_t)h.nx * p->nt;
  h.mixed = p->precision == AAO_MIXED;
  int s = build_tables(h);
  if (s == AAO_OK) s = tune_precond(h);
  if (s != AAO_OK) {
    free_handle(h);
    delete hd;
    return s;
  }
  *out = hd;
  return AAO_OK;
}

int aao_destroy(aao_handle* hd) {
  if (!hd) return AAO_OK;
  cudaStreamSynchronize(hd->h.stream);
  if (hd->host_b) cudaFree(hd->host_b);
  if (hd->host_x) cudaFree(hd->host_x);
  free_handle(hd->h);
  delete hd;
  return AAO_OK;
}

int aao_rhs(aao_handle* hd, double* b) {
  NvtxRange nv("aao_rhs");
  if (!hd || !b) { set_error("aao_rhs: null argument"); return AAO_EINVAL; }
  return launch_rhs(hd->h, b);
}

int aao_matvec(aao_handle* hd, const double* x, double* y) {
  NvtxRange nv("aao_matvec");
  if (!hd || !x || !y) { set_error("aao_matvec: null argument"); return AAO_EINVAL; }
  if (x == y) { set_error("aao_matvec: x and y must not alias"); return AAO_EINVAL; }
  return launch_matvec(hd->h, x, false, y, nullptr);
}

int precond_apply(aao_handle* hd, const double* v, double* z) {
  NvtxRange nv("precond_apply");
  if (!hd || !v || !z) { set_error("precond_apply: null argument"); return AAO_EINVAL; }
  Handle& h = hd->h;
  AAO_TRY(launch_precond(h, v, z, false));
  if (h.rz_err) {
    // the spectral step (b) of the symmetric Riesz operator runs on the tensor cores with bounded
    // waits: read (and clear) its error word, so that a product that gave up is reported here
    int e = 0;
    AAO_TRY_CUDA(cudaMemcpyAsync(&e, h.rz_err, sizeof(int), cudaMemcpyDeviceToHost, h.stream));
    AAO_TRY_CUDA(cudaStreamSynchronize(h.stream));
    if (e) {
      AAO_TRY_CUDA(cudaMemsetAsync(h.rz_err, 0, sizeof(int), h.stream));
      set_error("precond_apply: a tensor-core product of step (b) gave up a bounded wait; z is not valid");
      return AAO_TIMEOUT;
    }
  }
  return AAO_OK;
}

int aao_fault_inject(aao_handle* hd, int mask, double wait_ms) {
  if (!hd || (mask & ~AAO_INJECT_TC_NO_LOAD) != 0) { set_error("aao_fault_inject: bad argument"); return AAO_EINVAL; }
  Handle& h = hd->h;
  h.rz_inject = mask & AAO_INJECT_TC_NO_LOAD;
  h.rz_wait_ns = wait_ms > 0 ? (unsigned long long)(wait_ms * 1e6) : 2000000000ull;
  return AAO_OK;
}

int fgmres_solve(aao_handle* hd, const double* b, double* x, double tol, int m, int maxit, aao_stats* st) {
  NvtxRange nv("fgmres_solve");
  if (!hd || !b || !x) { set_error("fgmres_solve: null argument"); return AAO_EINVAL; }
  if (m < 1 || m > 64 || maxit < 1 || !(tol > 0)) { set_error("fgmres_solve: need 1 <= m <= 64, maxit >= 1, tol > 0"); return AAO_EINVAL; }
  return run_fgmres(hd->h, b, x, tol, m, maxit, st);
}

int fgmres_solve_zero(aao_handle* hd, const double* b, double* x, double tol, int m, int maxit, aao_stats* st) {
  NvtxRange nv("fgmres_solve_zero");
  if (!hd || !b || !x) { set_error("fgmres_solve_zero: null argument"); return AAO_EINVAL; }
  if (m < 1 || m > 64 || maxit < 1 || !(tol > 0)) { set_error("fgmres_solve_zero: need 1 <= m <= 64, maxit >= 1, tol > 0"); return AAO_EINVAL; }
  return run_fgmres(hd->h, b, x, tol, m, maxit, st, true);
}

int fgmres_solve_host(aao_handle* hd, const double* b_host, double* x_host, double tol, int m, int maxit,
                      aao_stats* st) {
  NvtxRange nv("fgmres_solve_host");
  if (!hd || !b_host || !x_host) { set_error("fgmres_solve_host: null argument"); return AAO_EINVAL; }
  if (m < 1 || m > 64 || maxit < 1 || !(tol > 0)) { set_error("fgmres_solve_host: need 1 <= m <= 64, maxit >= 1, tol > 0"); return AAO_EINVAL; }
  Handle& h = hd->h;
  const size_t bytes = sizeof(double) * h.n;
  if (!hd->host_b) AAO_TRY_CUDA(cudaMalloc(&hd->host_b, bytes));
  if (!hd->host_x) AAO_TRY_CUDA(cudaMalloc(&hd->host_x, bytes));
  double *b = hd->host_b, *x = hd->host_x;
  AAO_TRY_CUDA(cudaMemcpyAsync(b, b_host, bytes, cudaMemcpyHostToDevice, h.stream));
  int s = run_fgmres(h, b, x, tol, m, maxit, st, true);
  cudaError_t e = cudaMemcpyAsync(x_host, x, bytes, cudaMemcpyDeviceToHost, h.stream);
  cudaError_t e2 = cudaStreamSynchronize(h.stream);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    set_error(std::string("fgmres_solve_host: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    return AAO_ECUDA;
  }
  return s;
}

int aao_sym_eig(int n, double* A_host, double* w_host) {
  if (n < 1 || !A_host || !w_host) { set_error("aao_sym_eig: bad argument"); return AAO_EINVAL; }
  if (!sym_eig(n, A_host, w_host)) {
    set_error("aao_sym_eig: the symmetric QR iteration did not converge");
    return AAO_BREAKDOWN;
  }
  return AAO_OK;
}

unsigned int aao_check_failures(void) {
  cudaDeviceSynchronize();
  return check_word_precond() + check_word_krylov() + check_word_riesz() + check_word_heston();
}

const char* aao_last_error(void) { return t_last_error.c_str(); }

uint64_t aao_launch_count(void) { return g_launches.load(); }

int aao_profile_enable(int mask) {
  ProfState& st = prof();
  std::lock_guard<std::mutex> lk(st.mu);
  for (int c = 0; c < AAO_K_COUNT; ++c) {
    for (auto& pr : st.done[c]) {
      cudaEventSynchronize(pr.second);
      st.pool.push_back(pr.first);
      st.pool.push_back(pr.second);
    }
    st.done[c].clear();
    st.bytes[c] = 0.0;
    st.flops[c] = 0.0;
  }
  g_prof_mask.store(mask);
  return AAO_OK;
}

int aao_profile_read(int cls, int64_t* launches, double* total_ms, double* bytes, double* fp64_flops) {
  if (cls < 0 || cls >= AAO_K_COUNT || !launches || !total_ms || !bytes || !fp64_flops) { set_error("aao_profile_read: bad argument"); return AAO_EINVAL; }
  ProfState& st = prof();
  std::lock_guard<std::mutex> lk(st.mu);
  double tot = 0.0;
  for (auto& pr : st.done[cls]) {
    AAO_TRY_CUDA(cudaEventSynchronize(pr.second));
    float ms = 0.f;
    AAO_TRY_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
    tot += ms;
  }
  *launches = (int64_t)st.done[cls].size();
  *total_ms = tot;
  *bytes = st.bytes[cls];
  *fp64_flops = st.flops[cls];
  return AAO_OK;
}

}  // extern "C"

// Internal declarations of the GB300 all-at-once CN solver library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/aao.h"

namespace aao {

// ------------------------------------------------------------------ error plumbing
void set_error(const std::string& msg);
extern std::atomic<uint64_t> g_launches;

#define AAO_TRY_CUDA(expr)                                                              \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      (void)cudaGetLastError(); /* clear a non-sticky error so later calls do not see it */ \
      ::aao::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));             \
      return e_ == cudaErrorMemoryAllocation ? AAO_ENOMEM : AAO_ECUDA;                  \
    }                                                                                   \
  } while (0)

#define AAO_CHECK_LAUNCH()                                                              \
  do {                                                                                  \
    ::aao::g_launches.fetch_add(1, std::memory_order_relaxed);                          \
    cudaError_t e_ = cudaGetLastError();                                                \
    if (e_ != cudaSuccess) {                                                            \
      ::aao::set_error(std::string("kernel launch: ") + cudaGetErrorString(e_));         \
      return AAO_ECUDA;                                                                 \
    }                                                                                   \
  } while (0)

#define AAO_TRY(expr)            \
  do {                           \
    int s_ = (expr);             \
    if (s_ != AAO_OK) return s_; \
  } while (0)

// ------------------------------------------------------------------ bounds-checked build
// Built with -DAAO_CHECK (build.build(check=True): _build_check/libaao_check.so), device code tests
// the index of each global store it guards with AAO_DCHECK(cond): a failed test sets this
// translation unit's device word and the store is skipped (no fault); aao_check_failures() reads and
// clears the words of every unit. In the normal build AAO_DCHECK(cond) is the constant true and the
// tests compile away.
#ifdef AAO_CHECK
static __device__ unsigned int g_aao_check = 0u;
__device__ __forceinline__ bool aao_dcheck(bool ok) {
  if (!ok) atomicOr(&g_aao_check, 1u);
  return ok;
}
#define AAO_DCHECK(cond) ::aao::aao_dcheck((cond))
// this unit's word (read and cleared), and the sum over units
#define AAO_CHECK_WORD_FN(name)                                                        \
  unsigned int name() {                                                                \
    unsigned int v = 0u, z = 0u;                                                       \
    if (cudaMemcpyFromSymbol(&v, g_aao_check, sizeof v) != cudaSuccess) v = 1u;        \
    cudaMemcpyToSymbol(g_aao_check, &z, sizeof z);                                     \
    return v;                                                                          \
  }
#else
#define AAO_DCHECK(cond) true
#define AAO_CHECK_WORD_FN(name) \
  unsigned int name() { return 0u; }
#endif
unsigned int check_word_precond();
unsigned int check_word_krylov();
unsigned int check_word_riesz();
unsigned int check_word_heston();

// ------------------------------------------------------------------ device timing
// When enabled, every launch inside a ProfScope is bracketed by two CUDA events recorded on
// the launching stream; aao_profile_read sums their elapsed times per kernel class.
// Each scope also records the launch's algorithmic bytes (what it must read and write once) and
// its algorithmic FP64 flops (an FMA counts 2), so that a roofline can name the binding resource.
void prof_begin(int cls, cudaStream_t s);
void prof_end(int cls, cudaStream_t s, double bytes, double fp64_flops);
extern std::atomic<int> g_prof_mask;
struct ProfScope {
  int cls;
  cudaStream_t s;
  double bytes, flops;
  bool on;
  ProfScope(int c, cudaStream_t st, double b = 0.0, double f = 0.0) : cls(c), s(st), bytes(b), flops(f) {
    on = (g_prof_mask.load(std::memory_order_relaxed) >> c) & 1;
    if (on) prof_begin(cls, s);
  }
  ~ProfScope() {
    if (on) prof_end(cls, s, bytes, flops);
  }
};

// ------------------------------------------------------------------ complex helpers
template <typename R> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename R> using C_t = typename cplx<R>::type;

template <typename C> __host__ __device__ __forceinline__ C cmk(decltype(C::x) a, decltype(C::x) b) {
  C c; c.x = a; c.y = b; return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmk<C>(a.x, -a.y); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return cmk<C>(a.x * s, a.y * s); }
// multiply by -i
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { return cmk<C>(a.y, -a.x); }
// 1 / z
template <typename C> __device__ __forceinline__ C cinv(C a) {
  auto d = a.x * a.x + a.y * a.y;
  auto s = (decltype(C::x))1 / d;
  return cmk<C>(a.x * s, -a.y * s);
}

// ------------------------------------------------------------------ programmatic dependent launch
// The solver's kernels are launched with programmatic stream serialisation: a kernel's CTAs may
// be scheduled while the previous kernel's last CTAs still run; each kernel starts with
// pdl_sync(), which waits until the previous grid has completed (its writes visible) and then
// lets the next grid be scheduled once all of this grid's CTAs are resident. Launched without
// the attribute, both instructions return at once.
__device__ __forceinline__ void pdl_sync() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ------------------------------------------------------------------ conversions
// FP64 instructions (conversions included) share the slow FP64 pipe on this part, so the
// FP32 <-> FP64 conversions on the hot path are assembled from integer bit operations.
// widen: exact for normal numbers, zero, inf and NaN; FP32 subnormals become zero.
__device__ __forceinline__ double widen(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned mant = (e == 0u) ? 0u : (b & 0x7fffffu);
  unsigned ed = e + 896u;
  ed = (e == 0xffu) ? 2047u : ed;
  ed = (e == 0u) ? 0u : ed;
  const unsigned hi = (b & 0x80000000u) | (ed << 20) | (mant >> 3);
  return __hiloint2double((int)hi, (int)(mant << 29));
}
__device__ __forceinline__ double widen(double d) { return d; }

// twice: 2 x, exactly, from integer bit operations. FP32 input: widen with the exponent one
// higher (never overflows in FP64). FP64 input: a normal number gets exponent + 1 (the top binade
// overflows to inf); a zero or subnormal doubles its magnitude bits (the carry moves into the
// exponent field, which is the exact 2 x); inf and NaN are returned unchanged.
__device__ __forceinline__ double twice(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned mant = (e == 0u) ? 0u : (b & 0x7fffffu);
  unsigned ed = e + 897u;
  ed = (e == 0xffu) ? 2047u : ed;
  ed = (e == 0u) ? 0u : ed;
  const unsigned hi = (b & 0x80000000u) | (ed << 20) | (mant >> 3);
  return __hiloint2double((int)hi, (int)(mant << 29));
}
__device__ __forceinline__ double twice(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned e = (hi >> 20) & 0x7ffu, sign = hi & 0x80000000u;
  unsigned nhi = hi + 0x00100000u, nlo = lo;
  if (e == 0u) {
    nhi = sign | ((hi & 0x7fffffffu) << 1) | (lo >> 31);
    nlo = lo << 1;
  }
  if (e == 0x7feu) {
    nhi = sign | 0x7ff00000u;
    nlo = 0u;
  }
  if (e == 0x7ffu) {
    nhi = hi;
    nlo = lo;
  }
  return __hiloint2double((int)nhi, (int)nlo);
}

// narrow: round to nearest (ties away from zero) for results in the FP32 normal range;
// overflow gives inf, results below the normal range give zero, NaN stays NaN. Only 32-bit
// integer operations: the rounding carry from the low word is propagated by hand.
__device__ __forceinline__ float narrow(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned sign = hi & 0x80000000u, ehi = hi & 0x7fffffffu;
  const unsigned lo2 = lo + 0x10000000u;                 // half of the 29 dropped bits
  const unsigned hi2 = ehi + (lo2 < lo ? 1u : 0u);        // carry, possibly into the exponent
  const int fe = (int)(hi2 >> 20) - 896;
  unsigned fb = (((hi2 << 3) | (lo2 >> 29)) & 0x7fffffu) | ((unsigned)fe << 23);
  fb = fe >= 255 ? 0x7f800000u : fb;
  fb = fe <= 0 ? 0u : fb;
  fb = ehi >= 0x7ff00000u ? ((ehi > 0x7ff00000u || lo != 0u) ? 0x7fc00000u : 0x7f800000u) : fb;
  return __uint_as_float(sign | fb);
}

// NVTX range for the duration of a scope (entry points, FGMRES restart cycles): header-only
// NVTX v3, a no-op unless a profiler is attached
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ------------------------------------------------------------------ handle
// Stages of the mixed-radix FFT along t (nt not a power of two): nt = rad[0] rad[1] ...
// rad[nst-1], each radix 2, 3, 4, 5, 7 or 8; nst = 0 when nt is a power of two.
struct MrPlan {
  int nst;
  int rad[15];
};
// the stages for n (eights first), false when n has a prime factor above 7
inline bool mr_plan(int n, MrPlan& pl) {
  pl.nst = 0;
  for (int f : {8, 4, 2, 3, 5, 7})
    while (n % f == 0 && pl.nst < 15) { pl.rad[pl.nst++] = f; n /= f; }
  return n == 1;
}

struct Handle {
  aao_problem p;
  cudaStream_t stream = 0;
  int nx = 0, nt = 0, K = 0, log2n = 0;
  int pitch = 0;          // row pitch (complex elements) of the half spectrum [K][pitch]
  double tau = 0.0;
  size_t n = 0;           // nx * nt
  bool mixed = false;
  int coef_rows = 1;      // 1 (constant operator) or nt (time-dependent)

  // matvec coefficients: rows of nx, coef_rows rows each: lower and upper of (1/2) tau A_t and
  // the diagonal of I + (1/2) tau A_t. lower[0] and upper[nx-1] hold the Dirichlet-node
  // coefficients (used by aao_rhs only).
  double *mL = nullptr, *mD = nullptr, *mU = nullptr;
  double* gL = nullptr;   // left Dirichlet values at t_0..t_nt
  double* gR = nullptr;   // right Dirichlet values
  // preconditioner: tau * Abar diagonals, eigenvalue ratios mu_k = lambda1_k / lambda2_k,
  // 1/lambda2_k, Lambda_alpha and (Lambda_alpha^{-1} / nt), twiddles exp(-2 pi i m / nt)
  double *pL = nullptr, *pD = nullptr, *pU = nullptr;
  float *pLf = nullptr, *pDf = nullptr, *pUf = nullptr;
  double2 *mu = nullptr, *il2 = nullptr, *tw = nullptr;
  float2 *muf = nullptr, *il2f = nullptr, *twf = nullptr;
  double *lam = nullptr, *ilam = nullptr;
  float *lamf = nullptr, *ilamf = nullptr;
  void* spec = nullptr;   // half spectrum, K * pitch complex (float2 or double2)
  int fft_p = 0;          // FFT tile: 2*fft_p spatial columns per CTA (0 = heuristic)
  MrPlan mr{};            // mixed-radix stages when nt is not a power of two (mr.nst > 0)
  // step (b) partition: tri_T (a power of two) threads per bin, tri_ch rows each; coefficients a, diag, c chunk-
  // transposed ([j][l]) in one buffer of 3 * tri_ch * tri_T reals (precision of the preconditioner)
  void* tri = nullptr;
  int tri_T = 0, tri_ch = 0;
  // factors of step (b) per bin (complex, precision of the preconditioner): pivots and fill-in
  // [K][tri_T * tri_ch], reduction multipliers [K][2 lgT + 1][tri_T]; null where the
  // partition method does not fit in shared memory
  void *tri_fp = nullptr, *tri_fv = nullptr, *tri_fpcr = nullptr;
  // step (b) by k_tridiag_rc (pivots recomputed from tri, no per-bin tables) instead of the
  // factored partition method: where the factor tables do not fit, or by request (flags)
  bool tri_rc = false;

  // Riesz operator (dense Toeplitz): circulant-embedding spectrum (scaled by tau/2 / N2), its
  // twiddles, (tau/2) first column / row / left-exterior coefficients, inverses of step (b)
  int rz_n2 = 0, rz_log2n2 = 0;
  double2 *rz_chat = nullptr, *rz_tw = nullptr;
  double *rz_hcol = nullptr, *rz_hrow = nullptr, *rz_hcl = nullptr;
  float* Vf = nullptr;  // FP32 copy of the basis vector the next preconditioner apply reads (mixed)
  float2* rz_inv = nullptr;   // the inverses X_k of the shifted matrices, [k][i][j] (with drift)
  // symmetric Riesz operator (no drift): tau Abar = Q diag(lambda) Q^T; step (b) is
  // z2_k = Q diag(D_k) Q^T z1_k with D_k,j = (1/lambda_{2,k}) / (mu_k - lambda_j)
  bool rz_sym = false;
  float2* rz_dk = nullptr;  // D, [k][j] (FP32 complex)
  float2* rz_w = nullptr;   // the result of step (b) per bin, K x pitch complex (with drift)
  float2* rz_part = nullptr;  // partial products of the contraction segments
  int rz_ldq = 0;           // leading dimension of Q, Q^T, D and the workspaces
  int rz_kpad = 0;          // bins padded to whole 32-bin tiles of the tensor-core products
  int rz_nseg = 1;          // contraction segments of each tensor-core product
  float *rz_bh = nullptr, *rz_bl = nullptr;  // their complex operand, TF32 head and tail, tiled
  // TF32 head and tail (x = hi + lo) of Q (rows x, entries j) and of Q^T (rows j, entries x):
  // the tensor-core operands, zero-padded to rz_ldq and stored in 8 x 16-byte core-matrix tiles
  float *rz_qh = nullptr, *rz_ql = nullptr;
  float *rz_qth = nullptr, *rz_qtl = nullptr;
  int* rz_err = nullptr;    // set by a tensor-core product whose bounded wait gave up
  unsigned long long rz_wait_ns = 2000000000ull;  // bound of each wait in those products
  int rz_inject = 0;        // fault injection (aao_fault_inject): the products issue no operator load
  // TMA tensor maps (CUtensorMap, 128 bytes each) of the tiled Q^T head, tail, Q head, tail and of
  // the complex operand's head and tail
  alignas(64) unsigned char rz_tmap[6 * 128] = {};

  // Heston and SABR operators (AAO_OP_HESTON, AAO_OP_SABR): grid hs_ns x hs_nv (nx = hs_ns * hs_nv
  // unknowns per level);
  // per unknown the ten stencil coefficients of (tau/2) A (FP64 for the matvec, FP32 for step (b)),
  // tau f (boundary data), the payoff; step (b) per bin and v level: X_j = D_j^{-1},
  // G_j = X_j C'_j (j < nv - 1), H_0 = X_0 E_0 (FP32 complex, [j][k][ns][ns])
  int hs_ns = 0, hs_nv = 0;
  int hs_C = 1;  // CTAs per bin (thread-block cluster) of the step (b) apply
  double *hs_c = nullptr, *hs_tf = nullptr, *hs_u0 = nullptr;
  float* hs_cf = nullptr;
  float2 *hs_X = nullptr, *hs_G = nullptr, *hs_H = nullptr;

  // FGMRES workspace (grown on demand)
  int ws_m = 0;
  double* V = nullptr;    // (m+1) * n
  void* Z = nullptr;      // m * n (float when mixed, double otherwise)
  double* w = nullptr;    // n
  double* scal = nullptr; // small device scalars (see krylov.cu)
  double* part = nullptr; // block partial sums
  unsigned int* counter = nullptr;  // completion counter of the last-block reductions
  int part_blocks = 0;
  int sms = 0;            // multiprocessors of the handle's device
  double* host_scal = nullptr;  // pinned mirror
};

// launchers (return AAO_* codes)
int build_tables(Handle& h);
// vf (mixed precision only): an FP32 copy of v, read instead of v by the first kernel
int launch_precond(Handle& h, const double* v, void* z, bool z_is_float, const double* in_scale = nullptr,
                   const float* vf = nullptr);
int tune_precond(Handle& h);
// factors of the partitioned tridiagonal solves of step (b) (needs tri, mu/muf)
int build_tri_factors(Handle& h);
// The Riesz operator has no drift term ((r - sigma^2/2) u_x vanishes): its matrix is symmetric.
// the two-dimensional operators in (s, v), which share the grid, the stencil matvec and step (b)
inline bool op_2d(int op) { return op == AAO_OP_HESTON || op == AAO_OP_SABR; }
inline bool riesz_symmetric(const aao_problem& p) { return p.r - 0.5 * p.sigma * p.sigma == 0.0; }
// A = Q diag(w) Q^T for a dense symmetric n x n A (row-major, FP64, host); A is overwritten with
// Q^T. False if the symmetric QR iteration does not converge.
bool sym_eig(int n, double* A, double* w);
int riesz_build(Handle& h);
// in place: each of the K contiguous n x n complex matrices of M replaced by its inverse (blocked
// Gauss-Jordan without pivoting, the rank-64 updates on the tensor cores); synchronises the stream
int gj_invert_batched(cudaStream_t stream, float2* M, int n, int K);
// the Heston operator: stencil, boundary data and the step (b) block factors; matvec, b, step (b)
int heston_build(Handle& h);
int heston_matvec(Handle& h, const void* x, bool x_is_float, double* y, const double* b, const double* V, int nd,
                  int m);
int heston_rhs(Handle& h, double* b);
int heston_solve_bins(Handle& h, void* spec);
int riesz_matvec(Handle& h, const void* x, bool x_is_float, double* y, const double* b, const double* V, int nd, int m);
int riesz_rhs(Handle& h, double* b);
// step (b) of the Riesz operator on the half spectrum spec; *result: the buffer holding z2
// (spec itself, or the workspace rz_w)
int riesz_solve_bins(Handle& h, void* spec, void** result);
// yf (residual modes, mixed precision): also write an FP32 copy of y
int launch_matvec(Handle& h, const void* x, bool x_is_float, double* y, const double* b, const double* V = nullptr,
                  int nd = 0, int m = 0, bool with_bnorm = false, float* yf = nullptr);
int launch_rhs(Handle& h, double* b);
// zero_guess: x is output only and the solve starts from x_0 = 0 (the first residual is b)
int run_fgmres(Handle& h, const double* b, double* x, double tol, int m, int maxit, aao_stats* st,
               bool zero_guess = false);
void free_handle(Handle& h);

}  // namespace aao

// P_alpha^{-1} apply on GB300: the three steps of Eq. 3.2 with the conjugate-pair saving of
// Remark 1, as three kernels joined by the half spectrum in HBM/L2.
//
//   k_fft_fwd   step (a): Lambda_alpha scaling (first factor of V_alpha^{-1} = F Lambda_alpha)
//               fused with a real-to-complex FFT along t for a tile of 2P spatial columns.
//               Two real columns are packed into one complex column; the FFT is a Stockham
//               transform, radix 16/16/8 with 16 values per thread in registers for nt >= 128
//               (radix 4/2 in shared memory below). Output: bins k = 0..nt/2 of every
//               column, frequency-major [k][x] (the layout step (b) reads contiguously).
//   k_tridiag_part
//               step (b): for each bin k, T threads solve the complex-shifted tridiagonal system
//               (lambda_{1,k} I - lambda_{2,k} A~) z2_k = z1_k, A~ = tau * Abar, by the partition
//               method (chunks of ceil(nx/T) rows per thread, parallel cyclic reduction of the
//               T-row interface system in shared memory). The matrix-only parts (pivots,
//               fill-in, reduction multipliers) are factored once per bin when the handle is built
//               (k_tridiag_part_factor); an apply carries only the right-hand side. k_tridiag
//               (one bin per group of lanes, coefficients recomputed) serves the shapes whose
//               rows do not fit in shared memory.
//   k_fft_inv   step (c): complex-to-real inverse FFT along t (bins nt/2+1.. are the conjugates,
//               Remark 1) fused with Lambda_alpha^{-1} and the 1/nt normalisation.
//   k_fft_fwd_mr / k_fft_inv_mr
//               steps (a) and (c) for nt that is not a power of two (prime factors 2, 3, 5, 7):
//               shared-memory Stockham stages of radix 8, 4, 2, 3, 5, 7.
//
// The unitary DFT of Sec. 3.1 carries 1/sqrt(nt) in each direction; here the forward FFT is
// unnormalised and the single 1/nt is folded into the unscaling table.
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "precond_dev.cuh"

namespace aao {

namespace {

using namespace pdev;

constexpr size_t kTriSmemMax = 227 * 1024;  // dynamic shared memory per CTA

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) only when a launch needs more than was set
// before for that kernel on the current device (the attribute belongs to one device; the call is
// not free on the host, and the host's lead over the GPU matters after every status read-back of
// the solver)
int ensure_smem(const void* kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return AAO_OK;
  int dev = 0;
  AAO_TRY_CUDA(cudaGetDevice(&dev));
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> set;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = set[{dev, kernel}];
  if (bytes <= cur) return AAO_OK;
  AAO_TRY_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  cur = bytes;
  return AAO_OK;
}


// A launch with programmatic dependent launch (see launch_pdl) or, pdl false, a plain one: the
// kernel's CTAs are then scheduled only once the previous kernel has finished.
template <typename... KArgs, typename... Args>
cudaError_t launch_maybe_pdl(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args... args) {
  if (pdl) return launch_pdl(kernel, grid, block, smem, s, args...);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.numAttrs = 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// threads of the FFT kernels: kVals complex values per thread per stage, a multiple of 32,
// within the kernels' launch bounds
int fft_threads(int P, int N, size_t rsize) {
  int threads = (P * N + kVals - 1) / kVals;
  threads = ((threads + 31) / 32) * 32;
  if (threads < 64) threads = 64;
  const int tmax = rsize == 8 ? 512 : 1024;
  if (threads > tmax) threads = tmax;
  return threads;
}

// largest power of two P <= 16 with P*N within the register/shared-memory budget
int max_tile(int N, size_t rsize) {
  const int vmax = rsize == 4 ? 16384 : 8192;
  int P = 16;
  while (P > 1 && P * N > vmax) P >>= 1;
  return P;
}

int default_tile(int nx, int N, size_t rsize) {
  int P = max_tile(N, rsize);
  while (P > 1 && (nx + 2 * P - 1) / (2 * P) < 2 * 152) P >>= 1;
  return P;
}

// ------------------------------------------------------------ mixed-radix FFT along t
// For nt not a power of two (prime factors 2, 3, 5, 7): steps (a) and (c) by the mixed-radix
// column tiles of precond_dev.cuh (fft_fwd_mr_tile / fft_inv_mr_tile), one tile per CTA.
// Both kernels are launched with mr_threads<R>() threads (the tiles' strided loops assume it).
template <typename R, typename IN>
__global__ void __launch_bounds__(mr_threads<R>(), 2)
    k_fft_fwd_mr(const IN* __restrict__ v, C_t<R>* __restrict__ spec, int nx, int N, MrPlan pl, int lp, int pitch,
                 const R* __restrict__ lam, const C_t<R>* __restrict__ tw, const double* __restrict__ in_scale) {
  using C = C_t<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int P = 1 << lp;
  C* b0 = reinterpret_cast<C*>(smraw);
  C* b1 = b0 + (size_t)P * N;
  C* stw = b1 + (size_t)P * N;  // twiddle table copy (N complex)
  for (int m = threadIdx.x; m < N; m += blockDim.x) stw[m] = __ldg(&tw[m]);
  pdl_sync();
  const R sc = in_scale ? to_r<R>(*in_scale) : (R)1;
  fft_fwd_mr_tile<R, IN, mr_threads<R>()>(v, spec, nx, N, pl, lp, pitch, lam, sc, blockIdx.x * 2 * P, b0, b1, stw);
}

template <typename R, typename OUT>
__global__ void __launch_bounds__(mr_threads<R>(), 2)
    k_fft_inv_mr(const C_t<R>* __restrict__ spec, OUT* __restrict__ z, int nx, int N, MrPlan pl, int lp, int pitch,
                 const R* __restrict__ ilam, const C_t<R>* __restrict__ tw) {
  using C = C_t<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int P = 1 << lp;
  C* b0 = reinterpret_cast<C*>(smraw);
  C* b1 = b0 + (size_t)P * N;
  C* stw = b1 + (size_t)P * N;  // twiddle table copy (N complex)
  for (int m = threadIdx.x; m < N; m += blockDim.x) stw[m] = __ldg(&tw[m]);
  pdl_sync();
  fft_inv_mr_tile<R, OUT, mr_threads<R>()>(spec, z, nx, N, pl, lp, pitch, ilam, blockIdx.x * 2 * P, b0, b1, stw);
}

// tile of the mixed-radix kernels: the largest power of two P <= 16 with both buffers and the
// twiddle table within 112 KB (two CTAs per SM, each with its 1 KB reserve, in the SM's 228 KB)
size_t mr_smem(int P, int N, size_t csize) { return (2 * (size_t)P + 1) * N * csize; }
int mr_max_tile(int N, size_t csize) {
  int P = 16;
  while (P > 1 && mr_smem(P, N, csize) > 112 * 1024) P >>= 1;
  return P;
}

// partition-method layout of step (b): lgT, the odd chunk stride cs, coefficient staging and the
// bins per CTA G; false when one bin's rows do not fit in shared memory
struct TriPart {
  int lgT, cs, G;
  bool staged;
  size_t smem;
};
bool tri_part_layout(const Handle& h, size_t rsize, TriPart& t) {
  if (!h.tri || h.tri_T <= 0) return false;
  const int T = h.tri_T, ch = h.tri_ch;
  t.lgT = 0;
  while ((1 << t.lgT) < T) ++t.lgT;
  if (t.lgT > kTriMaxLgT) return false;
  t.cs = (ch & 1) ? ch + 2 : ch + 1;
  if (tri_part_bytes(1, T, t.cs, rsize, false) > kTriSmemMax) return false;
  t.staged = tri_part_bytes(1, T, t.cs, rsize, true) <= kTriSmemMax;
  t.G = 512 / T;
  while (t.G > 1 && tri_part_bytes(t.G, T, t.cs, rsize, t.staged) > kTriSmemMax) --t.G;
  t.smem = tri_part_bytes(t.G, T, t.cs, rsize, t.staged);
  return true;
}

// layout of k_tridiag_rc: lgT, the odd chunk stride cs, bins per CTA G (at most 512 threads), the
// coefficient planes staged in shared memory (sc) where they fit; per CTA at most 112 KB in FP32
// (two CTAs per SM) and one CTA's limit in FP64. False when one bin does not fit.
struct TriRc {
  int lgT, cs, G, CH;
  bool sc;
  size_t smem;
};
bool tri_rc_layout(const Handle& h, size_t rsize, TriRc& t) {
  if (!h.tri || h.tri_T <= 0 || h.tri_ch > 16) return false;
  const int T = h.tri_T, ch = h.tri_ch;
  t.lgT = 0;
  while ((1 << t.lgT) < T) ++t.lgT;
  if (t.lgT > kTriMaxLgT) return false;
  t.cs = (ch & 1) ? ch + 2 : ch + 1;
  t.CH = ch <= 4 ? 4 : (ch <= 8 ? 8 : 16);
  const size_t budget = rsize == 4 ? 112 * 1024 : kTriSmemMax;
  const size_t bin = tri_rc_bin_bytes(T, t.cs, 2 * rsize);
  for (int sc = 1; sc >= 0; --sc) {
    const size_t cb = sc ? ((3 * (size_t)ch * T * rsize) + 15) & ~(size_t)15 : 0;
    int G = 512 / T;
    if (G > 15) G = 15;  // named barriers 1..15, one per bin
    while (G > 1 && cb + G * bin > budget) --G;
    if (cb + G * bin <= budget) {
      t.G = G;
      t.sc = sc != 0;
      t.smem = cb + G * bin;
      return true;
    }
  }
  return false;
}

template <typename R, int CH, bool SC>
int launch_tri_rc_t(Handle& h, const TriRc& t, C_t<R>* spec, const C_t<R>* mu, const C_t<R>* il2) {
  AAO_TRY(ensure_smem((const void*)k_tridiag_rc<R, CH, SC>, t.smem));
  AAO_TRY_CUDA(launch_pdl(k_tridiag_rc<R, CH, SC>, (h.K + t.G - 1) / t.G, t.G << t.lgT, t.smem, h.stream, spec,
                          h.nx, h.K, h.pitch, h.tri_ch, t.cs, t.lgT, reinterpret_cast<const R*>(h.tri), mu, il2));
  return AAO_OK;
}

template <typename R>
int launch_tri_rc(Handle& h, const TriRc& t, C_t<R>* spec, const C_t<R>* mu, const C_t<R>* il2) {
  if (t.sc) {
    if (t.CH == 4) return launch_tri_rc_t<R, 4, true>(h, t, spec, mu, il2);
    if (t.CH == 8) return launch_tri_rc_t<R, 8, true>(h, t, spec, mu, il2);
    return launch_tri_rc_t<R, 16, true>(h, t, spec, mu, il2);
  }
  if (t.CH == 4) return launch_tri_rc_t<R, 4, false>(h, t, spec, mu, il2);
  if (t.CH == 8) return launch_tri_rc_t<R, 8, false>(h, t, spec, mu, il2);
  return launch_tri_rc_t<R, 16, false>(h, t, spec, mu, il2);
}

template <typename R>
int tri_factors_t(Handle& h, int lgT) {
  using C = C_t<R>;
  const int T = h.tri_T, ch = h.tri_ch, K = h.K;
  const size_t rows = (size_t)T * ch;
  AAO_TRY_CUDA(cudaMalloc(&h.tri_fp, sizeof(C) * rows * K));
  AAO_TRY_CUDA(cudaMalloc(&h.tri_fv, sizeof(C) * rows * K));
  AAO_TRY_CUDA(cudaMalloc(&h.tri_fpcr, sizeof(C) * tri_fact_pcr_elems(lgT, T) * K));
  const C* mu = (sizeof(R) == 4) ? (const C*)h.muf : (const C*)h.mu;
  k_tridiag_part_factor<R><<<K, T, 5 * T * sizeof(C), h.stream>>>(
      h.nx, ch, lgT, reinterpret_cast<const R*>(h.tri), mu, reinterpret_cast<C*>(h.tri_fp),
      reinterpret_cast<C*>(h.tri_fv), reinterpret_cast<C*>(h.tri_fpcr));
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

// skip_b: steps (a) and (c) only (the FFT-tile autotuner of the dense operators, whose step (b) does
// not depend on the tile and would dominate the timing)
template <typename R>
int run_precond(Handle& h, const double* v, void* z, bool z_is_float, const double* in_scale, const float* vf,
                bool skip_b = false) {
  using C = C_t<R>;
  const int N = h.nt, nx = h.nx;
  const bool mr = h.mr.nst > 0;  // nt not a power of two: the mixed-radix kernels
  const int P = h.fft_p > 0 ? h.fft_p : (mr ? mr_max_tile(N, sizeof(C)) : default_tile(nx, N, sizeof(R)));
  int threads = mr ? mr_threads<R>() : fft_threads(P, N, sizeof(R));
  int lp = 0;  // the mixed-radix tiles are powers of two
  while ((1 << lp) < P) ++lp;
  const size_t smem = mr ? mr_smem(P, N, sizeof(C)) : fft_tile_bytes(P, N, sizeof(C));
  const int grid = (nx + 2 * P - 1) / (2 * P);
  C* spec = reinterpret_cast<C*>(h.spec);
  const R* lam = (sizeof(R) == 4) ? (const R*)h.lamf : (const R*)h.lam;
  const R* ilam = (sizeof(R) == 4) ? (const R*)h.ilamf : (const R*)h.ilam;
  const C* tw = (sizeof(R) == 4) ? (const C*)h.twf : (const C*)h.tw;

  const double nsp = (double)h.K * nx * sizeof(C);   // half spectrum, bins 0..nt/2
  const double nv = (double)nx * N;
  if (mr) {
    ProfScope ps(AAO_K_FFT_FWD, h.stream, nv * (vf ? sizeof(float) : sizeof(double)) + nsp);
    if (vf && sizeof(R) == 4) {
      AAO_TRY(ensure_smem((const void*)k_fft_fwd_mr<R, float>, smem));
      AAO_TRY_CUDA(launch_pdl(k_fft_fwd_mr<R, float>, grid, threads, smem, h.stream, vf, spec, nx, N, h.mr, lp,
                              h.pitch, lam, tw, in_scale));
    } else {
      AAO_TRY(ensure_smem((const void*)k_fft_fwd_mr<R, double>, smem));
      AAO_TRY_CUDA(launch_pdl(k_fft_fwd_mr<R, double>, grid, threads, smem, h.stream, v, spec, nx, N, h.mr, lp,
                              h.pitch, lam, tw, in_scale));
    }
  } else if (vf && sizeof(R) == 4) {
    // the FP32 copy of v written by the kernel that produced v
    AAO_TRY(ensure_smem((const void*)k_fft_fwd<R, float>, smem));
    ProfScope ps(AAO_K_FFT_FWD, h.stream, nv * sizeof(float) + nsp);
    AAO_TRY_CUDA(launch_pdl(k_fft_fwd<R, float>, grid, threads, smem, h.stream, vf, spec, nx, N, h.log2n, P, h.pitch,
                            lam, tw, in_scale));
  } else {
    AAO_TRY(ensure_smem((const void*)k_fft_fwd<R, double>, smem));
    ProfScope ps(AAO_K_FFT_FWD, h.stream, nv * sizeof(double) + nsp);
    AAO_TRY_CUDA(launch_pdl(k_fft_fwd<R, double>, grid, threads, smem, h.stream, v, spec, nx, N, h.log2n, P, h.pitch,
                            lam, tw, in_scale));
  }
  AAO_CHECK_LAUNCH();

  C* spec_b = spec;  // where step (b) leaves its result for step (c)
  TriRc rc;
  // Step (c) by the register tiles follows the recomputing tridiagonal kernel without programmatic
  // dependent launch: scheduled early, the inverse transform's CTAs cost that kernel more than the
  // overlap saves (1.17 against 1.10 ms per 2047 x 2048 mixed solve). After the factored kernel, and
  // for the mixed-radix tiles after either, the overlap pays.
  bool pdl_c = true;
  if (skip_b) {
    // timing of steps (a) and (c) alone
  } else if (op_2d(h.p.op)) {
    // step (b) with the two-dimensional operator: block elimination over the v levels
    AAO_TRY(heston_solve_bins(h, spec));
  } else if (h.p.op == AAO_OP_RIESZ) {
    // step (b) with the dense Toeplitz operator: the inverses of the shifted matrices (with
    // drift) or the eigendecomposition (symmetric), both made by aao_create
    void* res = nullptr;
    AAO_TRY(riesz_solve_bins(h, spec, &res));
    spec_b = reinterpret_cast<C*>(res);
  } else if (h.tri_rc && tri_rc_layout(h, sizeof(R), rc)) {
    // step (b): partition method with every pivot recomputed from the shared diagonals (no
    // per-bin tables), G bins of 2^lgT threads per CTA
    const C* mu = (sizeof(R) == 4) ? (const C*)h.muf : (const C*)h.mu;
    const C* il2 = (sizeof(R) == 4) ? (const C*)h.il2f : (const C*)h.il2;
    ProfScope ps(AAO_K_TRIDIAG, h.stream, 2.0 * nsp);
    AAO_TRY(launch_tri_rc<R>(h, rc, spec, mu, il2));
    pdl_c = false;
  } else if (TriPart tp; h.tri_fp && tri_part_layout(h, sizeof(R), tp)) {
    // step (b): partition method with the per-bin factors built with the handle, G bins of
    // tri_T = 2^lgT threads per CTA
    const int ch = h.tri_ch;
    const C* il2 = (sizeof(R) == 4) ? (const C*)h.il2f : (const C*)h.il2;
    const R* tri = reinterpret_cast<const R*>(h.tri);
    const C* fp = reinterpret_cast<const C*>(h.tri_fp);
    const C* fv = reinterpret_cast<const C*>(h.tri_fv);
    const C* fpcr = reinterpret_cast<const C*>(h.tri_fpcr);
    const int T = h.tri_T;
    // right-hand side in and out, the pivots and the fill-in (the multipliers are ~T/ch smaller)
    ProfScope ps(AAO_K_TRIDIAG, h.stream, 2.0 * nsp + 2.0 * (double)h.K * T * ch * sizeof(C));
    if (tp.staged) {
      AAO_TRY(ensure_smem((const void*)k_tridiag_part<R, true>, tp.smem));
      AAO_TRY_CUDA(launch_pdl(k_tridiag_part<R, true>, (h.K + tp.G - 1) / tp.G, tp.G * T, tp.smem, h.stream, spec,
                              nx, h.K, h.pitch, ch, tp.cs, tp.lgT, tri, fp, fv, fpcr, il2));
    } else {
      AAO_TRY(ensure_smem((const void*)k_tridiag_part<R, false>, tp.smem));
      AAO_TRY_CUDA(launch_pdl(k_tridiag_part<R, false>, (h.K + tp.G - 1) / tp.G, tp.G * T, tp.smem, h.stream, spec,
                              nx, h.K, h.pitch, ch, tp.cs, tp.lgT, tri, fp, fv, fpcr, il2));
    }
  } else {
  // step (b): threads per bin T (multiple of 32, <= 512), chunk ch <= CH rows per thread
  constexpr int CH = sizeof(R) == 4 ? 16 : 8;
  int T = 32 * ((nx + 32 * CH - 1) / (32 * CH));
  if (T > 512) {
    set_error("precond_apply: nx too large for the tridiagonal solver");
    return AAO_EUNSUPPORTED;
  }
  int ch = (nx + T - 1) / T;
  if (ch < 2) ch = 2;
  const int cs = (ch & 1) ? ch + 2 : ch + 1;  // odd chunk stride: conflict-free shared memory
  const size_t gbytes = ((size_t)T * cs + 8 * (size_t)T) * sizeof(C);
  const size_t cbytes = ((3 * (size_t)T * cs * sizeof(R)) + 15) & ~(size_t)15;
  int G = (int)((96 * 1024 - cbytes) / gbytes);  // bins per CTA sharing the staged diagonals
  if (G > 512 / T) G = 512 / T;
  if (G > 4) G = 4;
  if (G < 1) G = 1;
  const size_t smem2 = cbytes + G * gbytes;
  const R* lo = (sizeof(R) == 4) ? (const R*)h.pLf : (const R*)h.pL;
  const R* di = (sizeof(R) == 4) ? (const R*)h.pDf : (const R*)h.pD;
  const R* up = (sizeof(R) == 4) ? (const R*)h.pUf : (const R*)h.pU;
  const C* mu = (sizeof(R) == 4) ? (const C*)h.muf : (const C*)h.mu;
  const C* il2 = (sizeof(R) == 4) ? (const C*)h.il2f : (const C*)h.il2;
  AAO_TRY(ensure_smem((const void*)k_tridiag<R, CH>, smem2));
  {
    ProfScope ps(AAO_K_TRIDIAG, h.stream, 2.0 * nsp);
    AAO_TRY_CUDA(launch_pdl(k_tridiag<R, CH>, (h.K + G - 1) / G, G * T, smem2, h.stream, spec, nx, h.K, h.pitch, ch,
                            cs, T, lo, di, up, mu, il2));
  }
  }  // tridiagonal operators
  AAO_CHECK_LAUNCH();

  if (mr) {
    ProfScope ps(AAO_K_FFT_INV, h.stream, nsp + nv * (z_is_float ? sizeof(float) : sizeof(double)));
    if (z_is_float) {
      AAO_TRY(ensure_smem((const void*)k_fft_inv_mr<R, float>, smem));
      AAO_TRY_CUDA(launch_maybe_pdl(true, k_fft_inv_mr<R, float>, grid, threads, smem, h.stream, spec_b, (float*)z, nx, N, h.mr,
                              lp, h.pitch, ilam, tw));
    } else {
      AAO_TRY(ensure_smem((const void*)k_fft_inv_mr<R, double>, smem));
      AAO_TRY_CUDA(launch_maybe_pdl(true, k_fft_inv_mr<R, double>, grid, threads, smem, h.stream, spec_b, (double*)z, nx, N, h.mr,
                              lp, h.pitch, ilam, tw));
    }
  } else if (z_is_float) {
    AAO_TRY(ensure_smem((const void*)k_fft_inv<R, float>, smem));
    ProfScope ps(AAO_K_FFT_INV, h.stream, nsp + nv * sizeof(float));
    AAO_TRY_CUDA(launch_maybe_pdl(pdl_c, k_fft_inv<R, float>, grid, threads, smem, h.stream, spec_b, (float*)z, nx, N, h.log2n, P,
                            h.pitch, ilam, tw));
  } else {
    AAO_TRY(ensure_smem((const void*)k_fft_inv<R, double>, smem));
    ProfScope ps(AAO_K_FFT_INV, h.stream, nsp + nv * sizeof(double));
    AAO_TRY_CUDA(launch_maybe_pdl(pdl_c, k_fft_inv<R, double>, grid, threads, smem, h.stream, spec_b, (double*)z, nx, N, h.log2n, P,
                            h.pitch, ilam, tw));
  }
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

}  // namespace

AAO_CHECK_WORD_FN(check_word_precond)

int launch_precond(Handle& h, const double* v, void* z, bool z_is_float, const double* in_scale, const float* vf) {
  if (h.mixed) return run_precond<float>(h, v, z, z_is_float, in_scale, vf);
  return run_precond<double>(h, v, z, z_is_float, in_scale, nullptr);
}

int build_tri_factors(Handle& h) {
  if (h.p.flags == AAO_FLAG_STEPB_RECOMPUTE) return AAO_OK;  // the recomputing solver needs none
  const size_t rsize = h.mixed ? sizeof(float) : sizeof(double);
  TriPart tp;
  if (!tri_part_layout(h, rsize, tp)) return AAO_OK;  // the per-bin fallback solver needs none
  return h.mixed ? tri_factors_t<float>(h, tp.lgT) : tri_factors_t<double>(h, tp.lgT);
}

// Tuning results per (device, nx, nt, precision, operator class, flags): a second handle of the
// same shape skips the timing (and, when the recomputing step (b) won, the factor tables).
struct TuneKey {
  int dev, nx, nt, mixed, riesz, flags;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, nx, nt, mixed, riesz, flags) < std::tie(o.dev, o.nx, o.nt, o.mixed, o.riesz, o.flags);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, bool>> g_tune;  // -> (fft_p, tri_rc)

// FFT tile autotuner: time the apply for every admissible tile width 2P (P = 1, 2, 4, ...) on this
// problem's sizes and keep the fastest: the whole apply for the tridiagonal operators, steps (a)
// and (c) alone for the dense ones (their step (b) is the same for every tile and would take most
// of the tuning time). Every tile width computes identical results (each column's transform runs
// the same operations in the same order); only speed differs.
int tune_precond(Handle& h) {
  const size_t rs = h.mixed ? 4 : 8;
  int dev = 0;
  AAO_TRY_CUDA(cudaGetDevice(&dev));
  // the operators whose step (b) is not the tridiagonal solver
  const bool riesz = h.p.op == AAO_OP_RIESZ || op_2d(h.p.op);
  const int opclass = op_2d(h.p.op) ? 3 : (h.p.op == AAO_OP_RIESZ ? (h.rz_sym ? 2 : 1) : 0);
  const TuneKey key{dev, h.nx, h.nt, h.mixed ? 1 : 0, opclass, h.p.flags};
  TriRc trc;
  TriPart tpart;
  const bool rc_fits = !riesz && tri_rc_layout(h, rs, trc);
  const bool fact_fits = !riesz && tri_part_layout(h, rs, tpart);
  if (!riesz) {
    if (h.p.flags == AAO_FLAG_STEPB_FACTORED && !fact_fits) {
      set_error("aao_create: the factored step (b) does not fit this nx; use AAO_FLAG_STEPB_RECOMPUTE or 0");
      return AAO_EUNSUPPORTED;
    }
    if (h.p.flags == AAO_FLAG_STEPB_RECOMPUTE && !rc_fits) {
      set_error("aao_create: the recomputing step (b) does not fit this nx");
      return AAO_EUNSUPPORTED;
    }
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      h.fft_p = it->second.first;
      h.tri_rc = it->second.second;
      if (!riesz && !h.tri_rc) return build_tri_factors(h);
      return AAO_OK;
    }
  }
  if (!riesz) {
    // the default: in mixed precision with nt a power of two the recomputing solver wherever it
    // fits (no tables; 1.092 against 1.105 ms per 2047 x 2048 solve); otherwise the factored one
    // (FP64: the recomputing solver pays FP64 divisions; mixed radix: 1.075 against 1.053 ms per
    // 2047 x 1536 solve). The per-bin tables of the factored solver are built only where it is
    // wanted and fits; without them the recomputing solver is the one.
    const bool want_rc = h.p.flags == AAO_FLAG_STEPB_RECOMPUTE ||
                         (h.p.flags == 0 && h.mixed && h.mr.nst == 0 && rc_fits);
    if (!want_rc) AAO_TRY(build_tri_factors(h));
    if (want_rc || (!h.tri_fp && rc_fits)) h.tri_rc = true;
  }
  auto remember = [&]() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = {h.fft_p, h.tri_rc};
  };
  const int pmax = h.mr.nst > 0 ? mr_max_tile(h.nt, 2 * rs) : max_tile(h.nt, rs);
  if (pmax == 1) {
    h.fft_p = 1;
    remember();
    return AAO_OK;
  }
  double *v = nullptr, *z = nullptr;
  AAO_TRY_CUDA(cudaMalloc(&v, sizeof(double) * h.n));
  AAO_TRY_CUDA(cudaMalloc(&z, sizeof(double) * h.n));
  AAO_TRY_CUDA(cudaMemsetAsync(v, 0, sizeof(double) * h.n, h.stream));
  cudaEvent_t e0, e1;
  AAO_TRY_CUDA(cudaEventCreate(&e0));
  AAO_TRY_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int bestp = h.mr.nst > 0 ? pmax : default_tile(h.nx, h.nt, rs);
  int rc = AAO_OK;
  // time the form the solver runs: mixed solves read an FP32 copy of the input (the zero bytes of
  // v serve as one)
  const float* vf = (h.mixed && !riesz) ? reinterpret_cast<const float*>(v) : nullptr;
  // widths: the powers of two up to pmax and, for the register FFT (nt >= 128, any width), the
  // widths whose tile count just fills the SMs once or twice (ceil(pairs / (k SMs))), so that no
  // SM is left without a tile
  std::vector<int> cand;
  for (int P = 1; P <= pmax; P <<= 1) cand.push_back(P);
  if (h.mr.nst == 0 && h.nt >= (1 << kRegFftMinLog2) && h.sms > 0) {
    const int pairs = (h.nx + 1) / 2;
    for (int k = 1; k <= 2; ++k) {
      const int P = (pairs + k * h.sms - 1) / (k * h.sms);
      if (P > 1 && P <= pmax && (P & (P - 1)) != 0) cand.push_back(P);
    }
  }
  // each width: one warm-up apply, then the fastest of five timed applies (robust to a slow rep)
  for (size_t ci = 0; ci < cand.size() && rc == AAO_OK; ++ci) {
    const int P = cand[ci];
    h.fft_p = P;
    auto apply = [&]() -> int {
      if (!riesz) return launch_precond(h, v, z, h.mixed, nullptr, vf);
      if (h.mixed) return run_precond<float>(h, v, z, h.mixed, nullptr, vf, true);
      return run_precond<double>(h, v, z, h.mixed, nullptr, nullptr, true);
    };
    rc = apply();
    float pbest = 1e30f;
    for (int r = 0; r < 5 && rc == AAO_OK; ++r) {
      cudaEventRecord(e0, h.stream);
      rc = apply();
      cudaEventRecord(e1, h.stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < pbest) pbest = ms;
    }
    if (rc != AAO_OK) break;
    if (pbest < best) { best = pbest; bestp = P; }
  }
  h.fft_p = bestp;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(v);
  cudaFree(z);
  if (rc == AAO_OK) remember();
  return rc;
}

}  // namespace aao

// Operator, right-hand side and FGMRES(m) for the CN all-at-once system on GB300.
//
//   k_build_coef  (1/2) tau A(t_{k+1/2}) for Black-Scholes (constant or local volatility),
//                 3-point central differences on S_i = i h; FP64. The diagonal is stored as
//                 1 + (1/2) tau a_ii (the matvec's form y_t = 2 x_t - (I + A~_t/2)(x_t + x_{t-1})).
//   k_rhs         b = xi + tau f (Eq. 2.2).
//   k_matvec      y = M x, block-bidiagonal M = B1 (x) I - B2 (x) A~ (Eq. 2.2; Eq. 5.8 form for
//                 time-dependent A): y_t = (x_t - x_{t-1}) - (1/2) A~_t (x_t + x_{t-1}), FP64;
//                 fused with the residual norm or with the first Gram-Schmidt projections.
//   k_update / k_mdot / k_xupdate / k_dot_self
//                 right-preconditioned flexible GMRES(m) (Sec. 5), FP64.
//
// FP64 is 1/64 of the FP32 rate on this part, so the Arnoldi process is arranged to issue as
// few FP64 instructions as possible:
//  * the Krylov basis is stored unnormalised (raw vectors V_i with scales sigma_i = 1/||V_i||);
//    the preconditioner reads sigma_j V_j (the scale is folded into its first kernel) and every
//    other normalisation into the Hessenberg scalars, so no pass rescales vectors;
//  * classical Gram-Schmidt runs once; a second pass (CGS2) runs only when cancellation
//    ||w'|| < kReorthEta ||w|| would lose more than ~1e-11 of orthogonality;
//  * block partial sums are finished by the last block of the producing kernel, in a fixed
//    order (deterministic), and the Givens update runs in that block as well;
//  * FP32 values are widened to FP64 by integer bit assembly, off the FP64 pipe.
#include <math.h>
#include <stdio.h>

#include <chrono>
#include <complex>
#include <map>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "krylov_dev.cuh"

namespace aao {

namespace {

using namespace kdev;

// After every block wrote its partial sums: true in the block that finishes last.
__device__ __forceinline__ bool last_block(unsigned int* counter, unsigned int nblocks) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = atomicAdd(counter, 1u) == nblocks - 1;
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}


__global__ void k_build_coef(double* __restrict__ L, double* __restrict__ D, double* __restrict__ U, int nx,
                             int rows, double h, double half_tau, double sigma, double r, double bump,
                             double tslope, double tau, const double* __restrict__ gS) {
  const size_t n = (size_t)nx * rows;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / nx), i = (int)(e - (size_t)k * nx);
    const double S = h * (double)(i + 1);
    double sig = sigma;
    if (bump != 0.0) {
      const double tm = tau * ((double)k + 0.5);
      sig = sigma + bump * gS[i] * (1.0 + tslope * tm);
    }
    const double diff = 0.5 * sig * sig * S * S / (h * h);
    const double conv = 0.5 * r * S / h;
    L[e] = half_tau * (diff - conv);
    D[e] = 1.0 + half_tau * (-2.0 * diff - r);  // diagonal of I + (1/2) tau A
    U[e] = half_tau * (diff + conv);
  }
}

__global__ void k_rhs(double* __restrict__ b, int nx, int nt, const double* __restrict__ L,
                      const double* __restrict__ D, const double* __restrict__ U, int rows,
                      const double* __restrict__ gL, const double* __restrict__ gR, double h, double K,
                      int payoff) {
  const size_t n = (size_t)nx * nt;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int t = (int)(e / nx), i = (int)(e - (size_t)t * nx);
    const size_t c0 = (rows == 1) ? 0 : (size_t)t * nx;
    double val = 0.0;
    // tau f^{t+1/2}: Dirichlet data averaged over t_t and t_{t+1}; (1/2) tau a enters twice
    if (i == 0) val += L[c0] * (gL[t] + gL[t + 1]);
    if (i == nx - 1) val += U[c0 + nx - 1] * (gR[t] + gR[t + 1]);
    if (t == 0) {
      auto u0 = [&](int j) {
        const double S = h * (double)(j + 1);
        return payoff == AAO_PUT ? fmax(K - S, 0.0) : fmax(S - K, 0.0);
      };
      double xi = D[i] * u0(i);  // D holds the diagonal of I + (1/2) tau A
      if (i > 0) xi += L[i] * u0(i - 1);
      if (i < nx - 1) xi += U[i] * u0(i + 1);
      val += xi;
    }
    b[e] = val;
  }
}

// y = M x over strips of kMvCols columns (one warp item each, with a halo column per side) and all
// time levels.
// MODE 0: y = M x.
// MODE 1: y = b - M x (the restart residual, written as the raw first basis vector); the last
//         block sets ||r||^2, sigma_0 = 1/||r|| and g = (||r||, 0, ...). MODE 3: MODE 1 and ||b||^2.
// MODE 2: y = M x and the first Gram-Schmidt projections d_q = V_q . y (q < nd <= 8),
//         finished by the last block into scal[S_D1 + q]. (||w||^2 is not formed: the update
//         kernel recovers it as ||w'||^2 + sum_q sigma_q^2 d_q^2.)
template <typename IN, int MODE, int ND>
__global__ void __launch_bounds__(kThreads) k_matvec(const IN* __restrict__ x, double* __restrict__ y,
                                                     const double* __restrict__ b, int nx, int nt,
                                                     const double* __restrict__ L, const double* __restrict__ D,
                                                     const double* __restrict__ U, int rows,
                                                     const double* __restrict__ V, size_t vstride,
                                                     double* __restrict__ part, double* __restrict__ scal,
                                                     unsigned int* __restrict__ counter, int m,
                                                     float* __restrict__ yf) {
  pdl_sync();
  constexpr int NA = MODE == 2 ? ND : (MODE == 3 ? 2 : 1);
  constexpr int nd = ND;
  // one wave of blocks: the (strip, time level) rows, strip-major, are split into one contiguous
  // range per warp, so every warp does the same work to within one row and keeps level t-1 in
  // registers along its range
  const int strips = (nx + kMvCols - 1) / kMvCols;
  const long long R = (long long)strips * nt;
  const long long W = (long long)gridDim.x * (kThreads / 32);
  const long long w = (long long)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  long long r = w * R / W;
  const long long r1 = (w + 1) * R / W;
  double acc[NA];
#pragma unroll
  for (int q = 0; q < NA; ++q) acc[q] = 0.0;
  while (r < r1) {
    const int strip = (int)(r / nt);
    const int t0 = (int)(r - (long long)strip * nt);
    const int t1 = (int)((long long)t0 + (r1 - r) < (long long)nt ? (long long)t0 + (r1 - r) : (long long)nt);
    if (!AAO_DCHECK(t0 >= 0 && t1 <= nt && strip * kMvCols < nx)) break;
    matvec_item<IN, MODE, ND, NA>(x, y, b, nx, t0, t1, strip * kMvCols, L, D, U, rows, V, vstride, acc, yf);
    r += t1 - t0;
  }
  if constexpr (MODE == 0) return;
  const unsigned int nblk = gridDim.x;
  const unsigned int bid = blockIdx.x;
  if constexpr (MODE == 2) {
    block_sums_wide<NA>(acc, nd, part + (size_t)bid * kPartLd);
  } else {
    block_sums_wide<NA>(acc, NA, part + (size_t)bid * kPartLd);
  }
  if (!last_block(counter, nblk)) return;
  if constexpr (MODE == 2) {
    finish_sums_wide<NA>(part, nblk, nd, [&](int q, double v) { scal[S_D1 + q] = v; }, counter);
  } else {
    finish_sums_wide<NA>(part, nblk, NA, [&](int q, double v) {
      if (q == 1) {
        scal[S_BNORM2] = v;
        return;
      }
      scal[S_BETA2] = v;
      const double beta = sqrt(v);
      scal[S_SIG] = beta > 0.0 ? 1.0 / beta : 0.0;
      scal[S_G] = beta;
      for (int k = 1; k <= m; ++k) scal[S_G + k] = 0.0;
      scal[S_FLAG] = isfinite(v) ? 0.0 : 1.0;
    }, counter);
  }
}

// out[c0 + q] = V_{c0+q} . w for q < NV (chunk of <= 8 basis vectors), finished by the last block
template <int NV>
__global__ void __launch_bounds__(kThreads) k_mdot(const double* __restrict__ V, int c0, size_t n,
                                                   const double* __restrict__ w, double* __restrict__ part,
                                                   double* __restrict__ out, unsigned int* __restrict__ counter) {
  pdl_sync();
  constexpr int nv = NV;
  double acc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = 0.0;
  const double* Vc = V + (size_t)c0 * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double wv = __ldg(w + e);
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = fma(__ldg(Vc + (size_t)q * n + e), wv, acc[q]);
  }
  block_sums_wide<NV>(acc, nv, part + (size_t)blockIdx.x * kPartLd);
  if (!last_block(counter, gridDim.x)) return;
  finish_sums_wide<NV>(part, gridDim.x, nv, [&](int q, double v) { out[c0 + q] = v; }, counter);
}

// Gram-Schmidt pass `pass` (1 or 2) on w (the raw vector V_{j+1}, updated in place):
//   w <- w - sum_{i<=j} sigma_i^2 d_i V_i,  d = scal[S_D1] (pass 1) or scal[S_D2] (pass 2),
// then ||w||^2 -> scal[S_WP2]. The last block decides: after pass 1 a second pass is requested
// (scal[S_REORTH] = 1) when ||w'||^2 < eta^2 ||w||^2; otherwise the Givens update of column j runs.
template <int NV>
__global__ void __launch_bounds__(kThreads) k_update(double* __restrict__ w, const double* __restrict__ V,
                                                     int j, size_t n, int pass, double* __restrict__ scal,
                                                     double* __restrict__ part, unsigned int* __restrict__ counter,
                                                     float* __restrict__ vf) {
  pdl_sync();
  // every scalar the kernel needs, the last block's tail included, is staged at the start, while
  // the loads are cheap; the tail then works out of shared memory
  __shared__ double cf[kLdH], sh_h[kLdH + 1], sh_cs[kLdH], sh_sn[kLdH], sh_g;
  const int nv = j + 1;
  const int off = pass == 1 ? S_D1 : S_D2;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    const double si = scal[S_SIG + i], di = scal[off + i];
    cf[i] = si * si * di;
    // column j of H before the rotations: sigma_i (d1_i + d2_i)
    sh_h[i] = si * (pass == 2 ? scal[S_D1 + i] + di : di);
    if (i < j) {
      sh_cs[i] = scal[S_CS + i];
      sh_sn[i] = scal[S_SN + i];
    }
  }
  if (threadIdx.x == 0) sh_g = scal[S_G + j];
  __syncthreads();
  double acc[1] = {0.0};
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if constexpr (NV > 0) {
    // two elements per step: all loads of both are issued before either is combined
    for (; e + stride < n; e += 2 * stride) {
      double wa = w[e], wb = w[e + stride], va[NV], vb[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        va[q] = __ldg(V + (size_t)q * n + e);
        vb[q] = __ldg(V + (size_t)q * n + e + stride);
      }
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        wa = fma(-cf[q], va[q], wa);
        wb = fma(-cf[q], vb[q], wb);
      }
      w[e] = wa;
      w[e + stride] = wb;
      if (vf) {
        vf[e] = narrow(wa);
        vf[e + stride] = narrow(wb);
      }
      acc[0] = fma(wa, wa, acc[0]);
      acc[0] = fma(wb, wb, acc[0]);
    }
  }
  for (; e < n; e += stride) {
    double wv = w[e];
    if constexpr (NV > 0) {
#pragma unroll
      for (int q = 0; q < NV; ++q) wv = fma(-cf[q], __ldg(V + (size_t)q * n + e), wv);
    } else {
      for (int q = 0; q < nv; ++q) wv = fma(-cf[q], __ldg(V + (size_t)q * n + e), wv);
    }
    w[e] = wv;
    if (vf) vf[e] = narrow(wv);
    acc[0] = fma(wv, wv, acc[0]);
  }
  block_sums_wide<1>(acc, 1, part + (size_t)blockIdx.x * kPartLd);
  if (!last_block(counter, gridDim.x)) return;
  __shared__ double wp2;
  finish_sums_wide<1>(part, gridDim.x, 1, [&](int, double v) {
    scal[S_WP2] = v;
    wp2 = v;
  }, counter);
  __syncthreads();
  // ||w||^2 = ||w'||^2 + sum_i sigma_i^2 d_i^2 (Pythagoras over the orthonormal basis; a sum of
  // positive terms, so no cancellation), compared with ||w'||^2 for the second-pass decision
  if (pass == 1) {
    double wn2 = wp2;
    for (int i = 0; i < nv; ++i) wn2 = fma(sh_h[i], sh_h[i], wn2);
    if (wp2 < kReorthEta * kReorthEta * wn2) {
      if (threadIdx.x == 0) scal[S_REORTH] = 1.0;
      return;
    }
  }
  if (threadIdx.x != 0) return;
  scal[S_REORTH] = 0.0;
  givens_column_staged(scal, j, wp2, sh_h, sh_cs, sh_sn, sh_g);
}

// x += sum_{i<jd} y_i Z_i with y = H(0:jd,0:jd)^{-1} g(0:jd) (each block solves the small
// triangular system itself); Z_i = P^{-1} v_i for the normalised basis vectors v_i
template <typename ZT>
__global__ void __launch_bounds__(kThreads) k_xupdate(double* __restrict__ x, const ZT* __restrict__ Z, int jd,
                                                      size_t n, const double* __restrict__ scal, int fresh) {
  pdl_sync();
  __shared__ double ys[128];
  if (threadIdx.x == 0) {
    for (int i = jd - 1; i >= 0; --i) {
      double s = scal[S_G + i];
      for (int k = i + 1; k < jd; ++k) s -= scal[S_HMAT + (size_t)k * kLdH + i] * ys[k];
      ys[i] = s / scal[S_HMAT + (size_t)i * kLdH + i];
    }
  }
  __syncthreads();
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  // two elements per step, loads first
  for (; e + stride < n; e += 2 * stride) {
    double va = fresh ? 0.0 : x[e], vb = fresh ? 0.0 : x[e + stride];
    int i = 0;
    for (; i + 2 <= jd; i += 2) {
      const double z0 = ld(Z + (size_t)i * n + e), z1 = ld(Z + (size_t)(i + 1) * n + e);
      const double z2 = ld(Z + (size_t)i * n + e + stride), z3 = ld(Z + (size_t)(i + 1) * n + e + stride);
      va = fma(ys[i], z0, va);
      vb = fma(ys[i], z2, vb);
      va = fma(ys[i + 1], z1, va);
      vb = fma(ys[i + 1], z3, vb);
    }
    if (i < jd) {
      va = fma(ys[i], ld(Z + (size_t)i * n + e), va);
      vb = fma(ys[i], ld(Z + (size_t)i * n + e + stride), vb);
    }
    x[e] = va;
    x[e + stride] = vb;
  }
  for (; e < n; e += stride) {
    double v = fresh ? 0.0 : x[e];
    for (int i = 0; i < jd; ++i) v = fma(ys[i], ld(Z + (size_t)i * n + e), v);
    x[e] = v;
  }
}

// The first restart residual from the zero initial guess, r = b: V_0 <- b (and its FP32 copy vf
// when the preconditioner reads one), ||b||^2 into both BETA2 and BNORM2, and sigma_0 = 1/beta,
// g = (beta, 0, ..., 0) and the finiteness flag as the residual matvec sets them.
__global__ void __launch_bounds__(kThreads) k_first_zero(const double* __restrict__ b, double* __restrict__ V0,
                                                         float* __restrict__ vf, size_t n, double* part,
                                                         double* __restrict__ scal, unsigned int* __restrict__ counter,
                                                         int m) {
  pdl_sync();
  double acc[1] = {0.0};
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double a = __ldg(b + e);
    if (AAO_DCHECK(e < n)) V0[e] = a;
    if (vf) vf[e] = narrow(a);
    acc[0] = fma(a, a, acc[0]);
  }
  block_sums_wide<1>(acc, 1, part + (size_t)blockIdx.x * kPartLd);
  if (!last_block(counter, gridDim.x)) return;
  finish_sums_wide<1>(part, gridDim.x, 1, [&](int, double v) {
    scal[S_BETA2] = v;
    scal[S_BNORM2] = v;
    const double beta = sqrt(v);
    scal[S_SIG] = beta > 0.0 ? 1.0 / beta : 0.0;
    scal[S_G] = beta;
    for (int k = 1; k <= m; ++k) scal[S_G + k] = 0.0;
    scal[S_FLAG] = isfinite(v) ? 0.0 : 1.0;
  }, counter);
}

// scal[slot] = v . v
__global__ void __launch_bounds__(kThreads) k_dot_self(const double* __restrict__ v, size_t n, double* part,
                                                       double* __restrict__ scal, int slot,
                                                       unsigned int* __restrict__ counter) {
  pdl_sync();
  double acc[1] = {0.0};
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double a = __ldg(v + e);
    acc[0] = fma(a, a, acc[0]);
  }
  block_sums_wide<1>(acc, 1, part + (size_t)blockIdx.x * kPartLd);
  if (!last_block(counter, gridDim.x)) return;
  finish_sums_wide<1>(part, gridDim.x, 1, [&](int, double s) { scal[slot] = s; }, counter);
}

int grid_for(size_t n) {
  size_t g = (n + kThreads - 1) / kThreads;
  return (int)(g < (size_t)kRedBlocks ? g : (size_t)kRedBlocks);
}

// Blocks of kThreads threads that are resident at once on h's device (one full wave, so that no
// partial second wave idles most SMs), at most `need` and at most kPartBlocks.
int wave_blocks(const Handle& h, const void* kernel, size_t need) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> occ;  // per (device, kernel)
  int o = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = occ.find({dev, kernel});
    if (it == occ.end()) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel, kThreads, 0) != cudaSuccess || o < 1) o = 1;
      occ[{dev, kernel}] = o;
    } else {
      o = it->second;
    }
  }
  size_t g = (size_t)o * (size_t)(h.sms > 0 ? h.sms : 1);
  if (g > need) g = need;
  if (g > (size_t)kPartBlocks) g = kPartBlocks;
  return (int)(g > 0 ? g : 1);
}

int ensure_workspace(Handle& h, int m) {
  if (h.ws_m >= m && h.V) return AAO_OK;
  if (h.V) cudaFree(h.V);
  if (h.Z) cudaFree(h.Z);
  if (h.Vf) cudaFree(h.Vf);
  h.V = nullptr; h.Z = nullptr; h.Vf = nullptr; h.ws_m = 0;
  AAO_TRY_CUDA(cudaMalloc(&h.V, sizeof(double) * h.n * (size_t)(m + 1)));
  AAO_TRY_CUDA(cudaMalloc(&h.Z, (h.mixed ? sizeof(float) : sizeof(double)) * h.n * (size_t)m));
  if (h.mixed) AAO_TRY_CUDA(cudaMalloc(&h.Vf, sizeof(float) * h.n));
  h.ws_m = m;
  return AAO_OK;
}

}  // namespace

AAO_CHECK_WORD_FN(check_word_krylov)

// ----------------------------------------------------------------------------------------
// tables
// ----------------------------------------------------------------------------------------

int build_tables(Handle& h) {
  const aao_problem& p = h.p;
  const int nx = h.nx, nt = h.nt, N = nt;
  h.tau = p.T / nt;
  const bool riesz = p.op == AAO_OP_RIESZ, heston = op_2d(p.op);
  const bool tridiag = !riesz && !heston;  // the one-dimensional Black-Scholes operators
  const double hS = p.s_max / (nx + 1);
  h.coef_rows = (p.op == AAO_OP_LOCALVOL) ? nt : 1;
  const size_t ncoef = (size_t)nx * h.coef_rows;

  // matvec coefficients on the device
  std::vector<double> gS(nx, 0.0);
  const double bump = (p.op == AAO_OP_LOCALVOL) ? p.lv_bump : 0.0;
  for (int i = 0; i < nx; ++i) {
    const double S = hS * (i + 1);
    const double l = log(S / p.K);
    gS[i] = exp(-l * l);
  }
  double* d_gS = nullptr;
  if (tridiag) {
  AAO_TRY_CUDA(cudaMalloc(&h.mL, sizeof(double) * ncoef));
  AAO_TRY_CUDA(cudaMalloc(&h.mD, sizeof(double) * ncoef));
  AAO_TRY_CUDA(cudaMalloc(&h.mU, sizeof(double) * ncoef));
  AAO_TRY_CUDA(cudaMalloc(&d_gS, sizeof(double) * nx));
  AAO_TRY_CUDA(cudaMemcpyAsync(d_gS, gS.data(), sizeof(double) * nx, cudaMemcpyHostToDevice, h.stream));
  k_build_coef<<<grid_for(ncoef), kThreads, 0, h.stream>>>(h.mL, h.mD, h.mU, nx, h.coef_rows, hS, 0.5 * h.tau,
                                                            p.sigma, p.r, bump, p.lv_tslope, h.tau, d_gS);
  AAO_CHECK_LAUNCH();

  // Dirichlet values at t_0..t_nt (t = time to maturity)
  std::vector<double> gl(nt + 1), gr(nt + 1);
  for (int k = 0; k <= nt; ++k) {
    const double t = h.tau * k;
    const double disc = p.K * exp(-p.r * t);
    gl[k] = p.payoff == AAO_PUT ? disc : 0.0;
    gr[k] = p.payoff == AAO_PUT ? 0.0 : p.s_max - disc;
  }
  AAO_TRY_CUDA(cudaMalloc(&h.gL, sizeof(double) * (nt + 1)));
  AAO_TRY_CUDA(cudaMalloc(&h.gR, sizeof(double) * (nt + 1)));
  AAO_TRY_CUDA(cudaMemcpyAsync(h.gL, gl.data(), sizeof(double) * (nt + 1), cudaMemcpyHostToDevice, h.stream));
  AAO_TRY_CUDA(cudaMemcpyAsync(h.gR, gr.data(), sizeof(double) * (nt + 1), cudaMemcpyHostToDevice, h.stream));
  }  // tridiag

  // preconditioner operator tau * Abar: time mean of sigma^2 in closed form,
  // mean_k (s0 + b_i c_k)^2 = s0^2 + 2 s0 b_i mean(c) + b_i^2 mean(c^2)
  double cm = 0.0, c2m = 0.0;
  for (int k = 0; k < nt; ++k) {
    const double c = 1.0 + p.lv_tslope * h.tau * (k + 0.5);
    cm += c;
    c2m += c * c;
  }
  cm /= nt;
  c2m /= nt;
  std::vector<double> pl(nx), pd(nx), pu(nx);
  std::vector<float> plf(nx), pdf(nx), puf(nx);
  for (int i = 0; i < nx; ++i) {
    const double bi = bump * gS[i];
    const double s2 = p.sigma * p.sigma + 2.0 * p.sigma * bi * cm + bi * bi * c2m;
    const double ii = (double)(i + 1);
    const double diff = 0.5 * s2 * ii * ii, conv = 0.5 * p.r * ii;
    pl[i] = h.tau * (diff - conv);
    pd[i] = h.tau * (-2.0 * diff - p.r);
    pu[i] = h.tau * (diff + conv);
    plf[i] = (float)pl[i]; pdf[i] = (float)pd[i]; puf[i] = (float)pu[i];
  }
  // eigenvalues of the alpha-circulant blocks: with a = alpha^{1/nt} and the forward DFT
  // exp(-2 pi i t k / nt), lambda1_k = 1 - a w^k, lambda2_k = (1 + a w^k) / 2, w = exp(-2 pi i / nt)
  const int K = h.K;
  const double a = pow(p.alpha, 1.0 / N);
  std::vector<double2> mu(K), il2(K), tw(N);
  std::vector<float2> muf(K), il2f(K), twf(N);
  for (int k = 0; k < K; ++k) {
    const double ang = -2.0 * M_PI * (double)k / N;
    const std::complex<double> wk(cos(ang), sin(ang));
    const std::complex<double> l1 = 1.0 - a * wk, l2 = 0.5 * (1.0 + a * wk);
    const std::complex<double> m = l1 / l2, il = 1.0 / l2;
    mu[k] = make_double2(m.real(), m.imag());
    il2[k] = make_double2(il.real(), il.imag());
    muf[k] = make_float2((float)m.real(), (float)m.imag());
    il2f[k] = make_float2((float)il.real(), (float)il.imag());
  }
  for (int m = 0; m < N; ++m) {
    const double ang = -2.0 * M_PI * (double)m / N;
    tw[m] = make_double2(cos(ang), sin(ang));
    twf[m] = make_float2((float)cos(ang), (float)sin(ang));
  }
  std::vector<double> lam(N), ilam(N);
  std::vector<float> lamf(N), ilamf(N);
  for (int t = 0; t < N; ++t) {
    lam[t] = pow(p.alpha, (double)t / N);
    ilam[t] = 1.0 / (lam[t] * N);
    lamf[t] = (float)lam[t];
    ilamf[t] = (float)ilam[t];
  }
  auto up = [&](auto** dst, const auto& src) -> int {
    using T = typename std::decay<decltype(src)>::type::value_type;
    AAO_TRY_CUDA(cudaMalloc((void**)dst, sizeof(T) * src.size()));
    AAO_TRY_CUDA(cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, h.stream));
    return AAO_OK;
  };
  if (tridiag) {
    AAO_TRY(up(&h.pL, pl)); AAO_TRY(up(&h.pD, pd)); AAO_TRY(up(&h.pU, pu));
    AAO_TRY(up(&h.pLf, plf)); AAO_TRY(up(&h.pDf, pdf)); AAO_TRY(up(&h.pUf, puf));
    // step (b) partition: T = 2^k >= 32 threads per bin with at most 16 rows each (up to T = 512),
    // rows l*ch .. l*ch+ch-1 on thread l; the coefficients a_i = -lo_i (0 for i = 0), diag_i,
    // c_i = -up_i (0 for i = nx-1) stored [j][l]
    int T = 32;
    while (T < 512 && (nx + T - 1) / T > 16) T *= 2;
    const int ch = (nx + T - 1) / T;
    const size_t plane = (size_t)ch * T;
    std::vector<double> tri(3 * plane, 0.0);
    for (int l = 0; l < T; ++l)
      for (int j = 0; j < ch; ++j) {
        const int i = l * ch + j;
        const size_t o = (size_t)j * T + l;
        tri[o] = (i > 0 && i < nx) ? -pl[i] : 0.0;
        tri[plane + o] = i < nx ? pd[i] : 0.0;
        tri[2 * plane + o] = (i < nx - 1) ? -pu[i] : 0.0;
      }
    h.tri_T = T;
    h.tri_ch = ch;
    if (h.mixed) {
      std::vector<float> trif(tri.size());
      for (size_t q = 0; q < tri.size(); ++q) trif[q] = (float)tri[q];
      float* d = nullptr;
      AAO_TRY(up(&d, trif));
      h.tri = d;
    } else {
      double* d = nullptr;
      AAO_TRY(up(&d, tri));
      h.tri = d;
    }
  }
  AAO_TRY(up(&h.mu, mu)); AAO_TRY(up(&h.il2, il2)); AAO_TRY(up(&h.tw, tw));
  AAO_TRY(up(&h.muf, muf)); AAO_TRY(up(&h.il2f, il2f)); AAO_TRY(up(&h.twf, twf));
  AAO_TRY(up(&h.lam, lam)); AAO_TRY(up(&h.ilam, ilam));
  AAO_TRY(up(&h.lamf, lamf)); AAO_TRY(up(&h.ilamf, ilamf));

  const size_t csz = h.mixed ? sizeof(float2) : sizeof(double2);
  AAO_TRY_CUDA(cudaMalloc(&h.spec, csz * (size_t)K * h.pitch));
  AAO_TRY_CUDA(cudaMalloc(&h.w, sizeof(double) * h.n));
  AAO_TRY_CUDA(cudaMalloc(&h.scal, sizeof(double) * S_TOTAL));
  AAO_TRY_CUDA(cudaMemsetAsync(h.scal, 0, sizeof(double) * S_TOTAL, h.stream));
  AAO_TRY_CUDA(cudaMalloc(&h.counter, sizeof(unsigned int) * 4));
  AAO_TRY_CUDA(cudaMemsetAsync(h.counter, 0, sizeof(unsigned int) * 4, h.stream));
  h.part_blocks = kRedBlocks;
  {
    int dev = 0;
    AAO_TRY_CUDA(cudaGetDevice(&dev));
    AAO_TRY_CUDA(cudaDeviceGetAttribute(&h.sms, cudaDevAttrMultiProcessorCount, dev));
  }
  AAO_TRY_CUDA(cudaMalloc(&h.part, sizeof(double) * (size_t)kPartBlocks * kPartLd));
  AAO_TRY_CUDA(cudaMallocHost(&h.host_scal, sizeof(double) * 8));
  // the temporary gS buffer must outlive the build kernel
  AAO_TRY_CUDA(cudaStreamSynchronize(h.stream));
  if (d_gS) cudaFree(d_gS);
  if (riesz) AAO_TRY(riesz_build(h));
  if (heston) AAO_TRY(heston_build(h));
  return AAO_OK;
}

void free_handle(Handle& h) {
  void* bufs[] = {h.mL, h.mD, h.mU, h.gL, h.gR, h.pL, h.pD, h.pU, h.pLf, h.pDf, h.pUf, h.mu, h.il2, h.tw,
                  h.muf, h.il2f, h.twf, h.lam, h.ilam, h.lamf, h.ilamf, h.spec, h.V, h.Z, h.w, h.scal, h.part,
                  h.counter, h.rz_chat, h.rz_tw, h.rz_hcol, h.rz_hrow, h.rz_hcl, h.tri, h.Vf, h.tri_fp,
                  h.tri_fv, h.tri_fpcr, h.rz_dk, h.rz_w,
                  h.rz_part, h.rz_qh, h.rz_ql, h.rz_qth, h.rz_qtl, h.rz_bh, h.rz_bl, h.rz_err, h.rz_inv, h.hs_c, h.hs_tf,
                  h.hs_u0, h.hs_cf, h.hs_X, h.hs_G, h.hs_H};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (h.host_scal) cudaFreeHost(h.host_scal);
}

// ----------------------------------------------------------------------------------------
// operator launches
// ----------------------------------------------------------------------------------------

namespace {

// time-chunk length: enough blocks to fill the GPU, at most kPartBlocks partial sums
template <typename IN>
int matvec_t(Handle& h, const IN* x, double* y, const double* b, const double* V, int nd, int m, double bytes,
             double flops, bool with_bnorm, float* yf) {
  const size_t rowsw = (size_t)((h.nx + kMvCols - 1) / kMvCols) * h.nt;  // warp rows
  const size_t need = (rowsw + kThreads / 32 - 1) / (kThreads / 32);
  ProfScope ps(AAO_K_MATVEC, h.stream, bytes, flops);
#define AAO_MV2(ND)                                                                                              \
  AAO_TRY_CUDA(launch_pdl(k_matvec<IN, 2, ND>, wave_blocks(h, (const void*)k_matvec<IN, 2, ND>, need), kThreads, 0, \
                          h.stream, x, y, nullptr, h.nx, h.nt, h.mL, h.mD, h.mU, h.coef_rows, V, h.n, h.part,      \
                          h.scal, h.counter, m, nullptr))
  if (V && nd > 0) {
    switch (nd) {
      case 1: AAO_MV2(1); break;
      case 2: AAO_MV2(2); break;
      case 3: AAO_MV2(3); break;
      case 4: AAO_MV2(4); break;
      case 5: AAO_MV2(5); break;
      case 6: AAO_MV2(6); break;
      case 7: AAO_MV2(7); break;
      default: AAO_MV2(8); break;
    }
  } else if (b && with_bnorm) {
    AAO_TRY_CUDA(launch_pdl(k_matvec<IN, 3, 0>, wave_blocks(h, (const void*)k_matvec<IN, 3, 0>, need), kThreads, 0,
                            h.stream, x, y, b, h.nx, h.nt, h.mL, h.mD, h.mU, h.coef_rows, nullptr, h.n, h.part, h.scal,
                            h.counter, m, yf));
  } else if (b) {
    AAO_TRY_CUDA(launch_pdl(k_matvec<IN, 1, 0>, wave_blocks(h, (const void*)k_matvec<IN, 1, 0>, need), kThreads, 0,
                            h.stream, x, y, b, h.nx, h.nt, h.mL, h.mD, h.mU, h.coef_rows, nullptr, h.n, h.part, h.scal,
                            h.counter, m, yf));
  } else {
    AAO_TRY_CUDA(launch_pdl(k_matvec<IN, 0, 0>, wave_blocks(h, (const void*)k_matvec<IN, 0, 0>, need), kThreads, 0,
                            h.stream, x, y, nullptr, h.nx, h.nt, h.mL, h.mD, h.mU, h.coef_rows, nullptr, h.n, h.part,
                            h.scal, h.counter, m, nullptr));
  }
#undef AAO_MV2
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

}  // namespace

// y = M x; with b: y = b - M x (restart residual); with V (nd <= 8): first Gram-Schmidt pass
int launch_matvec(Handle& h, const void* x, bool x_is_float, double* y, const double* b, const double* V, int nd,
                  int m, bool with_bnorm, float* yf) {
  if (h.p.op == AAO_OP_RIESZ || op_2d(h.p.op)) {
    if (b && with_bnorm) {
      ProfScope ps(AAO_K_OTHER, h.stream, 8.0 * (double)h.n);
      k_dot_self<<<wave_blocks(h, (const void*)k_dot_self, grid_for(h.n)), kThreads, 0, h.stream>>>(
          b, h.n, h.part, h.scal, S_BNORM2, h.counter);
      AAO_CHECK_LAUNCH();
    }
    if (op_2d(h.p.op)) return heston_matvec(h, x, x_is_float, y, b, V, nd, m);
    return riesz_matvec(h, x, x_is_float, y, b, V, nd, m);
  }
  const double nn = (double)h.n;
  // x once, coefficients (3 per row of the time-dependent operator), y, b and V_q if present
  const double bytes = nn * (x_is_float ? 4.0 : 8.0) + 3.0 * 8.0 * (double)h.nx * h.coef_rows + nn * 8.0 +
                       (b ? nn * 8.0 : 0.0) + (V ? nn * 8.0 * nd : 0.0);
  // per unknown, as executed: s = x_t + x_{t-1} (1 add; 2 x_t is an exponent increment), three
  // FMAs; residual: b - 2 x_t (1) and r.r (FMA), b.b (FMA); projections: nd FMAs
  const double flops = nn * (1.0 + 6.0 + (b ? 3.0 : 0.0) + (b && with_bnorm ? 2.0 : 0.0) + (V ? 2.0 * nd : 0.0));
  if (x_is_float) return matvec_t<float>(h, (const float*)x, y, b, V, nd, m, bytes, flops, with_bnorm, yf);
  return matvec_t<double>(h, (const double*)x, y, b, V, nd, m, bytes, flops, with_bnorm, yf);
}

void launch_rhs_raw(cudaStream_t s, double* b, int nx, int nt, const double* L, const double* D, const double* U,
                    int rows, const double* gL, const double* gR, double h, double K, int payoff) {
  k_rhs<<<grid_for((size_t)nx * nt), kThreads, 0, s>>>(b, nx, nt, L, D, U, rows, gL, gR, h, K, payoff);
}

void launch_coef_raw(cudaStream_t s, double* L, double* D, double* U, int nx, int rows, double h, double half_tau,
                     double sigma, double r, double bump, double tslope, double tau, const double* gS) {
  k_build_coef<<<grid_for((size_t)nx * rows), kThreads, 0, s>>>(L, D, U, nx, rows, h, half_tau, sigma, r, bump,
                                                                  tslope, tau, gS);
}

int launch_rhs(Handle& h, double* b) {
  if (h.p.op == AAO_OP_RIESZ) return riesz_rhs(h, b);
  if (op_2d(h.p.op)) return heston_rhs(h, b);
  k_rhs<<<grid_for(h.n), kThreads, 0, h.stream>>>(b, h.nx, h.nt, h.mL, h.mD, h.mU, h.coef_rows, h.gL, h.gR,
                                                   h.p.s_max / (h.nx + 1), h.p.K, h.p.payoff);
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

// ----------------------------------------------------------------------------------------
// FGMRES(m)
// ----------------------------------------------------------------------------------------

namespace {

int read_scalars(Handle& h, int first, int count) {
  AAO_TRY_CUDA(cudaMemcpyAsync(h.host_scal, h.scal + first, sizeof(double) * count, cudaMemcpyDeviceToHost, h.stream));
  AAO_TRY_CUDA(cudaStreamSynchronize(h.stream));
  return AAO_OK;
}

// out[c0 + q] = V_{c0+q} . w, q < cnt <= 8
int mdot(Handle& h, int c0, int cnt, const double* w, double* out) {
  const size_t n = h.n;
  const int g = grid_for(n);
  ProfScope ps(AAO_K_ARNOLDI, h.stream, 8.0 * (double)n * (cnt + 1), 2.0 * (double)n * cnt);
#define AAO_MD(NV)                                                                                      \
  AAO_TRY_CUDA(launch_pdl(k_mdot<NV>, wave_blocks(h, (const void*)k_mdot<NV>, g), kThreads, 0, h.stream, h.V, c0, n, \
                          w, h.part, out, h.counter))
  switch (cnt) {
    case 1: AAO_MD(1); break;
    case 2: AAO_MD(2); break;
    case 3: AAO_MD(3); break;
    case 4: AAO_MD(4); break;
    case 5: AAO_MD(5); break;
    case 6: AAO_MD(6); break;
    case 7: AAO_MD(7); break;
    default: AAO_MD(8); break;
  }
#undef AAO_MD
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

// second-pass projections of w onto V_0..V_{nv-1} into scal[S_D2..]
int projections(Handle& h, const double* w, int nv, int slot) {
  const size_t n = h.n;
  const int g = grid_for(n);
  for (int c0 = 0; c0 < nv; c0 += 8) {
    const int cnt = (nv - c0) < 8 ? (nv - c0) : 8;
    AAO_TRY(mdot(h, c0, cnt, w, h.scal + slot));
  }
  return AAO_OK;
}

int update(Handle& h, double* w, int j, int pass, float* vf) {
  const size_t n = h.n;
  const int g = grid_for(n);
  const int nv = j + 1;
  ProfScope ps(AAO_K_ARNOLDI, h.stream, 8.0 * (double)n * (nv + 2), 2.0 * (double)n * (nv + 1));
#define AAO_UP(NV)                                                                                        \
  AAO_TRY_CUDA(launch_pdl(k_update<NV>, wave_blocks(h, (const void*)k_update<NV>, g), kThreads, 0, h.stream, w, h.V, j, \
                          n, pass, h.scal, h.part, h.counter, vf))
  switch (nv) {
    case 1: AAO_UP(1); break;
    case 2: AAO_UP(2); break;
    case 3: AAO_UP(3); break;
    case 4: AAO_UP(4); break;
    case 5: AAO_UP(5); break;
    case 6: AAO_UP(6); break;
    case 7: AAO_UP(7); break;
    case 8: AAO_UP(8); break;
    default: AAO_UP(0); break;
  }
#undef AAO_UP
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

}  // namespace

int run_fgmres(Handle& h, const double* b, double* x, double tol, int m, int maxit, aao_stats* st, bool zero_guess) {
  const auto t0 = std::chrono::steady_clock::now();
  const uint64_t l0 = g_launches.load();
  AAO_TRY(ensure_workspace(h, m));
  const size_t n = h.n;
  const int g = grid_for(n);
  const size_t zsz = h.mixed ? sizeof(float) : sizeof(double);
  char* Zb = reinterpret_cast<char*>(h.Z);
  // mixed precision: the residual and update kernels also write an FP32 copy of the basis vector
  // that the next preconditioner apply reads (the Riesz matvec does not write one)
  float* vf = (h.mixed && h.p.op != AAO_OP_RIESZ && !op_2d(h.p.op)) ? h.Vf : nullptr;

  int its = 0, restarts = 0, status = AAO_OK;
  double rel = 0.0, est = 0.0, bnorm = 0.0;
  bool x_fresh = zero_guess;  // x holds nothing yet and stands for zero
  // the error word of the tensor-core step (b) reports this solve only
  if (h.rz_err) AAO_TRY_CUDA(cudaMemsetAsync(h.rz_err, 0, sizeof(int), h.stream));
  for (bool first = true;; first = false) {
    NvtxRange nv_cycle("fgmres_cycle");
    // restart residual r = b - M x, written as the raw first basis vector V_0 (the first one also
    // forms ||b||^2); from a zero guess the first one is b itself, and x is not read: the first
    // solution update writes it (x_fresh), or it is zeroed if the solve ends before one
    if (first && zero_guess) {
      ProfScope ps(AAO_K_OTHER, h.stream, (double)n * (16.0 + (vf ? 4.0 : 0.0)));
      AAO_TRY_CUDA(launch_pdl(k_first_zero, wave_blocks(h, (const void*)k_first_zero, g), kThreads, 0, h.stream, b,
                              h.V, vf, n, h.part, h.scal, h.counter, m));
      AAO_CHECK_LAUNCH();
    } else {
      AAO_TRY(launch_matvec(h, x, false, h.V, b, nullptr, 0, m, first, vf));
    }
    AAO_TRY(read_scalars(h, S_BETA2, 2));  // BETA2, BNORM2
    if (first) {
      bnorm = sqrt(h.host_scal[1]);
      if (!(bnorm > 0.0)) {
        AAO_TRY_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, h.stream));
        AAO_TRY_CUDA(cudaStreamSynchronize(h.stream));
        status = isfinite(bnorm) ? AAO_OK : AAO_BREAKDOWN;
        break;
      }
    }
    {
      const double beta = sqrt(h.host_scal[0]);
      rel = beta / bnorm;
      if (!isfinite(beta)) { status = AAO_BREAKDOWN; break; }
      if (beta <= tol * bnorm) { status = AAO_OK; break; }
      if (its >= maxit) { status = AAO_NOT_CONVERGED; break; }
      int jd = 0;
      for (int j = 0; j < m; ++j) {
        double* Vj = h.V + (size_t)j * n;
        double* W = h.V + (size_t)(j + 1) * n;  // raw next basis vector, orthogonalised in place
        void* Zj = Zb + zsz * (size_t)j * n;
        // z_j = P^{-1} (sigma_j V_j): the scale is applied inside the first FFT kernel
        AAO_TRY(launch_precond(h, Vj, Zj, h.mixed, h.scal + S_SIG + j, vf));
        const int nv = j + 1;
        const int nf = nv < 8 ? nv : 8;
        AAO_TRY(launch_matvec(h, Zj, h.mixed, W, nullptr, h.V, nf, m));
        if (nv > 8) {
          for (int c0 = 8; c0 < nv; c0 += 8) {
            const int cnt = (nv - c0) < 8 ? (nv - c0) : 8;
            AAO_TRY(mdot(h, c0, cnt, W, h.scal + S_D1));
          }
        }
        AAO_TRY(update(h, W, j, 1, vf));
        AAO_TRY(read_scalars(h, S_EST, 4));  // EST, HN, FLAG, REORTH
        if (h.host_scal[3] != 0.0) {
          AAO_TRY(projections(h, W, nv, S_D2));
          AAO_TRY(update(h, W, j, 2, vf));
          AAO_TRY(read_scalars(h, S_EST, 4));
        }
        est = h.host_scal[0];
        const double hn = h.host_scal[1];
        ++its;
        jd = j + 1;
        if (h.host_scal[2] != 0.0 || !isfinite(est)) { status = AAO_BREAKDOWN; break; }
        if (est <= tol * bnorm || hn <= 1e-300 || its >= maxit) break;
      }
      if (status == AAO_BREAKDOWN) break;
      {
        ProfScope ps(AAO_K_OTHER, h.stream, (double)n * (16.0 + zsz * jd));
        if (h.mixed)
          AAO_TRY_CUDA(launch_pdl(k_xupdate<float>, wave_blocks(h, (const void*)k_xupdate<float>, g), kThreads, 0,
                                  h.stream, x, (const float*)h.Z, jd, n, h.scal, x_fresh ? 1 : 0));
        else
          AAO_TRY_CUDA(launch_pdl(k_xupdate<double>, wave_blocks(h, (const void*)k_xupdate<double>, g), kThreads, 0,
                                  h.stream, x, (const double*)h.Z, jd, n, h.scal, x_fresh ? 1 : 0));
        x_fresh = false;
      }
      AAO_CHECK_LAUNCH();
      ++restarts;
    }
  }
  if (x_fresh) AAO_TRY_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, h.stream));
  if (h.rz_err) {
    // a tensor-core product of the spectral step (b) whose bounded wait gave up (its output was
    // skipped): report it rather than the solve's status
    int e = 0;
    AAO_TRY_CUDA(cudaMemcpyAsync(&e, h.rz_err, sizeof(int), cudaMemcpyDeviceToHost, h.stream));
    AAO_TRY_CUDA(cudaStreamSynchronize(h.stream));
    if (e) {
      AAO_TRY_CUDA(cudaMemsetAsync(h.rz_err, 0, sizeof(int), h.stream));
      status = AAO_TIMEOUT;
    }
  }
  const auto t1 = std::chrono::steady_clock::now();
  if (st) {
    st->status = status;
    st->iterations = its;
    st->restarts = restarts;
    st->launches = (int32_t)(g_launches.load() - l0);
    st->rel_residual = rel;
    st->est_residual = est / (bnorm > 0 ? bnorm : 1.0);
    st->ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  }
  if (status != AAO_OK) {
    char buf[160];
    snprintf(buf, sizeof buf, "fgmres_solve: status %d after %d iterations, relative residual %.3e", status, its, rel);
    set_error(buf);
  }
  return status;
}

}  // namespace aao

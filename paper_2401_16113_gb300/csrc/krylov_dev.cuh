// Device building blocks of the FP64 outer loop (CN matvec, Gram-Schmidt sums, Givens), shared
// by the single-instance kernels (krylov.cu) and the persistent batched solver (batch.cu).
#pragma once

#include <math.h>

#include "aao_internal.cuh"

namespace aao {
namespace kdev {

constexpr int kRedBlocks = 1216;   // 152 SMs x 8: blocks of the grid-stride kernels
constexpr int kPartBlocks = 4096;  // capacity (blocks) of the partial-sum buffer
constexpr int kPartLd = 16;        // partial sums per block
constexpr int kThreads = 256;
constexpr double kReorthEta = 1e-5;

// device scalar slots (offsets into Handle::scal)
enum : int {
  S_D1 = 0,       // raw first-pass projections V_i . w
  S_D2 = 128,     // raw second-pass projections
  S_SIG = 256,    // sigma_i = 1 / ||V_i||, i = 0..m
  // slot 330 unused: ||w||^2 before orthogonalisation is recovered from S_WP2 and the projections
  S_WP2 = 331,    // ||w'||^2 after the last pass
  S_EST = 332,    // |g_{j+1}| (residual estimate)
  S_HN = 333,     // h_{j+1,j}
  S_FLAG = 334,   // non-finite value seen
  S_REORTH = 335, // second pass requested
  S_BETA2 = 336,  // ||r||^2
  S_BNORM2 = 337, // ||b||^2
  S_G = 340,      // g, m+1
  S_CS = 420,     // Givens cosines, m
  S_SN = 500,     // Givens sines, m
  S_HMAT = 580,   // Hessenberg, column-major (m+1) x m, ld 65
  S_TOTAL = 580 + 65 * 64
};
constexpr int kLdH = 65;

template <typename T> __device__ __forceinline__ double ld(const T* p) { return widen(__ldg(p)); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// block-reduce `cnt` per-thread accumulators into out[0..cnt); blockDim.x == kThreads
template <int CNT>
__device__ __forceinline__ void block_sums(const double (&acc)[CNT], int cnt, double* out) {
  __shared__ double red[kThreads / 32][CNT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < CNT; ++q) {
    double v = warp_sum(acc[q]);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0.0;
#pragma unroll
    for (int wv = 0; wv < kThreads / 32; ++wv) s += red[wv][threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Shared scratch of CNT x kThreads doubles, one per CNT, used by the two reductions below (which
// never run at the same time).
template <int CNT>
__device__ __forceinline__ double (&red_scratch())[CNT][kThreads] {
  __shared__ double red[CNT][kThreads];
  return red;
}

// The same with fewer FP64 instructions, for kernels that can spare CNT * kThreads doubles of
// static shared memory: value q is summed by warp q mod 8, each lane adding the 8 partials of its
// lane position before one shuffle tree (12 FP64 warp instructions per value instead of 48).
template <int CNT>
__device__ __forceinline__ void block_sums_wide(const double (&acc)[CNT], int cnt, double* out) {
  auto& red = red_scratch<CNT>();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < CNT; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int q = warp; q < cnt; q += kThreads / 32) {
    double v = red[q][lane];
#pragma unroll
    for (int k = 1; k < kThreads / 32; ++k) v += red[q][lane + 32 * k];
    v = warp_sum(v);
    if (lane == 0) out[q] = v;
  }
  __syncthreads();
}

// Executed by the last block (blockDim.x == kThreads): out(q, total_q) for q < cnt <= CNT, total_q
// = the sum over blocks b < nblk of part[b * kPartLd + q] in a fixed order. All values are reduced
// at once (every thread loads its blocks' partials of every value, then warp q mod 8 reduces value
// q), so the serial tail of the kernel is one round trip and one shuffle tree; out runs on thread
// 0 in order of q. Resets the counter for the next kernel.
template <int CNT, typename OUT>
__device__ void finish_sums_wide(const double* part, int nblk, int cnt, OUT out, unsigned int* counter) {
  auto& red = red_scratch<CNT>();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double s[CNT];
#pragma unroll
  for (int q = 0; q < CNT; ++q) s[q] = 0.0;
#pragma unroll 4
  for (int b = threadIdx.x; b < nblk; b += kThreads) {
#pragma unroll
    for (int q = 0; q < CNT; ++q)
      if (q < cnt) s[q] += __ldcg(part + (size_t)b * kPartLd + q);
  }
#pragma unroll
  for (int q = 0; q < CNT; ++q) red[q][threadIdx.x] = s[q];
  __syncthreads();
  for (int q = warp; q < cnt; q += kThreads / 32) {
    double v = red[q][lane];
#pragma unroll
    for (int k = 1; k < kThreads / 32; ++k) v += red[q][lane + 32 * k];
    v = warp_sum(v);
    __syncwarp();
    if (lane == 0) red[q][0] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < cnt; ++q) out(q, red[q][0]);
    *counter = 0u;
  }
}

// Givens update of Hessenberg column j. w = M z_j with z_j = P^{-1} v_j for the normalised
// v_j = sigma_j V_j, so h_ij = v_i . w = sigma_i d_i and h_{j+1,j} = ||w'||; one thread.
__device__ inline void givens_column(double* __restrict__ scal, int j, const double* d1, const double* d2) {
  double* H = scal + S_HMAT + (size_t)j * kLdH;
  for (int i = 0; i <= j; ++i) H[i] = scal[S_SIG + i] * (d1[i] + (d2 ? d2[i] : 0.0));
  const double wn = sqrt(fmax(scal[S_WP2], 0.0));
  const double hn = wn;
  H[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = H[i], c = H[i + 1];
    H[i] = scal[S_CS + i] * a + scal[S_SN + i] * c;
    H[i + 1] = -scal[S_SN + i] * a + scal[S_CS + i] * c;
  }
  const double rho = hypot(H[j], H[j + 1]);
  const double cs = rho > 0.0 ? H[j] / rho : 1.0, sn = rho > 0.0 ? H[j + 1] / rho : 0.0;
  scal[S_CS + j] = cs;
  scal[S_SN + j] = sn;
  H[j] = rho;
  H[j + 1] = 0.0;
  const double g = scal[S_G + j];
  scal[S_G + j + 1] = -sn * g;
  scal[S_G + j] = cs * g;
  scal[S_EST] = fabs(sn * g);
  scal[S_HN] = hn;
  scal[S_SIG + j + 1] = wn > 0.0 ? 1.0 / wn : 0.0;
  if (!isfinite(rho) || !isfinite(hn)) scal[S_FLAG] = 1.0;
}

// givens_column on one thread with its inputs already in shared memory: h = column j of H before
// the rotations (sigma_i (d1_i + d2_i), i <= j; updated in place, needs j + 2 entries), cs/sn the
// previous rotations, g = g_j, wp2 = ||w'||^2. Writes the results to scal.
__device__ inline void givens_column_staged(double* __restrict__ scal, int j, double wp2, double* h, const double* cs_,
                                            const double* sn_, double g) {
  const double wn = sqrt(fmax(wp2, 0.0));
  h[j + 1] = wn;
  for (int i = 0; i < j; ++i) {
    const double a = h[i], c = h[i + 1];
    h[i] = cs_[i] * a + sn_[i] * c;
    h[i + 1] = -sn_[i] * a + cs_[i] * c;
  }
  const double rho = hypot(h[j], h[j + 1]);
  const double rr = rho > 0.0 ? 1.0 / rho : 0.0;
  const double cs = rho > 0.0 ? h[j] * rr : 1.0, sn = rho > 0.0 ? h[j + 1] * rr : 0.0;
  double* H = scal + S_HMAT + (size_t)j * kLdH;
  for (int i = 0; i < j; ++i) H[i] = h[i];
  H[j] = rho;
  H[j + 1] = 0.0;
  scal[S_CS + j] = cs;
  scal[S_SN + j] = sn;
  scal[S_G + j + 1] = -sn * g;
  scal[S_G + j] = cs * g;
  scal[S_EST] = fabs(sn * g);
  scal[S_HN] = wn;
  scal[S_SIG + j + 1] = wn > 0.0 ? 1.0 / wn : 0.0;
  if (!isfinite(rho) || !isfinite(wn)) scal[S_FLAG] = 1.0;
}

// One work item of the tiled matvec y = M x: this warp's kMvCols = 30 output columns
// [o0, o0 + 30) over time levels [t0, t1), keeping level t-1 in registers. Lane L holds column
// o0 - 1 + L (lanes 0 and 31 are the halo), so the spatial neighbours of s = x_t + x_{t-1} come
// from lane shuffles with no FP64 work of their own. With (L, D - 1, U) = tau/2 A_t and
// x_t - x_{t-1} = 2 x_t - s,
//  y_t,i = (x_t - x_{t-1})_i - [tau/2 A_t s]_i = 2 x_t,i - [L s_{i-1} + D s_i + U s_{i+1}],
// four FP64 operations per unknown (one add, three FMAs): 2 x is formed by integer bit operations.
// MODE 0: y only. MODE 1: y = b - M x = (b - 2 x_t) + [...], acc[0] += y.y, and the FP32 copy yf
// if given. MODE 3: as MODE 1, and acc[1] += b.b.
// MODE 2: acc[q] += V_q . y (q < ND, a compile-time count so that no predicated-off FP64
// instruction is issued), and acc[ND] += y.y when the caller has room for it (NA > ND).
constexpr int kMvCols = 30;
template <typename IN, int MODE, int ND, int NA>
__device__ __forceinline__ void matvec_item(const IN* __restrict__ x, double* __restrict__ y,
                                            const double* __restrict__ b, int nx, int t0, int t1, int o0,
                                            const double* __restrict__ L, const double* __restrict__ D,
                                            const double* __restrict__ U, int rows, const double* __restrict__ V,
                                            size_t vstride, double (&acc)[NA], float* __restrict__ yf = nullptr) {
  constexpr bool RES = MODE == 1 || MODE == 3;
  constexpr int NVQ = MODE == 2 ? ND : 0;
  const int lane = threadIdx.x & 31;
  const int i = o0 - 1 + lane;
  const bool in = i >= 0 && i < nx;               // the column exists (x is zero outside)
  const bool act = in && lane > 0 && lane < 31;   // an output column of this item
  double xp = 0.0;
  if (t0 > 0 && in) xp = ld(x + (size_t)(t0 - 1) * nx + i);
  // the loads of row t + 1 are issued before row t is computed (one row in flight ahead)
  IN xn = IN(0);
  double ln = 0.0, dn = 0.0, un = 0.0, bn = 0.0, vn[NVQ > 0 ? NVQ : 1];
  auto fetch = [&](int t) {
    const size_t r = (size_t)t * nx;
    xn = in ? __ldg(x + r + i) : IN(0);
    if (act) {
      const size_t c = rows == 1 ? (size_t)i : r + i;
      ln = __ldg(L + c);
      dn = __ldg(D + c);
      un = __ldg(U + c);
      if constexpr (RES) bn = __ldg(b + r + i);
#pragma unroll
      for (int q = 0; q < NVQ; ++q) vn[q] = __ldg(V + (size_t)q * vstride + r + i);
    }
  };
  if (t0 < t1) fetch(t0);
  for (int t = t0; t < t1; ++t) {
    const size_t r = (size_t)t * nx;
    const double xc = widen(xn), x2 = twice(xn);
    const double lc = ln, dc = dn, uc = un, bc = bn;
    double vc[NVQ > 0 ? NVQ : 1];
#pragma unroll
    for (int q = 0; q < NVQ; ++q) vc[q] = vn[q];
    if (t + 1 < t1) fetch(t + 1);
    if constexpr (RES) {
      // restart residual from a zero initial guess: when every value this warp reads is +-0
      // (integer test, warp-uniform), y = b - M x = b without any FP64 arithmetic
      auto z = [](double v) { return (__double_as_longlong(v) << 1) == 0; };
      if (__all_sync(0xffffffffu, z(xc) && z(xp))) {
        if (act) {
          acc[0] = fma(bc, bc, acc[0]);
          if constexpr (MODE == 3) acc[NA - 1] = fma(bc, bc, acc[NA - 1]);
          y[r + i] = bc;
          if (yf) yf[r + i] = narrow(bc);
        }
        xp = xc;
        continue;
      }
    }
    const double s = xc + xp;
    const double sl = __shfl_up_sync(0xffffffffu, s, 1);
    const double sr = __shfl_down_sync(0xffffffffu, s, 1);
    if (act) {
      double v;
      if constexpr (RES) {
        v = fma(dc, s, bc - x2);
        v = fma(lc, sl, v);
        v = fma(uc, sr, v);
        acc[0] = fma(v, v, acc[0]);
        if constexpr (MODE == 3) acc[NA - 1] = fma(bc, bc, acc[NA - 1]);
      } else {
        v = fma(-dc, s, x2);
        v = fma(-lc, sl, v);
        v = fma(-uc, sr, v);
      }
      y[r + i] = v;
      if constexpr (RES) {
        if (yf) yf[r + i] = narrow(v);
      }
      if constexpr (MODE == 2) {
#pragma unroll
        for (int q = 0; q < ND; ++q) acc[q] = fma(vc[q], v, acc[q]);
        if constexpr (NA > ND) acc[ND] = fma(v, v, acc[ND]);
      }
    }
    xp = xc;
  }
}

}  // namespace kdev
}  // namespace aao

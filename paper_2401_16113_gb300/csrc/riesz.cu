// The Riesz fractional operator (Eq. 1.2, second case) in log-price: a dense Toeplitz A.
//
//   A = -kappa h^-beta toeplitz(g_|i-j|) + (r - kappa)/(2h) (central first difference) - r I,
//   kappa = sigma^2/2, g_k = (-1)^k Gamma(beta+1)/(Gamma(beta/2-k+1) Gamma(beta/2+k+1)) (fractional
//   centred difference, computed by its recurrence g_{k+1} = g_k (k - beta/2)/(beta/2 + k + 1)).
//   The nodes beyond x = -x_max carry the left Dirichlet value K e^{-rt} - e^{-x_max}, those beyond
//   x = x_max carry 0; row i collects sum_{m > i} g_m = -g_0/2 - sum_{m=1}^{i} g_m of the left ones.
//
// Kernels:
//   k_rz_matvec  FP64 y = M x with the Toeplitz product A s by circulant embedding of length
//                N2 >= 2 nx - 1: two time levels are packed as the real and imaginary parts of one
//                complex FFT (A is real), forward FFT, pointwise product with the circulant's
//                spectrum, inverse FFT (shared-memory Stockham, FP64). Fused with the residual norm
//                or the first Gram-Schmidt projections, finished by the last block.
//   k_rz_rhs     b = xi + tau f (xi needs one dense product A u^0).
//   k_rz_form / k_lu_panel / k_lu_trsm / k_lu_update
//                at aao_create: the shifted matrices mu_k I - A~ of step (b) of Eq. 3.2 for the
//                nt/2+1 bins, factored in place by blocked right-looking LU without pivoting
//                (FP32 complex; the matrices are diagonally dominant, see the design notes).
//   k_rz_trsv    per apply: forward (unit L) and backward (U) blocked substitution of every bin.
//   k_rz_cgemm   step (b) when the operator is symmetric (no drift): with tau Abar = Q diag(lambda) Q^T
//                (eigendecomposition at aao_create), z2_k = Q diag(D_k) Q^T z1_k for every bin is two
//                products of the K x Nx complex half spectrum with the real Nx x Nx matrix Q.
#include <math.h>

#include <complex>
#include <vector>

#include "krylov_dev.cuh"
#include "precond_dev.cuh"

namespace aao {

namespace {

using namespace kdev;
using namespace pdev;

constexpr int kNB = 32;  // LU / substitution block

// ------------------------------------------------------------------- spectral step (b)
// Partial products P[s][k][n] = sum_{m in segment s} A[k][m] B[m][n] for bins k < Kb: A complex
// rows of pitch lda (FP32 complex), B real row-major with leading dimension ldb, segment s =
// [s Mseg, (s+1) Mseg) with Mseg a multiple of kGM, columns n < gridDim.x kGN <= ldb (the tables
// are zero-padded, so padded rows and columns contribute zeros). A CTA computes kGB bins x kGN
// columns of one segment; thread (tb, tn) holds bins 4 tb .. 4 tb + 3 and columns 4 tn + {0..3}
// and 64 + 4 tn + {0..3}: per contraction index 4 shared loads of 16 bytes feed 64 FMAs. Both
// tiles go through shared memory, the next chunk's loads are issued before the current products.
// The segments are summed in a fixed order by k_rz_cgemm_sum (deterministic, no atomics).
constexpr int kGB = 32, kGN = 128, kGM = 16, kGSplit = 4;
__global__ void __launch_bounds__(128) k_rz_cgemm(const float2* __restrict__ A, int lda, const float* __restrict__ B,
                                                  int ldb, float2* __restrict__ P, int ldp, int Kb, int Mseg) {
  __shared__ __align__(16) float2 As[kGM][kGB + 2];  // [m][bin], +2: transposed stores 2-way
  __shared__ __align__(16) float Bs[kGM][kGN];
  pdl_sync();
  const int tb = threadIdx.x >> 4, tn = threadIdx.x & 15;
  const int b0 = blockIdx.y * kGB, n0 = blockIdx.x * kGN, seg = blockIdx.z;
  const int mbeg = seg * Mseg, mend = mbeg + Mseg;
  const float2 zero = make_float2(0.f, 0.f);
  float2 acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[i][q] = zero;
  // A tile: 32 bins x 16 m complex (4 per thread: bin = e >> 4, m = e & 15, e = t + 128 i);
  // B tile: 16 rows x 128 floats (4 float4 per thread: row = e >> 5, column group = e & 31)
  float2 ra[4];
  float4 rb[4];
  auto fetch = [&](int m0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = threadIdx.x + 128 * i, bin = b0 + (e >> 4);
      ra[i] = bin < Kb ? __ldg(A + (size_t)bin * lda + m0 + (e & 15)) : zero;
      rb[i] = __ldg(reinterpret_cast<const float4*>(B + (size_t)(m0 + (e >> 5)) * ldb + n0 + 4 * (e & 31)));
    }
  };
  fetch(mbeg);
  for (int m0 = mbeg; m0 < mend; m0 += kGM) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = threadIdx.x + 128 * i;
      As[e & 15][e >> 4] = ra[i];
      *reinterpret_cast<float4*>(&Bs[e >> 5][4 * (e & 31)]) = rb[i];
    }
    __syncthreads();
    if (m0 + kGM < mend) fetch(m0 + kGM);
#pragma unroll
    for (int mm = 0; mm < kGM; ++mm) {
      const float4 a01 = *reinterpret_cast<const float4*>(&As[mm][4 * tb]);
      const float4 a23 = *reinterpret_cast<const float4*>(&As[mm][4 * tb + 2]);
      const float4 bl = *reinterpret_cast<const float4*>(&Bs[mm][4 * tn]);
      const float4 bh = *reinterpret_cast<const float4*>(&Bs[mm][64 + 4 * tn]);
      const float ar[4] = {a01.x, a01.z, a23.x, a23.z}, ai[4] = {a01.y, a01.w, a23.y, a23.w};
      const float bv[8] = {bl.x, bl.y, bl.z, bl.w, bh.x, bh.y, bh.z, bh.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          acc[i][q].x = fmaf(ar[i], bv[q], acc[i][q].x);
          acc[i][q].y = fmaf(ai[i], bv[q], acc[i][q].y);
        }
    }
    __syncthreads();
  }
  float2* Ps = P + (size_t)seg * Kb * ldp;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int b = b0 + 4 * tb + i;
    if (b >= Kb) continue;
    float4* lo = reinterpret_cast<float4*>(Ps + (size_t)b * ldp + n0 + 4 * tn);
    float4* hi = reinterpret_cast<float4*>(Ps + (size_t)b * ldp + n0 + 64 + 4 * tn);
    lo[0] = make_float4(acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y);
    lo[1] = make_float4(acc[i][2].x, acc[i][2].y, acc[i][3].x, acc[i][3].y);
    hi[0] = make_float4(acc[i][4].x, acc[i][4].y, acc[i][5].x, acc[i][5].y);
    hi[1] = make_float4(acc[i][6].x, acc[i][6].y, acc[i][7].x, acc[i][7].y);
  }
}

// C[k][n] = (D[k][n] *) sum_s P[s][k][n] for k < Kb, n < N (N even; pairs of complex per thread)
__global__ void __launch_bounds__(256) k_rz_cgemm_sum(const float2* __restrict__ P, int ldp, int Kb, int N,
                                                      float2* __restrict__ C, int ldc,
                                                      const float2* __restrict__ D, int ldd) {
  pdl_sync();
  const int half = N >> 1;
  const size_t total = (size_t)Kb * half, plane = (size_t)Kb * ldp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / half), n = 2 * (int)(e - (size_t)k * half);
    const float4* src = reinterpret_cast<const float4*>(P + (size_t)k * ldp + n);
    float4 v = __ldg(src);
#pragma unroll
    for (int s = 1; s < kGSplit; ++s) {
      const float4 w = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float2*>(src) + s * plane));
      v.x += w.x; v.y += w.y; v.z += w.z; v.w += w.w;
    }
    if (D) {
      const float4 d = __ldg(reinterpret_cast<const float4*>(D + (size_t)k * ldd + n));
      v = make_float4(v.x * d.x - v.y * d.y, v.x * d.y + v.y * d.x, v.z * d.z - v.w * d.w, v.z * d.w + v.w * d.z);
    }
    *reinterpret_cast<float4*>(C + (size_t)k * ldc + n) = v;
  }
}

// ------------------------------------------------------------------------------- matvec
template <typename IN, int MODE, int ND>
__global__ void __launch_bounds__(256) k_rz_matvec(const IN* __restrict__ x, double* __restrict__ y,
                                                   const double* __restrict__ b, int nx, int nt, int n2, int log2n2,
                                                   const double2* __restrict__ chat, const double2* __restrict__ tw2,
                                                   const double* __restrict__ V, size_t vstride,
                                                   double* __restrict__ part, double* __restrict__ scal,
                                                   unsigned int* __restrict__ counter, int m) {
  constexpr int NA = MODE == 2 ? ND : 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* data = reinterpret_cast<double2*>(smraw);
  double2* stw = data + n2;
  const int t0 = 2 * blockIdx.x, t1 = t0 + 1;
  const bool has1 = t1 < nt;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    stw[i] = tw2[i];
    double s0 = 0.0, s1 = 0.0;
    if (i < nx) {
      const double x0 = ld(x + (size_t)t0 * nx + i);
      const double xm = t0 > 0 ? ld(x + (size_t)(t0 - 1) * nx + i) : 0.0;
      s0 = x0 + xm;
      if (has1) s1 = ld(x + (size_t)t1 * nx + i) + x0;
    }
    data[i] = make_double2(s0, s1);
  }
  __syncthreads();
  smem_fft(data, log2n2, 0, stw);
  // pointwise product with the circulant spectrum (already scaled by tau/2 / N2), conjugated so
  // that a second forward transform gives the conjugate of the inverse transform
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    const double2 z = data[i], c = chat[i];
    data[i] = make_double2(z.x * c.x - z.y * c.y, -(z.x * c.y + z.y * c.x));
  }
  __syncthreads();
  smem_fft(data, log2n2, 0, stw);
  double acc[NA];
#pragma unroll
  for (int q = 0; q < NA; ++q) acc[q] = 0.0;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const double2 r = data[i];  // conj of (tau/2 A s): real part row t0, -imag part row t1
    for (int h = 0; h < 2; ++h) {
      const int t = t0 + h;
      if (t >= nt) break;
      const size_t e = (size_t)t * nx + i;
      const double xc = ld(x + e);
      const double xm = t > 0 ? ld(x + e - nx) : 0.0;
      double v = (xc - xm) - (h == 0 ? r.x : -r.y);
      if (MODE == 1) {
        v = __ldg(b + e) - v;
        acc[0] = fma(v, v, acc[0]);
      }
      y[e] = v;
      if (MODE == 2) {
#pragma unroll
        for (int q = 0; q < ND; ++q) acc[q] = fma(__ldg(V + (size_t)q * vstride + e), v, acc[q]);
      }
    }
  }
  if constexpr (MODE == 0) return;
  __shared__ double red[8][NA];
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const double v = warp_sum(acc[q]);
      if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < NA) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
      part[(size_t)blockIdx.x * kPartLd + threadIdx.x] = s;
    }
  }
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  if (threadIdx.x == 0) {
    for (int q = 0; q < NA; ++q) {
      double s = 0.0;
      for (unsigned bb = 0; bb < gridDim.x; ++bb) s += __ldcg(part + (size_t)bb * kPartLd + q);
      if (MODE == 2) {
        scal[S_D1 + q] = s;
      } else {
        scal[S_BETA2] = s;
        const double beta = sqrt(s);
        scal[S_SIG] = beta > 0.0 ? 1.0 / beta : 0.0;
        scal[S_G] = beta;
        for (int k = 1; k <= m; ++k) scal[S_G + k] = 0.0;
        scal[S_FLAG] = isfinite(s) ? 0.0 : 1.0;
      }
    }
    *counter = 0u;
  }
}

// b = xi + tau f: f from the left exterior value averaged over t_k and t_{k+1}; xi = u0 + A~ u0 / 2
__global__ void k_rz_rhs(double* __restrict__ b, int nx, int nt, const double* __restrict__ hcol,
                         const double* __restrict__ hrow, const double* __restrict__ hcl,
                         const double* __restrict__ gL, double xmax, double h, double K) {
  const size_t n = (size_t)nx * nt;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int t = (int)(e / nx), i = (int)(e - (size_t)t * nx);
    double v = hcl[i] * (gL[t] + gL[t + 1]);
    if (t == 0) {
      auto u0 = [&](int j) { return fmax(K - exp(-xmax + h * (j + 1)), 0.0); };
      double a = u0(i);
      for (int j = 0; j < nx; ++j) a = fma(j <= i ? hcol[i - j] : hrow[j - i], u0(j), a);
      v += a;
    }
    b[e] = v;
  }
}

// ------------------------------------------------------------------------------- LU at create
// M_k = mu_k I - A~ (row-major, complex FP32), A~ = tau A from its first column / row
__global__ void k_rz_form(float2* __restrict__ M, int nx, const double* __restrict__ tcol,
                          const double* __restrict__ trow, const float2* __restrict__ mu) {
  const int k = blockIdx.y;
  const size_t nn = (size_t)nx * nx;
  float2* Mk = M + (size_t)k * nn;
  const float2 muk = mu[k];
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / nx), j = (int)(e - (size_t)i * nx);
    const double a = j <= i ? tcol[i - j] : trow[j - i];
    Mk[e] = make_float2((float)((i == j ? (double)muk.x : 0.0) - a), i == j ? muk.y : 0.f);
  }
}

// unblocked LU of the panel rows [kb, n), columns [kb, kb+w): one CTA per bin
__global__ void __launch_bounds__(256) k_lu_panel(float2* __restrict__ M, int n, int kb, int w) {
  float2* A = M + (size_t)blockIdx.x * n * n;
  __shared__ float2 prow[kNB];
  for (int j = kb; j < kb + w; ++j) {
    if (threadIdx.x < kb + w - j) prow[threadIdx.x] = A[(size_t)j * n + j + threadIdx.x];
    __syncthreads();
    const float2 inv = cinv(prow[0]);
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
      float2* ri = A + (size_t)i * n;
      const float2 l = cmul(ri[j], inv);
      ri[j] = l;
      for (int c = 1; c < kb + w - j; ++c) ri[j + c] = csub(ri[j + c], cmul(l, prow[c]));
    }
    __syncthreads();
  }
}

// U12 = L11^{-1} A12 for rows [kb, kb+w) and columns [kb+w, n): one thread per column
__global__ void k_lu_trsm(float2* __restrict__ M, int n, int kb, int w) {
  float2* A = M + (size_t)blockIdx.y * n * n;
  const int c = kb + w + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  float2 col[kNB];
  for (int i = 0; i < w; ++i) col[i] = A[(size_t)(kb + i) * n + c];
  for (int i = 1; i < w; ++i) {
    float2 s = col[i];
    for (int j = 0; j < i; ++j) s = csub(s, cmul(A[(size_t)(kb + i) * n + kb + j], col[j]));
    col[i] = s;
  }
  for (int i = 1; i < w; ++i) A[(size_t)(kb + i) * n + c] = col[i];
}

// A22 -= L21 U12, rows and columns [kb+w, n), inner dimension w <= 32: 64 x 64 tiles, 4 x 4 per thread
__global__ void __launch_bounds__(256) k_lu_update(float2* __restrict__ M, int n, int kb, int w) {
  float2* A = M + (size_t)blockIdx.z * n * n;
  const int r0 = kb + w + blockIdx.y * 64, c0 = kb + w + blockIdx.x * 64;
  __shared__ float2 Ls[64][kNB + 1];
  __shared__ float2 Us[kNB][64 + 1];
  for (int e = threadIdx.x; e < 64 * kNB; e += blockDim.x) {
    const int r = e / kNB, k = e % kNB;
    Ls[r][k] = (r0 + r < n && k < w) ? A[(size_t)(r0 + r) * n + kb + k] : make_float2(0.f, 0.f);
    const int kk = e / 64, c = e % 64;
    Us[kk][c] = (c0 + c < n && kk < w) ? A[(size_t)(kb + kk) * n + c0 + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  float2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[a][q] = make_float2(0.f, 0.f);
  for (int k = 0; k < w; ++k) {
    float2 l[4], u[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) l[a] = Ls[tr + 16 * a][k];
#pragma unroll
    for (int q = 0; q < 4; ++q) u[q] = Us[k][tc + 16 * q];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[a][q].x = fmaf(l[a].x, u[q].x, fmaf(-l[a].y, u[q].y, acc[a][q].x));
        acc[a][q].y = fmaf(l[a].x, u[q].y, fmaf(l[a].y, u[q].x, acc[a][q].y));
      }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = r0 + tr + 16 * a, c = c0 + tc + 16 * q;
      if (r < n && c < n) {
        float2* p = A + (size_t)r * n + c;
        *p = csub(*p, acc[a][q]);
      }
    }
}

// ------------------------------------------------------------------------------- solves per apply
// Inverses of the diagonal kNB x kNB blocks of every bin's factors (at aao_create): block bi of
// bin k stores L_bb^{-1} (unit lower) and U_bb^{-1} (upper), row-major, zero beyond the block's
// width. One warp per triangle: lane c forms column c of the inverse by substitution.
__global__ void __launch_bounds__(64) k_rz_diaginv(const float2* __restrict__ LU, float2* __restrict__ dinv, int nx,
                                                   int nb) {
  __shared__ float2 blk[kNB][kNB + 1];
  const int bi = blockIdx.x, k = blockIdx.y;
  const int r0 = bi * kNB, w = min(kNB, nx - r0);
  const float2* A = LU + (size_t)k * nx * nx;
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int i = e / kNB, j = e % kNB;
    blk[i][j] = (i < w && j < w) ? A[(size_t)(r0 + i) * nx + r0 + j] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, tri = threadIdx.x >> 5;  // 0: L, 1: U
  float2* out = dinv + (((size_t)k * nb + bi) * 2 + tri) * kNB * kNB;
  float2 x[kNB];
  if (tri == 0) {
#pragma unroll
    for (int i = 0; i < kNB; ++i) {
      float2 v = make_float2(i == lane ? 1.f : 0.f, 0.f);
#pragma unroll
      for (int q = 0; q < i; ++q) v = csub(v, cmul(blk[i][q], x[q]));
      x[i] = (i < w && lane < w) ? v : make_float2(0.f, 0.f);
    }
  } else {
#pragma unroll
    for (int i = kNB - 1; i >= 0; --i) {
      float2 v = make_float2(i == lane ? 1.f : 0.f, 0.f);
#pragma unroll
      for (int q = i + 1; q < kNB; ++q) v = csub(v, cmul(blk[i][q], x[q]));
      x[i] = (i < w && lane < w) ? cmul(v, cinv(blk[i][i])) : make_float2(0.f, 0.f);
    }
  }
#pragma unroll
  for (int i = 0; i < kNB; ++i) out[i * kNB + lane] = x[i];
}

// Bin k: (mu_k I - A~) z = z1_k / lambda2_k with the LU factors; in place on the half spectrum.
// Blocked substitution: for each kNB-row block, the rows' products with the solved part of z
// (warps over rows, lanes over columns, eight loads in flight per lane), then the block itself by
// its stored inverse (one product instead of kNB dependent steps).
__global__ void __launch_bounds__(512) k_rz_trsv(float2* __restrict__ spec, int nx, int pitch,
                                                 const float2* __restrict__ LU, const float2* __restrict__ dinv,
                                                 const float2* __restrict__ il2) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* z = reinterpret_cast<float2*>(smraw);  // nx
  float2* t = z + nx;                            // kNB
  const int k = blockIdx.x;
  const float2* A = LU + (size_t)k * nx * nx;
  float2* row = spec + (size_t)k * pitch;
  const float2 sk = il2[k];
  for (int i = threadIdx.x; i < nx; i += blockDim.x) z[i] = cmul(row[i], sk);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nb = (nx + kNB - 1) / kNB;
  auto rowdot = [&](const float2* ri, int j0, int j1) {
    float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
    int j = j0 + lane;
    for (; j + 224 < j1; j += 256) {
      float2 l[8], v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) l[u] = __ldg(ri + j + 32 * u);
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = z[j + 32 * u];
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        ax = fmaf(l[u].x, v[u].x, fmaf(-l[u].y, v[u].y, ax));
        ay = fmaf(l[u].x, v[u].y, fmaf(l[u].y, v[u].x, ay));
        bx = fmaf(l[u + 1].x, v[u + 1].x, fmaf(-l[u + 1].y, v[u + 1].y, bx));
        by = fmaf(l[u + 1].x, v[u + 1].y, fmaf(l[u + 1].y, v[u + 1].x, by));
      }
    }
    for (; j < j1; j += 32) {
      const float2 l = __ldg(ri + j), v = z[j];
      ax = fmaf(l.x, v.x, fmaf(-l.y, v.y, ax));
      ay = fmaf(l.x, v.y, fmaf(l.y, v.x, ay));
    }
    float sx = ax + bx, sy = ay + by;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_down_sync(0xffffffffu, sx, o);
      sy += __shfl_down_sync(0xffffffffu, sy, o);
    }
    return make_float2(sx, sy);
  };
  // z_b <- Inv t over the block's w rows (warps over rows, lanes over columns)
  auto apply_inv = [&](const float2* inv, int r0, int w) {
    for (int i = warp; i < w; i += nw) {
      const float2 p = lane < w ? cmul(__ldg(inv + i * kNB + lane), t[lane]) : make_float2(0.f, 0.f);
      float px = p.x, py = p.y;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        px += __shfl_down_sync(0xffffffffu, px, o);
        py += __shfl_down_sync(0xffffffffu, py, o);
      }
      if (lane == 0) z[r0 + i] = make_float2(px, py);
    }
  };
  // forward: L y = z (unit lower)
  for (int bi = 0; bi < nb; ++bi) {
    const int r0 = bi * kNB, w = min(kNB, nx - r0);
    for (int i = warp; i < w; i += nw) {
      const float2 d = rowdot(A + (size_t)(r0 + i) * nx, 0, r0);
      if (lane == 0) t[i] = csub(z[r0 + i], d);
    }
    __syncthreads();
    apply_inv(dinv + (((size_t)k * nb + bi) * 2 + 0) * kNB * kNB, r0, w);
    __syncthreads();
  }
  // backward: U x = y
  for (int bi = nb - 1; bi >= 0; --bi) {
    const int r0 = bi * kNB, w = min(kNB, nx - r0);
    for (int i = warp; i < w; i += nw) {
      const float2 d = rowdot(A + (size_t)(r0 + i) * nx, r0 + w, nx);
      if (lane == 0) t[i] = csub(z[r0 + i], d);
    }
    __syncthreads();
    apply_inv(dinv + (((size_t)k * nb + bi) * 2 + 1) * kNB * kNB, r0, w);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < nx; i += blockDim.x) row[i] = z[i];
}

int grid_for(size_t n) {
  size_t g = (n + kThreads - 1) / kThreads;
  return (int)(g < (size_t)kRedBlocks ? g : (size_t)kRedBlocks);
}

}  // namespace

// ------------------------------------------------------------------------------- host
int riesz_build(Handle& h) {
  const aao_problem& p = h.p;
  const int nx = h.nx, nt = h.nt;
  const double xmax = p.s_max, hx = 2.0 * xmax / (nx + 1);
  const double kappa = 0.5 * p.sigma * p.sigma;
  const double c0 = -kappa * pow(hx, -p.beta);
  const double dr = (p.r - kappa) / (2.0 * hx);
  // fractional centred difference weights by recurrence
  std::vector<double> g(nx + 1);
  g[0] = tgamma(p.beta + 1.0) / (tgamma(0.5 * p.beta + 1.0) * tgamma(0.5 * p.beta + 1.0));
  for (int k = 0; k < nx; ++k) g[k + 1] = g[k] * ((double)k - 0.5 * p.beta) / (0.5 * p.beta + k + 1.0);
  // first column / row of A
  std::vector<double> col(nx), row(nx);
  for (int k = 0; k < nx; ++k) {
    col[k] = c0 * g[k] - (k == 1 ? dr : 0.0) - (k == 0 ? p.r : 0.0);
    row[k] = c0 * g[k] + (k == 1 ? dr : 0.0) - (k == 0 ? p.r : 0.0);
  }
  // left exterior coefficient: row i collects sum_{m > i} g_m = -g_0/2 - sum_{m=1}^{i} g_m, plus the
  // drift's coefficient on the left neighbour of row 0
  std::vector<double> cl(nx);
  double run = 0.0;  // sum_{m=1}^{i} g_m
  for (int i = 0; i < nx; ++i) {
    if (i >= 1) run += g[i];
    cl[i] = c0 * (-0.5 * g[0] - run) + (i == 0 ? -dr : 0.0);
  }
  // circulant embedding of length N2 >= 2 nx - 1 and its spectrum (direct DFT in FP64)
  int l2 = 0;
  while ((1 << l2) < 2 * nx - 1) ++l2;
  const int n2 = 1 << l2;
  h.rz_n2 = n2;
  h.rz_log2n2 = l2;
  std::vector<double> cc(n2, 0.0);
  for (int k = 0; k < nx; ++k) cc[k] = col[k];
  for (int k = 1; k < nx; ++k) cc[n2 - k] = row[k];
  std::vector<double> cs(n2), sn(n2);
  for (int q = 0; q < n2; ++q) {
    const double a = -2.0 * M_PI * (double)q / n2;
    cs[q] = cos(a);
    sn[q] = sin(a);
  }
  std::vector<double2> chat(n2), tw2(n2);
  const double sc = 0.5 * h.tau / n2;
  for (int f = 0; f < n2; ++f) {
    double re = 0.0, im = 0.0;
    for (int q = 0; q < n2; ++q) {
      if (cc[q] == 0.0) continue;
      const int idx = (int)(((long long)f * q) % n2);
      re += cc[q] * cs[idx];
      im += cc[q] * sn[idx];
    }
    chat[f] = make_double2(re * sc, im * sc);
    tw2[f] = make_double2(cs[f], sn[f]);
  }
  std::vector<double> hcol(nx), hrow(nx), hcl(nx), tcol(nx), trow(nx);
  for (int k = 0; k < nx; ++k) {
    hcol[k] = 0.5 * h.tau * col[k];
    hrow[k] = 0.5 * h.tau * row[k];
    hcl[k] = 0.5 * h.tau * cl[k];
    tcol[k] = h.tau * col[k];
    trow[k] = h.tau * row[k];
  }
  std::vector<double> gl(nt + 1);
  for (int k = 0; k <= nt; ++k) gl[k] = p.K * exp(-p.r * h.tau * k) - exp(-xmax);
  auto up = [&](auto** dst, const auto& src) -> int {
    using T = typename std::decay<decltype(src)>::type::value_type;
    AAO_TRY_CUDA(cudaMalloc((void**)dst, sizeof(T) * src.size()));
    AAO_TRY_CUDA(cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, h.stream));
    return AAO_OK;
  };
  double *d_tcol = nullptr, *d_trow = nullptr;
  AAO_TRY(up(&h.rz_chat, chat));
  AAO_TRY(up(&h.rz_tw, tw2));
  AAO_TRY(up(&h.rz_hcol, hcol));
  AAO_TRY(up(&h.rz_hrow, hrow));
  AAO_TRY(up(&h.rz_hcl, hcl));
  AAO_TRY(up(&h.gL, gl));
  AAO_TRY(up(&d_tcol, tcol));
  AAO_TRY(up(&d_trow, trow));
  const int K = h.K;
  const size_t nn = (size_t)nx * nx;
  if (riesz_symmetric(p)) {
    // no drift: tau Abar is the symmetric Toeplitz matrix of tcol; tau Abar = Q diag(lambda) Q^T
    std::vector<double> Ad(nn), lam(nx);
    for (int i = 0; i < nx; ++i)
      for (int j = 0; j < nx; ++j) Ad[(size_t)i * nx + j] = tcol[i > j ? i - j : j - i];
    if (!sym_eig(nx, Ad.data(), lam.data())) {
      set_error("aao_create: eigendecomposition of the symmetric Riesz operator did not converge");
      cudaFree(d_tcol);
      cudaFree(d_trow);
      return AAO_BREAKDOWN;
    }
    // Ad holds Q^T. Both orientations in FP32, zero-padded to ldq (a multiple of the products'
    // column tile, >= the spectrum's pitch)
    const int ldq = ((nx + kGN - 1) / kGN) * kGN;
    std::vector<float> q((size_t)ldq * ldq, 0.f), qt((size_t)ldq * ldq, 0.f);
    for (int j = 0; j < nx; ++j)
      for (int x = 0; x < nx; ++x) {
        const float v = (float)Ad[(size_t)j * nx + x];
        qt[(size_t)j * ldq + x] = v;
        q[(size_t)x * ldq + j] = v;
      }
    // D_k,j = (1/lambda_{2,k}) / (mu_k - lambda_j)
    std::vector<double2> mu(K), il2(K);
    AAO_TRY_CUDA(cudaMemcpyAsync(mu.data(), h.mu, sizeof(double2) * K, cudaMemcpyDeviceToHost, h.stream));
    AAO_TRY_CUDA(cudaMemcpyAsync(il2.data(), h.il2, sizeof(double2) * K, cudaMemcpyDeviceToHost, h.stream));
    AAO_TRY_CUDA(cudaStreamSynchronize(h.stream));
    std::vector<float2> dk((size_t)K * ldq, make_float2(0.f, 0.f));
    for (int k = 0; k < K; ++k) {
      const std::complex<double> m(mu[k].x, mu[k].y), s(il2[k].x, il2[k].y);
      for (int j = 0; j < nx; ++j) {
        const std::complex<double> v = s / (m - lam[j]);
        dk[(size_t)k * ldq + j] = make_float2((float)v.real(), (float)v.imag());
      }
    }
    AAO_TRY(up(&h.rz_q, q));
    AAO_TRY(up(&h.rz_qt, qt));
    AAO_TRY(up(&h.rz_dk, dk));
    AAO_TRY_CUDA(cudaMalloc(&h.rz_w, sizeof(float2) * (size_t)K * ldq));
    AAO_TRY_CUDA(cudaMalloc(&h.rz_part, sizeof(float2) * (size_t)kGSplit * K * ldq));
    h.rz_ldq = ldq;
    // the padding columns of the spectrum and of the workspace stay zero: every kernel writes
    // columns < nx only, or zeros
    AAO_TRY_CUDA(cudaMemsetAsync(h.rz_w, 0, sizeof(float2) * (size_t)K * ldq, h.stream));
    AAO_TRY_CUDA(cudaMemsetAsync(h.spec, 0, sizeof(float2) * (size_t)K * h.pitch, h.stream));
    AAO_TRY_CUDA(cudaStreamSynchronize(h.stream));
    h.rz_sym = true;
    cudaFree(d_tcol);
    cudaFree(d_trow);
    return AAO_OK;
  }
  // shifted matrices and their LU factors (FP32 complex)
  AAO_TRY_CUDA(cudaMalloc(&h.rz_lu, sizeof(float2) * nn * K));
  k_rz_form<<<dim3(256, K), 256, 0, h.stream>>>(h.rz_lu, nx, d_tcol, d_trow, h.muf);
  AAO_CHECK_LAUNCH();
  for (int kb = 0; kb < nx; kb += kNB) {
    const int w = nx - kb < kNB ? nx - kb : kNB;
    k_lu_panel<<<K, 256, 0, h.stream>>>(h.rz_lu, nx, kb, w);
    AAO_CHECK_LAUNCH();
    const int rest = nx - kb - w;
    if (rest > 0) {
      k_lu_trsm<<<dim3((rest + 127) / 128, K), 128, 0, h.stream>>>(h.rz_lu, nx, kb, w);
      AAO_CHECK_LAUNCH();
      k_lu_update<<<dim3((rest + 63) / 64, (rest + 63) / 64, K), 256, 0, h.stream>>>(h.rz_lu, nx, kb, w);
      AAO_CHECK_LAUNCH();
    }
  }
  {
    const int nb = (nx + kNB - 1) / kNB;
    AAO_TRY_CUDA(cudaMalloc(&h.rz_dinv, sizeof(float2) * (size_t)K * nb * 2 * kNB * kNB));
    k_rz_diaginv<<<dim3(nb, K), 64, 0, h.stream>>>(h.rz_lu, h.rz_dinv, nx, nb);
    AAO_CHECK_LAUNCH();
  }
  AAO_TRY_CUDA(cudaStreamSynchronize(h.stream));
  cudaFree(d_tcol);
  cudaFree(d_trow);
  return AAO_OK;
}

int riesz_matvec(Handle& h, const void* x, bool x_is_float, double* y, const double* b, const double* V, int nd,
                 int m) {
  const int grid = (h.nt + 1) / 2;
  const size_t smem = sizeof(double2) * 2 * (size_t)h.rz_n2;
  int threads = h.rz_n2 / 16;
  if (threads < 128) threads = 128;
  if (threads > 256) threads = 256;
  const double nn = (double)h.n;
  const double bytes = nn * (x_is_float ? 4.0 : 8.0) + nn * 8.0 + (b ? nn * 8.0 : 0.0) + (V ? nn * 8.0 * nd : 0.0);
  // two FP64 FFTs of length N2 per pair of time levels (5 N2 log2 N2 flops each), the product (6 N2)
  const double flops = (double)grid * (2.0 * 5.0 * h.rz_n2 * h.rz_log2n2 + 6.0 * h.rz_n2) +
                       nn * (3.0 + (b ? 3.0 : 0.0) + (V ? 2.0 * nd : 0.0));
  ProfScope ps(AAO_K_MATVEC, h.stream, bytes, flops);
#define RZ(IN, MODE, ND)                                                                                     \
  do {                                                                                                       \
    AAO_TRY_CUDA(cudaFuncSetAttribute(k_rz_matvec<IN, MODE, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                      (int)smem));                                                           \
    k_rz_matvec<IN, MODE, ND><<<grid, threads, smem, h.stream>>>(                                            \
        (const IN*)x, y, b, h.nx, h.nt, h.rz_n2, h.rz_log2n2, h.rz_chat, h.rz_tw, V, h.n, h.part, h.scal,    \
        h.counter, m);                                                                                       \
  } while (0)
  if (V && nd > 0) {
    if (x_is_float) {
      switch (nd) {
        case 1: RZ(float, 2, 1); break;
        case 2: RZ(float, 2, 2); break;
        case 3: RZ(float, 2, 3); break;
        case 4: RZ(float, 2, 4); break;
        case 5: RZ(float, 2, 5); break;
        case 6: RZ(float, 2, 6); break;
        case 7: RZ(float, 2, 7); break;
        default: RZ(float, 2, 8); break;
      }
    } else {
      switch (nd) {
        case 1: RZ(double, 2, 1); break;
        case 2: RZ(double, 2, 2); break;
        case 3: RZ(double, 2, 3); break;
        case 4: RZ(double, 2, 4); break;
        case 5: RZ(double, 2, 5); break;
        case 6: RZ(double, 2, 6); break;
        case 7: RZ(double, 2, 7); break;
        default: RZ(double, 2, 8); break;
      }
    }
  } else if (b) {
    if (x_is_float) RZ(float, 1, 0); else RZ(double, 1, 0);
  } else {
    if (x_is_float) RZ(float, 0, 0); else RZ(double, 0, 0);
  }
#undef RZ
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

int riesz_rhs(Handle& h, double* b) {
  const double hx = 2.0 * h.p.s_max / (h.nx + 1);
  k_rz_rhs<<<grid_for(h.n), kThreads, 0, h.stream>>>(b, h.nx, h.nt, h.rz_hcol, h.rz_hrow, h.rz_hcl, h.gL,
                                                      h.p.s_max, hx, h.p.K);
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

int riesz_solve_bins(Handle& h, void* spec) {
  if (h.rz_sym) {
    // W = (Z1 Q) o D, then Z2 = W Q^T (rows: bins; the half spectrum is [k][x]); each product in
    // kGSplit contraction segments, summed in order
    const int ldq = h.rz_ldq;
    const double nq = (double)ldq * ldq;
    ProfScope ps(AAO_K_TRIDIAG, h.stream, 2.0 * (nq * 4.0 + 2.0 * (double)h.K * ldq * 8.0));
    const dim3 grid(ldq / kGN, (h.K + kGB - 1) / kGB, kGSplit);
    const int sgrid = (int)((((size_t)h.K * ldq / 2) + 255) / 256);
    AAO_TRY_CUDA(launch_pdl(k_rz_cgemm, grid, 128, 0, h.stream, (const float2*)spec, h.pitch, (const float*)h.rz_q,
                            ldq, h.rz_part, ldq, h.K, h.pitch / kGSplit));
    AAO_TRY_CUDA(launch_pdl(k_rz_cgemm_sum, sgrid, 256, 0, h.stream, (const float2*)h.rz_part, ldq, h.K, ldq,
                            h.rz_w, ldq, (const float2*)h.rz_dk, ldq));
    AAO_TRY_CUDA(launch_pdl(k_rz_cgemm, grid, 128, 0, h.stream, (const float2*)h.rz_w, ldq, (const float*)h.rz_qt,
                            ldq, h.rz_part, ldq, h.K, ldq / kGSplit));
    AAO_TRY_CUDA(launch_pdl(k_rz_cgemm_sum, sgrid, 256, 0, h.stream, (const float2*)h.rz_part, ldq, h.K, h.pitch,
                            (float2*)spec, h.pitch, (const float2*)nullptr, ldq));
    AAO_CHECK_LAUNCH();
    return AAO_OK;
  }
  const size_t smem = sizeof(float2) * ((size_t)h.nx + kNB);
  const double bytes = (double)h.K * ((double)h.nx * h.nx * 8.0 + 2.0 * h.nx * 8.0);
  ProfScope ps(AAO_K_TRIDIAG, h.stream, bytes);
  k_rz_trsv<<<h.K, 512, smem, h.stream>>>((float2*)spec, h.nx, h.pitch, h.rz_lu, h.rz_dinv, h.il2f);
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

}  // namespace aao

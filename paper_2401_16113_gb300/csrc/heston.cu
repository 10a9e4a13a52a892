// The two-dimensional Heston operator of Sec. 5.1 (Eq. 5.1-5.5) on GB300.
//
//   u_t = 1/2 v s^2 u_ss + sigma rho s v u_sv + 1/2 sigma^2 v u_vv + r s u_s + kappa (eta - v) u_v - r u
//
// and, on the same grid with the same boundary conditions and the same kernels, the SABR operator of
// Sec. 5.2 (Eq. 5.7), D(t) = e^{-rt}:
//
//   u_t = 1/2 v^2 s^(2 beta) D^(2(1-beta)) u_ss + rho sigma s^beta D^(1-beta) v^2 u_sv
//         + 1/2 sigma^2 v^2 u_vv + r s u_s - r u,
//
// with the boundary equation u_t = r s u_s - r u at v = 0 (an all-zero row of A for r = 0). For
// r != 0 the operator depends on time: row k of the AaO system (Eq. 5.8) takes it at t_{k+1/2} (its
// coefficients as three sets, scaled per time level by 1, D^(2(1-beta)) and D^(1-beta)), and step (b)
// takes the time mean of those matrices.
//
// on a uniform grid: s_i = i h_s (i = 1..Ns, h_s = s_max / Ns), v_j = j h_v (j = 0..Nv-1,
// h_v = v_max / Nv); unknown (i, j) of a time level at p = j Ns + i - 1 (Ns Nv unknowns per level,
// so the FFT kernels of steps (a) and (c) see Ns Nv spatial columns). Second-order central
// differences, the mixed derivative by the four-point cross stencil; u(0, v) = 0; u(s, v_max) = s;
// u_s(s_max, v) = 1 through the ghost value u_{Ns+1} = u_{Ns-1} + 2 h_s; at v = 0 the boundary
// equation u_t = kappa eta u_v + r s u_s - r u with u_v = (-3 u_0 + 4 u_1 - u_2) / (2 h_v).
// Every row couples at most the ten offsets (di, dj) in {-1, 0, 1}^2 and (0, 2) (the last only on
// v = 0). The coefficients of (tau/2) A are built on the host in FP64 and kept per unknown.
//
// Kernels:
//   k_hs_matvec  FP64 y = M x (Eq. 2.2) from the stencil: y_t = (x_t - x_{t-1}) - (tau/2) A (x_t + x_{t-1}),
//                fused with the restart residual or the first Gram-Schmidt projections, finished
//                by the last block (the conventions of the other operators' matvecs);
//   k_hs_rhs     b = xi + tau f (f at t_{k+1/2}: constant in time but for SABR with r != 0);
//   step (b) of Eq. 3.2 by block elimination over the v levels. The shifted matrix of bin k,
//                S = mu_k I - tau A, is block tridiagonal in j (blocks Ns x Ns: B_j tridiagonal on
//                the diagonal, A_j and C_j tridiagonal below and above) except for the block E_0
//                (diagonal) that the one-sided u_v puts at (0, 2). At create, per bin:
//                D_0 = B_0, D_j = B_j - A_j G_{j-1}, X_j = D_j^{-1} (batched Gauss-Jordan on the tensor
//                cores, shared with the Riesz operator), G_j = X_j C'_j with C'_1 = C_1 - A_1 H_0 and
//                C'_j = C_j otherwise, H_0 = X_0 E_0. Per apply (k_hs_solve, one cluster of CTAs per bin):
//                w_0 = X_0 r_0, w_j = X_j (r_j - A_j w_{j-1}); x_{Nv-1} = w_{Nv-1},
//                x_j = w_j - G_j x_{j+1} (j >= 1), x_0 = w_0 - G_0 x_1 - H_0 x_2.
#include <math.h>

#include <algorithm>

#include <vector>

#include <cooperative_groups.h>

#include "krylov_dev.cuh"

namespace aao {

namespace {

using namespace kdev;
namespace cg = cooperative_groups;

constexpr int kHsOff = 10;  // stencil offsets, in this order:
__host__ __device__ constexpr int hs_di(int q) { return q < 9 ? (q % 3) - 1 : 0; }
__host__ __device__ constexpr int hs_dj(int q) { return q < 9 ? (q / 3) - 1 : 2; }

// SABR with a nonzero rate: Eq. 5.7 depends on time through D(t) = e^{-rt} (three coefficient sets)
bool hs_time_dependent(const aao_problem& p) { return p.op == AAO_OP_SABR && p.r != 0.0; }

template <typename T> __device__ __forceinline__ double ldx(const T* p) { return (double)*p; }
template <> __device__ __forceinline__ double ldx<float>(const float* p) { return widen(*p); }

// y = M x over all (t, p), by tiles of one time level t and rb v levels (grid-stride over the tiles).
// A tile first stages s = x_t + x_{t-1} on its rows and one row below and two above (the stencil's
// reach; rows outside the grid are zero) in shared memory, then each point sums the stencil from
// there: one FP64 addition per point for s instead of one per point and offset. The sums run over
// the offsets in the same order as a point-by-point evaluation, so y is the same bit for bit. MODE 0:
// y = M x; MODE 1: y = b - M x and ||y||^2 (restart residual; sigma_0, g set by the last block);
// MODE 2: y = M x and the projections V_q . y, q < ND. TD (SABR with r != 0): the coefficient of
// offset q at time level t is c0 + g2[t] c1 + g1[t] c2 from the three sets of c (each kHsOff x nsp),
// g = (g2[0..nt), g1[0..nt)); every offset is summed (no zero test: a zero coefficient multiplies a
// staged value inside the buffer).
template <typename IN, int MODE, int ND, bool TD>
__global__ void __launch_bounds__(256) k_hs_matvec(const IN* __restrict__ x, double* __restrict__ y,
                                                   const double* __restrict__ b, int ns, int nv, int nt, int rb,
                                                   const double* __restrict__ c, const double* __restrict__ g,
                                                   const double* __restrict__ V,
                                                   size_t vstride, double* __restrict__ part,
                                                   double* __restrict__ scal, unsigned int* __restrict__ counter,
                                                   int m) {
  extern __shared__ double s_sm[];  // (rb + 3) x ns: s on v rows j0 - 1 .. j0 + rb + 1
  pdl_sync();
  constexpr int NA = MODE == 2 ? ND : 1;
  double acc[NA];
#pragma unroll
  for (int q = 0; q < NA; ++q) acc[q] = 0.0;
  const int nsp = ns * nv;
  const int nrb = (nv + rb - 1) / rb;
  const int tiles = nt * nrb;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int t = tile / nrb, j0 = (tile - t * nrb) * rb;
    const int j1 = min(nv, j0 + rb);
    double g2 = 1.0, g1 = 1.0;
    if constexpr (TD) {
      g2 = __ldg(g + t);
      g1 = __ldg(g + nt + t);
    }
    const int hn = (j1 - j0 + 3) * ns;  // staged entries
    const IN* xt = x + (size_t)t * nsp;
    const IN* xm = t > 0 ? xt - nsp : nullptr;
    __syncthreads();  // the previous tile's reads of s_sm are done
    for (int e = threadIdx.x; e < hn; e += blockDim.x) {
      const int r = e / ns;
      const int jj = j0 - 1 + r;
      double v = 0.0;
      if (jj >= 0 && jj < nv) {
        const int p = jj * ns + (e - r * ns);
        v = ldx(xt + p) + (xm ? ldx(xm + p) : 0.0);
      }
      s_sm[e] = v;
    }
    __syncthreads();
    const int np = (j1 - j0) * ns;
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
      const int p = j0 * ns + e;  // spatial index; its staged entry is e + ns
      double as = 0.0;            // ((tau/2) A s)_p
      // Zero coefficients are skipped, tested on the bits of a 64-bit integer load (an FP64
      // comparison, which the compiler substitutes for a bit test of a double, takes the FP64 pipe). A nonzero coefficient never reaches past the grid (the boundary couplings are zero:
      // u(0, v) = 0, the ghost node folded into the i - 1 entry, no v - 1 entry on v = 0, u(s, v_max)
      // in the data), so the staged index is only clamped into the buffer; the offset (0, 2)
      // appears on the v = 0 row alone.
#pragma unroll
      for (int q = 0; q < kHsOff; ++q) {
        if (q == kHsOff - 1 && p >= ns) break;
        if constexpr (TD) {
          const size_t o = (size_t)q * nsp + p, cs = (size_t)kHsOff * nsp;
          const double cq = fma(g2, __ldg(c + cs + o), fma(g1, __ldg(c + 2 * cs + o), __ldg(c + o)));
          const int ln = min(max(e + ns + hs_di(q) + hs_dj(q) * ns, 0), hn - 1);
          as = fma(cq, s_sm[ln], as);
        } else {
          const long long cb = __ldg(reinterpret_cast<const long long*>(c) + (size_t)q * nsp + p);
          if ((cb << 1) != 0) {
            const int ln = min(max(e + ns + hs_di(q) + hs_dj(q) * ns, 0), hn - 1);
            as = fma(__longlong_as_double(cb), s_sm[ln], as);
          }
        }
      }
      const double x0 = ldx(xt + p), x1 = xm ? ldx(xm + p) : 0.0;
      double v = (x0 - x1) - as;
      const size_t ge = (size_t)t * nsp + p;
      if (MODE == 1) {
        v = __ldg(b + ge) - v;
        acc[0] = fma(v, v, acc[0]);
      }
      if (AAO_DCHECK(ge < (size_t)nsp * nt)) y[ge] = v;
      if (MODE == 2) {
#pragma unroll
        for (int q = 0; q < ND; ++q) acc[q] = fma(__ldg(V + (size_t)q * vstride + ge), v, acc[q]);
      }
    }
  }
  if constexpr (MODE == 0) return;
  // block partials, then the last block sums them with all its threads (one round trip)
  block_sums_wide<NA>(acc, NA, part + (size_t)blockIdx.x * kPartLd);
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  finish_sums_wide<NA>(part, (int)gridDim.x, NA, [&](int q, double v) {
    if (MODE == 2) {
      scal[S_D1 + q] = v;
    } else {
      scal[S_BETA2] = v;
      const double beta = sqrt(v);
      scal[S_SIG] = beta > 0.0 ? 1.0 / beta : 0.0;
      scal[S_G] = beta;
      for (int k = 1; k <= m; ++k) scal[S_G + k] = 0.0;
      scal[S_FLAG] = isfinite(v) ? 0.0 : 1.0;
    }
  }, counter);
}

// b_t = tau f + [t = 0] (u0 + (tau/2) A u0); with g (time-dependent SABR, the three sets of c and of
// tf as in k_hs_matvec) both at t_{t+1/2}: tau f = tf0 + g2[t] tf1 + g1[t] tf2, and A at t_{1/2}
__global__ void k_hs_rhs(double* __restrict__ b, int ns, int nsp, int nt, const double* __restrict__ c,
                         const double* __restrict__ tf, const double* __restrict__ u0,
                         const double* __restrict__ g) {
  const size_t n = (size_t)nsp * nt, cs = (size_t)kHsOff * nsp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int t = (int)(e / nsp), p = (int)(e - (size_t)t * nsp);
    double v = tf[p];
    if (g) v = fma(g[t], tf[nsp + p], fma(g[nt + t], tf[2 * (size_t)nsp + p], v));
    if (t == 0) {
      double au = 0.0;
      for (int q = 0; q < kHsOff; ++q) {
        double cq = c[(size_t)q * nsp + p];
        if (g) cq = fma(g[0], c[cs + (size_t)q * nsp + p], fma(g[nt], c[2 * cs + (size_t)q * nsp + p], cq));
        const int nb = p + hs_di(q) + hs_dj(q) * ns;
        if (cq != 0.0 && nb >= 0 && nb < nsp) au = fma(cq, u0[nb], au);
      }
      v += u0[p] + au;
    }
    b[e] = v;
  }
}

// ------------------------------------------------------------------------------- step (b): create
// Blocks of S_k = mu_k I - tau A for level j (rows r, columns c in 0..Ns-1); tau A = 2 (tau/2) A, the
// stencil coefficient of offset q at unknown (r, j) being hc[q][j Ns + r] (FP32 copy):
//   B_j[r][r + di] = mu_k [di = 0] - 2 hc[3 + di + 1][..], A_j[r][r + di] = -2 hc[di + 1][..],
//   C_j[r][r + di] = -2 hc[6 + di + 1][..], E_0[r][r] = -2 hc[9][r].
__device__ __forceinline__ float hcoef(const float* __restrict__ hc, int nsp, int q, int p) {
  return -2.f * __ldg(hc + (size_t)q * nsp + p);
}

// D[k] = B_j - A_j G (G = G_{j-1}[k], null for j = 0), one thread per entry, all bins (blockIdx.y)
__global__ void k_hs_form_d(float2* __restrict__ D, const float2* __restrict__ G, int ns, int nsp, int j,
                            const float* __restrict__ hc, const float2* __restrict__ mu) {
  const int k = blockIdx.y;
  const size_t nn = (size_t)ns * ns;
  float2* Dk = D + (size_t)k * nn;
  const float2* Gk = G ? G + (size_t)k * nn : nullptr;
  const float2 muk = mu[k];
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / ns), cc = (int)(e - (size_t)r * ns);
    const int p = j * ns + r;
    float2 v = make_float2(0.f, 0.f);
    const int di = cc - r;
    if (di >= -1 && di <= 1) v.x = hcoef(hc, nsp, 4 + di, p);
    if (di == 0) { v.x += muk.x; v.y += muk.y; }
    if (Gk) {
#pragma unroll
      for (int d = -1; d <= 1; ++d) {
        const int m = r + d;
        if (m < 0 || m >= ns) continue;
        const float a = hcoef(hc, nsp, 1 + d, p);
        if (a != 0.f) {
          const float2 g = Gk[(size_t)m * ns + cc];
          v.x -= a * g.x;
          v.y -= a * g.y;
        }
      }
    }
    Dk[e] = v;
  }
}

// G[k] = X[k] C_j (C_j tridiagonal) - (T ? X[k] T[k] : 0), T dense; one thread per entry
__global__ void k_hs_form_g(float2* __restrict__ G, const float2* __restrict__ X, const float2* __restrict__ T,
                            int ns, int nsp, int j, const float* __restrict__ hc) {
  const int k = blockIdx.y;
  const size_t nn = (size_t)ns * ns;
  const float2* Xk = X + (size_t)k * nn;
  const float2* Tk = T ? T + (size_t)k * nn : nullptr;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / ns), cc = (int)(e - (size_t)r * ns);
    float2 v = make_float2(0.f, 0.f);
    // (X C)[r][cc] = sum_di X[r][cc - di] C[cc - di][cc], C[m][m + di] = -2 hc[7 + di][(m, j)]
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
      const int m = cc - d;
      if (m < 0 || m >= ns) continue;
      const float cm = hcoef(hc, nsp, 7 + d, j * ns + m);
      if (cm != 0.f) {
        const float2 x = Xk[(size_t)r * ns + m];
        v.x += x.x * cm;
        v.y += x.y * cm;
      }
    }
    if (Tk) {
      float ax = 0.f, ay = 0.f;
      for (int m = 0; m < ns; ++m) {
        const float2 x = Xk[(size_t)r * ns + m], t = Tk[(size_t)m * ns + cc];
        ax = fmaf(x.x, t.x, fmaf(-x.y, t.y, ax));
        ay = fmaf(x.x, t.y, fmaf(x.y, t.x, ay));
      }
      v.x -= ax;
      v.y -= ay;
    }
    G[(size_t)k * nn + e] = v;
  }
}

// H[k] = X_0[k] E_0 (E_0 diagonal), and T[k] = A_1 H[k] (A_1 tridiagonal): the pieces of C'_1
__global__ void k_hs_form_h(float2* __restrict__ H, const float2* __restrict__ X0, int ns, int nsp,
                            const float* __restrict__ hc) {
  const int k = blockIdx.y;
  const size_t nn = (size_t)ns * ns;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
    const int cc = (int)(e % ns);
    const float ec = hcoef(hc, nsp, 9, cc);
    const float2 x = X0[(size_t)k * nn + e];
    H[(size_t)k * nn + e] = make_float2(x.x * ec, x.y * ec);
  }
}
__global__ void k_hs_form_t(float2* __restrict__ T, const float2* __restrict__ H, int ns, int nsp,
                            const float* __restrict__ hc) {
  const int k = blockIdx.y;
  const size_t nn = (size_t)ns * ns;
  const float2* Hk = H + (size_t)k * nn;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / ns), cc = (int)(e - (size_t)r * ns);
    const int p = ns + r;  // level j = 1
    float2 v = make_float2(0.f, 0.f);
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
      const int m = r + d;
      if (m < 0 || m >= ns) continue;
      const float a = hcoef(hc, nsp, 1 + d, p);
      const float2 h = Hk[(size_t)m * ns + cc];
      v.x += a * h.x;
      v.y += a * h.y;
    }
    T[(size_t)k * nn + e] = v;
  }
}

// ------------------------------------------------------------------------------- step (b): apply
// A thread-block cluster of C CTAs per bin (kHsThreads threads each). The sweeps are sequential in j,
// and each step is one dense Ns x Ns product, so the CTAs of a cluster split its rows: CTA c owns
// rows [c P, (c + 1) P), P = ceil(Ns / C), and a warp forms two of them at a time (lanes over the
// columns, four loads in flight per row and lane). Each finished entry is written into every CTA's
// copy of the vector (distributed shared memory), and one cluster barrier per step publishes it.
// The copies are double-buffered by the parity of j: a CTA writes step j's vector into slot j & 1
// while a slower CTA may still read step j - 1's from slot (j - 1) & 1, and step j + 1 reuses that
// slot only after the barrier of step j, which every CTA reaches after its reads. w_j reaches the
// bin's spectrum row (global) after that barrier, when no CTA still reads r_j there. Shared
// memory: the product's input t (Ns complex) and the two slots (2 Ns complex).
constexpr int kHsThreads = 256;
constexpr int kHsMaxC = 8;
constexpr int kHsPer = 2;  // entries of a level per thread (Ns <= 512)

// y_i = M_i . vec for the two rows M_0, M_1 (row 1 only if live1); every lane gets both sums.
// U loads per row and lane (U = ceil(Ns / 32) up to 8) are issued before the first is used, so a
// row of up to 256 columns takes one round and no load slot is masked off for the common widths.
template <int U>
__device__ __forceinline__ void dense_rows2(const float2* __restrict__ M0, const float2* __restrict__ M1, bool live1,
                                            const float2* __restrict__ vec, int ns, int lane, float2& y0, float2& y1) {
  float ax0 = 0.f, ay0 = 0.f, ax1 = 0.f, ay1 = 0.f;
  for (int m0 = 0; m0 < ns; m0 += 32 * U) {
    float2 a0[U], a1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int m = m0 + 32 * u + lane;
      a0[u] = m < ns ? __ldg(M0 + m) : make_float2(0.f, 0.f);
      a1[u] = (live1 && m < ns) ? __ldg(M1 + m) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int m = m0 + 32 * u + lane;
      const float2 b = m < ns ? vec[m] : make_float2(0.f, 0.f);
      ax0 = fmaf(a0[u].x, b.x, fmaf(-a0[u].y, b.y, ax0));
      ay0 = fmaf(a0[u].x, b.y, fmaf(a0[u].y, b.x, ay0));
      ax1 = fmaf(a1[u].x, b.x, fmaf(-a1[u].y, b.y, ax1));
      ay1 = fmaf(a1[u].x, b.y, fmaf(a1[u].y, b.x, ay1));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ax0 += __shfl_xor_sync(0xffffffffu, ax0, o);
    ay0 += __shfl_xor_sync(0xffffffffu, ay0, o);
    ax1 += __shfl_xor_sync(0xffffffffu, ax1, o);
    ay1 += __shfl_xor_sync(0xffffffffu, ay1, o);
  }
  y0 = make_float2(ax0, ay0);
  y1 = make_float2(ax1, ay1);
}

// Ask the L2 to fetch rows [r0, r1) of the Ns x Ns block M (one bulk prefetch; the start and end are
// rounded down to 16 bytes, so the range stays inside the block's allocation). A hint only: the
// next step's loads then find the rows in L2 while this step's barrier chain runs.
__device__ __forceinline__ void prefetch_rows_l2(const float2* M, int ns, int r0, int r1) {
  if (r1 <= r0) return;
  const uintptr_t a = reinterpret_cast<uintptr_t>(M + (size_t)r0 * ns);
  const uintptr_t e = reinterpret_cast<uintptr_t>(M + (size_t)r1 * ns);
  const uintptr_t a16 = a & ~(uintptr_t)15, e16 = e & ~(uintptr_t)15;
  if (e16 <= a16) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a16), "r"((unsigned)(e16 - a16)) : "memory");
}

template <int U>
__global__ void __launch_bounds__(kHsThreads) k_hs_solve(float2* __restrict__ spec, int pitch, int ns, int nv,
                                                         const float2* __restrict__ X, const float2* __restrict__ G,
                                                         const float2* __restrict__ H, const float* __restrict__ hc,
                                                         const float2* __restrict__ il2, int K) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* t = reinterpret_cast<float2*>(smraw);
  float2* slot = t + ns;  // slot[(j & 1) * ns + r]
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), c = (int)cl.block_rank();
  pdl_sync();
  const int k = blockIdx.x / C;
  const int nsp = ns * nv;
  const size_t nn = (size_t)ns * ns;
  float2* row = spec + (size_t)k * pitch;
  const float2 sk = il2[k];
  const int P = (ns + C - 1) / C;
  const int r0 = min(ns, c * P), r1 = min(ns, r0 + P);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  float2* peer = lane < C ? cl.map_shared_rank(slot, lane) : nullptr;  // lane q writes CTA q's copy
  const float2* Hk = H + (size_t)k * nn;
  if (threadIdx.x == 0) prefetch_rows_l2(X + (size_t)k * nn, ns, r0, r1);

  // forward: w_j = X_j (r_j - A_j w_{j-1}). For narrow blocks (U <= 4: Ns <= 128, where a step is
  // latency-bound) each thread's entries of r_{j+1} and of the coupling A_{j+1} (at most kHsPer per
  // thread) are loaded into registers before step j's cluster barrier: level j+1 of the spectrum row
  // is written only after step j+1's barrier, so the loads are safe then and the step after the
  // barrier starts from registers instead of an L2 round trip. Wider blocks load them after the
  // barrier (the registers would cost the bandwidth-bound product more than the round trip).
  constexpr bool kPre = U <= 4;
  float2 rr[kHsPer];
  float aa[kHsPer][3];
  auto load_level = [&](int j) {
#pragma unroll
    for (int q = 0; q < kHsPer; ++q) {
      const int r = threadIdx.x + q * kHsThreads, p = j * ns + r;
      rr[q] = r < ns ? row[p] : make_float2(0.f, 0.f);
#pragma unroll
      for (int d = -1; d <= 1; ++d) {
        const int m = r + d;
        aa[q][d + 1] = (j > 0 && r < ns && m >= 0 && m < ns) ? hcoef(hc, nsp, 1 + d, p) : 0.f;
      }
    }
  };
  if (kPre) load_level(0);
  for (int j = 0; j < nv; ++j) {
    if (threadIdx.x == 0)  // the next step's block: X_{j+1}, or G_{nv-2} for the first backward step
      prefetch_rows_l2(j + 1 < nv ? X + ((size_t)(j + 1) * K + k) * nn : G + ((size_t)(nv - 2) * K + k) * nn, ns, r0, r1);
    if (!kPre) load_level(j);
    const float2* wprev = slot + ((j - 1) & 1) * ns;
#pragma unroll
    for (int q = 0; q < kHsPer; ++q) {
      const int r = threadIdx.x + q * kHsThreads;
      if (r >= ns) break;
      float2 v = cmul(rr[q], sk);
      if (j > 0) {
#pragma unroll
        for (int d = -1; d <= 1; ++d) {
          const int m = r + d;
          if (m < 0 || m >= ns) continue;
          const float a = aa[q][d + 1];
          const float2 w = wprev[m];
          v.x -= a * w.x;
          v.y -= a * w.y;
        }
      }
      t[r] = v;
    }
    __syncthreads();
    const float2* Xj = X + ((size_t)j * K + k) * nn;
    const int off = (j & 1) * ns;
    for (int ra = r0 + warp; ra < r1; ra += 2 * nw) {
      const int rb = ra + nw;
      const bool lb = rb < r1;
      float2 ya, yb;
      dense_rows2<U>(Xj + (size_t)ra * ns, Xj + (size_t)(lb ? rb : ra) * ns, lb, t, ns, lane, ya, yb);
      if (peer && AAO_DCHECK(off + ra < 2 * ns)) {
        peer[off + ra] = ya;
        if (lb) peer[off + rb] = yb;
      }
    }
    if (kPre && j + 1 < nv) load_level(j + 1);
    cl.sync();
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x)
      if (AAO_DCHECK(j * ns + r < nsp && nsp <= pitch)) row[j * ns + r] = slot[off + r];
  }
  // backward: x_{nv-1} = w_{nv-1} (in slot (nv - 1) & 1); x_j = w_j - G_j x_{j+1}, and for j = 0
  // also - H_0 x_2 (x_1 in slot 1, x_2 in slot 0). x_0 is needed by no other row, so it goes to
  // the spectrum row only.
  for (int j = nv - 2; j >= 0; --j) {
    if (threadIdx.x == 0 && j > 0) {
      prefetch_rows_l2(G + ((size_t)(j - 1) * K + k) * nn, ns, r0, r1);
      if (j == 1) prefetch_rows_l2(Hk, ns, r0, r1);
    }
    const float2* xnext = slot + ((j + 1) & 1) * ns;
    const float2* Gj = G + ((size_t)j * K + k) * nn;
    const int off = (j & 1) * ns;
    for (int ra = r0 + warp; ra < r1; ra += 2 * nw) {
      const int rb = ra + nw;
      const bool lb = rb < r1;
      float2 sa, sb;
      dense_rows2<U>(Gj + (size_t)ra * ns, Gj + (size_t)(lb ? rb : ra) * ns, lb, xnext, ns, lane, sa, sb);
      if (j == 0) {
        float2 ha, hb;
        dense_rows2<U>(Hk + (size_t)ra * ns, Hk + (size_t)(lb ? rb : ra) * ns, lb, slot, ns, lane, ha, hb);
        sa.x += ha.x;
        sa.y += ha.y;
        sb.x += hb.x;
        sb.y += hb.y;
      }
      const float2 wa = row[j * ns + ra];
      const float2 xa = make_float2(wa.x - sa.x, wa.y - sa.y);
      float2 xb = make_float2(0.f, 0.f);
      if (lb) {
        const float2 wb = row[j * ns + rb];
        xb = make_float2(wb.x - sb.x, wb.y - sb.y);
      }
      if (lane == 0 && AAO_DCHECK(j * ns + ra < nsp)) {
        row[j * ns + ra] = xa;
        if (lb) row[j * ns + rb] = xb;
      }
      if (j > 0 && peer && AAO_DCHECK(off + ra < 2 * ns)) {
        peer[off + ra] = xa;
        if (lb) peer[off + rb] = xb;
      }
    }
    if (j > 0) cl.sync();
  }
}

}  // namespace

// ------------------------------------------------------------------------------- host
AAO_CHECK_WORD_FN(check_word_heston)

namespace {
int hs_grid(size_t n) {
  const size_t g = (n + 255) / 256;
  return (int)(g < (size_t)kRedBlocks ? g : (size_t)kRedBlocks);
}
int hs_grid2(size_t nn) {
  const size_t g = (nn + 255) / 256;
  return (int)(g < 256 ? g : 256);
}
}  // namespace

int heston_pick_cluster(Handle& h);

int heston_build(Handle& h) {
  const aao_problem& p = h.p;
  const int ns = p.nx, nv = p.nv, nsp = ns * nv, K = h.K;
  h.hs_ns = ns;
  h.hs_nv = nv;
  const double hs = p.s_max / ns, hv = p.v_max / nv, tau = h.tau;
  const double r = p.r, kap = p.kappa, eta = p.eta, sig = p.sigma, rho = p.rho;
  const bool sabr = p.op == AAO_OP_SABR;
  // SABR with r != 0: Eq. 5.7 depends on time through D(t) = e^{-rt}; its coefficients are kept as
  // three sets, the terms without D (set 0), the u_ss term at D = 1 (set 1, times D^(2(1-beta)))
  // and the u_sv term at D = 1 (set 2, times D^(1-beta))
  const bool td = hs_time_dependent(p);
  const int nset = td ? 3 : 1;
  const size_t cset = (size_t)kHsOff * nsp;  // one coefficient set
  std::vector<double> c(nset * cset, 0.0), f((size_t)nset * nsp + (td ? 2 * (size_t)h.nt : 0), 0.0), u0(nsp);
  int set = 0;  // the set that add() writes
  // coefficient w of u(ii, jj) in the equation of unknown (i, j) (i, ii 1-based in s)
  auto add = [&](int i, int j, int ii, int jj, double w) {
    const int pt = j * ns + i - 1;
    if (jj == nv) {  // v = v_max: u = s
      f[(size_t)set * nsp + pt] += w * ii * hs;
      return;
    }
    if (ii == 0) return;  // s = 0: u = 0
    if (ii == ns + 1) {   // the ghost beyond s_max: u_{Ns+1} = u_{Ns-1} + 2 h_s
      f[(size_t)set * nsp + pt] += w * 2.0 * hs;
      ii = ns - 1;
    }
    const int di = ii - i, dj = jj - j;
    const int q = dj == 2 ? 9 : (dj + 1) * 3 + (di + 1);
    c[set * cset + (size_t)q * nsp + pt] += w;
  };
  for (int j = 0; j < nv; ++j) {
    const double v = hv * j;
    for (int i = 1; i <= ns; ++i) {
      const double s = hs * i;
      u0[j * ns + i - 1] = s > p.K ? s - p.K : 0.0;  // call payoff
      if (j == 0 && sabr) {  // u_t = r s u_s - r u (nothing for r = 0)
        if (r != 0.0) {
          add(i, 0, i, 0, -r);
          add(i, 0, i + 1, 0, r * s / (2.0 * hs));
          add(i, 0, i - 1, 0, -r * s / (2.0 * hs));
        }
        continue;
      }
      if (td) {  // the three sets of Eq. 5.7's interior row
        const double sb = pow(s, p.beta);
        const double dss = 0.5 * v * v * sb * sb / (hs * hs), dvv = 0.5 * sig * sig * v * v / (hv * hv);
        const double dsv = rho * sig * sb * v * v / (4.0 * hs * hv), cs1 = r * s / (2.0 * hs);
        set = 0;
        add(i, j, i, j, -2.0 * dvv - r);
        add(i, j, i + 1, j, cs1);
        add(i, j, i - 1, j, -cs1);
        add(i, j, i, j + 1, dvv);
        add(i, j, i, j - 1, dvv);
        set = 1;
        add(i, j, i, j, -2.0 * dss);
        add(i, j, i + 1, j, dss);
        add(i, j, i - 1, j, dss);
        set = 2;
        add(i, j, i + 1, j + 1, dsv);
        add(i, j, i - 1, j - 1, dsv);
        add(i, j, i + 1, j - 1, -dsv);
        add(i, j, i - 1, j + 1, -dsv);
        set = 0;
        continue;
      }
      if (j == 0) {  // u_t = kappa eta u_v + r s u_s - r u, u_v one-sided to second order
        add(i, 0, i, 0, -3.0 * kap * eta / (2.0 * hv) - r);
        add(i, 0, i, 1, 4.0 * kap * eta / (2.0 * hv));
        add(i, 0, i, 2, -kap * eta / (2.0 * hv));
        add(i, 0, i + 1, 0, r * s / (2.0 * hs));
        add(i, 0, i - 1, 0, -r * s / (2.0 * hs));
        continue;
      }
      double dss, dvv, dsv, cs, cv;
      if (sabr) {
        const double sb = pow(s, p.beta);  // s^beta; s^(2 beta) = sb^2
        dss = 0.5 * v * v * sb * sb / (hs * hs);
        dvv = 0.5 * sig * sig * v * v / (hv * hv);
        dsv = rho * sig * sb * v * v / (4.0 * hs * hv);
        cs = 0.0;
        cv = 0.0;
      } else {
        dss = 0.5 * v * s * s / (hs * hs);
        dvv = 0.5 * sig * sig * v / (hv * hv);
        dsv = sig * rho * s * v / (4.0 * hs * hv);
        cs = r * s / (2.0 * hs);
        cv = kap * (eta - v) / (2.0 * hv);
      }
      add(i, j, i, j, -2.0 * dss - 2.0 * dvv - r);
      add(i, j, i + 1, j, dss + cs);
      add(i, j, i - 1, j, dss - cs);
      add(i, j, i, j + 1, dvv + cv);
      add(i, j, i, j - 1, dvv - cv);
      add(i, j, i + 1, j + 1, dsv);
      add(i, j, i - 1, j - 1, dsv);
      add(i, j, i + 1, j - 1, -dsv);
      add(i, j, i - 1, j + 1, -dsv);
    }
  }
  for (size_t e = 0; e < c.size(); ++e) c[e] *= 0.5 * tau;  // (tau/2) A
  for (size_t q = 0; q < (size_t)nset * nsp; ++q) f[q] *= tau;  // tau f
  // step (b) takes the time mean of A(t_{k+1/2}) (for constant coefficients A itself): the sets
  // weighted by the means of their factors, in FP32
  double m2 = 1.0, m1 = 1.0;
  if (td) {
    // per time level k the factors g2 = D^(2(1-beta)), g1 = D^(1-beta), D = e^{-r t_{k+1/2}}, kept
    // after the three boundary vectors
    double* g = f.data() + (size_t)3 * nsp;
    m2 = m1 = 0.0;
    for (int k = 0; k < h.nt; ++k) {
      const double D = exp(-r * tau * (k + 0.5));
      g[k] = pow(D, 2.0 * (1.0 - p.beta));
      g[h.nt + k] = pow(D, 1.0 - p.beta);
      m2 += g[k];
      m1 += g[h.nt + k];
    }
    m2 /= h.nt;
    m1 /= h.nt;
  }
  std::vector<float> cf(cset);
  for (size_t e = 0; e < cset; ++e) cf[e] = (float)(td ? c[e] + m2 * c[cset + e] + m1 * c[2 * cset + e] : c[e]);
  auto up = [&](auto** dst, const auto& src) -> int {
    using T = typename std::decay<decltype(src)>::type::value_type;
    AAO_TRY_CUDA(cudaMalloc((void**)dst, sizeof(T) * src.size()));
    AAO_TRY_CUDA(cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, h.stream));
    return AAO_OK;
  };
  AAO_TRY(up(&h.hs_c, c));
  AAO_TRY(up(&h.hs_cf, cf));
  AAO_TRY(up(&h.hs_tf, f));
  AAO_TRY(up(&h.hs_u0, u0));

  // step (b): block elimination over the v levels for every bin at once
  const size_t nn = (size_t)ns * ns, slice = (size_t)K * nn;
  AAO_TRY_CUDA(cudaMalloc(&h.hs_X, sizeof(float2) * slice * nv));
  AAO_TRY_CUDA(cudaMalloc(&h.hs_G, sizeof(float2) * slice * (nv - 1)));
  AAO_TRY_CUDA(cudaMalloc(&h.hs_H, sizeof(float2) * slice));
  float2* T = nullptr;
  AAO_TRY_CUDA(cudaMalloc(&T, sizeof(float2) * slice));
  const dim3 g2(hs_grid2(nn), K);
  int rc = AAO_OK;
  for (int j = 0; j < nv && rc == AAO_OK; ++j) {
    float2* Xj = h.hs_X + (size_t)j * slice;
    k_hs_form_d<<<g2, 256, 0, h.stream>>>(Xj, j > 0 ? h.hs_G + (size_t)(j - 1) * slice : nullptr, ns, nsp, j, h.hs_cf,
                                          h.muf);
    rc = [&]() -> int { AAO_CHECK_LAUNCH(); return AAO_OK; }();
    if (rc == AAO_OK) rc = gj_invert_batched(h.stream, Xj, ns, K);
    if (rc != AAO_OK) break;
    if (j == 0) {
      k_hs_form_h<<<g2, 256, 0, h.stream>>>(h.hs_H, Xj, ns, nsp, h.hs_cf);
      rc = [&]() -> int { AAO_CHECK_LAUNCH(); return AAO_OK; }();
    }
    if (rc == AAO_OK && j == 1) {
      k_hs_form_t<<<g2, 256, 0, h.stream>>>(T, h.hs_H, ns, nsp, h.hs_cf);
      rc = [&]() -> int { AAO_CHECK_LAUNCH(); return AAO_OK; }();
    }
    if (rc == AAO_OK && j < nv - 1) {
      k_hs_form_g<<<g2, 256, 0, h.stream>>>(h.hs_G + (size_t)j * slice, Xj, j == 1 ? T : nullptr, ns, nsp, j,
                                            h.hs_cf);
      rc = [&]() -> int { AAO_CHECK_LAUNCH(); return AAO_OK; }();
    }
  }
  cudaStreamSynchronize(h.stream);
  cudaFree(T);
  if (rc == AAO_OK) rc = heston_pick_cluster(h);
  return rc;
}

int heston_rhs(Handle& h, double* b) {
  const double* g = hs_time_dependent(h.p) ? h.hs_tf + (size_t)3 * h.nx : nullptr;
  k_hs_rhs<<<hs_grid(h.n), 256, 0, h.stream>>>(b, h.hs_ns, h.nx, h.nt, h.hs_c, h.hs_tf, h.hs_u0, g);
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

int heston_matvec(Handle& h, const void* x, bool x_is_float, double* y, const double* b, const double* V, int nd,
                  int m) {
  // tiles of rb v levels: at most about 2048 points, and at least kRedBlocks tiles where the grid
  // allows (small grids otherwise leave SMs idle); an equal number of tiles per block
  const int ns = h.hs_ns, nv = h.hs_nv;
  const int per_t = (kRedBlocks + h.nt - 1) / h.nt;  // v-level blocks per time level wanted
  const int rb = std::max(1, std::min({nv, 2048 / ns, (nv + per_t - 1) / per_t}));
  const size_t tiles = (size_t)h.nt * ((nv + rb - 1) / rb);
  const size_t per = (tiles + kRedBlocks - 1) / kRedBlocks;
  const int grid = (int)((tiles + per - 1) / per);
  const size_t smem = sizeof(double) * (size_t)(rb + 3) * ns;
  const double nn = (double)h.n;
  const bool td = hs_time_dependent(h.p);
  const double* g = td ? h.hs_tf + (size_t)3 * h.nx : nullptr;
  const double bytes = nn * (x_is_float ? 4.0 : 8.0) + nn * 8.0 + (b ? nn * 8.0 : 0.0) + (V ? nn * 8.0 * nd : 0.0) +
                       8.0 * kHsOff * h.nx * (td ? 3 : 1);
  const double flops = nn * (2.0 * kHsOff + 3.0 + (b ? 3.0 : 0.0) + (V ? 2.0 * nd : 0.0));
  ProfScope ps(AAO_K_MATVEC, h.stream, bytes, flops);
#define HS(IN, MODE, ND)                                                                                       \
  do {                                                                                                         \
    if (td)                                                                                                    \
      AAO_TRY_CUDA(launch_pdl(k_hs_matvec<IN, MODE, ND, true>, grid, 256, smem, h.stream, (const IN*)x, y, b, ns, \
                              nv, h.nt, rb, h.hs_c, g, V, h.n, h.part, h.scal, h.counter, m));                  \
    else                                                                                                       \
      AAO_TRY_CUDA(launch_pdl(k_hs_matvec<IN, MODE, ND, false>, grid, 256, smem, h.stream, (const IN*)x, y, b, ns, \
                              nv, h.nt, rb, h.hs_c, g, V, h.n, h.part, h.scal, h.counter, m));                  \
  } while (0)
  if (V && nd > 0) {
    if (x_is_float) {
      switch (nd) {
        case 1: HS(float, 2, 1); break;
        case 2: HS(float, 2, 2); break;
        case 3: HS(float, 2, 3); break;
        case 4: HS(float, 2, 4); break;
        case 5: HS(float, 2, 5); break;
        case 6: HS(float, 2, 6); break;
        case 7: HS(float, 2, 7); break;
        default: HS(float, 2, 8); break;
      }
    } else {
      switch (nd) {
        case 1: HS(double, 2, 1); break;
        case 2: HS(double, 2, 2); break;
        case 3: HS(double, 2, 3); break;
        case 4: HS(double, 2, 4); break;
        case 5: HS(double, 2, 5); break;
        case 6: HS(double, 2, 6); break;
        case 7: HS(double, 2, 7); break;
        default: HS(double, 2, 8); break;
      }
    }
  } else if (b) {
    if (x_is_float) HS(float, 1, 0); else HS(double, 1, 0);
  } else {
    if (x_is_float) HS(float, 0, 0); else HS(double, 0, 0);
  }
#undef HS
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

namespace {
// the instance of k_hs_solve for Ns: U = ceil(Ns / 32) loads per row and lane, at most 8
const void* hs_solve_kernel(int ns) {
  switch ((ns + 31) / 32) {
    case 1: return (const void*)k_hs_solve<1>;
    case 2: return (const void*)k_hs_solve<2>;
    case 3: return (const void*)k_hs_solve<3>;
    case 4: return (const void*)k_hs_solve<4>;
    case 5: return (const void*)k_hs_solve<5>;
    case 6: return (const void*)k_hs_solve<6>;
    case 7: return (const void*)k_hs_solve<7>;
    default: return (const void*)k_hs_solve<8>;
  }
}

cudaLaunchConfig_t hs_solve_config(const Handle& h, int C, cudaLaunchAttribute* attr) {
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(h.K * C);
  cfg.blockDim = dim3(kHsThreads);
  cfg.dynamicSmemBytes = 3 * sizeof(float2) * (size_t)h.hs_ns;
  cfg.stream = h.stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}
}  // namespace

// Cluster size of step (b): the time of one apply goes as (waves of clusters) x (rows per CTA), so
// take C in {1, 2, 4, 8} minimising ceil(K / clusters resident at once) / C; on a tie the smaller C,
// which needs fewer waves (each wave pays the chain of per-step barriers again).
int heston_pick_cluster(Handle& h) {
  int best = 0;
  double cost = 0.0;
  for (int C = 1; C <= kHsMaxC; C <<= 1) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = hs_solve_config(h, C, attr);
    cfg.gridDim = dim3(C);
    int nc = 0;
    AAO_TRY_CUDA(cudaOccupancyMaxActiveClusters(&nc, hs_solve_kernel(h.hs_ns), &cfg));
    if (nc < 1) continue;
    const double c = (double)((h.K + nc - 1) / nc) / C;
    if (best == 0 || c < cost) {
      best = C;
      cost = c;
    }
  }
  if (best == 0) {
    set_error("aao_create: no cluster of the Heston step (b) kernel fits on the GPU");
    return AAO_EUNSUPPORTED;
  }
  h.hs_C = best;
  return AAO_OK;
}

int heston_solve_bins(Handle& h, void* spec) {
  const double nn = (double)h.hs_ns * h.hs_ns;
  const double bytes = (double)h.K * ((2.0 * h.hs_nv) * nn * 8.0 + 2.0 * h.nx * 8.0);
  ProfScope ps(AAO_K_TRIDIAG, h.stream, bytes);
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = hs_solve_config(h, h.hs_C, attr);
  void* args[] = {&spec, (void*)&h.pitch, (void*)&h.hs_ns, (void*)&h.hs_nv, (void*)&h.hs_X, (void*)&h.hs_G,
                  (void*)&h.hs_H, (void*)&h.hs_cf, (void*)&h.il2f, (void*)&h.K};
  AAO_TRY_CUDA(cudaLaunchKernelExC(&cfg, hs_solve_kernel(h.hs_ns), args));
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

}  // namespace aao

// Operator, right-hand side and FGMRES(m) for the CN all-at-once system on GB300.
//
//   k_build_coef  (1/2) tau A(t_{k+1/2}) for Black-Scholes (constant or local volatility),
//                 3-point central differences on S_i = i h; FP64.
//   k_rhs         b = xi + tau f (Eq. 2.2).
//   k_matvec      y = M x, block-bidiagonal M = B1 (x) I - B2 (x) A~ (Eq. 2.2; Eq. 5.8 form for
//                 time-dependent A): y_t = (x_t - x_{t-1}) - (1/2) A~_t (x_t + x_{t-1}), FP64;
//                 optionally r = b - M x with block partial sums of r.r.
//   k_mdot / k_update / k_vnext / k_givens / k_lsq / k_xupdate
//                 right-preconditioned flexible GMRES(m) (Sec. 5): classical Gram-Schmidt
//                 applied twice, Givens rotations, FP64 throughout. Block partial sums are
//                 reduced in a fixed order, so results are deterministic.
#include <math.h>
#include <stdio.h>

#include <chrono>
#include <complex>
#include <vector>

#include "aao_internal.cuh"

namespace aao {

namespace {

constexpr int kRedBlocks = 1216;  // 152 SMs x 8: partial-sum blocks of the reductions
constexpr int kThreads = 256;

// device scalar slots (offsets into Handle::scal)
enum : int {
  S_H1 = 0,        // 128 first-pass projections
  S_H2 = 128,      // 128 second-pass projections
  S_NRM2 = 256,    // ||w'||^2
  S_EST = 257,     // |g_{j+1}|
  S_HN = 258,      // h_{j+1,j}
  S_INVHN = 259,   // 1 / h_{j+1,j}
  S_BETA2 = 260,   // ||r||^2
  S_INVB = 261,    // 1 / ||r||
  S_FLAG = 262,    // non-finite detected
  S_G = 320,       // g (m+1)
  S_CS = 400,      // cosines (m)
  S_SN = 480,      // sines (m)
  S_Y = 560,       // least-squares solution (m)
  S_HMAT = 640,    // Hessenberg, column-major (m+1) x m, ld 65
  S_TOTAL = 640 + 65 * 64
};
constexpr int kLdH = 65;

template <typename T> __device__ __forceinline__ double ld(const T* p) { return (double)__ldg(p); }

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
    D[e] = half_tau * (-2.0 * diff - r);
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
      double xi = u0(i) + D[i] * u0(i);
      if (i > 0) xi += L[i] * u0(i - 1);
      if (i < nx - 1) xi += U[i] * u0(i + 1);
      val += xi;
    }
    b[e] = val;
  }
}

// y = M x  (b == nullptr)   or   y = b - M x with partial sums of y.y  (b != nullptr)
template <typename IN>
__global__ void __launch_bounds__(kThreads) k_matvec(const IN* __restrict__ x, double* __restrict__ y,
                                                     const double* __restrict__ b, int nx, int nt,
                                                     const double* __restrict__ L, const double* __restrict__ D,
                                                     const double* __restrict__ U, int rows,
                                                     double* __restrict__ part) {
  const size_t n = (size_t)nx * nt;
  double acc[1] = {0.0};
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int t = (int)(e / nx), i = (int)(e - (size_t)t * nx);
    const size_t c = (rows == 1) ? (size_t)i : e;
    const double xc = ld(x + e);
    const double xl = i > 0 ? ld(x + e - 1) : 0.0;
    const double xr = i < nx - 1 ? ld(x + e + 1) : 0.0;
    double pc = 0.0, pl = 0.0, pr = 0.0;
    if (t > 0) {
      pc = ld(x + e - nx);
      pl = i > 0 ? ld(x + e - nx - 1) : 0.0;
      pr = i < nx - 1 ? ld(x + e - nx + 1) : 0.0;
    }
    double v = xc - pc;
    v = fma(-__ldg(L + c), xl + pl, v);
    v = fma(-__ldg(D + c), xc + pc, v);
    v = fma(-__ldg(U + c), xr + pr, v);
    if (b) {
      v = __ldg(b + e) - v;
      acc[0] = fma(v, v, acc[0]);
    }
    y[e] = v;
  }
  if (b) block_sums<1>(acc, 1, part + blockIdx.x);
}

// part[blk * nv + i] = sum over the block's elements of V_i . w  (nv <= 8 per launch chunk)
__global__ void __launch_bounds__(kThreads) k_mdot(const double* __restrict__ V, int nv, size_t n,
                                                   const double* __restrict__ w, double* __restrict__ part,
                                                   int part_ld) {
  double acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double wv = __ldg(w + e);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < nv) acc[q] = fma(__ldg(V + (size_t)q * n + e), wv, acc[q]);
  }
  block_sums<8>(acc, nv, part + (size_t)blockIdx.x * part_ld);
}

// w <- w - sum_i h_i V_i ; part[blk*ld + i] = V_i . w (i < nv, chunked by 8) and part[.. + nv] = w.w
__global__ void __launch_bounds__(kThreads) k_update(double* __restrict__ w, const double* __restrict__ V,
                                                     int nv, size_t n, const double* __restrict__ hc,
                                                     double* __restrict__ part, int part_ld) {
  __shared__ double hs[128];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = hc[i];
  __syncthreads();
  for (int c0 = 0; c0 <= nv; c0 += 8) {
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
      double wv;
      if (c0 == 0) {
        wv = w[e];
        for (int i = 0; i < nv; ++i) wv = fma(-hs[i], __ldg(V + (size_t)i * n + e), wv);
        w[e] = wv;
      } else {
        wv = w[e];
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int i = c0 + q;
        if (i < nv) acc[q] = fma(__ldg(V + (size_t)i * n + e), wv, acc[q]);
        else if (i == nv) acc[q] = fma(wv, wv, acc[q]);
      }
    }
    const int cnt = (nv + 1 - c0) < 8 ? (nv + 1 - c0) : 8;
    block_sums<8>(acc, cnt, part + (size_t)blockIdx.x * part_ld + c0);
  }
}

// out[i] = sum_blk part[blk*ld + i], fixed order; one warp per value
__global__ void k_reduce(const double* __restrict__ part, int nblk, int cnt, int ld, double* __restrict__ out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= cnt) return;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += part[(size_t)b * ld + warp];
  s = warp_sum(s);
  if (lane == 0) out[warp] = s;
}

// v_next = (w - sum_i h2_i V_i) / h_{j+1,j}
__global__ void __launch_bounds__(kThreads) k_vnext(const double* __restrict__ w, const double* __restrict__ V,
                                                    int nv, size_t n, const double* __restrict__ scal,
                                                    double* __restrict__ out) {
  __shared__ double hs[128];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = scal[S_H2 + i];
  __syncthreads();
  const double inv = scal[S_INVHN];
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double wv = __ldg(w + e);
    for (int i = 0; i < nv; ++i) wv = fma(-hs[i], __ldg(V + (size_t)i * n + e), wv);
    out[e] = wv * inv;
  }
}

// Hessenberg column j from the two Gram-Schmidt passes, previous rotations, new rotation.
__global__ void k_givens(double* __restrict__ scal, int j) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* H = scal + S_HMAT + (size_t)j * kLdH;
  double h2n = 0.0;
  for (int i = 0; i <= j; ++i) {
    const double a = scal[S_H1 + i], c = scal[S_H2 + i];
    H[i] = a + c;
    h2n += c * c;
  }
  double hn2 = scal[S_NRM2] - h2n;
  const double hn = hn2 > 0.0 ? sqrt(hn2) : 0.0;
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
  scal[S_INVHN] = hn > 0.0 ? 1.0 / hn : 0.0;
  if (!isfinite(rho) || !isfinite(hn)) scal[S_FLAG] = 1.0;
}

// y = H(0:jd, 0:jd)^{-1} g(0:jd), upper triangular after the rotations
__global__ void k_lsq(double* __restrict__ scal, int jd) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = jd - 1; i >= 0; --i) {
    double s = scal[S_G + i];
    for (int k = i + 1; k < jd; ++k) s -= scal[S_HMAT + (size_t)k * kLdH + i] * scal[S_Y + k];
    scal[S_Y + i] = s / scal[S_HMAT + (size_t)i * kLdH + i];
  }
}

// x += sum_i y_i Z_i
template <typename ZT>
__global__ void __launch_bounds__(kThreads) k_xupdate(double* __restrict__ x, const ZT* __restrict__ Z, int jd,
                                                      size_t n, const double* __restrict__ scal) {
  __shared__ double ys[128];
  for (int i = threadIdx.x; i < jd; i += blockDim.x) ys[i] = scal[S_Y + i];
  __syncthreads();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double v = x[e];
    for (int i = 0; i < jd; ++i) v = fma(ys[i], (double)__ldg(Z + (size_t)i * n + e), v);
    x[e] = v;
  }
}

// v = r / ||r||, starts a cycle: g = (beta, 0, ...)
__global__ void __launch_bounds__(kThreads) k_start(const double* __restrict__ r, double* __restrict__ v, size_t n,
                                                    double* __restrict__ scal, int m) {
  const double beta = sqrt(scal[S_BETA2]);
  const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    v[e] = r[e] * inv;
  if (blockIdx.x == 0 && threadIdx.x <= m) scal[S_G + threadIdx.x] = threadIdx.x == 0 ? beta : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) scal[S_FLAG] = 0.0;
}

__global__ void __launch_bounds__(kThreads) k_dot_self(const double* __restrict__ v, size_t n, double* part) {
  double acc[1] = {0.0};
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double a = __ldg(v + e);
    acc[0] = fma(a, a, acc[0]);
  }
  block_sums<1>(acc, 1, part + blockIdx.x);
}

int grid_for(size_t n) {
  size_t g = (n + kThreads - 1) / kThreads;
  return (int)(g < (size_t)kRedBlocks ? g : (size_t)kRedBlocks);
}

int reduce_to(Handle& h, int nblk, int cnt, int ld, double* out) {
  const int warps = cnt;
  const int threads = 256;
  const int blocks = (warps * 32 + threads - 1) / threads;
  ProfScope ps(AAO_K_OTHER, h.stream, 8.0 * (double)nblk * cnt);
  k_reduce<<<blocks, threads, 0, h.stream>>>(h.part, nblk, cnt, ld, out);
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

int ensure_workspace(Handle& h, int m) {
  if (h.ws_m >= m && h.V) return AAO_OK;
  if (h.V) cudaFree(h.V);
  if (h.Z) cudaFree(h.Z);
  h.V = nullptr; h.Z = nullptr; h.ws_m = 0;
  AAO_TRY_CUDA(cudaMalloc(&h.V, sizeof(double) * h.n * (size_t)(m + 1)));
  AAO_TRY_CUDA(cudaMalloc(&h.Z, (h.mixed ? sizeof(float) : sizeof(double)) * h.n * (size_t)m));
  h.ws_m = m;
  return AAO_OK;
}

}  // namespace

// ----------------------------------------------------------------------------------------
// tables
// ----------------------------------------------------------------------------------------

int build_tables(Handle& h) {
  const aao_problem& p = h.p;
  const int nx = h.nx, nt = h.nt, N = nt;
  h.tau = p.T / nt;
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
  AAO_TRY(up(&h.pL, pl)); AAO_TRY(up(&h.pD, pd)); AAO_TRY(up(&h.pU, pu));
  AAO_TRY(up(&h.pLf, plf)); AAO_TRY(up(&h.pDf, pdf)); AAO_TRY(up(&h.pUf, puf));
  AAO_TRY(up(&h.mu, mu)); AAO_TRY(up(&h.il2, il2)); AAO_TRY(up(&h.tw, tw));
  AAO_TRY(up(&h.muf, muf)); AAO_TRY(up(&h.il2f, il2f)); AAO_TRY(up(&h.twf, twf));
  AAO_TRY(up(&h.lam, lam)); AAO_TRY(up(&h.ilam, ilam));
  AAO_TRY(up(&h.lamf, lamf)); AAO_TRY(up(&h.ilamf, ilamf));

  const size_t csz = h.mixed ? sizeof(float2) : sizeof(double2);
  AAO_TRY_CUDA(cudaMalloc(&h.spec, csz * (size_t)K * h.pitch));
  AAO_TRY_CUDA(cudaMalloc(&h.w, sizeof(double) * h.n));
  AAO_TRY_CUDA(cudaMalloc(&h.scal, sizeof(double) * S_TOTAL));
  AAO_TRY_CUDA(cudaMemsetAsync(h.scal, 0, sizeof(double) * S_TOTAL, h.stream));
  h.part_blocks = kRedBlocks;
  AAO_TRY_CUDA(cudaMalloc(&h.part, sizeof(double) * (size_t)kRedBlocks * 136));
  AAO_TRY_CUDA(cudaMallocHost(&h.host_scal, sizeof(double) * 8));
  // the temporary gS buffer must outlive the build kernel
  AAO_TRY_CUDA(cudaStreamSynchronize(h.stream));
  cudaFree(d_gS);
  return AAO_OK;
}

void free_handle(Handle& h) {
  void* bufs[] = {h.mL, h.mD, h.mU, h.gL, h.gR, h.pL, h.pD, h.pU, h.pLf, h.pDf, h.pUf, h.mu, h.il2, h.tw,
                  h.muf, h.il2f, h.twf, h.lam, h.ilam, h.lamf, h.ilamf, h.spec, h.V, h.Z, h.w, h.scal, h.part};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (h.host_scal) cudaFreeHost(h.host_scal);
}

// ----------------------------------------------------------------------------------------
// operator launches
// ----------------------------------------------------------------------------------------

int launch_matvec(Handle& h, const void* x, bool x_is_float, double* y, const double* b) {
  const int g = grid_for(h.n);
  const double nn = (double)h.n;
  // x once, coefficients (3 per row of the time-dependent operator), y, and b if present
  const double bytes = nn * (x_is_float ? 4.0 : 8.0) + 3.0 * 8.0 * (double)h.nx * h.coef_rows + nn * 8.0 +
                       (b ? nn * 8.0 : 0.0);
  ProfScope ps(AAO_K_MATVEC, h.stream, bytes);
  if (x_is_float)
    k_matvec<float><<<g, kThreads, 0, h.stream>>>((const float*)x, y, b, h.nx, h.nt, h.mL, h.mD, h.mU, h.coef_rows, h.part);
  else
    k_matvec<double><<<g, kThreads, 0, h.stream>>>((const double*)x, y, b, h.nx, h.nt, h.mL, h.mD, h.mU, h.coef_rows, h.part);
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

int launch_rhs(Handle& h, double* b) {
  k_rhs<<<grid_for(h.n), kThreads, 0, h.stream>>>(b, h.nx, h.nt, h.mL, h.mD, h.mU, h.coef_rows, h.gL, h.gR,
                                                   h.p.s_max / (h.nx + 1), h.p.K, h.p.payoff);
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

// ----------------------------------------------------------------------------------------
// FGMRES(m)
// ----------------------------------------------------------------------------------------

namespace {

int residual(Handle& h, const double* b, const double* x, double* r, double* beta2_host) {
  AAO_TRY(launch_matvec(h, x, false, r, b));
  const int g = grid_for(h.n);
  AAO_TRY(reduce_to(h, g, 1, 1, h.scal + S_BETA2));
  AAO_TRY_CUDA(cudaMemcpyAsync(h.host_scal, h.scal + S_BETA2, sizeof(double), cudaMemcpyDeviceToHost, h.stream));
  AAO_TRY_CUDA(cudaStreamSynchronize(h.stream));
  *beta2_host = h.host_scal[0];
  return AAO_OK;
}

}  // namespace

int run_fgmres(Handle& h, const double* b, double* x, double tol, int m, int maxit, aao_stats* st) {
  const auto t0 = std::chrono::steady_clock::now();
  const uint64_t l0 = g_launches.load();
  AAO_TRY(ensure_workspace(h, m));
  const size_t n = h.n;
  const int g = grid_for(n);
  const size_t zsz = h.mixed ? sizeof(float) : sizeof(double);
  char* Zb = reinterpret_cast<char*>(h.Z);

  // ||b||
  k_dot_self<<<g, kThreads, 0, h.stream>>>(b, n, h.part);
  AAO_CHECK_LAUNCH();
  AAO_TRY(reduce_to(h, g, 1, 1, h.scal + S_BETA2));
  AAO_TRY_CUDA(cudaMemcpyAsync(h.host_scal, h.scal + S_BETA2, sizeof(double), cudaMemcpyDeviceToHost, h.stream));
  AAO_TRY_CUDA(cudaStreamSynchronize(h.stream));
  const double bnorm = sqrt(h.host_scal[0]);

  int its = 0, restarts = 0, status = AAO_OK;
  double rel = 0.0, est = 0.0;
  if (!(bnorm > 0.0)) {
    AAO_TRY_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, h.stream));
    AAO_TRY_CUDA(cudaStreamSynchronize(h.stream));
    status = isfinite(bnorm) ? AAO_OK : AAO_BREAKDOWN;
  } else {
    for (;;) {
      double beta2 = 0.0;
      AAO_TRY(residual(h, b, x, h.w, &beta2));
      const double beta = sqrt(beta2);
      rel = beta / bnorm;
      if (!isfinite(beta)) { status = AAO_BREAKDOWN; break; }
      if (beta <= tol * bnorm) { status = AAO_OK; break; }
      if (its >= maxit) { status = AAO_NOT_CONVERGED; break; }
      k_start<<<g, kThreads, 0, h.stream>>>(h.w, h.V, n, h.scal, m);
      AAO_CHECK_LAUNCH();
      int jd = 0;
      bool stop_cycle = false;
      for (int j = 0; j < m && !stop_cycle; ++j) {
        double* Vj = h.V + (size_t)j * n;
        void* Zj = Zb + zsz * (size_t)j * n;
        AAO_TRY(launch_precond(h, Vj, Zj, h.mixed));
        AAO_TRY(launch_matvec(h, Zj, h.mixed, h.w, nullptr));
        const int nv = j + 1;
        // first Gram-Schmidt pass: projections in chunks of 8 basis vectors
        for (int c0 = 0; c0 < nv; c0 += 8) {
          const int cnt = (nv - c0) < 8 ? (nv - c0) : 8;
          ProfScope ps(AAO_K_ARNOLDI, h.stream, 8.0 * (double)n * (cnt + 1));
          k_mdot<<<g, kThreads, 0, h.stream>>>(h.V + (size_t)c0 * n, cnt, n, h.w, h.part + c0, 136);
          AAO_CHECK_LAUNCH();
        }
        AAO_TRY(reduce_to(h, g, nv, 136, h.scal + S_H1));
        // subtract, second pass projections and ||w'||^2
        {
          ProfScope ps(AAO_K_ARNOLDI, h.stream, 8.0 * (double)n * (nv + 2));
          k_update<<<g, kThreads, 0, h.stream>>>(h.w, h.V, nv, n, h.scal + S_H1, h.part, 136);
        }
        AAO_CHECK_LAUNCH();
        AAO_TRY(reduce_to(h, g, nv + 1, 136, h.scal + S_H2));  // S_H2[0..nv) and S_H2[nv] = ||w'||^2
        // move ||w'||^2 to its slot
        AAO_TRY_CUDA(cudaMemcpyAsync(h.scal + S_NRM2, h.scal + S_H2 + nv, sizeof(double), cudaMemcpyDeviceToDevice, h.stream));
        k_givens<<<1, 32, 0, h.stream>>>(h.scal, j);
        AAO_CHECK_LAUNCH();
        AAO_TRY_CUDA(cudaMemcpyAsync(h.host_scal, h.scal + S_EST, sizeof(double) * 2, cudaMemcpyDeviceToHost, h.stream));
        AAO_TRY_CUDA(cudaMemcpyAsync(h.host_scal + 2, h.scal + S_FLAG, sizeof(double), cudaMemcpyDeviceToHost, h.stream));
        AAO_TRY_CUDA(cudaStreamSynchronize(h.stream));
        est = h.host_scal[0];
        const double hn = h.host_scal[1];
        ++its;
        jd = j + 1;
        if (h.host_scal[2] != 0.0 || !isfinite(est)) { stop_cycle = true; status = AAO_BREAKDOWN; break; }
        if (est <= tol * bnorm || hn <= 1e-300 || its >= maxit) { stop_cycle = true; break; }
        {
          ProfScope ps(AAO_K_ARNOLDI, h.stream, 8.0 * (double)n * (nv + 2));
          k_vnext<<<g, kThreads, 0, h.stream>>>(h.w, h.V, nv, n, h.scal, h.V + (size_t)(j + 1) * n);
        }
        AAO_CHECK_LAUNCH();
      }
      if (status == AAO_BREAKDOWN) break;
      k_lsq<<<1, 32, 0, h.stream>>>(h.scal, jd);
      AAO_CHECK_LAUNCH();
      if (h.mixed)
        k_xupdate<float><<<g, kThreads, 0, h.stream>>>(x, (const float*)h.Z, jd, n, h.scal);
      else
        k_xupdate<double><<<g, kThreads, 0, h.stream>>>(x, (const double*)h.Z, jd, n, h.scal);
      AAO_CHECK_LAUNCH();
      ++restarts;
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

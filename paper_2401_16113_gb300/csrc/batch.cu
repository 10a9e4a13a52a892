// Batched AaO solves in one persistent launch.
//
// Each CTA takes the next instance from a queue (largest first) and runs the whole
// right-preconditioned FGMRES(m) of that instance by itself: the P_alpha^{-1} apply (FFT tiles
// along t, shifted tridiagonal solves by groups of threads, inverse FFT tiles), the CN matvec
// fused with the first Gram-Schmidt projections, the update, the Givens rotations and the
// convergence test. All reductions are CTA-local, so an instance never waits on another CTA
// and never goes back to the host; each instance carries its own status (its convergence
// mask). The same arithmetic as the single-instance path (precond_dev.cuh, krylov_dev.cuh):
// FP32-complex preconditioner, FP64 matvec, Gram-Schmidt, Givens and solution update.
//
// batch_submit replays a CUDA graph (pointer upload, queue reset, the persistent kernel,
// status download) captured on the first call. The FFT column tile of every nt class is
// autotuned at aao_batch_create.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <chrono>
#include <complex>
#include <map>
#include <string>
#include <vector>

#include <cooperative_groups.h>

#include "krylov_dev.cuh"
#include "precond_dev.cuh"

namespace cg = cooperative_groups;

namespace aao {
namespace {

using namespace kdev;
using namespace pdev;

constexpr int kBT = 256;       // threads of a batched-solver CTA
constexpr int kCH = 16;        // tridiagonal rows per thread (at most)
constexpr int kMaxM = 40;      // restart length bound of the batched solver
constexpr int kMaxC = 8;       // largest cluster (CTAs per instance)

struct BatchInst {
  int nx, nt, log2n, K, pitch, P, tgrp, ch, cs, rows, m, pad;
  MrPlan mr;  // stages of the mixed-radix transform (nst = 0: nt is a power of two)
  size_t n;
  const double* b;
  double* x;
  double* V;
  float* Z;
  float2* spec;
  const double *mL, *mD, *mU;
  const float *pL, *pD, *pU;
  const float2 *mu, *il2, *tw;
  const float *lam, *ilam;
  double* scal;
};

// ---------------------------------------------------------------- cluster-level building blocks
// A cluster of C CTAs (C = cluster size) works on one instance. Work is split by cluster rank;
// phases that read what other CTAs wrote are separated by cluster barriers (release/acquire at
// cluster scope, so global-memory writes before the barrier are visible after it). Sums are
// formed per CTA, then every CTA adds the C partials from distributed shared memory in rank
// order: all CTAs hold identical, deterministic totals. Each CTA keeps its own copy of the
// instance's scalars (Hessenberg, Givens, scales) and runs the scalar updates redundantly.

struct Ctx {
  int rank, C;
};

__device__ __forceinline__ Ctx ctx() {
  cg::cluster_group cl = cg::this_cluster();
  return Ctx{(int)cl.block_rank(), (int)cl.num_blocks()};
}

__device__ __forceinline__ void cluster_sync() { cg::this_cluster().sync(); }

// cluster sum of CNT per-thread accumulators -> out[0..cnt) (CTA-local shared, in every CTA)
template <int CNT>
__device__ __forceinline__ void cluster_sums(const double (&acc)[CNT], int cnt, double* part_sm, double* out) {
  block_sums<CNT>(acc, cnt, part_sm);
  cg::cluster_group cl = cg::this_cluster();
  cl.sync();
  if (threadIdx.x < cnt) {
    double s = 0.0;
    for (unsigned r = 0; r < cl.num_blocks(); ++r) s += cl.map_shared_rank(part_sm, r)[threadIdx.x];
    out[threadIdx.x] = s;
  }
  cl.sync();
}

// y = M x over the instance: warp (rank, w) takes work items rank*8 + w, + C*8, ... (32-column
// strip x 16 time levels)
template <typename IN, int MODE, int ND, int NA>
__device__ __forceinline__ void cl_matvec(const BatchInst& I, Ctx c, const IN* x, double* y, const double* b,
                                          const double* V, double (&acc)[NA]) {
  const int warp = threadIdx.x >> 5;
  const int strips = (I.nx + kMvCols - 1) / kMvCols, chunks = (I.nt + 15) / 16;
  for (int it = c.rank * (kBT / 32) + warp; it < strips * chunks; it += c.C * (kBT / 32)) {
    const int sidx = it % strips, cidx = it / strips;
    const int t0 = cidx * 16, t1 = min(I.nt, t0 + 16);
    matvec_item<IN, MODE, ND, NA>(x, y, b, I.nx, t0, t1, sidx * kMvCols, I.mL, I.mD, I.mU, I.rows, V, I.n, acc);
  }
}

// restart residual r = b - M x into V_0; ||r||^2 -> out[0]
__device__ __noinline__ void cl_residual(const BatchInst& I, Ctx c, double* psm, double* out) {
  double acc[1] = {0.0};
  cl_matvec<double, 1, 0, 1>(I, c, I.x, I.V, I.b, nullptr, acc);
  cluster_sums<1>(acc, 1, psm, out);
}

// W = M z_j with the first-pass projections V_q . W (q < ND) -> out[0..ND) (||W||^2 is recovered
// by the update from ||W'||^2 and the projections)
template <int ND>
__device__ __noinline__ void cl_matvec_proj(const BatchInst& I, Ctx c, const float* z, double* W, double* psm,
                                            double* out) {
  double acc[ND];
#pragma unroll
  for (int q = 0; q < ND; ++q) acc[q] = 0.0;
  cl_matvec<float, 2, ND, ND>(I, c, z, W, nullptr, I.V, acc);
  cluster_sums<ND>(acc, ND, psm, out);
}

// the twiddle table of the mixed-radix tiles, after their two P x nt buffers
__device__ __forceinline__ float2* cl_mr_twiddles(const BatchInst& I, unsigned char* smem) {
  float2* stw = reinterpret_cast<float2*>(smem) + 2 * (size_t)I.P * I.nt;
  for (int m = threadIdx.x; m < I.nt; m += blockDim.x) stw[m] = I.tw[m];
  return stw;  // made visible by the first barrier of the tile
}

// P_alpha^{-1} (scale * v) -> z (FP32), Eq. 3.2 with Remark 1; tiles and bins split by rank. nt
// a power of two: the register or shared-memory tiles; otherwise the mixed-radix tiles (two
// buffers of P x nt and the twiddle table in shared memory).
__device__ __noinline__ void cl_precond(const BatchInst& I, Ctx c, const double* v, float scale, float* z,
                                        unsigned char* smem) {
  const int W = 2 * I.P;
  if (I.mr.nst > 0) {
    const int lp = __ffs(I.P) - 1;
    float2* b0 = reinterpret_cast<float2*>(smem);
    const float2* stw = cl_mr_twiddles(I, smem);
    for (int x0 = c.rank * W; x0 < I.nx; x0 += c.C * W) {
      fft_fwd_mr_tile<float, double, kBT>(v, I.spec, I.nx, I.nt, I.mr, lp, I.pitch, I.lam, scale, x0, b0,
                                          b0 + (size_t)I.P * I.nt, stw);
      __syncthreads();
    }
  } else {
    for (int x0 = c.rank * W; x0 < I.nx; x0 += c.C * W) {
      fft_fwd_tile<float>(v, I.spec, I.nx, I.nt, I.log2n, I.P, I.pitch, I.lam, I.tw, scale, x0, smem);
      __syncthreads();
    }
  }
  cluster_sync();
  const int G = kBT / I.tgrp;
  const int g = threadIdx.x / I.tgrp, tid = threadIdx.x - g * I.tgrp;
  const size_t gbytes = ((size_t)I.tgrp * I.cs + 8 * (size_t)I.tgrp) * sizeof(float2);
  float* sa = reinterpret_cast<float*>(smem);
  float* sd = sa + (size_t)I.tgrp * I.cs;
  float* sc = sd + (size_t)I.tgrp * I.cs;
  unsigned char* groups = smem + (((3 * (size_t)I.tgrp * I.cs * sizeof(float)) + 15) & ~(size_t)15);
  tridiag_stage<float>(I.pL, I.pD, I.pU, I.nx, I.tgrp, I.ch, I.cs, sa, sd, sc);
  __syncthreads();
  for (int k0 = c.rank * G; k0 < I.K; k0 += c.C * G) {
    const int k = k0 + g;
    tridiag_bin<float, kCH>(I.spec, I.nx, I.pitch, I.ch, I.cs, sa, sd, sc, I.mu, I.il2, k < I.K ? k : 0, tid,
                            I.tgrp, k < I.K, groups + g * gbytes);
    __syncthreads();
  }
  cluster_sync();
  if (I.mr.nst > 0) {
    const int lp = __ffs(I.P) - 1;
    float2* b0 = reinterpret_cast<float2*>(smem);
    const float2* stw = cl_mr_twiddles(I, smem);
    for (int x0 = c.rank * W; x0 < I.nx; x0 += c.C * W) {
      fft_inv_mr_tile<float, float, kBT>(I.spec, z, I.nx, I.nt, I.mr, lp, I.pitch, I.ilam, x0, b0,
                                         b0 + (size_t)I.P * I.nt, stw);
      __syncthreads();
    }
  } else {
    for (int x0 = c.rank * W; x0 < I.nx; x0 += c.C * W) {
      fft_inv_tile<float, float>(I.spec, z, I.nx, I.nt, I.log2n, I.P, I.pitch, I.ilam, I.tw, x0, smem);
      __syncthreads();
    }
  }
  cluster_sync();
}

// out[c0 + q] = V_{c0+q} . w, q < CNT <= 8 (into this CTA's scalar copy)
template <int CNT>
__device__ __noinline__ void cl_mdot_t(const BatchInst& I, Ctx c, int c0, const double* w, double* out, double* psm,
                                       double* tot) {
  double acc[CNT];
#pragma unroll
  for (int q = 0; q < CNT; ++q) acc[q] = 0.0;
  const double* Vc = I.V + (size_t)c0 * I.n;
  for (size_t e = (size_t)c.rank * kBT + threadIdx.x; e < I.n; e += (size_t)c.C * kBT) {
    const double wv = w[e];
#pragma unroll
    for (int q = 0; q < CNT; ++q) acc[q] = fma(Vc[(size_t)q * I.n + e], wv, acc[q]);
  }
  cluster_sums<CNT>(acc, CNT, psm, tot);
  if (threadIdx.x < CNT) out[c0 + threadIdx.x] = tot[threadIdx.x];
  __syncthreads();
}

__device__ void cl_mdot(const BatchInst& I, Ctx c, int c0, int cnt, const double* w, double* out, double* psm,
                        double* tot) {
  switch (cnt) {
    case 1: cl_mdot_t<1>(I, c, c0, w, out, psm, tot); break;
    case 2: cl_mdot_t<2>(I, c, c0, w, out, psm, tot); break;
    case 3: cl_mdot_t<3>(I, c, c0, w, out, psm, tot); break;
    case 4: cl_mdot_t<4>(I, c, c0, w, out, psm, tot); break;
    case 5: cl_mdot_t<5>(I, c, c0, w, out, psm, tot); break;
    case 6: cl_mdot_t<6>(I, c, c0, w, out, psm, tot); break;
    case 7: cl_mdot_t<7>(I, c, c0, w, out, psm, tot); break;
    default: cl_mdot_t<8>(I, c, c0, w, out, psm, tot); break;
  }
}

// Gram-Schmidt pass: w -= sum sigma_i^2 d_i V_i, then ||w||^2; thread 0 of every CTA decides on a
// second pass or runs the Givens update of column j on its own scalar copy
__device__ __noinline__ void cl_update(const BatchInst& I, Ctx c, double* scal, int j, int pass, double* w,
                                       double* psm, double* tot) {
  const int nv = j + 1;
  const int off = pass == 1 ? S_D1 : S_D2;
  __shared__ double cf[kMaxM + 1];
  for (int i = threadIdx.x; i < nv; i += kBT) {
    const double si = scal[S_SIG + i];
    cf[i] = si * si * scal[off + i];
  }
  __syncthreads();
  double acc[1] = {0.0};
  for (size_t e = (size_t)c.rank * kBT + threadIdx.x; e < I.n; e += (size_t)c.C * kBT) {
    double wv = w[e];
    for (int q = 0; q < nv; ++q) wv = fma(-cf[q], I.V[(size_t)q * I.n + e], wv);
    w[e] = wv;
    acc[0] = fma(wv, wv, acc[0]);
  }
  cluster_sums<1>(acc, 1, psm, tot);
  if (threadIdx.x == 0) {
    const double v = tot[0];
    scal[S_WP2] = v;
    // ||w||^2 = ||w'||^2 + sum_i (sigma_i d_i)^2 (Pythagoras over the orthonormal basis)
    double wn2 = v;
    if (pass == 1)
      for (int i = 0; i < nv; ++i) {
        const double hi = scal[S_SIG + i] * scal[S_D1 + i];
        wn2 = fma(hi, hi, wn2);
      }
    if (pass == 1 && v < kReorthEta * kReorthEta * wn2) {
      scal[S_REORTH] = 1.0;
    } else {
      scal[S_REORTH] = 0.0;
      givens_column(scal, j, scal + S_D1, pass == 2 ? scal + S_D2 : nullptr);
    }
  }
  __syncthreads();
}

// x += sum_{i<jd} y_i Z_i, y = H^{-1} g
__device__ __noinline__ void cl_xupdate(const BatchInst& I, Ctx c, const double* scal, int jd) {
  __shared__ double ys[kMaxM];
  if (threadIdx.x == 0) {
    for (int i = jd - 1; i >= 0; --i) {
      double s = scal[S_G + i];
      for (int k = i + 1; k < jd; ++k) s -= scal[S_HMAT + (size_t)k * kLdH + i] * ys[k];
      ys[i] = s / scal[S_HMAT + (size_t)i * kLdH + i];
    }
  }
  __syncthreads();
  for (size_t e = (size_t)c.rank * kBT + threadIdx.x; e < I.n; e += (size_t)c.C * kBT) {
    double v = I.x[e];
    for (int i = 0; i < jd; ++i) v = fma(ys[i], widen(I.Z[(size_t)i * I.n + e]), v);
    I.x[e] = v;
  }
  cluster_sync();
}

// FGMRES(m) of one instance by one cluster
__device__ __noinline__ void cl_solve(const BatchInst& I, Ctx c, double tol, int maxit, aao_stats* st,
                                      unsigned char* smem) {
  __shared__ double psm[16];
  __shared__ double tot[16];
  double* scal = I.scal + (size_t)c.rank * S_TOTAL;
  const int m = I.m;
  {
    double acc[1] = {0.0};
    for (size_t e = (size_t)c.rank * kBT + threadIdx.x; e < I.n; e += (size_t)c.C * kBT)
      acc[0] = fma(I.b[e], I.b[e], acc[0]);
    cluster_sums<1>(acc, 1, psm, tot);
  }
  const double bnorm = sqrt(tot[0]);
  int its = 0, restarts = 0, status = AAO_OK;
  double rel = 0.0, est = 0.0;
  if (!(bnorm > 0.0)) {
    for (size_t e = (size_t)c.rank * kBT + threadIdx.x; e < I.n; e += (size_t)c.C * kBT) I.x[e] = 0.0;
    status = isfinite(bnorm) ? AAO_OK : AAO_BREAKDOWN;
  } else {
    for (;;) {
      cl_residual(I, c, psm, tot);
      const double beta = sqrt(tot[0]);
      rel = beta / bnorm;
      if (!isfinite(beta)) { status = AAO_BREAKDOWN; break; }
      if (beta <= tol * bnorm) { status = AAO_OK; break; }
      if (its >= maxit) { status = AAO_NOT_CONVERGED; break; }
      if (threadIdx.x == 0) {
        scal[S_SIG] = 1.0 / beta;
        scal[S_G] = beta;
        for (int k = 1; k <= m; ++k) scal[S_G + k] = 0.0;
        scal[S_FLAG] = 0.0;
      }
      __syncthreads();
      int jd = 0;
      for (int j = 0; j < m; ++j) {
        double* Vj = I.V + (size_t)j * I.n;
        double* W = I.V + (size_t)(j + 1) * I.n;
        float* Zj = I.Z + (size_t)j * I.n;
        cl_precond(I, c, Vj, (float)scal[S_SIG + j], Zj, smem);
        const int nv = j + 1;
        const int nf = nv < 8 ? nv : 8;
        switch (nf) {
          case 1: cl_matvec_proj<1>(I, c, Zj, W, psm, tot); break;
          case 2: cl_matvec_proj<2>(I, c, Zj, W, psm, tot); break;
          case 3: cl_matvec_proj<3>(I, c, Zj, W, psm, tot); break;
          case 4: cl_matvec_proj<4>(I, c, Zj, W, psm, tot); break;
          case 5: cl_matvec_proj<5>(I, c, Zj, W, psm, tot); break;
          case 6: cl_matvec_proj<6>(I, c, Zj, W, psm, tot); break;
          case 7: cl_matvec_proj<7>(I, c, Zj, W, psm, tot); break;
          default: cl_matvec_proj<8>(I, c, Zj, W, psm, tot); break;
        }
        if (threadIdx.x < nf) scal[S_D1 + threadIdx.x] = tot[threadIdx.x];
        __syncthreads();
        for (int c0 = 8; c0 < nv; c0 += 8) cl_mdot(I, c, c0, min(8, nv - c0), W, scal + S_D1, psm, tot);
        cl_update(I, c, scal, j, 1, W, psm, tot);
        if (scal[S_REORTH] != 0.0) {
          for (int c0 = 0; c0 < nv; c0 += 8) cl_mdot(I, c, c0, min(8, nv - c0), W, scal + S_D2, psm, tot);
          cl_update(I, c, scal, j, 2, W, psm, tot);
        }
        est = scal[S_EST];
        const double hn = scal[S_HN];
        const bool bad = scal[S_FLAG] != 0.0 || !isfinite(est);
        __syncthreads();
        ++its;
        jd = j + 1;
        if (bad) { status = AAO_BREAKDOWN; break; }
        if (est <= tol * bnorm || hn <= 1e-300 || its >= maxit) break;
      }
      if (status == AAO_BREAKDOWN) break;
      cl_xupdate(I, c, scal, jd);
      ++restarts;
    }
  }
  if (c.rank == 0 && threadIdx.x == 0) {
    st->status = status;
    st->iterations = its;
    st->restarts = restarts;
    st->launches = 0;
    st->rel_residual = rel;
    st->est_residual = est / (bnorm > 0 ? bnorm : 1.0);
    st->ms = 0.0;
  }
  cluster_sync();
}

// mode 0: solve; mode 1: two preconditioner applies only (FFT tile tuning). Rank 0 of each
// cluster takes the next instance from the queue and the cluster reads it from its shared memory.
__global__ void __launch_bounds__(kBT, 2) k_batch(const BatchInst* __restrict__ insts, const int* __restrict__ order,
                                                  int n, unsigned int* __restrict__ next, double tol, int maxit,
                                                  aao_stats* __restrict__ st, int mode) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int cur;
  const Ctx c = ctx();
  cg::cluster_group cl = cg::this_cluster();
  for (;;) {
    if (c.rank == 0 && threadIdx.x == 0) cur = (int)atomicAdd(next, 1u);
    cl.sync();
    const int q = *cl.map_shared_rank(&cur, 0);
    cl.sync();
    if (q >= n) return;
    const int id = order[q];
    const BatchInst& I = insts[id];
    if (mode == 1) {
      cl_precond(I, c, I.V, 1.0f, I.Z, smem);
      cl_precond(I, c, I.V, 1.0f, I.Z, smem);
    } else {
      cl_solve(I, c, tol, maxit, st + id, smem);
    }
  }
}

size_t al(size_t b) { return (b + 255) & ~size_t(255); }

int tile_P(int nt, int cap) {
  int P = 16;
  while (P > 1 && P * nt > cap) P >>= 1;
  return P;
}

// the largest FFT tile of an nt class within the batch kernel's shared memory: P nt <= 16 kBT
// complex for the power-of-two tiles, 2 P nt <= 16 kBT for the mixed-radix ones (two buffers)
int tile_P_max(int nt) {
  const bool pow2 = (nt & (nt - 1)) == 0;
  return tile_P(nt, pow2 ? 16 * kBT : 8 * kBT);
}

}  // namespace

// ---------------------------------------------------------------- host side

struct Batch {
  int n = 0, m = 0;
  cudaStream_t user = 0, s = 0;
  void* pool = nullptr;
  BatchInst* d_inst = nullptr;
  int* d_order = nullptr;
  unsigned int* d_next = nullptr;
  aao_stats* d_st = nullptr;
  std::vector<BatchInst> inst;
  std::vector<aao_problem> prob;
  std::vector<int> order;
  BatchInst* h_inst = nullptr;      // pinned copy of the descriptors (graph upload source)
  aao_stats* h_st = nullptr;        // pinned
  std::vector<double*> gL, gR;      // per instance Dirichlet values (device)
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  double g_tol = -1.0;
  int g_maxit = -1;
  size_t smem = 0;
  int C = 4;          // CTAs per instance (thread-block cluster size)
  int nclusters = 1;  // clusters resident at once for C
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

// host tables of one instance (same definitions as the single-instance path)
void host_tables(const aao_problem& p, int nx, int nt, std::vector<float>& pl, std::vector<float>& pd,
                 std::vector<float>& pu, std::vector<float2>& mu, std::vector<float2>& il2,
                 std::vector<float2>& tw, std::vector<float>& lam, std::vector<float>& ilam) {
  const double tau = p.T / nt;
  const double hS = p.s_max / (nx + 1);
  const double bump = p.op == AAO_OP_LOCALVOL ? p.lv_bump : 0.0;
  const double tslope = p.op == AAO_OP_LOCALVOL ? p.lv_tslope : 0.0;
  double cm = 0.0, c2m = 0.0;
  for (int k = 0; k < nt; ++k) {
    const double c = 1.0 + tslope * tau * (k + 0.5);
    cm += c;
    c2m += c * c;
  }
  cm /= nt;
  c2m /= nt;
  pl.resize(nx); pd.resize(nx); pu.resize(nx);
  for (int i = 0; i < nx; ++i) {
    const double S = hS * (i + 1), l = log(S / p.K);
    const double bi = bump * exp(-l * l);
    const double s2 = p.sigma * p.sigma + 2.0 * p.sigma * bi * cm + bi * bi * c2m;
    const double ii = i + 1.0;
    const double diff = 0.5 * s2 * ii * ii, conv = 0.5 * p.r * ii;
    pl[i] = (float)(tau * (diff - conv));
    pd[i] = (float)(tau * (-2.0 * diff - p.r));
    pu[i] = (float)(tau * (diff + conv));
  }
  const int K = nt / 2 + 1;
  const double a = pow(p.alpha, 1.0 / nt);
  mu.resize(K); il2.resize(K); tw.resize(nt); lam.resize(nt); ilam.resize(nt);
  for (int k = 0; k < K; ++k) {
    const double ang = -2.0 * M_PI * (double)k / nt;
    const std::complex<double> wk(cos(ang), sin(ang));
    const std::complex<double> l1 = 1.0 - a * wk, l2 = 0.5 * (1.0 + a * wk);
    const std::complex<double> q = l1 / l2, il = 1.0 / l2;
    mu[k] = make_float2((float)q.real(), (float)q.imag());
    il2[k] = make_float2((float)il.real(), (float)il.imag());
  }
  for (int t = 0; t < nt; ++t) {
    const double ang = -2.0 * M_PI * (double)t / nt;
    tw[t] = make_float2((float)cos(ang), (float)sin(ang));
    const double l = pow(p.alpha, (double)t / nt);
    lam[t] = (float)l;
    ilam[t] = (float)(1.0 / (l * nt));
  }
}

// launch the persistent kernel with clusters of B.C CTAs, as many clusters as fit at once
int launch_k_batch(Batch& B, int mode, double tol, int maxit) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = B.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kBT);
  cfg.dynamicSmemBytes = B.smem;
  cfg.stream = B.s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(B.C * std::min(B.n, B.nclusters));
  AAO_TRY_CUDA(cudaLaunchKernelEx(&cfg, k_batch, (const BatchInst*)B.d_inst, (const int*)B.d_order, B.n, B.d_next,
                                  tol, maxit, B.d_st, mode));
  return AAO_OK;
}

int set_cluster(Batch& B, int C) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kBT);
  cfg.dynamicSmemBytes = B.smem;
  cfg.gridDim = dim3(C);
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nc = 0;
  AAO_TRY_CUDA(cudaOccupancyMaxActiveClusters(&nc, (const void*)k_batch, &cfg));
  if (nc < 1) {
    set_error("aao_batch: no cluster of this size fits on the GPU");
    return AAO_EUNSUPPORTED;
  }
  B.C = C;
  B.nclusters = nc;
  return AAO_OK;
}

int run_batch(Batch& B, int mode, double tol, int maxit) {
  AAO_TRY_CUDA(cudaMemsetAsync(B.d_next, 0, sizeof(unsigned int), B.s));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return launch_k_batch(B, mode, tol, maxit);
}

// FFT column tile per nt class: time two preconditioner applies of that class's instances
// with the largest admissible tile and with half of it; keep the faster (results are identical).
int tune_tiles(Batch& B) {
  std::map<int, std::vector<int>> cls;
  for (int i = 0; i < B.n; ++i) cls[B.inst[i].nt].push_back(i);
  cudaEvent_t e0, e1;
  AAO_TRY_CUDA(cudaEventCreate(&e0));
  AAO_TRY_CUDA(cudaEventCreate(&e1));
  int rc = AAO_OK;
  for (auto& kv : cls) {
    const int nt = kv.first;
    const std::vector<int>& ids = kv.second;
    const int pmax = tile_P_max(nt);
    int bestP = pmax;
    float best = 1e30f;
    for (int P = pmax; P >= 1 && P >= pmax / 4 && rc == AAO_OK; P >>= 1) {
      for (int i : ids) B.inst[i].P = P;
      memcpy(B.h_inst, B.inst.data(), sizeof(BatchInst) * B.n);
      if (cudaMemcpyAsync(B.d_inst, B.h_inst, sizeof(BatchInst) * B.n, cudaMemcpyHostToDevice, B.s) != cudaSuccess ||
          cudaMemcpyAsync(B.d_order, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice, B.s) != cudaSuccess) {
        rc = AAO_ECUDA;
        break;
      }
      // run_batch uses B.n; time only this class
      const int n_save = B.n;
      B.n = (int)ids.size();
      cudaEventRecord(e0, B.s);
      rc = run_batch(B, 1, 1.0, 1);
      cudaEventRecord(e1, B.s);
      B.n = n_save;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; bestP = P; }
    }
    for (int i : ids) B.inst[i].P = bestP;
  }
  memcpy(B.h_inst, B.inst.data(), sizeof(BatchInst) * B.n);
  if (rc == AAO_OK && cudaMemcpyAsync(B.d_inst, B.h_inst, sizeof(BatchInst) * B.n, cudaMemcpyHostToDevice, B.s) != cudaSuccess)
    rc = AAO_ECUDA;
  // cluster size: time the preconditioner pass over the whole batch (largest first) for each size
  if (rc == AAO_OK) {
    std::vector<int> ord(B.n);
    for (int i = 0; i < B.n; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return B.inst[a].n > B.inst[b].n; });
    if (cudaMemcpyAsync(B.d_order, ord.data(), sizeof(int) * B.n, cudaMemcpyHostToDevice, B.s) != cudaSuccess) rc = AAO_ECUDA;
    float best = 1e30f;
    int bestC = B.C;
    for (int C : {2, 4, 8}) {
      if (rc != AAO_OK) break;
      if (set_cluster(B, C) != AAO_OK) continue;
      cudaEventRecord(e0, B.s);
      rc = run_batch(B, 1, 1.0, 1);
      cudaEventRecord(e1, B.s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; bestC = C; }
    }
    if (rc == AAO_OK) rc = set_cluster(B, bestC);
  }
  cudaStreamSynchronize(B.s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace

void launch_rhs_raw(cudaStream_t s, double* b, int nx, int nt, const double* L, const double* D, const double* U,
                    int rows, const double* gL, const double* gR, double h, double K, int payoff);
void launch_coef_raw(cudaStream_t s, double* L, double* D, double* U, int nx, int rows, double h, double half_tau,
                     double sigma, double r, double bump, double tslope, double tau, const double* gS);

}  // namespace aao

struct aao_batch {
  aao::Batch B;
};

using namespace aao;

static void batch_free(Batch& B) {
  if (B.exec) cudaGraphExecDestroy(B.exec);
  if (B.graph) cudaGraphDestroy(B.graph);
  if (B.pool) cudaFree(B.pool);
  if (B.h_inst) cudaFreeHost(B.h_inst);
  if (B.h_st) cudaFreeHost(B.h_st);
  if (B.ev0) cudaEventDestroy(B.ev0);
  if (B.ev1) cudaEventDestroy(B.ev1);
  if (B.s) cudaStreamDestroy(B.s);
}

extern "C" int aao_batch_create(const aao_problem* ps, int n, int m, aao_batch** out) {
  if (!out) { set_error("aao_batch_create: null output"); return AAO_EINVAL; }
  *out = nullptr;
  if (!ps || n < 1) { set_error("aao_batch_create: need n >= 1 problems"); return AAO_EINVAL; }
  if (m < 1 || m > kMaxM) { set_error("aao_batch_create: need 1 <= m <= 40"); return AAO_EINVAL; }
  for (int i = 0; i < n; ++i) {
    const aao_problem& p = ps[i];
    MrPlan pl;
    const bool radix_ok = p.nt > 0 && mr_plan(p.nt, pl);  // prime factors 2, 3, 5 and 7 only
    if ((p.op != AAO_OP_BS && p.op != AAO_OP_LOCALVOL) || p.precision != AAO_MIXED || !radix_ok || p.nt < 2 ||
        p.nt > 4096 || p.nx < 2 || p.nx > 4096 || !(p.T > 0) || !(p.K > 0) || !(p.sigma > 0) || !(p.s_max > 0) ||
        !(p.r >= 0) || !(p.alpha > 0) || !(p.alpha <= 1) || (p.payoff != AAO_PUT && p.payoff != AAO_CALL)) {
      char buf[200];
      snprintf(buf, sizeof buf,
               "aao_batch_create: problem %d unsupported (mixed precision, op BS or LOCALVOL, "
               "2 <= nt <= 4096 with prime factors 2, 3, 5, 7 only, 2 <= nx <= 4096, valid parameters)", i);
      set_error(buf);
      return AAO_EINVAL;
    }
  }
  aao_batch* bt = new aao_batch();
  Batch& B = bt->B;
  B.n = n;
  B.m = m;
  B.user = (cudaStream_t)ps[0].stream;
  B.prob.assign(ps, ps + n);
  auto fail = [&](int code) {
    batch_free(B);
    delete bt;
    return code;
  };
#define BTRY(expr)                                                                        \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      set_error(std::string("aao_batch_create: ") + #expr + ": " + cudaGetErrorString(e_)); \
      return fail(e_ == cudaErrorMemoryAllocation ? AAO_ENOMEM : AAO_ECUDA);              \
    }                                                                                     \
  } while (0)
  BTRY(cudaStreamCreateWithFlags(&B.s, cudaStreamNonBlocking));
  BTRY(cudaEventCreateWithFlags(&B.ev0, cudaEventDisableTiming));
  BTRY(cudaEventCreateWithFlags(&B.ev1, cudaEventDisableTiming));

  // layout of the pool
  struct Off { size_t V, Z, spec, mL, mD, mU, gL, gR, gS, tab, scal; size_t pl, pd, pu, mu, il2, tw, lam, ilam; };
  std::vector<Off> off(n);
  size_t o = 0;
  B.inst.resize(n);
  for (int i = 0; i < n; ++i) {
    const aao_problem& p = ps[i];
    const int nx = p.nx, nt = p.nt, K = nt / 2 + 1, pitch = ((nx + 63) / 64) * 64;
    const size_t nn = (size_t)nx * nt;
    const int rows = p.op == AAO_OP_LOCALVOL ? nt : 1;
    Off& f = off[i];
    f.V = o; o = al(o + sizeof(double) * nn * (m + 1));
    f.Z = o; o = al(o + sizeof(float) * nn * m);
    f.spec = o; o = al(o + sizeof(float2) * (size_t)K * pitch);
    f.mL = o; o = al(o + sizeof(double) * (size_t)nx * rows);
    f.mD = o; o = al(o + sizeof(double) * (size_t)nx * rows);
    f.mU = o; o = al(o + sizeof(double) * (size_t)nx * rows);
    f.gL = o; o = al(o + sizeof(double) * (nt + 1));
    f.gR = o; o = al(o + sizeof(double) * (nt + 1));
    f.gS = o; o = al(o + sizeof(double) * nx);
    f.scal = o; o = al(o + sizeof(double) * S_TOTAL * kMaxC);  // one scalar copy per cluster rank
    f.tab = o;
    f.pl = o; o = al(o + sizeof(float) * nx);
    f.pd = o; o = al(o + sizeof(float) * nx);
    f.pu = o; o = al(o + sizeof(float) * nx);
    f.mu = o; o = al(o + sizeof(float2) * K);
    f.il2 = o; o = al(o + sizeof(float2) * K);
    f.tw = o; o = al(o + sizeof(float2) * nt);
    f.lam = o; o = al(o + sizeof(float) * nt);
    f.ilam = o; o = al(o + sizeof(float) * nt);
    BatchInst& I = B.inst[i];
    I.nx = nx; I.nt = nt; I.K = K; I.pitch = pitch; I.rows = rows; I.m = m; I.n = nn;
    int l = 0;
    while ((1 << l) < nt) ++l;
    I.log2n = l;
    I.tgrp = 32 * ((nx + 32 * kCH - 1) / (32 * kCH));
    if (I.tgrp > kBT) { set_error("aao_batch_create: nx too large"); return fail(AAO_EINVAL); }
    I.ch = (nx + I.tgrp - 1) / I.tgrp;
    if (I.ch < 2) I.ch = 2;
    I.cs = (I.ch & 1) ? I.ch + 2 : I.ch + 1;
    I.P = tile_P_max(nt);
    if (!(nt & (nt - 1))) I.mr.nst = 0;
    else mr_plan(nt, I.mr);
  }
  const size_t tail = o;
  size_t dsz = al(sizeof(BatchInst) * n) + al(sizeof(int) * n) + 256 + al(sizeof(aao_stats) * n);
  BTRY(cudaMalloc(&B.pool, tail + dsz));
  char* base = static_cast<char*>(B.pool);
  B.d_inst = reinterpret_cast<BatchInst*>(base + tail);
  B.d_order = reinterpret_cast<int*>(base + tail + al(sizeof(BatchInst) * n));
  B.d_next = reinterpret_cast<unsigned int*>(base + tail + al(sizeof(BatchInst) * n) + al(sizeof(int) * n));
  B.d_st = reinterpret_cast<aao_stats*>(base + tail + al(sizeof(BatchInst) * n) + al(sizeof(int) * n) + 256);
  BTRY(cudaMallocHost(&B.h_inst, sizeof(BatchInst) * n));
  BTRY(cudaMallocHost(&B.h_st, sizeof(aao_stats) * n));
  BTRY(cudaMemsetAsync(B.pool, 0, tail, B.s));  // workspace and scalars start defined

  // tables (host, staged in one pinned buffer per instance region), coefficients (device)
  size_t smem = 0;
  for (int i = 0; i < n; ++i) {
    const aao_problem& p = ps[i];
    const Off& f = off[i];
    BatchInst& I = B.inst[i];
    std::vector<float> pl, pd, pu, lam, ilam;
    std::vector<float2> mu, il2, tw;
    host_tables(p, I.nx, I.nt, pl, pd, pu, mu, il2, tw, lam, ilam);
    const size_t tab_end = f.ilam + sizeof(float) * I.nt;
    std::vector<char> stage(tab_end - f.tab, 0);  // this instance's table region
    auto put = [&](size_t at, const void* src, size_t bytes) { memcpy(stage.data() + (at - f.tab), src, bytes); };
    put(f.pl, pl.data(), sizeof(float) * I.nx);
    put(f.pd, pd.data(), sizeof(float) * I.nx);
    put(f.pu, pu.data(), sizeof(float) * I.nx);
    put(f.mu, mu.data(), sizeof(float2) * I.K);
    put(f.il2, il2.data(), sizeof(float2) * I.K);
    put(f.tw, tw.data(), sizeof(float2) * I.nt);
    put(f.lam, lam.data(), sizeof(float) * I.nt);
    put(f.ilam, ilam.data(), sizeof(float) * I.nt);
    BTRY(cudaMemcpyAsync(base + f.tab, stage.data(), stage.size(), cudaMemcpyHostToDevice, B.s));
    // Dirichlet values and the local-volatility shape exp(-ln^2(S/K))
    std::vector<double> gl(I.nt + 1), gr(I.nt + 1), gS(I.nx);
    const double tau = p.T / I.nt, hS = p.s_max / (I.nx + 1);
    for (int k = 0; k <= I.nt; ++k) {
      const double disc = p.K * exp(-p.r * tau * k);
      gl[k] = p.payoff == AAO_PUT ? disc : 0.0;
      gr[k] = p.payoff == AAO_PUT ? 0.0 : p.s_max - disc;
    }
    for (int x = 0; x < I.nx; ++x) {
      const double l = log(hS * (x + 1) / p.K);
      gS[x] = exp(-l * l);
    }
    BTRY(cudaMemcpyAsync(base + f.gL, gl.data(), sizeof(double) * (I.nt + 1), cudaMemcpyHostToDevice, B.s));
    BTRY(cudaMemcpyAsync(base + f.gR, gr.data(), sizeof(double) * (I.nt + 1), cudaMemcpyHostToDevice, B.s));
    BTRY(cudaMemcpyAsync(base + f.gS, gS.data(), sizeof(double) * I.nx, cudaMemcpyHostToDevice, B.s));
    BTRY(cudaStreamSynchronize(B.s));  // host staging buffers are released at scope end
    double* mL = reinterpret_cast<double*>(base + f.mL);
    double* mD = reinterpret_cast<double*>(base + f.mD);
    double* mU = reinterpret_cast<double*>(base + f.mU);
    launch_coef_raw(B.s, mL, mD, mU, I.nx, I.rows, hS, 0.5 * tau, p.sigma, p.r,
                    p.op == AAO_OP_LOCALVOL ? p.lv_bump : 0.0, p.op == AAO_OP_LOCALVOL ? p.lv_tslope : 0.0, tau,
                    reinterpret_cast<const double*>(base + f.gS));
    BTRY(cudaGetLastError());
    I.V = reinterpret_cast<double*>(base + f.V);
    I.Z = reinterpret_cast<float*>(base + f.Z);
    I.spec = reinterpret_cast<float2*>(base + f.spec);
    I.mL = mL; I.mD = mD; I.mU = mU;
    I.pL = reinterpret_cast<const float*>(base + f.pl);
    I.pD = reinterpret_cast<const float*>(base + f.pd);
    I.pU = reinterpret_cast<const float*>(base + f.pu);
    I.mu = reinterpret_cast<const float2*>(base + f.mu);
    I.il2 = reinterpret_cast<const float2*>(base + f.il2);
    I.tw = reinterpret_cast<const float2*>(base + f.tw);
    I.lam = reinterpret_cast<const float*>(base + f.lam);
    I.ilam = reinterpret_cast<const float*>(base + f.ilam);
    I.scal = reinterpret_cast<double*>(base + f.scal);
    B.gL.push_back(reinterpret_cast<double*>(base + f.gL));
    B.gR.push_back(reinterpret_cast<double*>(base + f.gR));
    // shared memory: the FFT tile and twiddles ((P + 1) * nt complex, P * nt <= 16 * kBT) or the
    // staged diagonals plus the tridiagonal groups
    const size_t tri_b = ((3 * (size_t)I.tgrp * I.cs * sizeof(float) + 15) & ~(size_t)15) +
                         (size_t)(kBT / I.tgrp) * ((size_t)I.tgrp * I.cs + 8 * (size_t)I.tgrp) * sizeof(float2);
    smem = std::max(smem, tri_b);
    smem = std::max(smem, (size_t)(16 * kBT + I.nt) * sizeof(float2));
  }
  B.smem = smem;
  BTRY(cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  BTRY(cudaStreamSynchronize(B.s));
  int rc = set_cluster(B, 4);
  if (rc == AAO_OK) rc = tune_tiles(B);
  if (rc != AAO_OK) return fail(rc);
  B.order.resize(n);
  for (int i = 0; i < n; ++i) B.order[i] = i;
  std::stable_sort(B.order.begin(), B.order.end(), [&](int a, int b) { return B.inst[a].n > B.inst[b].n; });
  BTRY(cudaMemcpyAsync(B.d_order, B.order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, B.s));
  BTRY(cudaStreamSynchronize(B.s));
  *out = bt;
  return AAO_OK;
#undef BTRY
}

extern "C" int aao_batch_rhs(aao_batch* bt, double* const* b) {
  if (!bt || !b) { set_error("aao_batch_rhs: null argument"); return AAO_EINVAL; }
  Batch& B = bt->B;
  AAO_TRY_CUDA(cudaEventRecord(B.ev0, B.user));
  AAO_TRY_CUDA(cudaStreamWaitEvent(B.s, B.ev0, 0));
  for (int i = 0; i < B.n; ++i) {
    if (!b[i]) { set_error("aao_batch_rhs: null b pointer"); return AAO_EINVAL; }
    const aao_problem& p = B.prob[i];
    const BatchInst& I = B.inst[i];
    launch_rhs_raw(B.s, b[i], I.nx, I.nt, I.mL, I.mD, I.mU, I.rows, B.gL[i], B.gR[i], p.s_max / (I.nx + 1), p.K,
                   p.payoff);
    AAO_CHECK_LAUNCH();
  }
  AAO_TRY_CUDA(cudaEventRecord(B.ev1, B.s));
  AAO_TRY_CUDA(cudaStreamWaitEvent(B.user, B.ev1, 0));
  return AAO_OK;
}

extern "C" int batch_submit(aao_batch* bt, double* const* b, double* const* x, double tol, int maxit,
                            aao_stats* st) {
  NvtxRange nv("batch_submit");
  if (!bt || !b || !x) { set_error("batch_submit: null argument"); return AAO_EINVAL; }
  if (!(tol > 0) || maxit < 1) { set_error("batch_submit: need tol > 0 and maxit >= 1"); return AAO_EINVAL; }
  Batch& B = bt->B;
  const auto t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < B.n; ++i) {
    if (!b[i] || !x[i]) { set_error("batch_submit: null vector pointer"); return AAO_EINVAL; }
    B.inst[i].b = b[i];
    B.inst[i].x = x[i];
  }
  memcpy(B.h_inst, B.inst.data(), sizeof(BatchInst) * B.n);
  if (!B.exec || B.g_tol != tol || B.g_maxit != maxit) {
    if (B.exec) { cudaGraphExecDestroy(B.exec); B.exec = nullptr; }
    if (B.graph) { cudaGraphDestroy(B.graph); B.graph = nullptr; }
    AAO_TRY_CUDA(cudaStreamBeginCapture(B.s, cudaStreamCaptureModeThreadLocal));
    cudaMemcpyAsync(B.d_inst, B.h_inst, sizeof(BatchInst) * B.n, cudaMemcpyHostToDevice, B.s);
    cudaMemsetAsync(B.d_next, 0, sizeof(unsigned int), B.s);
    const int lrc = launch_k_batch(B, 0, tol, maxit);
    cudaMemcpyAsync(B.h_st, B.d_st, sizeof(aao_stats) * B.n, cudaMemcpyDeviceToHost, B.s);
    cudaError_t ec = cudaStreamEndCapture(B.s, &B.graph);
    if (lrc != AAO_OK) return lrc;
    if (ec != cudaSuccess) {
      set_error(std::string("batch_submit: graph capture: ") + cudaGetErrorString(ec));
      return AAO_ECUDA;
    }
    AAO_TRY_CUDA(cudaGraphInstantiate(&B.exec, B.graph, 0));
    B.g_tol = tol;
    B.g_maxit = maxit;
  }
  AAO_TRY_CUDA(cudaEventRecord(B.ev0, B.user));
  AAO_TRY_CUDA(cudaStreamWaitEvent(B.s, B.ev0, 0));
  AAO_TRY_CUDA(cudaGraphLaunch(B.exec, B.s));
  g_launches.fetch_add(1, std::memory_order_relaxed);  // the graph holds one kernel
  AAO_TRY_CUDA(cudaStreamSynchronize(B.s));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  int worst = AAO_OK;
  for (int i = 0; i < B.n; ++i) {
    if (st) {
      st[i] = B.h_st[i];
      st[i].ms = ms;
      st[i].launches = i == 0 ? 1 : 0;
    }
    if (B.h_st[i].status != AAO_OK && worst == AAO_OK) worst = B.h_st[i].status;
  }
  if (worst != AAO_OK) set_error("batch_submit: at least one instance did not converge");
  return worst;
}

extern "C" int aao_batch_set_alpha(aao_batch* bt, const double* alpha) {
  if (!bt || !alpha) { set_error("aao_batch_set_alpha: null argument"); return AAO_EINVAL; }
  Batch& B = bt->B;
  for (int i = 0; i < B.n; ++i)
    if (!(alpha[i] > 0) || !(alpha[i] <= 1)) { set_error("aao_batch_set_alpha: need 0 < alpha <= 1"); return AAO_EINVAL; }
  AAO_TRY_CUDA(cudaStreamSynchronize(B.s));
  for (int i = 0; i < B.n; ++i) {
    B.prob[i].alpha = alpha[i];
    const BatchInst& I = B.inst[i];
    std::vector<float> pl, pd, pu, lam, ilam;
    std::vector<float2> mu, il2, tw;
    host_tables(B.prob[i], I.nx, I.nt, pl, pd, pu, mu, il2, tw, lam, ilam);
    AAO_TRY_CUDA(cudaMemcpyAsync((void*)I.mu, mu.data(), sizeof(float2) * I.K, cudaMemcpyHostToDevice, B.s));
    AAO_TRY_CUDA(cudaMemcpyAsync((void*)I.il2, il2.data(), sizeof(float2) * I.K, cudaMemcpyHostToDevice, B.s));
    AAO_TRY_CUDA(cudaMemcpyAsync((void*)I.lam, lam.data(), sizeof(float) * I.nt, cudaMemcpyHostToDevice, B.s));
    AAO_TRY_CUDA(cudaMemcpyAsync((void*)I.ilam, ilam.data(), sizeof(float) * I.nt, cudaMemcpyHostToDevice, B.s));
    AAO_TRY_CUDA(cudaStreamSynchronize(B.s));  // host vectors are released at scope end
  }
  return AAO_OK;
}

extern "C" int aao_batch_destroy(aao_batch* bt) {
  if (!bt) return AAO_OK;
  cudaStreamSynchronize(bt->B.s);
  batch_free(bt->B);
  delete bt;
  return AAO_OK;
}

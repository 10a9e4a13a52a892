// Device building blocks of the P_alpha^{-1} apply (steps (a)-(c) of Eq. 3.2), shared by the
// single-instance kernels (precond.cu) and the persistent batched solver (batch.cu).
#pragma once

#include "aao_internal.cuh"

namespace aao {
namespace pdev {

constexpr int kVals = 16;  // complex values held per thread per FFT stage

// forward 4-point DFT (omega_4 = -i), in place
template <typename C>
__device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  C s02 = cadd(a0, a2), d02 = csub(a0, a2);
  C s13 = cadd(a1, a3), d13 = cmul_mi(csub(a1, a3));
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, d13);
  a3 = csub(d02, d13);
}

// One in-place Stockham stage of radix R = 2^LR (4 or 2) over P = 2^lp interleaved columns
// stored [t][P]. Butterfly j (0 <= j < N/R) of column p reads elements j + r N/R, twiddles them
// by exp(-2 pi i r (j mod Ns) / (Ns R)), Ns = 2^lns, and writes (j / Ns) Ns R + (j mod Ns) + r Ns.
// All index arithmetic is shifts and masks (every size is a power of two).
template <typename C, int LR>
__device__ __forceinline__ void stockham_stage(C* __restrict__ data, int log2n, int lp, int lns,
                                               const C* __restrict__ tw) {
  constexpr int R = 1 << LR;
  constexpr int B = kVals / R;
  const int nbf = 1 << (lp + log2n - LR);
  const int stride_in = 1 << (log2n - LR);
  const int lts = log2n - lns - LR;  // log2 of the twiddle-table step N / (Ns R)
  const int pm = (1 << lp) - 1, nsm = (1 << lns) - 1;
  C reg[B][R];
#pragma unroll
  for (int q = 0; q < B; ++q) {
    const int b = threadIdx.x + q * blockDim.x;
    if (b < nbf) {
      const int p = b & pm, j = b >> lp, k = j & nsm;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C a = data[((j + r * stride_in) << lp) + p];
        if (r > 0 && k > 0) a = cmul(a, tw[(r * k) << lts]);
        reg[q][r] = a;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < B; ++q) {
    const int b = threadIdx.x + q * blockDim.x;
    if (b < nbf) {
      const int p = b & pm, j = b >> lp, k = j & nsm;
      if (R == 4) {
        dft4(reg[q][0], reg[q][1], reg[q][2], reg[q][3]);
      } else {
        C t0 = reg[q][0];
        reg[q][0] = cadd(t0, reg[q][1]);
        reg[q][1] = csub(t0, reg[q][1]);
      }
      const int base = ((j >> lns) << (lns + LR)) + k;
#pragma unroll
      for (int r = 0; r < R; ++r) data[((base + (r << lns)) << lp) + p] = reg[q][r];
    }
  }
  __syncthreads();
}

// Forward DFT (exp(-2 pi i t k / N)) of P = 2^lp columns of length N = 2^log2n in shared memory.
template <typename C>
__device__ void smem_fft(C* data, int log2n, int lp, const C* tw) {
  int lns = 0;
  for (int s = 0; s < log2n / 2; ++s) {
    stockham_stage<C, 2>(data, log2n, lp, lns, tw);
    lns += 2;
  }
  if (log2n & 1) stockham_stage<C, 1>(data, log2n, lp, lns, tw);
}

template <typename R> __device__ __forceinline__ R to_r(double v);
template <> __device__ __forceinline__ float to_r<float>(double v) { return narrow(v); }
template <> __device__ __forceinline__ double to_r<double>(double v) { return v; }

// step (a) for the column tile starting at x0 (all threads of the CTA; smem holds (P+1)*N complex:
// the tile, then a copy of the twiddle table).
// Ends without a barrier: synchronise before reusing smem.
template <typename R>
__device__ __forceinline__ void fft_fwd_tile(const double* __restrict__ v, C_t<R>* __restrict__ spec, int nx, int N,
                                             int log2n, int P, int pitch, const R* __restrict__ lam,
                                             const C_t<R>* __restrict__ tw, R sc, int x0, unsigned char* smraw) {
  using C = C_t<R>;
  C* data = reinterpret_cast<C*>(smraw);
  R* flat = reinterpret_cast<R*>(smraw);
  C* stw = data + (size_t)P * N;  // twiddle table copy (N complex) after the tile
  for (int m = threadIdx.x; m < N; m += blockDim.x) stw[m] = __ldg(&tw[m]);
  // P is a power of two <= 16 and blockDim.x a multiple of 32, so W = 2P divides blockDim.x:
  // thread owns tile column c and rows t = tr, tr + tstep, ... (independent loads in flight)
  const int W = 2 * P;
  const int c = threadIdx.x & (W - 1), tr = threadIdx.x / W, tstep = blockDim.x / W;
  const int x = x0 + c;
  const bool ok = x < nx;
  const double* src = v + x;
#pragma unroll 8
  for (int t = tr; t < N; t += tstep) {
    R val = (R)0;
    if (ok) val = to_r<R>(__ldg(src + (size_t)t * nx)) * (__ldg(&lam[t]) * sc);
    flat[t * W + c] = val;  // complex column c/2: real part for even c, imaginary for odd c
  }
  __syncthreads();
  const int lp = __ffs(P) - 1;
  smem_fft(data, log2n, lp, stw);
  const int half = N / 2;
  for (int e = threadIdx.x; e < (half + 1) * P; e += blockDim.x) {
    const int k = e >> lp, p = e & (P - 1);
    const C zk = data[k * P + p];
    const C zn = data[((N - k) & (N - 1)) * P + p];
    const R h = (R)0.5;
    const C xa = cmk<C>(h * (zk.x + zn.x), h * (zk.y - zn.y));
    const C xb = cmk<C>(h * (zk.y + zn.y), h * (zn.x - zk.x));
    const int x = x0 + 2 * p;
    C* out = spec + (size_t)k * pitch + x;
    if (x < nx) out[0] = xa;
    if (x + 1 < nx) out[1] = xb;
  }
}

template <typename R>
__global__ void __launch_bounds__(sizeof(R) == 8 ? 512 : 1024) k_fft_fwd(const double* __restrict__ v, C_t<R>* __restrict__ spec,
                                                  int nx, int N, int log2n, int P, int pitch,
                                                  const R* __restrict__ lam, const C_t<R>* __restrict__ tw,
                                                  const double* __restrict__ in_scale) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const R sc = in_scale ? (R)(*in_scale) : (R)1;
  fft_fwd_tile<R>(v, spec, nx, N, log2n, P, pitch, lam, tw, sc, blockIdx.x * 2 * P, smraw);
}

// step (c) for the column tile starting at x0 (all threads of the CTA; smem holds (P+1)*N complex:
// the tile, then a copy of the twiddle table).
// Ends without a barrier: synchronise before reusing smem.
template <typename R, typename OUT>
__device__ __forceinline__ void fft_inv_tile(const C_t<R>* __restrict__ spec, OUT* __restrict__ z, int nx, int N,
                                             int log2n, int P, int pitch, const R* __restrict__ ilam,
                                             const C_t<R>* __restrict__ tw, int x0, unsigned char* smraw) {
  using C = C_t<R>;
  C* data = reinterpret_cast<C*>(smraw);
  C* stw = data + (size_t)P * N;  // twiddle table copy (N complex) after the tile
  for (int m = threadIdx.x; m < N; m += blockDim.x) stw[m] = __ldg(&tw[m]);
  const int W = 2 * P;
  const int half = N / 2;
  const int lp = __ffs(P) - 1;
  for (int e = threadIdx.x; e < (half + 1) * P; e += blockDim.x) {
    const int k = e >> lp, p = e & (P - 1);
    const int x = x0 + 2 * p;
    const C* in = spec + (size_t)k * pitch + x;
    C A = cmk<C>(0, 0), B = cmk<C>(0, 0);
    if (x < nx) A = in[0];
    if (x + 1 < nx) B = in[1];
    if (k == 0 || k == half) { A.y = 0; B.y = 0; }  // DC / Nyquist bins of a real signal
    // Z[k] = A + iB; stored conjugated (inverse DFT via the forward transform)
    data[k * P + p] = cmk<C>(A.x - B.y, -(A.y + B.x));
    if (k > 0 && k < half) {
      // Z[N-k] = conj(A) + i conj(B)
      data[(N - k) * P + p] = cmk<C>(A.x + B.y, A.y - B.x);
    }
  }
  __syncthreads();
  smem_fft(data, log2n, lp, stw);
  const int c = threadIdx.x & (W - 1), tr = threadIdx.x / W, tstep = blockDim.x / W;
  const int x = x0 + c;
  if (x < nx) {
    OUT* dst = z + x;
#pragma unroll 8
    for (int t = tr; t < N; t += tstep) {
      const C y = data[t * P + (c >> 1)];
      const R val = ((c & 1) ? -y.y : y.x) * __ldg(&ilam[t]);
      dst[(size_t)t * nx] = (OUT)val;
    }
  }
}

template <typename R, typename OUT>
__global__ void __launch_bounds__(sizeof(R) == 8 ? 512 : 1024) k_fft_inv(const C_t<R>* __restrict__ spec, OUT* __restrict__ z,
                                                  int nx, int N, int log2n, int P, int pitch,
                                                  const R* __restrict__ ilam, const C_t<R>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smraw[];
  fft_inv_tile<R, OUT>(spec, z, nx, N, log2n, P, pitch, ilam, tw, blockIdx.x * 2 * P, smraw);
}

// step (b): one CTA per frequency bin k. Row i of (mu_k I - A~), mu_k = lambda_{1,k}/lambda_{2,k},
// right-hand side z1_k / lambda_{2,k}: a_i = -lo_i, b_i = mu_k - di_i, c_i = -up_i. Thread l owns
// rows [l ch, (l+1) ch) (padding rows beyond nx are identity rows). A modified Thomas sweep
// expresses every row of the chunk through the chunk's first and last unknowns (multipliers in
// registers, right-hand sides in shared memory); the 2T first/last rows form a tridiagonal
// interface system solved by parallel cyclic reduction in shared memory; back substitution
// recovers the interior rows.
// Stage the diagonals of tau*Abar for the row layout of tridiag_bin: row i = L*ch + j goes to
// L*cs + j (odd stride cs: conflict-free per-thread chunks). a_i = -lo_i (0 for i = 0), c_i =
// -up_i (0 for i = nx-1), rows i >= nx are padding. All threads of the CTA; synchronise after.
template <typename R>
__device__ __forceinline__ void tridiag_stage(const R* __restrict__ lo, const R* __restrict__ di,
                                              const R* __restrict__ up, int nx, int T, int ch, int cs, R* sa,
                                              R* sd, R* sc) {
  for (int i = threadIdx.x; i < T * ch; i += blockDim.x) {
    const int L = i / ch, j = i - L * ch, o = L * cs + j;
    sa[o] = (i > 0 && i < nx) ? -__ldg(&lo[i]) : (R)0;
    sd[o] = i < nx ? __ldg(&di[i]) : (R)0;
    sc[o] = (i < nx - 1) ? -__ldg(&up[i]) : (R)0;
  }
}

// The solve of bin k by a group of T threads (thread tid of the group) with smem region smraw of
// (T*cs + 8T) complex and the staged diagonals sa, sd, sc. Every thread of the CTA must call it
// together (it uses __syncthreads); a group with valid == false takes part in the barriers only.
template <typename R, int CH>
__device__ __forceinline__ void tridiag_bin(C_t<R>* __restrict__ spec, int nx, int pitch, int ch, int cs,
                                            const R* __restrict__ sa, const R* __restrict__ sd,
                                            const R* __restrict__ sc, const C_t<R>* __restrict__ mu,
                                            const C_t<R>* __restrict__ il2, int k, int tid, int T, bool valid,
                                            unsigned char* smraw) {
  using C = C_t<R>;
  C* dd = reinterpret_cast<C*>(smraw);
  C* pa = dd + (size_t)T * cs;
  C* pb = pa + 2 * T;
  C* pc = pb + 2 * T;
  C* pd = pc + 2 * T;
  const C zero = cmk<C>(0, 0), one = cmk<C>(1, 0);
  const C muk = valid ? mu[k] : one, sk = valid ? il2[k] : one;
  C* row = spec + (size_t)k * pitch;
  for (int i = tid; i < T * ch; i += T) {
    const int L = i / ch, j = i - L * ch;
    dd[L * cs + j] = (valid && i < nx) ? cmul(row[i], sk) : zero;
  }
  __syncthreads();

  const int s = tid * ch;
  C* d_ = dd + tid * cs;
  C ap[CH], cp[CH];
  C dprev = zero, A1 = zero, C1 = zero, D1 = zero;
#pragma unroll
  for (int j = 0; j < CH; ++j) {
    if (j < ch) {
      const int i = s + j;
      const int o = tid * cs + j;
      const C a = cmk<C>(sa[o], 0), c = cmk<C>(sc[o], 0);
      const C b = i < nx ? cmk<C>(muk.x - sd[o], muk.y) : one;
      C dj;
      if (j < 2) {
        const C ib = cinv(b);
        ap[j] = cmul(a, ib);
        cp[j] = cmul(c, ib);
        dj = cmul(d_[j], ib);
      } else {
        const C r = cinv(csub(b, cmul(a, cp[j - 1])));
        dj = cmul(r, csub(d_[j], cmul(a, dprev)));
        ap[j] = cscale(cmul(r, cmul(a, ap[j - 1])), (R)-1);
        cp[j] = cmul(r, c);
      }
      d_[j] = dj;
      dprev = dj;
      if (j == ch - 1) { A1 = ap[j]; C1 = cp[j]; D1 = dj; }
    }
  }
  C A0 = ap[0], C0 = cp[0], D0 = d_[0];
  if (ch >= 3) {
    C dn = d_[ch - 2];
#pragma unroll
    for (int j = CH - 3; j >= 1; --j) {
      if (j <= ch - 3) {
        dn = csub(d_[j], cmul(cp[j], dn));
        ap[j] = csub(ap[j], cmul(cp[j], ap[j + 1]));
        cp[j] = cscale(cmul(cp[j], cp[j + 1]), (R)-1);
        d_[j] = dn;
      }
    }
    const C r = cinv(csub(one, cmul(C0, ap[1])));
    D0 = cmul(r, csub(D0, cmul(C0, d_[1])));
    A0 = cmul(r, A0);
    C0 = cscale(cmul(r, cmul(C0, cp[1])), (R)-1);
  }
  // interface system: row 2l couples x_{2l-1}, x_{2l}, x_{2l+1}; row 2l+1 couples x_{2l}..x_{2l+2}
  const int R2 = 2 * T;
  pa[2 * tid] = A0; pb[2 * tid] = one; pc[2 * tid] = C0; pd[2 * tid] = D0;
  pa[2 * tid + 1] = A1; pb[2 * tid + 1] = one; pc[2 * tid + 1] = C1; pd[2 * tid + 1] = D1;
  __syncthreads();
  for (int delta = 1; delta < R2; delta <<= 1) {
    C nA[2], nB[2], nC[2], nD[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = 2 * tid + h;
      C lA = zero, lB = one, lC = zero, lD = zero, hA = zero, hB = one, hC = zero, hD = zero;
      if (q - delta >= 0) { lA = pa[q - delta]; lB = pb[q - delta]; lC = pc[q - delta]; lD = pd[q - delta]; }
      if (q + delta < R2) { hA = pa[q + delta]; hB = pb[q + delta]; hC = pc[q + delta]; hD = pd[q + delta]; }
      const C k1 = cmul(pa[q], cinv(lB)), k2 = cmul(pc[q], cinv(hB));
      nA[h] = cscale(cmul(lA, k1), (R)-1);
      nC[h] = cscale(cmul(hC, k2), (R)-1);
      nB[h] = csub(csub(pb[q], cmul(lC, k1)), cmul(hA, k2));
      nD[h] = csub(csub(pd[q], cmul(lD, k1)), cmul(hD, k2));
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = 2 * tid + h;
      pa[q] = nA[h]; pb[q] = nB[h]; pc[q] = nC[h]; pd[q] = nD[h];
    }
    __syncthreads();
  }
  const C xs = cmul(pd[2 * tid], cinv(pb[2 * tid]));
  const C xe = cmul(pd[2 * tid + 1], cinv(pb[2 * tid + 1]));
#pragma unroll
  for (int j = 1; j < CH - 1; ++j)
    if (j < ch - 1) d_[j] = csub(csub(d_[j], cmul(ap[j], xs)), cmul(cp[j], xe));
  d_[0] = xs;
  d_[ch - 1] = xe;
  __syncthreads();
  if (valid) {
    for (int i = tid; i < nx; i += T) {
      const int L = i / ch, j = i - L * ch;
      row[i] = dd[L * cs + j];
    }
  }
}

// G groups of T threads per CTA, one bin per group (bins blockIdx.x * G + g); the diagonals are
// staged once per CTA and shared by the groups.
template <typename R, int CH>
__global__ void __launch_bounds__(512) k_tridiag(C_t<R>* __restrict__ spec, int nx, int K, int pitch, int ch,
                                                 int cs, int T, const R* __restrict__ lo, const R* __restrict__ di,
                                                 const R* __restrict__ up, const C_t<R>* __restrict__ mu,
                                                 const C_t<R>* __restrict__ il2) {
  extern __shared__ __align__(16) unsigned char smraw[];
  using C = C_t<R>;
  const int G = blockDim.x / T;
  R* sa = reinterpret_cast<R*>(smraw);
  R* sd = sa + (size_t)T * cs;
  R* sc = sd + (size_t)T * cs;
  unsigned char* groups = reinterpret_cast<unsigned char*>(sc + (size_t)T * cs);
  groups = reinterpret_cast<unsigned char*>(((size_t)groups + 15) & ~(size_t)15);
  tridiag_stage<R>(lo, di, up, nx, T, ch, cs, sa, sd, sc);
  __syncthreads();
  const int g = threadIdx.x / T, tid = threadIdx.x - g * T;
  const int k = blockIdx.x * G + g;
  const size_t gbytes = ((size_t)T * cs + 8 * (size_t)T) * sizeof(C);
  tridiag_bin<R, CH>(spec, nx, pitch, ch, cs, sa, sd, sc, mu, il2, k < K ? k : 0, tid, T, k < K, groups + g * gbytes);
}


}  // namespace pdev
}  // namespace aao

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
// an input element (FP64, or an FP32 copy made by the kernel that produced the vector) as R
template <typename R> __device__ __forceinline__ R in_r(double v) { return to_r<R>(v); }
template <typename R> __device__ __forceinline__ R in_r(float v) { return (R)v; }

// step (a) for the column tile starting at x0, N < 128 (all threads of the CTA; smem holds
// (P+1)*N complex: the tile, then a copy of the twiddle table).
// Ends without a barrier: synchronise before reusing smem.
template <typename R, typename IN>
__device__ __forceinline__ void fft_fwd_tile_smem(const IN* __restrict__ v, C_t<R>* __restrict__ spec, int nx, int N,
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
  const IN* src = v + x;
#pragma unroll 8
  for (int t = tr; t < N; t += tstep) {
    R val = (R)0;
    if (ok) val = in_r<R>(__ldg(src + (size_t)t * nx)) * (__ldg(&lam[t]) * sc);
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
    if (!AAO_DCHECK(k <= half && x + 1 <= pitch)) continue;
    if (x < nx) out[0] = xa;
    if (x + 1 < nx) out[1] = xb;
  }
}

// step (c) for the column tile starting at x0, N < 128 (all threads of the CTA; smem holds
// (P+1)*N complex: the tile, then a copy of the twiddle table).
// Ends without a barrier: synchronise before reusing smem.
template <typename R, typename OUT>
__device__ __forceinline__ void fft_inv_tile_smem(const C_t<R>* __restrict__ spec, OUT* __restrict__ z, int nx, int N,
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
      if (AAO_DCHECK(t < N)) dst[(size_t)t * nx] = (OUT)val;
    }
  }
}

// ------------------------------------------------------------------ register FFT, N >= 128
// For N = 2^log2n >= 128 each column transform is a sequence of Stockham stages (the same
// recursion as stockham_stage) in which every thread holds 16 complex values of one column in
// registers: radix-16 stages, one stage of radix 2, 4 or 8 to use up log2n - 3 bits, and a final
// radix-8 stage. The first stage reads global memory and the last writes it, so a transform of
// 2^11 points makes two shared-memory round trips (instead of seven radix-4/2 passes).
// Virtual thread (p, u), p < P the complex column, u < N/16, is CTA thread u*P + p.
// Shared tile: element t of column p at (t + t/16) * P + p; the pad row per 16 rows keeps the
// stride-16 scatter of the first stage free of bank conflicts.
constexpr int kRegFftMinLog2 = 7;

__host__ __device__ __forceinline__ size_t reg_fft_elems(int P, int N) { return (size_t)P * (N + N / 16); }

__device__ __forceinline__ int tix(int t, int P, int p) { return (t + (t >> 4)) * P + p; }

// a * (c + i s)
template <typename C>
__device__ __forceinline__ C cmulc(C a, decltype(C::x) c, decltype(C::x) s) {
  return cmk<C>(a.x * c - a.y * s, a.x * s + a.y * c);
}

template <typename C>
__device__ __forceinline__ void dft2(C& a, C& b) {
  const C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

// forward 8-point DFT in registers, natural order in and out: 8 = 2 x 4 (radix 2 over the
// stride-4 index, twiddles w8^(n2 k1), radix 4 over n2; X[k1 + 2 k2] lands in a[4 k1 + k2])
template <typename C>
__device__ __forceinline__ void dft8(C* a) {
  using R = decltype(C::x);
  const R h = (R)0.70710678118654752440;  // cos(pi/4)
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft2(a[n2], a[4 + n2]);
  a[5] = cmulc(a[5], h, -h);   // w8^1
  a[6] = cmul_mi(a[6]);        // w8^2 = -i
  a[7] = cmulc(a[7], -h, -h);  // w8^3
  dft4(a[0], a[1], a[2], a[3]);
  dft4(a[4], a[5], a[6], a[7]);
  const C x1 = a[4], x2 = a[1], x3 = a[5], x4 = a[2], x5 = a[6], x6 = a[3];
  a[1] = x1; a[2] = x2; a[3] = x3; a[4] = x4; a[5] = x5; a[6] = x6;
}

// forward 16-point DFT in registers, natural order in and out: 16 = 4 x 4 (radix 4 over the
// stride-4 index, twiddles w16^(n2 k1), radix 4 over n2; X[k1 + 4 k2] lands in a[4 k1 + k2])
template <typename C>
__device__ __forceinline__ void dft16(C* a) {
  using R = decltype(C::x);
  const R c1 = (R)0.92387953251128675613, s1 = (R)0.38268343236508977173;  // cos, sin(pi/8)
  const R h = (R)0.70710678118654752440;
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4(a[n2], a[4 + n2], a[8 + n2], a[12 + n2]);
  a[5] = cmulc(a[5], c1, -s1);    // w16^1
  a[6] = cmulc(a[6], h, -h);      // w16^2
  a[7] = cmulc(a[7], s1, -c1);    // w16^3
  a[9] = cmulc(a[9], h, -h);      // w16^2
  a[10] = cmul_mi(a[10]);         // w16^4 = -i
  a[11] = cmulc(a[11], -h, -h);   // w16^6
  a[13] = cmulc(a[13], s1, -c1);  // w16^3
  a[14] = cmulc(a[14], -h, -h);   // w16^6
  a[15] = cmulc(a[15], -c1, s1);  // w16^9
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
  C t;
  t = a[1]; a[1] = a[4]; a[4] = t;
  t = a[2]; a[2] = a[8]; a[8] = t;
  t = a[3]; a[3] = a[12]; a[12] = t;
  t = a[6]; a[6] = a[9]; a[9] = t;
  t = a[7]; a[7] = a[13]; a[13] = t;
  t = a[11]; a[11] = a[14]; a[14] = t;
}

template <int LR, typename C>
__device__ __forceinline__ void dft_pow2(C* a) {
  if constexpr (LR == 1) dft2(a[0], a[1]);
  else if constexpr (LR == 2) dft4(a[0], a[1], a[2], a[3]);
  else if constexpr (LR == 3) dft8(a);
  else dft16(a);
}

// One shared-to-shared Stockham stage of radix 2^LR with Ns = 2^lns: virtual thread (p, u) takes
// butterflies j = u + q N/16 (q < 16 / 2^LR) of column p. Two barriers (reads, then writes).
template <typename C, int LR>
__device__ __forceinline__ void reg_stage(C* __restrict__ data, int log2n, int P, int lns,
                                          const C* __restrict__ tw, int p, int u, bool act) {
  constexpr int RR = 1 << LR, B = 16 / RR;
  const int n16 = 1 << (log2n - 4), stride = 1 << (log2n - LR), lts = log2n - lns - LR;
  const int nsm = (1 << lns) - 1;
  C a[16];
  if (act) {
#pragma unroll
    for (int q = 0; q < B; ++q) {
      const int j = u + q * n16, k = j & nsm;
      a[q * RR] = data[tix(j, P, p)];
#pragma unroll
      for (int r = 1; r < RR; ++r) a[q * RR + r] = cmul(data[tix(j + r * stride, P, p)], __ldg(tw + ((r * k) << lts)));
    }
  }
  __syncthreads();
  if (act) {
#pragma unroll
    for (int q = 0; q < B; ++q) {
      const int j = u + q * n16, k = j & nsm;
      dft_pow2<LR>(a + q * RR);
      const int base = ((j >> lns) << (lns + LR)) + k;
#pragma unroll
      for (int r = 0; r < RR; ++r) data[tix(base + (r << lns), P, p)] = a[q * RR + r];
    }
  }
  __syncthreads();
}

// The stages between the first (radix 16, from global memory) and the last (radix 8); on entry
// the first stage's output is in shared memory and a barrier has passed.
template <typename C>
__device__ __forceinline__ void reg_middle(C* data, int log2n, int P, const C* tw, int p, int u, bool act) {
  int lns = 4;
  for (; lns + 4 <= log2n - 3; lns += 4) reg_stage<C, 4>(data, log2n, P, lns, tw, p, u, act);
  switch (log2n - 3 - lns) {
    case 1: reg_stage<C, 1>(data, log2n, P, lns, tw, p, u, act); break;
    case 2: reg_stage<C, 2>(data, log2n, P, lns, tw, p, u, act); break;
    case 3: reg_stage<C, 3>(data, log2n, P, lns, tw, p, u, act); break;
    default: break;
  }
}

// The last stage (radix 8, Ns = N/8) for virtual thread u: butterflies ja = u and jb = Ns - u
// (u = 0: 0 and Ns/2), so that bin k and its mirror N - k sit in the same thread. Element r of
// butterfly j is bin j + r Ns. Reads shared memory only (no barrier needed afterwards).
template <typename C>
__device__ __forceinline__ void reg_last(const C* __restrict__ data, int log2n, int P, const C* __restrict__ tw,
                                         int p, int u, C (&a)[8], C (&b)[8], int& ja, int& jb) {
  const int ns = 1 << (log2n - 3);
  ja = u;
  jb = u == 0 ? ns / 2 : ns - u;
  a[0] = data[tix(ja, P, p)];
  b[0] = data[tix(jb, P, p)];
#pragma unroll
  for (int r = 1; r < 8; ++r) {
    a[r] = cmul(data[tix(ja + r * ns, P, p)], __ldg(tw + r * ja));
    b[r] = cmul(data[tix(jb + r * ns, P, p)], __ldg(tw + r * jb));
  }
  dft8(a);
  dft8(b);
}

template <typename C>
__device__ __forceinline__ void store_pair(C* out, C xa, C xb, bool ok0, bool ok1) {
  if (ok1) {
    if constexpr (sizeof(C) == 8) {
      *reinterpret_cast<float4*>(out) = make_float4(xa.x, xa.y, xb.x, xb.y);
    } else {
      out[0] = xa;
      out[1] = xb;
    }
  } else if (ok0) {
    out[0] = xa;
  }
}

template <typename C>
__device__ __forceinline__ void load_pair(const C* in, C& A, C& B, bool ok0, bool ok1) {
  A = cmk<C>(0, 0);
  B = cmk<C>(0, 0);
  if (ok1) {
    if constexpr (sizeof(C) == 8) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(in));
      A = cmk<C>(q.x, q.y);
      B = cmk<C>(q.z, q.w);
    } else {
      A = __ldg(in);
      B = __ldg(in + 1);
    }
  } else if (ok0) {
    A = __ldg(in);
  }
}

// step (a) for the column tile starting at x0, N >= 128 (spec rows 16-byte aligned, x0 even;
// smem holds reg_fft_elems(P, N) complex). Ends without a barrier: synchronise before reusing smem.
template <typename R, typename IN>
__device__ __forceinline__ void fft_fwd_tile_reg(const IN* __restrict__ v, C_t<R>* __restrict__ spec, int nx,
                                                 int N, int log2n, int P, int pitch, const R* __restrict__ lam,
                                                 const C_t<R>* __restrict__ tw, R sc, int x0, unsigned char* smraw) {
  using C = C_t<R>;
  C* data = reinterpret_cast<C*>(smraw);
  const int n16 = N >> 4;
  const bool act = (int)threadIdx.x < P * n16;  // P need not be a power of two here
  const int u = (int)threadIdx.x / P, p = (int)threadIdx.x - u * P;
  const int x = x0 + 2 * p;
  const bool ok0 = x < nx, ok1 = x + 1 < nx;
  if (act) {
    // first stage: radix 16 over rows u + r N/16, scaled by Lambda_alpha and the input scale
    C a[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int t = u + r * n16;
      const IN* row = v + (size_t)t * nx + x;
      const R l = __ldg(&lam[t]) * sc;
      R re = (R)0, im = (R)0;
      if (ok0) re = in_r<R>(__ldg(row)) * l;
      if (ok1) im = in_r<R>(__ldg(row + 1)) * l;
      a[r] = cmk<C>(re, im);
    }
    dft16(a);
#pragma unroll
    for (int r = 0; r < 16; ++r) data[tix(u * 16 + r, P, p)] = a[r];
  }
  __syncthreads();
  reg_middle(data, log2n, P, tw, p, u, act);
  if (act) {
    C a[8], b[8];
    int ja, jb;
    reg_last(data, log2n, P, tw, p, u, a, b, ja, jb);
    // Z = A + iB packs the two real columns; A[k] = (Z[k] + conj Z[N-k]) / 2,
    // B[k] = (Z[k] - conj Z[N-k]) / 2i, for the bins k <= N/2 this thread holds
    const int ns = N >> 3;
    const R h = (R)0.5;
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      if (r < 4 || u == 0) {
        const C zk = a[r];
        const C zn = u == 0 ? a[(8 - r) & 7] : b[7 - r];
        const C xa = cmk<C>(h * (zk.x + zn.x), h * (zk.y - zn.y));
        const C xb = cmk<C>(h * (zk.y + zn.y), h * (zn.x - zk.x));
        if (AAO_DCHECK(ja + r * ns <= N / 2 && x + 1 <= pitch))
          store_pair(spec + (size_t)(ja + r * ns) * pitch + x, xa, xb, ok0, ok1);
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const C zk = b[r];
      const C zn = u == 0 ? b[7 - r] : a[7 - r];
      const C xa = cmk<C>(h * (zk.x + zn.x), h * (zk.y - zn.y));
      const C xb = cmk<C>(h * (zk.y + zn.y), h * (zn.x - zk.x));
      if (AAO_DCHECK(jb + r * ns <= N / 2 && x + 1 <= pitch))
        store_pair(spec + (size_t)(jb + r * ns) * pitch + x, xa, xb, ok0, ok1);
    }
  }
}

// step (c) for the column tile starting at x0, N >= 128 (spec rows 16-byte aligned, x0 even;
// smem holds reg_fft_elems(P, N) complex). Ends without a barrier: synchronise before reusing smem.
template <typename R, typename OUT>
__device__ __forceinline__ void fft_inv_tile_reg(const C_t<R>* __restrict__ spec, OUT* __restrict__ z, int nx, int N,
                                                 int log2n, int P, int pitch, const R* __restrict__ ilam,
                                                 const C_t<R>* __restrict__ tw, int x0, unsigned char* smraw) {
  using C = C_t<R>;
  C* data = reinterpret_cast<C*>(smraw);
  const int n16 = N >> 4, half = N >> 1;
  const bool act = (int)threadIdx.x < P * n16;  // P need not be a power of two here
  const int u = (int)threadIdx.x / P, p = (int)threadIdx.x - u * P;
  const int x = x0 + 2 * p;
  const bool ok0 = x < nx, ok1 = x + 1 < nx;
  if (act) {
    // first stage: the conjugate of the full spectrum Z = A + iB, bins above N/2 from their
    // mirrors (Remark 1), so that the forward transform gives the conjugated inverse DFT
    C a[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int t = u + r * n16;
      const int k = t <= half ? t : N - t;
      C A, B;
      load_pair(spec + (size_t)k * pitch + x, A, B, ok0, ok1);
      if (k == 0 || k == half) { A.y = 0; B.y = 0; }  // DC / Nyquist bins of a real signal
      a[r] = t <= half ? cmk<C>(A.x - B.y, -(A.y + B.x)) : cmk<C>(A.x + B.y, A.y - B.x);
    }
    dft16(a);
#pragma unroll
    for (int r = 0; r < 16; ++r) data[tix(u * 16 + r, P, p)] = a[r];
  }
  __syncthreads();
  reg_middle(data, log2n, P, tw, p, u, act);
  if (act) {
    C a[8], b[8];
    int ja, jb;
    reg_last(data, log2n, P, tw, p, u, a, b, ja, jb);
    const int ns = N >> 3;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int ta = ja + r * ns, tb = jb + r * ns;
      const R la = __ldg(&ilam[ta]), lb = __ldg(&ilam[tb]);
      OUT* da = z + (size_t)ta * nx + x;
      OUT* db = z + (size_t)tb * nx + x;
      if (!AAO_DCHECK(ta < N && tb < N)) continue;
      if (ok0) { da[0] = (OUT)(a[r].x * la); db[0] = (OUT)(b[r].x * lb); }
      if (ok1) { da[1] = (OUT)(-a[r].y * la); db[1] = (OUT)(-b[r].y * lb); }
    }
  }
}

// shared memory of one FFT tile (both directions)
__host__ __device__ __forceinline__ size_t fft_tile_bytes(int P, int N, size_t csize) {
  return (N >= (1 << kRegFftMinLog2) ? reg_fft_elems(P, N) : (size_t)(P + 1) * N) * csize;
}

template <typename R, typename IN = double>
__device__ __forceinline__ void fft_fwd_tile(const IN* __restrict__ v, C_t<R>* __restrict__ spec, int nx, int N,
                                             int log2n, int P, int pitch, const R* __restrict__ lam,
                                             const C_t<R>* __restrict__ tw, R sc, int x0, unsigned char* smraw) {
  if (log2n >= kRegFftMinLog2) fft_fwd_tile_reg<R, IN>(v, spec, nx, N, log2n, P, pitch, lam, tw, sc, x0, smraw);
  else fft_fwd_tile_smem<R, IN>(v, spec, nx, N, log2n, P, pitch, lam, tw, sc, x0, smraw);
}

template <typename R, typename OUT>
__device__ __forceinline__ void fft_inv_tile(const C_t<R>* __restrict__ spec, OUT* __restrict__ z, int nx, int N,
                                             int log2n, int P, int pitch, const R* __restrict__ ilam,
                                             const C_t<R>* __restrict__ tw, int x0, unsigned char* smraw) {
  if (log2n >= kRegFftMinLog2) fft_inv_tile_reg<R, OUT>(spec, z, nx, N, log2n, P, pitch, ilam, tw, x0, smraw);
  else fft_inv_tile_smem<R, OUT>(spec, z, nx, N, log2n, P, pitch, ilam, tw, x0, smraw);
}

template <typename R, typename IN>
__global__ void __launch_bounds__(sizeof(R) == 8 ? 512 : 1024) k_fft_fwd(const IN* __restrict__ v, C_t<R>* __restrict__ spec,
                                                  int nx, int N, int log2n, int P, int pitch,
                                                  const R* __restrict__ lam, const C_t<R>* __restrict__ tw,
                                                  const double* __restrict__ in_scale) {
  extern __shared__ __align__(16) unsigned char smraw[];
  pdl_sync();
  const R sc = in_scale ? to_r<R>(*in_scale) : (R)1;
  fft_fwd_tile<R, IN>(v, spec, nx, N, log2n, P, pitch, lam, tw, sc, blockIdx.x * 2 * P, smraw);
}

template <typename R, typename OUT>
__global__ void __launch_bounds__(sizeof(R) == 8 ? 512 : 1024) k_fft_inv(const C_t<R>* __restrict__ spec, OUT* __restrict__ z,
                                                  int nx, int N, int log2n, int P, int pitch,
                                                  const R* __restrict__ ilam, const C_t<R>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smraw[];
  pdl_sync();
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
      if (AAO_DCHECK(i < pitch)) row[i] = dd[L * cs + j];
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
  pdl_sync();
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


// ------------------------------------------------------------------ partitioned tridiagonal solve
// step (b) by the partition method, T = 2^lgT >= 32 threads per bin and G bins per CTA: thread l
// of a bin owns the chunk of rows [l ch, (l+1) ch), rows >= nx being identity rows. For the
// system (mu_k I - Abar) x = d of bin k (a_i, c_i the off-diagonals as stored, dg_i the diagonal):
//  (1) downward elimination inside the chunk, the previous chunk's last unknown y_{l-1} kept as a
//      parameter: x_i + c'_i x_{i+1} = d'_i + v_i y_{l-1}, with p_i = 1 / (mu_k - dg_i - a_i c'_{i-1}),
//      c'_i = c_i p_i, d'_i = (d_i - a_i d'_{i-1}) p_i, v_i = -a_i v_{i-1} p_i (v = 1 before the chunk);
//  (2) an upward recurrence writing the chunk's first unknown as x_s = G + H y_{l-1} + J y_l,
//      y_l the chunk's last unknown;
//  the T last-row unknowns then satisfy a tridiagonal system (row e_l of (1) with x_{e+1} taken
//  from chunk l+1's (G, H, J)), solved by parallel cyclic reduction;
//  (3) upward back substitution x_i = d'_i + v_i y_{l-1} - c'_i x_{i+1} from x_e = y_l.
// Everything that depends on the matrix alone -- the pivots p_i, the fill-in v_i, H and J, the
// reduced system and the multipliers of every reduction level -- is the same for every apply, so
// k_tridiag_part_factor computes it once per bin when the handle is built. An apply carries only
// the right-hand side through the recurrences: d' (one real FMA pair and a complex product per
// row), G, the reduced right-hand side and the back substitution.
// Factor tables, per bin k: p and v at [k][i] (i = l ch + j < T ch, identity rows included), and
// [k][2 s][l], [k][2 s + 1][l] the level-s multipliers (s < lgT), [k][2 lgT][l] 1 / the final
// reduced diagonal. An apply stages the bin's p and v rows (before waiting for the previous kernel:
// programmatic dependent launch), its right-hand side and the a and c planes of the coefficient
// table (shared by the CTA's G bins) in shared memory with asynchronous copies, all in flight at
// once; thread l keeps rows l*cs + j (odd stride cs: conflict-free). G bins per CTA fill shared
// memory (at most 512 threads).
constexpr int kTriMaxLgT = 9;  // T <= 512
__host__ __device__ __forceinline__ size_t tri_fact_pcr_elems(int lgT, int T) { return (size_t)(2 * lgT + 1) * T; }
__host__ __device__ __forceinline__ size_t tri_part_bin_elems(int T, int cs) { return 3 * (size_t)T * cs + 2 * (size_t)T; }
__host__ __device__ __forceinline__ size_t tri_part_coef_bytes(int T, int cs, size_t rsize, bool staged) {
  return staged ? (((2 * (size_t)T * cs * rsize) + 15) & ~(size_t)15) : 0;
}
__host__ __device__ __forceinline__ size_t tri_part_bytes(int G, int T, int cs, size_t rsize, bool staged) {
  return tri_part_coef_bytes(T, cs, rsize, staged) + (size_t)G * tri_part_bin_elems(T, cs) * 2 * rsize;
}

template <typename R>
__device__ __forceinline__ C_t<R> crcp(C_t<R> a);
template <>
__device__ __forceinline__ float2 crcp<float>(float2 a) {
  float s;  // hardware reciprocal (about 1 ulp): the FP32 preconditioner needs no correct rounding
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(fmaf(a.x, a.x, a.y * a.y)));
  return make_float2(a.x * s, -a.y * s);
}
template <>
__device__ __forceinline__ double2 crcp<double>(double2 a) {
  const double s = 1.0 / fma(a.x, a.x, a.y * a.y);
  return make_double2(a.x * s, -a.y * s);
}

// asynchronous global -> shared copy of 4, 8 or 16 bytes (both addresses aligned to the size)
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(gmem_src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Factor kernel: one bin per CTA of T threads (shared memory: 5 T complex). The coefficient table
// is chunk-transposed: planes a, dg, c of T ch reals each, entry (j, l) at j T + l.
template <typename R>
__global__ void __launch_bounds__(512) k_tridiag_part_factor(int nx, int ch, int lgT, const R* __restrict__ tri,
                                                             const C_t<R>* __restrict__ mu, C_t<R>* __restrict__ fp,
                                                             C_t<R>* __restrict__ fv, C_t<R>* __restrict__ fpcr) {
  using C = C_t<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int T = 1 << lgT, l = threadIdx.x, k = blockIdx.x;
  C* pa = reinterpret_cast<C*>(smraw);
  C* pb = pa + T;
  C* pc = pb + T;
  C* ph = pc + T;
  C* pj = ph + T;
  const C zero = cmk<C>(0, 0), one = cmk<C>(1, 0);
  const C muk = mu[k];
  const size_t plane = (size_t)T * ch, rows = (size_t)T * ch;
  C* P = fp + (size_t)k * rows + (size_t)l * ch;
  C* Vv = fv + (size_t)k * rows + (size_t)l * ch;
  const int nrow = nx - l * ch;
  C cpr = zero, vpr = one;
  for (int j = 0; j < ch; ++j) {
    const size_t o = (size_t)j * T + l;
    const R a = tri[o], dg = tri[plane + o], c = tri[2 * plane + o];
    const C b = j < nrow ? cmk<C>(muk.x - dg, muk.y) : one;
    const C inv = crcp<R>(cmk<C>(b.x - a * cpr.x, b.y - a * cpr.y));
    cpr = cscale(inv, c);
    vpr = cmul(cscale(vpr, -a), inv);
    P[j] = inv;
    Vv[j] = vpr;
  }
  // (2) H and J (this thread re-reads its own stores)
  C Hs = zero, Js = one;
  for (int j = ch - 2; j >= 0; --j) {
    const C cj = cscale(P[j], tri[2 * plane + (size_t)j * T + l]);
    Hs = csub(Vv[j], cmul(cj, Hs));
    Js = cscale(cmul(cj, Js), (R)-1);
  }
  ph[l] = Hs;
  pj[l] = Js;
  __syncthreads();
  const C Hn = l + 1 < T ? ph[l + 1] : zero, Jn = l + 1 < T ? pj[l + 1] : zero;
  // row l of the reduced system: -v_e y_{l-1} + (1 + c'_e H_{l+1}) y_l + c'_e J_{l+1} y_{l+1}
  pa[l] = cscale(vpr, (R)-1);
  pb[l] = cadd(one, cmul(cpr, Hn));
  pc[l] = cmul(cpr, Jn);
  __syncthreads();
  C* F = fpcr + (size_t)k * tri_fact_pcr_elems(lgT, T) + l;
  for (int s = 0; s < lgT; ++s) {
    const int delta = 1 << s;
    C lA = zero, lB = one, lC = zero, hA = zero, hB = one, hC = zero;
    if (l - delta >= 0) { lA = pa[l - delta]; lB = pb[l - delta]; lC = pc[l - delta]; }
    if (l + delta < T) { hA = pa[l + delta]; hB = pb[l + delta]; hC = pc[l + delta]; }
    const C k1 = l - delta >= 0 ? cmul(pa[l], crcp<R>(lB)) : zero;
    const C k2 = l + delta < T ? cmul(pc[l], crcp<R>(hB)) : zero;
    const C nA = cscale(cmul(lA, k1), (R)-1);
    const C nC = cscale(cmul(hC, k2), (R)-1);
    const C nB = csub(csub(pb[l], cmul(lC, k1)), cmul(hA, k2));
    F[(size_t)(2 * s) * T] = k1;
    F[(size_t)(2 * s + 1) * T] = k2;
    __syncthreads();
    pa[l] = nA; pb[l] = nB; pc[l] = nC;
    __syncthreads();
  }
  F[(size_t)(2 * lgT) * T] = crcp<R>(pb[l]);
}

// Apply kernel: G bins of T threads per CTA. STAGED = false (large Nx, where the coefficient planes
// do not fit beside one bin): the sweeps read them from global memory, one row ahead.
template <typename R, bool STAGED>
__global__ void __launch_bounds__(512) k_tridiag_part(C_t<R>* __restrict__ spec, int nx, int K, int pitch, int ch,
                                                      int cs, int lgT, const R* __restrict__ tri,
                                                      const C_t<R>* __restrict__ fp, const C_t<R>* __restrict__ fv,
                                                      const C_t<R>* __restrict__ fpcr,
                                                      const C_t<R>* __restrict__ il2) {
  using C = C_t<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int T = 1 << lgT, G = blockDim.x >> lgT;
  const int g = threadIdx.x >> lgT, l = threadIdx.x & (T - 1);
  const int k = blockIdx.x * G + g;
  const bool valid = k < K;
  const int kk = valid ? k : 0;
  R* sa = reinterpret_cast<R*>(smraw);
  R* sc = sa + (size_t)T * cs;
  const size_t coef = tri_part_coef_bytes(T, cs, sizeof(R), STAGED);
  C* sd = reinterpret_cast<C*>(smraw + coef) + (size_t)g * tri_part_bin_elems(T, cs);
  C* sp = sd + (size_t)T * cs;
  C* sv = sp + (size_t)T * cs;
  C* pd = sv + (size_t)T * cs;
  C* pg = pd + T;
  const C zero = cmk<C>(0, 0);
  C* row = spec + (size_t)kk * pitch;
  const size_t rows = (size_t)T * ch, plane = (size_t)T * ch;
  const C* gp = fp + (size_t)kk * rows;
  const C* gv = fv + (size_t)kk * rows;
  C m1[kTriMaxLgT], m2[kTriMaxLgT];
  const C* F = fpcr + (size_t)kk * tri_fact_pcr_elems(lgT, T) + l;
#pragma unroll
  for (int s = 0; s < kTriMaxLgT; ++s) {
    m1[s] = s < lgT ? __ldg(F + (size_t)(2 * s) * T) : zero;
    m2[s] = s < lgT ? __ldg(F + (size_t)(2 * s + 1) * T) : zero;
  }
  const C rb = __ldg(F + (size_t)(2 * lgT) * T);
  if constexpr (STAGED) {
    for (int e = threadIdx.x; e < 2 * ch * T; e += blockDim.x) {
      const int jq = e >> lgT, L = e & (T - 1);
      const int q = jq >= ch ? 1 : 0, j = jq - q * ch;
      cp_async<sizeof(R)>(sa + (size_t)q * T * cs + L * cs + j, tri + (q == 0 ? 0 : 2 * plane) + (size_t)j * T + L);
    }
  }
  const int dL = T / ch, dj = T - dL * ch;
  for (int L = l / ch, j = l - (l / ch) * ch; L < T;) {
    const int i = L * ch + j;
    const int o = L * cs + j;
    cp_async<sizeof(C)>(sp + o, gp + i);
    cp_async<sizeof(C)>(sv + o, gv + i);
    j += dj;
    L += dL;
    if (j >= ch) { j -= ch; ++L; }
  }
  pdl_sync();
  for (int L = l / ch, j = l - (l / ch) * ch; L < T;) {
    const int i = L * ch + j;
    const int o = L * cs + j;
    if (valid && i < nx) cp_async<sizeof(C)>(sd + o, row + i);
    else sd[o] = zero;
    j += dj;
    L += dL;
    if (j >= ch) { j -= ch; ++L; }
  }
  cp_async_wait_all();
  __syncthreads();
  C* D = sd + l * cs;
  const C* Pp = sp + l * cs;
  const C* Vv = sv + l * cs;
  const R* A = sa + l * cs;
  const R* CC = sc + l * cs;
  auto coef_a = [&](int j) -> R {
    if constexpr (STAGED) return A[j];
    else return __ldg(tri + (size_t)j * T + l);
  };
  auto coef_c = [&](int j) -> R {
    if constexpr (STAGED) return CC[j];
    else return __ldg(tri + 2 * plane + (size_t)j * T + l);
  };
  C dpr = zero;
  R an = coef_a(0);
  for (int j = 0; j < ch; ++j) {
    const R a = an;
    if (j + 1 < ch) an = coef_a(j + 1);
    const C dj = D[j];
    dpr = cmul(cmk<C>(dj.x - a * dpr.x, dj.y - a * dpr.y), Pp[j]);
    D[j] = dpr;
  }
  const C cpe = cscale(Pp[ch - 1], coef_c(ch - 1));
  C Gs = zero;
  R cn = ch >= 2 ? coef_c(ch - 2) : (R)0;
  for (int j = ch - 2; j >= 0; --j) {
    const R c = cn;
    if (j > 0) cn = coef_c(j - 1);
    Gs = csub(D[j], cmul(cscale(Pp[j], c), Gs));
  }
  pg[l] = Gs;
  __syncthreads();
  const C Gn = l + 1 < T ? pg[l + 1] : zero;
  C cur = csub(dpr, cmul(cpe, Gn));
  pd[l] = cur;
  __syncthreads();
#pragma unroll
  for (int s = 0; s < kTriMaxLgT; ++s) {
    if (s < lgT) {
      const int delta = 1 << s;
      const C lD = l - delta >= 0 ? pd[l - delta] : zero;
      const C hD = l + delta < T ? pd[l + delta] : zero;
      cur = csub(csub(cur, cmul(lD, m1[s])), cmul(hD, m2[s]));
      __syncthreads();
      pd[l] = cur;
      __syncthreads();
    }
  }
  const C y = cmul(cur, rb);
  pg[l] = y;
  __syncthreads();
  const C yp = l > 0 ? pg[l - 1] : zero;
  C x = y;
  D[ch - 1] = x;
  cn = ch >= 2 ? coef_c(ch - 2) : (R)0;
  for (int j = ch - 2; j >= 0; --j) {
    const R c = cn;
    if (j > 0) cn = coef_c(j - 1);
    x = csub(cadd(D[j], cmul(Vv[j], yp)), cmul(cscale(Pp[j], c), x));
    D[j] = x;
  }
  __syncthreads();
  if (valid) {
    const C sk = il2[k];
    for (int L = l / ch, j = l - (l / ch) * ch; L < T;) {
      const int i = L * ch + j;
      if (i >= nx) break;
      if (AAO_DCHECK(k < K && i < pitch)) row[i] = cmul(sd[L * cs + j], sk);
      j += dj;
      L += dL;
      if (j >= ch) { j -= ch; ++L; }
    }
  }
}

// ------------------------------------------------------------------ step (b) without factor tables
// k_tridiag_rc: the partition method of k_tridiag_part with nothing stored per bin. Every pivot is
// recomputed from the three real diagonals of tau*Abar (the chunk-transposed table, shared by all
// bins) and mu_k; ALU work is cheap here, while per-bin tables of pivots and
// fill-in tripled the bytes a bin moves and filled shared memory. Thread l of a bin keeps the
// right-hand sides of its chunk (rows s = l ch .. e = s + ch - 1) in registers; with the row
// equations a_j x_{j-1} + b_j x_j + c_j x_{j+1} = d_j (b_j = mu_k - dg_j, identity rows beyond nx):
//  (A1) a reverse sweep over rows e-1 .. s with x_e = y_l and x_{s-1} = y_{l-1} kept as parameters:
//       x_j = G_j + H_j x_{j-1} + J_j y_l, q_j = 1 / (b_j + c_j H_{j+1}), G_j = (d_j - c_j G_{j+1}) q_j,
//       H_j = -a_j q_j, J_j = -c_j J_{j+1} q_j (G, J start from q_{e-1}); at row s it gives
//       x_s = G + H y_{l-1} + J y_l;
//  (A2) a forward sweep over rows s .. e with y_{l-1} kept as a parameter:
//       x_j + c'_j x_{j+1} = d'_j + v_j y_{l-1}, p_j = 1 / (b_j - a_j c'_{j-1}), c'_j = c_j p_j,
//       d'_j = (d_j - a_j d'_{j-1}) p_j, v_j = -a_j v_{j-1} p_j; the pivots p_j are kept in
//       shared memory for (B).
//  (A1) and (A2) only read the right-hand sides, so they run interleaved (two independent
//  dependency chains). Row e of (A2) with x_{e+1} taken from chunk l+1's (G, H, J) is row l of the
//  T-row reduced system -v_e y_{l-1} + (1 + c'_e H_{l+1}) y_l + c'_e J_{l+1} y_{l+1} =
//  d'_e - c'_e G_{l+1}, solved by parallel cyclic reduction in shared memory (named barriers of
//  the bin's T threads);
//  (B) with y_{l-1} and y_l known: d''_j = (d_j - a_j d''_{j-1}) p_j from d''_{s-1} = y_{l-1},
//      then x_j = d''_j - c_j p_j x_{j+1} upward from x_e = y_l.
// G bins per CTA. Shared memory: the three coefficient planes [3][ch][T] (staged with cp.async
// before the kernel waits for its predecessor: they do not depend on it), then per bin the chunk
// rows (odd stride cs, conflict-free; the right-hand side on the way in, the pivots, the solution
// on the way out) and one buffer of 4 T complex for the exchanges and the reduction (two named
// barriers per level). The rows are scaled by 1/lambda_{2,k} on the way out (the solve is linear).
template <typename C>
struct RcRow {  // one row of the reduced system
  C a, b, c, d;  // sub-diagonal, diagonal, super-diagonal, right-hand side
};
__device__ __forceinline__ void bin_barrier(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__host__ __device__ __forceinline__ size_t tri_rc_bin_bytes(int T, int cs, size_t csize) {
  return ((size_t)T * cs + 4 * (size_t)T) * csize;
}
// SC: the coefficient planes staged in shared memory (else read from global memory through L1,
// where they do not fit beside the bins' rows: FP64 at the largest nx)
template <typename R, int CH, bool SC>
__global__ void __launch_bounds__(512, sizeof(R) == 4 ? 2 : 1)
    k_tridiag_rc(C_t<R>* __restrict__ spec, int nx, int K, int pitch, int ch, int cs, int lgT,
                 const R* __restrict__ tri, const C_t<R>* __restrict__ mu, const C_t<R>* __restrict__ il2) {
  using C = C_t<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int T = 1 << lgT;
  const int g = threadIdx.x >> lgT, l = threadIdx.x & (T - 1);
  const int k = blockIdx.x * (blockDim.x >> lgT) + g;
  const bool valid = k < K;
  const int kk = valid ? k : 0;
  const size_t plane = (size_t)ch * T;
  R* sco = reinterpret_cast<R*>(smraw);  // [3][ch][T] when SC
  const size_t cbytes = SC ? ((3 * plane * sizeof(R)) + 15) & ~(size_t)15 : 0;
  C* W = reinterpret_cast<C*>(smraw + cbytes + (size_t)g * tri_rc_bin_bytes(T, cs, sizeof(C)));
  C* buf = W + (size_t)T * cs;
  const int bar = 1 + g;
  const C zero = cmk<C>(0, 0), one = cmk<C>(1, 0);
  // the coefficient planes do not depend on the previous kernel: stage them before waiting for it
  if constexpr (SC) {
    const int n16 = (int)(3 * plane * sizeof(R) / 16);
    for (int e = threadIdx.x; e < n16; e += blockDim.x)
      cp_async<16>(reinterpret_cast<unsigned char*>(sco) + 16 * (size_t)e,
                   reinterpret_cast<const unsigned char*>(tri) + 16 * (size_t)e);
  }
  const C muk = __ldg(mu + kk);
  C* row = spec + (size_t)kk * pitch;
  pdl_sync();
  {
    const int dL = T / ch, dj = T - dL * ch;
    for (int L = l / ch, j = l - (l / ch) * ch; L < T;) {
      const int i = L * ch + j;
      W[L * cs + j] = (valid && i < nx) ? row[i] : zero;
      j += dj;
      L += dL;
      if (j >= ch) { j -= ch; ++L; }
    }
  }
  cp_async_wait_all();
  __syncthreads();
  C d[CH];
  C* Wl = W + l * cs;
#pragma unroll
  for (int j = 0; j < CH; ++j) d[j] = j < ch ? Wl[j] : zero;
  const int nrow = nx - l * ch;
  const R* cb = SC ? sco : tri;
  const R* sa = cb + l;
  const R* sg = cb + plane + l;
  const R* sc = cb + 2 * plane + l;
  C Gs = zero, Hs = zero, Js = one;
  C cpr = zero, dpr = zero, vpr = one;
#pragma unroll
  for (int u = 0; u < CH; ++u) {
    if (u < ch) {
      const R a = sa[u * T], c = sc[u * T];
      const C b = u < nrow ? cmk<C>(muk.x - sg[u * T], muk.y) : one;
      const C p = crcp<R>(cmk<C>(b.x - a * cpr.x, b.y - a * cpr.y));
      cpr = cscale(p, c);
      dpr = cmul(cmk<C>(d[u].x - a * dpr.x, d[u].y - a * dpr.y), p);
      vpr = cmul(cscale(vpr, -a), p);
      Wl[u] = p;
    }
    const int j = CH - 1 - u;
    if (j <= ch - 2) {
      const R a = sa[j * T], c = sc[j * T];
      const C b = j < nrow ? cmk<C>(muk.x - sg[j * T], muk.y) : one;
      if (j == ch - 2) {
        const C q = crcp<R>(b);
        Gs = cmul(d[j], q);
        Js = cscale(q, -c);
        Hs = cscale(q, -a);
      } else {
        const C q = crcp<R>(cmk<C>(b.x + c * Hs.x, b.y + c * Hs.y));
        Gs = cmul(cmk<C>(d[j].x - c * Gs.x, d[j].y - c * Gs.y), q);
        Js = cmul(cscale(Js, -c), q);
        Hs = cscale(q, -a);
      }
    }
  }
  buf[l] = Gs;
  buf[T + l] = Hs;
  buf[2 * T + l] = Js;
  bin_barrier(bar, T);
  RcRow<C> rr;
  {
    const bool last = l + 1 >= T;
    const C Gn = last ? zero : buf[l + 1], Hn = last ? zero : buf[T + l + 1], Jn = last ? zero : buf[2 * T + l + 1];
    rr.a = cscale(vpr, (R)-1);
    rr.b = cadd(one, cmul(cpr, Hn));
    rr.c = cmul(cpr, Jn);
    rr.d = csub(dpr, cmul(cpr, Gn));
  }
#pragma unroll 1
  for (int s = 0; s < lgT; ++s) {
    bin_barrier(bar, T);  // the previous reads of buf are done
    buf[l] = rr.a;
    buf[T + l] = crcp<R>(rr.b);
    buf[2 * T + l] = rr.c;
    buf[3 * T + l] = rr.d;
    bin_barrier(bar, T);
    const int delta = 1 << s;
    C anew = zero, cnew = zero, bnew = rr.b, dnew = rr.d;
    if (l - delta >= 0) {
      const C k1 = cmul(rr.a, buf[T + l - delta]);
      anew = cscale(cmul(buf[l - delta], k1), (R)-1);
      bnew = csub(bnew, cmul(buf[2 * T + l - delta], k1));
      dnew = csub(dnew, cmul(buf[3 * T + l - delta], k1));
    }
    if (l + delta < T) {
      const C k2 = cmul(rr.c, buf[T + l + delta]);
      cnew = cscale(cmul(buf[2 * T + l + delta], k2), (R)-1);
      bnew = csub(bnew, cmul(buf[l + delta], k2));
      dnew = csub(dnew, cmul(buf[3 * T + l + delta], k2));
    }
    rr.a = anew;
    rr.b = bnew;
    rr.c = cnew;
    rr.d = dnew;
  }
  const C y = cmul(rr.d, crcp<R>(rr.b));
  bin_barrier(bar, T);
  buf[l] = y;
  bin_barrier(bar, T);
  const C yp = l > 0 ? buf[l - 1] : zero;
  {
    C dd = yp;
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      if (j <= ch - 2) {
        const R a = sa[j * T];
        dd = cmul(cmk<C>(d[j].x - a * dd.x, d[j].y - a * dd.y), Wl[j]);
        d[j] = dd;
      }
    }
  }
  const C sk = valid ? __ldg(il2 + k) : one;
  C x = y;
#pragma unroll
  for (int j = CH - 1; j >= 0; --j) {
    if (j < ch) {
      if (j < ch - 1) x = csub(d[j], cmul(cscale(Wl[j], sc[j * T]), x));
      Wl[j] = cmul(x, sk);
    }
  }
  bin_barrier(bar, T);
  if (valid) {
    const int dL = T / ch, dj = T - dL * ch;
    for (int L = l / ch, j = l - (l / ch) * ch; L < T;) {
      const int i = L * ch + j;
      if (i >= nx) break;
      if (AAO_DCHECK(k < K && i < pitch)) row[i] = W[L * cs + j];
      j += dj;
      L += dL;
      if (j >= ch) { j -= ch; ++L; }
    }
  }
}

// ------------------------------------------------------------------ mixed-radix column tiles
// For nt not a power of two (prime factors 2, 3, 5, 7): the same steps (a) and (c) as the
// power-of-two tiles (two real columns per complex column, Lambda_alpha fused, bins 0..nt/2
// written frequency-major), the transform a shared-memory Stockham recursion over the stages of
// MrPlan (radix 8, 4, 2, 3, 5, 7), out of place between two buffers of P columns x N.
// A stage of radix Q with Ns = the product of the earlier radices: butterfly j < N/Q of column
// p reads elements j + q N/Q (q < Q), twiddles element q by w^(q (j mod Ns)), w = exp(-2 pi i /
// (Ns Q)), takes their Q-point DFT and writes output m to (j / Ns) Ns Q + (j mod Ns) + m Ns.
// Twiddle indices into tw[m] = exp(-2 pi i m / N): q (j mod Ns) N / (Ns Q) < N.
// P = 2^lp columns per tile; j / Ns by a multiply-high with ceil(2^32 / Ns), exact for
// j < 2^14 and Ns <= 2^13 (j < N/2 <= 4096 here).
template <typename R> __host__ __device__ constexpr int mr_threads() { return sizeof(R) == 4 ? 512 : 256; }

template <typename C, int Q>
__device__ __forceinline__ void mr_stage(const C* __restrict__ in, C* __restrict__ out, int N, int lp, int Ns,
                                         const C* __restrict__ tw) {
  const int P = 1 << lp;
  const int L = N / Q, ts = N / (Ns * Q);
  const unsigned mag = Ns > 1 ? (unsigned)((0x100000000ull + (unsigned)Ns - 1) / (unsigned)Ns) : 0u;
  C w[Q];  // Q-th roots of unity exp(-2 pi i s / Q)
#pragma unroll
  for (int s = 0; s < Q; ++s) w[s] = tw[s * L];
  for (int e = threadIdx.x; e < L * P; e += blockDim.x) {
    const int j = e >> lp, p = e & (P - 1);
    const int jq = mag ? (int)__umulhi((unsigned)j, mag) : j;  // j / Ns
    const int k = j - jq * Ns;
    C a[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) a[q] = in[(j + q * L) * P + p];
    if (k > 0) {
#pragma unroll
      for (int q = 1; q < Q; ++q) a[q] = cmul(a[q], tw[q * k * ts]);
    }
    C o[Q];
    if constexpr (Q == 8) {
      dft8(a);
#pragma unroll
      for (int m = 0; m < 8; ++m) o[m] = a[m];
    } else if constexpr (Q == 4) {
      dft4(a[0], a[1], a[2], a[3]);
#pragma unroll
      for (int m = 0; m < 4; ++m) o[m] = a[m];
    } else if constexpr (Q == 2) {
      o[0] = cadd(a[0], a[1]);
      o[1] = csub(a[0], a[1]);
    } else {
      // the Q-point DFT by its definition: o_m = sum_q a_q w^(q m mod Q)
#pragma unroll
      for (int m = 0; m < Q; ++m) {
        C acc = a[0];
#pragma unroll
        for (int q = 1; q < Q; ++q) acc = cadd(acc, cmul(a[q], w[(q * m) % Q]));
        o[m] = acc;
      }
    }
    const int base = jq * Ns * Q + k;
#pragma unroll
    for (int m = 0; m < Q; ++m) out[(base + m * Ns) * P + p] = o[m];
  }
}

// forward DFT of the P columns in b0 (tw: the twiddle table in shared memory); returns the
// buffer that holds the result
template <typename C>
__device__ C* mr_fft(C* b0, C* b1, int N, int lp, const MrPlan& pl, const C* __restrict__ tw) {
  C* in = b0;
  C* out = b1;
  int Ns = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int Q = pl.rad[s];
    switch (Q) {
      case 2: mr_stage<C, 2>(in, out, N, lp, Ns, tw); break;
      case 3: mr_stage<C, 3>(in, out, N, lp, Ns, tw); break;
      case 4: mr_stage<C, 4>(in, out, N, lp, Ns, tw); break;
      case 5: mr_stage<C, 5>(in, out, N, lp, Ns, tw); break;
      case 7: mr_stage<C, 7>(in, out, N, lp, Ns, tw); break;
      default: mr_stage<C, 8>(in, out, N, lp, Ns, tw); break;
    }
    __syncthreads();
    Ns *= Q;
    C* t = in;
    in = out;
    out = t;
  }
  return in;
}

// Step (a) for the mixed-radix column tile at x0 (2P real columns): load and scale, transform,
// untangle the two real columns' bins 0..N/2 into spec. b0, b1: two P x N complex buffers; stw:
// the twiddle table (N complex) in shared memory, written before the call (the first barrier
// here makes it visible). NT = the CTA's threads (the strided loops assume blockDim.x == NT).
// Ends without a barrier: synchronise before reusing the buffers.
template <typename R, typename IN, int NT>
__device__ __forceinline__ void fft_fwd_mr_tile(const IN* __restrict__ v, C_t<R>* __restrict__ spec, int nx, int N,
                                                const MrPlan& pl, int lp, int pitch, const R* __restrict__ lam, R sc,
                                                int x0, C_t<R>* b0, C_t<R>* b1, const C_t<R>* stw) {
  using C = C_t<R>;
  const int P = 1 << lp, W = 2 * P;
  R* flat = reinterpret_cast<R*>(b0);
  // real column c of the tile is the real (c even) or imaginary (c odd) part of complex column c/2;
  // unrolled so that a thread's global loads are in flight together
#pragma unroll 8
  for (int e = threadIdx.x; e < N * W; e += NT) {
    const int t = e >> (lp + 1), c = e & (W - 1), x = x0 + c;
    R val = (R)0;
    if (x < nx) val = in_r<R>(__ldg(v + (size_t)t * nx + x)) * (__ldg(&lam[t]) * sc);
    flat[e] = val;
  }
  __syncthreads();
  const C* Z = mr_fft(b0, b1, N, lp, pl, stw);
  // bins 0..N/2 of the two real columns: X_a = (Z_k + conj Z_{N-k}) / 2, X_b = (Z_k - conj Z_{N-k}) / 2i
  const int K = N / 2 + 1;
  for (int e = threadIdx.x; e < K * P; e += NT) {
    const int k = e >> lp, p = e & (P - 1);
    const C zk = Z[k * P + p];
    const C zn = Z[(k == 0 ? 0 : N - k) * P + p];
    const R h = (R)0.5;
    const int x = x0 + 2 * p;
    C* out = spec + (size_t)k * pitch + x;
    if (!AAO_DCHECK(k <= N / 2 && x + 1 <= pitch)) continue;
    if (x < nx) out[0] = cmk<C>(h * (zk.x + zn.x), h * (zk.y - zn.y));
    if (x + 1 < nx) out[1] = cmk<C>(h * (zk.y + zn.y), h * (zn.x - zk.x));
  }
}

// Step (c) for the mixed-radix column tile at x0: the full spectrum of the two real columns from
// their half spectra, the transform, Lambda_alpha^{-1}, the real columns out. Buffers and NT as for
// fft_fwd_mr_tile. Ends without a barrier.
template <typename R, typename OUT, int NT>
__device__ __forceinline__ void fft_inv_mr_tile(const C_t<R>* __restrict__ spec, OUT* __restrict__ z, int nx, int N,
                                                const MrPlan& pl, int lp, int pitch, const R* __restrict__ ilam,
                                                int x0, C_t<R>* b0, C_t<R>* b1, const C_t<R>* stw) {
  using C = C_t<R>;
  const int P = 1 << lp, W = 2 * P;
  const int K = N / 2 + 1;
  // Z_k = A_k + i B_k for all k from the half spectra (A_{N-k} = conj A_k), stored conjugated:
  // the inverse DFT is the conjugate of the forward DFT of the conjugate
#pragma unroll 4
  for (int e = threadIdx.x; e < K * P; e += NT) {
    const int k = e >> lp, p = e & (P - 1);
    const int x = x0 + 2 * p;
    const C* in = spec + (size_t)k * pitch + x;
    C A = cmk<C>(0, 0), B = cmk<C>(0, 0);
    if (x < nx) A = in[0];
    if (x + 1 < nx) B = in[1];
    const bool self = (k == 0) || (2 * k == N);  // DC and (N even) Nyquist bins of a real signal
    if (self) { A.y = 0; B.y = 0; }
    b0[k * P + p] = cmk<C>(A.x - B.y, -(A.y + B.x));
    if (!self) b0[(N - k) * P + p] = cmk<C>(A.x + B.y, A.y - B.x);
  }
  __syncthreads();
  const C* Y = mr_fft(b0, b1, N, lp, pl, stw);
#pragma unroll 4
  for (int e = threadIdx.x; e < N * W; e += NT) {
    const int t = e >> (lp + 1), c = e & (W - 1), x = x0 + c;
    if (x < nx) {
      const C y = Y[t * P + (c >> 1)];
      const R val = ((c & 1) ? -y.y : y.x) * __ldg(&ilam[t]);
      if (AAO_DCHECK(t < N)) z[(size_t)t * nx + x] = (OUT)val;
    }
  }
}

}  // namespace pdev
}  // namespace aao

// P_alpha^{-1} apply on GB300: the three steps of Eq. 3.2 with the conjugate-pair saving of
// Remark 1, as three kernels joined by the half spectrum in HBM/L2.
//
//   k_fft_fwd   step (a): Lambda_alpha scaling (first factor of V_alpha^{-1} = F Lambda_alpha)
//               fused with a real-to-complex FFT along t for a tile of 2P spatial columns.
//               Two real columns are packed into one complex column; the FFT is a Stockham
//               radix-4/2 transform in shared memory. Output: bins k = 0..nt/2 of every
//               column, frequency-major [k][x] (the layout step (b) reads contiguously).
//   k_tridiag   step (b): for each bin k one warp solves the complex-shifted tridiagonal system
//               (lambda_{1,k} I - lambda_{2,k} A~) z2_k = z1_k, A~ = tau * Abar, by a partitioned
//               Thomas sweep per lane (chunks of ceil(nx/32) rows) and parallel cyclic reduction
//               of the 64-row interface system across the warp with shuffles.
//   k_fft_inv   step (c): complex-to-real inverse FFT along t (bins nt/2+1.. are the conjugates,
//               Remark 1) fused with Lambda_alpha^{-1} and the 1/nt normalisation.
//
// The unitary DFT of Sec. 3.1 carries 1/sqrt(nt) in each direction; here the forward FFT is
// unnormalised and the single 1/nt is folded into the unscaling table.
#include "aao_internal.cuh"

namespace aao {

namespace {

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
        if (r > 0 && k > 0) a = cmul(a, __ldg(&tw[(r * k) << lts]));
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
template <> __device__ __forceinline__ float to_r<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ double to_r<double>(double v) { return v; }

// step (a)
template <typename R>
__global__ void __launch_bounds__(sizeof(R) == 8 ? 512 : 1024) k_fft_fwd(const double* __restrict__ v, C_t<R>* __restrict__ spec,
                                                  int nx, int N, int log2n, int P, int pitch,
                                                  const R* __restrict__ lam, const C_t<R>* __restrict__ tw,
                                                  const double* __restrict__ in_scale) {
  using C = C_t<R>;
  const R sc = in_scale ? (R)(*in_scale) : (R)1;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* data = reinterpret_cast<C*>(smraw);
  R* flat = reinterpret_cast<R*>(smraw);
  // P is a power of two <= 16 and blockDim.x a multiple of 32, so W = 2P divides blockDim.x:
  // thread owns tile column c and rows t = tr, tr + tstep, ... (independent loads in flight)
  const int W = 2 * P;
  const int x0 = blockIdx.x * W;
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
  smem_fft(data, log2n, lp, tw);
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

// step (c)
template <typename R, typename OUT>
__global__ void __launch_bounds__(sizeof(R) == 8 ? 512 : 1024) k_fft_inv(const C_t<R>* __restrict__ spec, OUT* __restrict__ z,
                                                  int nx, int N, int log2n, int P, int pitch,
                                                  const R* __restrict__ ilam, const C_t<R>* __restrict__ tw) {
  using C = C_t<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* data = reinterpret_cast<C*>(smraw);
  const int W = 2 * P;
  const int x0 = blockIdx.x * W;
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
  smem_fft(data, log2n, lp, tw);
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

// step (b): one CTA per frequency bin k. Row i of (mu_k I - A~), mu_k = lambda_{1,k}/lambda_{2,k},
// right-hand side z1_k / lambda_{2,k}: a_i = -lo_i, b_i = mu_k - di_i, c_i = -up_i. Thread l owns
// rows [l ch, (l+1) ch) (padding rows beyond nx are identity rows). A modified Thomas sweep
// expresses every row of the chunk through the chunk's first and last unknowns (multipliers in
// registers, right-hand sides in shared memory); the 2T first/last rows form a tridiagonal
// interface system solved by parallel cyclic reduction in shared memory; back substitution
// recovers the interior rows.
template <typename R, int CH>
__global__ void __launch_bounds__(512) k_tridiag(C_t<R>* __restrict__ spec, int nx, int pitch, int ch, int cs,
                                                 const R* __restrict__ lo, const R* __restrict__ di,
                                                 const R* __restrict__ up, const C_t<R>* __restrict__ mu,
                                                 const C_t<R>* __restrict__ il2) {
  using C = C_t<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int T = blockDim.x, tid = threadIdx.x, k = blockIdx.x;
  C* dd = reinterpret_cast<C*>(smraw);
  C* pa = dd + (size_t)T * cs;
  C* pb = pa + 2 * T;
  C* pc = pb + 2 * T;
  C* pd = pc + 2 * T;
  const C muk = mu[k], sk = il2[k];
  C* row = spec + (size_t)k * pitch;
  const C zero = cmk<C>(0, 0), one = cmk<C>(1, 0);
  for (int i = tid; i < T * ch; i += T) {
    const int L = i / ch, j = i - L * ch;
    dd[L * cs + j] = (i < nx) ? cmul(row[i], sk) : zero;
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
      C a = zero, b = one, c = zero;
      if (i < nx) {
        a = cmk<C>(i > 0 ? -__ldg(&lo[i]) : (R)0, 0);
        b = cmk<C>(muk.x - __ldg(&di[i]), muk.y);
        c = cmk<C>(i < nx - 1 ? -__ldg(&up[i]) : (R)0, 0);
      }
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
  for (int i = tid; i < nx; i += T) {
    const int L = i / ch, j = i - L * ch;
    row[i] = dd[L * cs + j];
  }
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

template <typename R>
int run_precond(Handle& h, const double* v, void* z, bool z_is_float, const double* in_scale) {
  using C = C_t<R>;
  const int N = h.nt, nx = h.nx;
  const int P = h.fft_p > 0 ? h.fft_p : default_tile(nx, N, sizeof(R));
  int threads = fft_threads(P, N, sizeof(R));
  const size_t smem = (size_t)P * N * sizeof(C);
  const int grid = (nx + 2 * P - 1) / (2 * P);
  C* spec = reinterpret_cast<C*>(h.spec);
  const R* lam = (sizeof(R) == 4) ? (const R*)h.lamf : (const R*)h.lam;
  const R* ilam = (sizeof(R) == 4) ? (const R*)h.ilamf : (const R*)h.ilam;
  const C* tw = (sizeof(R) == 4) ? (const C*)h.twf : (const C*)h.tw;

  AAO_TRY_CUDA(cudaFuncSetAttribute(k_fft_fwd<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const double nsp = (double)h.K * nx * sizeof(C);   // half spectrum, bins 0..nt/2
  const double nv = (double)nx * N;
  {
    ProfScope ps(AAO_K_FFT_FWD, h.stream, nv * sizeof(double) + nsp);
    k_fft_fwd<R><<<grid, threads, smem, h.stream>>>(v, spec, nx, N, h.log2n, P, h.pitch, lam, tw, in_scale);
  }
  AAO_CHECK_LAUNCH();

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
  const size_t smem2 = ((size_t)T * cs + 8 * (size_t)T) * sizeof(C);
  const R* lo = (sizeof(R) == 4) ? (const R*)h.pLf : (const R*)h.pL;
  const R* di = (sizeof(R) == 4) ? (const R*)h.pDf : (const R*)h.pD;
  const R* up = (sizeof(R) == 4) ? (const R*)h.pUf : (const R*)h.pU;
  const C* mu = (sizeof(R) == 4) ? (const C*)h.muf : (const C*)h.mu;
  const C* il2 = (sizeof(R) == 4) ? (const C*)h.il2f : (const C*)h.il2;
  AAO_TRY_CUDA(cudaFuncSetAttribute(k_tridiag<R, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
  {
    ProfScope ps(AAO_K_TRIDIAG, h.stream, 2.0 * nsp);
    k_tridiag<R, CH><<<h.K, T, smem2, h.stream>>>(spec, nx, h.pitch, ch, cs, lo, di, up, mu, il2);
  }
  AAO_CHECK_LAUNCH();

  if (z_is_float) {
    AAO_TRY_CUDA(cudaFuncSetAttribute(k_fft_inv<R, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope ps(AAO_K_FFT_INV, h.stream, nsp + nv * sizeof(float));
    k_fft_inv<R, float><<<grid, threads, smem, h.stream>>>(spec, (float*)z, nx, N, h.log2n, P, h.pitch, ilam, tw);
  } else {
    AAO_TRY_CUDA(cudaFuncSetAttribute(k_fft_inv<R, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope ps(AAO_K_FFT_INV, h.stream, nsp + nv * sizeof(double));
    k_fft_inv<R, double><<<grid, threads, smem, h.stream>>>(spec, (double*)z, nx, N, h.log2n, P, h.pitch, ilam, tw);
  }
  AAO_CHECK_LAUNCH();
  return AAO_OK;
}

}  // namespace

int launch_precond(Handle& h, const double* v, void* z, bool z_is_float, const double* in_scale) {
  if (h.mixed) return run_precond<float>(h, v, z, z_is_float, in_scale);
  return run_precond<double>(h, v, z, z_is_float, in_scale);
}

// FFT tile autotuner: time the whole apply for every admissible tile width 2P (P = 1, 2, 4, ...)
// on this problem's sizes and keep the fastest. Every tile width computes identical results
// (each column's transform runs the same operations in the same order); only speed differs.
int tune_precond(Handle& h) {
  const size_t rs = h.mixed ? 4 : 8;
  const int pmax = max_tile(h.nt, rs);
  if (pmax == 1) {
    h.fft_p = 1;
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
  int bestp = default_tile(h.nx, h.nt, rs);
  int rc = AAO_OK;
  for (int P = 1; P <= pmax && rc == AAO_OK; P <<= 1) {
    h.fft_p = P;
    rc = launch_precond(h, v, z, h.mixed);
    if (rc != AAO_OK) break;
    cudaEventRecord(e0, h.stream);
    for (int r = 0; r < 3 && rc == AAO_OK; ++r) rc = launch_precond(h, v, z, h.mixed);
    cudaEventRecord(e1, h.stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; bestp = P; }
  }
  h.fft_p = bestp;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(v);
  cudaFree(z);
  return rc;
}

}  // namespace aao

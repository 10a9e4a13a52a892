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

// One in-place Stockham stage of radix R (4 or 2) over P interleaved columns stored [t][P].
// Butterfly j (0 <= j < N/R) of column p reads elements j + r N/R, twiddles them by
// exp(-2 pi i r (j mod Ns) / (Ns R)), and writes (j / Ns) Ns R + (j mod Ns) + r Ns.
template <typename C, int R>
__device__ __forceinline__ void stockham_stage(C* __restrict__ data, int N, int P, int Ns,
                                               const C* __restrict__ tw) {
  constexpr int B = kVals / R;
  const int nbf = P * (N / R);
  const int stride_in = N / R;
  const int tstep = N / (Ns * R);
  C reg[B][R];
#pragma unroll
  for (int q = 0; q < B; ++q) {
    const int b = threadIdx.x + q * blockDim.x;
    if (b < nbf) {
      const int p = b % P, j = b / P, k = j % Ns;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C a = data[(j + r * stride_in) * P + p];
        if (r > 0 && k > 0) a = cmul(a, __ldg(&tw[r * k * tstep]));
        reg[q][r] = a;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < B; ++q) {
    const int b = threadIdx.x + q * blockDim.x;
    if (b < nbf) {
      const int p = b % P, j = b / P, k = j % Ns;
      if (R == 4) {
        dft4(reg[q][0], reg[q][1], reg[q][2], reg[q][3]);
      } else {
        C t0 = reg[q][0];
        reg[q][0] = cadd(t0, reg[q][1]);
        reg[q][1] = csub(t0, reg[q][1]);
      }
      const int base = (j / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) data[(base + r * Ns) * P + p] = reg[q][r];
    }
  }
  __syncthreads();
}

// Forward DFT (exp(-2 pi i t k / N)) of P columns of length N = 2^log2n in shared memory.
template <typename C>
__device__ void smem_fft(C* data, int N, int log2n, int P, const C* tw) {
  int Ns = 1;
  for (int s = 0; s < log2n / 2; ++s) {
    stockham_stage<C, 4>(data, N, P, Ns, tw);
    Ns *= 4;
  }
  if (log2n & 1) stockham_stage<C, 2>(data, N, P, Ns, tw);
}

template <typename R> __device__ __forceinline__ R to_r(double v);
template <> __device__ __forceinline__ float to_r<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ double to_r<double>(double v) { return v; }

// step (a)
template <typename R>
__global__ void __launch_bounds__(sizeof(R) == 8 ? 512 : 1024) k_fft_fwd(const double* __restrict__ v, C_t<R>* __restrict__ spec,
                                                  int nx, int N, int log2n, int P, int pitch,
                                                  const R* __restrict__ lam, const C_t<R>* __restrict__ tw) {
  using C = C_t<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* data = reinterpret_cast<C*>(smraw);
  R* flat = reinterpret_cast<R*>(smraw);
  const int W = 2 * P;
  const int x0 = blockIdx.x * W;
  for (int e = threadIdx.x; e < N * W; e += blockDim.x) {
    const int t = e / W, c = e - t * W;
    const int x = x0 + c;
    R val = (R)0;
    if (x < nx) val = to_r<R>(__ldg(&v[(size_t)t * nx + x])) * __ldg(&lam[t]);
    flat[e] = val;  // complex column c/2, real part for even c, imaginary for odd c
  }
  __syncthreads();
  smem_fft(data, N, log2n, P, tw);
  const int half = N / 2;
  for (int e = threadIdx.x; e < (half + 1) * P; e += blockDim.x) {
    const int k = e / P, p = e - k * P;
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
  for (int e = threadIdx.x; e < (half + 1) * P; e += blockDim.x) {
    const int k = e / P, p = e - k * P;
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
  smem_fft(data, N, log2n, P, tw);
  for (int e = threadIdx.x; e < N * W; e += blockDim.x) {
    const int t = e / W, c = e - t * W;
    const int x = x0 + c;
    if (x < nx) {
      const C y = data[t * P + (c >> 1)];
      const R val = ((c & 1) ? -y.y : y.x) * __ldg(&ilam[t]);
      z[(size_t)t * nx + x] = (OUT)val;
    }
  }
}

// step (b)
template <typename R>
__global__ void __launch_bounds__(256) k_tridiag(C_t<R>* __restrict__ spec, int nx, int K, int pitch, int ch,
                                                 int cs, const R* __restrict__ lo, const R* __restrict__ di,
                                                 const R* __restrict__ up, const C_t<R>* __restrict__ mu,
                                                 const C_t<R>* __restrict__ il2) {
  using C = C_t<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * (blockDim.x >> 5) + warp;
  if (k >= K) return;  // the whole warp leaves together; only warp-level sync below
  const int span = 32 * cs;
  C* dd = reinterpret_cast<C*>(smraw) + (size_t)warp * 3 * span;
  C* aa = dd + span;
  C* cc = aa + span;
  const C muk = mu[k], sk = il2[k];
  C* row = spec + (size_t)k * pitch;
  const C zero = cmk<C>(0, 0);
  const int npad = 32 * ch;
  for (int i = lane; i < npad; i += 32) {
    const int L = i / ch, j = i - L * ch;
    dd[L * cs + j] = (i < nx) ? cmul(row[i], sk) : zero;
  }
  __syncwarp();

  // Row i of (mu I - A~): a_i = -lo_i, b_i = mu - di_i, c_i = -up_i; padding rows are identity.
  auto coef = [&](int i, C& a, C& b, C& c) {
    if (i < nx) {
      a = cmk<C>(i > 0 ? -__ldg(&lo[i]) : (R)0, 0);
      b = cmk<C>(muk.x - __ldg(&di[i]), muk.y);
      c = cmk<C>(i < nx - 1 ? -__ldg(&up[i]) : (R)0, 0);
    } else {
      a = zero; b = cmk<C>(1, 0); c = zero;
    }
  };

  const int s = lane * ch;
  C* d_ = dd + lane * cs;
  C* a_ = aa + lane * cs;
  C* c_ = cc + lane * cs;
  // forward sweep: rows 0, 1 normalised; rows j >= 2 expressed in terms of x_s and x_{j+1}
  C ap, cp, dp;
  for (int j = 0; j < 2; ++j) {
    C a, b, c;
    coef(s + j, a, b, c);
    const C ib = cinv(b);
    ap = cmul(a, ib); cp = cmul(c, ib); dp = cmul(d_[j], ib);
    a_[j] = ap; c_[j] = cp; d_[j] = dp;
  }
  for (int j = 2; j < ch; ++j) {
    C a, b, c;
    coef(s + j, a, b, c);
    const C r = cinv(csub(b, cmul(a, cp)));
    dp = cmul(r, csub(d_[j], cmul(a, dp)));
    ap = cscale(cmul(r, cmul(a, ap)), (R)-1);
    cp = cmul(r, c);
    a_[j] = ap; c_[j] = cp; d_[j] = dp;
  }
  C A0, C0, D0, A1, C1, D1;
  A1 = a_[ch - 1]; C1 = c_[ch - 1]; D1 = d_[ch - 1];
  if (ch >= 3) {
    // backward sweep: rows 1..ch-2 expressed in terms of x_s and x_e
    C an = a_[ch - 2], cn = c_[ch - 2], dn = d_[ch - 2];
    for (int j = ch - 3; j >= 1; --j) {
      const C cj = c_[j];
      dn = csub(d_[j], cmul(cj, dn));
      an = csub(a_[j], cmul(cj, an));
      cn = cscale(cmul(cj, cn), (R)-1);
      a_[j] = an; c_[j] = cn; d_[j] = dn;
    }
    // row 0: eliminate x_1 with row 1
    const C c0 = c_[0];
    const C r = cinv(csub(cmk<C>(1, 0), cmul(c0, a_[1])));
    D0 = cmul(r, csub(d_[0], cmul(c0, d_[1])));
    A0 = cmul(r, a_[0]);
    C0 = cscale(cmul(r, cmul(c0, c_[1])), (R)-1);
  } else {
    A0 = a_[0]; C0 = c_[0]; D0 = d_[0];
  }
  // parallel cyclic reduction of the 64-row interface system, rows 2*lane (x_s), 2*lane+1 (x_e)
  C B0 = cmk<C>(1, 0), B1 = cmk<C>(1, 0);
  auto shfl = [](C v, int src) { return cmk<C>(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)); };
  for (int delta = 1; delta < 64; delta <<= 1) {
    C lA0, lB0, lC0, lD0, hA0, hB0, hC0, hD0;  // neighbours of row 2L
    C lA1, lB1, lC1, lD1, hA1, hB1, hC1, hD1;  // neighbours of row 2L+1
    const C one = cmk<C>(1, 0);
    if (delta == 1) {
      const int src = lane > 0 ? lane - 1 : 0;
      lA0 = shfl(A1, src); lB0 = shfl(B1, src); lC0 = shfl(C1, src); lD0 = shfl(D1, src);
      if (lane == 0) { lA0 = zero; lB0 = one; lC0 = zero; lD0 = zero; }
      hA0 = A1; hB0 = B1; hC0 = C1; hD0 = D1;
      lA1 = A0; lB1 = B0; lC1 = C0; lD1 = D0;
      const int srh = lane < 31 ? lane + 1 : 31;
      hA1 = shfl(A0, srh); hB1 = shfl(B0, srh); hC1 = shfl(C0, srh); hD1 = shfl(D0, srh);
      if (lane == 31) { hA1 = zero; hB1 = one; hC1 = zero; hD1 = zero; }
    } else {
      const int o = delta >> 1;
      const int sl = lane >= o ? lane - o : lane, sh = lane + o < 32 ? lane + o : lane;
      lA0 = shfl(A0, sl); lB0 = shfl(B0, sl); lC0 = shfl(C0, sl); lD0 = shfl(D0, sl);
      hA0 = shfl(A0, sh); hB0 = shfl(B0, sh); hC0 = shfl(C0, sh); hD0 = shfl(D0, sh);
      lA1 = shfl(A1, sl); lB1 = shfl(B1, sl); lC1 = shfl(C1, sl); lD1 = shfl(D1, sl);
      hA1 = shfl(A1, sh); hB1 = shfl(B1, sh); hC1 = shfl(C1, sh); hD1 = shfl(D1, sh);
      if (lane < o) { lA0 = zero; lB0 = one; lC0 = zero; lD0 = zero; lA1 = zero; lB1 = one; lC1 = zero; lD1 = zero; }
      if (lane + o >= 32) { hA0 = zero; hB0 = one; hC0 = zero; hD0 = zero; hA1 = zero; hB1 = one; hC1 = zero; hD1 = zero; }
    }
    {
      const C k1 = cmul(A0, cinv(lB0)), k2 = cmul(C0, cinv(hB0));
      const C nA = cscale(cmul(lA0, k1), (R)-1), nC = cscale(cmul(hC0, k2), (R)-1);
      const C nB = csub(csub(B0, cmul(lC0, k1)), cmul(hA0, k2));
      const C nD = csub(csub(D0, cmul(lD0, k1)), cmul(hD0, k2));
      A0 = nA; B0 = nB; C0 = nC; D0 = nD;
    }
    {
      const C k1 = cmul(A1, cinv(lB1)), k2 = cmul(C1, cinv(hB1));
      const C nA = cscale(cmul(lA1, k1), (R)-1), nC = cscale(cmul(hC1, k2), (R)-1);
      const C nB = csub(csub(B1, cmul(lC1, k1)), cmul(hA1, k2));
      const C nD = csub(csub(D1, cmul(lD1, k1)), cmul(hD1, k2));
      A1 = nA; B1 = nB; C1 = nC; D1 = nD;
    }
  }
  const C xs = cmul(D0, cinv(B0)), xe = cmul(D1, cinv(B1));
  // back substitution of the chunk interior
  for (int j = 1; j < ch - 1; ++j) d_[j] = csub(csub(d_[j], cmul(a_[j], xs)), cmul(c_[j], xe));
  d_[0] = xs;
  d_[ch - 1] = xe;
  __syncwarp();
  for (int i = lane; i < nx; i += 32) {
    const int L = i / ch, j = i - L * ch;
    row[i] = dd[L * cs + j];
  }
}

template <typename R>
int run_precond(Handle& h, const double* v, void* z, bool z_is_float) {
  using C = C_t<R>;
  const int N = h.nt, nx = h.nx;
  const int vmax = (sizeof(R) == 4) ? 16384 : 8192;  // P * N bound from registers / smem
  int P = nx / 512;
  if (P < 1) P = 1;
  if (P > vmax / N) P = vmax / N;
  if (P < 1) P = 1;
  int threads = (P * N + kVals - 1) / kVals;
  threads = ((threads + 31) / 32) * 32;
  if (threads < 64) threads = 64;
  const int tmax = sizeof(R) == 8 ? 512 : 1024;  // the kernels' launch bounds
  if (threads > tmax) threads = tmax;
  // also cover the load/post loops comfortably
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
    k_fft_fwd<R><<<grid, threads, smem, h.stream>>>(v, spec, nx, N, h.log2n, P, h.pitch, lam, tw);
  }
  AAO_CHECK_LAUNCH();

  const int ch = nx <= 64 ? 2 : (nx + 31) / 32;
  const int cs = (ch & 1) ? ch + 2 : ch + 1;
  const size_t per_warp = (size_t)3 * 32 * cs * sizeof(C);
  int wpb = (int)((100 * 1024) / per_warp);
  if (wpb < 1) wpb = 1;
  if (wpb > 8) wpb = 8;
  const size_t smem2 = per_warp * wpb;
  if (smem2 > 220 * 1024) {
    set_error("precond_apply: nx too large for the shared-memory tridiagonal solver");
    return AAO_EUNSUPPORTED;
  }
  const R* lo = (sizeof(R) == 4) ? (const R*)h.pLf : (const R*)h.pL;
  const R* di = (sizeof(R) == 4) ? (const R*)h.pDf : (const R*)h.pD;
  const R* up = (sizeof(R) == 4) ? (const R*)h.pUf : (const R*)h.pU;
  const C* mu = (sizeof(R) == 4) ? (const C*)h.muf : (const C*)h.mu;
  const C* il2 = (sizeof(R) == 4) ? (const C*)h.il2f : (const C*)h.il2;
  AAO_TRY_CUDA(cudaFuncSetAttribute(k_tridiag<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
  {
    ProfScope ps(AAO_K_TRIDIAG, h.stream, 2.0 * nsp);
    k_tridiag<R><<<(h.K + wpb - 1) / wpb, 32 * wpb, smem2, h.stream>>>(spec, nx, h.K, h.pitch, ch, cs, lo, di, up, mu, il2);
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

int launch_precond(Handle& h, const double* v, void* z, bool z_is_float) {
  if (h.mixed) return run_precond<float>(h, v, z, z_is_float);
  return run_precond<double>(h, v, z, z_is_float);
}

}  // namespace aao

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
//   k_rz_form / k_gj_pivot / k_gj_rowscale / k_gj_update_tc / k_gj_colfix
//                at aao_create: the shifted matrices mu_k I - A~ of step (b) of Eq. 3.2 for the
//                nt/2+1 bins, inverted in place, X_k = (mu_k I - A~)^{-1}, by blocked Gauss-Jordan
//                elimination without pivoting (FP32 complex; the matrices are diagonally dominant);
//                the rank-64 updates that carry the work run on the tensor cores (tcgen05, 3xTF32).
//   k_rz_gemv    per apply: z2_k = X_k z1_k / lambda_2,k for every bin, a dense complex
//                matrix-vector product that streams the inverses once (HBM-bound).
//   k_rz_tc      step (b) when the operator is symmetric (no drift): with tau Abar = Q diag(lambda) Q^T
//                (eigendecomposition at aao_create), z2_k = Q diag(D_k) Q^T z1_k for every bin is two
//                products of the K x Nx complex half spectrum with the real Nx x Nx matrix Q, on the
//                tensor cores (3xTF32). k_rz_split makes each product's complex operand (TF32 head
//                and tail, tiled for TMA); k_rz_cgemm_sum adds the last contraction segments in order.
#include <math.h>
#include <string.h>

#include <complex>
#include <thread>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "krylov_dev.cuh"
#include "precond_dev.cuh"

namespace aao {

namespace {

using namespace kdev;
using namespace pdev;

// ------------------------------------------------------------------- spectral step (b)
// C[k][n] = (D[k][n] *) sum_{s < nseg} P[s][k][n] for k < Kb, n < N (N even; pairs of complex
// per thread), the segments added in order
__global__ void __launch_bounds__(256) k_rz_cgemm_sum(const float2* __restrict__ P, int ldp, int Kb, int N,
                                                      int nseg, float2* __restrict__ C, int ldc,
                                                      const float2* __restrict__ D, int ldd) {
  pdl_sync();
  const int half = N >> 1;
  const size_t total = (size_t)Kb * half, plane = (size_t)Kb * ldp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / half), n = 2 * (int)(e - (size_t)k * half);
    const float4* src = reinterpret_cast<const float4*>(P + (size_t)k * ldp + n);
    float4 v = __ldg(src);
    for (int s = 1; s < nseg; ++s) {
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

// ------------------------------------------------------- spectral step (b) on tensor cores
// The same two products on the 5th-generation tensor cores (tcgen05.mma, FP32 accumulator in
// TMEM). A CTA owns 128 output columns n and 32 bins of one contraction segment:
//   D[n][(bin, c)] = sum_m Op[n][m] * Z[bin][m].c,  c = re, im  (MMA M = 128, N = 64, K = 8),
// Op = Q^T (first product) or Q (second), both stored K-major ([n][m]). TF32 keeps 10 mantissa
// bits, and step (c) multiplies errors by up to 1/alpha, so each operand is split into a TF32
// head and a TF32 tail (x = hi + lo) and three products are accumulated,
// hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32 rounding): FP32 accuracy. Q's split is
// made at create; the complex operand's by k_rz_split, which writes it in the same tiled layout
// (row 2 bin + c), so that both operands reach shared memory by TMA. Operand tiles use the
// K-major layout without swizzling: 8-row x 16-byte core matrices, adjacent along K 128 bytes
// apart and along the rows 1024 bytes apart (32 contraction entries per chunk). A producer warp
// streams the chunks into S buffers; one thread issues the MMAs of each chunk as soon as it has
// landed and releases the buffer with a tcgen05.commit. Every wait is bounded in time (the global
// nanosecond timer): when one gives up, the CTA raises a shared abort flag, the producer stops
// issuing, the TMA loads and the MMAs already issued are waited for (bounded as well), and only
// then is TMEM freed; the kernel records an error code and skips its output (the solve then
// reports AAO_TIMEOUT instead of hanging).
namespace tcg {
constexpr int kM = 128, kN = 64, kKC = 32, kBins = kN / 2;
constexpr int kSegMax = 8;                                     // contraction segments, at most
// chunk buffers per CTA: 144 KB, one CTA per SM, the producer up to 3 chunks ahead. Step (b) of the
// symmetric Riesz operator at 1023 x 512 takes 36.5 us per apply with 3, 38.6 with 4 and 40.9 with 2
// (two CTAs per SM)
constexpr int kStages = 3;
constexpr uint32_t kAop = kM * kKC * 4, kBop = kN * kKC * 4;  // bytes of one operand tile
constexpr uint32_t kStage = 2 * kAop + 2 * kBop;               // hi and lo of both operands
// dynamic shared memory of k_rz_tc<S>: S stages, 2 S + 1 mbarriers and the TMEM slot, alignment
constexpr uint32_t smem_bytes(int S) { return (uint32_t)S * kStage + 16u * S + 16u + 1024u; }
constexpr unsigned long long kWaitNs = 2000000000ull;          // 2 s: far above any legitimate wait

// A staged operand tile (rows x 32 contraction entries, K-major, no swizzling) keeps entry
// (row r, k) at byte ((r / 8) * 8 + k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4: 8-row x 16-byte core
// matrices, the 8 K groups of a row group contiguous.
// shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading byte offset (next
// core matrix along K) >> 4 (bits 16-29), stride byte offset (next 8-row group) >> 4 (bits
// 32-45), descriptor version 1 (bits 46-47), no swizzle (bits 61-63 zero)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(1024u >> 4) << 32) |
         (1ull << 46);
}
// instruction descriptor, kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9 and 10-12 =
// 2), both K-major (bits 15, 16 = 0), N >> 3 (bits 17-22), M >> 4 (bits 24-28)
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kM >> 4) << 24);

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(kIdesc), "r"(acc));
}
__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait for the completion of phase `parity` of an mbarrier: false once wait_ns have passed,
// or (abort != nullptr) as soon as *abort is set by another thread of the CTA
__device__ __forceinline__ bool wait_parity(uint32_t mbar, uint32_t parity, unsigned long long wait_ns,
                                            const volatile int* abort = nullptr) {
  const unsigned long long t0 = now_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (abort && *abort) return false;
    if (now_ns() - t0 > wait_ns) return false;
  }
}
}  // namespace tcg

// TMA load of one operand tile: a box of 256 floats (8 core matrices of one row group) x `rows / 8`
// row groups from a tiled operand (see the tensor maps made at create), completing on mbar
__device__ __forceinline__ void tma_tile(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
// all 128 threads of warps 0-3: true iff every one of them passes true (named barrier 1)
__device__ __forceinline__ bool warps03_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, 1, 128, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

// The complex operand of a tensor-core product, B[2 bin + c][m] (c = re, im) for bin < Kpad and
// m < L, written as TF32 head and tail in the tiled layout of the operands: entry (row r, m) at
// float ((r/8 (L/4) + m/4) 8 + r%8) 4 + m%4. B[bin][m] = D[bin][m] sum_{s < nseg} P[s][bin][m]
// (the segments added in order; no D factor when D is null) for bin < Kb and m < ncols, zero
// elsewhere. One thread per (bin, group of 4 m): four lanes fill one 128-byte core matrix.
__global__ void __launch_bounds__(256) k_rz_split(const float2* __restrict__ P, int ldp, size_t plane, int nseg,
                                                  int Kb, int ncols, const float2* __restrict__ D, int ldd,
                                                  float* __restrict__ Bh, float* __restrict__ Bl, int L, int Kpad) {
  pdl_sync();
  const int ng = L >> 2;
  const size_t total = (size_t)Kpad * ng;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t t = e >> 2;  // (row group, K group) = (t / ng, t % ng)
    const int b = (int)(e & 3);
    const int kg = (int)(t % ng), bin = 4 * (int)(t / ng) + b, m0 = 4 * kg;
    float4 re = make_float4(0.f, 0.f, 0.f, 0.f), im = re;
    if (bin < Kb && m0 < ncols) {
      const float4* src = reinterpret_cast<const float4*>(P + (size_t)bin * ldp + m0);
      float4 u = __ldg(src), w = __ldg(src + 1);
      for (int s = 1; s < nseg; ++s) {
        const float4* q = reinterpret_cast<const float4*>(P + s * plane + (size_t)bin * ldp + m0);
        const float4 u2 = __ldg(q), w2 = __ldg(q + 1);
        u.x += u2.x; u.y += u2.y; u.z += u2.z; u.w += u2.w;
        w.x += w2.x; w.y += w2.y; w.z += w2.z; w.w += w2.w;
      }
      if (D) {
        const float4* dp = reinterpret_cast<const float4*>(D + (size_t)bin * ldd + m0);
        const float4 d0 = __ldg(dp), d1 = __ldg(dp + 1);
        u = make_float4(u.x * d0.x - u.y * d0.y, u.x * d0.y + u.y * d0.x, u.z * d0.z - u.w * d0.w,
                        u.z * d0.w + u.w * d0.z);
        w = make_float4(w.x * d1.x - w.y * d1.y, w.x * d1.y + w.y * d1.x, w.z * d1.z - w.w * d1.w,
                        w.z * d1.w + w.w * d1.z);
      }
      re = make_float4(u.x, u.z, w.x, w.z);
      im = make_float4(u.y, u.w, w.y, w.w);
    }
    const float4 rh = make_float4(tcg::tf32_rna(re.x), tcg::tf32_rna(re.y), tcg::tf32_rna(re.z), tcg::tf32_rna(re.w));
    const float4 ih = make_float4(tcg::tf32_rna(im.x), tcg::tf32_rna(im.y), tcg::tf32_rna(im.z), tcg::tf32_rna(im.w));
    const size_t o = (t * 8 + 2 * b) * 4;  // row 2 b (re) of the core matrix; row 2 b + 1 (im) follows
    *reinterpret_cast<float4*>(Bh + o) = rh;
    *reinterpret_cast<float4*>(Bh + o + 4) = ih;
    *reinterpret_cast<float4*>(Bl + o) = make_float4(tcg::tf32_rna(re.x - rh.x), tcg::tf32_rna(re.y - rh.y),
                                                     tcg::tf32_rna(re.z - rh.z), tcg::tf32_rna(re.w - rh.w));
    *reinterpret_cast<float4*>(Bl + o + 4) = make_float4(tcg::tf32_rna(im.x - ih.x), tcg::tf32_rna(im.y - ih.y),
                                                         tcg::tf32_rna(im.z - ih.z), tcg::tf32_rna(im.w - ih.w));
  }
}

// P[seg][k][n] for k < Kb (see above). ahi / alo: tensor maps of the real operator's head and tail
// (rows n, stored tiled at create); bhi / blo: those of the complex operand made by k_rz_split
// (rows 2 bin + c, padded to a multiple of 32 bins). Segment seg = blockIdx.z covers contraction
// entries [seg Mseg, (seg+1) Mseg), Mseg a multiple of 32. err: set to 1 if a wait gave up. wait_ns
// bounds every wait; inject != 0 (fault injection for tests of the timeout path) makes the
// producer issue no load, so that the first wait for a chunk runs out with nothing in flight.
// Warp 4 is the TMA producer, running ahead as far as the S buffers allow; thread 0 issues the
// MMAs; warps 0-3 then move the accumulator out of TMEM. Per buffer: `full` completes when the
// four tiles of a chunk have landed (transaction count), `empty` when the MMAs that read the
// buffer have finished (tcgen05.commit); `done` when all MMAs of the CTA have.
// Timeout path: the thread whose wait gives up raises the shared abort flag; every other wait
// returns at once when it sees the flag. The producer then issues nothing more and waits for the
// `full` phases of the last load it issued into each buffer, and thread 0 commits what it issued
// to `done` and waits for it, so that no copy into this CTA's shared memory and no MMA is pending
// when TMEM is freed and the CTA exits. These drain waits ignore the flag and are bounded by
// wait_ns too.
template <int S>
__global__ void __launch_bounds__(160) k_rz_tc(const __grid_constant__ CUtensorMap ahi,
                                               const __grid_constant__ CUtensorMap alo,
                                               const __grid_constant__ CUtensorMap bhi,
                                               const __grid_constant__ CUtensorMap blo, float2* __restrict__ P,
                                               int ldp, int Kb, int Mseg, int* __restrict__ err,
                                               unsigned long long wait_ns, int inject) {
  using namespace tcg;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ volatile int abort_flag;
  const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(smraw);
  const uint32_t base = (s0 + 1023u) & ~1023u;  // 1024-aligned operand tiles
  unsigned char* gbase = smraw + (base - s0);
  // full[S] at +0, empty[S] at +8 S, done at +16 S, TMEM slot at +16 S + 8
  const uint32_t bars = base + S * kStage;
  const uint32_t full0 = bars, empty0 = bars + 8 * S, done = bars + 16 * S, slot = done + 8;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int n0 = blockIdx.x * kM, b0 = blockIdx.y * kBins;
  const int nch = Mseg / kKC, c0 = blockIdx.z * nch;  // chunks of this segment: [c0, c0 + nch)
  auto raise_abort = [&]() {
    abort_flag = 1;
    __threadfence_block();
  };

  // set-up that reads nothing the previous kernel writes, before the wait for it (programmatic
  // dependent launch): barriers, the TMEM columns, the tensor maps (kernel parameters)
  if (tid == 0) {
    abort_flag = 0;
    for (int i = 0; i < 2 * S + 1; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bars + 8 * i) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid == 128) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ahi)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&alo)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&bhi)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&blo)) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(kN) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(gbase + (slot - base));
  pdl_sync();

  if (warp == 4) {
    // producer: chunk c into buffer c % S once the MMAs of chunk c - S have released it
    if ((tid & 31) == 0) {
      bool ok = true;
      int issued = 0;
      for (int c = 0; c < nch && !inject; ++c) {
        const int buf = c % S;
        if (abort_flag) break;
        if (c >= S && !wait_parity(empty0 + 8 * buf, ((c - S) / S) & 1, wait_ns, &abort_flag)) {
          if (!abort_flag) { ok = false; raise_abort(); }
          break;
        }
        const uint32_t st = base + buf * kStage, fb = full0 + 8 * buf;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(kStage) : "memory");
        const int x = (c0 + c) * 256;
        tma_tile(st, &ahi, x, n0 / 8, fb);
        tma_tile(st + kAop, &alo, x, n0 / 8, fb);
        tma_tile(st + 2 * kAop, &bhi, x, b0 / 4, fb);
        tma_tile(st + 2 * kAop + kBop, &blo, x, b0 / 4, fb);
        issued = c + 1;
      }
      // drain: the last load issued into each buffer has landed (none newer shares its phase)
      for (int c = issued - S > 0 ? issued - S : 0; c < issued; ++c)
        if (!wait_parity(full0 + 8 * (c % S), (c / S) & 1, wait_ns)) ok = false;
      if (!ok) atomicExch(err, 1);
    }
    __syncwarp();  // the producer lane rejoins its warp before the final barrier
  } else {
    bool mma_ok = true;
    if (tid == 0) {
      int committed = 0;
      for (int c = 0; c < nch; ++c) {
        const int buf = c % S;
        if (!wait_parity(full0 + 8 * buf, (c / S) & 1, wait_ns, &abort_flag)) {
          if (!abort_flag) raise_abort();
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = base + buf * kStage;
#pragma unroll
        for (int ks = 0; ks < kKC / 8; ++ks) {
          const uint32_t ko = ks * 256;  // two core matrices along K per MMA
          const uint64_t ah = sdesc(st + ko), al = sdesc(st + kAop + ko);
          const uint64_t bh = sdesc(st + 2 * kAop + ko), bl = sdesc(st + 2 * kAop + kBop + ko);
          mma(tmem, ah, bh, (c > 0 || ks > 0) ? 1u : 0u);
          mma(tmem, ah, bl, 1u);
          mma(tmem, al, bh, 1u);
        }
        commit(empty0 + 8 * buf);
        committed = c + 1;
      }
      // all MMAs issued by this thread finished (on the timeout path as well: a drain that
      // ignores the flag)
      if (committed > 0) {
        commit(done);
        if (!wait_parity(done, 0, wait_ns)) committed = -1;
      }
      mma_ok = committed == nch;
      if (!mma_ok && !abort_flag) raise_abort();
    }
    __syncwarp();
    const bool ok = warps03_all(mma_ok);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      // warp w reads TMEM lanes 32 w .. 32 w + 31 (output columns n0 + 32 w + lane), 64 columns
      const int n = n0 + 32 * warp + (tid & 31);
      float2* Ps = P + (size_t)blockIdx.z * Kb * ldp;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + 32 * half;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int bin = b0 + 16 * half + j;
          if (bin < Kb && AAO_DCHECK(n < ldp))
            Ps[(size_t)bin * ldp + n] = make_float2(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]));
        }
      }
    } else if (tid == 0) {
      atomicExch(err, 1);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kN) : "memory");
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
  // the last block sums the partials with all its threads (one round trip), then thread 0 writes
  __shared__ double fin[8][NA];
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      double s = 0.0;
      for (unsigned bb = threadIdx.x; bb < gridDim.x; bb += blockDim.x) s += __ldcg(part + (size_t)bb * kPartLd + q);
      s = warp_sum(s);
      if (lane == 0) fin[warp][q] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < NA; ++q) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += fin[w][q];
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

// ------------------------------------------------------------------------------- inverse at create
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

// The inverses X_k = M_k^{-1} by blocked Gauss-Jordan elimination in place, without pivoting (the
// shifted matrices are diagonally dominant), over pivot blocks of kGW columns. Round p, block
// [p0, p0 + wp):
//   k_gj_pivot     P = (A_pp)^{-1}, a kGW x kGW Gauss-Jordan in shared memory (one CTA per bin);
//   k_gj_rowscale  A_pj <- P A_pj for the column tiles j outside the block;
//   k_gj_update_tc A_ij <- A_ij - A_ip A_pj for i, j outside the block: the rank-kGW update that
//                  carries almost all of the work, on the tensor cores (below);
//   k_gj_colfix    A_ip <- -A_ip P for the row tiles i outside the block, and A_pp <- P.
// After the last round A holds M^{-1}. The update reads the block's rows after rowscale and its
// columns before colfix, and writes neither.
constexpr int kGW = 64;

// one bin per CTA of 4 kGW threads; P[k] is kGW x kGW row-major, identity beyond wp. Thread
// (h, j) = (tid / kGW, tid % kGW) owns column j on the kGW/4 rows h kGW/4 ... Step c: the pivot
// column is copied (one entry per thread of the first quarter) and row c read, both before the
// step's first barrier; after it every thread eliminates column c from its rows
// (S[i][j] -= S[i][c] S[c][j] / S[c][c]; column c itself becomes -S[i][c] / S[c][c]) in one
// unrolled, branch-free pass, and the owner of row c then stores the scaled row entry
// S[c][j] / S[c][c] (1 / S[c][c] in column c) over what the pass wrote there. Rows are padded to
// kGW + 1 entries so that the column copy does not hit one bank.
constexpr int kGjPivThreads = 4 * kGW;
__global__ void __launch_bounds__(kGjPivThreads) k_gj_pivot(const float2* __restrict__ M, int nx, int p0, int wp,
                                                            float2* __restrict__ P) {
  constexpr int kR = kGW / 4;  // rows per thread
  __shared__ float2 S[kGW][kGW + 1];
  __shared__ float2 col[kGW];
  const int k = blockIdx.x, j = threadIdx.x % kGW, h = threadIdx.x / kGW;
  const int i0 = h * kR;
  const float2* A = M + (size_t)k * nx * nx;
#pragma unroll 4
  for (int a = i0; a < i0 + kR; ++a)
    S[a][j] = (a < wp && j < wp) ? A[(size_t)(p0 + a) * nx + p0 + j] : make_float2(a == j ? 1.f : 0.f, 0.f);
  __syncthreads();
  for (int c = 0; c < kGW; ++c) {
    if (h == 0) col[j] = S[j][c];
    const float2 scj = S[c][j];  // read by every quarter before the owner of row c rewrites it
    __syncthreads();
    const float2 inv = cinv(col[c]);
    const float2 rc = j == c ? inv : cmul(scj, inv);  // row c of the result, column j
    const bool pc = j == c;
#pragma unroll
    for (int u = 0; u < kR; ++u) {
      const int i = i0 + u;
      const float2 ci = col[i];
      const float2 v = pc ? cscale(cmul(ci, inv), -1.f) : csub(S[i][j], cmul(ci, rc));
      S[i][j] = v;
    }
    if (c >= i0 && c < i0 + kR) S[c][j] = rc;
    __syncthreads();
  }
  float2* Pk = P + (size_t)k * kGW * kGW;
#pragma unroll 4
  for (int a = i0; a < i0 + kR; ++a) Pk[a * kGW + j] = S[a][j];
}

// Products of two kGW x kGW complex tiles in shared memory, for rowscale and colfix: thread t
// forms the 4 x 4 block of outputs (rows 4 (t / 16) .., columns 4 (t % 16) ..), so one round of
// loads (four entries of L's column, two float4 of R's row) feeds 16 complex FMAs.
// acc[u][v] = sum_c L[(4 (t / 16) + u) kGW + c] R[c kGW + 4 (t % 16) + v], c < cn.
__device__ __forceinline__ void tile_mm4x4(const float2* __restrict__ L, const float2* __restrict__ R, int cn,
                                           float2 (&acc)[4][4]) {
  const int r0 = 4 * (threadIdx.x >> 4), c0 = 4 * (threadIdx.x & 15);
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = make_float2(0.f, 0.f);
  for (int c = 0; c < cn; ++c) {
    float2 l[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) l[u] = L[(r0 + u) * kGW + c];
    const float4 ra = *reinterpret_cast<const float4*>(R + c * kGW + c0);
    const float4 rb = *reinterpret_cast<const float4*>(R + c * kGW + c0 + 2);
    const float2 rr[4] = {make_float2(ra.x, ra.y), make_float2(ra.z, ra.w), make_float2(rb.x, rb.y),
                          make_float2(rb.z, rb.w)};
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        acc[u][v].x = fmaf(l[u].x, rr[v].x, fmaf(-l[u].y, rr[v].y, acc[u][v].x));
        acc[u][v].y = fmaf(l[u].x, rr[v].y, fmaf(l[u].y, rr[v].x, acc[u][v].y));
      }
  }
}

// A_pj <- P A_pj on column tile blockIdx.x (kGW columns), bin blockIdx.y; the block's own tile is
// left to k_gj_colfix. Shared memory: P and the tile, 2 kGW^2 complex.
__global__ void __launch_bounds__(256) k_gj_rowscale(float2* __restrict__ M, int nx, int p0, int wp,
                                                     const float2* __restrict__ P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int j0 = blockIdx.x * kGW, k = blockIdx.y;
  if (j0 == p0) return;
  float2* Ps = reinterpret_cast<float2*>(smraw);  // [a][b]
  float2* Ts = Ps + kGW * kGW;                    // [b][jj]
  float2* A = M + (size_t)k * nx * nx;
  const float2* Pk = P + (size_t)k * kGW * kGW;
  for (int e = threadIdx.x; e < kGW * kGW; e += blockDim.x) {
    Ps[e] = Pk[e];
    const int b = e / kGW, jj = e % kGW;
    Ts[e] = (b < wp && j0 + jj < nx) ? A[(size_t)(p0 + b) * nx + j0 + jj] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2 acc[4][4];
  tile_mm4x4(Ps, Ts, wp, acc);
  const int a0 = 4 * (threadIdx.x >> 4), jj0 = 4 * (threadIdx.x & 15);
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int a = a0 + u, jj = jj0 + v;
      if (a < wp && j0 + jj < nx) A[(size_t)(p0 + a) * nx + j0 + jj] = acc[u][v];
    }
}

// A_ip <- -A_ip P on row tile blockIdx.x (kGW rows), bin blockIdx.y; the block's own tile becomes P.
__global__ void __launch_bounds__(256) k_gj_colfix(float2* __restrict__ M, int nx, int p0, int wp,
                                                   const float2* __restrict__ P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int i0 = blockIdx.x * kGW, k = blockIdx.y;
  float2* A = M + (size_t)k * nx * nx;
  const float2* Pk = P + (size_t)k * kGW * kGW;
  if (i0 == p0) {
    for (int e = threadIdx.x; e < kGW * kGW; e += blockDim.x) {
      const int a = e / kGW, b = e % kGW;
      if (a < wp && b < wp) A[(size_t)(p0 + a) * nx + p0 + b] = Pk[e];
    }
    return;
  }
  float2* Ps = reinterpret_cast<float2*>(smraw);  // [a][b]
  float2* Ts = Ps + kGW * kGW;                    // [ii][a]
  for (int e = threadIdx.x; e < kGW * kGW; e += blockDim.x) {
    Ps[e] = Pk[e];
    const int ii = e / kGW, a = e % kGW;
    Ts[e] = (i0 + ii < nx && a < wp) ? A[(size_t)(i0 + ii) * nx + p0 + a] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2 acc[4][4];
  tile_mm4x4(Ts, Ps, wp, acc);
  const int ii0 = 4 * (threadIdx.x >> 4), b0 = 4 * (threadIdx.x & 15);
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int ii = ii0 + u, b = b0 + v;
      if (i0 + ii < nx && b < wp) A[(size_t)(i0 + ii) * nx + p0 + b] = make_float2(-acc[u][v].x, -acc[u][v].y);
    }
}

// The rank-kGW update A_ij -= sum_q A_iq A_qj (q in the pivot block) on the tensor cores. A CTA
// owns 128 rows (i0 ..) and NT column tiles of 32 complex columns (j0 ..); per column tile one
// accumulation D (128 x 64 FP32 in TMEM) = A' B'^T with the complex product embedded in a real one
// along the contraction index kappa = 2q + s:
//   A'[r][2q] = Re A_iq, A'[r][2q+1] = Im A_iq;
//   B'[2j][2q] = Re B_qj, B'[2j][2q+1] = -Im B_qj, B'[2j+1][2q] = Im B_qj, B'[2j+1][2q+1] = Re B_qj,
// so that D[r][2j] + i D[r][2j+1] = sum_q A_iq B_qj. Each operand is split into a TF32 head and
// tail and three products are accumulated (3xTF32, FP32 accuracy), with the operand layout, the
// descriptors and the instruction descriptor of k_rz_tc (K-major, no swizzle, 8-row x 16-byte core
// matrices; M = 128, N = 64, K = 8 per MMA): four 32-entry chunks of kappa per operand. 256 threads
// stage float4 = one 16-byte core-matrix row, eight consecutive rows per quarter warp (conflict-free);
// thread 0 issues the MMAs; the eight warps read the accumulator back by lane quadrant and half.
// Rows and columns inside the pivot block, and beyond nx, are not written. The wait for the MMAs
// is bounded by wait_ns; on a timeout the CTA sets *err, waits (bounded) once more so that no MMA is
// pending, frees TMEM and returns without writing.
constexpr uint32_t kGjA = 4 * 16384u, kGjB = 4 * 8192u;  // one operand (hi or lo), bytes
constexpr uint32_t kGjSmem = 2 * kGjA + 2 * kGjB + 64 + 1024;
constexpr int kGjThreads = 256;
template <int NT>
__global__ void __launch_bounds__(kGjThreads, 1) k_gj_update_tc(float2* __restrict__ M, int nx, int p0, int wp,
                                                                int* __restrict__ err, unsigned long long wait_ns) {
  using namespace tcg;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int k = blockIdx.z, i0 = blockIdx.y * 128, jbase = blockIdx.x * 32 * NT;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float2* A = M + (size_t)k * nx * nx;
  const int pe = p0 + wp;
  // nothing to write: all rows in the pivot block (cannot happen for 128 rows) or all columns in it
  if (jbase >= p0 && jbase + 32 * NT <= pe) return;
  const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(smraw);
  const uint32_t base = (s0 + 1023u) & ~1023u;
  unsigned char* gbase = smraw + (base - s0);
  const uint32_t aHi = base, aLo = base + kGjA, bHi = base + 2 * kGjA, bLo = bHi + kGjB;
  const uint32_t mbar = base + 2 * kGjA + 2 * kGjB, slot = mbar + 8;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(kN) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // A' (rows i0.., the block's columns): float4 e = (row r, q pair qp) at chunk qp >> 3; the loads of
  // four pieces are issued before any of them is converted
  constexpr int kBatch = 8;
  for (int it0 = 0; it0 < 4096 / kGjThreads; it0 += kBatch) {
    float4 v[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = (it0 + u) * kGjThreads + tid;
      const int r = ((e >> 8) << 3) | (e & 7), qp = (e >> 3) & 31;
      const int i = i0 + r, q = 2 * qp;
      v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < nx) {
        const float2* src = A + (size_t)i * nx + p0 + q;
        if (q < wp) { const float2 t = src[0]; v[u].x = t.x; v[u].y = t.y; }
        if (q + 1 < wp) { const float2 t = src[1]; v[u].z = t.x; v[u].w = t.y; }
      }
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = (it0 + u) * kGjThreads + tid;
      const int r = ((e >> 8) << 3) | (e & 7), qp = (e >> 3) & 31;
      const uint32_t off = (uint32_t)((qp >> 3) * 16384 + (((r >> 3) << 3) + (qp & 7)) * 128 + (r & 7) * 16);
      const float4 hi = make_float4(tf32_rna(v[u].x), tf32_rna(v[u].y), tf32_rna(v[u].z), tf32_rna(v[u].w));
      const float4 lo = make_float4(tf32_rna(v[u].x - hi.x), tf32_rna(v[u].y - hi.y), tf32_rna(v[u].z - hi.z),
                                    tf32_rna(v[u].w - hi.w));
      *reinterpret_cast<float4*>(gbase + off) = hi;
      *reinterpret_cast<float4*>(gbase + kGjA + off) = lo;
    }
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(gbase + 2 * kGjA + 2 * kGjB + 8);
  bool ok = true;
  int phase = 0;  // commits issued so far: the mbarrier phase of the next one
  for (int nt = 0; nt < NT && ok; ++nt) {
    const int j0 = jbase + 32 * nt;
    if (j0 >= nx) break;
    if (j0 >= p0 && j0 + 32 <= pe) continue;  // every column of this tile is in the block
    // B' (the block's rows, columns j0..j0+31): float4 e = (row n = 2 j + t, q pair qp); all loads
    // of a thread issued before any is used
    constexpr int kIt = 2048 / kGjThreads;
    float2 bq[kIt][2];
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int e = it * kGjThreads + tid;
      const int n = ((e >> 8) << 3) | (e & 7), qp = (e >> 3) & 31;
      const int j = j0 + (n >> 1), q = 2 * qp;
      bq[it][0] = bq[it][1] = make_float2(0.f, 0.f);
      if (j < nx) {
        if (q < wp) bq[it][0] = A[(size_t)(p0 + q) * nx + j];
        if (q + 1 < wp) bq[it][1] = A[(size_t)(p0 + q + 1) * nx + j];
      }
    }
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int e = it * kGjThreads + tid;
      const int n = ((e >> 8) << 3) | (e & 7), qp = (e >> 3) & 31;
      const int t = n & 1;
      const float2 b0 = bq[it][0], b1 = bq[it][1];
      const float4 v = t == 0 ? make_float4(b0.x, -b0.y, b1.x, -b1.y) : make_float4(b0.y, b0.x, b1.y, b1.x);
      const uint32_t off = (uint32_t)((qp >> 3) * 8192 + (((n >> 3) << 3) + (qp & 7)) * 128 + (n & 7) * 16);
      const float4 hi = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
      const float4 lo = make_float4(tf32_rna(v.x - hi.x), tf32_rna(v.y - hi.y), tf32_rna(v.z - hi.z),
                                    tf32_rna(v.w - hi.w));
      *reinterpret_cast<float4*>(gbase + 2 * kGjA + off) = hi;
      *reinterpret_cast<float4*>(gbase + 2 * kGjA + kGjB + off) = lo;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int c = 0; c < 4; ++c) {
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t ko = ks * 256;
          const uint64_t ah = sdesc(aHi + c * 16384 + ko), al = sdesc(aLo + c * 16384 + ko);
          const uint64_t bh = sdesc(bHi + c * 8192 + ko), bl = sdesc(bLo + c * 8192 + ko);
          mma(tmem, ah, bh, (c > 0 || ks > 0) ? 1u : 0u);
          mma(tmem, ah, bl, 1u);
          mma(tmem, al, bh, 1u);
        }
      }
      commit(mbar);
    }
    // this thread's 16 entries of C (row i, complex columns j0 + 16 (w >> 2) ..), loaded while the
    // MMAs run
    const int i = i0 + 32 * (warp & 3) + lane;
    const bool row_ok = i < nx && (i < p0 || i >= pe);
    const int jc = j0 + 16 * (warp >> 2);
    float2 cv[16];
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      const int j = jc + jj;
      cv[jj] = (row_ok && j < nx) ? A[(size_t)i * nx + j] : make_float2(0.f, 0.f);
    }
    // the MMAs of this tile are done (thread 0 waits; the outcome is shared at the barrier)
    __shared__ int done_s;
    if (tid == 0) {
      const bool d = wait_parity(mbar, (uint32_t)(phase & 1), wait_ns);
      if (!d) {
        atomicExch(err, 1);
        (void)wait_parity(mbar, (uint32_t)(phase & 1), wait_ns);  // drain before TMEM is freed
      }
      done_s = d ? 1 : 0;
    }
    __syncthreads();
    ++phase;
    ok = done_s != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) break;
    // epilogue: warp w reads TMEM lanes 32 (w & 3) .. (rows i0 + 32 (w & 3) + lane) and columns
    // 32 (w >> 2) .. (complex columns jc ..)
    {
      const int half = warp >> 2;
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 32 * half;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row_ok) {
        float2* dst = A + (size_t)i * nx;
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int j = jc + jj;
          if (j < nx && (j < p0 || j >= pe) && AAO_DCHECK(i < nx))
            dst[j] = make_float2(cv[jj].x - __uint_as_float(v[2 * jj]), cv[jj].y - __uint_as_float(v[2 * jj + 1]));
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // TMEM read and B' consumed before the next tile's staging and MMAs
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kN) : "memory");
}

// Step (b) per apply for the Riesz operator with drift: z_k = X_k (z1_k / lambda_2,k) for every
// bin, a dense complex matrix-vector product (the inverses made at create). A CTA owns 16 rows of
// one bin, a warp one row (lanes over columns, eight loads in flight per lane); the bin's
// right-hand side is staged in shared memory. The result goes to out (the half spectrum's shape),
// not in place: other CTAs of the bin still read the right-hand side.
constexpr int kRzGemvRows = 16;
__global__ void __launch_bounds__(32 * kRzGemvRows) k_rz_gemv(const float2* __restrict__ spec, float2* __restrict__ out,
                                                            int nx, int pitch, const float2* __restrict__ X,
                                                            const float2* __restrict__ il2) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* zb = reinterpret_cast<float2*>(smraw);  // nx
  pdl_sync();
  const int k = blockIdx.y, i = blockIdx.x * kRzGemvRows + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  const float2 sk = il2[k];
  const float2* rhs = spec + (size_t)k * pitch;
  for (int j = threadIdx.x; j < nx; j += blockDim.x) zb[j] = cmul(rhs[j], sk);
  __syncthreads();
  if (i >= nx) return;
  const float2* xr = X + ((size_t)k * nx + i) * nx;
  float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
  int j = lane;
  for (; j + 224 < nx; j += 256) {
    float2 l[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) l[u] = __ldg(xr + j + 32 * u);
#pragma unroll
    for (int u = 0; u < 8; u += 2) {
      const float2 va = zb[j + 32 * u], vb = zb[j + 32 * (u + 1)];
      ax = fmaf(l[u].x, va.x, fmaf(-l[u].y, va.y, ax));
      ay = fmaf(l[u].x, va.y, fmaf(l[u].y, va.x, ay));
      bx = fmaf(l[u + 1].x, vb.x, fmaf(-l[u + 1].y, vb.y, bx));
      by = fmaf(l[u + 1].x, vb.y, fmaf(l[u + 1].y, vb.x, by));
    }
  }
  for (; j < nx; j += 32) {
    const float2 l = __ldg(xr + j), v = zb[j];
    ax = fmaf(l.x, v.x, fmaf(-l.y, v.y, ax));
    ay = fmaf(l.x, v.y, fmaf(l.y, v.x, ay));
  }
  float sx = ax + bx, sy = ay + by;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_down_sync(0xffffffffu, sx, o);
    sy += __shfl_down_sync(0xffffffffu, sy, o);
  }
  if (lane == 0 && AAO_DCHECK(i < pitch)) out[(size_t)k * pitch + i] = make_float2(sx, sy);
}

}  // namespace

AAO_CHECK_WORD_FN(check_word_riesz)

int gj_invert_batched(cudaStream_t stream, float2* M, int n, int K) {
  float2* piv = nullptr;
  int* err = nullptr;
  AAO_TRY_CUDA(cudaMalloc(&piv, sizeof(float2) * (size_t)K * kGW * kGW));
  AAO_TRY_CUDA(cudaMalloc(&err, sizeof(int)));
  int rc = AAO_OK;
  if (cudaMemsetAsync(err, 0, sizeof(int), stream) != cudaSuccess) rc = AAO_ECUDA;
  const size_t tsm = 2 * sizeof(float2) * kGW * kGW;
  if (rc == AAO_OK &&
      (cudaFuncSetAttribute(k_gj_rowscale, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm) != cudaSuccess ||
       cudaFuncSetAttribute(k_gj_colfix, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm) != cudaSuccess ||
       cudaFuncSetAttribute(k_gj_update_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGjSmem) !=
           cudaSuccess ||
       cudaFuncSetAttribute(k_gj_update_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGjSmem) !=
           cudaSuccess))
    rc = AAO_ECUDA;
  const int nbt = (n + kGW - 1) / kGW;
  // column tiles per CTA of the update: 16 for wide matrices (the staged pivot columns A' serve
  // more tiles: 55 -> 51 ms for the 257 inverses of order 1023), 4 for narrow ones, which would
  // otherwise leave too few CTAs (the Heston blocks of order 192: 52 against 53 ms)
  const int NT = n >= 512 ? 16 : 4;
  const dim3 gup((n + 32 * NT - 1) / (32 * NT), (n + 127) / 128, K);
  for (int p0 = 0; p0 < n && rc == AAO_OK; p0 += kGW) {
    const int wp = n - p0 < kGW ? n - p0 : kGW;
    k_gj_pivot<<<K, kGjPivThreads, 0, stream>>>(M, n, p0, wp, piv);
    k_gj_rowscale<<<dim3(nbt, K), 256, tsm, stream>>>(M, n, p0, wp, piv);
    if (NT == 16)
      k_gj_update_tc<16><<<gup, kGjThreads, kGjSmem, stream>>>(M, n, p0, wp, err, tcg::kWaitNs);
    else
      k_gj_update_tc<4><<<gup, kGjThreads, kGjSmem, stream>>>(M, n, p0, wp, err, tcg::kWaitNs);
    k_gj_colfix<<<dim3(nbt, K), 256, tsm, stream>>>(M, n, p0, wp, piv);
    g_launches.fetch_add(3, std::memory_order_relaxed);
    rc = [&]() -> int { AAO_CHECK_LAUNCH(); return AAO_OK; }();
  }
  int e = 0;
  if (rc == AAO_OK) {
    if (cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      rc = AAO_ECUDA;
  }
  cudaFree(piv);
  cudaFree(err);
  if (rc == AAO_ECUDA) set_error("gauss-jordan inversion: a CUDA call failed");
  if (rc != AAO_OK) return rc;
  if (e) {
    set_error("aao_create: a tensor-core update of the step (b) inverses gave up a bounded wait");
    return AAO_TIMEOUT;
  }
  return AAO_OK;
}

namespace {

int grid_for(size_t n) {
  size_t g = (n + kThreads - 1) / kThreads;
  return (int)(g < (size_t)kRedBlocks ? g : (size_t)kRedBlocks);
}

}  // namespace

// ------------------------------------------------------------------------------- host
namespace {
// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    cudaGetLastError();
  }
  return fn;
}
// the 2-D map over a tiled operator: rows of ldq * 8 floats (one row group: ldq / 4 core
// matrices of 8 rows x 4 entries), ldq / 8 row groups; boxes of 256 floats x 16 row groups
// tensor map of an operand stored tiled (see k_rz_tc): `rows` rows of L contraction entries, as
// L * 8 floats per 8-row group; one TMA box is 32 entries (8 core matrices) x box_rows rows
int encode_tiled_map(void* map, float* tiled, int L, int rows, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) {
    set_error("aao_create: cuTensorMapEncodeTiled is not available");
    return AAO_ECUDA;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)L * 8, (cuuint64_t)rows / 8};
  const cuuint64_t strides[1] = {(cuuint64_t)L * 8 * sizeof(float)};
  const cuuint32_t box[2] = {256, (cuuint32_t)box_rows / 8};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, tiled, dims, strides,
                         box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("aao_create: cuTensorMapEncodeTiled failed for an operand of the spectral step");
    return AAO_ECUDA;
  }
  return AAO_OK;
}
}  // namespace

// f(begin, end) over [0, n) on the host's cores (contiguous chunks, the caller taking the first)
template <typename F>
void host_parallel(int n, F f) {
  const unsigned hw = std::thread::hardware_concurrency();
  const int T = (int)std::max(1u, std::min(hw == 0 ? 1u : hw, 32u));
  if (T <= 1 || n < 2 * T) {
    f(0, n);
    return;
  }
  const int per = (n + T - 1) / T;
  std::vector<std::thread> th;
  for (int t = 1; t < T; ++t) {
    const int b = t * per, e = std::min(n, b + per);
    if (b < e) th.emplace_back([&f, b, e] { f(b, e); });
  }
  f(0, std::min(n, per));
  for (auto& x : th) x.join();
}

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
  // circulant embedding of length N2 >= 2 nx - 1 and its spectrum (radix-2 FFT in FP64)
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
  {
    // chat[f] = sc sum_q cc[q] exp(-2 pi i f q / N2): iterative radix-2 decimation in time, inputs
    // in bit-reversed order, twiddles exp(-2 pi i j / len) = (cs, sn)[j N2 / len]
    std::vector<double> re(n2), im(n2, 0.0);
    for (int q = 0; q < n2; ++q) {
      int rq = 0;
      for (int b = 0; b < l2; ++b) rq |= ((q >> b) & 1) << (l2 - 1 - b);
      re[rq] = cc[q];
    }
    for (int len = 2; len <= n2; len <<= 1) {
      const int half = len >> 1, step = n2 / len;
      for (int i0 = 0; i0 < n2; i0 += len)
        for (int j = 0; j < half; ++j) {
          const double wr = cs[j * step], wi = sn[j * step];
          const int a = i0 + j, b = a + half;
          const double tr = wr * re[b] - wi * im[b], ti = wr * im[b] + wi * re[b];
          re[b] = re[a] - tr;
          im[b] = im[a] - ti;
          re[a] += tr;
          im[a] += ti;
        }
    }
    for (int f = 0; f < n2; ++f) {
      chat[f] = make_double2(re[f] * sc, im[f] * sc);
      tw2[f] = make_double2(cs[f], sn[f]);
    }
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
    // column tile, >= the spectrum's pitch): q[r][k] = Q[r][k] = Ad[k][r], qt[r][k] = Ad[r][k]
    const int ldq = ((nx + tcg::kM - 1) / tcg::kM) * tcg::kM;
    // D_k,j = (1/lambda_{2,k}) / (mu_k - lambda_j)
    std::vector<double2> mu(K), il2(K);
    AAO_TRY_CUDA(cudaMemcpyAsync(mu.data(), h.mu, sizeof(double2) * K, cudaMemcpyDeviceToHost, h.stream));
    AAO_TRY_CUDA(cudaMemcpyAsync(il2.data(), h.il2, sizeof(double2) * K, cudaMemcpyDeviceToHost, h.stream));
    AAO_TRY_CUDA(cudaStreamSynchronize(h.stream));
    std::vector<float2> dk((size_t)K * ldq, make_float2(0.f, 0.f));
    host_parallel(K, [&](int k0, int k1) {
      for (int k = k0; k < k1; ++k) {
        const std::complex<double> m(mu[k].x, mu[k].y), s(il2[k].x, il2[k].y);
        for (int j = 0; j < nx; ++j) {
          const std::complex<double> v = s / (m - lam[j]);
          dk[(size_t)k * ldq + j] = make_float2((float)v.real(), (float)v.imag());
        }
      }
    });
    // TF32 head and tail of Q and Q^T for the tensor-core products (x = hi + lo)
    auto tf32 = [](float x) {
      uint32_t u;
      memcpy(&u, &x, 4);
      if ((u & 0x7f800000u) != 0x7f800000u) {
        u += 0x0fffu + ((u >> 13) & 1u);  // round to nearest even at 10 mantissa bits
        u &= 0xffffe000u;
      }
      float r;
      memcpy(&r, &u, 4);
      return r;
    };
    // stored tiled for the TMA boxes: entry (row r, contraction index k) at float
    // ((r/8 (ldq/4) + k/4) 8 + r%8) 4 + k%4, i.e. 8 x 16-byte core matrices, K groups of a row
    // group contiguous; row groups of 8 are split over the host threads
    const size_t qn = (size_t)ldq * ldq;
    std::vector<float> qh(qn), ql(qn), qth(qn), qtl(qn);
    host_parallel(ldq / 8, [&](int g0, int g1) {
      for (int r = 8 * g0; r < 8 * g1; ++r)
        for (int k = 0; k < ldq; ++k) {
          const size_t t = ((((size_t)(r >> 3) * (ldq / 4) + (k >> 2)) * 8 + (r & 7)) * 4) + (k & 3);
          const bool in = r < nx && k < nx;
          const float a = in ? (float)Ad[(size_t)k * nx + r] : 0.f, b = in ? (float)Ad[(size_t)r * nx + k] : 0.f;
          qh[t] = tf32(a);
          ql[t] = tf32(a - qh[t]);
          qth[t] = tf32(b);
          qtl[t] = tf32(b - qth[t]);
        }
    });
    AAO_TRY(up(&h.rz_qh, qh));
    AAO_TRY(up(&h.rz_ql, ql));
    AAO_TRY(up(&h.rz_qth, qth));
    AAO_TRY(up(&h.rz_qtl, qtl));
    // the complex operand of the products (TF32 head and tail, tiled, 2 Kpad rows)
    const int Kpad = ((K + tcg::kBins - 1) / tcg::kBins) * tcg::kBins;
    const size_t nb = (size_t)2 * Kpad * ldq;
    AAO_TRY_CUDA(cudaMalloc(&h.rz_bh, sizeof(float) * nb));
    AAO_TRY_CUDA(cudaMalloc(&h.rz_bl, sizeof(float) * nb));
    AAO_TRY_CUDA(cudaMemsetAsync(h.rz_bh, 0, sizeof(float) * nb, h.stream));
    AAO_TRY_CUDA(cudaMemsetAsync(h.rz_bl, 0, sizeof(float) * nb, h.stream));
    AAO_TRY(encode_tiled_map(h.rz_tmap + 0 * 128, h.rz_qth, ldq, ldq, tcg::kM));
    AAO_TRY(encode_tiled_map(h.rz_tmap + 1 * 128, h.rz_qtl, ldq, ldq, tcg::kM));
    AAO_TRY(encode_tiled_map(h.rz_tmap + 2 * 128, h.rz_qh, ldq, ldq, tcg::kM));
    AAO_TRY(encode_tiled_map(h.rz_tmap + 3 * 128, h.rz_ql, ldq, ldq, tcg::kM));
    AAO_TRY(encode_tiled_map(h.rz_tmap + 4 * 128, h.rz_bh, ldq, 2 * Kpad, tcg::kN));
    AAO_TRY(encode_tiled_map(h.rz_tmap + 5 * 128, h.rz_bl, ldq, 2 * Kpad, tcg::kN));
    AAO_TRY_CUDA(cudaMalloc(&h.rz_err, sizeof(int)));
    AAO_TRY_CUDA(cudaMemsetAsync(h.rz_err, 0, sizeof(int), h.stream));
    const uint32_t tc_smem = tcg::smem_bytes(tcg::kStages);
    AAO_TRY_CUDA(cudaFuncSetAttribute(k_rz_tc<tcg::kStages>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem));
    // contraction segments: the fewest (a power of two dividing the ldq / 32 chunks, at most
    // kSegMax) whose grid fills 90% of the resident CTA slots
    int per_sm = 0, sms = h.sms;
    AAO_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rz_tc<tcg::kStages>, 160, tc_smem));
    if (sms <= 0) {
      int dev = 0;
      AAO_TRY_CUDA(cudaGetDevice(&dev));
      AAO_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const long slots = (long)(per_sm > 0 ? per_sm : 1) * sms, ctas = (long)(ldq / tcg::kM) * (Kpad / tcg::kBins);
    int nseg = 1;
    while (2 * nseg <= tcg::kSegMax && (ldq / tcg::kKC) % (2 * nseg) == 0 && 10 * ctas * nseg < 9 * slots) nseg *= 2;
    h.rz_nseg = nseg;
    h.rz_kpad = Kpad;
    AAO_TRY(up(&h.rz_dk, dk));
    AAO_TRY_CUDA(cudaMalloc(&h.rz_part, sizeof(float2) * (size_t)nseg * K * ldq));
    h.rz_ldq = ldq;
    // the padding columns of the spectrum stay zero: every kernel writes columns < nx only, or zeros
    AAO_TRY_CUDA(cudaMemsetAsync(h.spec, 0, sizeof(float2) * (size_t)K * h.pitch, h.stream));
    AAO_TRY_CUDA(cudaStreamSynchronize(h.stream));
    h.rz_sym = true;
    cudaFree(d_tcol);
    cudaFree(d_trow);
    return AAO_OK;
  }
  // the shifted matrices, inverted in place by blocked Gauss-Jordan (FP32 complex; the rank-kGW
  // updates on the tensor cores): an apply is then one matrix-vector product per bin
  AAO_TRY_CUDA(cudaMalloc(&h.rz_inv, sizeof(float2) * nn * K));
  k_rz_form<<<dim3(256, K), 256, 0, h.stream>>>(h.rz_inv, nx, d_tcol, d_trow, h.muf);
  AAO_CHECK_LAUNCH();
  {
    AAO_TRY(gj_invert_batched(h.stream, h.rz_inv, nx, K));
    AAO_TRY_CUDA(cudaMalloc(&h.rz_w, sizeof(float2) * (size_t)K * h.pitch));
    AAO_TRY_CUDA(cudaMemsetAsync(h.rz_w, 0, sizeof(float2) * (size_t)K * h.pitch, h.stream));
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

int riesz_solve_bins(Handle& h, void* spec, void** result) {
  *result = spec;
  if (h.rz_sym) {
    // W = (Z1 Q) o D, then Z2 = W Q^T (rows: bins; the half spectrum is [k][x]) on the tensor
    // cores: k_rz_split tiles and splits the complex operand (for the second product it also adds
    // the first one's contraction segments in order and multiplies by D), k_rz_tc forms the
    // segments' partial products, k_rz_cgemm_sum adds the second product's
    const int ldq = h.rz_ldq, Kpad = h.rz_kpad, nseg = h.rz_nseg;
    const double nq = (double)ldq * ldq;
    ProfScope ps(AAO_K_TRIDIAG, h.stream, 2.0 * (nq * 8.0 + 2.0 * (double)h.K * ldq * 8.0));
    const dim3 g(ldq / tcg::kM, Kpad / tcg::kBins, nseg);
    const uint32_t smem = tcg::smem_bytes(tcg::kStages);
    const int bgrid = (int)(((size_t)Kpad * (ldq / 4) + 255) / 256);
    const int sgrid = (int)((((size_t)h.K * ldq / 2) + 255) / 256);
    CUtensorMap m[6];
    memcpy(m, h.rz_tmap, sizeof m);
    AAO_TRY_CUDA(launch_pdl(k_rz_split, bgrid, 256, 0, h.stream, (const float2*)spec, h.pitch, (size_t)0, 1, h.K,
                            h.pitch, (const float2*)nullptr, 0, h.rz_bh, h.rz_bl, ldq, Kpad));
    AAO_TRY_CUDA(launch_pdl(k_rz_tc<tcg::kStages>, g, 160, smem, h.stream, m[0], m[1], m[4], m[5], h.rz_part, ldq, h.K,
                            ldq / nseg, h.rz_err, h.rz_wait_ns, h.rz_inject));
    AAO_TRY_CUDA(launch_pdl(k_rz_split, bgrid, 256, 0, h.stream, (const float2*)h.rz_part, ldq, (size_t)h.K * ldq, nseg,
                            h.K, ldq, (const float2*)h.rz_dk, ldq, h.rz_bh, h.rz_bl, ldq, Kpad));
    AAO_TRY_CUDA(launch_pdl(k_rz_tc<tcg::kStages>, g, 160, smem, h.stream, m[2], m[3], m[4], m[5], h.rz_part, ldq, h.K,
                            ldq / nseg, h.rz_err, h.rz_wait_ns, h.rz_inject));
    AAO_TRY_CUDA(launch_pdl(k_rz_cgemm_sum, sgrid, 256, 0, h.stream, (const float2*)h.rz_part, ldq, h.K, h.pitch, nseg,
                            (float2*)spec, h.pitch, (const float2*)nullptr, ldq));
    AAO_CHECK_LAUNCH();
    return AAO_OK;
  }
  // with drift: z2_k = X_k (z1_k / lambda_2,k) into the workspace
  const size_t smem = sizeof(float2) * (size_t)h.nx;
  const double bytes = (double)h.K * ((double)h.nx * h.nx * 8.0 + 2.0 * h.nx * 8.0);
  ProfScope ps(AAO_K_TRIDIAG, h.stream, bytes);
  AAO_TRY_CUDA(launch_pdl(k_rz_gemv, dim3((h.nx + kRzGemvRows - 1) / kRzGemvRows, h.K), 32 * kRzGemvRows, smem, h.stream,
                          (const float2*)spec, h.rz_w, h.nx, h.pitch, (const float2*)h.rz_inv, (const float2*)h.il2f));
  AAO_CHECK_LAUNCH();
  *result = h.rz_w;
  return AAO_OK;
}

}  // namespace aao

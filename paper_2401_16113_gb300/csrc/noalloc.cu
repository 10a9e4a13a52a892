// precond_apply_static: the P_alpha^{-1} apply for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the preconditioner: host
// code under a fixed device-memory budget (a pool handed out up front, or a process that must
// never grow its footprint after start-up), and real-time paths where an allocation's implicit
// synchronisation or its failure mode is not acceptable. aao_create allocates the handle's
// tables and the half-spectrum workspace, so it is not usable there.
//
// This entry point needs nothing but the caller's input and output vectors. Its scratch
// (the FFT twiddles, Lambda_alpha tables, shifted eigenvalues, the tau*Abar diagonals and the
// half spectrum) lives in one file-scope device array of kStaticBytes (32 MiB), reserved on
// every GPU that loads this library until the process exits. Every call rewrites the tables
// and the spectrum it reads, so nothing has to start at zero and no state carries over from
// a previous call's contents. Because all calls on a device share the one array, calls whose
// work overlaps on the GPU (different streams, or different host threads, without ordering
// between them) race on it: order them, for example by using one stream.
//
// The device address of the array is looked up with cudaGetSymbolAddress the first time the
// entry point runs on a device (with that device current) and cached for the life of the
// process: a cudaDeviceReset between calls would leave the cached address stale, so the library
// supports no reset while it is in use. Make that first call before starting any stream capture
// that will contain later calls.
#include <math.h>

#include <atomic>
#include <mutex>

#include "aao_internal.cuh"

namespace aao {
namespace {

constexpr size_t kStaticBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

// device address of g_static_scratch on the current device (looked up once per device)
int scratch_address(void** out) {
  int dev = 0;
  AAO_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("precond_apply_static: device ordinal out of range");
    return AAO_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    AAO_TRY_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return AAO_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

struct Layout {
  size_t tw, lam, ilam, mu, il2, pl, pd, pu, spec, total;
};

Layout layout(int nx, int nt, int pitch, size_t rs) {
  const size_t cs = 2 * rs;  // complex
  const int K = nt / 2 + 1;
  Layout L{};
  size_t o = 0;
  L.tw = o;   o = align256(o + cs * nt);
  L.lam = o;  o = align256(o + rs * nt);
  L.ilam = o; o = align256(o + rs * nt);
  L.mu = o;   o = align256(o + cs * K);
  L.il2 = o;  o = align256(o + cs * K);
  L.pl = o;   o = align256(o + rs * nx);
  L.pd = o;   o = align256(o + rs * nx);
  L.pu = o;   o = align256(o + rs * nx);
  L.spec = o; o = align256(o + cs * (size_t)K * pitch);
  L.total = o;
  return L;
}

// Tables of the apply, written into the static scratch (same definitions as aao_create:
// lambda1_k = 1 - a w^k, lambda2_k = (1 + a w^k)/2, a = alpha^{1/nt}, w = exp(-2 pi i/nt);
// tau*Abar from the time mean of sigma^2, here in closed form over the midpoints t_{k+1/2}).
template <typename R>
__global__ void k_static_tables(unsigned char* base, Layout L, int nx, int nt, double T, double r, double K,
                                double sigma, double s_max, double bump, double tslope, double alpha) {
  using C = C_t<R>;
  C* tw = reinterpret_cast<C*>(base + L.tw);
  R* lam = reinterpret_cast<R*>(base + L.lam);
  R* ilam = reinterpret_cast<R*>(base + L.ilam);
  C* mu = reinterpret_cast<C*>(base + L.mu);
  C* il2 = reinterpret_cast<C*>(base + L.il2);
  R* pl = reinterpret_cast<R*>(base + L.pl);
  R* pd = reinterpret_cast<R*>(base + L.pd);
  R* pu = reinterpret_cast<R*>(base + L.pu);
  const int Kb = nt / 2 + 1;
  const double tau = T / nt;
  const double a = pow(alpha, 1.0 / nt);
  const double cm = 1.0 + tslope * T * 0.5;
  const double c2m = 1.0 + tslope * T + tslope * tslope * tau * tau * (4.0 * (double)nt * nt - 1.0) / 12.0;
  const double hS = s_max / (nx + 1);
  const int total = nt + Kb + nx;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    if (e < nt) {
      double s, c;
      sincospi(-2.0 * (double)e / nt, &s, &c);
      tw[e] = cmk<C>((R)c, (R)s);
      const double l = pow(alpha, (double)e / nt);
      lam[e] = (R)l;
      ilam[e] = (R)(1.0 / (l * nt));
    } else if (e < nt + Kb) {
      const int k = e - nt;
      double s, c;
      sincospi(-2.0 * (double)k / nt, &s, &c);
      const double l1r = 1.0 - a * c, l1i = -a * s;
      const double l2r = 0.5 * (1.0 + a * c), l2i = 0.5 * a * s;
      const double d = l2r * l2r + l2i * l2i;
      mu[k] = cmk<C>((R)((l1r * l2r + l1i * l2i) / d), (R)((l1i * l2r - l1r * l2i) / d));
      il2[k] = cmk<C>((R)(l2r / d), (R)(-l2i / d));
    } else {
      const int i = e - nt - Kb;
      const double S = hS * (i + 1);
      const double lg = log(S / K);
      const double bi = bump * exp(-lg * lg);
      const double s2 = sigma * sigma + 2.0 * sigma * bi * cm + bi * bi * c2m;
      const double ii = (double)(i + 1);
      const double diff = 0.5 * s2 * ii * ii, conv = 0.5 * r * ii;
      pl[i] = (R)(tau * (diff - conv));
      pd[i] = (R)(tau * (-2.0 * diff - r));
      pu[i] = (R)(tau * (diff + conv));
    }
  }
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace
}  // namespace aao

using namespace aao;

extern "C" int precond_apply_static(const aao_problem* p, const double* v, double* z) {
  if (!p || !v || !z) {
    set_error("precond_apply_static: null argument");
    return AAO_EINVAL;
  }
  if (p->op != AAO_OP_BS && p->op != AAO_OP_LOCALVOL) {
    set_error("precond_apply_static: op must be AAO_OP_BS or AAO_OP_LOCALVOL");
    return AAO_EUNSUPPORTED;
  }
  if (p->precision != AAO_FP64 && p->precision != AAO_MIXED) {
    set_error("precond_apply_static: unknown precision");
    return AAO_EINVAL;
  }
  const bool mixed = p->precision == AAO_MIXED;
  MrPlan plan;
  const bool nt_ok = p->nt >= 1 && (is_pow2(p->nt) || mr_plan(p->nt, plan));
  if (p->nx < 2 || !nt_ok || p->nt > (mixed ? 8192 : 4096) || p->nx > (mixed ? 8192 : 4096)) {
    set_error("precond_apply_static: need nx >= 2 (<= 8192 mixed, <= 4096 FP64) and nt with no prime factor "
              "above 7 (<= 8192 mixed, <= 4096 FP64)");
    return AAO_EINVAL;
  }
  if (!(p->T > 0) || !(p->K > 0) || !(p->sigma > 0) || !(p->s_max > 0) || !(p->r >= 0) || !(p->alpha > 0) ||
      !(p->alpha <= 1)) {
    set_error("precond_apply_static: need T, K, sigma, s_max > 0, r >= 0 and 0 < alpha <= 1");
    return AAO_EINVAL;
  }
  const int pitch = ((p->nx + 63) / 64) * 64;
  const size_t rs = mixed ? sizeof(float) : sizeof(double);
  const Layout L = layout(p->nx, p->nt, pitch, rs);
  if (L.total > kStaticBytes) {
    set_error("precond_apply_static: problem needs more than the 32 MiB static scratch "
              "(roughly (nt/2+1) * ceil(nx/64)*64 complex values plus tables); use precond_apply");
    return AAO_EINVAL;
  }
  void* base = nullptr;
  AAO_TRY(scratch_address(&base));
  unsigned char* b = static_cast<unsigned char*>(base);

  // a handle view onto the static scratch: no allocation
  Handle h;
  h.p = *p;
  h.stream = (cudaStream_t)p->stream;
  h.nx = p->nx;
  h.nt = p->nt;
  h.K = p->nt / 2 + 1;
  int l = 0;
  while ((1 << l) < p->nt) ++l;
  h.log2n = l;
  if (!is_pow2(p->nt)) h.mr = plan;  // the mixed-radix FFT kernels
  h.pitch = pitch;
  h.n = (size_t)p->nx * p->nt;
  h.mixed = mixed;
  h.spec = b + L.spec;
  const double bump = p->op == AAO_OP_LOCALVOL ? p->lv_bump : 0.0;
  const double tslope = p->op == AAO_OP_LOCALVOL ? p->lv_tslope : 0.0;
  const int total = p->nt + h.K + p->nx;
  const int grid = (total + 255) / 256;
  if (mixed) {
    k_static_tables<float><<<grid, 256, 0, h.stream>>>(b, L, p->nx, p->nt, p->T, p->r, p->K, p->sigma, p->s_max,
                                                       bump, tslope, p->alpha);
    h.twf = reinterpret_cast<float2*>(b + L.tw);
    h.lamf = reinterpret_cast<float*>(b + L.lam);
    h.ilamf = reinterpret_cast<float*>(b + L.ilam);
    h.muf = reinterpret_cast<float2*>(b + L.mu);
    h.il2f = reinterpret_cast<float2*>(b + L.il2);
    h.pLf = reinterpret_cast<float*>(b + L.pl);
    h.pDf = reinterpret_cast<float*>(b + L.pd);
    h.pUf = reinterpret_cast<float*>(b + L.pu);
  } else {
    k_static_tables<double><<<grid, 256, 0, h.stream>>>(b, L, p->nx, p->nt, p->T, p->r, p->K, p->sigma, p->s_max,
                                                        bump, tslope, p->alpha);
    h.tw = reinterpret_cast<double2*>(b + L.tw);
    h.lam = reinterpret_cast<double*>(b + L.lam);
    h.ilam = reinterpret_cast<double*>(b + L.ilam);
    h.mu = reinterpret_cast<double2*>(b + L.mu);
    h.il2 = reinterpret_cast<double2*>(b + L.il2);
    h.pL = reinterpret_cast<double*>(b + L.pl);
    h.pD = reinterpret_cast<double*>(b + L.pd);
    h.pU = reinterpret_cast<double*>(b + L.pu);
  }
  AAO_CHECK_LAUNCH();
  // the three kernels of the apply, reading the tables and the spectrum from the static scratch
  return launch_precond(h, v, z, false);
}

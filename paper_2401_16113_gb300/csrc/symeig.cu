// Dense symmetric eigendecomposition on the host, FP64: the setup of the spectral step (b) for a
// symmetric spatial operator (Riesz without drift), where (mu_k I - tau Abar)^{-1} =
// Q diag(1 / (mu_k - lambda_j)) Q^T for every frequency k once tau Abar = Q diag(lambda) Q^T.
//
// Two classical stages (Golub and Van Loan, Matrix Computations, Sec. 8.3):
//  1. Householder tridiagonalisation (their Algorithm 8.3.1): T = Q1^T A Q1 with Q1 = H_0 ... H_{n-3},
//     H_k = I - beta_k v_k v_k^T zeroing column k below the subdiagonal, the trailing block updated
//     by the symmetric rank-2 form B - v w^T - w v^T;
//  2. the symmetric QR algorithm (their Algorithms 8.3.2 and 8.3.3): off-diagonal entries below
//     eps (|a_i| + |a_{i+1}|) are set to zero, and the last unreduced block is reduced by implicit
//     QR steps with the Wilkinson shift (the eigenvalue of its trailing 2 x 2 block nearer to the
//     last diagonal entry), each step a chase of the bulge down the block by plane rotations.
// The QR iteration touches only the tridiagonal (O(n) per step), so it runs first and records its
// rotations; the eigenvector matrix Q = Q1 G_1 G_2 ... is then formed by applying the reflectors and
// the recorded rotations to blocks of rows in parallel, each block streaming through the whole list
// once (rows of Q are independent under both kinds of update). For n = 1023 the 6 n^3 flops of the
// rotations dominate; they run on all host cores.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <functional>
#include <thread>
#include <vector>

#include "aao_internal.cuh"

namespace aao {
namespace {

// A pool of host threads kept spinning for the duration of one decomposition, so that the ~2n
// parallel regions of the Householder stage cost a wake-up of a few microseconds each. run(n, f)
// calls f(begin, end) over [0, n) in contiguous chunks, the caller taking the first; run_beside
// leaves the caller free for other work meanwhile.
class SpinPool {
 public:
  explicit SpinPool(int threads) : nthr_(std::max(1, threads)) {
    for (int t = 1; t < nthr_; ++t) th_.emplace_back([this, t] { worker(t); });
  }
  ~SpinPool() {
    stop_.store(true, std::memory_order_release);
    for (auto& t : th_) t.join();
  }
  int threads() const { return nthr_; }
  void run(int n, const std::function<void(int, int)>& f) {
    if (nthr_ == 1 || n < 2 * nthr_) {
      f(0, n);
      return;
    }
    start(n, f, false);
    chunk(0);
    wait();
  }
  // f over [0, n) on the pool's other threads while the caller runs g
  void run_beside(int n, const std::function<void(int, int)>& f, const std::function<void()>& g) {
    if (nthr_ == 1) {
      g();
      f(0, n);
      return;
    }
    start(n, f, true);
    g();
    wait();
  }

 private:
  void start(int n, const std::function<void(int, int)>& f, bool beside) {
    job_ = &f;
    n_ = n;
    beside_ = beside;
    done_.store(0, std::memory_order_relaxed);
    gen_.fetch_add(1, std::memory_order_acq_rel);
  }
  void wait() {
    while (done_.load(std::memory_order_acquire) < nthr_ - 1) std::this_thread::yield();
  }
  void chunk(int t) {
    const int parts = beside_ ? nthr_ - 1 : nthr_, idx = beside_ ? t - 1 : t;
    const int per = (n_ + parts - 1) / parts;
    const int b = idx * per, e = std::min(n_, b + per);
    if (b < e) (*job_)(b, e);
  }
  void worker(int t) {
    int seen = 0;
    for (;;) {
      int g;
      while ((g = gen_.load(std::memory_order_acquire)) == seen) {
        if (stop_.load(std::memory_order_acquire)) return;
        std::this_thread::yield();
      }
      seen = g;
      chunk(t);
      done_.fetch_add(1, std::memory_order_acq_rel);
    }
  }
  int nthr_;
  std::vector<std::thread> th_;
  std::atomic<int> gen_{0}, done_{0};
  std::atomic<bool> stop_{false};
  const std::function<void(int, int)>* job_ = nullptr;
  int n_ = 0;
  bool beside_ = false;
};

int host_threads(size_t work) {
  if (work < (size_t)1 << 16) return 1;  // not worth the threads
  const unsigned hw = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(hw == 0 ? 1u : hw, 32u));
}

struct Rotation {
  int k;        // plane (k, k+1)
  double c, s;  // columns k, k+1 of Q become c q_k + s q_{k+1} and -s q_k + c q_{k+1}
};

// Householder vector of x (length m): v = x - sub e_0 with sub = -sign(x_0) ||x|| (no cancellation
// in v_0), beta = 2 / ||v||^2; beta = 0 and sub = x_0 when x = 0.
void householder(const double* x, int m, std::vector<double>& v, double& sub, double& bk) {
  v.assign(x, x + m);
  double s2 = 0.0;
  for (int i = 0; i < m; ++i) s2 += v[i] * v[i];
  sub = v[0];
  bk = 0.0;
  if (s2 > 0.0) {
    const double nrm = sqrt(s2);
    sub = v[0] >= 0.0 ? -nrm : nrm;
    v[0] -= sub;
    const double vv = s2 - 2.0 * sub * (v[0] + sub) + sub * sub;  // ||x - sub e_0||^2
    bk = vv > 0.0 ? 2.0 / vv : 0.0;
  }
}

// Householder stage on A (n x n row-major, overwritten). Returns the diagonal a, the off-diagonal
// b (b[i] couples i and i+1), the reflectors (v_k of length n-k-1) and their beta_k.
// Step k on the trailing block B (rows and columns k+1..): p = beta B v, w = p - (beta/2)(v^T p) v,
// B <- B - v w^T - w v^T. The next step's reflector depends only on column k+1 of the updated B,
// which costs O(m) to form, so it is built first and one pass over B per step both applies the
// update and accumulates the next step's B v (over the same entries in the same order as a separate
// pass would).
void tridiagonalise(SpinPool& pool, int n, double* A, std::vector<double>& a, std::vector<double>& b,
                    std::vector<std::vector<double>>& refl, std::vector<double>& beta) {
  const size_t N = (size_t)n;
  a.assign(N, 0.0);
  b.assign(N > 0 ? N - 1 : 0, 0.0);
  std::vector<double> p(N), w(N), col(N);
  std::vector<double> v, vn;
  double sub = 0.0, bk = 0.0;
  if (n >= 3) {
    const int m = n - 1;
    for (int i = 0; i < m; ++i) col[i] = A[(size_t)(1 + i) * N];
    householder(col.data(), m, v, sub, bk);
    if (bk != 0.0)
      pool.run(m, [&](int r0, int r1) {
        for (int i = r0; i < r1; ++i) {
          const double* Bi = A + (size_t)(1 + i) * N + 1;
          double acc = 0.0;
          for (int j = 0; j < m; ++j) acc += Bi[j] * v[j];
          p[i] = bk * acc;
        }
      });
  }
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    const size_t o = (size_t)k + 1;
    if (bk != 0.0) {
      double vp = 0.0;
      for (int i = 0; i < m; ++i) vp += v[i] * p[i];
      const double h = 0.5 * bk * vp;
      for (int i = 0; i < m; ++i) w[i] = p[i] - h * v[i];
    }
    a[k] = A[(size_t)k * N + k];
    b[k] = sub;
    // the next step's reflector, from column k+1 below the diagonal after this step's update
    const bool next = k + 3 < n;
    double subn = 0.0, bkn = 0.0;
    if (next) {
      for (int i = 1; i < m; ++i) {
        const double bi = A[(o + i) * N + o];
        col[i - 1] = bk != 0.0 ? bi - (v[i] * w[0] + w[i] * v[0]) : bi;
      }
      householder(col.data(), m - 1, vn, subn, bkn);
    }
    const bool upd = bk != 0.0, mv = next && bkn != 0.0;
    if (upd || mv)
      pool.run(m, [&](int r0, int r1) {
        for (int i = r0; i < r1; ++i) {
          double* Bi = A + (o + i) * N + o;
          if (upd) {
            const double vi = v[i], wi = w[i];
            for (int j = 0; j < m; ++j) Bi[j] -= vi * w[j] + wi * v[j];
          }
          if (mv && i >= 1) {
            double acc = 0.0;
            for (int j = 1; j < m; ++j) acc += Bi[j] * vn[j - 1];
            p[i - 1] = bkn * acc;
          }
        }
      });
    refl.push_back(std::move(v));
    beta.push_back(bk);
    v = std::move(vn);
    vn.clear();
    sub = subn;
    bk = bkn;
  }
  if (n >= 2) {
    a[n - 2] = A[(N - 2) * N + (N - 2)];
    b[n - 2] = A[(N - 1) * N + (N - 2)];
  }
  a[n - 1] = A[(N - 1) * N + (N - 1)];
}

// Symmetric QR algorithm on (a, b); the rotations are appended to rot in the order applied.
// False if some block needs more than 64 QR steps per eigenvalue found.
bool symmetric_qr(int n, std::vector<double>& a, std::vector<double>& b, std::vector<Rotation>& rot) {
  const double eps = 2.220446049250313e-16;
  int m = n - 1;  // rows m+1.. are finished (diagonal)
  int steps = 0;
  while (m > 0) {
    // deflation: negligible couplings become zero
    for (int i = 0; i < m; ++i)
      if (fabs(b[i]) <= eps * (fabs(a[i]) + fabs(a[i + 1]))) b[i] = 0.0;
    while (m > 0 && b[m - 1] == 0.0) --m;  // a[m] is an eigenvalue
    if (m == 0) break;
    int l = m - 1;
    while (l > 0 && b[l - 1] != 0.0) --l;  // [l, m] is the last unreduced block
    if (++steps > 64 * n) return false;
    // Wilkinson shift: the eigenvalue of [[a_{m-1}, b_{m-1}], [b_{m-1}, a_m]] nearer to a_m
    const double dlt = 0.5 * (a[m - 1] - a[m]);
    const double bb = b[m - 1];
    const double den = dlt + (dlt >= 0.0 ? 1.0 : -1.0) * hypot(dlt, bb);
    const double mu = a[m] - (den != 0.0 ? bb * bb / den : 0.0);
    // implicit QR step: the first rotation is fixed by the first column of T - mu I, the later
    // ones chase the bulge (an entry at (k+1, k-1)) down to the end of the block
    double x = a[l] - mu, z = b[l];
    for (int k = l; k < m; ++k) {
      const double r = hypot(x, z);
      double c = 1.0, s = 0.0;
      if (r > 0.0) {
        c = x / r;
        s = z / r;
      }
      if (k > l) b[k - 1] = r;  // the bulge is absorbed
      // similarity by [[c, s], [-s, c]] on rows and columns (k, k+1)
      const double ak = a[k], ak1 = a[k + 1], bk = b[k];
      const double cs = c * s;
      a[k] = c * c * ak + 2.0 * cs * bk + s * s * ak1;
      a[k + 1] = s * s * ak - 2.0 * cs * bk + c * c * ak1;
      b[k] = cs * (ak1 - ak) + (c * c - s * s) * bk;
      if (k + 1 < m) {
        z = s * b[k + 1];  // the new bulge at (k+2, k)
        b[k + 1] *= c;
        x = b[k];
      }
      rot.push_back({k, c, s});
    }
  }
  return true;
}

}  // namespace

bool sym_eig(int n, double* A, double* w) {
  if (n <= 0) return true;
  const size_t N = (size_t)n;
  SpinPool pool(host_threads(N * N));
  std::vector<double> a, b, beta;
  std::vector<std::vector<double>> refl;
  tridiagonalise(pool, n, A, a, b, refl, beta);
  // Q = Q1 G_1 G_2 ..., formed by blocks of kRows rows: row r of Q1 = e_r^T H_0 ... H_{n-3} (the
  // reflectors in order; H_k changes entries k+1.. only), then the rotations in order. A block is
  // held transposed (entry j of the block's row r at j kRows + r), so that each update touches kRows
  // contiguous values. The reflector stage needs no rotation, so it runs on the pool's other threads
  // while this thread runs the QR iteration.
  constexpr int kRows = 16;
  const int blocks = (n + kRows - 1) / kRows;
  std::vector<double> qall((size_t)blocks * N * kRows);
  std::vector<Rotation> rot;
  rot.reserve(4 * N * N / 2 + 16);
  bool converged = true;
  pool.run_beside(blocks, [&](int b0, int b1) {
    for (int blk = b0; blk < b1; ++blk) {
      double* qb = qall.data() + (size_t)blk * N * kRows;
      const int r0 = blk * kRows, nr = std::min(n, r0 + kRows) - r0;
      for (int r = 0; r < nr; ++r) qb[(size_t)(r0 + r) * kRows + r] = 1.0;
      for (size_t k = 0; k < refl.size(); ++k) {
        if (beta[k] == 0.0) continue;
        const double* v = refl[k].data();
        const int m = (int)refl[k].size();
        double* q = qb + (k + 1) * kRows;
        double dot[kRows] = {};
        for (int j = 0; j < m; ++j)
          for (int r = 0; r < kRows; ++r) dot[r] += q[(size_t)j * kRows + r] * v[j];
        for (int r = 0; r < kRows; ++r) dot[r] *= beta[k];
        for (int j = 0; j < m; ++j)
          for (int r = 0; r < kRows; ++r) q[(size_t)j * kRows + r] -= dot[r] * v[j];
      }
    }
  }, [&]() { converged = symmetric_qr(n, a, b, rot); });
  if (!converged) return false;

  // The rotations of one QR step act on neighbouring planes (k, k+1), (k+1, k+2), ...: the column
  // that a rotation leaves in plane k+1 is the one the next rotation takes in, so it is carried in
  // registers along such a chain (and written back when the chain breaks) instead of being stored
  // and loaded again between the two.
  std::vector<double> Q(N * N);
  pool.run(blocks, [&](int b0, int b1) {
    for (int blk = b0; blk < b1; ++blk) {
      double* qb = qall.data() + (size_t)blk * N * kRows;
      const int r0 = blk * kRows, nr = std::min(n, r0 + kRows) - r0;
      double xv[kRows];
      int cur = -1;  // the column held in xv
      for (const Rotation& g : rot) {
        if (g.k != cur) {
          if (cur >= 0)
            for (int r = 0; r < kRows; ++r) qb[(size_t)cur * kRows + r] = xv[r];
          for (int r = 0; r < kRows; ++r) xv[r] = qb[(size_t)g.k * kRows + r];
        }
        double* x = qb + (size_t)g.k * kRows;
        const double* y = x + kRows;
        for (int r = 0; r < kRows; ++r) {
          const double xr = xv[r], yr = y[r];
          x[r] = g.c * xr + g.s * yr;
          xv[r] = g.c * yr - g.s * xr;
        }
        cur = g.k + 1;
      }
      if (cur >= 0)
        for (int r = 0; r < kRows; ++r) qb[(size_t)cur * kRows + r] = xv[r];
      for (int r = 0; r < nr; ++r)
        for (size_t j = 0; j < N; ++j) Q[(size_t)(r0 + r) * N + j] = qb[j * kRows + r];
    }
  });
  // A <- Q^T (row j = the eigenvector of a[j])
  for (size_t r = 0; r < N; ++r)
    for (size_t j = 0; j < N; ++j) A[j * N + r] = Q[r * N + j];
  for (int j = 0; j < n; ++j) w[j] = a[j];
  return true;
}

}  // namespace aao

// Host float64 construction of the least-misfit gridding function, its look-up table
// and the grid-correction factors (Section 2.1; Appendices A, B, E, F).
//
// Design variables: h(x) on the Ng+1 = 33 nodes x_k = k x0/Ng (h(0) = 1), mirrored to
// 2Ng+1 nodes on [-x0, x0] with trapezoid weights. For a given h the gridding weights
// C_r(s) minimise the integrated misfit separately for every table coordinate s: the
// normal equations A C = B(s) (Eqs. 17-19, Cholesky) for W <= 11 and Householder-QR least
// squares for W > 11 (Appendices B and E). The outer problem minimises
// E = (1/2x0) int l(x) dx (Eq. 16, l from Eq. 11 with the s-integral on Mg = 16 points)
// over h(x_1..x_Ng) with a Levenberg-Marquardt iteration (Appendix A).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <thread>

#include "lmg_internal.h"

namespace lmg {
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

// Quadrature of Appendix A. s-nodes: midpoints of Mg equal cells of (0, 1/2).
struct Nodes {
  int K;                      // 2Ng+1
  std::vector<double> x, w;   // nodes on [-x0, x0], trapezoid weights
  std::vector<double> s;      // Mg design values of s
};

Nodes make_nodes(double x0p) {
  Nodes n;
  n.K = 2 * kNg + 1;
  n.x.resize(n.K);
  n.w.resize(n.K);
  for (int i = 0; i < n.K; ++i) {
    n.x[i] = x0p * double(i - kNg) / kNg;
    n.w[i] = x0p / kNg;
  }
  n.w[0] *= 0.5;
  n.w[n.K - 1] *= 0.5;
  n.s.resize(kMg);
  for (int j = 0; j < kMg; ++j) n.s[j] = (j + 0.5) / (2.0 * kMg);
  return n;
}

// In-place Cholesky of a symmetric positive definite W x W matrix (lower factor).
bool cholesky(std::vector<double>& a, int W) {
  for (int j = 0; j < W; ++j) {
    double d = a[j * W + j];
    for (int k = 0; k < j; ++k) d -= a[j * W + k] * a[j * W + k];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    a[j * W + j] = d;
    for (int i = j + 1; i < W; ++i) {
      double v = a[i * W + j];
      for (int k = 0; k < j; ++k) v -= a[i * W + k] * a[j * W + k];
      a[i * W + j] = v / d;
    }
  }
  return true;
}

void cholesky_solve(const std::vector<double>& L, int W, double* b) {
  for (int i = 0; i < W; ++i) {
    double v = b[i];
    for (int k = 0; k < i; ++k) v -= L[i * W + k] * b[k];
    b[i] = v / L[i * W + i];
  }
  for (int i = W - 1; i >= 0; --i) {
    double v = b[i];
    for (int k = i + 1; k < W; ++k) v -= L[k * W + i] * b[k];
    b[i] = v / L[i * W + i];
  }
}

// Least squares min ||M c - rhs|| for a dense m x W matrix (column-major work copy) by
// Householder QR; c receives W values.
bool householder_lstsq(std::vector<double>& M, int m, int W, std::vector<double>& rhs, double* c) {
  for (int k = 0; k < W; ++k) {
    double* col = &M[size_t(k) * m];
    double norm = 0.0;
    for (int i = k; i < m; ++i) norm += col[i] * col[i];
    norm = std::sqrt(norm);
    if (norm == 0.0) return false;
    double alpha = col[k] > 0 ? -norm : norm;
    double v0 = col[k] - alpha;
    // v = (v0, col[k+1..m-1]); H = I - 2 v v^T / (v^T v)
    double vtv = v0 * v0;
    for (int i = k + 1; i < m; ++i) vtv += col[i] * col[i];
    col[k] = v0;
    for (int jc = k + 1; jc < W; ++jc) {
      double* cj = &M[size_t(jc) * m];
      double dot = 0.0;
      for (int i = k; i < m; ++i) dot += col[i] * cj[i];
      double f = 2.0 * dot / vtv;
      for (int i = k; i < m; ++i) cj[i] -= f * col[i];
    }
    double dot = 0.0;
    for (int i = k; i < m; ++i) dot += col[i] * rhs[i];
    double f = 2.0 * dot / vtv;
    for (int i = k; i < m; ++i) rhs[i] -= f * col[i];
    col[k] = alpha;  // R diagonal
  }
  for (int i = W - 1; i >= 0; --i) {
    double v = rhs[i];
    for (int jc = i + 1; jc < W; ++jc) v -= M[size_t(jc) * m + i] * c[jc];
    c[i] = v / M[size_t(i) * m + i];
  }
  return true;
}

// Solver for C_r(s) given the 2Ng+1 values of h.
class CSolver {
 public:
  CSolver(const Nodes& nd, int W) : nd_(nd), W_(W), use_qr_(W > 11) {}

  // Prepare for a new h (factor A for the normal-equation route).
  bool set_h(const std::vector<double>& h) {
    h_ = h;
    if (use_qr_) return true;
    // Toeplitz A[a][b] = sum_i w_i h_i^2 cos(2 pi (a-b) x_i)
    std::vector<double> t(W_, 0.0);
    for (int m = 0; m < W_; ++m) {
      double acc = 0.0;
      for (int i = 0; i < nd_.K; ++i) acc += nd_.w[i] * h[i] * h[i] * std::cos(kTwoPi * m * nd_.x[i]);
      t[m] = acc;
    }
    L_.assign(size_t(W_) * W_, 0.0);
    for (int a = 0; a < W_; ++a)
      for (int b = 0; b < W_; ++b) L_[a * W_ + b] = t[std::abs(a - b)];
    return cholesky(L_, W_);
  }

  // b <- A^-1 b (normal-equation route only).
  void solve_A(double* b) const { cholesky_solve(L_, W_, b); }

  // C_j(s), j = 0..W-1, for offsets d_j = j - W/2 + s.
  bool solve(double s, double* c) const {
    const int K = nd_.K;
    if (!use_qr_) {
      for (int a = 0; a < W_; ++a) {
        double d = a - 0.5 * W_ + s, acc = 0.0;
        for (int i = 0; i < K; ++i) acc += nd_.w[i] * h_[i] * std::cos(kTwoPi * d * nd_.x[i]);
        c[a] = acc;
      }
      cholesky_solve(L_, W_, c);
      return true;
    }
    const int m = 2 * K;
    std::vector<double> M(size_t(m) * W_), rhs(m, 0.0);
    for (int a = 0; a < W_; ++a) {
      double d = a - 0.5 * W_ + s;
      for (int i = 0; i < K; ++i) {
        double sw = std::sqrt(nd_.w[i]) * h_[i], ph = kTwoPi * d * nd_.x[i];
        M[size_t(a) * m + i] = sw * std::cos(ph);
        M[size_t(a) * m + K + i] = sw * std::sin(ph);
      }
    }
    for (int i = 0; i < K; ++i) rhs[i] = std::sqrt(nd_.w[i]);
    return householder_lstsq(M, m, W_, rhs, c);
  }

 private:
  const Nodes& nd_;
  int W_;
  bool use_qr_;
  std::vector<double> h_, L_;
};

// Trigonometric tables of one design problem (they do not depend on h):
// ce/se[j][a][i] = cos/sin(2 pi d_a(s_j) x_i), ca[m][i] = cos(2 pi m x_i).
struct Design {
  const Nodes& nd;
  int W;
  double x0p;
  std::vector<double> ce, se, ca;
  Design(const Nodes& n, int W_, double x0p_) : nd(n), W(W_), x0p(x0p_) {
    const int K = nd.K;
    ce.resize(size_t(kMg) * W * K);
    se.resize(ce.size());
    ca.resize(size_t(W) * K);
    for (int j = 0; j < kMg; ++j)
      for (int a = 0; a < W; ++a)
        for (int i = 0; i < K; ++i) {
          double ph = kTwoPi * (a - 0.5 * W + nd.s[j]) * nd.x[i];
          ce[(size_t(j) * W + a) * K + i] = std::cos(ph);
          se[(size_t(j) * W + a) * K + i] = std::sin(ph);
        }
    for (int m = 0; m < W; ++m)
      for (int i = 0; i < K; ++i) ca[size_t(m) * K + i] = std::cos(kTwoPi * m * nd.x[i]);
  }
};

// Residual vector r (size 2 Mg K) with |r|^2 = E for h on the Ng+1 nodes (h[0] = 1).
// r = sqrt(w_i / (2 x0 Mg)) (1 - h_i a(x_i; s_j)), real parts then imaginary parts.
bool residuals(const Design& dz, const std::vector<double>& h_half, std::vector<double>& r) {
  const Nodes& nd = dz.nd;
  const int K = nd.K, W = dz.W;
  std::vector<double> h(K), wh(K);
  for (int i = 0; i < K; ++i) {
    h[i] = h_half[std::abs(i - kNg)];
    wh[i] = nd.w[i] * h[i];
  }
  r.assign(size_t(2) * kMg * K, 0.0);
  double c[kMaxW];
  std::vector<double> L;
  if (W <= 11) {
    L.assign(size_t(W) * W, 0.0);
    double tt[kMaxW];
    for (int m = 0; m < W; ++m) {
      double acc = 0.0;
      for (int i = 0; i < K; ++i) acc += wh[i] * h[i] * dz.ca[size_t(m) * K + i];
      tt[m] = acc;
    }
    for (int a = 0; a < W; ++a)
      for (int b = 0; b < W; ++b) L[a * W + b] = tt[std::abs(a - b)];
    if (!cholesky(L, W)) return false;
  }
  std::vector<double> M, rhs;
  for (int j = 0; j < kMg; ++j) {
    const double* cej = &dz.ce[size_t(j) * W * K];
    const double* sej = &dz.se[size_t(j) * W * K];
    if (W <= 11) {
      for (int a = 0; a < W; ++a) {
        double acc = 0.0;
        for (int i = 0; i < K; ++i) acc += wh[i] * cej[size_t(a) * K + i];
        c[a] = acc;
      }
      cholesky_solve(L, W, c);
    } else {
      const int m = 2 * K;
      M.assign(size_t(m) * W, 0.0);
      rhs.assign(m, 0.0);
      for (int a = 0; a < W; ++a)
        for (int i = 0; i < K; ++i) {
          double sw = std::sqrt(nd.w[i]) * h[i];
          M[size_t(a) * m + i] = sw * cej[size_t(a) * K + i];
          M[size_t(a) * m + K + i] = sw * sej[size_t(a) * K + i];
        }
      for (int i = 0; i < K; ++i) rhs[i] = std::sqrt(nd.w[i]);
      if (!householder_lstsq(M, m, W, rhs, c)) return false;
    }
    for (int i = 0; i < K; ++i) {
      double re = 0.0, im = 0.0;
      for (int a = 0; a < W; ++a) {
        re += c[a] * cej[size_t(a) * K + i];
        im += c[a] * sej[size_t(a) * K + i];
      }
      double sc = std::sqrt(nd.w[i] / (2.0 * dz.x0p * kMg));
      r[size_t(j) * K + i] = sc * (1.0 - h[i] * re);
      r[size_t(kMg) * K + size_t(j) * K + i] = -sc * h[i] * im;
    }
  }
  return true;
}

double sumsq(const std::vector<double>& r) {
  double s = 0.0;
  for (double v : r) s += v * v;
  return s;
}

// Levenberg-Marquardt on h(x_1..x_Ng) with h(0) = 1 (Appendix A), Marquardt diagonal
// scaling and a forward-difference Jacobian. Returns the number of iterations or -1.
int levenberg_marquardt(const Design& dz, std::vector<double>& h_half, double& E) {
  const int P = kNg;  // parameters h_1..h_Ng
  std::vector<double> r, rt, J;
  if (!residuals(dz, h_half, r)) return -1;
  const size_t R = r.size();
  double F = sumsq(r);
  double lambda = 1e-3, nu = 2.0;
  int stall = 0, it = 0;
  const int max_iter = 20000;
  std::vector<double> JtJ(P * P), g(P), step(P), A(P * P), trial;
  for (it = 0; it < max_iter; ++it) {
    // Jacobian by forward differences.
    J.assign(R * P, 0.0);
    std::vector<double> hp = h_half;
    for (int k = 0; k < P; ++k) {
      double hk = h_half[k + 1];
      double dh = 1.4901161193847656e-08 * std::max(std::fabs(hk), 1e-3);
      hp[k + 1] = hk + dh;
      if (!residuals(dz, hp, rt)) return -1;
      hp[k + 1] = hk;
      for (size_t q = 0; q < R; ++q) J[q * P + k] = (rt[q] - r[q]) / dh;
    }
    for (int a = 0; a < P; ++a) {
      double ga = 0.0;
      for (size_t q = 0; q < R; ++q) ga += J[q * P + a] * r[q];
      g[a] = ga;
      for (int b = a; b < P; ++b) {
        double v = 0.0;
        for (size_t q = 0; q < R; ++q) v += J[q * P + a] * J[q * P + b];
        JtJ[a * P + b] = JtJ[b * P + a] = v;
      }
    }
    bool accepted = false;
    for (int tries = 0; tries < 40 && !accepted; ++tries) {
      A = JtJ;
      for (int a = 0; a < P; ++a) A[a * P + a] += lambda * std::max(JtJ[a * P + a], 1e-300);
      if (!cholesky(A, P)) { lambda *= nu; nu *= 2.0; continue; }
      for (int a = 0; a < P; ++a) step[a] = -g[a];
      cholesky_solve(A, P, step.data());
      trial = h_half;
      for (int a = 0; a < P; ++a) trial[a + 1] += step[a];
      std::vector<double> rtrial;
      if (!residuals(dz, trial, rtrial)) { lambda *= nu; nu *= 2.0; continue; }
      double Ft = sumsq(rtrial);
      // predicted reduction of the local quadratic model
      double pred = 0.0;
      for (int a = 0; a < P; ++a) pred += step[a] * (lambda * std::max(JtJ[a * P + a], 1e-300) * step[a] - g[a]);
      if (Ft < F) {
        double rho = pred > 0 ? (F - Ft) / pred : 1.0;
        double rel = (F - Ft) / F;
        h_half = trial;
        r.swap(rtrial);
        F = Ft;
        double t = 2.0 * rho - 1.0;
        lambda *= std::max(1.0 / 3.0, 1.0 - t * t * t);
        nu = 2.0;
        accepted = true;
        double snorm = 0.0, hnorm = 0.0;
        for (int a = 0; a < P; ++a) { snorm += step[a] * step[a]; hnorm += h_half[a + 1] * h_half[a + 1]; }
        stall = (rel < 1e-13 && snorm < 1e-26 * hnorm) ? stall + 1 : 0;
      } else {
        lambda *= nu;
        nu *= 2.0;
      }
    }
    if (!accepted || stall >= 3) break;
  }
  E = F;
  return it;
}

}  // namespace

int build_least_misfit(int W, double x0p, int Ms, lmg_table* t) {
  Nodes nd = make_nodes(x0p);
  // Initial guesses of Appendix A: h = 1 for W <= 4, h_W = h_{W-1}^2 / h_{W-2} above,
  // so W' = 3, 4, ..., W are optimised in turn.
  std::vector<double> ones(kNg + 1, 1.0), prev1, prev2, cur;
  double E = 0.0;
  int iters = 0;
  for (int Wp = (W <= 4 ? W : 3); Wp <= W; ++Wp) {
    if (Wp <= 4) {
      cur = ones;
    } else {
      cur.resize(kNg + 1);
      for (int k = 0; k <= kNg; ++k) cur[k] = prev1[k] * prev1[k] / prev2[k];
    }
    Design dz(nd, Wp, x0p);
    iters = levenberg_marquardt(dz, cur, E);
    if (iters < 0) return set_error(LMG_ENOCONV, "least-misfit optimisation failed (singular system)");
    prev2 = prev1;
    prev1 = cur;
  }
  t->h_nodes = cur;
  t->E = E;
  t->iterations = iters;
  // Look-up table (Appendix E): row i at s = i / Ms, i = 0..Ms.
  std::vector<double> h(nd.K);
  for (int i = 0; i < nd.K; ++i) h[i] = cur[std::abs(i - kNg)];
  t->C.assign(size_t(Ms + 1) * W, 0.0);
  unsigned nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  if (Ms < 4096) nth = 1;
  std::vector<int> ok(nth, 1);
  auto work = [&](unsigned tid) {
    CSolver solver(nd, W);
    if (!solver.set_h(h)) { ok[tid] = 0; return; }
    for (int i = int(tid); i <= Ms; i += int(nth))
      if (!solver.solve(double(i) / Ms, &t->C[size_t(i) * W])) ok[tid] = 0;
  };
  std::vector<std::thread> pool;
  for (unsigned k = 1; k < nth; ++k) pool.emplace_back(work, k);
  work(0);
  for (auto& th : pool) th.join();
  for (int v : ok)
    if (!v) return set_error(LMG_ENOCONV, "table solve failed (singular system)");
  return LMG_OK;
}

// Direct calculation (Section 5.2): A is Toeplitz and does not depend on s, so
// C(s) = A^-1 B(s) with B_a(s) = sum_i w_i h_i cos(2 pi (a - W/2 + s) x_i). The nodes are
// symmetric (x_{-k} = -x_k, h even), so B_a folds onto k = 0..Ng with weights omega_k and
// angles theta_k = k phi, phi = 2 pi x0 / Ng; expanding cos(theta_k (a - W/2) + theta_k s)
// gives C_a(s) = sum_k alpha[a][k] cos(k phi s) + beta[a][k] sin(k phi s) with
// alpha[a][k] = sum_b Ainv[a][b] omega_k cos(theta_k (b - W/2)) and
// beta[a][k] = -sum_b Ainv[a][b] omega_k sin(theta_k (b - W/2)).
int direct_coefficients(const lmg_table* t, std::vector<double>& out) {
  const int W = t->W, Kn = kNg + 1;
  if (W > kDirectMaxW) return set_error(LMG_EUNSUPPORTED, "direct calculation needs W <= 11 (normal equations)");
  if (t->h_nodes.size() != size_t(Kn) || !(t->h_nodes[0] > 0.0))
    return set_error(LMG_EINVAL, "direct calculation needs a least-misfit table (h is unknown for caller tables)");
  Nodes nd = make_nodes(t->x0p);
  std::vector<double> h(nd.K);
  for (int i = 0; i < nd.K; ++i) h[i] = t->h_nodes[size_t(std::abs(i - kNg))];
  CSolver solver(nd, W);
  if (!solver.set_h(h)) return set_error(LMG_ENOCONV, "direct calculation: A is not positive definite");
  // A^-1, column by column through the Cholesky factor
  std::vector<double> Ainv(size_t(W) * W);
  for (int b = 0; b < W; ++b) {
    std::vector<double> e(W, 0.0);
    e[b] = 1.0;
    solver.solve_A(e.data());
    for (int a = 0; a < W; ++a) Ainv[size_t(a) * W + b] = e[a];
  }
  const double phi = kTwoPi * t->x0p / kNg;
  out.assign(1 + size_t(2) * W * Kn, 0.0);
  out[0] = phi;
  for (int k = 0; k < Kn; ++k) {
    const double omega = (k == 0 ? 1.0 : 2.0) * nd.w[size_t(kNg + k)] * h[size_t(kNg + k)];
    for (int a = 0; a < W; ++a) {
      double al = 0.0, be = 0.0;
      for (int b = 0; b < W; ++b) {
        const double th = k * phi * (b - 0.5 * W);
        al += Ainv[size_t(a) * W + b] * omega * std::cos(th);
        be -= Ainv[size_t(a) * W + b] * omega * std::sin(th);
      }
      out[1 + size_t(a) * Kn + k] = al;
      out[1 + size_t(W + a) * Kn + k] = be;
    }
  }
  return LMG_OK;
}

// c(x) = int_0^1 ds sum_j C_j(s) cos(2 pi d_j x), D(x) = int_0^1 ds |sum_j C_j(s) e^{i 2 pi d_j x}|^2
// (Eqs. 12-14) for the interpolated table function; h = c / D (Eq. 15) or 1 / c.
void correction_factors(const lmg_table* t, int64_t n_image, int64_t N, bool single_precision,
                        double* h_out) {
  const int W = t->W, Ms = t->Ms;
  std::vector<double> T(t->C);
  if (single_precision)
    for (double& v : T) v = double(float(v));
  // 8-point Gauss-Legendre nodes/weights on [-1, 1].
  static const double gx[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290,
                               -0.1834346424956498, 0.1834346424956498,  0.5255324099163290,
                               0.7966664774136267,  0.9602898564975363};
  static const double gw[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873,
                               0.3626837833783620, 0.3626837833783620, 0.3137066458778873,
                               0.2223810344533745, 0.1012285362903763};
  // Integration pieces: one per table piece (linear: [k, k+1]/Ms; nearest: centred on
  // the rows); beyond 4096 pieces, 4096 equal pieces (the kinks then sit far below
  // double-precision relevance).
  std::vector<double> edges;
  const bool direct = t->interp == LMG_INTERP_DIRECT;
  if (direct) {  // the exact function is smooth in s: 64 equal pieces
    for (int k = 0; k <= 64; ++k) edges.push_back(double(k) / 64);
  } else if (Ms <= 4096) {
    if (t->interp == LMG_INTERP_LINEAR) {
      for (int k = 0; k <= Ms; ++k) edges.push_back(double(k) / Ms);
    } else if (t->interp == LMG_INTERP_NEAREST) {
      edges.push_back(0.0);
      for (int k = 0; k < Ms; ++k) edges.push_back((k + 0.5) / Ms);
      edges.push_back(1.0);
    } else {  // degree 2, 3: half-row pieces contain every change of stencil
      for (int k = 0; k <= 2 * Ms; ++k) edges.push_back(double(k) / (2.0 * Ms));
    }
  } else {
    for (int k = 0; k <= 4096; ++k) edges.push_back(double(k) / 4096);
  }
  const size_t npieces = edges.size() - 1;
  std::vector<double> sn(npieces * 8), sw(npieces * 8), Cn(npieces * 8 * W);
  Nodes nd = make_nodes(t->x0p);
  std::vector<double> hfull(nd.K);
  for (int i = 0; i < nd.K; ++i) hfull[i] = t->h_nodes.empty() ? 0.0 : t->h_nodes[size_t(std::abs(i - kNg))];
  CSolver exact(nd, W);
  if (direct) exact.set_h(hfull);
  for (size_t p = 0; p < npieces; ++p) {
    double lo = edges[p], hi = edges[p + 1], half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
    for (int g = 0; g < 8; ++g) {
      size_t q = p * 8 + g;
      double s = mid + half * gx[g];
      sn[q] = s;
      sw[q] = half * gw[g];
      if (direct) {
        exact.solve(s, &Cn[q * W]);
      } else if (t->interp == LMG_INTERP_LINEAR) {
        double tt = s * Ms;
        int k = std::min(int(std::floor(tt)), Ms - 1);
        double f = tt - k;
        for (int j = 0; j < W; ++j)
          Cn[q * W + j] = (1.0 - f) * T[size_t(k) * W + j] + f * T[size_t(k + 1) * W + j];
      } else if (t->interp >= LMG_INTERP_QUADRATIC) {
        // Lagrange interpolation of degree d through rows k0 .. k0 + d (Appendix F)
        const int d = t->interp;
        const double tt = s * Ms;
        int k0 = int(std::floor(tt - 0.5 * (d - 1)));
        k0 = std::max(0, std::min(k0, Ms - d));
        const double x = tt - k0;
        double L[4];
        for (int m = 0; m <= d; ++m) {
          double v = 1.0;
          for (int jj = 0; jj <= d; ++jj)
            if (jj != m) v *= (x - jj) / double(m - jj);
          L[m] = v;
        }
        for (int j = 0; j < W; ++j) {
          double v = 0.0;
          for (int m = 0; m <= d; ++m) v += L[m] * T[size_t(k0 + m) * W + j];
          Cn[q * W + j] = v;
        }
      } else {
        int k = int(std::floor(s * Ms + 0.5));
        for (int j = 0; j < W; ++j) Cn[q * W + j] = T[size_t(k) * W + j];
      }
    }
  }
  // h is even: evaluate |x| once per distinct value.
  const int64_t half_n = n_image / 2;
  std::vector<double> hpos(size_t(half_n) + 1);
  unsigned nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  auto work = [&](unsigned tid) {
    for (int64_t a = tid; a <= half_n; a += nth) {
      double x = double(a) / double(N);
      double c = 0.0, D = 0.0;
      const double zr = std::cos(kTwoPi * x), zi = std::sin(kTwoPi * x);
      for (size_t q = 0; q < sn.size(); ++q) {
        // sum_j C_j z^j by Horner, then times exp(i 2 pi (s - W/2) x)
        double pr = 0.0, pi = 0.0;
        for (int j = W - 1; j >= 0; --j) {
          double nr = pr * zr - pi * zi + Cn[q * W + j];
          double ni = pr * zi + pi * zr;
          pr = nr;
          pi = ni;
        }
        double ph = kTwoPi * (sn[q] - 0.5 * W) * x;
        double er = std::cos(ph), ei = std::sin(ph);
        double ar = pr * er - pi * ei, ai = pr * ei + pi * er;
        c += sw[q] * ar;
        D += sw[q] * (ar * ar + ai * ai);
      }
      hpos[size_t(a)] = (t->correction == LMG_CORR_INV_C) ? 1.0 / c : c / D;
    }
  };
  std::vector<std::thread> pool;
  for (unsigned k = 1; k < nth; ++k) pool.emplace_back(work, k);
  work(0);
  for (auto& th : pool) th.join();
  for (int64_t p = 0; p < n_image; ++p) h_out[p] = hpos[size_t(std::llabs(p - half_n))];
}

}  // namespace lmg

// Host-side discretisation tables of libsg: quadrature, nodal bases, the dG(r)
// time matrices, the Hermite chaos index set and triple products, and the
// coefficient values at the quadrature points.  Everything here runs once per
// sg_setup; the per-apply work is in sg_apply.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>

#include "sg_internal.h"

namespace sg {

// Legendre polynomial P_n(x) and its derivative by the three-term recurrence.
static void legendre(int n, double x, double& p, double& dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { p = 1.0; dp = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = pk;
  }
  p = p1;
  if (std::fabs(x) < 1.0) dp = n * (x * p1 - p0) / (x * x - 1.0);
  else dp = 0.5 * n * (n + 1) * ((x > 0 || (n % 2)) ? 1.0 : -1.0);  // P_n'(+-1)
}

Rule1D gauss_legendre(int n) {
  // Newton on P_n from the Chebyshev-like guesses, then map [-1,1] -> [0,1].
  Rule1D r;
  r.x.resize(n);
  r.w.resize(n);
  for (int i = 0; i < n; ++i) {
    double x = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(n, x, p, dp);
      double dx = p / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    double p, dp;
    legendre(n, x, p, dp);
    r.x[n - 1 - i] = 0.5 * (x + 1.0);
    r.w[n - 1 - i] = 1.0 / ((1.0 - x * x) * dp * dp);  // 2/((1-x^2)P'^2) halved
  }
  return r;
}

std::vector<double> lobatto_nodes(int k) {
  if (k == 1) return {0.0, 1.0};
  if (k == 2) return {0.0, 0.5, 1.0};
  if (k == 3) {
    double s = 1.0 / std::sqrt(5.0);
    return {0.0, 0.5 * (1.0 - s), 0.5 * (1.0 + s), 1.0};
  }
  return {};
}

std::vector<double> radau_right_nodes(int r) {
  // Roots of q(x) = P_r(x) - P_{r+1}(x) on [-1, 1]; x = 1 is one of them.
  std::vector<double> out;
  if (r == 0) return {1.0};
  auto q = [&](double x) {
    double a, da, b, db;
    legendre(r, x, a, da);
    legendre(r + 1, x, b, db);
    return a - b;
  };
  const int n_scan = 4000;
  double xa = -1.0, qa = q(xa);
  for (int s = 1; s <= n_scan; ++s) {
    double xb = -1.0 + 2.0 * s / n_scan;
    if (s == n_scan) xb = 1.0 - 1e-9;
    double qb = q(xb);
    if (qa == 0.0) { out.push_back(xa); }
    else if (qa * qb < 0.0) {
      double lo = xa, hi = xb, flo = qa;
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi), fm = q(mid);
        if (fm == 0.0 || hi - lo < 1e-17) { lo = hi = mid; break; }
        if (flo * fm < 0.0) hi = mid; else { lo = mid; flo = fm; }
      }
      out.push_back(0.5 * (lo + hi));
    }
    xa = xb;
    qa = qb;
  }
  out.push_back(1.0);
  for (double& v : out) v = 0.5 * (v + 1.0);
  std::sort(out.begin(), out.end());
  return out;
}

double lagrange(const std::vector<double>& nodes, int i, double t) {
  double v = 1.0;
  for (size_t j = 0; j < nodes.size(); ++j)
    if ((int)j != i) v *= (t - nodes[j]) / (nodes[i] - nodes[j]);
  return v;
}

double lagrange_deriv(const std::vector<double>& nodes, int i, double t) {
  double s = 0.0;
  for (size_t k = 0; k < nodes.size(); ++k) {
    if ((int)k == i) continue;
    double term = 1.0 / (nodes[i] - nodes[k]);
    for (size_t j = 0; j < nodes.size(); ++j)
      if ((int)j != i && j != k) term *= (t - nodes[j]) / (nodes[i] - nodes[j]);
    s += term;
  }
  return s;
}

void time_matrices(int r, std::vector<double>& A, std::vector<double>& B) {
  const int n = r + 1;
  std::vector<double> nodes = radau_right_nodes(r);
  Rule1D g = gauss_legendre(r + 2);
  A.assign(n * n, 0.0);
  B.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double a = lagrange(nodes, j, 0.0) * lagrange(nodes, i, 0.0);  // jump at t_{n-1}^+
      double b = 0.0;
      for (size_t q = 0; q < g.x.size(); ++q) {
        a += g.w[q] * lagrange_deriv(nodes, j, g.x[q]) * lagrange(nodes, i, g.x[q]);
        b += g.w[q] * lagrange(nodes, j, g.x[q]) * lagrange(nodes, i, g.x[q]);
      }
      A[i * n + j] = a;
      B[i * n + j] = b;
    }
}

std::vector<int> chaos_indices(int M, int p) {
  std::vector<int> out;
  std::vector<int> cur(M, 0);
  // all alpha with |alpha| = deg, alpha_1 descending first, recursively
  std::function<void(int, int)> rec = [&](int m, int left) {
    if (m == M - 1) {
      cur[m] = left;
      out.insert(out.end(), cur.begin(), cur.end());
      return;
    }
    for (int a = left; a >= 0; --a) {
      cur[m] = a;
      rec(m + 1, left - a);
    }
  };
  for (int d = 0; d <= p; ++d) rec(0, d);
  return out;
}

double hermite_triple(int a, int b, int c) {
  // Selection rule: a+b+c even and |a-b| <= c <= a+b.
  if ((a + b + c) % 2 || c < std::abs(a - b) || c > a + b) return 0.0;
  // psi_a(J) e_b, with J the Jacobi matrix of the orthonormal Hermite basis
  // (xi psi_n = sqrt(n+1) psi_{n+1} + sqrt(n) psi_{n-1}); its c-th entry is
  // E[psi_a psi_b psi_c].
  const int L = a + b + 2;
  std::vector<double> wm(L, 0.0), w(L, 0.0), wn(L, 0.0);
  w[b] = 1.0;  // psi_0(J) e_b
  auto applyJ = [&](const std::vector<double>& v, std::vector<double>& o) {
    for (int n = 0; n < L; ++n) {
      double s = 0.0;
      if (n > 0) s += std::sqrt((double)n) * v[n - 1];
      if (n + 1 < L) s += std::sqrt((double)(n + 1)) * v[n + 1];
      o[n] = s;
    }
  };
  for (int s = 0; s < a; ++s) {
    applyJ(w, wn);
    for (int n = 0; n < L; ++n)
      wn[n] = (wn[n] - std::sqrt((double)s) * wm[n]) / std::sqrt((double)(s + 1));
    wm = w;
    w = wn;
  }
  return w[c];
}

double factor_value(int kind, int k, double s) {
  switch (kind) {
    case SG_F_ONE: return 1.0;
    case SG_F_SIN: return std::sin(k * M_PI * s);
    case SG_F_POW: return std::pow(s, (double)k);
  }
  return 0.0;
}

sg_status build_host_problem(const sg_mesh* mesh, int k, int r, int n_slabs, double T,
                             int M, int p, const sg_coeff* coef, HostProblem& hp,
                             std::string& msg) {
  if (!mesh || !coef) { msg = "null mesh or coefficient"; return SG_ERR_ARG; }
  if (coef->n_pieces < 1 || !coef->mu || !coef->amp || !coef->factor_kind || !coef->factor_k) {
    msg = "coefficient needs at least one piece and all arrays";
    return SG_ERR_ARG;
  }
  if (M < 1 || M > 16) { msg = "invalid M"; return SG_ERR_ARG; }
  int64_t n_cells = 1;
  for (int d = 0; d < mesh->dim && d < 3; ++d) n_cells *= std::max(1, mesh->cells[d]);
  std::vector<Piece> pieces;
  sg_status st = parse_pieces(coef, M, n_cells, pieces, msg);
  if (st != SG_OK) return st;
  return build_host_problem_pieces(mesh, k, r, n_slabs, T, M, p, pieces, hp, msg);
}

sg_status parse_pieces(const sg_coeff* coef, int M, int64_t n_cells, std::vector<Piece>& pieces, std::string& msg) {
  if (!coef) { msg = "null coefficient"; return SG_ERR_ARG; }
  if (coef->n_pieces < 1 || !coef->mu || !coef->amp || !coef->factor_kind || !coef->factor_k) {
    msg = "coefficient needs at least one piece and all arrays";
    return SG_ERR_ARG;
  }
  pieces.assign(coef->n_pieces, Piece());
  for (int pc = 0; pc < coef->n_pieces; ++pc) {
    Piece& q = pieces[pc];
    q.mu.assign(coef->mu + (size_t)pc * M, coef->mu + (size_t)(pc + 1) * M);
    q.amp = coef->amp[pc];
    for (int d = 0; d < 3; ++d) {
      q.kind[d] = coef->factor_kind[pc * 3 + d];
      q.k[d] = coef->factor_k[pc * 3 + d];
    }
    if (coef->cell_scale && coef->cell_scale[pc])
      q.scale.assign(coef->cell_scale[pc], coef->cell_scale[pc] + n_cells);
  }
  return SG_OK;
}

sg_status build_host_problem_pieces(const sg_mesh* mesh, int k, int r, int n_slabs, double T,
                                    int M, int p, const std::vector<Piece>& pieces,
                                    HostProblem& hp, std::string& msg) {
  if (!mesh) { msg = "null mesh"; return SG_ERR_ARG; }
  if (mesh->dim != 2 && mesh->dim != 3) { msg = "dim must be 2 or 3"; return SG_ERR_UNSUPPORTED; }
  if (k < 1 || k > kMaxK || (mesh->dim == 3 && k > 2)) { msg = "fe_degree not built"; return SG_ERR_UNSUPPORTED; }
  if (r < 0 || r + 1 > kMaxNT) { msg = "time_degree not built"; return SG_ERR_UNSUPPORTED; }
  if (n_slabs < 1 || !(T > 0.0) || M < 1 || p < 0 || M > 16 || p > 12) { msg = "invalid slabs, T, M or order"; return SG_ERR_ARG; }
  if (pieces.empty()) { msg = "coefficient needs at least one piece"; return SG_ERR_ARG; }
  hp.pieces = pieces;
  hp.dim = mesh->dim; hp.k = k; hp.r = r; hp.M = M; hp.p = p; hp.n_slabs = n_slabs; hp.T = T;
  hp.tau = T / n_slabs;
  hp.n_x = 1; hp.n_cells = 1;
  for (int d = 0; d < 3; ++d) {
    if (d < hp.dim) {
      if (mesh->cells[d] < 1 || !(mesh->hi[d] > mesh->lo[d])) { msg = "invalid mesh extent"; return SG_ERR_ARG; }
      hp.cells[d] = mesh->cells[d];
      hp.lo[d] = mesh->lo[d];
      hp.h[d] = (mesh->hi[d] - mesh->lo[d]) / mesh->cells[d];
      hp.nn[d] = k * mesh->cells[d] + 1;
    } else {
      hp.cells[d] = 1; hp.nn[d] = 1; hp.lo[d] = 0.0; hp.h[d] = 1.0;
    }
    hp.n_x *= hp.nn[d];
    hp.n_cells *= hp.cells[d];
  }
  // chaos
  hp.idx = chaos_indices(M, p);
  hp.n_xi = (int)(hp.idx.size() / M);
  hp.n_t = r + 1;
  if ((long long)hp.n_xi * hp.n_t * hp.n_x > (1LL << 40) || hp.n_x >= (1LL << 31) || hp.n_cells >= (1LL << 31)) {
    msg = "problem too large";
    return SG_ERR_ARG;
  }
  // active coefficient terms (first appearance order)
  hp.mus.clear();
  const int n_pieces = (int)pieces.size();
  std::vector<int> piece_term(n_pieces);
  for (int pc = 0; pc < n_pieces; ++pc) {
    const std::vector<int>& mu = pieces[pc].mu;
    if ((int)mu.size() != M) { msg = "coefficient index of wrong length"; return SG_ERR_ARG; }
    for (int v : mu) if (v < 0) { msg = "negative chaos index in coefficient"; return SG_ERR_ARG; }
    auto it = std::find(hp.mus.begin(), hp.mus.end(), mu);
    if (it == hp.mus.end()) { piece_term[pc] = (int)hp.mus.size(); hp.mus.push_back(mu); }
    else piece_term[pc] = (int)(it - hp.mus.begin());
    for (int d = 0; d < hp.dim; ++d) {
      int kd = pieces[pc].kind[d];
      if (kd != SG_F_ONE && kd != SG_F_SIN && kd != SG_F_POW) { msg = "unknown factor kind"; return SG_ERR_ARG; }
      if (kd == SG_F_POW && pieces[pc].k[d] < 0) { msg = "negative power"; return SG_ERR_ARG; }
    }
    if (!pieces[pc].scale.empty() && (int64_t)pieces[pc].scale.size() != hp.n_cells) {
      msg = "cell scale of wrong length";
      return SG_ERR_ARG;
    }
  }
  hp.piece_term = piece_term;
  hp.n_terms = (int)hp.mus.size();
  // stochastic coupling table, row by row
  hp.g.row.assign(hp.n_xi + 1, 0);
  hp.g.col.clear(); hp.g.term.clear(); hp.g.val.clear();
  for (int a = 0; a < hp.n_xi; ++a) {
    for (int t = 0; t < hp.n_terms; ++t)
      for (int b = 0; b < hp.n_xi; ++b) {
        double g = 1.0;
        for (int m = 0; m < M && g != 0.0; ++m)
          g *= hermite_triple(hp.mus[t][m], hp.idx[a * M + m], hp.idx[b * M + m]);
        if (g != 0.0) {
          hp.g.col.push_back(b);
          hp.g.term.push_back(t);
          hp.g.val.push_back(g);
        }
      }
    hp.g.row[a + 1] = (int)hp.g.col.size();
  }
  // time
  time_matrices(r, hp.A_hat, hp.B_hat);
  for (int i = 0; i < hp.n_t; ++i)
    for (int j = 0; j < hp.n_t; ++j)
      if (i != j && std::fabs(hp.B_hat[i * hp.n_t + j]) > 1e-13) {
        msg = "time mass matrix is not diagonal";
        return SG_ERR_UNSUPPORTED;
      }
  // chaos rows ordered by their number of coupling entries (warp uniformity)
  hp.perm.resize(hp.n_xi);
  for (int a = 0; a < hp.n_xi; ++a) hp.perm[a] = a;
  std::stable_sort(hp.perm.begin(), hp.perm.end(), [&](int a, int b) {
    return hp.g.row[a + 1] - hp.g.row[a] > hp.g.row[b + 1] - hp.g.row[b];
  });
  // 1D spatial bases at the (k+1)-point Gauss rule
  const int nq = k + 1;
  Rule1D g = gauss_legendre(nq);
  std::vector<double> gll = lobatto_nodes(k);
  hp.wq = g.w;
  hp.S.assign(nq * nq, 0.0);
  hp.Dhat.assign(nq * nq, 0.0);
  hp.dS.assign(nq * nq, 0.0);
  for (int q = 0; q < nq; ++q)
    for (int n = 0; n < nq; ++n) {
      hp.S[q * nq + n] = lagrange(gll, n, g.x[q]);
      hp.Dhat[q * nq + n] = lagrange_deriv(g.x, n, g.x[q]);
      hp.dS[q * nq + n] = lagrange_deriv(gll, n, g.x[q]);
    }
  return fill_ctab(hp, msg);
}

sg_status fill_ctab(HostProblem& hp, std::string& msg) {
  // coefficient values at the tensor Gauss points of every cell, times w_q |J|
  const int nq = hp.k + 1;
  Rule1D g = gauss_legendre(nq);
  const std::vector<Piece>& pieces = hp.pieces;
  const std::vector<int>& piece_term = hp.piece_term;
  const int n_pieces = (int)pieces.size();
  const int nqd = hp.dim == 2 ? nq * nq : nq * nq * nq;
  double detJ = 1.0;
  for (int d = 0; d < hp.dim; ++d) detJ *= hp.h[d];
  try {
    hp.ctab.assign((size_t)hp.n_cells * hp.n_terms * nqd, 0.0);
  } catch (...) {
    msg = "host allocation of the coefficient table failed";
    return SG_ERR_OOM;
  }
  for (int64_t c = 0; c < hp.n_cells; ++c) {
    int cc[3] = {(int)(c % hp.cells[0]), (int)((c / hp.cells[0]) % hp.cells[1]),
                 (int)(c / ((int64_t)hp.cells[0] * hp.cells[1]))};
    for (int qd = 0; qd < nqd; ++qd) {
      int qi[3] = {qd % nq, (qd / nq) % nq, qd / (nq * nq)};
      double xq[3], w = detJ;
      for (int d = 0; d < hp.dim; ++d) {
        xq[d] = hp.lo[d] + (cc[d] + g.x[qi[d]]) * hp.h[d];
        w *= g.w[qi[d]];
      }
      for (int pc = 0; pc < n_pieces; ++pc) {
        double v = pieces[pc].amp;
        for (int d = 0; d < hp.dim; ++d) v *= factor_value(pieces[pc].kind[d], pieces[pc].k[d], xq[d]);
        if (!pieces[pc].scale.empty()) v *= pieces[pc].scale[c];
        hp.ctab[((size_t)c * hp.n_terms + piece_term[pc]) * nqd + qd] += w * v / (hp.h[0] * hp.h[0]);
      }
    }
  }
  return SG_OK;
}

}  // namespace sg

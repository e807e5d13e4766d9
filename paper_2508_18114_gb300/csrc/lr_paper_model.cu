// Host-side builder of the paper's own readout model (Sec. S2.A, S2.D, S2.E)
// as the CSR operator set of the sparse engine. No device code.
//
//  1. Transmon: 4 Ec n^2 - Ej cos(phi) in the charge basis n = -n_cut..n_cut
//     (cos(phi) = (|n><n+1| + |n+1><n|)/2, offset charge 0), diagonalised by
//     cyclic Jacobi rotations (Golub & Van Loan, Matrix Computations, Sec.
//     8.5); lowest Nt levels; eigenvector signs with n_{j,j+1} > 0.
//  2. Normal modes (Sec. S2.D): for c = alpha a + beta f + gamma a^dag +
//     delta f^dag the condition [H_rf, c] = -w c is (Omega - w) x = 0 with
//     Omega = [[wr, J, 0, J], [J, wf, J, 0], [0, -J, -wr, -J], [-J, 0, -J, -wf]].
//     Its positive eigenvalues come in closed form: H_rf is two oscillators
//     coupled through their momenta (a^dag - a = -i sqrt(2) p), with normal
//     frequencies w^2 = m -+ sqrt(((wr^2 - wf^2)/2)^2 + 4 J^2 wr wf),
//     m = (wr^2 + wf^2)/2. Each null vector is a column of adj(Omega - w);
//     normalised to alpha^2 + beta^2 - gamma^2 - delta^2 = 1, beta > 0. The
//     inverse map is a = sum_i (alpha_i c_i - gamma_i c_i^dag) and
//     f = sum_i (beta_i c_i - delta_i c_i^dag) (from [a, c_i^dag] = alpha_i,
//     [a, c_i] = gamma_i), so s13 = alpha_l, s12 = -gamma_l, s14 = alpha_u,
//     s11 = -gamma_u, s23 = beta_l, s22 = -delta_l, s24 = beta_u, s21 = -delta_u.
//  3. Readout: the filter field, beta = tr(rho f) (Fig. 2), as
//     f(t) = s23 c_l + s24 c_u + e^{2i w_d t} (s21 c_u^dag + s22 c_l^dag) in the
//     frame of the drive (e^{i w_d t} times the lab-frame operator).
//  4. Operators as sums of "ladder words": a coefficient, a time channel and a
//     product of elementary operators applied right to left to a basis state;
//     an intermediate state outside the cutoffs ends the word (truncated
//     products, as matrix products of the truncated operators give).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "lr_internal.cuh"

namespace {

using cd = std::complex<double>;

// ------------------------------------------------------------- transmon
bool jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double x = A[(size_t)i * n + j] * A[(size_t)i * n + j];
        tot += x;
        if (i != j) off += x;
      }
    if (off <= 1e-30 * tot) return true;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double tau = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
        const double t = tau >= 0.0 ? 1.0 / (tau + sqrt(1.0 + tau * tau)) : -1.0 / (-tau + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {   // A <- J^T A
          const double akp = A[(size_t)p * n + k], akq = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * akp - s * akq;
          A[(size_t)q * n + k] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {   // A <- A J, V <- V J
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  return false;
}

// eps[0..Nt), nn[j] = n_{j,j+1}
bool transmon_levels(double Ec, double Ej, int n_cut, int Nt, std::vector<double>& eps, std::vector<double>& nn) {
  const int d = 2 * n_cut + 1;
  std::vector<double> A((size_t)d * d, 0.0), V;
  for (int i = 0; i < d; ++i) {
    const double n = i - n_cut;
    A[(size_t)i * d + i] = 4.0 * Ec * n * n;
    if (i + 1 < d) A[(size_t)i * d + i + 1] = A[(size_t)(i + 1) * d + i] = -0.5 * Ej;
  }
  if (!jacobi_eigen(d, A, V)) return false;
  std::vector<int> order(d);
  for (int i = 0; i < d; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return A[(size_t)x * d + x] < A[(size_t)y * d + y]; });
  std::vector<std::vector<double>> v(Nt, std::vector<double>(d));
  eps.assign(Nt, 0.0);
  for (int j = 0; j < Nt; ++j) {
    eps[j] = A[(size_t)order[j] * d + order[j]];
    for (int i = 0; i < d; ++i) v[j][i] = V[(size_t)i * d + order[j]];
  }
  auto nel = [&](int j, int k) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) s += v[j][i] * (i - n_cut) * v[k][i];
    return s;
  };
  nn.assign(Nt > 1 ? Nt - 1 : 0, 0.0);
  for (int j = 0; j + 1 < Nt; ++j) {
    if (nel(j, j + 1) < 0.0)
      for (int i = 0; i < d; ++i) v[j + 1][i] = -v[j + 1][i];
    nn[j] = nel(j, j + 1);
  }
  return true;
}

// --------------------------------------------------------- normal modes
double det3(const double m[4][4], int r0, int r1, int r2, int c0, int c1, int c2) {
  return m[r0][c0] * (m[r1][c1] * m[r2][c2] - m[r1][c2] * m[r2][c1]) -
         m[r0][c1] * (m[r1][c0] * m[r2][c2] - m[r1][c2] * m[r2][c0]) +
         m[r0][c2] * (m[r1][c0] * m[r2][c1] - m[r1][c1] * m[r2][c0]);
}

// null vector of the rank-3 matrix Omega - w: the largest column of its adjugate
bool null_vector(double wr, double wf, double J, double w, double x[4]) {
  const double O[4][4] = {{wr - w, J, 0.0, J}, {J, wf - w, J, 0.0}, {0.0, -J, -wr - w, -J}, {-J, 0.0, -J, -wf - w}};
  double best = -1.0;
  for (int col = 0; col < 4; ++col) {   // column `col` of adj = cofactors C_{col, i}
    double y[4], nrm = 0.0;
    for (int i = 0; i < 4; ++i) {
      int rr[3], cc[3], a = 0, b = 0;
      for (int k = 0; k < 4; ++k) {
        if (k != col) rr[a++] = k;
        if (k != i) cc[b++] = k;
      }
      const double sgn = ((i + col) % 2) ? -1.0 : 1.0;
      y[i] = sgn * det3(O, rr[0], rr[1], rr[2], cc[0], cc[1], cc[2]);
      nrm += y[i] * y[i];
    }
    if (nrm > best) {
      best = nrm;
      for (int i = 0; i < 4; ++i) x[i] = y[i];
    }
  }
  if (!(best > 0.0)) return false;
  const double s = x[0] * x[0] + x[1] * x[1] - x[2] * x[2] - x[3] * x[3];
  if (!(s > 0.0)) return false;
  const double inv = (x[1] < 0.0 ? -1.0 : 1.0) / sqrt(s);
  for (int i = 0; i < 4; ++i) x[i] *= inv;
  return true;
}

struct Derived {
  double wl, wu, mu_l, mu_u, nu_l, nu_u, s21, s22, s23, s24;
  std::vector<double> eps, nn;
};

bool derive(const lr_paper_params& p, Derived& D) {
  if (!transmon_levels(p.Ec, p.Ej, p.n_cut, p.Nt, D.eps, D.nn)) return false;
  const double m = 0.5 * (p.wr * p.wr + p.wf * p.wf);
  const double h = 0.5 * (p.wr * p.wr - p.wf * p.wf);
  const double dd = sqrt(h * h + 4.0 * p.J * p.J * p.wr * p.wf);
  if (!(m - dd > 0.0)) return false;
  D.wl = sqrt(m - dd);
  D.wu = sqrt(m + dd);
  double xl[4], xu[4];   // (alpha, beta, gamma, delta) of c_l, c_u
  if (!null_vector(p.wr, p.wf, p.J, D.wl, xl) || !null_vector(p.wr, p.wf, p.J, D.wu, xu)) return false;
  const double s11 = -xu[2], s12 = -xl[2], s13 = xl[0], s14 = xu[0];
  D.s21 = -xu[3];
  D.s22 = -xl[3];
  D.s23 = xl[1];
  D.s24 = xu[1];
  D.mu_u = s14 - s11;
  D.mu_l = s13 - s12;
  D.nu_u = D.s24 - D.s21;
  D.nu_l = D.s23 - D.s22;
  return true;
}

// ------------------------------------------------------------ operators
enum Op : int { LP, LM, UP, UM, TP_, TM_, BL, BR, NL, NU, ET };  // c_l^dag, c_l, c_u^dag, c_u, n^-, n^+, b, b^dag, N_l, N_u, H_t'
struct Word {
  cd coef;
  int chan;
  int n;
  int op[2];   // product op[0] op[1]: op[n-1] acts first
};
struct State {
  int l, u, t;
};

bool apply_op(int op, State& s, double& w, const lr_paper_params& p, const Derived& D) {
  switch (op) {
    case LP: if (s.l + 1 >= p.Nl) return false; w *= sqrt(s.l + 1.0); ++s.l; return true;
    case LM: if (s.l == 0) return false; w *= sqrt((double)s.l); --s.l; return true;
    case UP: if (s.u + 1 >= p.Nu) return false; w *= sqrt(s.u + 1.0); ++s.u; return true;
    case UM: if (s.u == 0) return false; w *= sqrt((double)s.u); --s.u; return true;
    case TP_: if (s.t + 1 >= p.Nt) return false; w *= D.nn[s.t]; ++s.t; return true;   // n^- |j> = n_{j,j+1} |j+1>
    case TM_: if (s.t == 0) return false; w *= D.nn[s.t - 1]; --s.t; return true;      // n^+ |j> = n_{j-1,j} |j-1>
    case BL: if (s.t == 0) return false; w *= sqrt((double)s.t); --s.t; return true;
    case BR: if (s.t + 1 >= p.Nt) return false; w *= sqrt(s.t + 1.0); ++s.t; return true;
    case NL: w *= s.l; return true;
    case NU: w *= s.u; return true;
    case ET: w *= D.eps[s.t] - D.eps[0] - s.t * p.wd; return true;
  }
  return false;
}

int chan(int a, int q) { return 5 * a + q + 2; }

std::vector<std::vector<Word>> words(const lr_paper_params& p, const Derived& D) {
  const cd I(0.0, 1.0);
  std::vector<Word> H, A, L1, L2, R;
  auto w1 = [](std::vector<Word>& v, cd c, int ch, int a) { v.push_back(Word{c, ch, 1, {a, 0}}); };
  auto w2 = [](std::vector<Word>& v, cd c, int ch, int a, int b) { v.push_back(Word{c, ch, 2, {a, b}}); };
  // Hamiltonian in the frame of the drive, Eq. S(hamiltonian_rotated)
  w1(H, 1.0, chan(0, 0), ET);
  w1(H, D.wl - p.wd, chan(0, 0), NL);
  w1(H, D.wu - p.wd, chan(0, 0), NU);
  const int up[2] = {LP, UP}, dn[2] = {LM, UM};
  const double mu[2] = {D.mu_l, D.mu_u}, nu[2] = {D.nu_l, D.nu_u};
  // frame 1, Eq. S(hamiltonian_rwa): the same terms without the explicitly
  // time-dependent ones (channels q != 0)
  const bool rwa = p.frame == 1;
  for (int x = 0; x < 2; ++x) {
    w2(H, I * p.g * mu[x], chan(0, 0), TM_, up[x]);     //  i g mu n^+ c^dag
    w2(H, -I * p.g * mu[x], chan(0, 0), TP_, dn[x]);    // -i g mu n^- c
    w1(H, -0.5 * nu[x], chan(1, 0), up[x]);             // -(nu/2) Omega (c^dag + c)
    w1(H, -0.5 * nu[x], chan(1, 0), dn[x]);
    if (rwa) continue;
    w2(H, -I * p.g * mu[x], chan(0, -2), TM_, dn[x]);   // -i g mu n^+ c e^{-2i w_d t}
    w2(H, I * p.g * mu[x], chan(0, 2), TP_, up[x]);     //  i g mu n^- c^dag e^{2i w_d t}
    w1(H, 0.5 * nu[x], chan(1, 2), up[x]);              // +(nu/2) Omega c^dag e^{2i w_d t}
    w1(H, 0.5 * nu[x], chan(1, -2), dn[x]);             // +(nu/2) Omega c e^{-2i w_d t}
  }
  for (const Word& w : H) A.push_back(Word{-I * w.coef, w.chan, w.n, {w.op[0], w.op[1]}});
  // -1/2 L_1^dag L_1 with L_1 = sqrt(kappa) (Aop + e^{2i w_d t} Bop),
  // Aop = s23 c_l + s24 c_u, Bop = s21 c_u^dag + s22 c_l^dag
  const double k2 = -0.5 * p.kappa;
  const int aop[2] = {LM, UM}, bop[2] = {UP, LP};
  const double ac[2] = {D.s23, D.s24}, bc[2] = {D.s21, D.s22};
  const int aopd[2] = {LP, UP}, bopd[2] = {UM, LM};   // adjoints
  // (RWA: L_1 = sqrt(kappa) Aop, its slow part)
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      w2(A, k2 * ac[i] * ac[j], chan(0, 0), aopd[i], aop[j]);   // Aop^dag Aop
      if (rwa) continue;
      w2(A, k2 * bc[i] * bc[j], chan(0, 0), bopd[i], bop[j]);   // Bop^dag Bop
      w2(A, k2 * ac[i] * bc[j], chan(0, 2), aopd[i], bop[j]);   // Aop^dag Bop e^{2i w_d t}
      w2(A, k2 * bc[i] * ac[j], chan(0, -2), bopd[i], aop[j]);  // Bop^dag Aop e^{-2i w_d t}
    }
  w2(A, -0.5 * p.gamma, chan(0, 0), BR, BL);   // -1/2 gamma b^dag b
  const double sk = sqrt(p.kappa);
  w1(L1, sk * D.s23, chan(0, 0), LM);
  w1(L1, sk * D.s24, chan(0, 0), UM);
  if (!rwa) {
    w1(L1, sk * D.s21, chan(0, 2), UP);
    w1(L1, sk * D.s22, chan(0, 2), LP);
  }
  w1(L2, sqrt(p.gamma), chan(0, 0), BL);
  // readout: the filter field f in the frame of the drive, e^{i w_d t} times the
  // lab-frame f (RWA: its slow part)
  w1(R, D.s23, chan(0, 0), LM);
  w1(R, D.s24, chan(0, 0), UM);
  if (!rwa) {
    w1(R, D.s21, chan(0, 2), UP);
    w1(R, D.s22, chan(0, 2), LP);
  }
  return {A, L1, L2, R};
}

struct Entry {
  int row, col, ch;
  cd v;
};

bool params_ok(const lr_paper_params* p) {
  if (!p) return false;
  if (p->Nl < 1 || p->Nu < 1 || p->Nt < 1 || p->Nt > LR_MAX_NT) return false;
  if (p->n_cut < p->Nt || p->n_cut > 64) return false;
  const double N = (double)p->Nl * p->Nu * p->Nt;
  if (N > (double)(1 << 24)) return false;
  const double v[] = {p->Ec, p->Ej, p->wr, p->wf, p->g, p->J, p->kappa, p->gamma, p->wd};
  for (double x : v)
    if (!isfinite(x)) return false;
  if (p->frame != 0 && p->frame != 1) return false;
  return p->Ec > 0.0 && p->Ej > 0.0 && p->wr > 0.0 && p->wf > 0.0 && p->kappa >= 0.0 && p->gamma >= 0.0;
}

// Builds the four operators; returns false on failure.
bool assemble(const lr_paper_params& p, std::vector<std::vector<Entry>>& ops, Derived& D) {
  if (!derive(p, D)) return false;
  const auto W = words(p, D);
  const int N = p.Nl * p.Nu * p.Nt;
  ops.assign(W.size(), {});
  for (size_t o = 0; o < W.size(); ++o) {
    std::vector<Entry>& E = ops[o];
    for (int c = 0; c < N; ++c) {
      const State s0{c / (p.Nu * p.Nt), (c / p.Nt) % p.Nu, c % p.Nt};
      for (const Word& w : W[o]) {
        State s = s0;
        double amp = 1.0;
        bool ok = true;
        for (int k = w.n - 1; k >= 0 && ok; --k) ok = apply_op(w.op[k], s, amp, p, D);
        if (!ok || amp == 0.0) continue;
        E.push_back(Entry{(s.l * p.Nu + s.u) * p.Nt + s.t, c, w.chan, w.coef * amp});
      }
    }
    std::sort(E.begin(), E.end(), [](const Entry& x, const Entry& y) {
      if (x.row != y.row) return x.row < y.row;
      if (x.col != y.col) return x.col < y.col;
      return x.ch < y.ch;
    });
    std::vector<Entry> merged;
    for (const Entry& e : E) {
      if (!merged.empty() && merged.back().row == e.row && merged.back().col == e.col && merged.back().ch == e.ch)
        merged.back().v += e.v;
      else
        merged.push_back(e);
    }
    E.clear();
    for (const Entry& e : merged)
      if (e.v != cd(0.0, 0.0)) E.push_back(e);
  }
  return true;
}

}  // namespace

extern "C" lr_status lr_paper_model_size(const lr_paper_params* p, int* N, long* nnz) {
  if (!params_ok(p) || !N || !nnz) return LR_ERR_ARG;
  std::vector<std::vector<Entry>> ops;
  Derived D;
  if (!assemble(*p, ops, D)) return LR_ERR_ARG;
  long tot = 0;
  for (const auto& E : ops) tot += (long)E.size();
  *N = p->Nl * p->Nu * p->Nt;
  *nnz = tot;
  return LR_OK;
}

extern "C" lr_status lr_paper_model_build(const lr_paper_params* p, int* rowptr, int* col, double* val,
                                          unsigned char* chan_out, int* level, double* derived) {
  if (!params_ok(p) || !rowptr || !col || !val || !chan_out || !level) return LR_ERR_ARG;
  std::vector<std::vector<Entry>> ops;
  Derived D;
  if (!assemble(*p, ops, D)) return LR_ERR_ARG;
  const int N = p->Nl * p->Nu * p->Nt;
  long pos = 0;
  for (size_t o = 0; o < ops.size(); ++o) {
    int* rp = rowptr + o * (size_t)(N + 1);
    size_t e = 0;
    for (int n = 0; n <= N; ++n) {
      rp[n] = (int)(pos + e);
      while (n < N && e < ops[o].size() && ops[o][e].row == n) ++e;
    }
    for (const Entry& x : ops[o]) {
      col[pos] = x.col;
      val[2 * pos] = x.v.real();
      val[2 * pos + 1] = x.v.imag();
      chan_out[pos] = (unsigned char)x.ch;
      ++pos;
    }
  }
  for (int n = 0; n < N; ++n) level[n] = n % p->Nt;
  if (derived) {
    for (int i = 0; i < LR_PAPER_DERIVED; ++i) derived[i] = 0.0;
    const double v[10] = {D.wl, D.wu, D.mu_l, D.mu_u, D.nu_l, D.nu_u, D.s21, D.s22, D.s23, D.s24};
    for (int i = 0; i < 10; ++i) derived[i] = v[i];
    if (p->Nt >= 2) derived[10] = D.eps[1] - D.eps[0];
    if (p->Nt >= 3) derived[11] = D.eps[2] - 2.0 * D.eps[1] + D.eps[0];
  }
  return LR_OK;
}

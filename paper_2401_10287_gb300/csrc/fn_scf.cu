// Mulliken partial charges for Algorithm 1 (host code).
//
// Algorithm 1 decides the electrons per atom of an ion from partial charges, which the
// method takes from a Mulliken population analysis of a Hartree-Fock calculation in the
// STO-6G basis (pretraining paragraph and the LiH+ example of the ionic charge
// initialisation section).  This file computes them for molecules of H..Ne:
//   * basis: STO-6G (Hehre, Stewart & Pople, J. Chem. Phys. 51, 2657 (1969)): six
//     Gaussians per Slater shell, 2s and 2p sharing exponents, scaled by zeta^2 with the
//     standard molecular exponents of each element;
//   * integrals over contracted Cartesian s and p Gaussians by the Obara-Saika
//     recurrences (overlap, kinetic energy, nuclear attraction, and the two-electron
//     vertical recurrence on all four centres);
//   * unrestricted Hartree-Fock: symmetric orthogonalisation; six starts (core Hamiltonian,
//     generalised Wolfsberg-Helmholz, four symmetric perturbations of the core Hamiltonian), damped
//     iterations then DIIS on both spins, the lowest converged energy kept; Jacobi diagonalisation;
//   * q_A = Z_A - sum over the functions mu on A of (P S)_mu,mu, P = P_alpha + P_beta.
// A diatomic takes milliseconds; the computation is set-up for the sampler, not part of
// the per-walker path, and runs once per molecule.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "fn_internal.cuh"

namespace fn {
namespace scf {

// STO-6G expansions of the Slater functions with exponent 1; coefficients multiply
// normalised primitives.
constexpr double kExp1s[6] = {23.10303149, 4.235915534, 1.185056519, 0.4070988982, 0.1580884151, 0.06510953954};
constexpr double kCoef1s[6] = {0.009163596281, 0.04936149294, 0.1685383049, 0.3705627997, 0.4164915298,
                               0.1303340841};
constexpr double kExp2sp[6] = {10.30869372, 2.040359519, 0.6341422097, 0.2439773411, 0.1059595374, 0.04856900860};
constexpr double kCoef2s[6] = {-0.01325278809, -0.04699171014, -0.03378537151, 0.2502417861, 0.5951172526,
                               0.2407061763};
constexpr double kCoef2p[6] = {0.003759696623, 0.03767936984, 0.1738967435, 0.4180364347, 0.4258595477,
                               0.1017082955};
// Standard molecular Slater exponents (1s, 2sp) of H..Ne.
constexpr double kZeta1s[11] = {0, 1.24, 1.69, 2.69, 3.68, 4.68, 5.67, 6.67, 7.66, 8.65, 9.64};
constexpr double kZeta2sp[11] = {0, 0, 0, 0.80, 1.15, 1.50, 1.72, 1.95, 2.25, 2.55, 2.88};

constexpr double kPi = 3.14159265358979323846;
// The two-electron integrals cost n^4 / 8 contracted quartets of 6^4 primitives each.
constexpr int kMaxBasis = 20;

struct Shell {        // one contracted Cartesian function
  double c[3];
  int l[3];
  double a[6], w[6];  // exponents and weights (contraction coefficient x primitive norm)
  int atom;
};

// Boys function F_m(T), m = 0..mmax: the series for F_mmax (any T below 40) and downward
// recursion F_m = (2T F_(m+1) + e^-T) / (2m + 1); above T = 40 the asymptotic form with
// upward recursion (e^-T < 5e-18 is dropped).
static void boys(int mmax, double T, double* F) {
  if (T < 1e-14) {
    for (int m = 0; m <= mmax; ++m) F[m] = 1.0 / (2 * m + 1);
    return;
  }
  if (T > 40.0) {
    F[0] = 0.5 * std::sqrt(kPi / T);
    for (int m = 0; m < mmax; ++m) F[m + 1] = (2 * m + 1) / (2 * T) * F[m];
    return;
  }
  double term = 1.0 / (2 * mmax + 1), sum = term;
  for (int k = 1; k < 400; ++k) {
    term *= 2 * T / (2 * mmax + 2 * k + 1);
    sum += term;
    if (term < 1e-17 * sum) break;
  }
  const double et = std::exp(-T);
  F[mmax] = et * sum;
  for (int m = mmax - 1; m >= 0; --m) F[m] = (2 * T * F[m + 1] + et) / (2 * m + 1);
}

static double prim_norm(double a, const int* l) {
  const int L = l[0] + l[1] + l[2];   // s or p: (2l - 1)!! = 1
  return std::pow(2 * a / kPi, 0.75) * std::pow(4 * a, 0.5 * L);
}

// One Cartesian direction of a primitive pair with powers i, j <= 1 (Obara-Saika): the
// overlap factor S_ij and the kinetic-energy factor T_ij.
static void os_1d(int i, int j, double a, double b, double PA, double PB, double XAB, double* S_out, double* T_out) {
  const double p = a + b, mu = a * b / p;
  double S[2][2] = {}, T[2][2] = {};
  S[0][0] = std::sqrt(kPi / p) * std::exp(-mu * XAB * XAB);
  for (int ii = 0; ii <= i; ++ii)
    for (int jj = 0; jj <= j; ++jj) {
      if (ii == 0 && jj == 0) continue;
      if (ii > 0) {
        const int u = ii - 1;
        S[ii][jj] = PA * S[u][jj] + (1 / (2 * p)) * ((u > 0 ? u * S[u - 1][jj] : 0) + (jj > 0 ? jj * S[u][jj - 1] : 0));
      } else {
        const int v = jj - 1;
        S[ii][jj] = PB * S[ii][v] + (1 / (2 * p)) * (v > 0 ? v * S[ii][v - 1] : 0);
      }
    }
  T[0][0] = (a - 2 * a * a * (PA * PA + 1 / (2 * p))) * S[0][0];
  for (int ii = 0; ii <= i; ++ii)
    for (int jj = 0; jj <= j; ++jj) {
      if (ii == 0 && jj == 0) continue;
      if (ii > 0) {
        const int u = ii - 1;
        T[ii][jj] = PA * T[u][jj] + (1 / (2 * p)) * ((u > 0 ? u * T[u - 1][jj] : 0) + (jj > 0 ? jj * T[u][jj - 1] : 0)) +
                    (b / p) * (2 * a * S[ii][jj] - (u > 0 ? u * S[u - 1][jj] : 0));
      } else {
        const int v = jj - 1;
        T[ii][jj] = PB * T[ii][v] + (1 / (2 * p)) * (v > 0 ? v * T[ii][v - 1] : 0) +
                    (a / p) * (2 * b * S[ii][jj] - (v > 0 ? v * S[ii][v - 1] : 0));
      }
    }
  *S_out = S[i][j];
  *T_out = T[i][j];
}

static void one_electron(const Shell& f, const Shell& g, double* s_out, double* t_out) {
  double s = 0, t = 0;
  for (int x = 0; x < 6; ++x)
    for (int y = 0; y < 6; ++y) {
      const double a = f.a[x], b = g.a[y], p = a + b;
      double Sd[3], Td[3];
      for (int d = 0; d < 3; ++d) {
        const double P = (a * f.c[d] + b * g.c[d]) / p;
        os_1d(f.l[d], g.l[d], a, b, P - f.c[d], P - g.c[d], f.c[d] - g.c[d], &Sd[d], &Td[d]);
      }
      const double w = f.w[x] * g.w[y];
      s += w * Sd[0] * Sd[1] * Sd[2];
      t += w * (Td[0] * Sd[1] * Sd[2] + Sd[0] * Td[1] * Sd[2] + Sd[0] * Sd[1] * Td[2]);
    }
  *s_out = s;
  *t_out = t;
}

static int axis_of(const int* l) { return l[0] ? 0 : (l[1] ? 1 : (l[2] ? 2 : -1)); }

// <f| 1/|r - C| |g> for s and p functions (Obara-Saika with the auxiliary index m).
static double nuclear(const Shell& f, const Shell& g, const double* C) {
  const int i = axis_of(f.l), j = axis_of(g.l);
  double tot = 0;
  for (int x = 0; x < 6; ++x)
    for (int y = 0; y < 6; ++y) {
      const double a = f.a[x], b = g.a[y], p = a + b, mu = a * b / p;
      double P[3], AB2 = 0, PC2 = 0;
      for (int d = 0; d < 3; ++d) {
        P[d] = (a * f.c[d] + b * g.c[d]) / p;
        AB2 += (f.c[d] - g.c[d]) * (f.c[d] - g.c[d]);
        PC2 += (P[d] - C[d]) * (P[d] - C[d]);
      }
      double F[3];
      boys(2, p * PC2, F);
      const double k = 2 * kPi / p * std::exp(-mu * AB2);
      double ss[3];
      for (int m = 0; m < 3; ++m) ss[m] = k * F[m];
      double v;
      if (i < 0 && j < 0) {
        v = ss[0];
      } else if (j < 0) {
        v = (P[i] - f.c[i]) * ss[0] - (P[i] - C[i]) * ss[1];
      } else if (i < 0) {
        v = (P[j] - g.c[j]) * ss[0] - (P[j] - C[j]) * ss[1];
      } else {
        const double ps0 = (P[i] - f.c[i]) * ss[0] - (P[i] - C[i]) * ss[1];
        const double ps1 = (P[i] - f.c[i]) * ss[1] - (P[i] - C[i]) * ss[2];
        v = (P[j] - g.c[j]) * ps0 - (P[j] - C[j]) * ps1 + (i == j ? (ss[0] - ss[1]) / (2 * p) : 0.0);
      }
      tot += f.w[x] * g.w[y] * v;
    }
  return tot;
}

// Two-electron primitives [ab|cd]^(m) by the Obara-Saika vertical recurrence applied to
// the first function of the quartet that still carries angular momentum.
struct Quartet {
  double p, q, rho;
  double PA[3], PB[3], QC[3], QD[3], WP[3], WQ[3];
  double F[5], base;
};

static double vrr(const Quartet& Q, int la[3], int lb[3], int lc[3], int ld[3], int m) {
  int* L[4] = {la, lb, lc, ld};
  for (int s = 0; s < 4; ++s)
    for (int d = 0; d < 3; ++d) {
      if (L[s][d] == 0) continue;
      L[s][d] -= 1;   // reduce function s along axis d; the others keep their momentum
      const bool bra = s < 2;
      const double X = bra ? (s == 0 ? Q.PA[d] : Q.PB[d]) : (s == 2 ? Q.QC[d] : Q.QD[d]);
      const double W = bra ? Q.WP[d] : Q.WQ[d];
      const double z = bra ? Q.p : Q.q;
      double v = X * vrr(Q, la, lb, lc, ld, m) + W * vrr(Q, la, lb, lc, ld, m + 1);
      // same-side partners: this function itself and the other function of its pair
      const int same[2] = {s, bra ? 1 - s : 5 - s};
      const int opposite[2] = {bra ? 2 : 0, bra ? 3 : 1};
      for (int t : same) {
        const int n = L[t][d];
        if (n > 0) {
          L[t][d] -= 1;
          v += n / (2 * z) * (vrr(Q, la, lb, lc, ld, m) - Q.rho / z * vrr(Q, la, lb, lc, ld, m + 1));
          L[t][d] += 1;
        }
      }
      // opposite-side functions
      for (int t : opposite) {
        const int n = L[t][d];
        if (n > 0) {
          L[t][d] -= 1;
          v += n / (2 * (Q.p + Q.q)) * vrr(Q, la, lb, lc, ld, m + 1);
          L[t][d] += 1;
        }
      }
      L[s][d] += 1;
      return v;
    }
  return Q.base * Q.F[m];
}

static double eri(const Shell& f, const Shell& g, const Shell& h, const Shell& k) {
  double tot = 0;
  for (int x = 0; x < 6; ++x)
    for (int y = 0; y < 6; ++y) {
      const double a = f.a[x], b = g.a[y], p = a + b;
      double P[3], AB2 = 0;
      for (int d = 0; d < 3; ++d) {
        P[d] = (a * f.c[d] + b * g.c[d]) / p;
        AB2 += (f.c[d] - g.c[d]) * (f.c[d] - g.c[d]);
      }
      const double kab = std::exp(-a * b / p * AB2), wab = f.w[x] * g.w[y];
      for (int z = 0; z < 6; ++z)
        for (int u = 0; u < 6; ++u) {
          const double c = h.a[z], d2 = k.a[u], q = c + d2;
          Quartet Q;
          double Qc[3], CD2 = 0, PQ2 = 0;
          for (int d = 0; d < 3; ++d) {
            Qc[d] = (c * h.c[d] + d2 * k.c[d]) / q;
            CD2 += (h.c[d] - k.c[d]) * (h.c[d] - k.c[d]);
            PQ2 += (P[d] - Qc[d]) * (P[d] - Qc[d]);
          }
          Q.p = p;
          Q.q = q;
          Q.rho = p * q / (p + q);
          for (int d = 0; d < 3; ++d) {
            const double W = (p * P[d] + q * Qc[d]) / (p + q);
            Q.PA[d] = P[d] - f.c[d];
            Q.PB[d] = P[d] - g.c[d];
            Q.QC[d] = Qc[d] - h.c[d];
            Q.QD[d] = Qc[d] - k.c[d];
            Q.WP[d] = W - P[d];
            Q.WQ[d] = W - Qc[d];
          }
          boys(4, Q.rho * PQ2, Q.F);
          Q.base = 2 * std::pow(kPi, 2.5) / (p * q * std::sqrt(p + q)) * kab * std::exp(-c * d2 / q * CD2);
          int la[3] = {f.l[0], f.l[1], f.l[2]}, lb[3] = {g.l[0], g.l[1], g.l[2]};
          int lc[3] = {h.l[0], h.l[1], h.l[2]}, ld[3] = {k.l[0], k.l[1], k.l[2]};
          tot += wab * h.w[z] * k.w[u] * vrr(Q, la, lb, lc, ld, 0);
        }
    }
  return tot;
}

// Jacobi eigen-decomposition of a symmetric n x n matrix (row-major); eigenvalues ascending,
// eigenvectors in the columns of V.
static void jacobi(int n, std::vector<double> A, std::vector<double>* evals, std::vector<double>* V) {
  V->assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) (*V)[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
    if (off < 1e-30) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1));
        const double c = 1 / std::sqrt(t * t + 1), s = t * c;
        for (int k = 0; k < n; ++k) {   // columns p, q
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {   // rows p, q
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = (*V)[(size_t)k * n + p], vkq = (*V)[(size_t)k * n + q];
          (*V)[(size_t)k * n + p] = c * vkp - s * vkq;
          (*V)[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  for (int i = 0; i < n; ++i)   // selection sort by eigenvalue
    for (int j = i + 1; j < n; ++j)
      if (A[(size_t)order[j] * n + order[j]] < A[(size_t)order[i] * n + order[i]]) std::swap(order[i], order[j]);
  evals->resize(n);
  std::vector<double> Vs((size_t)n * n);
  for (int c = 0; c < n; ++c) {
    (*evals)[c] = A[(size_t)order[c] * n + order[c]];
    for (int r = 0; r < n; ++r) Vs[(size_t)r * n + c] = (*V)[(size_t)r * n + order[c]];
  }
  *V = Vs;
}

using Mat = std::vector<double>;

static Mat matmul(int n, const Mat& A, const Mat& B, bool ta = false) {
  Mat C((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      const double aik = ta ? A[(size_t)k * n + i] : A[(size_t)i * n + k];
      for (int j = 0; j < n; ++j) C[(size_t)i * n + j] += aik * B[(size_t)k * n + j];
    }
  return C;
}

// Density of the n_occ lowest orbitals of F in the orthogonalised basis X.
static Mat density(int n, const Mat& F, const Mat& X, int n_occ) {
  const Mat Fp = matmul(n, matmul(n, X, F, true), X);
  std::vector<double> e;
  Mat Cp;
  jacobi(n, Fp, &e, &Cp);
  const Mat C = matmul(n, X, Cp);
  Mat P((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int o = 0; o < n_occ; ++o) P[(size_t)i * n + j] += C[(size_t)i * n + o] * C[(size_t)j * n + o];
  return P;
}

// Solves the (m+1) x (m+1) DIIS system by Gaussian elimination with partial pivoting.
static bool solve(int n, std::vector<double> A, std::vector<double> b, std::vector<double>* x) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
    if (std::fabs(A[(size_t)piv * n + c]) < 1e-300) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; ++r) {
      const double f = A[(size_t)r * n + c] / A[(size_t)c * n + c];
      for (int k = c; k < n; ++k) A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
      b[r] -= f * b[c];
    }
  }
  x->assign(n, 0.0);
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int k = r + 1; k < n; ++k) s -= A[(size_t)r * n + k] * (*x)[k];
    (*x)[r] = s / A[(size_t)r * n + r];
  }
  return true;
}

// UHF iterations from the starting Fock matrix F0: kDampIters damped steps (P <- (P + P_new) / 2),
// then DIIS on both spins.  Returns false if not converged in 500 iterations; on success the
// energy and the total density P_alpha + P_beta.
constexpr int kDampIters = 30;

static bool scf_from(const Mat& F0, int n, const Mat& S, const Mat& H, const std::vector<double>& G, const Mat& X,
                     int n_a, int n_b, double e_nn, double* e_out, Mat* P_out, Mat* Fa_out = nullptr,
                     Mat* Fb_out = nullptr) {
  const size_t n2 = (size_t)n * n;
  Mat Pa = density(n, F0, X, n_a), Pb = density(n, F0, X, n_b);
  std::vector<Mat> hF_a, hF_b, hErr;
  double e_old = 0;
  for (int it = 0; it < 500; ++it) {
    Mat Fa = H, Fb = H;
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q) {
        double J = 0, Ka = 0, Kb = 0;
        for (int r = 0; r < n; ++r)
          for (int s = 0; s < n; ++s) {
            const double prs = Pa[(size_t)r * n + s] + Pb[(size_t)r * n + s];
            J += G[(((size_t)p * n + q) * n + r) * n + s] * prs;
            const double x = G[(((size_t)p * n + r) * n + q) * n + s];
            Ka += x * Pa[(size_t)r * n + s];
            Kb += x * Pb[(size_t)r * n + s];
          }
        Fa[(size_t)p * n + q] += J - Ka;
        Fb[(size_t)p * n + q] += J - Kb;
      }
    double e = e_nn;
    for (size_t k = 0; k < n2; ++k) e += 0.5 * ((H[k] + Fa[k]) * Pa[k] + (H[k] + Fb[k]) * Pb[k]);
    // DIIS error F P S - S P F for both spins
    const Mat FPSa = matmul(n, matmul(n, Fa, Pa), S), FPSb = matmul(n, matmul(n, Fb, Pb), S);
    Mat err(2 * n2);
    double emax = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        err[(size_t)i * n + j] = FPSa[(size_t)i * n + j] - FPSa[(size_t)j * n + i];
        err[n2 + (size_t)i * n + j] = FPSb[(size_t)i * n + j] - FPSb[(size_t)j * n + i];
      }
    for (double v : err) emax = std::max(emax, std::fabs(v));
    if (it > 0 && std::fabs(e - e_old) < 1e-11 && emax < 1e-8) {
      P_out->assign(n2, 0.0);
      for (size_t k = 0; k < n2; ++k) (*P_out)[k] = Pa[k] + Pb[k];
      *e_out = e;
      if (Fa_out) *Fa_out = Fa;
      if (Fb_out) *Fb_out = Fb;
      return true;
    }
    e_old = e;
    if (it < kDampIters) {
      const Mat Na = density(n, Fa, X, n_a), Nb = density(n, Fb, X, n_b);
      for (size_t k = 0; k < n2; ++k) {
        Pa[k] = 0.5 * (Pa[k] + Na[k]);
        Pb[k] = 0.5 * (Pb[k] + Nb[k]);
      }
      continue;
    }
    hF_a.push_back(Fa);
    hF_b.push_back(Fb);
    hErr.push_back(err);
    if (hErr.size() > 8) {
      hF_a.erase(hF_a.begin());
      hF_b.erase(hF_b.begin());
      hErr.erase(hErr.begin());
    }
    const int m = (int)hErr.size();
    std::vector<double> Bm((size_t)(m + 1) * (m + 1), -1.0), rhs(m + 1, 0.0), c;
    Bm[(size_t)m * (m + 1) + m] = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        double d = 0;
        for (size_t k = 0; k < 2 * n2; ++k) d += hErr[i][k] * hErr[j][k];
        Bm[(size_t)i * (m + 1) + j] = d;
      }
    rhs[m] = -1.0;
    Mat Fa_x(n2, 0.0), Fb_x(n2, 0.0);
    if (solve(m + 1, Bm, rhs, &c)) {
      for (int i = 0; i < m; ++i)
        for (size_t k = 0; k < n2; ++k) {
          Fa_x[k] += c[i] * hF_a[i][k];
          Fb_x[k] += c[i] * hF_b[i][k];
        }
    } else {
      Fa_x = Fa;
      Fb_x = Fb;
    }
    Pa = density(n, Fa_x, X, n_a);
    Pb = density(n, Fb_x, X, n_b);
  }
  return false;
}

// Occupied UHF orbitals of the converged state (the targets of the Eq. 5 pretraining loss):
// the eigenvectors of each spin's Fock matrix in the orthogonalised basis, the n_occ lowest in
// order of orbital energy, back-transformed (C = X C'), each signed so that its
// largest-magnitude coefficient is positive.
struct HfOrbitals {
  std::vector<Shell> basis;
  Mat C[2];              // [nbf][n_occ] per spin
  int n_occ[2] = {0, 0};
  double energy = 0;
};

static bool occupied_orbitals(int n, const Mat& F, const Mat& X, int n_occ, Mat* C_out) {
  const Mat Fp = matmul(n, matmul(n, X, F, true), X);
  std::vector<double> e;
  Mat Cp;
  jacobi(n, Fp, &e, &Cp);
  const Mat C = matmul(n, X, Cp);
  // a degenerate highest occupied level, or degenerate occupied levels, make the target not unique
  if (n_occ > 0 && n_occ < n && std::fabs(e[n_occ] - e[n_occ - 1]) < 1e-8) return false;
  for (int o = 1; o < n_occ; ++o)
    if (std::fabs(e[o] - e[o - 1]) < 1e-8) return false;
  C_out->assign((size_t)n * n_occ, 0.0);
  for (int o = 0; o < n_occ; ++o) {
    int big = 0;
    for (int mu = 1; mu < n; ++mu)
      if (std::fabs(C[(size_t)mu * n + o]) > std::fabs(C[(size_t)big * n + o])) big = mu;
    const double sg = C[(size_t)big * n + o] < 0 ? -1.0 : 1.0;
    for (int mu = 0; mu < n; ++mu) (*C_out)[(size_t)mu * n_occ + o] = sg * C[(size_t)mu * n + o];
  }
  return true;
}

static fn_status run(const double* nuc, const double* Z, int M, int n_a, int n_b, double* q_out, double* e_out,
                     HfOrbitals* orb = nullptr) {
  std::vector<Shell> bas;
  for (int A = 0; A < M; ++A) {
    const int z = (int)std::lround(Z[A]);
    auto add = [&](const double* ex, const double* co, double zeta, int lx, int ly, int lz) {
      Shell s{};
      for (int d = 0; d < 3; ++d) s.c[d] = nuc[3 * A + d];
      s.l[0] = lx; s.l[1] = ly; s.l[2] = lz;
      for (int k = 0; k < 6; ++k) {
        s.a[k] = ex[k] * zeta * zeta;
        s.w[k] = co[k] * prim_norm(s.a[k], s.l);
      }
      s.atom = A;
      bas.push_back(s);
    };
    add(kExp1s, kCoef1s, kZeta1s[z], 0, 0, 0);
    if (z >= 3) {
      add(kExp2sp, kCoef2s, kZeta2sp[z], 0, 0, 0);
      add(kExp2sp, kCoef2p, kZeta2sp[z], 1, 0, 0);
      add(kExp2sp, kCoef2p, kZeta2sp[z], 0, 1, 0);
      add(kExp2sp, kCoef2p, kZeta2sp[z], 0, 0, 1);
    }
  }
  const int n = (int)bas.size();
  if (n > kMaxBasis) {
    set_error("at most " + std::to_string(kMaxBasis) + " STO-6G functions (four first-row atoms)");
    return FN_ERR_UNSUPPORTED;
  }
  if (n_a > n || n_b > n) { set_error("more electrons of a spin than STO-6G functions"); return FN_ERR_ARG; }
  for (Shell& s : bas) {   // normalise each contraction
    double ss, tt;
    one_electron(s, s, &ss, &tt);
    for (int k = 0; k < 6; ++k) s.w[k] /= std::sqrt(ss);
  }
  Mat S((size_t)n * n), H((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s, t;
      one_electron(bas[i], bas[j], &s, &t);
      double v = 0;
      for (int A = 0; A < M; ++A) v -= Z[A] * nuclear(bas[i], bas[j], nuc + 3 * A);
      S[(size_t)i * n + j] = s;
      H[(size_t)i * n + j] = t + v;
    }
  const size_t n2 = (size_t)n * n;
  std::vector<double> G(n2 * n2);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j)
      for (int k = 0; k < n; ++k)
        for (int l = 0; l <= k; ++l) {
          if (i * (i + 1) / 2 + j < k * (k + 1) / 2 + l) continue;
          const double x = eri(bas[i], bas[j], bas[k], bas[l]);
          const int idx[8][4] = {{i, j, k, l}, {j, i, k, l}, {i, j, l, k}, {j, i, l, k},
                                 {k, l, i, j}, {l, k, i, j}, {k, l, j, i}, {l, k, j, i}};
          for (auto& t : idx) G[(((size_t)t[0] * n + t[1]) * n + t[2]) * n + t[3]] = x;
        }
  double e_nn = 0;
  for (int A = 0; A < M; ++A)
    for (int B = 0; B < A; ++B) {
      double r2 = 0;
      for (int d = 0; d < 3; ++d) r2 += (nuc[3 * A + d] - nuc[3 * B + d]) * (nuc[3 * A + d] - nuc[3 * B + d]);
      if (!(r2 > 1e-12)) { set_error("two nuclei at the same position"); return FN_ERR_ARG; }
      e_nn += Z[A] * Z[B] / std::sqrt(r2);
    }
  // X = S^(-1/2)
  std::vector<double> s_ev;
  Mat U;
  jacobi(n, S, &s_ev, &U);
  Mat X(n2, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) X[(size_t)i * n + j] += U[(size_t)i * n + k] * U[(size_t)j * n + k] / std::sqrt(s_ev[k]);
  // Starts: the core Hamiltonian and the generalised Wolfsberg-Helmholz guess (k = 1.75), each
  // with damped iterations before DIIS (DIIS from the first iteration can settle on an excited
  // self-consistent solution).  The lowest converged energy is the ground state kept.
  Mat gwh(n2);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      gwh[(size_t)i * n + j] = i == j ? H[(size_t)i * n + i]
                                      : 1.75 * S[(size_t)i * n + j] * 0.5 * (H[(size_t)i * n + i] + H[(size_t)j * n + j]);
  // Open shells with degenerate levels have several self-consistent solutions: four more starts
  // perturb the core Hamiltonian symmetrically (0.3 x (R + R^T), R uniform in [-1, 1) from a
  // 64-bit linear congruential generator with a fixed seed) to break the symmetry.
  std::vector<Mat> starts = {H, gwh};
  uint64_t state = 0x9E3779B97F4A7C15ull;
  auto uniform = [&state]() {
    state = state * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(state >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  };
  for (int k = 0; k < 16; ++k) {
    Mat R(n2), F0 = H;
    for (size_t i = 0; i < n2; ++i) R[i] = uniform();
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) F0[(size_t)i * n + j] += 0.3 * (R[(size_t)i * n + j] + R[(size_t)j * n + i]);
    starts.push_back(F0);
  }
  bool found = false;
  double e_best = 0;
  Mat P_best, Fa_best, Fb_best;
  for (const Mat& F0 : starts) {
    double e;
    Mat P, Fa, Fb;
    if (scf_from(F0, n, S, H, G, X, n_a, n_b, e_nn, &e, &P, &Fa, &Fb) && (!found || e < e_best - 1e-9)) {
      found = true;
      e_best = e;
      P_best = P;
      Fa_best = Fa;
      Fb_best = Fb;
    }
  }
  if (!found) {
    set_error("Hartree-Fock did not converge in 500 iterations");
    return FN_ERR_NUMERIC;
  }
  if (q_out) {
    const Mat PS = matmul(n, P_best, S);
    for (int A = 0; A < M; ++A) q_out[A] = Z[A];
    for (int mu = 0; mu < n; ++mu) q_out[bas[mu].atom] -= PS[(size_t)mu * n + mu];
  }
  if (e_out) *e_out = e_best;
  if (orb) {
    orb->basis = bas;
    orb->energy = e_best;
    orb->n_occ[0] = n_a;
    orb->n_occ[1] = n_b;
    if (!occupied_orbitals(n, Fa_best, X, n_a, &orb->C[0]) || !occupied_orbitals(n, Fb_best, X, n_b, &orb->C[1])) {
      set_error("degenerate occupied Hartree-Fock levels: the pretraining target is not unique");
      return FN_ERR_UNSUPPORTED;
    }
  }
  return FN_OK;
}

// Uploads the UHF state of the system (STO-6G, the system's own n_up / n_down) for the Eq. 5
// pretraining loss: per basis function 18 doubles (centre, Cartesian powers, six exponents,
// six weights), then C_up [nbf][n_up] and C_down [nbf][n_down].
fn_status upload_hf_state(fn_system* s, double* e_out) {
  for (int m = 0; m < s->M; ++m) {
    const double z = s->charges[m];
    if (!(z >= 1.0 && z <= 10.0)) {
      set_error("STO-6G Hartree-Fock is provided for H..Ne (integer Z from 1 to 10)");
      return FN_ERR_ARG;
    }
  }
  HfOrbitals orb;
  fn_status st = run(s->nuclei.data(), s->charges.data(), s->M, s->n_up, s->n_dn, nullptr, e_out, &orb);
  if (st != FN_OK) return st;
  const int nbf = (int)orb.basis.size();
  std::vector<double> buf;
  for (const Shell& f : orb.basis) {
    for (int d = 0; d < 3; ++d) buf.push_back(f.c[d]);
    for (int d = 0; d < 3; ++d) buf.push_back((double)f.l[d]);
    for (int k = 0; k < 6; ++k) buf.push_back(f.a[k]);
    for (int k = 0; k < 6; ++k) buf.push_back(f.w[k]);
  }
  for (int q = 0; q < 2; ++q) buf.insert(buf.end(), orb.C[q].begin(), orb.C[q].end());
  if (s->d_hf) {
    cudaFreeAsync(s->d_hf, cudaStreamPerThread);
    s->d_hf = nullptr;
  }
  cudaError_t e = cudaMallocAsync(&s->d_hf, sizeof(double) * buf.size(), cudaStreamPerThread);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_hf, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice, cudaStreamPerThread);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamPerThread);
  if (e != cudaSuccess) return cuda_status(e, "Hartree-Fock state upload");
  s->hf_nbf = nbf;
  return FN_OK;
}

}  // namespace scf

fn_status upload_hf_state(fn_system* s, double* e_out) { return scf::upload_hf_state(s, e_out); }

}  // namespace fn

extern "C" fn_status fn_mulliken_charges(const double* h_nuclei, const double* h_charges, int n_nuclei, int n_up,
                                         int n_down, double* h_partial_charges, double* h_energy) {
  using namespace fn;
  if (!h_nuclei || !h_charges || !h_partial_charges || n_nuclei < 1 || n_nuclei > kMaxNuclei || n_up < 0 ||
      n_down < 0 || n_up + n_down == 0) {
    set_error("invalid argument");
    return FN_ERR_ARG;
  }
  for (int m = 0; m < n_nuclei; ++m) {
    const double z = h_charges[m];
    if (!(z >= 1.0 && z <= 10.0) || std::fabs(z - std::round(z)) > 1e-12) {
      set_error("STO-6G charges are provided for H..Ne (integer Z from 1 to 10)");
      return FN_ERR_ARG;
    }
  }
  return scf::run(h_nuclei, h_charges, n_nuclei, std::max(n_up, n_down), std::min(n_up, n_down), h_partial_charges,
                  h_energy);
}

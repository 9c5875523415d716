// Host-side construction of the 1D expansion bases of Sec. 2 and their
// tables at Gauss-Legendre points.  Float64 throughout.
//
// Steps, in the order of Sec. 2:
//   * standard basis psi: Lagrange polynomials on the P+1 Gauss-Lobatto-
//     Legendre points (eqs. lagrangian, shape_functions_lag), evaluated in
//     barycentric form, or the Jacobi modal basis (eq. BasePadrao1D);
//   * 1D mass and stiffness (eqs. Matrizesmassa, Matrizesrigidez) by
//     Gauss-Legendre quadrature with P+2 points (exact for degree 2P);
//   * vertex/internal blocks (eq. BlocosMassa);
//   * simultaneous diagonalisation of the internal block (eqs. diagMassa, L,
//     diagL, Y) with a cyclic Jacobi symmetric eigensolver;
//   * minimum-energy vertex modes (eq. ExtensaoMEmassa) with
//     alpha = G_vi G_ii^{-1}, G = M, K or K + lambda M (eqs. alphaMassa,
//     alphaRigidez, alphaKN).
// Each SD internal function is signed so that its derivative at -1 is
// positive, and internal functions are ordered by ascending eigenvalue of L;
// this fixes the eigenvectors' free signs independently of the solver.
#include "basis1d.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace sdme {
namespace {

constexpr double kPi = 3.14159265358979323846;

// Legendre polynomial L_m(x) and its derivative by the Bonnet recurrence.
void legendre(int m, double x, double* Lm, double* dLm) {
  double p0 = 1.0, p1 = x;
  if (m == 0) { *Lm = 1.0; *dLm = 0.0; return; }
  for (int k = 2; k <= m; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *Lm = p1;
  // (1 - x^2) L_m' = m (L_{m-1} - x L_m)
  double den = 1.0 - x * x;
  *dLm = (den != 0.0) ? m * (p0 - x * p1) / den : 0.5 * m * (m + 1) * (x > 0 ? 1.0 : (m % 2 ? 1.0 : -1.0));
}

// Jacobi P_m^{a,b}(x) by the three-term recurrence, and its derivative
// d/dx P_m^{a,b} = (m + a + b + 1)/2 P_{m-1}^{a+1,b+1}.
double jacobi(int m, double a, double b, double x) {
  if (m == 0) return 1.0;
  double p0 = 1.0;
  double p1 = 0.5 * ((a + b + 2.0) * x + (a - b));
  for (int k = 1; k < m; ++k) {
    double s = 2.0 * k + a + b;
    double c1 = 2.0 * (k + 1) * (k + a + b + 1) * s;
    double c2 = (s + 1.0) * ((s + 2.0) * s * x + a * a - b * b);
    double c3 = 2.0 * (k + a) * (k + b) * (s + 2.0);
    double p2 = (c2 * p1 - c3 * p0) / c1;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

double jacobi_d(int m, double a, double b, double x) {
  if (m == 0) return 0.0;
  return 0.5 * (m + a + b + 1.0) * jacobi(m - 1, a + 1.0, b + 1.0, x);
}

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (row-major).
// On return A holds nothing useful, w the eigenvalues ascending and V the
// eigenvectors as columns (V[i*n + j] = component i of vector j).
void sym_eig(int n, std::vector<double> A, std::vector<double>& w, std::vector<double>& V) {
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) (i == j ? diag : off) += A[i * n + j] * A[i * n + j];
    if (off <= 1e-32 * diag || off == 0.0) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (apq == 0.0) continue;
        double app = A[p * n + p], aqq = A[q * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
  // ascending order
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return w[a] < w[b]; });
  std::vector<double> w2(n), V2(n * n);
  for (int j = 0; j < n; ++j) {
    w2[j] = w[idx[j]];
    for (int i = 0; i < n; ++i) V2[i * n + j] = V[i * n + idx[j]];
  }
  w = w2;
  V = V2;
}

// Solve the small dense system A X = Bm (A m x m, Bm m x r) by Gaussian
// elimination with partial pivoting.  Row-major; result in Bm.
bool dense_solve(int m, int r, std::vector<double> A, std::vector<double>& Bm) {
  for (int col = 0; col < m; ++col) {
    int piv = col;
    for (int i = col + 1; i < m; ++i)
      if (std::fabs(A[i * m + col]) > std::fabs(A[piv * m + col])) piv = i;
    if (A[piv * m + col] == 0.0) return false;
    if (piv != col) {
      for (int k = 0; k < m; ++k) std::swap(A[col * m + k], A[piv * m + k]);
      for (int k = 0; k < r; ++k) std::swap(Bm[col * r + k], Bm[piv * r + k]);
    }
    for (int i = col + 1; i < m; ++i) {
      double f = A[i * m + col] / A[col * m + col];
      for (int k = col; k < m; ++k) A[i * m + k] -= f * A[col * m + k];
      for (int k = 0; k < r; ++k) Bm[i * r + k] -= f * Bm[col * r + k];
    }
  }
  for (int i = m - 1; i >= 0; --i) {
    for (int k = 0; k < r; ++k) {
      double s = Bm[i * r + k];
      for (int j = i + 1; j < m; ++j) s -= A[i * m + j] * Bm[j * r + k];
      Bm[i * r + k] = s / A[i * m + i];
    }
  }
  return true;
}

}  // namespace

void gauss_legendre(int Q, double* x, double* w) {
  // Newton iteration on L_Q from the Chebyshev-like initial guesses.
  for (int i = 0; i < Q; ++i) {
    double z = -std::cos(kPi * (i + 0.75) / (Q + 0.5));
    double L = 0.0, dL = 0.0;
    for (int it = 0; it < 100; ++it) {
      legendre(Q, z, &L, &dL);
      double dz = L / dL;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    legendre(Q, z, &L, &dL);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dL * dL);
  }
}

void gauss_lobatto_legendre(int P, double* x) {
  // End points and the P-1 roots of L_P' found by Newton on L_P'.  With
  // f = L_P', (1 - z^2) f' = 2 z f - P (P + 1) L_P.
  x[0] = -1.0;
  x[P] = 1.0;
  for (int i = 1; i < P; ++i) {
    double z = -std::cos(kPi * i / P);
    for (int it = 0; it < 100; ++it) {
      double L, dL;
      legendre(P, z, &L, &dL);
      double d2L = (2.0 * z * dL - P * (P + 1.0) * L) / (1.0 - z * z);
      double dz = dL / d2L;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
}

// Barycentric Lagrange evaluation: values and derivatives of all n basis
// polynomials through nodes xn at point x.
void lagrange_eval(int n, const double* xn, double x, double* val, double* der) {
  std::vector<double> wb(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) wb[j] /= (xn[j] - xn[k]);
  for (int j = 0; j < n; ++j) {
    if (x == xn[j]) {
      for (int a = 0; a < n; ++a) val[a] = (a == j) ? 1.0 : 0.0;
      // derivative at a node: l_a'(x_j) = (w_a / w_j) / (x_j - x_a), a != j;
      // l_j'(x_j) = -sum of the others
      double s = 0.0;
      for (int a = 0; a < n; ++a) {
        if (a == j) continue;
        der[a] = (wb[a] / wb[j]) / (xn[j] - xn[a]);
        s += der[a];
      }
      der[j] = -s;
      return;
    }
  }
  // l_a(x) = ell(x) w_a / (x - x_a); ell' / ell = sum 1/(x - x_k)
  double ell = 1.0, sinv = 0.0;
  for (int k = 0; k < n; ++k) {
    ell *= (x - xn[k]);
    sinv += 1.0 / (x - xn[k]);
  }
  for (int a = 0; a < n; ++a) {
    double d = x - xn[a];
    val[a] = ell * wb[a] / d;
    der[a] = val[a] * (sinv - 1.0 / d);
  }
}

void gauss_lobatto_weights(int P, const double* x, double* w) {
  for (int i = 0; i <= P; ++i) {
    double l0 = 1.0, l1 = x[i];
    for (int k = 1; k < P; ++k) {
      const double l2 = ((2 * k + 1) * x[i] * l1 - k * l0) / (k + 1);
      l0 = l1;
      l1 = l2;
    }
    w[i] = 2.0 / (P * (P + 1) * l1 * l1);
  }
}

bool Basis1D::build(int P_, int kind_, double k, double lam, bool start_nodal, double ja, double jb) {
  if (P_ < 1 || P_ > kMaxP) return false;
  P = P_;
  kind = kind_;
  n = P + 1;
  nodal = (kind == 0) || (kind >= 2 && start_nodal);
  alpha = ja;
  beta = jb;
  if (nodal) {
    gll.resize(n);
    gauss_lobatto_legendre(P, gll.data());
  }
  // T maps standard functions (paper order) to the final functions.
  T.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) T[i * n + i] = 1.0;
  std::vector<double> M, K;
  std::vector<double> Ts = T;
  T = Ts;
  matrices(M, K, /*final=*/false);
  if (kind >= 2 && P >= 2) {
    const int m = P - 1;
    std::vector<double> Mii(m * m), Kii(m * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        Mii[i * m + j] = M[(i + 2) * n + j + 2];
        Kii[i * m + j] = K[(i + 2) * n + j + 2];
      }
    std::vector<double> lamM, X;
    sym_eig(m, Mii, lamM, X);
    // A = X Lambda_M^{-1/2}
    std::vector<double> A(m * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) A[i * m + j] = X[i * m + j] / std::sqrt(lamM[j]);
    // L = A^T Kii A
    std::vector<double> KA(m * m, 0.0), L(m * m, 0.0);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        double s = 0.0;
        for (int l = 0; l < m; ++l) s += Kii[i * m + l] * A[l * m + j];
        KA[i * m + j] = s;
      }
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        double s = 0.0;
        for (int l = 0; l < m; ++l) s += A[l * m + i] * KA[l * m + j];
        L[i * m + j] = s;
      }
    for (int i = 0; i < m; ++i)
      for (int j = i + 1; j < m; ++j) L[i * m + j] = L[j * m + i] = 0.5 * (L[i * m + j] + L[j * m + i]);
    std::vector<double> Z;
    sym_eig(m, L, lamS, Z);
    // Y = (A Z Lambda_S^{-k/2})^T : row j of Y = column j of A Z, scaled
    std::vector<double> Y(m * m);
    for (int j = 0; j < m; ++j) {
      double sc = std::pow(lamS[j], -0.5 * k);
      for (int i = 0; i < m; ++i) {
        double s = 0.0;
        for (int l = 0; l < m; ++l) s += A[i * m + l] * Z[l * m + j];
        Y[j * m + i] = s * sc;
      }
    }
    // sign: derivative at -1 of each new internal function positive
    std::vector<double> v(n), d(n);
    eval_standard(-1.0, v.data(), d.data());
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int i = 0; i < m; ++i) s += Y[j * m + i] * d[i + 2];
      if (s < 0.0)
        for (int i = 0; i < m; ++i) Y[j * m + i] = -Y[j * m + i];
    }
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < m; ++i) T[(j + 2) * n + i + 2] = Y[j * m + i];
    // ME: alpha = G_vi G_ii^{-1}  <=>  G_ii^T alpha^T = G_vi^T
    std::vector<double> G(n * n);
    for (int i = 0; i < n * n; ++i) {
      if (kind == 2) G[i] = M[i];
      else if (kind == 3) G[i] = K[i];
      else G[i] = K[i] + lam * M[i];
    }
    std::vector<double> Gii(m * m), rhs(m * 2);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) Gii[i * m + j] = G[(j + 2) * n + i + 2];  // transpose
    for (int i = 0; i < m; ++i)
      for (int v2 = 0; v2 < 2; ++v2) rhs[i * 2 + v2] = G[v2 * n + i + 2];
    if (!dense_solve(m, 2, Gii, rhs)) return false;
    for (int v2 = 0; v2 < 2; ++v2)
      for (int i = 0; i < m; ++i) T[v2 * n + i + 2] = -rhs[i * 2 + v2];
  }
  return true;
}

void Basis1D::eval_standard(double x, double* v, double* d) const {
  if (nodal) {
    std::vector<double> lv(n), ld(n);
    lagrange_eval(n, gll.data(), x, lv.data(), ld.data());
    // paper order: L_0, L_P, L_1 .. L_{P-1}
    v[0] = lv[0];
    d[0] = ld[0];
    v[1] = lv[P];
    d[1] = ld[P];
    for (int p = 2; p < n; ++p) {
      v[p] = lv[p - 1];
      d[p] = ld[p - 1];
    }
  } else {
    v[0] = 0.5 * (1.0 - x);
    d[0] = -0.5;
    v[1] = 0.5 * (1.0 + x);
    d[1] = 0.5;
    double bub = 0.25 * (1.0 - x) * (1.0 + x), dbub = -0.5 * x;
    for (int p = 2; p < n; ++p) {
      double J = jacobi(p - 2, alpha, beta, x), dJ = jacobi_d(p - 2, alpha, beta, x);
      v[p] = bub * J;
      d[p] = dbub * J + bub * dJ;
    }
  }
}

void Basis1D::eval(double x, double* v, double* d) const {
  std::vector<double> sv(n), sd(n);
  eval_standard(x, sv.data(), sd.data());
  for (int i = 0; i < n; ++i) {
    double a = 0.0, b = 0.0;
    for (int j = 0; j < n; ++j) {
      a += T[i * n + j] * sv[j];
      b += T[i * n + j] * sd[j];
    }
    v[i] = a;
    d[i] = b;
  }
}

void Basis1D::matrices(std::vector<double>& M, std::vector<double>& K, bool final_basis) const {
  const int nq = P + 2;
  std::vector<double> xq(nq), wq(nq), v(n), d(n);
  gauss_legendre(nq, xq.data(), wq.data());
  M.assign(n * n, 0.0);
  K.assign(n * n, 0.0);
  for (int q = 0; q < nq; ++q) {
    if (final_basis) eval(xq[q], v.data(), d.data());
    else eval_standard(xq[q], v.data(), d.data());
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        M[i * n + j] += wq[q] * v[i] * v[j];
        K[i * n + j] += wq[q] * d[i] * d[j];
      }
  }
}

int Basis1D::lattice_to_paper(int j) const {
  if (j == 0) return 0;
  if (j == P) return 1;
  return j + 1;
}

void Basis1D::tables(int Q, const double* xq, double* B, double* D) const {
  std::vector<double> v(n), d(n);
  for (int q = 0; q < Q; ++q) {
    eval(xq[q], v.data(), d.data());
    for (int j = 0; j < n; ++j) {
      int pj = lattice_to_paper(j);
      if (B) B[q * n + j] = v[pj];
      if (D) D[q * n + j] = d[pj];
    }
  }
}

void collocation_derivative(int Q, const double* xq, double* DQ) {
  std::vector<double> v(Q), d(Q);
  for (int q = 0; q < Q; ++q) {
    lagrange_eval(Q, xq, xq[q], v.data(), d.data());
    for (int m = 0; m < Q; ++m) DQ[q * Q + m] = d[m];
  }
}

}  // namespace sdme

// Host-side 1D basis construction (Sec. 2).  See basis1d.cpp.
#pragma once
#include <vector>

namespace sdme {

constexpr int kMaxP = 8;

void gauss_legendre(int Q, double* x, double* w);
void gauss_lobatto_legendre(int P, double* x);
// Weights of the P + 1 point Gauss-Lobatto-Legendre rule at the nodes x:
// w_i = 2 / (P (P + 1) L_P(x_i)^2).
void gauss_lobatto_weights(int P, const double* x, double* w);
void lagrange_eval(int n, const double* xn, double x, double* val, double* der);
// DQ[q*Q + m] = derivative of the m-th Lagrange polynomial through the Q
// points xq, evaluated at xq[q] (exact derivative of degree < Q polynomials
// from their point values).
void collocation_derivative(int Q, const double* xq, double* DQ);

struct Basis1D {
  int P = 0, n = 0, kind = 0;
  bool nodal = false;
  double alpha = 1.0, beta = 1.0;
  std::vector<double> gll;     // GLL nodes (nodal start)
  std::vector<double> T;       // final = T * standard, paper order, n x n
  std::vector<double> lamS;    // eigenvalues of L (SD kinds)

  // kind: 0 nodal, 1 modal, 2 SDME-M, 3 SDME-K, 4 SDME-H
  bool build(int P, int kind, double k, double lambda, bool start_nodal, double ja, double jb);
  void eval_standard(double x, double* v, double* d) const;   // paper order
  void eval(double x, double* v, double* d) const;            // paper order
  void matrices(std::vector<double>& M, std::vector<double>& K, bool final_basis) const;
  int lattice_to_paper(int j) const;
  // B[q*n + j], D[q*n + j] in lattice order
  void tables(int Q, const double* xq, double* B, double* D) const;
};

}  // namespace sdme

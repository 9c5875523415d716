// Even-odd ("mirror") factorisation of the 1D tables used by the element
// kernels.  Host-only, no allocation (fixed-size local arrays), shared by the
// context set-up and the allocation-free entry point.
//
// Every 1D basis of the engine is mirror symmetric under xi -> -xi on the
// symmetric Gauss points:
//  * SDME (SD internal modes are the eigenfunctions of a symmetric pencil,
//    with alternating parity in ascending-eigenvalue order; the ME vertex
//    modes satisfy phi_0(-xi) = phi_P(xi)) and the modal basis with
//    alpha = beta (bubble p has the parity of P_{p-2}) have the "canonical"
//    structure: lattice positions 0 and n-1 are a mirror pair, internal
//    position j (1 <= j <= n-2) is even for odd j and odd for even j;
//  * the nodal basis on GLL points is reversal symmetric, L_a(-xi) =
//    L_{n-1-a}(xi); replacing each mirrored internal pair (i, n-1-i) by
//    (L_i + L_{n-1-i})/2 and (L_i - L_{n-1-i})/2 (even, odd; the middle node
//    stays) gives the canonical structure.  The kernels apply that change of
//    coefficients on the fly ("pairs" flag): c_e = u_i + u_j, c_o = u_i - u_j
//    on loads and r_i = r_e + r_o, r_j = r_e - r_o on stores.
// With the structure known, a line contraction over n modes and Q points
// splits into an even and an odd half, halving its multiply-adds:
//   out[q] = S + D, out[Q-1-q] = S - D,  S = TE[q] . e,  D = TO[q] . o,
//   e = (in_0 + in_{n-1}, in_1, in_3, ...),  o = (in_0 - in_{n-1}, in_2, in_4, ...),
// with TE[q][0] = (B[q][0] + B[q][n-1]) / 2, TE[q][k] = B[q][2k-1],
// TO[q][0] = (B[q][0] - B[q][n-1]) / 2, TO[q][k] = B[q][2k], and for odd Q the
// middle point row TEm.  The collocation-derivative matrix on the Gauss
// points is antisymmetric under point reflection, DQ[Q-1-q][Q-1-m] =
// -DQ[q][m], which gives AH = (DQ[q][m] - DQ[q][Q-1-m]) / 2,
// CH = (DQ[q][m] + DQ[q][Q-1-m]) / 2, CM[q] = DQ[q][mid], DM[m] = DQ[mid][m].
#pragma once

#include <cmath>

namespace sdme {

enum EoSymmetry { kEoNone = 0, kEoCanonical = 1, kEoNodalPairs = 2 };

// Sizes for order P (n = P + 1 modes, Q = P + 2 points).
struct EoSizes {
  int n, Q, QH, NE, NO;
  explicit EoSizes(int P) : n(P + 1), Q(P + 2), QH((P + 2) / 2), NE(1 + P / 2), NO(1 + (P - 1) / 2) {}
};

// Builds the half tables from the natural tables B (Q x n, lattice order)
// and DQ (Q x Q).  Returns the symmetry class found (kEoNone when the basis
// is not mirror symmetric to `tol` relative; the outputs are then unset).
// Output sizes: TE[QH*NE], TO[QH*NO], TEm[NE], AH[QH*QH], CH[QH*QH],
// CM[QH], DM[QH] (TEm, CM, DM are zero for even Q).
inline int build_eo_tables(int P, const double* B, const double* DQ, double* TE, double* TO, double* TEm,
                           double* AH, double* CH, double* CM, double* DM, double tol = 1e-11) {
  const EoSizes z(P);
  const int n = z.n, Q = z.Q, QH = z.QH;
  double scale = 0.0;
  for (int i = 0; i < Q * n; ++i) scale = std::fmax(scale, std::fabs(B[i]));
  double dscale = 0.0;
  for (int i = 0; i < Q * Q; ++i) dscale = std::fmax(dscale, std::fabs(DQ[i]));
  // canonical-structure table Bc (Q x n), possibly after the nodal pairing
  double Bc[16 * 16];
  auto canonical_ok = [&](const double* Bt) {
    for (int q = 0; q < Q; ++q) {
      const int r = Q - 1 - q;
      if (std::fabs(Bt[r * n + 0] - Bt[q * n + n - 1]) > tol * scale) return false;
      if (std::fabs(Bt[r * n + n - 1] - Bt[q * n + 0]) > tol * scale) return false;
      for (int j = 1; j <= n - 2; ++j) {
        const double sgn = (j % 2 == 1) ? 1.0 : -1.0;
        if (std::fabs(Bt[r * n + j] - sgn * Bt[q * n + j]) > tol * scale) return false;
      }
    }
    return true;
  };
  int sym = kEoNone;
  for (int i = 0; i < Q * n; ++i) Bc[i] = B[i];
  if (canonical_ok(Bc)) {
    sym = kEoCanonical;
  } else {
    // nodal pairing: pair i = 1..np -> positions 2i-1 (even), 2i (odd);
    // middle node (P even) -> position n-2
    const int np = (n - 2) / 2;
    for (int q = 0; q < Q; ++q) {
      double* row = Bc + q * n;
      const double* src = B + q * n;
      row[0] = src[0];
      row[n - 1] = src[n - 1];
      for (int i = 1; i <= np; ++i) {
        row[2 * i - 1] = 0.5 * (src[i] + src[n - 1 - i]);
        row[2 * i] = 0.5 * (src[i] - src[n - 1 - i]);
      }
      if ((n - 2) % 2 == 1) row[n - 2] = src[(n - 1) / 2];
    }
    if (canonical_ok(Bc)) sym = kEoNodalPairs;
  }
  if (sym == kEoNone) return kEoNone;
  for (int q = 0; q < Q; ++q)
    for (int m = 0; m < Q; ++m)
      if (std::fabs(DQ[(Q - 1 - q) * Q + (Q - 1 - m)] + DQ[q * Q + m]) > tol * dscale) return kEoNone;
  for (int q = 0; q < QH; ++q) {
    const double* row = Bc + q * n;
    TE[q * z.NE + 0] = 0.5 * (row[0] + row[n - 1]);
    TO[q * z.NO + 0] = 0.5 * (row[0] - row[n - 1]);
    for (int k = 1; k < z.NE; ++k) TE[q * z.NE + k] = row[2 * k - 1];
    for (int k = 1; k < z.NO; ++k) TO[q * z.NO + k] = row[2 * k];
  }
  const bool odd = (Q % 2) == 1;
  for (int k = 0; k < z.NE; ++k) TEm[k] = 0.0;
  if (odd) {
    const double* row = Bc + QH * n;
    TEm[0] = row[0];
    for (int k = 1; k < z.NE; ++k) TEm[k] = row[2 * k - 1];
  }
  for (int q = 0; q < QH; ++q) {
    for (int m = 0; m < QH; ++m) {
      AH[q * QH + m] = 0.5 * (DQ[q * Q + m] - DQ[q * Q + (Q - 1 - m)]);
      CH[q * QH + m] = 0.5 * (DQ[q * Q + m] + DQ[q * Q + (Q - 1 - m)]);
    }
    CM[q] = odd ? DQ[q * Q + QH] : 0.0;
    DM[q] = odd ? DQ[QH * Q + q] : 0.0;
  }
  return sym;
}

}  // namespace sdme

// Host-side generator of the per-level 1D operators used by the kernels.
//
// For a level with n nodes on the sub-element reference interval [-1/2, 1/2]
// (Sec. 2.2 of the paper, eq. sub-element), it produces, in double precision from
// long-double arithmetic:
//   R      = P^-1, reconstruction from n subcell means to n nodal values (eq. trafo-mv-nodal)
//   P      projection from nodal values to n subcell means (Sec. 2.3)
//   Dn     nodal differentiation matrix D_ij = l_j'(xi_i) (Sec. 2.2)
//   Dhat   = P Dvol, Dvol = M^-1 D^T M (eqs. semi-discrete-dg, dgfv-operators)
//   Bh0/Bhn the two nonzero columns of Bhat = P B^(0) (eqs. tweak-boundary-
//          evaluation-matrix, dgfv-operators)
//   IRf    (n+1) x n: values at the n+1 subcell interfaces of the polynomial
//          reconstructed from the n means, i.e. I_face R (eq. subcell-fv-
//          interpolation-operator composed with eq. trafo-mv-nodal)
//   w      quadrature weights (sum 1)
//   C, c0, cn  telescoping (subcell-flux) form of the level's right-hand side: with
//          F_L, F_R the common fluxes at the sub-element's two boundaries and f the
//          nodal fluxes, the flux at interior interface k (1..n-1) is
//          G_k = c0_k F_L + cn_k F_R - (1/n) sum_j C_kj f_j, where
//          C_kj = sum_{i<=k} Dhat_ij, c0_k = 1 + (1/n) sum_{i<=k} Bhat_i0 and
//          cn_k = (1/n) sum_{i<=k} Bhat_in; then (M/n)(Dhat f - Bhat F)_i / dx =
//          -(M/dx)(G_i - G_{i-1}) with G_0 = F_L, G_n = F_R. This follows from the
//          zero column sums of Dhat and the boundary sums of Bhat (eqs.
//          dg-vol-mat-property, projection-mat-property, dg-surf-mat-property).
// Node families: Gauss-Legendre (the paper's choice) and Gauss-Lobatto.
#pragma once

namespace sesc {

struct LevelOps {
  int n;
  double R[64], P[64], Dn[64], Dhat[64], IRf[72], Bh0[8], Bhn[8], w[8], nodes[8];
  double C[64], c0[8], cn[8];   // rows k = 1..n-1 stored at k-1
};

// Fills `out` for n in {2, 4, 8}; family 0 = Gauss-Legendre, 1 = Gauss-Lobatto.
// Returns false for unsupported arguments.
bool make_level_ops(int n, int family, LevelOps* out);

}  // namespace sesc

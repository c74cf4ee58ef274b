// Reference-element operators of the ADER-DG scheme, generated on the host.
//
// Basis (Sec. 4.1 names Dubiner's basis; B_N = C(N+3,3)): the orthonormal
// Dubiner product basis on the reference tetrahedron (0,0,0),(1,0,0),(0,1,0),
// (0,0,1), ordered by total degree, then i, then j (k = n - i - j):
//   phi_ijk ~ s^i P_i^(0,0)(2 xi/s - 1) t^j P_j^(2i+1,0)(2 eta/t - 1)
//             P_k^(2i+2j+2,0)(2 zeta - 1),  s = 1 - eta - zeta, t = 1 - zeta,
// scaled to unit L2 norm with a positive constant.  Here every basis function
// is expanded into monomials (scaled Jacobi recurrences in homogeneous form)
// and every integral is taken exactly from int x^a y^b z^c = a!b!c!/(a+b+c+3)!
// in long double; no quadrature is involved.
//
// Face f of the tet is the face opposite vertex f; its vertices in increasing
// local order (a,b,c) define x(chi) = Va + chi1 (Vb - Va) + chi2 (Vc - Va).
// Face data are nodal on the (N+1)(N+2)/2 equispaced points of the reference
// triangle, chi = (i1/N, i2/N); the point set is invariant under the six vertex
// permutations, so re-orienting a neighbour's trace is a permutation of nodes.
#pragma once
#include <vector>

namespace adg {

inline int nbasis(int n) { return n < 0 ? 0 : (n + 1) * (n + 2) * (n + 3) / 6; }
inline int nface(int n) { return (n + 1) * (n + 2) / 2; }

struct RefOps {
  int N = 0, B = 0, Bf = 0, B1 = 0;
  // kt[a][m][l] = int phi_l dphi_m/dxi_a ... see refmat.cpp for exact meaning
  std::vector<double> kt;     // (3, B, B):  kt[a][m][l] = int phi_m * dphi_l/dxi_a   (CK, strong form)
  std::vector<double> kvol;   // (3, B, B1): kvol[a][m][l] = int dphi_m/dxi_a * phi_l (l < B_{N-1})
  std::vector<double> efc;    // (4, Bf, B): efc[f][n][l] = phi_l at node n of face f
  std::vector<double> lift;   // (4, B, Bf): lift[f][m][n] = int_tri phi_m(face f) * ell_n
  std::vector<int> perm;      // (6, Bf): node permutation for each vertex permutation
  std::vector<double> node_chi;  // (Bf, 2)
  std::vector<int> vperm;     // (6, 3) the vertex permutations in perm order
  double max_orth_err = 0.0;  // |M - I|_max, checked at generation
};

RefOps make_ref_ops(int N);
// phi_l(xi) for a point (used for receivers / projections on the host)
void eval_basis(const RefOps& ops, const double xi[3], double* out /*B*/);

}  // namespace adg

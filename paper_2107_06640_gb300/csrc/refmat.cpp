// Host generation of the reference operators (see refmat.hpp for the basis,
// face and node conventions).  Exact monomial arithmetic in long double.
#include "refmat.hpp"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace adg {
namespace {

typedef long double ld;

// Dense polynomial in (x, y, z) with exponents < D per variable.
struct P3 {
  int D;
  std::vector<ld> c;
  explicit P3(int d = 1) : D(d), c((size_t)d * d * d, 0.0L) {}
  ld& at(int a, int b, int e) { return c[(size_t)a + D * (b + (size_t)D * e)]; }
  ld get(int a, int b, int e) const { return c[(size_t)a + D * (b + (size_t)D * e)]; }
};

P3 konst(int D, ld v) { P3 p(D); p.at(0, 0, 0) = v; return p; }
P3 lin(int D, ld c0, ld cx, ld cy, ld cz) {
  P3 p(D);
  p.at(0, 0, 0) = c0;
  p.at(1, 0, 0) = cx;
  p.at(0, 1, 0) = cy;
  p.at(0, 0, 1) = cz;
  return p;
}
P3 add(const P3& a, const P3& b, ld sa = 1, ld sb = 1) {
  P3 r(a.D);
  for (size_t i = 0; i < r.c.size(); ++i) r.c[i] = sa * a.c[i] + sb * b.c[i];
  return r;
}
P3 mul(const P3& a, const P3& b) {
  const int D = a.D;
  P3 r(D);
  for (int a1 = 0; a1 < D; ++a1)
    for (int b1 = 0; b1 < D; ++b1)
      for (int c1 = 0; c1 < D; ++c1) {
        ld va = a.get(a1, b1, c1);
        if (va == 0) continue;
        for (int a2 = 0; a1 + a2 < D; ++a2)
          for (int b2 = 0; b1 + b2 < D; ++b2)
            for (int c2 = 0; c1 + c2 < D; ++c2) {
              ld vb = b.get(a2, b2, c2);
              if (vb != 0) r.at(a1 + a2, b1 + b2, c1 + c2) += va * vb;
            }
      }
  // overflow check: product must fit (total degree bound respected by callers)
  return r;
}
P3 deriv(const P3& p, int dir) {
  P3 r(p.D);
  for (int a = 0; a < p.D; ++a)
    for (int b = 0; b < p.D; ++b)
      for (int e = 0; e < p.D; ++e) {
        int ex[3] = {a, b, e};
        if (ex[dir] == 0) continue;
        ld v = p.get(a, b, e) * ex[dir];
        ex[dir] -= 1;
        r.at(ex[0], ex[1], ex[2]) += v;
      }
  return r;
}
ld fact(int n) { ld r = 1; for (int i = 2; i <= n; ++i) r *= i; return r; }
// int over the reference tet of x^a y^b z^c = a! b! c! / (a+b+c+3)!
ld tet_int(const P3& p) {
  ld s = 0;
  for (int a = 0; a < p.D; ++a)
    for (int b = 0; b < p.D; ++b)
      for (int e = 0; e < p.D; ++e) {
        ld v = p.get(a, b, e);
        if (v != 0) s += v * fact(a) * fact(b) * fact(e) / fact(a + b + e + 3);
      }
  return s;
}
ld eval(const P3& p, ld x, ld y, ld z) {
  ld s = 0;
  for (int e = p.D - 1; e >= 0; --e) {
    ld sy = 0;
    for (int b = p.D - 1; b >= 0; --b) {
      ld sx = 0;
      for (int a = p.D - 1; a >= 0; --a) sx = sx * x + p.get(a, b, e);
      sy = sy * y + sx;
    }
    s = s * z + sy;
  }
  return s;
}

// tau^n P_n^(alpha,0)(2 x/tau - 1) for linear polynomials x, tau, via the
// three-term Jacobi recurrence multiplied through by tau^n.
P3 scaled_jacobi(int n, int alpha, const P3& x, const P3& tau) {
  const int D = x.D;
  P3 q0 = konst(D, 1.0L);
  if (n == 0) return q0;
  const ld al = alpha;
  // P_1 = (alpha+1) + (alpha+2)(y-1)/2  ->  (alpha+1) tau + (alpha+2)(x - tau)
  P3 q1 = add(tau, add(x, tau, 1, -1), al + 1, al + 2);
  if (n == 1) return q1;
  P3 two_x_minus_tau = add(x, tau, 2, -1);
  P3 tau2 = mul(tau, tau);
  for (int m = 2; m <= n; ++m) {
    ld a = 2 * m + al;
    ld lhs = 2.0L * m * (m + al) * (a - 2);
    ld c1 = (a - 1);
    P3 t1 = add(two_x_minus_tau, tau, a * (a - 2), al * al);  // a(a-2)(2x-tau) + alpha^2 tau
    P3 term1 = mul(t1, q1);
    P3 term2 = mul(tau2, q0);
    ld c2 = 2.0L * (m + al - 1) * (m - 1) * a;
    P3 q2 = add(term1, term2, c1 / lhs, -c2 / lhs);
    q0 = q1;
    q1 = q2;
  }
  return q1;
}

struct Tri { int i, j, k; };
std::vector<Tri> triples(int N) {
  std::vector<Tri> t;
  for (int n = 0; n <= N; ++n)
    for (int i = 0; i <= n; ++i)
      for (int j = 0; j <= n - i; ++j) t.push_back({i, j, n - i - j});
  return t;
}

const ld kRefV[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
const int kFaceV[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

// Polynomial in (chi1, chi2) stored as P3 with z exponent 0.
P3 restrict_to_face(const P3& p, int f, int D) {
  // x(chi) = Va + chi1 (Vb - Va) + chi2 (Vc - Va), each coordinate linear in chi
  const ld* A = kRefV[kFaceV[f][0]];
  const ld* Bv = kRefV[kFaceV[f][1]];
  const ld* C = kRefV[kFaceV[f][2]];
  P3 X[3];
  for (int d = 0; d < 3; ++d) X[d] = lin(D, A[d], Bv[d] - A[d], C[d] - A[d], 0);
  // Horner-free expansion: sum c_abe X^a Y^b Z^e
  std::vector<P3> px(p.D, konst(D, 1)), py(p.D, konst(D, 1)), pz(p.D, konst(D, 1));
  for (int i = 1; i < p.D; ++i) {
    px[i] = mul(px[i - 1], X[0]);
    py[i] = mul(py[i - 1], X[1]);
    pz[i] = mul(pz[i - 1], X[2]);
  }
  P3 r(D);
  for (int a = 0; a < p.D; ++a)
    for (int b = 0; a + b < p.D; ++b)
      for (int e = 0; a + b + e < p.D; ++e) {
        ld v = p.get(a, b, e);
        if (v == 0) continue;
        P3 m = mul(mul(px[a], py[b]), pz[e]);
        r = add(r, m, 1, v);
      }
  return r;
}
// int over the reference triangle of chi1^a chi2^b = a! b! / (a+b+2)!
ld tri_int(const P3& p) {
  ld s = 0;
  for (int a = 0; a < p.D; ++a)
    for (int b = 0; b < p.D; ++b) {
      ld v = p.get(a, b, 0);
      if (v != 0) s += v * fact(a) * fact(b) / fact(a + b + 2);
    }
  return s;
}

// Gauss-Jordan inverse (long double, partial pivoting)
std::vector<ld> invert(std::vector<ld> A, int n) {
  std::vector<ld> I((size_t)n * n, 0);
  for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs((double)A[(size_t)r * n + c]) > std::fabs((double)A[(size_t)piv * n + c])) piv = r;
    if (A[(size_t)piv * n + c] == 0) throw std::runtime_error("singular face Vandermonde");
    for (int k = 0; k < n; ++k) {
      std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
      std::swap(I[(size_t)c * n + k], I[(size_t)piv * n + k]);
    }
    ld d = A[(size_t)c * n + c];
    for (int k = 0; k < n; ++k) { A[(size_t)c * n + k] /= d; I[(size_t)c * n + k] /= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      ld m = A[(size_t)r * n + c];
      if (m == 0) continue;
      for (int k = 0; k < n; ++k) {
        A[(size_t)r * n + k] -= m * A[(size_t)c * n + k];
        I[(size_t)r * n + k] -= m * I[(size_t)c * n + k];
      }
    }
  }
  return I;
}

std::vector<P3> build_basis(int N, int D) {
  std::vector<P3> phi;
  P3 xi = lin(D, 0, 1, 0, 0), eta = lin(D, 0, 0, 1, 0), zeta = lin(D, 0, 0, 0, 1);
  P3 s = lin(D, 1, 0, -1, -1), t = lin(D, 1, 0, 0, -1), one = konst(D, 1);
  for (const Tri& tr : triples(N)) {
    P3 f1 = scaled_jacobi(tr.i, 0, xi, s);
    P3 f2 = scaled_jacobi(tr.j, 2 * tr.i + 1, eta, t);
    // P_k^(alpha,0)(2 zeta - 1) = scaled form with x = zeta, tau = 1
    P3 f3 = scaled_jacobi(tr.k, 2 * tr.i + 2 * tr.j + 2, zeta, one);
    P3 p = mul(mul(f1, f2), f3);
    ld nrm = std::sqrt(tet_int(mul(p, p)));
    for (auto& v : p.c) v /= nrm;
    phi.push_back(p);
  }
  return phi;
}

}  // namespace

RefOps make_ref_ops(int N) {
  if (N < 1 || N > 7) throw std::runtime_error("degree must be in [1, 7]");
  RefOps r;
  r.N = N;
  r.B = nbasis(N);
  r.Bf = nface(N);
  r.B1 = nbasis(N - 1);
  const int B = r.B, Bf = r.Bf, B1 = r.B1;
  const int D = 2 * N + 2;  // room for products of two degree-N polynomials
  std::vector<P3> phi = build_basis(N, D);
  std::vector<P3> dphi[3];
  for (int a = 0; a < 3; ++a)
    for (int l = 0; l < B; ++l) dphi[a].push_back(deriv(phi[l], a));
  // orthonormality check
  for (int k = 0; k < B; ++k)
    for (int l = 0; l <= k; ++l) {
      double m = (double)tet_int(mul(phi[k], phi[l]));
      r.max_orth_err = std::max(r.max_orth_err, std::fabs(m - (k == l ? 1.0 : 0.0)));
    }
  r.kt.assign((size_t)3 * B * B, 0.0);
  r.kvol.assign((size_t)3 * B * B1, 0.0);
  for (int a = 0; a < 3; ++a)
    for (int m = 0; m < B; ++m)
      for (int l = 0; l < B; ++l) {
        double v = (double)tet_int(mul(phi[m], dphi[a][l]));  // int phi_m dphi_l/dxi_a
        r.kt[((size_t)a * B + m) * B + l] = v;
        if (l < B1) r.kvol[((size_t)a * B + m) * B1 + l] = (double)tet_int(mul(dphi[a][m], phi[l]));
      }
  // face nodes: chi = (i1/N, i2/N), i2 outer, i1 inner
  std::vector<int> n1, n2;
  for (int i2 = 0; i2 <= N; ++i2)
    for (int i1 = 0; i1 + i2 <= N; ++i1) {
      n1.push_back(i1);
      n2.push_back(i2);
      r.node_chi.push_back((double)i1 / N);
      r.node_chi.push_back((double)i2 / N);
    }
  // Lagrange basis on the nodes: invert the monomial Vandermonde
  std::vector<std::pair<int, int>> mono;
  for (int a = 0; a <= N; ++a)
    for (int b = 0; a + b <= N; ++b) mono.push_back({a, b});
  std::vector<ld> V((size_t)Bf * Bf);
  for (int n = 0; n < Bf; ++n)
    for (int j = 0; j < Bf; ++j) {
      ld x = (ld)n1[n] / N, y = (ld)n2[n] / N;
      V[(size_t)n * Bf + j] = std::pow(x, mono[j].first) * std::pow(y, mono[j].second);
    }
  std::vector<ld> Vi = invert(V, Bf);  // coefficients of ell_n: column n of V^-1
  std::vector<P3> ell;
  for (int n = 0; n < Bf; ++n) {
    P3 p(D);
    for (int j = 0; j < Bf; ++j) p.at(mono[j].first, mono[j].second, 0) = Vi[(size_t)j * Bf + n];
    ell.push_back(p);
  }
  r.efc.assign((size_t)4 * Bf * B, 0.0);
  r.lift.assign((size_t)4 * B * Bf, 0.0);
  for (int f = 0; f < 4; ++f) {
    const ld* A = kRefV[kFaceV[f][0]];
    const ld* Bv = kRefV[kFaceV[f][1]];
    const ld* C = kRefV[kFaceV[f][2]];
    for (int n = 0; n < Bf; ++n) {
      ld c1 = (ld)n1[n] / N, c2 = (ld)n2[n] / N;
      ld x[3];
      for (int d = 0; d < 3; ++d) x[d] = A[d] + c1 * (Bv[d] - A[d]) + c2 * (C[d] - A[d]);
      for (int l = 0; l < B; ++l) r.efc[((size_t)f * Bf + n) * B + l] = (double)eval(phi[l], x[0], x[1], x[2]);
    }
    for (int m = 0; m < B; ++m) {
      P3 pf = restrict_to_face(phi[m], f, D);
      for (int n = 0; n < Bf; ++n) r.lift[((size_t)f * B + m) * Bf + n] = (double)tri_int(mul(pf, ell[n]));
    }
  }
  // vertex permutations sigma: my barycentric slot s takes the neighbour's slot sigma[s]
  const int vp[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  r.perm.assign((size_t)6 * Bf, -1);
  for (int p = 0; p < 6; ++p) {
    for (int s = 0; s < 3; ++s) r.vperm.push_back(vp[p][s]);
    for (int n = 0; n < Bf; ++n) {
      int bary[3] = {N - n1[n] - n2[n], n1[n], n2[n]};
      int nb[3];
      for (int s = 0; s < 3; ++s) nb[vp[p][s]] = bary[s];
      // find node with barycentric (nb0, nb1, nb2): i1 = nb1, i2 = nb2
      for (int q = 0; q < Bf; ++q)
        if (n1[q] == nb[1] && n2[q] == nb[2]) r.perm[(size_t)p * Bf + n] = q;
    }
  }
  return r;
}

void eval_basis(const RefOps& ops, const double xi[3], double* out) {
  // basis values through the face evaluation is not general; rebuild on demand
  static thread_local int cachedN = -1;
  static thread_local std::vector<P3> phi;
  if (cachedN != ops.N) {
    phi = build_basis(ops.N, 2 * ops.N + 2);
    cachedN = ops.N;
  }
  for (int l = 0; l < ops.B; ++l) out[l] = (double)eval(phi[l], xi[0], xi[1], xi[2]);
}

}  // namespace adg

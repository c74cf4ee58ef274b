// Host side of the C ABI (include/adg.h): mesh set-up, geometry, clustering,
// Godunov flux matrices, device memory, the rate-2 LTS tick schedule and the
// per-macro-step CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/adg.h"
#include "kernels.cuh"
#include "refmat.hpp"
#include "adg_internal.hpp"

using namespace adg;

namespace {

const int kFaceV[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

using Err = adg::AdgError;

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t _e = (call);                                                              \
    if (_e != cudaSuccess) throw Err(ADG_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// ---------------- small dense 9x9 helpers (row-major) ----------------
typedef std::array<double, 81> M9;
M9 mm(const M9& a, const M9& b) {
  M9 r{};
  for (int i = 0; i < 9; ++i)
    for (int k = 0; k < 9; ++k) {
      double v = a[i * 9 + k];
      if (v == 0) continue;
      for (int j = 0; j < 9; ++j) r[i * 9 + j] += v * b[k * 9 + j];
    }
  return r;
}
M9 madd(const M9& a, const M9& b) { M9 r; for (int i = 0; i < 81; ++i) r[i] = a[i] + b[i]; return r; }

// x-Jacobian of Eq. (elasticity-pde) (the rotated 1-D problem uses A only)
M9 jac_x(double rho, double lam, double mu) {
  M9 A{};
  A[0 * 9 + 6] = -(lam + 2 * mu);
  A[1 * 9 + 6] = -lam;
  A[2 * 9 + 6] = -lam;
  A[3 * 9 + 7] = -mu;
  A[5 * 9 + 8] = -mu;
  A[6 * 9 + 0] = -1.0 / rho;
  A[7 * 9 + 3] = -1.0 / rho;
  A[8 * 9 + 5] = -1.0 / rho;
  return A;
}

// Orthonormal frame (n, s, t) and the maps T (rotated -> global) and T^-1.
void frame(const double n[3], double R[3][3]) {
  int k = 0;
  for (int d = 1; d < 3; ++d)
    if (std::fabs(n[d]) < std::fabs(n[k])) k = d;
  double a[3] = {0, 0, 0};
  a[k] = 1;
  double dot = a[0] * n[0] + a[1] * n[1] + a[2] * n[2];
  double s[3] = {a[0] - dot * n[0], a[1] - dot * n[1], a[2] - dot * n[2]};
  double ns = std::sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
  for (double& v : s) v /= ns;
  double t[3] = {n[1] * s[2] - n[2] * s[1], n[2] * s[0] - n[0] * s[2], n[0] * s[1] - n[1] * s[0]};
  for (int d = 0; d < 3; ++d) { R[d][0] = n[d]; R[d][1] = s[d]; R[d][2] = t[d]; }
}
const int kVo[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {1, 2}, {0, 2}};
// out = rotate(vec): fwd => stress R S R^T, vel R v ; inverse => R^T S R, R^T v
void rot9(const double R[3][3], const double* in, double* out, bool to_global) {
  double S[3][3];
  for (int c = 0; c < 6; ++c) { S[kVo[c][0]][kVo[c][1]] = in[c]; S[kVo[c][1]][kVo[c][0]] = in[c]; }
  double Rm[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Rm[i][j] = to_global ? R[i][j] : R[j][i];
  double Y[3][3];
  for (int i = 0; i < 3; ++i)
    for (int l = 0; l < 3; ++l) {
      double acc = 0;
      for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) acc += Rm[i][j] * S[j][k] * Rm[l][k];
      Y[i][l] = acc;
    }
  for (int c = 0; c < 6; ++c) out[c] = Y[kVo[c][0]][kVo[c][1]];
  for (int i = 0; i < 3; ++i) {
    double acc = 0;
    for (int j = 0; j < 3; ++j) acc += Rm[i][j] * in[6 + j];
    out[6 + i] = acc;
  }
}
void rot_mats(const double n[3], M9& T, M9& Ti) {
  double R[3][3];
  frame(n, R);
  for (int c = 0; c < 9; ++c) {
    double e[9] = {0}, o[9];
    e[c] = 1;
    rot9(R, e, o, true);
    for (int r = 0; r < 9; ++r) T[r * 9 + c] = o[r];
    rot9(R, e, o, false);
    for (int r = 0; r < 9; ++r) Ti[r * 9 + c] = o[r];
  }
}

// Middle state w^b = Mm w^- + Mp w^+ (Sec. 4.2, Eq. boundary-state; solid-solid
// shear with the same welded form using Z_s).
void middle_state(double Zpm, double Zpp, double Zsm, double Zsp, M9& Mm, M9& Mp) {
  Mm.fill(0);
  Mp.fill(0);
  const double c = Zpm * Zpp / (Zpm + Zpp);
  Mm[0 * 9 + 0] = 1 - c / Zpp; Mm[0 * 9 + 6] = -c;
  Mp[0 * 9 + 0] = c / Zpp;     Mp[0 * 9 + 6] = c;
  Mm[6 * 9 + 0] = -c / (Zpp * Zpm); Mm[6 * 9 + 6] = 1 - c / Zpm;
  Mp[6 * 9 + 0] = c / (Zpp * Zpm);  Mp[6 * 9 + 6] = c / Zpm;
  for (int r : {1, 2, 4}) Mm[r * 9 + r] = 1;  // irrelevant components (zero columns of A)
  const int pairs[2][2] = {{3, 7}, {5, 8}};
  for (auto& pr : pairs) {
    const int ts = pr[0], tv = pr[1];
    if (Zsm > 0 && Zsp > 0) {
      const double cs = Zsm * Zsp / (Zsm + Zsp);
      Mm[ts * 9 + ts] = 1 - cs / Zsp; Mm[ts * 9 + tv] = -cs;
      Mp[ts * 9 + ts] = cs / Zsp;     Mp[ts * 9 + tv] = cs;
      Mm[tv * 9 + ts] = -cs / (Zsp * Zsm); Mm[tv * 9 + tv] = 1 - cs / Zsm;
      Mp[tv * 9 + ts] = cs / (Zsp * Zsm);  Mp[tv * 9 + tv] = cs / Zsm;
    } else {
      Mm[tv * 9 + tv] = 1;
      if (Zsm > 0) Mm[tv * 9 + ts] = -1.0 / Zsm;
    }
  }
}

M9 diag9(std::initializer_list<double> d) {
  M9 r{};
  int i = 0;
  for (double v : d) { r[i * 9 + i] = v; ++i; }
  return r;
}

// Godunov flux matrices of a face in the global frame (Sec. 4.2, Eq.
// numerical-flux): with TA = T A^- and Ti = T^-1 for the face's normal, the
// flux T A^- w^b, w^b = Mm T^-1 q^- + Mp T^-1 q^+, is Fm q^- + Fp q^+.
void godunov_pair(const M9& TA, const M9& Ti, double Zpm, double Zpp, double Zsm, double Zsp, M9& Fm, M9& Fp) {
  M9 Mm, Mp;
  middle_state(Zpm, Zpp, Zsm, Zsp, Mm, Mp);
  Fm = mm(mm(TA, Mm), Ti);
  Fp = mm(mm(TA, Mp), Ti);
}

// Linear boundaries (Sec. 4.3): the ghost state w^+ = G w^- (free surface:
// traction w1, w4, w6 mirrored; rigid wall: w7, w4, w6 mirrored; absorbing:
// G = 0) with the minus material folds into Fm = T A^- (Mm + Mp G) T^-1.
M9 boundary_matrix(const M9& TA, const M9& Ti, double Zp, double Zs, int tag) {
  M9 Mm, Mp;
  middle_state(Zp, Zp, Zs, Zs, Mm, Mp);
  M9 G{};
  if (tag == ADG_TAG_FREE) G = diag9({-1, 1, 1, -1, 1, -1, 1, 1, 1});
  else if (tag == ADG_TAG_RIGID) G = diag9({1, 1, 1, -1, 1, -1, -1, 1, 1});
  return mm(mm(TA, madd(Mm, mm(Mp, G))), Ti);
}

// ---------------- Gauss-Legendre on [0,1] (Newton on P_n) ----------------
void gauss01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1, p2 = 0;
      for (int j = 1; j <= n; ++j) { double p3 = p2; p2 = p1; p1 = ((2 * j - 1) * z * p2 - (j - 1) * p3) / j; }
      pp = n * (z * p1 - p2) / (z * z - 1);
      double dz = p1 / pp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (1 - z);
    w[i] = 1.0 / ((1 - z * z) * pp * pp);  // = 0.5 * 2/((1-z^2) P'^2)
  }
}

}  // namespace

// ======================================================================
namespace adg {

[[noreturn]] void throw_err(int code, const std::string& m) { throw Err(code, m); }

template <typename T>
static void* upload_vec(const std::vector<double>& h, std::vector<void*>& owned, int64_t& bytes) {
  std::vector<T> t(h.begin(), h.end());
  void* d = nullptr;
  if (t.empty()) return nullptr;
  CK(cudaMalloc(&d, t.size() * sizeof(T)));
  owned.push_back(d);
  bytes += t.size() * sizeof(T);
  CK(cudaMemcpy(d, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice));
  return d;
}
template <typename T>
static T* upload_raw(const std::vector<T>& h, std::vector<void*>& owned, int64_t& bytes) {
  if (h.empty()) return nullptr;
  void* d = nullptr;
  CK(cudaMalloc(&d, h.size() * sizeof(T)));
  owned.push_back(d);
  bytes += h.size() * sizeof(T);
  CK(cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return (T*)d;
}
static void* dalloc(size_t n, std::vector<void*>& owned, int64_t& bytes) {
  if (n == 0) return nullptr;
  void* d = nullptr;
  CK(cudaMalloc(&d, n));
  owned.push_back(d);
  bytes += n;
  CK(cudaMemset(d, 0, n));
  return d;
}

// Host-side plan of the mesh in the caller's element order: geometry, face
// connectivity with node permutations, CFL time steps and rate-2 clusters
// (Sec. 4.4).  Needs no device; adg_init and adg_plan both use it.
void Ctx::plan_mesh(const RefOps& o, int degree, MeshPlan& plan) const {
  const int64_t E = nt;
  // ---- geometry (user order)
  plan.Jinv.assign(9 * E, 0.0); plan.detJ.assign(E, 0.0); plan.area.assign(4 * E, 0.0); plan.nrm.assign(12 * E, 0.0);
  plan.fcen.assign(12 * E, 0.0); plan.h.assign(E, 0.0);
  std::vector<double>&Jinv = plan.Jinv, &detJ = plan.detJ, &area = plan.area, &nrm = plan.nrm, &fcen = plan.fcen, &h = plan.h;
  for (int64_t e = 0; e < E; ++e) {
    const double* P[4];
    for (int k = 0; k < 4; ++k) {
      int64_t vid = tets[4 * e + k];
      if (vid < 0 || vid >= nv) throw Err(ADG_E_MESH, "vertex index out of range");
      P[k] = &xyz[3 * vid];
    }
    double J[3][3];
    for (int d = 0; d < 3; ++d)
      for (int c = 0; c < 3; ++c) J[d][c] = P[c + 1][d] - P[0][d];
    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                 J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                 J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    if (!(det > 0)) throw Err(ADG_E_MESH, "inverted or degenerate tetrahedron " + std::to_string(e));
    detJ[e] = det;
    // inverse: Jinv[a][d] = d xi_a / d x_d
    double Ji[3][3];
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    for (int a = 0; a < 3; ++a)
      for (int d = 0; d < 3; ++d) Jinv[9 * e + 3 * a + d] = Ji[a][d];
    double asum = 0;
    for (int f = 0; f < 4; ++f) {
      const double* A = P[kFaceV[f][0]];
      const double* Bv = P[kFaceV[f][1]];
      const double* C = P[kFaceV[f][2]];
      double u[3], w[3], cr[3];
      for (int d = 0; d < 3; ++d) { u[d] = Bv[d] - A[d]; w[d] = C[d] - A[d]; }
      cr[0] = u[1] * w[2] - u[2] * w[1];
      cr[1] = u[2] * w[0] - u[0] * w[2];
      cr[2] = u[0] * w[1] - u[1] * w[0];
      double ar = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
      double out = 0;
      for (int d = 0; d < 3; ++d) out += cr[d] * (A[d] - P[f][d]);
      double sg = out > 0 ? 1.0 : -1.0;
      for (int d = 0; d < 3; ++d) {
        nrm[12 * e + 3 * f + d] = sg * cr[d] / ar;
        fcen[12 * e + 3 * f + d] = (A[d] + Bv[d] + C[d]) / 3.0;
      }
      area[4 * e + f] = 0.5 * ar;
      asum += 0.5 * ar;
    }
    h[e] = 6.0 * (det / 6.0) / asum;  // insphere diameter 2 r_in = 6 V / sum(A)
  }

  // ---- face connectivity: interior/fault by vertex triples, periodic by partner
  plan.nbr.assign(4 * E, -1); plan.nface.assign(4 * E, -1); plan.nperm.assign(4 * E, -1);
  std::vector<int64_t>& nbr_u = plan.nbr;
  std::vector<int>&nface_u = plan.nface, &nperm_u = plan.nperm;
  {
    // match interior/fault faces by their sorted vertex triples: sort all
    // triples, then equal neighbours in the sorted list are the two sides
    struct FK {
      int64_t v0, v1, v2, id;
    };
    std::vector<FK> keys;
    keys.reserve((size_t)(4 * E));
    for (int64_t e = 0; e < E; ++e)
      for (int f = 0; f < 4; ++f) {
        int tg = tag[4 * e + f];
        if (tg < 0 || tg > 6) throw Err(ADG_E_MESH, "unknown face tag");
        if (tg != ADG_TAG_INTERIOR && tg != ADG_TAG_FAULT) continue;
        int64_t v[3] = {tets[4 * e + kFaceV[f][0]], tets[4 * e + kFaceV[f][1]], tets[4 * e + kFaceV[f][2]]};
        std::sort(v, v + 3);
        keys.push_back({v[0], v[1], v[2], 4 * e + f});
      }
    auto less = [](const FK& a, const FK& b) {
      if (a.v0 != b.v0) return a.v0 < b.v0;
      if (a.v1 != b.v1) return a.v1 < b.v1;
      if (a.v2 != b.v2) return a.v2 < b.v2;
      return a.id < b.id;
    };
    std::sort(keys.begin(), keys.end(), less);
    auto same = [](const FK& a, const FK& b) { return a.v0 == b.v0 && a.v1 == b.v1 && a.v2 == b.v2; };
    for (size_t k = 0; k < keys.size();) {
      if (k + 1 >= keys.size() || !same(keys[k], keys[k + 1]))
        throw Err(ADG_E_MESH, "interior face without a matching neighbour (tet " + std::to_string(keys[k].id / 4) + ")");
      if (k + 2 < keys.size() && same(keys[k], keys[k + 2])) throw Err(ADG_E_MESH, "face shared by more than two tets");
      const int64_t e = keys[k].id / 4, e2 = keys[k + 1].id / 4;
      const int f = (int)(keys[k].id % 4), f2 = (int)(keys[k + 1].id % 4);
      if (tag[4 * e2 + f2] != tag[4 * e + f]) throw Err(ADG_E_MESH, "fault face tagged on one side only");
      nbr_u[4 * e + f] = e2; nface_u[4 * e + f] = f2;
      nbr_u[4 * e2 + f2] = e; nface_u[4 * e2 + f2] = f;
      k += 2;
    }
    for (int64_t e = 0; e < E; ++e)
      for (int f = 0; f < 4; ++f) {
        if (tag[4 * e + f] != ADG_TAG_PERIODIC) continue;
        if (partner.empty()) throw Err(ADG_E_MESH, "periodic face without partner array");
        int64_t p = partner[4 * e + f];
        if (p < 0 || p >= 4 * E || tag[p] != ADG_TAG_PERIODIC) throw Err(ADG_E_MESH, "bad periodic partner");
        nbr_u[4 * e + f] = p / 4;
        nface_u[4 * e + f] = (int)(p % 4);
      }
    // orientation: node permutation so that my node n sits on the neighbour's node perm[n]
    for (int64_t e = 0; e < E; ++e)
      for (int f = 0; f < 4; ++f) {
        int64_t e2 = nbr_u[4 * e + f];
        if (e2 < 0) continue;
        int f2 = nface_u[4 * e + f];
        int sig[3];
        for (int s = 0; s < 3; ++s) {
          int64_t gv = tets[4 * e + kFaceV[f][s]];
          sig[s] = -1;
          if (tag[4 * e + f] == ADG_TAG_PERIODIC) {
            double sh[3];
            for (int d = 0; d < 3; ++d) sh[d] = fcen[12 * e2 + 3 * f2 + d] - fcen[12 * e + 3 * f + d];
            double best = 1e300;
            for (int s2 = 0; s2 < 3; ++s2) {
              const double* X = &xyz[3 * tets[4 * e2 + kFaceV[f2][s2]]];
              double dd = 0;
              for (int d = 0; d < 3; ++d) { double df = X[d] - (xyz[3 * gv + d] + sh[d]); dd += df * df; }
              if (dd < best) { best = dd; sig[s] = s2; }
            }
          } else {
            for (int s2 = 0; s2 < 3; ++s2)
              if (tets[4 * e2 + kFaceV[f2][s2]] == gv) sig[s] = s2;
          }
        }
        int pid = -1;
        for (int p = 0; p < 6; ++p)
          if (o.vperm[3 * p] == sig[0] && o.vperm[3 * p + 1] == sig[1] && o.vperm[3 * p + 2] == sig[2]) pid = p;
        if (pid < 0) throw Err(ADG_E_MESH, "could not orient a face pair");
        nperm_u[4 * e + f] = pid;
      }
  }

  // ---- CFL time steps and rate-2 clusters (Sec. 4.4)
  plan.dte.assign(E, 0.0);
  std::vector<double>& dte = plan.dte;
  double& dt_min = plan.dtmin;
  dt_min = 1e300;
  for (int64_t e = 0; e < E; ++e) {
    double cp = std::sqrt((lam[e] + 2 * mu[e]) / rho[e]);
    if (!(cp > 0) || !(rho[e] > 0) || mu[e] < 0) throw Err(ADG_E_INVALID, "bad material");
    dte[e] = cfg.cfl / (2 * degree + 1) * h[e] / cp;
    dt_min = std::min(dt_min, dte[e]);
  }
  plan.cl.assign(E, 0);
  std::vector<int>& cl = plan.cl;
  const int cmaxcap = std::max(1, std::min(cfg.max_clusters, 16)) - 1;
  for (int64_t e = 0; e < E; ++e) {
    int c = (int)std::floor(std::log2(dte[e] / dt_min) + 1e-12);
    cl[e] = std::max(0, std::min(c, cmaxcap));
  }
  for (bool changed = true; changed;) {
    changed = false;
    for (int64_t e = 0; e < E; ++e)
      for (int f = 0; f < 4; ++f) {
        int64_t e2 = nbr_u[4 * e + f];
        if (e2 < 0) continue;
        int lim = tag[4 * e + f] == ADG_TAG_FAULT ? cl[e2] : cl[e2] + 1;
        if (cl[e] > lim) { cl[e] = lim; changed = true; }
      }
  }
  plan.ncl = 0;
  for (int64_t e = 0; e < E; ++e) plan.ncl = std::max(plan.ncl, cl[e] + 1);
}

// The flux matrices setup() builds for face f of user tet eu (global frame,
// row-major): interior and periodic faces Fm, Fp; free, rigid and absorbing
// faces Fm (Fp zero); gravitational and fault faces zero (their fluxes come
// from the (eta, H) ODE and the friction solve).
void Ctx::face_flux(const MeshPlan& pl, int64_t eu, int f, double* Fm, double* Fp) const {
  M9 FmM{}, FpM{};
  const int tg = tag[4 * eu + f];
  const double Zpm = std::sqrt(rho[eu] * (lam[eu] + 2 * mu[eu])), Zsm = std::sqrt(rho[eu] * mu[eu]);
  M9 T, Ti;
  rot_mats(&pl.nrm[12 * eu + 3 * f], T, Ti);
  const M9 TA = mm(T, jac_x(rho[eu], lam[eu], mu[eu]));
  if (tg == ADG_TAG_INTERIOR || tg == ADG_TAG_PERIODIC) {
    const int64_t e2u = pl.nbr[4 * eu + f];
    const double Zpp = std::sqrt(rho[e2u] * (lam[e2u] + 2 * mu[e2u])), Zsp = std::sqrt(rho[e2u] * mu[e2u]);
    godunov_pair(TA, Ti, Zpm, Zpp, Zsm, Zsp, FmM, FpM);
  } else if (tg == ADG_TAG_FREE || tg == ADG_TAG_RIGID || tg == ADG_TAG_ABSORB) {
    FmM = boundary_matrix(TA, Ti, Zpm, Zsm, tg);
  }
  if (Fm) std::copy(FmM.begin(), FmM.end(), Fm);
  if (Fp) std::copy(FpM.begin(), FpM.end(), Fp);
}

// Face f of user tet eu seen from its neighbour (interior, periodic and fault
// faces): the neighbour tet and local face, and node_map[n] = the neighbour's
// face node at the place of my face node n (the permutation the neighbour
// kernel applies to the neighbour's trace); nb = -1 for faces without one.
void Ctx::face_neighbour(const MeshPlan& pl, const RefOps& o, int64_t eu, int f, int64_t* nb, int* nf,
                         int32_t* node_map) const {
  const int64_t e2 = pl.nbr[4 * eu + f];
  if (nb) *nb = e2;
  if (nf) *nf = e2 < 0 ? -1 : pl.nface[4 * eu + f];
  if (e2 < 0 || !node_map) return;
  const int pid = pl.nperm[4 * eu + f];
  for (int n = 0; n < o.Bf; ++n) node_map[n] = o.perm[(size_t)pid * o.Bf + n];
}

void Ctx::setup() {
  if (!has_mesh || !has_mat) throw Err(ADG_E_STATE, "upload mesh and material before adg_init");
  CK(cudaSetDevice(cfg.device));
  const int64_t E = nt;
  N = cfg.degree;
  S = cfg.ensemble;
  fp64 = cfg.precision == ADG_FP64;
  tc = cfg.precision == ADG_3XTF32 && (cfg.degree == 5 || cfg.degree == 4);
  ops = make_ref_ops(N);
  if (ops.max_orth_err > 1e-12) throw Err(ADG_E_INVALID, "reference basis not orthonormal");
  B = ops.B; Bf = ops.Bf; B1 = ops.B1;

  MeshPlan pl;
  plan_mesh(ops, N, pl);
  const std::vector<double>&Jinv = pl.Jinv, &detJ = pl.detJ, &area = pl.area, &nrm = pl.nrm;
  const std::vector<int64_t>& nbr_u = pl.nbr;
  const std::vector<int>&nface_u = pl.nface, &nperm_u = pl.nperm, &cl = pl.cl;
  dtmin = pl.dtmin;
  ncl = pl.ncl;
  // ---- internal order: by cluster, stable; with the tensor-core kernels,
  // the elements of a cluster without gravitational face, fault face or
  // finer neighbour come first (those with a coarser neighbour, which the
  // tensor-core kernels handle at some extra cost, at the end of that range,
  // so that they fill few tiles)
  // (special: 1 a coarser neighbour, 3 one gravitational face or a finer
  // neighbour (both on the tensor-core kernels, 3 on their special local
  // instantiation), 2 the CUDA-core kernels: a fault face or more than one
  // gravitational face)
  std::vector<char> special(E, 0), lts_face(E, 0);
  if (tc)
    for (int64_t e = 0; e < E; ++e) {
      int ng_e = 0;
      bool cc = false, coarser = false, finer = false;
      for (int f = 0; f < 4; ++f) {
        const int tg = tag[4 * e + f];
        const int64_t e2 = nbr_u[4 * e + f];
        ng_e += tg == ADG_TAG_GRAVITY;
        cc = cc || tg == ADG_TAG_FAULT;
        coarser = coarser || (e2 >= 0 && cl[e2] > cl[e]);
        finer = finer || (e2 >= 0 && cl[e2] < cl[e]);
      }
      special[e] = (cc || ng_e > 1) ? 2 : ((ng_e == 1 || finer) ? 3 : (coarser ? 1 : 0));
      lts_face[e] = coarser || finer;
    }
  // order key within a cluster: 0 plain elastic, 1 plain fluid on the
  // acoustic local kernel, 2 with a coarser neighbour, 3 with a gravitational
  // face or a finer neighbour (all four on the tensor-core kernels), 4 the
  // CUDA-core rest
  std::vector<char> key(E, 0);
  for (int64_t e = 0; e < E; ++e)
    key[e] = special[e] == 1 ? 2 : special[e] == 3 ? 3 : special[e] == 2 ? 4
                                 : (char)(tc && acoustic && mu[e] == 0.0 ? 1 : 0);
  order.resize(E);
  for (int64_t e = 0; e < E; ++e) order[e] = e;
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    return cl[a] != cl[b] ? cl[a] < cl[b] : key[a] < key[b];
  });
  inv.assign(E, 0);
  for (int64_t i = 0; i < E; ++i) inv[order[i]] = i;
  cl_begin.assign(ncl + 1, 0);
  cl_plain.assign(ncl, 0);
  cl_elastic.assign(ncl, 0);
  cl_fluid.assign(ncl, 0);
  cl_grav.assign(ncl, 0);
  cl_tc_lts.assign(ncl, 0);
  for (int64_t i = 0; i < E; ++i) {
    const int k = key[order[i]], c = cl[order[i]];
    cl_begin[c + 1]++;
    if (tc && k < 4) cl_plain[c]++;
    if (tc && k == 0) cl_elastic[c]++;
    if (tc && k == 1) cl_fluid[c]++;
    if (tc && k == 3) cl_grav[c]++;
    if (tc && (k == 2 || k == 3) && lts_face[order[i]]) cl_tc_lts[c] = 1;  // (the neighbour kernel's LTS-face code)
  }
  for (int c = 0; c < ncl; ++c) cl_begin[c + 1] += cl_begin[c];
  cluster.resize(E);
  for (int64_t i = 0; i < E; ++i) cluster[i] = cl[order[i]];

  // ---- per-element / per-face device data (internal order)
  std::vector<double> par((size_t)E * PAR), Fm((size_t)E * 324, 0.0), Fp((size_t)E * 324, 0.0);
  std::vector<float> frec(tc ? (size_t)E * 4 * FREC : 0, 0.f);
  std::vector<int> nbr((size_t)E * 4, -1), ninfo((size_t)E * 4, 0), gslot((size_t)E * 4, -1),
      bslot(E, -1), dslot((size_t)E * 4, -1);
  std::vector<double> gpar;
  gfaces.clear();
  int nb_slots = 0, nd_slots = 0, ng = 0;
  // gravity faces in increasing user (tet*4+face) order
  for (int64_t eu = 0; eu < E; ++eu)
    for (int f = 0; f < 4; ++f)
      if (tag[4 * eu + f] == ADG_TAG_GRAVITY) gfaces.push_back(4 * eu + f);
  for (size_t g = 0; g < gfaces.size(); ++g) {
    int64_t eu = gfaces[g] / 4;
    gslot[inv[eu] * 4 + gfaces[g] % 4] = (int)g;
  }
  ng = (int)gfaces.size();
  gpar.assign((size_t)ng * GPAR, 0.0);
  // per element in parallel; LTS/fault slots are flagged here and numbered in
  // element order afterwards
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t i = 0; i < E; ++i) {
    const int64_t eu = order[i];
    for (int k = 0; k < 9; ++k) par[i * PAR + k] = Jinv[9 * eu + k];
    par[i * PAR + 9] = rho[eu];
    par[i * PAR + 10] = lam[eu];
    par[i * PAR + 11] = mu[eu];
    for (int f = 0; f < 4; ++f) par[i * PAR + 12 + f] = 2.0 * area[4 * eu + f] / detJ[eu];
    const double Zpm = std::sqrt(rho[eu] * (lam[eu] + 2 * mu[eu])), Zsm = std::sqrt(rho[eu] * mu[eu]);
    const M9 Am = jac_x(rho[eu], lam[eu], mu[eu]);
    bool has_coarse = false;
    for (int f = 0; f < 4; ++f) {
      const double* n = &nrm[12 * eu + 3 * f];
      M9 T, Ti;
      rot_mats(n, T, Ti);
      const M9 TA = mm(T, Am);
      const int tg = tag[4 * eu + f];
      M9 Mm, Mp, FmM{}, FpM{};
      int kind = NK_NONE;
      float* rec = tc ? &frec[((size_t)i * 4 + f) * FREC] : nullptr;
      if (rec) {
        for (int d = 0; d < 3; ++d) rec[d] = (float)n[d];
        rec[5] = (float)(tg == ADG_TAG_FREE ? FACE_FREE
                         : tg == ADG_TAG_RIGID ? FACE_RIGID
                         : tg == ADG_TAG_ABSORB ? FACE_ABSORB : FACE_NEIGHBOUR);
      }
      if (tg == ADG_TAG_INTERIOR || tg == ADG_TAG_PERIODIC) {
        const int64_t e2u = nbr_u[4 * eu + f];
        const double Zpp = std::sqrt(rho[e2u] * (lam[e2u] + 2 * mu[e2u])), Zsp = std::sqrt(rho[e2u] * mu[e2u]);
        if (rec) {
          rec[3] = (float)Zpp;
          rec[4] = (float)Zsp;
        }
        godunov_pair(TA, Ti, Zpm, Zpp, Zsm, Zsp, FmM, FpM);
        const int64_t e2 = inv[e2u];
        nbr[i * 4 + f] = (int)e2;
        const int c1 = cluster[i], c2 = cluster[e2];
        kind = c1 == c2 ? NK_SAME : (c2 > c1 ? NK_COARSE : NK_FINE);
        if (kind == NK_COARSE) has_coarse = true;
        if (kind == NK_FINE) dslot[i * 4 + f] = 1;
        ninfo[i * 4 + f] = nface_u[4 * eu + f] | (nperm_u[4 * eu + f] << 2) | (kind << 5);
      } else if (tg == ADG_TAG_GRAVITY) {
        if (rec) {
          const int g = gslot[i * 4 + f];
          rec[5] = (float)FACE_GRAVITY;
          std::memcpy(&rec[6], &g, sizeof(int));
        }
        middle_state(Zpm, Zpm, Zsm, Zsm, Mm, Mp);
        // time-integrated middle state: w1 = -rho g H, w7 = eta^{n+1}-eta^n, w4 = w6 = 0,
        // w8/w9 = w8/w9 - w4/w6 / Z_s (solid) ; Fg applies the shear part to int q^-
        M9 Sm{};
        const int pairs[2][2] = {{3, 7}, {5, 8}};
        for (auto& pr : pairs) {
          Sm[pr[1] * 9 + pr[1]] = 1;
          if (Zsm > 0) Sm[pr[1] * 9 + pr[0]] = -1.0 / Zsm;
        }
        const M9 Fg = mm(mm(TA, Sm), Ti);
        const int g = gslot[i * 4 + f];
        double* gp = &gpar[(size_t)g * GPAR];
        gp[0] = n[0]; gp[1] = n[1]; gp[2] = n[2];
        gp[3] = Zpm;
        gp[4] = rho[eu] * cfg.gravity / Zpm;
        gp[5] = rho[eu] * cfg.gravity;
        for (int k = 0; k < 81; ++k) gp[6 + k] = Fg[k];
        for (int q = 0; q < 9; ++q) { gp[87 + q] = TA[q * 9 + 0]; gp[96 + q] = TA[q * 9 + 6]; }
      } else if (tg == ADG_TAG_FAULT) {
        kind = NK_FAULT;  // flux supplied by the rupture solver from both sides' derivative traces
        dslot[i * 4 + f] = 1;
        nbr[i * 4 + f] = (int)inv[nbr_u[4 * eu + f]];
        ninfo[i * 4 + f] = nface_u[4 * eu + f] | (nperm_u[4 * eu + f] << 2) | (kind << 5);
      } else {
        FmM = boundary_matrix(TA, Ti, Zpm, Zsm, tg);  // free, rigid, absorbing
      }
      for (int k = 0; k < 81; ++k) {
        Fm[(i * 4 + f) * 81 + k] = FmM[k];
        Fp[(i * 4 + f) * 81 + k] = FpM[k];
      }
    }
    if (has_coarse) bslot[i] = 1;
  }
  for (int64_t i = 0; i < E; ++i) {
    if (bslot[i] == 1) bslot[i] = nb_slots++;
    for (int f = 0; f < 4; ++f)
      if (dslot[i * 4 + f] == 1) dslot[i * 4 + f] = nd_slots++;
  }
  n_bslots = nb_slots;
  n_dslots = nd_slots;
  n_gslots = ng;
  // the tensor-core kernels handle same-cluster and coarser neighbours and
  // linear boundaries: check that the ordering gave them nothing else
  if (tc)
    for (int c = 0; c < ncl; ++c)
      for (int64_t i = cl_begin[c]; i < cl_begin[c] + cl_plain[c]; ++i) {
        // (the last cl_grav[c] of them may have one gravitational face and faces
        // with a finer neighbour)
        const bool spec = i >= cl_begin[c] + cl_plain[c] - cl_grav[c];
        bool ok = true;
        int ngf = 0;
        for (int f = 0; f < 4; ++f) {
          const int kind = (ninfo[i * 4 + f] >> 5) & 7;
          ngf += gslot[i * 4 + f] >= 0;
          ok = ok && (kind == NK_SAME || kind == NK_NONE || kind == NK_COARSE || (spec && kind == NK_FINE)) &&
               (dslot[i * 4 + f] < 0 || (spec && kind == NK_FINE));
        }
        ok = ok && ngf <= (spec ? 1 : 0);
        if (!ok) throw Err(ADG_E_STATE, "internal: element order for the tensor-core kernels is inconsistent");
      }
  // ---- fault faces: one entry per tet pair, minus side = lower user tet index,
  // listed in internal (cluster) order; both sides share a cluster by construction
  fface.clear(); fgeo.clear(); fminus_user.clear(); fplus_user.clear();
  std::vector<int> fslot((size_t)E * 4, -1);
  fcl_begin.assign(ncl + 1, 0);
  for (int64_t i = 0; i < E; ++i) {
    const int64_t eu = order[i];
    for (int f = 0; f < 4; ++f) {
      if (tag[4 * eu + f] != ADG_TAG_FAULT) continue;
      const int64_t e2u = nbr_u[4 * eu + f];
      if (e2u < eu) continue;  // listed from the minus side
      const int f2 = nface_u[4 * eu + f];
      const int64_t e2 = inv[e2u];
      const int64_t fi = (int64_t)fface.size() / 5;
      fface.insert(fface.end(), {(int)i, f, (int)e2, f2, nperm_u[4 * eu + f]});
      fslot[i * 4 + f] = (int)(2 * fi);
      fslot[e2 * 4 + f2] = (int)(2 * fi + 1);
      fminus_user.push_back(4 * eu + f);
      fplus_user.push_back(4 * e2u + f2);
      const double* n = &nrm[12 * eu + 3 * f];
      fgeo.insert(fgeo.end(), {n[0], n[1], n[2], rho[eu], lam[eu], mu[eu], rho[e2u], lam[e2u], mu[e2u]});
      if (!(mu[eu] > 0 && mu[e2u] > 0)) throw Err(ADG_E_MESH, "fault faces must separate two solids");
      fcl_begin[cluster[i] + 1]++;
    }
  }
  nff = (int64_t)fface.size() / 5;
  for (int c = 0; c < ncl; ++c) fcl_begin[c + 1] += fcl_begin[c];
  n_fault_faces = nff;
  fault_set = false;

  // ---- reference operators in device layouts (l-major / n-major)
  std::vector<double> ktT((size_t)3 * B * B), kvolT((size_t)3 * B1 * B), efcT((size_t)4 * B * Bf),
      liftT((size_t)4 * Bf * B);
  for (int a = 0; a < 3; ++a)
    for (int m = 0; m < B; ++m) {
      for (int l = 0; l < B; ++l) ktT[((size_t)a * B + l) * B + m] = ops.kt[((size_t)a * B + m) * B + l];
      for (int l = 0; l < B1; ++l) kvolT[((size_t)a * B1 + l) * B + m] = ops.kvol[((size_t)a * B + m) * B1 + l];
    }
  for (int f = 0; f < 4; ++f)
    for (int n = 0; n < Bf; ++n)
      for (int l = 0; l < B; ++l) {
        efcT[((size_t)f * B + l) * Bf + n] = ops.efc[((size_t)f * Bf + n) * B + l];
        liftT[((size_t)f * Bf + n) * B + l] = ops.lift[((size_t)f * B + l) * Bf + n];
      }

  // ---- device allocations
  if (cfg.cuda_stream) {
    stream = (cudaStream_t)cfg.cuda_stream;
  } else {
    CK(cudaStreamCreateWithFlags(&own_stream, cudaStreamNonBlocking));
    stream = own_stream;
  }
  const size_t ts = fp64 ? 8 : 4;
  const int64_t V = E * S;
  dQ = dalloc((size_t)V * 9 * B * ts, owned, dev_bytes);
  dTrace = dalloc((size_t)V * 4 * face_stride(N) * ts, owned, dev_bytes);
  dOrder = upload_raw(order, owned, dev_bytes);
  dBtrace = (double*)dalloc((size_t)nb_slots * S * 36 * Bf * 8, owned, dev_bytes);
  dDtrace = dalloc((size_t)nd_slots * S * (N + 1) * 9 * Bf * ts, owned, dev_bytes);
  dEta = (double*)dalloc((size_t)ng * S * Bf * 8, owned, dev_bytes);
  dGflux = dalloc((size_t)ng * S * 9 * Bf * ts, owned, dev_bytes);
  if (fp64) {
    dPar = upload_vec<double>(par, owned, dev_bytes);
    dFm = upload_vec<double>(Fm, owned, dev_bytes);
    dFp = upload_vec<double>(Fp, owned, dev_bytes);
    dKt = upload_vec<double>(ktT, owned, dev_bytes);
    dKvol = upload_vec<double>(kvolT, owned, dev_bytes);
    dEfc = upload_vec<double>(efcT, owned, dev_bytes);
    dLift = upload_vec<double>(liftT, owned, dev_bytes);
  } else {
    dPar = upload_vec<float>(par, owned, dev_bytes);
    dFm = upload_vec<float>(Fm, owned, dev_bytes);
    dFp = upload_vec<float>(Fp, owned, dev_bytes);
    dKt = upload_vec<float>(ktT, owned, dev_bytes);
    dKvol = upload_vec<float>(kvolT, owned, dev_bytes);
    dEfc = upload_vec<float>(efcT, owned, dev_bytes);
    dLift = upload_vec<float>(liftT, owned, dev_bytes);
  }
  dNbr = upload_raw<int>(nbr, owned, dev_bytes);
  dNinfo = upload_raw<int>(ninfo, owned, dev_bytes);
  dGslot = ng ? upload_raw<int>(gslot, owned, dev_bytes) : nullptr;
  dBslot = nb_slots ? upload_raw<int>(bslot, owned, dev_bytes) : nullptr;
  dDslot = nd_slots ? upload_raw<int>(dslot, owned, dev_bytes) : nullptr;
  dGpar = ng ? upload_raw<double>(gpar, owned, dev_bytes) : nullptr;
  dPerm = upload_raw<int>(ops.perm, owned, dev_bytes);
  CK(cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, cfg.device));
  if (tc) {
    std::vector<float> tl(local_tc_floats(N));
    pack_local_tc(N, ops.kt.data(), ops.kvol.data(), ops.efc.data(), tl.data());
    dTcLocal = upload_raw<float>(tl, owned, dev_bytes);
    std::vector<float> tf(lift_tc_floats(N));
    pack_lift_tc(N, ops.lift.data(), tf.data());
    dTcLift = upload_raw<float>(tf, owned, dev_bytes);
    dFrec = upload_raw<float>(frec, owned, dev_bytes);
    int64_t ngrav = 0;
    for (int c = 0; c < ncl; ++c) ngrav += cl_grav[c];
    if (ngrav > 0 && n_gslots > 0)
      dGscr = (float*)dalloc((size_t)n_gslots * S * gscr_floats(N) * sizeof(float), owned, dev_bytes);
  }
  dErr = (unsigned int*)dalloc(sizeof(unsigned int), owned, dev_bytes);
  if (acoustic) {
    std::vector<int64_t> fl;
    for (int64_t i = 0; i < E; ++i)
      if (mu[order[i]] == 0.0) fl.push_back(i);
    n_fluid = (int64_t)fl.size();
    dFluid = n_fluid ? upload_raw<int64_t>(fl, owned, dev_bytes) : nullptr;
  }
  if (nff) {
    dFface = upload_raw<int>(fface, owned, dev_bytes);
    dFslot = upload_raw<int>(fslot, owned, dev_bytes);
    dFgeo = upload_raw<double>(fgeo, owned, dev_bytes);
    dFpar = (double*)dalloc((size_t)nff * S * Bf * FPAR * 8, owned, dev_bytes);
    dFstate = (double*)dalloc((size_t)nff * S * Bf * FSTATE * 8, owned, dev_bytes);
    dDrout = dalloc((size_t)nff * S * 2 * 9 * Bf * ts, owned, dev_bytes);
    dNewton = (unsigned long long*)dalloc(2 * sizeof(unsigned long long), owned, dev_bytes);
    dMlp = (float*)dalloc(MLP_NPARAM * sizeof(float), owned, dev_bytes);
    dCapCount = (unsigned long long*)dalloc(sizeof(unsigned long long), owned, dev_bytes);
  }
  // configure kernels once (outside any stream capture)
  StepArgs a0 = base_args();
  const Segs none = make_segs(nullptr, 0, 1);
  int rc = launch_local(fp64, N, a0, none, stream);
  if (!rc && tc) rc = launch_local_tc(N, a0, none, n_sms, stream, false);
  if (!rc && tc) rc = launch_neighbour_tc(N, a0, none, n_sms, stream, false);
  if (rc) throw Err(ADG_E_CUDA, std::string("kernel configuration: ") + cudaGetErrorString((cudaError_t)rc));
  tick = 0;
  time = 0.0;
  inited = true;
}

StepArgs Ctx::base_args() const {
  StepArgs a{};
  a.Q = dQ; a.trace = dTrace; a.btrace = dBtrace; a.dtrace = dDtrace; a.eta = dEta;
  a.par = dPar; a.Fm = dFm; a.Fp = dFp; a.nbr = dNbr; a.ninfo = dNinfo;
  a.gslot = dGslot; a.bslot = dBslot; a.dslot = dDslot;
  a.ktT = dKt; a.kvolT = dKvol; a.efcT = dEfc; a.liftT = dLift; a.perm = dPerm; a.gpar = dGpar;
  a.S = S; a.err = dErr;
  a.fslot = dFslot; a.drout = dDrout; a.gflux = dGflux; a.tc_local = dTcLocal; a.tc_lift = dTcLift;
  a.frec = dFrec; a.gscr = dGscr;
  return a;
}

static void taylor_int(int N, double ta, double tb, double* out) {
  double fa = ta, fb = tb, fac = 1;
  for (int k = 0; k <= N; ++k) {
    fac *= (k + 1);
    out[k] = (fb - fa) / fac;
    fa *= ta;
    fb *= tb;
  }
}

// Launch the work of tick s of the rate-2 schedule with fine step dtm (Sec.
// 4.4): first the local phase of every cluster that starts a step at this
// tick, then the friction solves and the neighbour phase of every cluster
// that ends one.  Each phase is one launch per kernel kind covering all its
// clusters (a segment per cluster with that cluster's step and coefficients):
// the tensor-core kernels take the plain elements, the CUDA-core kernels the
// rest (all elements without the tensor-core form).
void Ctx::launch_tick(int s, double dtm) {
  StepArgs a = base_args();
  for (int phase = 0; phase < 2; ++phase) {
    // per kernel kind the clusters' segments: tensor-core elastic, tensor-core
    // acoustic and gravitational-face (local phase only), CUDA-core
    // (tcb: the local phase's elements with a coarser neighbour outside the
    // special range, on the instantiation with the LTS-buffer code)
    std::vector<Seg> tcs, tcb, fls, grs, ccs;
    bool ltsf = false;
    for (int c = 0; c < ncl; ++c) {
      const bool active = phase == 0 ? s % (1 << c) == 0 : (s + 1) % (1 << c) == 0;
      const int64_t n = cl_begin[c + 1] - cl_begin[c];
      if (!active || !n) continue;
      const double dt = (double)(1 << c) * dtm;
      Seg sg{};
      sg.dt = dt;
      if (phase == 0) {
        taylor_int(N, 0.0, dt, sg.tcoef);
        sg.btrace_mode = (s % (1 << (c + 1)) == 0) ? 1 : 2;
      } else {
        // position of this step inside the coarser neighbour's (2x longer) step
        const int half = ((s + 1) / (1 << c) - 1) % 2;
        taylor_int(N, half * dt, (half + 1) * dt, sg.ccoef);
        if (fcl_begin.size() > (size_t)c + 1 && fcl_begin[c + 1] > fcl_begin[c]) launch_rupture_cluster(c, dt);
      }
      auto seg = [&](int64_t first, int64_t count) {
        Seg t = sg;
        t.v_begin = first * S;
        t.n = count * S;
        return t;
      };
      const int64_t np = tc ? cl_plain[c] : 0;
      if (np > 0) {
        ltsf = ltsf || cl_tc_lts[c] != 0;
        const int64_t n0 = cl_elastic[c], n1 = cl_fluid[c], ng_c = cl_grav[c], n2 = np - ng_c - n0 - n1;
        if (phase == 0) {
          // plain elastic, acoustic, coarser-neighbour and special ranges, each on
          // its own kernel
          if (n0 > 0) tcs.push_back(seg(cl_begin[c], n0));
          if (n1 > 0) fls.push_back(seg(cl_begin[c] + n0, n1));
          if (n2 > 0) tcb.push_back(seg(cl_begin[c] + n0 + n1, n2));
          if (ng_c > 0) grs.push_back(seg(cl_begin[c] + np - ng_c, ng_c));
        } else {
          tcs.push_back(seg(cl_begin[c], np));
        }
      }
      if (n > np) ccs.push_back(seg(cl_begin[c] + np, n - np));
    }
    if (tcs.empty() && tcb.empty() && fls.empty() && grs.empty() && ccs.empty()) continue;
    ProfEv ev{phase, nullptr, nullptr, 0};
    if (prof) {
      CK(cudaEventCreate(&ev.a));
      CK(cudaEventCreate(&ev.b));
      CK(cudaEventRecord(ev.a, stream));
    }
    int rc = 0;
    // one launch per kind and at most kMaxSeg segments
    auto launch = [&](const std::vector<Seg>& v, int unit, auto&& fn) {
      for (size_t i = 0; i < v.size() && !rc; i += kMaxSeg) {
        const int k = (int)std::min<size_t>(kMaxSeg, v.size() - i);
        rc = fn(make_segs(v.data() + i, k, unit, unit == 1 ? 1 : tc_chunk[phase]));
        ev.launches++;
      }
    };
    launch(tcs, kTileElems, [&](const Segs& g) {
      return phase == 0 ? launch_local_tc(N, a, g, n_sms, stream, false)
                        : launch_neighbour_tc(N, a, g, n_sms, stream, ltsf);
    });
    launch(tcb, kTileElems, [&](const Segs& g) { return launch_local_tc(N, a, g, n_sms, stream, true); });
    launch(fls, kTileElemsFluid, [&](const Segs& g) { return launch_local_tc(N, a, g, n_sms, stream, false, true); });
    launch(grs, kTileElems,
           [&](const Segs& g) { return launch_local_tc(N, a, g, n_sms, stream, true, false, true); });
    if (prof && (!tcs.empty() || !tcb.empty() || !fls.empty() || !grs.empty())) {  // the tensor-core launches alone
      CK(cudaEventCreate(&ev.m));
      CK(cudaEventRecord(ev.m, stream));
    }
    launch(ccs, 1, [&](const Segs& g) {
      return phase == 0 ? launch_local(fp64, N, a, g, stream, cc_threads[0])
                        : launch_neighbour(fp64, N, a, g, stream, cc_threads[1]);
    });
    if (prof) { CK(cudaEventRecord(ev.b, stream)); prof->push_back(ev); }
    if (rc)
      throw Err(ADG_E_CUDA, std::string(phase == 0 ? "local kernel: " : "neighbour kernel: ") +
                                cudaGetErrorString((cudaError_t)rc));
  }
}

// Friction solve on the fault faces of cluster c over its step dt (before the
// neighbour kernel of that cluster, which lifts the fault fluxes).
void Ctx::launch_rupture_cluster(int c, double dt) {
  if (!fault_set) throw Err(ADG_E_STATE, "fault faces present: call adg_set_fault before stepping");
  DRArgs d{};
  d.dtrace = dDtrace; d.dslot = dDslot; d.fface = dFface; d.fgeo = dFgeo; d.fpar = dFpar;
  d.fstate = dFstate; d.drout = dDrout; d.perm = dPerm;
  d.f_begin = fcl_begin[c];
  d.n_faces = fcl_begin[c + 1] - fcl_begin[c];
  d.S = S;
  d.dt = dt;
  std::vector<double> x, w;
  gauss01(N + 1, x, w);
  for (int j = 0; j <= N; ++j) { d.tp[j] = dt * x[j]; d.tw[j] = dt * w[j]; }
  d.newton = dNewton; d.err = dErr;
  d.mlp = mlp_on ? dMlp : nullptr;
  d.capture = cap_on ? dCapture : nullptr;
  d.cap_count = dCapCount;
  d.cap_capacity = cap_capacity;
  d.law = fric_law;
  ProfEv ev{2, nullptr, nullptr, 1};
  if (prof) {
    CK(cudaEventCreate(&ev.a));
    CK(cudaEventCreate(&ev.b));
    CK(cudaEventRecord(ev.a, stream));
  }
  int rc = launch_rupture(fp64, N, d, stream);
  if (prof) { CK(cudaEventRecord(ev.b, stream)); prof->push_back(ev); }
  if (rc) throw Err(ADG_E_CUDA, std::string("rupture kernel: ") + cudaGetErrorString((cudaError_t)rc));
}

int64_t Ctx::launches_per_macro() const {
  int64_t L = 0;
  const int ticks = 1 << (ncl - 1);
  for (int s = 0; s < ticks; ++s)
    for (int phase = 0; phase < 2; ++phase) {
      bool tcl = false, tbl = false, fll = false, grl = false, ccl = false;
      for (int c = 0; c < ncl; ++c) {
        const int64_t n = cl_begin[c + 1] - cl_begin[c];
        if (!n || (phase == 0 ? s % (1 << c) : (s + 1) % (1 << c))) continue;
        if (phase == 1 && fcl_begin[c + 1] > fcl_begin[c]) L += 1;  // friction solve per cluster
        const int64_t np = tc ? cl_plain[c] : 0;
        if (phase == 0 && np > 0) {
          const int64_t n0 = cl_elastic[c], nf = cl_fluid[c], ngr = cl_grav[c];
          tcl = tcl || n0 > 0;
          fll = fll || nf > 0;
          tbl = tbl || np - ngr - n0 - nf > 0;
          grl = grl || ngr > 0;
        } else {
          tcl = tcl || np > 0;
        }
        ccl = ccl || n > np;
      }
      L += tcl + tbl + fll + grl + ccl;
    }
  return L;
}

void Ctx::project_fluid(bool sync) {
  if (!acoustic || !n_fluid) return;
  const int rc = launch_isotropic_fluid(fp64, dQ, dFluid, n_fluid, S * B, B, stream);
  if (rc) throw Err(ADG_E_CUDA, std::string("fluid projection: ") + cudaGetErrorString((cudaError_t)rc));
  if (sync) CK(cudaStreamSynchronize(stream));
}

void Ctx::aio_setup() {
  if (aio.in) return;  // (created last: everything else is in place)
  const size_t bytes = (size_t)nt * S * 9 * B * sizeof(float);
  for (int b = 0; b < 2; ++b) {
    if (!aio.dIn[b]) aio.dIn[b] = static_cast<float*>(dalloc(bytes, owned, dev_bytes));
    if (!aio.dOut[b]) aio.dOut[b] = static_cast<float*>(dalloc(bytes, owned, dev_bytes));
    for (cudaEvent_t* e : {&aio.in_copied[b], &aio.in_used[b], &aio.out_made[b], &aio.out_copied[b]})
      if (!*e) CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  if (!aio.out) CK(cudaStreamCreateWithFlags(&aio.out, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&aio.in, cudaStreamNonBlocking));
}

void Ctx::aio_sync() {
  if (aio.in) CK(cudaStreamSynchronize(aio.in));
  if (aio.out) CK(cudaStreamSynchronize(aio.out));
}

void Ctx::aio_free() {
  for (cudaStream_t st : {aio.in, aio.out})
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  for (int b = 0; b < 2; ++b)
    for (cudaEvent_t e : {aio.in_copied[b], aio.in_used[b], aio.out_made[b], aio.out_copied[b]})
      if (e) cudaEventDestroy(e);
  aio = AsyncIo{};  // (the staging buffers are among the owned allocations)
}

void Ctx::run_macro(double scale) {
  const int ticks = 1 << (ncl - 1);
  const double dtm = dtmin * scale;
  if (scale == 1.0 && use_graph) {
    if (!graph_exec) {
      cudaGraph_t g;
      CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
      try {
        for (int s = 0; s < ticks; ++s) launch_tick(s, dtm);
      } catch (...) {
        cudaStreamEndCapture(stream, &g);
        throw;
      }
      CK(cudaStreamEndCapture(stream, &g));
      CK(cudaGraphInstantiate(&graph_exec, g, 0));
      CK(cudaGraphDestroy(g));
    }
    CK(cudaGraphLaunch(graph_exec, stream));
  } else {
    for (int s = 0; s < ticks; ++s) launch_tick(s, dtm);
  }
  time += ticks * dtm;
}

// Cadence recording: after a macro step of adg_advance / adg_advance_to, take
// the samples that are due into their device ring slots on the library stream
// and queue each slot's copy to the pinned host ring on the recording stream.
void Ctx::record_after_macro() {
  for (int k = 0; k < 2; ++k) {
    Recorder& r = rec[k];
    if (!r.every || ++r.macro % r.every) continue;
    const int64_t slot = r.count % r.cap;
    if (r.count - r.read >= r.cap) {  // the oldest unread sample is overwritten
      r.read++;
      r.dropped++;
    }
    CK(cudaStreamWaitEvent(stream, r.copied[slot], 0));  // the slot's previous copy is done
    double* d = r.dRing + slot * r.sample;
    if (k == 0) {
      const int rc = launch_receivers(fp64, B, dQ, S, n_rec, dRecElem, dRecPhi, d, stream);
      if (rc) throw Err(ADG_E_CUDA, std::string("receiver kernel: ") + cudaGetErrorString((cudaError_t)rc));
    } else {
      CK(cudaMemcpyAsync(d, dEta, r.sample * 8, cudaMemcpyDeviceToDevice, stream));
    }
    CK(cudaEventRecord(r.taken[slot], stream));
    CK(cudaStreamWaitEvent(rec_stream, r.taken[slot], 0));
    CK(cudaMemcpyAsync(r.hRing + slot * r.sample, d, r.sample * 8, cudaMemcpyDeviceToHost, rec_stream));
    CK(cudaEventRecord(r.copied[slot], rec_stream));
    r.t[slot] = time;
    r.count++;
  }
}

void Ctx::record_free(int kind) {
  Recorder& r = rec[kind];
  if (rec_stream) cudaStreamSynchronize(rec_stream);
  if (r.dRing) cudaFree(r.dRing);
  if (r.hRing) cudaFreeHost(r.hRing);
  for (cudaEvent_t e : r.taken) cudaEventDestroy(e);
  for (cudaEvent_t e : r.copied) cudaEventDestroy(e);
  r = Recorder();
}

void Ctx::check_err() {
  CK(cudaStreamSynchronize(stream));
  unsigned int h = 0;
  CK(cudaMemcpy(&h, dErr, sizeof(h), cudaMemcpyDeviceToHost));
  if (h) {
    CK(cudaMemset(dErr, 0, sizeof(unsigned int)));
    if (h & ERR_NAN) throw Err(ADG_E_NAN, "non-finite dofs detected");
    if (h & ERR_NEWTON) throw Err(ADG_E_NEWTON, "friction Newton solve did not converge");
    if (h & ERR_TIMEOUT) throw Err(ADG_E_TIMEOUT, "bounded device wait ran out");
  }
}

Ctx::~Ctx() {
  record_free(0);
  record_free(1);
  aio_free();
  if (rec_stream) cudaStreamDestroy(rec_stream);
  if (graph_exec) cudaGraphExecDestroy(graph_exec);
  for (void* p : owned) cudaFree(p);
  if (hstage) cudaFreeHost(hstage);
  if (own_stream) cudaStreamDestroy(own_stream);
}

// Volume quadrature for projections: collapsed Gauss-Legendre, exact for degree deg.
void tet_rule(int deg, std::vector<double>& pts, std::vector<double>& w) {
  int n = std::max(1, (deg + 4) / 2);
  std::vector<double> x, wx;
  gauss01(n, x, wx);
  pts.clear();
  w.clear();
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        double u = x[i], v = x[j], s = x[k];
        pts.push_back(u * (1 - v) * (1 - s));
        pts.push_back(v * (1 - s));
        pts.push_back(s);
        w.push_back(wx[i] * wx[j] * wx[k] * (1 - v) * (1 - s) * (1 - s));
      }
}

}  // namespace adg

// ADER-DG element-update kernels (CUDA cores), templated on the working
// precision T (double or float) and the polynomial degree N.
//
// Per element v (virtual index; ensembles stack S scenarios per element) over
// one own step:
//   local kernel      Sec. 4.1: Cauchy-Kovalewski predictor
//                       D^{k+1} = -sum_a KT_a D^k A*_a^T,  KT_a[m][l] = int phi_m dphi_l/dxi_a,
//                     time integral I = sum_k dt^{k+1}/(k+1)! D^k (Eq. taylor),
//                     volume sum_a K_a I A*_a^T, its own nodal face traces
//                     (and LTS buffers / derivative traces); gravitational
//                     faces (Sec. 4.3): exact (eta, H) Taylor recursion in
//                     FP64 at the face nodes and that face's time-integrated
//                     flux from int w1^b = -rho g H and int w7^b = eta^{n+1} - eta^n.
//   neighbour kernel  Godunov fluxes of all four faces (Sec. 4.2, Eq.
//                     numerical-flux): F^- on the own traces, F^+ on the
//                     neighbours' (re-oriented by a node permutation), the
//                     stored fluxes of gravitational and fault faces; one lift.
// Dofs layout: Q[v][9][B] (basis fastest); traces [v][4][face_stride(N)], each face
// block [9][Bf] (node fastest) followed by padding.
#pragma once
#include <cstdint>

namespace adg {

__host__ __device__ constexpr int nb3(int n) { return n < 0 ? 0 : (n + 1) * (n + 2) * (n + 3) / 6; }
__host__ __device__ constexpr int nb2(int n) { return (n + 1) * (n + 2) / 2; }
// floats of one face's traces in the trace array: 9 x Bf values [quantity][node],
// padded to a multiple of 4 so that every face block starts on 16 bytes
__host__ __device__ constexpr int face_stride(int n) { return (9 * nb2(n) + 3) / 4 * 4; }

// neighbour-face kinds (ninfo bits 5..7)
enum { NK_NONE = 0, NK_SAME = 1, NK_COARSE = 2, NK_FINE = 3, NK_FAULT = 4 };

// per-element parameters (stride PAR): Jinv[9] (d xi_a/d x_d, row a), rho, lam, mu, scale[4]
constexpr int PAR = 16;
// per-gravity-face parameters (double, stride GPAR):
//   n[3], Z, kappa = rho g / Z, rho*g, Fg[81], a1[9], a7[9]
constexpr int GPAR = 6 + 81 + 18;

struct StepArgs {
  void* Q;              // T [V][9][B]
  void* trace;          // T [V][4][face_stride(N)]: [9][Bf] per face + padding
  double* btrace;       // [nbslot*S][4][9][Bf]  (LTS buffer, FP64)
  void* dtrace;         // T [ndslot*S][N+1][9][Bf] (LTS derivative traces)
  double* eta;          // [ngslot*S][Bf]
  const void* par;      // T [E][PAR]
  const void* Fm;       // T [E][4][81]  row-major F[q][p]
  const void* Fp;       // T [E][4][81]
  const int* nbr;       // [E][4] internal neighbour element or -1
  const int* ninfo;     // [E][4] j | perm<<2 | kind<<5
  const int* gslot;     // [E][4] gravity slot or -1
  const int* bslot;     // [E]    LTS buffer slot or -1
  const int* dslot;     // [E][4] LTS derivative-trace slot or -1
  const void* ktT;      // T [3][B(l)][B(m)]   KT_a[m][l] stored l-major
  const void* kvolT;    // T [3][B1(l)][B(m)]  K_a[m][l]  stored l-major
  const void* efcT;     // T [4][B(l)][Bf(n)]  phi_l at node n stored l-major
  const void* liftT;    // T [4][Bf(n)][B(m)]  lift[f][m][n] stored n-major
  const int* perm;      // [6][Bf]
  const double* gpar;   // [ngslot][GPAR]
  int S;                // ensemble size
  unsigned int* err;    // device error word
  const int* fslot;     // [E][4] 2*fault + side for fault faces, else -1
  const void* drout;    // T [nff*S][2][9][Bf] time-integrated fault flux per side
  void* gflux;          // T [ngslot*S][9][Bf] time-integrated flux of gravitational faces
  const float* tc_local; // tensor-core operands of the local kernel (hi/lo, canonical layout), degree 5 or 4
  const float* tc_lift;  // tensor-core lift operand of the neighbour kernel (hi/lo, canonical layout), degree 5 or 4
  const float* frec;     // [E][4][FREC] face records of the tensor-core neighbour kernel (FP32 dofs)
  float* gscr;           // [ngslot*S][gscr_floats(N)] scratch of the tensor-core local kernel's gravity faces
};
// Per gravity slot and scenario, the tensor-core local kernel's scratch: the
// normal-projected derivative rows g_m[l] = sum_p w_p D^m[p][l] (m = 0..N,
// l < B(N - m); w: v_n - sigma_nn / Z), then the own-trace flux part
// sum_p Fg[q][p] V[p][n] (q < 9, n < Bf).
__host__ __device__ constexpr int gscr_off(int n, int m) { return m <= 0 ? 0 : gscr_off(n, m - 1) + nb3(n - m + 1); }
__host__ __device__ constexpr int gscr_floats(int n) { return gscr_off(n, n + 1) + 9 * nb2(n); }

// Face record of the tensor-core neighbour kernel (floats): the outward unit
// normal n[3], the plus side's impedances Zp+, Zs+ (interior and periodic
// faces), the face code (FACE_* below), two zeros.  The kernel forms the
// Godunov flux of Sec. 4.2 from it and the element's own material.
constexpr int FREC = 8;
// (FACE_GRAVITY: a gravitational free surface; the record's seventh float
// holds the bits of its gravity slot, and the kernel lifts the flux the local
// kernel stored for it)
enum { FACE_NEIGHBOUR = 0, FACE_FREE = 1, FACE_RIGID = 2, FACE_ABSORB = 3, FACE_GRAVITY = 4 };

// The clusters of one LTS phase (Sec. 4.4) in a single launch: segment i
// covers the virtual elements [v_begin, v_begin + n) of one cluster with that
// cluster's time coefficients, and the launch's work units (tiles of the
// tensor-core kernels, blocks of the CUDA-core kernels) [first[i], first[i+1]).
// The launch takes the table by value (kernel parameter space), so a CUDA
// graph keeps it and no device buffer is involved.
constexpr int kMaxSeg = 16;
// virtual elements per tile of the tensor-core kernels (12 x 9 quantities =
// the 128 rows of one MMA)
constexpr int kTileElems = 12;
// ... and of the acoustic (4-quantity, ocean) instantiation of the local one
constexpr int kTileElemsFluid = 32;
struct Seg {
  int64_t v_begin, n;
  double tcoef[8];   // dt^{k+1}/(k+1)!, k = 0..N (the cluster's own step)
  double ccoef[8];   // (tb^{k+1}-ta^{k+1})/(k+1)! on a coarser neighbour's expansion
  double dt;         // the cluster's step (gravity ODE)
  int btrace_mode;   // 0 none, 1 overwrite, 2 accumulate (LTS buffers)
};
struct Segs {
  int n;                        // segments
  int chunk;                    // tensor-core kernels: consecutive tiles a CTA slot takes per sweep
  int64_t first[kMaxSeg + 1];   // first work unit of each segment; first[n] = all units
  Seg s[kMaxSeg];
};
// Tensor-core kernels: the i-th tile of slot `slot` (of `slots`, over all CTAs)
// when every slot takes `chunk` consecutive tiles per sweep; increasing in i.
// (Tile counts stay below 2^31.)
__host__ __device__ inline int slot_tile(int i, int slot, int slots, int chunk) {
  const int q = i / chunk;
  return (q * slots + slot) * chunk + (i - q * chunk);
}
// segment of work unit u (segments are few: a linear scan)
__host__ __device__ inline int seg_find(const Segs& g, int64_t u) {
  int i = 0;
  while (i + 1 < g.n && u >= g.first[i + 1]) ++i;
  return i;
}
// segment of work unit u in a launch that may have several (kMulti) or has one
template <bool kMulti>
__host__ __device__ inline int seg_of(const Segs& g, int64_t u) {
  return kMulti ? seg_find(g, u) : 0;
}
// Segs of the given segments with `unit` virtual elements per work unit
Segs make_segs(const Seg* s, int n, int unit, int chunk = 1);

// tensor-core (tcgen05, 3xTF32) local kernel, degree 5 or 4, FP32 dofs
// (local_tc.cuh; one translation unit per degree), for elements without
// gravitational faces, fault faces or finer LTS neighbours
// buffers: the launch's elements include some with an LTS buffer (a coarser neighbour)
// acoustic: the launch's elements are fluid (mu = 0) without LTS buffer, on the
// 4-quantity (p, v) instantiation; their stress must be isotropic (-p I)
// (other degrees: cudaErrorInvalidValue)
// grav: the launch's elements have one gravitational face or a finer LTS
// neighbour (elastic instantiation; the face's (eta, H) update in FP64 and
// the derivative traces of every level on faces with a finer neighbour)
int launch_local_tc(int degree, const StepArgs& a, const Segs& g, int n_sms, void* stream, bool buffers,
                    bool acoustic = false, bool grav = false);
void pack_local_tc(int degree, const double* kt, const double* kvol, const double* efc, float* out);
int local_tc_floats(int degree);
// tensor-core (tcgen05, 3xTF32) neighbour kernel, degree 5 or 4, FP32 dofs
// (neighbour_tc.cuh), for the same elements
// coarse: the launch's elements include some with a coarser LTS neighbour
int launch_neighbour_tc(int degree, const StepArgs& a, const Segs& g, int n_sms, void* stream, bool coarse);
void pack_lift_tc(int degree, const double* lift, float* out);
int lift_tc_floats(int degree);

// ---- dynamic rupture (rupture.cu) ----
// per-node fault parameters (double, stride FPAR), in this order:
//   a, b, L, f0, V0, f_w, V_w, sigma_n0, tau0_x, tau0_y, tau0_z, psi_init, V_init
// (linear slip weakening: mu_s, mu_d, D_c, cohesion in the first four slots)
constexpr int FPAR = 13;
// per-node fault state (double, stride FSTATE): |V|, psi, slip_xyz, traction_xyz
constexpr int FSTATE = 8;
// per-fault-face geometry (double, stride FGEO): n (minus outward), rho-, lam-, mu-, rho+, lam+, mu+
constexpr int FGEO = 9;
// friction-guess network: inputs, hidden width (two tanh layers), parameters
constexpr int MLP_IN = 6, MLP_H = 32;
constexpr int MLP_NPARAM = MLP_IN * MLP_H + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1 + 2 * MLP_IN + 2;

struct DRArgs {
  const void* dtrace;   // derivative traces of both sides (see StepArgs)
  const int* dslot;
  const int* fface;     // [nff][5] minus elem, minus face, plus elem, plus face, perm
  const double* fgeo;   // [nff][FGEO]
  const double* fpar;   // [nff*S][Bf][FPAR]
  double* fstate;       // [nff*S][Bf][FSTATE]
  void* drout;          // T [nff*S][2][9][Bf]
  const int* perm;      // [6][Bf]
  int64_t f_begin, n_faces;
  int S;
  double dt;
  double tp[8], tw[8];  // Gauss-Legendre time points / weights on [0, dt]
  unsigned long long* newton;  // [0] solves, [1] iterations
  unsigned int* err;
  const float* mlp;     // network parameters (or null: plain start)
  float* capture;       // training samples [cap][MLP_IN + 1] (or null)
  unsigned long long* cap_count;
  int64_t cap_capacity;
  int law;              // FRIC_RS or FRIC_LSW
};

enum { FRIC_RS = 0, FRIC_LSW = 1 };  // the ADG_FRICTION_* values of adg.h

int launch_rupture(int fp64, int N, const DRArgs& a, void* stream);

enum { ERR_NAN = 1u, ERR_TIMEOUT = 2u, ERR_NEWTON = 4u };

// host-side launchers (kernels_f64.cu / kernels_f32.cu); return cudaError_t as int
// (threads: per element block, a multiple of 32 up to 256)
int launch_local(int fp64, int N, const StepArgs& a, const Segs& g, void* stream, int threads = 128);
int launch_neighbour(int fp64, int N, const StepArgs& a, const Segs& g, void* stream, int threads = 128);
int local_smem_bytes(int fp64, int N);

}  // namespace adg

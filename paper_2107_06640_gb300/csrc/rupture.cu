// Dynamic-rupture friction solve (Sec. 3, Eq. bc-dynrup) on fault faces,
// FP64, one thread per fault node and scenario.
//
// Readings (the paper names fast-velocity-weakening rate and state friction
// but prints neither f nor g):
//   f(V, psi)  = a asinh(V/(2 V0) exp(psi/a))
//   dpsi/dt    = -(V/L)(psi - psi_ss(V)),  psi_ss = a ln((2V0/V) sinh(f_ss/a)),
//   f_ss       = f_w + (f0 - (b-a) ln(V/V0) - f_w) / (1 + (V/V_w)^8)^(1/8);
//   strength S = max(0, -(sigma_n0 + sigma_n^b)) with sigma_n^b the welded P
//   middle state; locked shear traction theta = eta_s [(u+ - u-) + tau+/Zs+ +
//   tau-/Zs-], eta_s = Zs- Zs+/(Zs- + Zs+); |V| solves
//   Theta - eta_s |V| = S f(|V|, psi), Theta = |tau0 + theta|, V parallel to
//   tau0 + theta.  Per step: N+1 Gauss-Legendre time points; at each, two
//   passes of [exact psi relaxation for a frozen slip rate (pass 0: the
//   previous one, pass 1: the mid-point of previous and pass-0 rates), Newton
//   on x = ln |V| clamped to [-700, ln(Theta/eta_s)], |dx| <= 1e-10]; the
//   learned guess only seeds the pass-0 Newton, so the answer does not
//   depend on it.
// Learned start (the paper has none): the network predicts ln V* - x_a, x_a
// the large-argument asymptote of asinh; at time points j >= 1 the pass-0
// Newton starts from the warm start plus the change of the predicted ln V*
// since point j-1 (exact where nothing changes), at j = 0 from the warm
// start; a start that fails falls back to the warm start.
// Linear slip weakening (law FRIC_LSW; the Scenario-A fault of Sec. 5, law of
// Andrews 1976): the parameter slots a, b, L, f0 hold mu_s, mu_d, D_c and the
// cohesion C; psi is the slip path length, dpsi/dt = |V|,
// f = mu_s - (mu_s - mu_d) min(psi/D_c, 1), strength tau_S = C + f S and
// |V| = max(0, Theta - tau_S)/eta_s in closed form, with the same time points
// and two passes (psi advanced exactly for a frozen slip rate: psi + |V| h).
// Output per fault face: the time-integrated flux n.(A,B,C) q^b for the minus
// element (minus node order) and -n.(A,B,C) q^c for the plus element (plus
// node order); the neighbour kernel lifts them.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace adg {

namespace {

constexpr double kTol = 1e-10;
constexpr int kMaxIter = 100;
constexpr double kXFloor = -700.0;

struct FricPar {
  double a, b, L, f0, V0, fw, Vw;
};

// (lnV = ln V, l2v0 = ln(2 V0): shared with the caller's other uses)
__device__ double f_ss(double V, double lnV, double l2v0, const FricPar& p) {
  const double fLV = p.f0 - (p.b - p.a) * (lnV - (l2v0 - 0.6931471805599453));
  const double r = V / p.Vw;
  const double r2 = r * r, r4 = r2 * r2, r8 = r4 * r4;
  // (1 + r8 rounds to 1 below 2^-53: the power is then exactly 1)
  return p.fw + (fLV - p.fw) / (r8 < 1e-17 ? 1.0 : pow(1.0 + r8, 0.125));
}

__device__ double psi_relax(double psi, double V, double h, double l2v0, const FricPar& p) {
  // exact solution of dpsi/dt = -(V/L)(psi - psi_ss(V)) for frozen V over h
  // (V floored at 1e-300: for V -> 0 the state does not change)
  V = fmax(V, 1e-300);
  const double lnV = log(V);
  const double x = f_ss(V, lnV, l2v0, p) / p.a;
  // ln sinh(x) = x + ln(1 - e^{-2x}) - ln 2; above x = 20 the middle term is below
  // half an ulp of x and the sum is x - ln 2 exactly
  const double lsinh = (x > 20.0 ? x : x + log1p(-exp(-2.0 * x))) - 0.6931471805599453;
  const double ss = p.a * ((l2v0 - lnV) + lsinh);
  return ss + (psi - ss) * exp(-V * h / p.L);
}

// Newton on x = ln V for Theta - eta V - S a asinh(c V) = 0 (decreasing, concave in x);
// lc = ln c = psi / a - ln(2 V0) and hi = ln(Theta / eta) (the root's upper
// bound) come from the caller, which shares them between the two passes and
// the network's features; *xout = the final x (ln V)
__device__ double newton_v(double Th, double S, double eta, double lc, double hi, const FricPar& p, double x0,
                           int* iters, bool* ok, double* xout) {
  *iters = 0;
  *ok = true;
  *xout = kXFloor;
  if (!(Th > 0)) return 0.0;
  if (S == 0.0) {
    *xout = hi;
    return Th / eta;
  }
  double x = fmin(fmax(x0, kXFloor), hi);
  for (int it = 0; it < kMaxIter; ++it) {
    const double V = exp(x);
    const double cv = exp(lc + x);
    const double g = Th - eta * V - S * p.a * asinh(cv);
    const double dg = -eta * V - S * p.a * cv / sqrt(1.0 + cv * cv);
    const double xn = fmin(fmax(x - g / dg, kXFloor), hi);
    const double step = fabs(xn - x);
    x = xn;
    if (step <= kTol) {
      *iters = it + 1;
      *xout = x;
      return exp(x);
    }
  }
  *iters = kMaxIter;
  *ok = false;
  *xout = x;
  return exp(x);
}

// n.(A,B,C) applied to a state with traction t = sigma n and velocity v
__device__ void ahat(const double n[3], const double t[3], const double v[3], double rho, double lam, double mu,
                     double sgn, double w, double* acc) {
  const double nv = n[0] * v[0] + n[1] * v[1] + n[2] * v[2];
  const int pi[6] = {0, 1, 2, 0, 1, 0}, pj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    double s = -mu * (n[pj[c]] * v[pi[c]] + n[pi[c]] * v[pj[c]]);
    if (c < 3) s -= lam * nv;
    acc[c] += sgn * w * s;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) acc[6 + i] += sgn * w * (-t[i] / rho);
}

__device__ void traction(const double q[9], const double n[3], double t[3]) {
  t[0] = q[0] * n[0] + q[3] * n[1] + q[5] * n[2];
  t[1] = q[3] * n[0] + q[1] * n[1] + q[4] * n[2];
  t[2] = q[5] * n[0] + q[4] * n[1] + q[2] * n[2];
}

__device__ __forceinline__ float tanh_hw(float x) {  // the hardware tanh approximation (MUFU)
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// friction-guess network (FP32, weights W in shared memory, 16-byte aligned
// rows): features -> predicted ln V* - x_a
__device__ float mlp_eval(const float* W, const float f[MLP_IN]) {
  const float* W1 = W;
  const float* b1 = W1 + MLP_IN * MLP_H;
  const float* W2 = b1 + MLP_H;
  const float* b2 = W2 + MLP_H * MLP_H;
  const float* w3 = b2 + MLP_H;
  const float* b3 = w3 + MLP_H;
  const float* mu = b3 + 1;
  const float* sd = mu + MLP_IN;
  const float* osc = sd + MLP_IN;  // output shift, scale
  float x[MLP_IN], h1[MLP_H];
#pragma unroll
  for (int i = 0; i < MLP_IN; ++i) x[i] = (f[i] - mu[i]) / sd[i];
#pragma unroll
  for (int j = 0; j < MLP_H; ++j) {
    float s = b1[j];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) s += W1[j * MLP_IN + i] * x[i];
    h1[j] = tanh_hw(s);
  }
  float y = b3[0];
#pragma unroll 4
  for (int j = 0; j < MLP_H; ++j) {
    const float4* w = reinterpret_cast<const float4*>(W2 + j * MLP_H);
    float s = b2[j];
#pragma unroll
    for (int i = 0; i < MLP_H / 4; ++i) {
      const float4 q = w[i];
      s += q.x * h1[4 * i] + q.y * h1[4 * i + 1] + q.z * h1[4 * i + 2] + q.w * h1[4 * i + 3];
    }
    y += w3[j] * tanh_hw(s);
  }
  return osc[0] + osc[1] * y;
}

// kNet: the launch evaluates the friction-guess network or captures training
// samples (without, that code stays out of the kernel)
template <typename T, int N, bool kNet>
__global__ void __launch_bounds__(128) rupture_kernel(DRArgs a) {
  constexpr int Bf = nb2(N);
  __shared__ __align__(16) float sW[(MLP_NPARAM + 3) / 4 * 4];  // the network's weights, once per block
  if (kNet && a.mlp) {
    for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x) sW[i] = a.mlp[i];
  }
  __syncthreads();
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = a.n_faces * a.S * Bf;
  if (id >= total) return;
  const int n = (int)(id % Bf);
  const int64_t fs = id / Bf;
  const int64_t fi = a.f_begin + fs / a.S;
  const int s = (int)(fs % a.S);
  const int* ff = a.fface + fi * 5;
  const int em = ff[0], fm = ff[1], ep = ff[2], fp = ff[3], pm = ff[4];
  const double* g = a.fgeo + fi * FGEO;
  const double nrm[3] = {g[0], g[1], g[2]};
  const double rhom = g[3], lamm = g[4], mum = g[5], rhop = g[6], lamp = g[7], mup = g[8];
  const double Zpm = sqrt(rhom * (lamm + 2 * mum)), Zsm = sqrt(rhom * mum);
  const double Zpp = sqrt(rhop * (lamp + 2 * mup)), Zsp = sqrt(rhop * mup);
  const double eta = Zsm * Zsp / (Zsm + Zsp);
  const int np_ = a.perm[pm * Bf + n];
  const T* dm = reinterpret_cast<const T*>(a.dtrace) + ((int64_t)a.dslot[em * 4 + fm] * a.S + s) * (N + 1) * 9 * Bf;
  const T* dp = reinterpret_cast<const T*>(a.dtrace) + ((int64_t)a.dslot[ep * 4 + fp] * a.S + s) * (N + 1) * 9 * Bf;
  const double* par = a.fpar + ((fi * a.S + s) * Bf + n) * FPAR;
  double* st = a.fstate + ((fi * a.S + s) * Bf + n) * FSTATE;
  const FricPar p{par[0], par[1], par[2], par[3], par[4], par[5], par[6]};
  const double sn0 = par[7];
  double t0s[3] = {par[8], par[9], par[10]};
  {
    const double t0n = t0s[0] * nrm[0] + t0s[1] * nrm[1] + t0s[2] * nrm[2];
    for (int i = 0; i < 3; ++i) t0s[i] -= t0n * nrm[i];
  }
  double V = st[0], psi = st[1];
  const double l2v0 = log(2.0 * p.V0);  // (ln c = psi / a - ln(2 V0))
  double slip[3] = {st[2], st[3], st[4]};
  double tau_tot[3] = {st[5], st[6], st[7]};
  double Gm[9] = {0}, Gp[9] = {0};
  double tprev = 0.0;
  double xhat_prev = 0.0;  // the network's ln V* at the previous time point
  bool have_prev = false;
  // the first-pass Newton at the previous time point needed more than one
  // iteration: the state is changing here, and only then is the network
  // evaluated (where the warm start already converges it cannot help)
  bool busy = false;
  unsigned long long n_solves = 0, n_iters = 0;
  bool all_ok = true;
#pragma unroll 1
  for (int j = 0; j <= N; ++j) {
    const double t = a.tp[j];
    // Taylor weights t^k / k!, formed once per time point
    double tk[N + 1];
    tk[0] = 1.0;
#pragma unroll
    for (int k = 1; k <= N; ++k) tk[k] = tk[k - 1] * t / (double)k;
    double qm[9], qp[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      double am = 0, ap = 0;
#pragma unroll
      for (int k = 0; k <= N; ++k) {
        am += tk[k] * (double)dm[(k * 9 + c) * Bf + n];
        ap += tk[k] * (double)dp[(k * 9 + c) * Bf + np_];
      }
      qm[c] = am;
      qp[c] = ap;
    }
    double Tm[3], Tp[3];
    traction(qm, nrm, Tm);
    traction(qp, nrm, Tp);
    const double snm = Tm[0] * nrm[0] + Tm[1] * nrm[1] + Tm[2] * nrm[2];
    const double snp = Tp[0] * nrm[0] + Tp[1] * nrm[1] + Tp[2] * nrm[2];
    const double vnm = qm[6] * nrm[0] + qm[7] * nrm[1] + qm[8] * nrm[2];
    const double vnp = qp[6] * nrm[0] + qp[7] * nrm[1] + qp[8] * nrm[2];
    double taum[3], taup[3], um[3], up[3], Thv[3];
    const double a1 = Zpm * Zpp / (Zpm + Zpp) * ((snm - snp) / Zpp + vnm - vnp);
    const double sn_b = snm - a1, vn_b = vnm - a1 / Zpm;
    for (int i = 0; i < 3; ++i) {
      taum[i] = Tm[i] - snm * nrm[i];
      taup[i] = Tp[i] - snp * nrm[i];
      um[i] = qm[6 + i] - vnm * nrm[i];
      up[i] = qp[6 + i] - vnp * nrm[i];
      Thv[i] = t0s[i] + eta * ((up[i] - um[i]) + taup[i] / Zsp + taum[i] / Zsm);
    }
    const double Th = sqrt(Thv[0] * Thv[0] + Thv[1] * Thv[1] + Thv[2] * Thv[2]);
    const double S = fmax(0.0, -(sn0 + sn_b));
    const double h = t - tprev;
    const double Vold = V;
    const double xw = log(fmax(V, 1e-300));  // warm start: the previous ln|V|
    const double hi = Th > 0 ? log(Th / eta) : 0.0;  // the root's upper bound ln(Theta / eta)
    double x0 = xw;
    double xa = 0.0;  // asinh asymptote: the base of the network's prediction
    float feat[MLP_IN];
    const bool lsw = a.law == FRIC_LSW;
    const bool solve = (Th > 0) && (S > 0) && !lsw;
    bool learned = false;
    // the features only where the network runs or a training sample is
    // captured, in FP64: the start moves the warm start by the change of the
    // prediction between time points, which rounding noise in the features
    // would swamp
    if (kNet && solve && ((a.mlp && busy) || a.capture)) {
      const double lc = psi / p.a - l2v0;
      const double xhi = hi;
      const double r = fmin(Th / (S * p.a), 700.0);
      const double xwc = fmin(fmax(xw, kXFloor), xhi);
      xa = fmin(fmax(r - lc - 0.6931471805599453, kXFloor), xhi);
      feat[0] = (float)r;
      feat[1] = (float)lc;
      feat[2] = (float)xhi;
      feat[3] = (float)xwc;
      feat[4] = (float)fmin(fmax(log(eta / (S * p.a)), -50.0), 50.0);
      feat[5] = (float)xa;
      if (a.mlp && busy) {
        // predicted ln V* = x_a + network; when it was also evaluated at the
        // previous time point, the start is the warm start moved by the change
        // of that prediction
        const double xhat = xa + (double)mlp_eval(sW, feat);
        if (have_prev) {
          x0 = fmin(fmax(xwc + (xhat - xhat_prev), kXFloor), xhi);
          learned = true;
        }
        xhat_prev = xhat;
        have_prev = true;
      } else {
        have_prev = false;
      }
    } else {
      have_prev = false;
    }
    double Vcur = 0.0;
    double xs = x0;  // the Newton start (ln V): pass 0 from x0, pass 1 from pass 0's root
    double psi_new = psi;
    if (lsw) {
      // mu_s, mu_d, D_c, C in the slots a, b, L, f0
      Vcur = V;
      for (int pass = 0; pass < 2; ++pass) {
        const double Vmid = pass == 0 ? Vold : 0.5 * (Vold + Vcur);
        psi_new = psi + Vmid * h;
        const double f = p.a - (p.a - p.b) * fmin(psi_new / p.L, 1.0);
        Vcur = fmax(0.0, Th - (p.f0 + f * S)) / eta;
      }
    }
    for (int pass = 0; pass < (lsw ? 0 : 2); ++pass) {
      // the start guess only seeds Newton; pass 0 relaxes psi with the previous
      // slip rate, pass 1 with the mid-point of the previous and pass-0 rates
      const double Vmid = pass == 0 ? Vold : 0.5 * (Vold + Vcur);
      psi_new = psi_relax(psi, Vmid, h, l2v0, p);
      const double lcn = psi_new / p.a - l2v0;
      int it;
      bool ok;
      double xo;
      Vcur = newton_v(Th, S, eta, lcn, hi, p, xs, &it, &ok, &xo);
      if (pass == 0 && learned && !ok) {
        // fallback: rerun from the warm start
        int it_w;
        Vcur = newton_v(Th, S, eta, lcn, hi, p, xw, &it_w, &ok, &xo);
        it += it_w;
      }
      xs = xo;
      all_ok &= ok;
      if (solve) {
        n_solves++;
        n_iters += it;
      }
      if (pass == 0) busy = solve && it > 1;
      if (kNet && pass == 0 && solve && a.capture) {
        const unsigned long long k = atomicAdd(a.cap_count, 1ull);
        if ((int64_t)k < a.cap_capacity) {
          float* row = a.capture + k * (MLP_IN + 1);
          for (int i = 0; i < MLP_IN; ++i) row[i] = feat[i];
          row[MLP_IN] = (float)(xs - xa);
        }
      }
    }
    psi = psi_new;
    V = Vcur;
    double d[3] = {0, 0, 0};
    if (Th > 0)
      for (int i = 0; i < 3; ++i) d[i] = Thv[i] / Th;
    double tb[3], vb[3], vc[3];
    for (int i = 0; i < 3; ++i) {
      tau_tot[i] = (Th - eta * V) * d[i];
      const double tp_ = tau_tot[i] - t0s[i];
      tb[i] = sn_b * nrm[i] + tp_;
      vb[i] = vn_b * nrm[i] + um[i] + (tp_ - taum[i]) / Zsm;
      vc[i] = vn_b * nrm[i] + up[i] - (tp_ - taup[i]) / Zsp;
      slip[i] += a.tw[j] * V * d[i];
    }
    ahat(nrm, tb, vb, rhom, lamm, mum, 1.0, a.tw[j], Gm);
    ahat(nrm, tb, vc, rhop, lamp, mup, -1.0, a.tw[j], Gp);
    tprev = t;
  }
  psi = a.law == FRIC_LSW ? psi + V * (a.dt - tprev) : psi_relax(psi, V, a.dt - tprev, l2v0, p);
  st[0] = V;
  st[1] = psi;
  for (int i = 0; i < 3; ++i) {
    st[2 + i] = slip[i];
    st[5 + i] = tau_tot[i];
  }
  T* out = reinterpret_cast<T*>(a.drout) + (fi * a.S + s) * 2 * 9 * Bf;
  for (int c = 0; c < 9; ++c) {
    out[c * Bf + n] = (T)Gm[c];
    out[(9 + c) * Bf + np_] = (T)Gp[c];
  }
  if (!all_ok) atomicOr(a.err, ERR_NEWTON);
  atomicAdd(&a.newton[0], n_solves);
  atomicAdd(&a.newton[1], n_iters);
}

template <typename T>
int dispatch(int N, const DRArgs& a, cudaStream_t st) {
  const int64_t total = a.n_faces * a.S * nb2(N);
  if (total <= 0) return 0;
  const unsigned grid = (unsigned)((total + 127) / 128);
  const bool net = a.mlp || a.capture;
#define ADG_RK(n) (net ? rupture_kernel<T, n, true> : rupture_kernel<T, n, false>)<<<grid, 128, 0, st>>>(a)
  switch (N) {
    case 1: ADG_RK(1); break;
    case 2: ADG_RK(2); break;
    case 3: ADG_RK(3); break;
    case 4: ADG_RK(4); break;
    case 5: ADG_RK(5); break;
    default: return (int)cudaErrorInvalidValue;
  }
#undef ADG_RK
  return (int)cudaGetLastError();
}

}  // namespace

int launch_rupture(int fp64, int N, const DRArgs& a, void* stream) {
  return fp64 ? dispatch<double>(N, a, (cudaStream_t)stream) : dispatch<float>(N, a, (cudaStream_t)stream);
}

}  // namespace adg

// Template bodies of the element-update kernels (see kernels.cuh).
//
// Shared-memory working arrays keep the 9 quantities of one basis function
// (or face node) contiguous, padded to P values so that a row is read with
// vector loads; inside a warp the threads usually read the same row, so one
// broadcast load feeds 9 FMAs per thread.  Star products use the Jacobian
// form  sum_a A*_a Y_a = sum_d A_d X_d,  X_d = sum_a (dxi_a/dx_d) Y_a,  with
// the sparse A_d of Eq. (elasticity-pde) written out (material in registers).
#pragma once
#include <cuda_runtime.h>

#include "func_attr.hpp"
#include "kernels.cuh"

namespace adg {

// threads per element block: a launch-time choice (the autotuner's), up to this
constexpr int kMaxThreads = 256;

// 1/k (k = 1..47; entry 0 unused) and 1/m! (m = 0..5), correctly rounded
// constants: the gravity-face series multiplies by them instead of dividing
static __constant__ double kRecipInt[48] = {0.0, 1.0 / 1.0, 1.0 / 2.0, 1.0 / 3.0, 1.0 / 4.0, 1.0 / 5.0, 1.0 / 6.0, 1.0 / 7.0, 1.0 / 8.0, 1.0 / 9.0, 1.0 / 10.0, 1.0 / 11.0, 1.0 / 12.0, 1.0 / 13.0, 1.0 / 14.0, 1.0 / 15.0, 1.0 / 16.0, 1.0 / 17.0, 1.0 / 18.0, 1.0 / 19.0, 1.0 / 20.0, 1.0 / 21.0, 1.0 / 22.0, 1.0 / 23.0, 1.0 / 24.0, 1.0 / 25.0, 1.0 / 26.0, 1.0 / 27.0, 1.0 / 28.0, 1.0 / 29.0, 1.0 / 30.0, 1.0 / 31.0, 1.0 / 32.0, 1.0 / 33.0, 1.0 / 34.0, 1.0 / 35.0, 1.0 / 36.0, 1.0 / 37.0, 1.0 / 38.0, 1.0 / 39.0, 1.0 / 40.0, 1.0 / 41.0, 1.0 / 42.0, 1.0 / 43.0, 1.0 / 44.0, 1.0 / 45.0, 1.0 / 46.0, 1.0 / 47.0};
static __constant__ double kInvFact[6] = {1.0, 1.0, 1.0 / 2.0, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0};

__host__ __device__ constexpr int doff_rows(int k, int N) {  // first row of D^k in the derivative stack
  int s = 0;
  for (int j = 0; j < k; ++j) s += nb3(N - j);
  return s;
}

template <typename T>
struct Pad;
template <>
struct Pad<float> {
  static constexpr int P = 12;  // 3 x float4
};
template <>
struct Pad<double> {
  static constexpr int P = 10;  // 5 x double2
};

__device__ __forceinline__ void load9(const float* p, float o[9]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  const float4 b = *reinterpret_cast<const float4*>(p + 4);
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
  o[8] = p[8];
}
__device__ __forceinline__ void load9(const double* p, double o[9]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double2 a = *reinterpret_cast<const double2*>(p + 2 * i);
    o[2 * i] = a.x;
    o[2 * i + 1] = a.y;
  }
  o[8] = p[8];
}
__device__ __forceinline__ void store9(float* p, const float o[9]) {
  *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
  *reinterpret_cast<float4*>(p + 4) = make_float4(o[4], o[5], o[6], o[7]);
  p[8] = o[8];
}
__device__ __forceinline__ void store9(double* p, const double o[9]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) *reinterpret_cast<double2*>(p + 2 * i) = make_double2(o[2 * i], o[2 * i + 1]);
  p[8] = o[8];
}

// out = sum_d A_d X_d for the Jacobians of Eq. (elasticity-pde)
template <typename T>
__device__ __forceinline__ void jac_sum(const T X0[9], const T X1[9], const T X2[9], T lam, T mu, T irho, T out[9]) {
  const T l2m = lam + T(2) * mu;
  out[0] = -(l2m * X0[6] + lam * X1[7] + lam * X2[8]);
  out[1] = -(lam * X0[6] + l2m * X1[7] + lam * X2[8]);
  out[2] = -(lam * X0[6] + lam * X1[7] + l2m * X2[8]);
  out[3] = -mu * (X1[6] + X0[7]);
  out[4] = -mu * (X2[7] + X1[8]);
  out[5] = -mu * (X2[6] + X0[8]);
  out[6] = -irho * (X0[0] + X1[3] + X2[5]);
  out[7] = -irho * (X0[3] + X1[1] + X2[4]);
  out[8] = -irho * (X0[5] + X1[4] + X2[2]);
}
// out = A_d x for one direction d
template <typename T>
__device__ __forceinline__ void jac_dir(int d, const T x[9], T lam, T mu, T irho, T out[9]) {
  const T vd = x[6 + d];
#pragma unroll
  for (int i = 0; i < 3; ++i) out[i] = -lam * vd;
  out[d] -= T(2) * mu * vd;
  out[3] = -mu * ((d == 1 ? x[6] : T(0)) + (d == 0 ? x[7] : T(0)));
  out[4] = -mu * ((d == 2 ? x[7] : T(0)) + (d == 1 ? x[8] : T(0)));
  out[5] = -mu * ((d == 2 ? x[6] : T(0)) + (d == 0 ? x[8] : T(0)));
  // velocity rows: -(1/rho) s_{i d}
  const int s0 = d == 0 ? 0 : (d == 1 ? 3 : 5);  // s_{x d}
  const int s1 = d == 0 ? 3 : (d == 1 ? 1 : 4);  // s_{y d}
  const int s2 = d == 0 ? 5 : (d == 1 ? 4 : 2);  // s_{z d}
  out[6] = -irho * x[s0];
  out[7] = -irho * x[s1];
  out[8] = -irho * x[s2];
}

template <typename T, int N>
struct Smem {
  static constexpr int P = Pad<T>::P;
  static constexpr int B = nb3(N), Bf = nb2(N), B1 = nb3(N - 1);
  static constexpr int nDrows = doff_rows(N + 1, N);
  // derivative stack | time integral | Y / Z scratch (3 x B1 rows) | face traces | dQ partials | params
  static constexpr int oD = 0, oI = oD + nDrows * P, oY = oI + B * P, oV = oY + 3 * B1 * P,
                       oQ = oV + 4 * Bf * P, oP = oQ + 3 * B * P, oEnd = oP + PAR;
  static constexpr int nGrav = (N + 1) * Bf;  // doubles
  static constexpr int bytes = ((oEnd * (int)sizeof(T) + 15) / 16) * 16 + nGrav * 8;
};

template <typename T, int N>
__global__ void __launch_bounds__(kMaxThreads) local_kernel(StepArgs a, const __grid_constant__ Segs segs) {
  using S = Smem<T, N>;
  constexpr int P = S::P, B = S::B, Bf = S::Bf, B1 = S::B1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* sD = sm + S::oD;
  T* sI = sm + S::oI;
  T* sY = sm + S::oY;
  T* sV = sm + S::oV;
  T* sQp = sm + S::oQ;
  T* sP = sm + S::oP;
  double* sF = reinterpret_cast<double*>(smem_raw + ((S::oEnd * (int)sizeof(T) + 15) / 16) * 16);

  const int tid = threadIdx.x, nth = blockDim.x;
  const Seg& sg = segs.s[seg_find(segs, blockIdx.x)];
  const int64_t v = sg.v_begin + ((int64_t)blockIdx.x - segs.first[&sg - segs.s]);
  const int64_t e = v / a.S;
  const int s = (int)(v - e * a.S);
  T* Q = reinterpret_cast<T*>(a.Q) + v * 9 * B;
  const T* ktT = reinterpret_cast<const T*>(a.ktT);
  const T* kvolT = reinterpret_cast<const T*>(a.kvolT);
  const T* efcT = reinterpret_cast<const T*>(a.efcT);

  if (tid < PAR) sP[tid] = reinterpret_cast<const T*>(a.par)[e * PAR + tid];
  for (int r = tid; r < 9 * B; r += nth) {  // Q[p][l] -> D^0[l][p]
    const int p = r / B, l = r % B;
    sD[l * P + p] = Q[r];
  }
  __syncthreads();
  T g[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) g[i] = sP[i];  // g[a*3+d] = d xi_a / d x_d
  const T lam = sP[10], mu = sP[11], irho = T(1) / sP[9];

  // ---- Cauchy-Kovalewski: Y_a = KT_a D^k (rows < B_{N-k-1}), D^{k+1} = -sum_d A_d X_d
#pragma unroll 1
  for (int k = 0; k < N; ++k) {
    const int Bl = nb3(N - k), Bm = nb3(N - k - 1);
    const T* Dk = sD + doff_rows(k, N) * P;
    T* Dn = sD + doff_rows(k + 1, N) * P;
    for (int r = tid; r < 3 * Bm; r += nth) {
      const int ax = r / Bm, m = r % Bm;
      T acc[9];
#pragma unroll
      for (int p = 0; p < 9; ++p) acc[p] = T(0);
      const T* kk = ktT + (size_t)ax * B * B + m;
      for (int l = 0; l < Bl; ++l) {
        const T w = kk[(size_t)l * B];
        T d9[9];
        load9(Dk + l * P, d9);
#pragma unroll
        for (int p = 0; p < 9; ++p) acc[p] += w * d9[p];
      }
      store9(sY + (ax * B1 + m) * P, acc);
    }
    __syncthreads();
    for (int m = tid; m < Bm; m += nth) {
      T y0[9], y1[9], y2[9], X0[9], X1[9], X2[9], o[9];
      load9(sY + (0 * B1 + m) * P, y0);
      load9(sY + (1 * B1 + m) * P, y1);
      load9(sY + (2 * B1 + m) * P, y2);
#pragma unroll
      for (int p = 0; p < 9; ++p) {
        X0[p] = g[0] * y0[p] + g[3] * y1[p] + g[6] * y2[p];
        X1[p] = g[1] * y0[p] + g[4] * y1[p] + g[7] * y2[p];
        X2[p] = g[2] * y0[p] + g[5] * y1[p] + g[8] * y2[p];
      }
      jac_sum(X0, X1, X2, lam, mu, irho, o);
#pragma unroll
      for (int p = 0; p < 9; ++p) o[p] = -o[p];
      store9(Dn + m * P, o);
    }
    __syncthreads();
  }

  // ---- time integral over the own step
  for (int l = tid; l < B; l += nth) {
    T acc[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) acc[p] = T(0);
#pragma unroll
    for (int k = 0; k <= N; ++k) {
      if (l < nb3(N - k)) {
        T d9[9];
        load9(sD + (doff_rows(k, N) + l) * P, d9);
        const T c = T(sg.tcoef[k]);
#pragma unroll
        for (int p = 0; p < 9; ++p) acc[p] += c * d9[p];
      }
    }
    store9(sI + l * P, acc);
  }
  // ---- LTS: derivative traces E_f D^k for faces with a finer neighbour or a fault
  if (a.dslot) {
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
      const int ds = a.dslot[e * 4 + f];  // block-uniform
      if (ds < 0) continue;
      T* out = reinterpret_cast<T*>(a.dtrace) + ((int64_t)ds * a.S + s) * (N + 1) * 9 * Bf;
      for (int r = tid; r < (N + 1) * Bf; r += nth) {
        const int k = r / Bf, n = r % Bf;
        const int Bk = nb3(N - k);
        const T* Dk = sD + doff_rows(k, N) * P;
        T acc[9];
#pragma unroll
        for (int p = 0; p < 9; ++p) acc[p] = T(0);
        for (int l = 0; l < Bk; ++l) {
          const T w = efcT[((size_t)f * B + l) * Bf + n];
          T d9[9];
          load9(Dk + l * P, d9);
#pragma unroll
          for (int p = 0; p < 9; ++p) acc[p] += w * d9[p];
        }
#pragma unroll
        for (int p = 0; p < 9; ++p) out[(k * 9 + p) * Bf + n] = acc[p];
      }
    }
  }
  __syncthreads();

  // ---- volume operand Z_a[l] = A*_a I[l] (l < B_{N-1}) and face traces V = E_f I
  for (int l = tid; l < B1; l += nth) {
    T x[9], u0[9], u1[9], u2[9];
    load9(sI + l * P, x);
    jac_dir(0, x, lam, mu, irho, u0);
    jac_dir(1, x, lam, mu, irho, u1);
    jac_dir(2, x, lam, mu, irho, u2);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      T z[9];
#pragma unroll
      for (int p = 0; p < 9; ++p) z[p] = g[ax * 3 + 0] * u0[p] + g[ax * 3 + 1] * u1[p] + g[ax * 3 + 2] * u2[p];
      store9(sY + (ax * B1 + l) * P, z);
    }
  }
  constexpr int FS = face_stride(N);
  T* trace = reinterpret_cast<T*>(a.trace) + v * 4 * FS;
  double* bt = nullptr;
  if (sg.btrace_mode && a.bslot) {
    const int bs = a.bslot[e];
    if (bs >= 0) bt = a.btrace + ((int64_t)bs * a.S + s) * 36 * Bf;
  }
  for (int r = tid; r < 4 * Bf; r += nth) {
    const int f = r / Bf, n = r % Bf;
    T acc[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) acc[p] = T(0);
    const T* ee = efcT + (size_t)f * B * Bf + n;
    for (int l = 0; l < B; ++l) {
      const T w = ee[(size_t)l * Bf];
      T d9[9];
      load9(sI + l * P, d9);
#pragma unroll
      for (int p = 0; p < 9; ++p) acc[p] += w * d9[p];
    }
    store9(sV + r * P, acc);
#pragma unroll
    for (int p = 0; p < 9; ++p) trace[f * FS + p * Bf + n] = acc[p];
    if (bt) {
#pragma unroll
      for (int p = 0; p < 9; ++p) {
        double* b = bt + (f * 9 + p) * Bf + n;
        *b = (sg.btrace_mode == 1 ? 0.0 : *b) + (double)acc[p];
      }
    }
  }
  __syncthreads();
  // ---- volume: dQ[m] = sum_a sum_l K_a[m][l] Z_a[l]   (three partial sums, one per a)
  for (int r = tid; r < 3 * B; r += nth) {
    const int ax = r / B, m = r % B;
    T acc[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) acc[p] = T(0);
    const T* kv = kvolT + (size_t)ax * B1 * B + m;
    const T* z = sY + ax * B1 * P;
    for (int l = 0; l < B1; ++l) {
      const T w = kv[(size_t)l * B];
      T z9[9];
      load9(z + l * P, z9);
#pragma unroll
      for (int p = 0; p < 9; ++p) acc[p] += w * z9[p];
    }
    store9(sQp + (ax * B + m) * P, acc);
  }
  __syncthreads();
  // ---- Q += volume term (face terms follow in the neighbour kernel)
  for (int r = tid; r < 9 * B; r += nth) {
    const int p = r / B, m = r % B;
    Q[r] = sD[m * P + p] + ((sQp[m * P + p] + sQp[(B + m) * P + p]) + sQp[(2 * B + m) * P + p]);
  }
  // ---- gravitational faces: (eta, H) ODE per node in FP64, then that face's flux
  if (a.gslot) {
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
      const int gs = a.gslot[e * 4 + f];  // block-uniform
      if (gs < 0) continue;
      const double* gp = a.gpar + (size_t)gs * GPAR;
      __syncthreads();
      // Taylor coefficients f_m(node) of v_n^- + p^-/Z = n.v - s_nn/Z, divided by m!
      for (int r = tid; r < (N + 1) * Bf; r += nth) {
        const int m = r / Bf, n = r % Bf;
        const int Bk = nb3(N - m);
        const T* Dm = sD + doff_rows(m, N) * P;
        T acc[9];
#pragma unroll
        for (int p = 0; p < 9; ++p) acc[p] = T(0);
        for (int l = 0; l < Bk; ++l) {
          const T w = efcT[((size_t)f * B + l) * Bf + n];
          T d9[9];
          load9(Dm + l * P, d9);
#pragma unroll
          for (int p = 0; p < 9; ++p) acc[p] += w * d9[p];
        }
        // n.sigma.n and n.v in the dofs precision (the traces are in it)
        const T nx = (T)gp[0], ny = (T)gp[1], nz = (T)gp[2];
        const T snn = nx * nx * acc[0] + ny * ny * acc[1] + nz * nz * acc[2] +
                      T(2) * (nx * ny * acc[3] + ny * nz * acc[4] + nx * nz * acc[5]);
        const T vn = nx * acc[6] + ny * acc[7] + nz * acc[8];
        sF[r] = ((double)vn - (double)snn * (1.0 / gp[3])) * kInvFact[m];
      }
      __syncthreads();
      if (tid < Bf) {
        const int n = tid;
        double* eta = a.eta + ((int64_t)gs * a.S + s) * Bf;
        const double kappa = gp[4], rg = gp[5], dt = sg.dt;
        const double eta0 = eta[n];
        double c = eta0, e1 = eta0, H = eta0 * dt, pw = 1.0;
        for (int m = 0; m < N + 40; ++m) {
          const double fm = (m <= N) ? sF[m * Bf + n] : 0.0;
          c = (fm - kappa * c) * kRecipInt[m + 1];
          pw *= dt;
          const double term = c * pw;
          e1 += term;
          H += term * dt * kRecipInt[m + 2];
          if (m > N && fabs(term) <= 1e-17 * fabs(e1)) break;
        }
        eta[n] = e1;
        const double* Fg = gp + 6;
        const double* a1 = gp + 87;
        const double* a7 = gp + 96;
        T* gfl = reinterpret_cast<T*>(a.gflux) + ((int64_t)gs * a.S + s) * 9 * Bf;
        for (int q = 0; q < 9; ++q) {
          // the own trace's part in the dofs precision, the (eta, H) part in FP64
          T fv = T(0);
          for (int p = 0; p < 9; ++p) fv += (T)Fg[q * 9 + p] * sV[(f * Bf + n) * P + p];
          gfl[q * Bf + n] = (T)(a1[q] * (-rg * H) + a7[q] * (e1 - eta0) + (double)fv);
        }
      }
    }
  }
}

template <typename T, int N>
struct SmemN {
  static constexpr int P = Pad<T>::P;
  static constexpr int B = nb3(N), Bf = nb2(N);
};

template <typename T, int N>
__global__ void __launch_bounds__(kMaxThreads) neighbour_kernel(StepArgs a, const __grid_constant__ Segs segs) {
  constexpr int P = Pad<T>::P, B = nb3(N), Bf = nb2(N);
  __shared__ __align__(16) T sVo[4 * Bf * P];  // own traces [f][n][p]
  __shared__ __align__(16) T sVn[4 * Bf * P];  // neighbours' traces in this face's node order
  __shared__ __align__(16) T sG[4 * Bf * P];   // scaled face fluxes
  __shared__ __align__(16) T sPart[2 * B * P];
  __shared__ T sF[4 * 162];                    // per face: F- (81) then F+ (81)
  __shared__ T sScale[4];
  __shared__ int sKind[4];
  __shared__ int sGrav[4];
  const int tid = threadIdx.x, nth = blockDim.x;
  const Seg& sg = segs.s[seg_find(segs, blockIdx.x)];
  const int64_t v = sg.v_begin + ((int64_t)blockIdx.x - segs.first[&sg - segs.s]);
  const int64_t e = v / a.S;
  const int s = (int)(v - e * a.S);
  const T* liftT = reinterpret_cast<const T*>(a.liftT);
  if (tid < 4) {
    sScale[tid] = reinterpret_cast<const T*>(a.par)[e * PAR + 12 + tid];
    sKind[tid] = (a.ninfo[e * 4 + tid] >> 5) & 7;
    sGrav[tid] = a.gslot ? a.gslot[e * 4 + tid] : -1;
  }
  for (int r = tid; r < 4 * 81; r += nth) {
    const int f = r / 81, k = r % 81;
    sF[f * 162 + k] = reinterpret_cast<const T*>(a.Fm)[e * 4 * 81 + r];
    sF[f * 162 + 81 + k] = reinterpret_cast<const T*>(a.Fp)[e * 4 * 81 + r];
  }
  constexpr int FS = face_stride(N);
  const T* own = reinterpret_cast<const T*>(a.trace) + v * 4 * FS;
  for (int r = tid; r < 36 * Bf; r += nth) {  // [f][p][n] -> [f][n][p]
    const int f = r / (9 * Bf), p = (r / Bf) % 9, n = r % Bf;
    sVo[(f * Bf + n) * P + p] = own[f * FS + p * Bf + n];
  }
  __syncthreads();
  for (int r = tid; r < 36 * Bf; r += nth) {
    const int f = r / (9 * Bf), p = (r / Bf) % 9, n = r % Bf;
    const int kind = sKind[f];
    T val = T(0);
    if (kind == NK_SAME || kind == NK_FINE || kind == NK_COARSE) {
      const int info = a.ninfo[e * 4 + f];
      const int64_t nb = a.nbr[e * 4 + f];
      const int j = info & 3, pm = (info >> 2) & 7;
      const int src = a.perm[pm * Bf + n];
      if (kind == NK_SAME) {
        val = reinterpret_cast<const T*>(a.trace)[((nb * a.S + s) * 4 + j) * FS + p * Bf + src];
      } else if (kind == NK_FINE) {
        const int bs = a.bslot[nb];
        val = (T)a.btrace[(((int64_t)bs * a.S + s) * 4 + j) * 9 * Bf + p * Bf + src];
      } else {  // NK_COARSE: integrate the coarser neighbour's expansion over this sub-interval
        const int ds = a.dslot[nb * 4 + j];
        const T* dt = reinterpret_cast<const T*>(a.dtrace) + ((int64_t)ds * a.S + s) * (N + 1) * 9 * Bf;
        T acc = T(0);
#pragma unroll
        for (int k = 0; k <= N; ++k) acc += T(sg.ccoef[k]) * dt[(k * 9 + p) * Bf + src];
        val = acc;
      }
    }
    sVn[(f * Bf + n) * P + p] = val;
  }
  __syncthreads();
  // face fluxes: F- (own) + F+ (neighbour) on interior faces, F- with the ghost
  // folded in on linear boundaries, stored fluxes on gravitational / fault faces
  for (int r = tid; r < 4 * Bf; r += nth) {
    const int f = r / Bf, n = r % Bf;
    T gq[9];
    if (sKind[f] == NK_FAULT) {
      const int fsl = a.fslot[e * 4 + f];
      const T* src = reinterpret_cast<const T*>(a.drout) + (((int64_t)(fsl >> 1) * a.S + s) * 2 + (fsl & 1)) * 9 * Bf;
#pragma unroll
      for (int q = 0; q < 9; ++q) gq[q] = src[q * Bf + n];
    } else if (sGrav[f] >= 0) {
      const T* src = reinterpret_cast<const T*>(a.gflux) + ((int64_t)sGrav[f] * a.S + s) * 9 * Bf;
#pragma unroll
      for (int q = 0; q < 9; ++q) gq[q] = src[q * Bf + n];
    } else {
      T vo[9];
      load9(sVo + r * P, vo);
      const T* Fm = sF + f * 162;
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        T acc = T(0);
#pragma unroll
        for (int p = 0; p < 9; ++p) acc += Fm[q * 9 + p] * vo[p];
        gq[q] = acc;
      }
      if (sKind[f] != NK_NONE) {
        T vn[9];
        load9(sVn + r * P, vn);
        const T* Fp = sF + f * 162 + 81;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          T acc = T(0);
#pragma unroll
          for (int p = 0; p < 9; ++p) acc += Fp[q * 9 + p] * vn[p];
          gq[q] += acc;
        }
      }
    }
    const T sc = sScale[f];
#pragma unroll
    for (int q = 0; q < 9; ++q) gq[q] *= sc;
    store9(sG + r * P, gq);
  }
  __syncthreads();
  // lift: two partial sums per basis function (faces 0-1 and 2-3)
  for (int r = tid; r < 2 * B; r += nth) {
    const int half = r / B, m = r % B;
    T acc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] = T(0);
    for (int fn = half * 2 * Bf; fn < (half + 1) * 2 * Bf; ++fn) {  // fn = f*Bf + n
      const T w = liftT[(size_t)fn * B + m];
      T g9[9];
      load9(sG + fn * P, g9);
#pragma unroll
      for (int q = 0; q < 9; ++q) acc[q] += w * g9[q];
    }
    store9(sPart + r * P, acc);
  }
  __syncthreads();
  T* Q = reinterpret_cast<T*>(a.Q) + v * 9 * B;
  bool bad = false;
  for (int r = tid; r < 9 * B; r += nth) {
    const int q = r / B, m = r % B;
    const T nq = Q[r] - (sPart[m * P + q] + sPart[(B + m) * P + q]);
    Q[r] = nq;
    bad |= !isfinite((double)nq);
  }
  if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0) atomicOr(a.err, ERR_NAN);
}

template <typename T, int N>
int launch_local_t(const StepArgs& a, const Segs& g, int threads, cudaStream_t st) {
  const int64_t nblocks = g.n ? g.first[g.n] : 0;
  constexpr int bytes = Smem<T, N>::bytes;
  const int rc = configure_on_device((const void*)local_kernel<T, N>, [] {
    return cudaFuncSetAttribute(local_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  });
  if (rc) return rc;
  if (nblocks <= 0) return 0;
  if (threads < 32 || threads > kMaxThreads || threads % 32) return (int)cudaErrorInvalidValue;
  local_kernel<T, N><<<(unsigned)nblocks, threads, bytes, st>>>(a, g);
  return (int)cudaGetLastError();
}

template <typename T, int N>
int launch_neighbour_t(const StepArgs& a, const Segs& g, int threads, cudaStream_t st) {
  const int64_t nblocks = g.n ? g.first[g.n] : 0;
  if (nblocks <= 0) return 0;
  if (threads < 32 || threads > kMaxThreads || threads % 32) return (int)cudaErrorInvalidValue;
  neighbour_kernel<T, N><<<(unsigned)nblocks, threads, 0, st>>>(a, g);
  return (int)cudaGetLastError();
}

template <typename T>
int dispatch_local(int N, const StepArgs& a, const Segs& nb, int th, cudaStream_t st) {
  switch (N) {
    case 1: return launch_local_t<T, 1>(a, nb, th, st);
    case 2: return launch_local_t<T, 2>(a, nb, th, st);
    case 3: return launch_local_t<T, 3>(a, nb, th, st);
    case 4: return launch_local_t<T, 4>(a, nb, th, st);
    case 5: return launch_local_t<T, 5>(a, nb, th, st);
  }
  return (int)cudaErrorInvalidValue;
}
template <typename T>
int dispatch_neighbour(int N, const StepArgs& a, const Segs& nb, int th, cudaStream_t st) {
  switch (N) {
    case 1: return launch_neighbour_t<T, 1>(a, nb, th, st);
    case 2: return launch_neighbour_t<T, 2>(a, nb, th, st);
    case 3: return launch_neighbour_t<T, 3>(a, nb, th, st);
    case 4: return launch_neighbour_t<T, 4>(a, nb, th, st);
    case 5: return launch_neighbour_t<T, 5>(a, nb, th, st);
  }
  return (int)cudaErrorInvalidValue;
}
template <typename T>
int smem_of(int N) {
  switch (N) {
    case 1: return Smem<T, 1>::bytes;
    case 2: return Smem<T, 2>::bytes;
    case 3: return Smem<T, 3>::bytes;
    case 4: return Smem<T, 4>::bytes;
    case 5: return Smem<T, 5>::bytes;
  }
  return 0;
}

}  // namespace adg

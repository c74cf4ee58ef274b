// Template bodies of the element-update kernels (see kernels.cuh).
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace adg {

constexpr int kThreads = 128;

__host__ __device__ constexpr int doff(int k, int N) {
  int s = 0;
  for (int j = 0; j < k; ++j) s += 9 * nb3(N - j);
  return s;
}

// Entry (q, p) of the Jacobian A_d of Eq. (elasticity-pde) for material (rho, lam, mu).
template <typename T>
__device__ __forceinline__ T jac_entry(int d, int q, int p, T rho, T lam, T mu) {
  if (q < 3) {
    if (p != 6 + d) return T(0);
    return -lam - (q == d ? T(2) * mu : T(0));
  }
  if (q < 6) {
    const int i = (q == 4) ? 1 : 0;
    const int j = (q == 3) ? 1 : 2;
    T r = T(0);
    if (d == j && p == 6 + i) r -= mu;
    if (d == i && p == 6 + j) r -= mu;
    return r;
  }
  const int i = q - 6;
  // Voigt index of s_{i d}
  int s;
  if (i == d) s = i;
  else if ((i == 0 && d == 1) || (i == 1 && d == 0)) s = 3;
  else if ((i == 1 && d == 2) || (i == 2 && d == 1)) s = 4;
  else s = 5;
  return p == s ? -T(1) / rho : T(0);
}

// star[a][q][p] = sum_d Jinv[a][d] A_d[q][p]
template <typename T>
__device__ __forceinline__ void build_star(const T* par, T* star) {
  const T rho = par[9], lam = par[10], mu = par[11];
  for (int r = threadIdx.x; r < 243; r += blockDim.x) {
    const int a = r / 81, q = (r / 9) % 9, p = r % 9;
    T s = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) s += par[a * 3 + d] * jac_entry<T>(d, q, p, rho, lam, mu);
    star[r] = s;
  }
}

template <typename T, int N>
struct Smem {
  static constexpr int B = nb3(N), Bf = nb2(N), B1 = nb3(N - 1);
  static constexpr int nD = doff(N + 1, N);
  static constexpr int nY = 27 * B1;
  // D | I | Y | dQ | star | V | G | par | gravity scratch (double)
  static constexpr int oD = 0, oI = oD + nD, oY = oI + 9 * B, odQ = oY + nY, oS = odQ + 9 * B,
                       oV = oS + 243, oG = oV + 36 * Bf, oP = oG + 36 * Bf, oEnd = oP + PAR;
  static constexpr int nGrav = (N + 1) * Bf;  // doubles
  static constexpr int bytes = ((oEnd * (int)sizeof(T) + 15) / 16) * 16 + nGrav * 8;
};

template <typename T, int N>
__global__ void __launch_bounds__(kThreads) local_kernel(StepArgs a) {
  using S = Smem<T, N>;
  constexpr int B = S::B, Bf = S::Bf, B1 = S::B1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* sD = sm + S::oD;
  T* sI = sm + S::oI;
  T* sY = sm + S::oY;
  T* sdQ = sm + S::odQ;
  T* sStar = sm + S::oS;
  T* sV = sm + S::oV;
  T* sG = sm + S::oG;
  T* sP = sm + S::oP;
  double* sF = reinterpret_cast<double*>(smem_raw + ((S::oEnd * (int)sizeof(T) + 15) / 16) * 16);

  const int tid = threadIdx.x, nth = blockDim.x;
  const int64_t v = a.v_begin + blockIdx.x;
  const int64_t e = v / a.S;
  const int s = (int)(v - e * a.S);
  T* Q = reinterpret_cast<T*>(a.Q) + v * 9 * B;
  const T* ktT = reinterpret_cast<const T*>(a.ktT);
  const T* kvolT = reinterpret_cast<const T*>(a.kvolT);
  const T* efcT = reinterpret_cast<const T*>(a.efcT);
  const T* liftT = reinterpret_cast<const T*>(a.liftT);

  if (tid < PAR) sP[tid] = reinterpret_cast<const T*>(a.par)[e * PAR + tid];
  for (int r = tid; r < 9 * B; r += nth) sD[r] = Q[r];
  __syncthreads();
  build_star<T>(sP, sStar);
  __syncthreads();

  // ---- Cauchy-Kovalewski: D^{k+1} = -sum_a KT_a D^k A*_a^T, truncated to B_{N-k-1} rows
#pragma unroll 1
  for (int k = 0; k < N; ++k) {
    const int Bl = nb3(N - k), Bm = nb3(N - k - 1);
    const T* Dk = sD + doff(k, N);
    T* Dn = sD + doff(k + 1, N);
    for (int r = tid; r < 3 * Bm; r += nth) {
      const int ax = r / Bm, m = r % Bm;
      T acc[9];
#pragma unroll
      for (int p = 0; p < 9; ++p) acc[p] = T(0);
      const T* kk = ktT + (size_t)ax * B * B + m;
      for (int l = 0; l < Bl; ++l) {
        const T w = kk[(size_t)l * B];
#pragma unroll
        for (int p = 0; p < 9; ++p) acc[p] += w * Dk[p * Bl + l];
      }
#pragma unroll
      for (int p = 0; p < 9; ++p) sY[(ax * 9 + p) * Bm + m] = acc[p];
    }
    __syncthreads();
    for (int r = tid; r < 9 * Bm; r += nth) {
      const int q = r / Bm, m = r % Bm;
      T acc = T(0);
#pragma unroll
      for (int ax = 0; ax < 3; ++ax)
#pragma unroll
        for (int p = 0; p < 9; ++p) {
          const T st = sStar[(ax * 9 + q) * 9 + p];
          if (st != T(0)) acc += st * sY[(ax * 9 + p) * Bm + m];
        }
      Dn[q * Bm + m] = -acc;
    }
    __syncthreads();
  }

  // ---- time integral over the own step
  for (int r = tid; r < 9 * B; r += nth) {
    const int p = r / B, l = r % B;
    T acc = T(0);
#pragma unroll
    for (int k = 0; k <= N; ++k) {
      const int Bk = nb3(N - k);
      if (l < Bk) acc += T(a.tcoef[k]) * sD[doff(k, N) + p * Bk + l];
    }
    sI[r] = acc;
  }
  // ---- LTS: derivative traces for finer neighbours
  if (a.dslot) {
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
      const int ds = a.dslot[e * 4 + f];
      if (ds < 0) continue;
      T* out = reinterpret_cast<T*>(a.dtrace) + ((int64_t)ds * a.S + s) * (N + 1) * 9 * Bf;
      for (int r = tid; r < (N + 1) * 9 * Bf; r += nth) {
        const int k = r / (9 * Bf), p = (r / Bf) % 9, n = r % Bf;
        const int Bk = nb3(N - k);
        const T* Dk = sD + doff(k, N) + p * Bk;
        T acc = T(0);
        for (int l = 0; l < Bk; ++l) acc += efcT[((size_t)f * B + l) * Bf + n] * Dk[l];
        out[r] = acc;
      }
    }
  }
  __syncthreads();

  // ---- volume: dQ = sum_a K_a (I A*_a^T)
  for (int r = tid; r < 27 * B1; r += nth) {
    const int ax = r / (9 * B1), q = (r / B1) % 9, l = r % B1;
    T acc = T(0);
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      const T st = sStar[(ax * 9 + q) * 9 + p];
      if (st != T(0)) acc += st * sI[p * B + l];
    }
    sY[r] = acc;  // Z[a][q][l]
  }
  // ---- own face traces V[f][p][n] = sum_l E_f[n][l] I[p][l]
  T* trace = reinterpret_cast<T*>(a.trace) + v * 36 * Bf;
  for (int r = tid; r < 36 * Bf; r += nth) {
    const int f = r / (9 * Bf), p = (r / Bf) % 9, n = r % Bf;
    T acc = T(0);
    const T* ee = efcT + (size_t)f * B * Bf + n;
    for (int l = 0; l < B; ++l) acc += ee[(size_t)l * Bf] * sI[p * B + l];
    sV[r] = acc;
    trace[r] = acc;
  }
  if (a.btrace_mode && a.bslot) {
    const int bs = a.bslot[e];
    if (bs >= 0) {
      __syncthreads();
      double* bt = a.btrace + ((int64_t)bs * a.S + s) * 36 * Bf;
      for (int r = tid; r < 36 * Bf; r += nth) bt[r] = (a.btrace_mode == 1 ? 0.0 : bt[r]) + (double)sV[r];
    }
  }
  __syncthreads();
  for (int r = tid; r < 9 * B; r += nth) {
    const int q = r / B, m = r % B;
    T acc = T(0);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const T* kv = kvolT + (size_t)ax * B1 * B + m;
      const T* z = sY + (ax * 9 + q) * B1;
      for (int l = 0; l < B1; ++l) acc += kv[(size_t)l * B] * z[l];
    }
    sdQ[r] = acc;
  }
  // ---- the local flux F^- V of ordinary faces is applied, together with the
  // neighbour flux, by the neighbour kernel (one lift per step); here only the
  // gravitational faces need the own derivatives:
  // (eta, H) ODE per node in FP64, then that face's flux into gflux
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
        const T* Dm = sD + doff(m, N);
        double val[9];
#pragma unroll
        for (int p = 0; p < 9; ++p) {
          T acc = T(0);
          for (int l = 0; l < Bk; ++l) acc += efcT[((size_t)f * B + l) * Bf + n] * Dm[p * Bk + l];
          val[p] = (double)acc;
        }
        const double nx = gp[0], ny = gp[1], nz = gp[2], Z = gp[3];
        const double snn = nx * nx * val[0] + ny * ny * val[1] + nz * nz * val[2] +
                           2.0 * (nx * ny * val[3] + ny * nz * val[4] + nx * nz * val[5]);
        const double vn = nx * val[6] + ny * val[7] + nz * val[8];
        double fac = 1.0;
        for (int j = 2; j <= m; ++j) fac *= j;
        sF[r] = (vn - snn / Z) / fac;
      }
      __syncthreads();
      if (tid < Bf) {
        const int n = tid;
        double* eta = a.eta + ((int64_t)gs * a.S + s) * Bf;
        const double kappa = gp[4], rg = gp[5], dt = a.dt;
        const double eta0 = eta[n];
        double c = eta0, e1 = eta0, H = eta0 * dt, pw = 1.0;
        for (int m = 0; m < N + 40; ++m) {
          const double fm = (m <= N) ? sF[m * Bf + n] : 0.0;
          c = (fm - kappa * c) / (m + 1);
          pw *= dt;
          const double term = c * pw;
          e1 += term;
          H += term * dt / (m + 2);
          if (m > N && fabs(term) <= 1e-17 * fabs(e1)) break;
        }
        eta[n] = e1;
        const double* Fg = gp + 6;
        const double* a1 = gp + 87;
        const double* a7 = gp + 96;
        T* gfl = reinterpret_cast<T*>(a.gflux) + ((int64_t)gs * a.S + s) * 9 * Bf;
        for (int q = 0; q < 9; ++q) {
          double acc = a1[q] * (-rg * H) + a7[q] * (e1 - eta0);
          for (int p = 0; p < 9; ++p) acc += Fg[q * 9 + p] * (double)sV[(f * 9 + p) * Bf + n];
          gfl[q * Bf + n] = (T)acc;
        }
      }
    }
  }
  __syncthreads();
  // ---- Q += volume term (the face terms follow in the neighbour kernel)
  for (int r = tid; r < 9 * B; r += nth) Q[r] = sD[r] + sdQ[r];
}

template <typename T, int N>
__global__ void __launch_bounds__(kThreads) neighbour_kernel(StepArgs a) {
  constexpr int B = nb3(N), Bf = nb2(N);
  __shared__ T sV[36 * Bf];   // neighbours' time-integrated traces (this face's node order)
  __shared__ T sVo[36 * Bf];  // own time-integrated traces
  __shared__ T sG[36 * Bf];
  __shared__ T sFp[4 * 81];
  __shared__ T sFm[4 * 81];
  __shared__ T sScale[4];
  __shared__ int sKind[4];
  __shared__ int sGrav[4];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int64_t v = a.v_begin + blockIdx.x;
  const int64_t e = v / a.S;
  const int s = (int)(v - e * a.S);
  const T* liftT = reinterpret_cast<const T*>(a.liftT);
  if (tid < 4) {
    sScale[tid] = reinterpret_cast<const T*>(a.par)[e * PAR + 12 + tid];
    sKind[tid] = (a.ninfo[e * 4 + tid] >> 5) & 7;
    sGrav[tid] = a.gslot ? a.gslot[e * 4 + tid] : -1;
  }
  for (int r = tid; r < 4 * 81; r += nth) {
    sFp[r] = reinterpret_cast<const T*>(a.Fp)[e * 4 * 81 + r];
    sFm[r] = reinterpret_cast<const T*>(a.Fm)[e * 4 * 81 + r];
  }
  for (int r = tid; r < 36 * Bf; r += nth) sVo[r] = reinterpret_cast<const T*>(a.trace)[v * 36 * Bf + r];
  __syncthreads();
  for (int r = tid; r < 36 * Bf; r += nth) {
    const int f = r / (9 * Bf), p = (r / Bf) % 9, n = r % Bf;
    const int info = a.ninfo[e * 4 + f];
    const int kind = (info >> 5) & 7;
    T val = T(0);
    if (kind != NK_NONE && kind != NK_FAULT) {
      const int64_t nb = a.nbr[e * 4 + f];
      const int j = info & 3, pm = (info >> 2) & 7;
      const int src = a.perm[pm * Bf + n];
      if (kind == NK_SAME) {
        val = reinterpret_cast<const T*>(a.trace)[((nb * a.S + s) * 4 + j) * 9 * Bf + p * Bf + src];
      } else if (kind == NK_FINE) {
        const int bs = a.bslot[nb];
        val = (T)a.btrace[(((int64_t)bs * a.S + s) * 4 + j) * 9 * Bf + p * Bf + src];
      } else {  // NK_COARSE: integrate the coarser neighbour's expansion over this sub-interval
        const int ds = a.dslot[nb * 4 + j];
        const T* dt = reinterpret_cast<const T*>(a.dtrace) + ((int64_t)ds * a.S + s) * (N + 1) * 9 * Bf;
        T acc = T(0);
#pragma unroll
        for (int k = 0; k <= N; ++k) acc += T(a.ccoef[k]) * dt[(k * 9 + p) * Bf + src];
        val = acc;
      }
    }
    sV[r] = val;
  }
  __syncthreads();
  // face fluxes G[f][q][n]: F^- (own) + F^+ (neighbour) on interior faces,
  // F^- with the ghost folded in on linear boundaries, the precomputed fluxes on
  // gravitational (local kernel) and fault faces (rupture kernel)
  for (int r = tid; r < 36 * Bf; r += nth) {
    const int f = r / (9 * Bf), q = (r / Bf) % 9, n = r % Bf;
    T acc = T(0);
    if (sKind[f] == NK_FAULT) {
      // time-integrated fault flux of this side, already in this face's node order
      const int fsl = a.fslot[e * 4 + f];
      acc = reinterpret_cast<const T*>(a.drout)[((((int64_t)(fsl >> 1) * a.S + s) * 2 + (fsl & 1)) * 9 + q) * Bf + n];
    } else if (sGrav[f] >= 0) {
      acc = reinterpret_cast<const T*>(a.gflux)[((int64_t)sGrav[f] * a.S + s) * 9 * Bf + q * Bf + n];
    } else {
#pragma unroll
      for (int p = 0; p < 9; ++p) acc += sFm[f * 81 + q * 9 + p] * sVo[(f * 9 + p) * Bf + n];
      if (sKind[f] != NK_NONE) {
#pragma unroll
        for (int p = 0; p < 9; ++p) acc += sFp[f * 81 + q * 9 + p] * sV[(f * 9 + p) * Bf + n];
      }
    }
    sG[r] = acc;
  }
  __syncthreads();
  T* Q = reinterpret_cast<T*>(a.Q) + v * 9 * B;
  bool bad = false;
  for (int r = tid; r < 9 * B; r += nth) {
    const int q = r / B, m = r % B;
    T acc = T(0);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      T af = T(0);
      const T* lf = liftT + (size_t)f * Bf * B + m;
      const T* g = sG + (f * 9 + q) * Bf;
      for (int n = 0; n < Bf; ++n) af += lf[(size_t)n * B] * g[n];
      acc += sScale[f] * af;
    }
    const T nq = Q[r] - acc;
    Q[r] = nq;
    bad |= !isfinite((double)nq);
  }
  if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0) atomicOr(a.err, ERR_NAN);
}

template <typename T, int N>
int launch_local_t(const StepArgs& a, int64_t nblocks, cudaStream_t st) {
  constexpr int bytes = Smem<T, N>::bytes;
  static bool configured = false;
  if (!configured) {
    cudaError_t ce = cudaFuncSetAttribute(local_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (ce != cudaSuccess) return (int)ce;
    configured = true;
  }
  if (nblocks <= 0) return 0;
  local_kernel<T, N><<<(unsigned)nblocks, kThreads, bytes, st>>>(a);
  return (int)cudaGetLastError();
}

template <typename T, int N>
int launch_neighbour_t(const StepArgs& a, int64_t nblocks, cudaStream_t st) {
  if (nblocks <= 0) return 0;
  neighbour_kernel<T, N><<<(unsigned)nblocks, kThreads, 0, st>>>(a);
  return (int)cudaGetLastError();
}

template <typename T>
int dispatch_local(int N, const StepArgs& a, int64_t nb, cudaStream_t st) {
  switch (N) {
    case 1: return launch_local_t<T, 1>(a, nb, st);
    case 2: return launch_local_t<T, 2>(a, nb, st);
    case 3: return launch_local_t<T, 3>(a, nb, st);
    case 4: return launch_local_t<T, 4>(a, nb, st);
    case 5: return launch_local_t<T, 5>(a, nb, st);
  }
  return (int)cudaErrorInvalidValue;
}
template <typename T>
int dispatch_neighbour(int N, const StepArgs& a, int64_t nb, cudaStream_t st) {
  switch (N) {
    case 1: return launch_neighbour_t<T, 1>(a, nb, st);
    case 2: return launch_neighbour_t<T, 2>(a, nb, st);
    case 3: return launch_neighbour_t<T, 3>(a, nb, st);
    case 4: return launch_neighbour_t<T, 4>(a, nb, st);
    case 5: return launch_neighbour_t<T, 5>(a, nb, st);
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

// Local element kernel on the tensor cores (tcgen05, 3xTF32), degrees 5 and
// 4, FP32 dofs: Cauchy-Kovalewski predictor, time integral, face traces and
// volume term of Sec. 4.1 for elements without fault faces or two or more
// gravitational faces (those take the CUDA-core kernel); an element with a
// coarser LTS neighbour also adds its
// traces to its FP64 LTS buffer; elements with one gravitational face or a
// finer LTS neighbour take a special instantiation that also forms the
// gravitational face's (eta, H) update and the derivative traces of every
// level on faces with a finer neighbour.
//
// A tile is 12 (virtual) elements x 9 quantities = the 128 rows of the MMAs,
// one row per TMEM lane: warp w of a warpgroup holds elements 3w..3w+2, the
// j-th of them in lanes 9j..9j+8 (lane 9j+p = quantity p); lanes 27..31 are
// zero padding.  Every product with a reference matrix is then
//   rows(element, quantity) x reference matrix^T
// with the element data as the A operand in TMEM (split into tf32 hi + lo by
// the threads that own the rows) and the reference matrices as B operands,
// resident in shared memory in the canonical K-major layout (hi and lo);
// A_hi B_hi + A_hi B_lo + A_lo B_hi accumulate in fp32 in TMEM.  Per tile:
//   levels k < N - 2:  Y = D^k [KT_0; KT_1; KT_2]^T on the tensor cores,
//     then X_d = sum_a (dxi_a/dx_d) Y_a and D^{k+1} = -sum_d A_d X_d on the CUDA
//     cores (Jacobian form of the star product; the quantities of an element
//     are exchanged with warp shuffles);
//   the last two levels (4 and 1 rows) on the CUDA cores from registers;
//   I = sum_k dt^{k+1}/(k+1)! D^k in registers (Eq. taylor);
//   traces V_f = E_f I on the tensor cores, staged per face in shared memory
//     and written to the trace array with bulk copies (cp.async.bulk);
//   volume: W_a = K_a I for the three axes on the tensor cores, then
//     Q += sum_a A*_a W_a on the CUDA cores (Jacobian form, shuffles).
// The operand image reaches shared memory once per CTA by TMA bulk copies.
// A CTA keeps two tiles in flight (TMEM columns [0, 256) and [256, 512)), each
// worked on by two warpgroups that split every stage by 8-column chunks (even
// chunks: first half, odd chunks: second half); one thread per tile issues
// its MMAs and waits for their completion with a bounded mbarrier wait.
//
// Acoustic ocean (Sec. 4.1: the fluid is the elastic system with mu = 0;
// stress -p I): the fluid instantiation works on the 4 quantities (p, v) only,
// stored as the sigma_xx row (sigma_yy = sigma_zz = sigma_xx, no shear) and
// the velocity rows.  A tile is then 32 elements x 4 quantities (warp w:
// elements 8w..8w+7, lane 4j+p), all 128 rows in use; the star product is the
// acoustic one, dsigma/dt = lambda div v and dv/dt = grad(sigma_xx) / rho in
// the same Jacobian form; the element's face blocks are written in the full
// 9-quantity layout (three equal normal-stress rows, zero shear), so
// neighbours and the neighbour kernel see ordinary traces.
//
// Degree 4 (35 basis functions): a dofs row is 140 bytes, not a multiple of 16,
// so the tile's rows are staged in shared memory with coalesced loads at the
// start of the tile (its rows are consecutive in memory) and written back the
// same way after the volume update.
//
// This header holds the kernel for both degrees; local_tc.cu and local_tc4.cu
// instantiate it (one degree per translation unit, compiled in parallel).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "func_attr.hpp"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace adg {

namespace {

constexpr int kThreadsL = 512;  // two tiles in flight, two warpgroups (halves) per tile

// The medium of an instantiation: quantities per element (rows of the tile),
// elements per warp and per tile, and the dofs row of quantity p.
struct Elastic {
  static constexpr bool fluid = false;
  static constexpr int Q = 9, EW = 3, TE = kTileElems;
  static __device__ __forceinline__ int row(int p) { return p; }
};
struct Acoustic {
  static constexpr bool fluid = true;
  static constexpr int Q = 4, EW = 8, TE = kTileElemsFluid;
  static __device__ __forceinline__ int row(int p) { return p == 0 ? 0 : 5 + p; }  // sigma_xx, v_x, v_y, v_z
};
static_assert(Elastic::TE == 4 * Elastic::EW && Acoustic::TE == 4 * Acoustic::EW, "tile of 4 warps");
constexpr int kWaitIters = 1 << 24;

constexpr int r8(int x) { return (x + 7) / 8 * 8; }
constexpr int r16(int x) { return (x + 15) / 16 * 16; }

// Shapes of degree N.  Predictor level l on the tensor cores multiplies D^l
// (KU[l] rows used, K[l] padded to 8) by the three stacked KT_a, keeping the
// M[l] rows of D^{l+1} per axis (padded to MP[l]; N = NN[l] = 3 MP[l] padded
// to 16); the last tensor-core level leaves the 10 rows of D^{N-2}, and the
// CUDA cores take D^{N-1} (4 rows) and D^N (1 row).  TS: floats per element in
// the trace staging buffer (the face block, then zeros; 16-byte multiple).
template <int N>
struct LDeg;
template <>
struct LDeg<5> {
  static constexpr int B = 56, B1 = 35, BF = 21, NL = 3, TS = 196;
  static constexpr int K[3] = {56, 40, 24}, KU[3] = {56, 35, 20}, M[3] = {35, 20, 10}, MP[3] = {40, 24, 16},
                       NN[3] = {128, 80, 48};
};
template <>
struct LDeg<4> {
  static constexpr int B = 35, B1 = 20, BF = 15, NL = 2, TS = 140;
  static constexpr int K[3] = {40, 24, 0}, KU[3] = {35, 20, 0}, M[3] = {20, 10, 0}, MP[3] = {24, 16, 0},
                       NN[3] = {80, 48, 0};
};

// derived shapes and the shared-memory image of the operands (floats), hi
// block then lo block each
template <int N>
struct LImg : LDeg<N> {
  using D = LDeg<N>;
  static constexpr int B = D::B, B1 = D::B1, BF = D::BF, NL = D::NL;
  static constexpr int BP = r8(B);            // a row padded to whole 8-column chunks
  static constexpr int NCH = BP / 8;          // 8-column chunks of a row
  static constexpr int FS = face_stride(N);   // floats per face block of the trace array
  static constexpr int NT = r16(4 * BF);      // traces: 4 faces x BF nodes, padded; K = BP
  static constexpr int NTCH = (4 * BF + 7) / 8;  // 8-column chunks holding traces
  static constexpr int KV = r8(B1);           // volume: K = the B1 rows of I that K_a reads
  static constexpr int NV = r16(3 * BP);      // volume: axis a, basis m at column BP a + m
  static constexpr bool kAligned = B % 4 == 0;  // dofs rows 16-byte aligned (float4 access)
  static constexpr int oP0 = 0, sP0 = D::NN[0] * D::K[0];
  static constexpr int oP1 = oP0 + 2 * sP0, sP1 = D::NN[1] * D::K[1];
  static constexpr int oP2 = oP1 + 2 * sP1, sP2 = D::NN[2] * D::K[2];
  static constexpr int oV = oP2 + 2 * sP2, sV = NV * KV;
  static constexpr int oT = oV + 2 * sV, sT = NT * BP;
  static constexpr int oK3 = oT + 2 * sT;     // kt[a][m][l], m < 4, l < 10
  static constexpr int oK4 = oK3 + 120;       // kt[a][0][l], l < 4
  static constexpr int floats = ((oK4 + 12 + 3) / 4) * 4;
  // degree 4: per slot, two buffers of a tile's dofs rows [row][B] (32 x 4 acoustic rows at most)
  static constexpr int oQ = floats, sQ = kAligned ? 0 : 128 * B;
  static constexpr int bytes = (floats + 2 * 2 * sQ) * 4;
  // A hi at [0, 64), lo at [64, 128), accumulators from 128; volume: A at [0, 2 KV), accumulators after
  static_assert(BP <= 64 && D::NN[0] <= 128 && NT <= 128 && 2 * KV + NV <= 256, "TMEM columns of a slot");
};

// trace staging: per warp pair one face of its elements, two buffers
// alternating over the faces (sized for degree 5, the larger)
constexpr int kTB = 3 * LDeg<5>::TS;
static_assert(LImg<5>::bytes + 2 * (2 * 128 + 4 * 2 * kTB) * 4 + 64 <= 232448 &&
                  LImg<4>::bytes + 2 * (2 * 128 + 4 * 2 * kTB) * 4 + 64 <= 232448,
              "operands exceed the shared memory of one CTA");

// the kernel's shared memory besides the operand image (dynamic): per slot the
// MMA barrier, abort flag, rows 8, 9 of D^3 handed from half 1 to half 0, and
// per warp pair two trace staging buffers
__shared__ __align__(8) uint64_t s_mbar[2];
__shared__ int s_abort[2];
__shared__ float s_X[2][2 * 128];
__shared__ __align__(16) float s_T[2][4][2 * kTB];
extern __shared__ __align__(1024) unsigned char smem_raw[];

// per-warpgroup TMEM columns: A hi [0, 64), A lo [64, 128), accumulators [128, 256)
constexpr uint32_t cAh = 0, cAl = 64, cAcc = 128;

// Per-thread star-product data: the quantity p of this lane's row, the lanes
// of the quantities each output reads and their material coefficients.
// D^{k+1}[p] = sum_d c_d X_d[src_d] with X_d = sum_a (dxi_a/dx_d) Y_a, the
// Jacobian form of -sum_a A*_a Y_a (Eq. elasticity-pde); the volume operand
// is Z_a[p] = -sum_d (dxi_a/dx_d) c_d I[src_d].
struct Star {
  float g[9];    // g[a*3+d] = d xi_a / d x_d
  float c[3];    // coefficients of the three directions
  int src[3];    // source lanes
};

__device__ __forceinline__ void star_setup(int lane, bool valid, const float* par, Star& s) {
  const int j = lane / 9, p = lane - 9 * (lane / 9);
  const int base = 9 * j;
  float lam = 0.f, mu = 0.f, irho = 0.f;
  if (valid) {
#pragma unroll
    for (int k = 0; k < 9; ++k) s.g[k] = par[k];
    irho = 1.f / par[9];
    lam = par[10];
    mu = par[11];
  } else {
#pragma unroll
    for (int k = 0; k < 9; ++k) s.g[k] = 0.f;
  }
  const float l2m = lam + 2.f * mu;
  // (source quantity, coefficient) per direction d for output quantity p
  int q0 = p, q1 = p, q2 = p;
  float c0 = 0.f, c1 = 0.f, c2 = 0.f;
  switch (p) {
    case 0: q0 = 6; c0 = l2m; q1 = 7; c1 = lam; q2 = 8; c2 = lam; break;
    case 1: q0 = 6; c0 = lam; q1 = 7; c1 = l2m; q2 = 8; c2 = lam; break;
    case 2: q0 = 6; c0 = lam; q1 = 7; c1 = lam; q2 = 8; c2 = l2m; break;
    case 3: q0 = 7; c0 = mu; q1 = 6; c1 = mu; break;
    case 4: q1 = 8; c1 = mu; q2 = 7; c2 = mu; break;
    case 5: q0 = 8; c0 = mu; q2 = 6; c2 = mu; break;
    case 6: q0 = 0; c0 = irho; q1 = 3; c1 = irho; q2 = 5; c2 = irho; break;
    case 7: q0 = 3; c0 = irho; q1 = 1; c1 = irho; q2 = 4; c2 = irho; break;
    default: q0 = 5; c0 = irho; q1 = 4; c1 = irho; q2 = 2; c2 = irho; break;
  }
  if (lane >= 27) { q0 = q1 = q2 = 0; c0 = c1 = c2 = 0.f; }
  s.c[0] = c0; s.c[1] = c1; s.c[2] = c2;
  s.src[0] = (lane >= 27 ? lane : base + q0);
  s.src[1] = (lane >= 27 ? lane : base + q1);
  s.src[2] = (lane >= 27 ? lane : base + q2);
}

// The acoustic star data of lane 4j + p (p = 0: sigma_xx = -p_pressure,
// p = 1..3: v_x, v_y, v_z): the normal stress reads the three velocities with
// lambda (mu = 0), velocity component d reads the normal stress in direction
// d with 1/rho, the other two directions nothing.
__device__ __forceinline__ void star_setup_acoustic(int lane, bool valid, const float* par, Star& s) {
  const int p = lane & 3, base = lane & ~3;
  float lam = 0.f, irho = 0.f;
  if (valid) {
#pragma unroll
    for (int k = 0; k < 9; ++k) s.g[k] = par[k];
    irho = 1.f / par[9];
    lam = par[10];
  } else {
#pragma unroll
    for (int k = 0; k < 9; ++k) s.g[k] = 0.f;
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    s.c[d] = p == 0 ? lam : (p == d + 1 ? irho : 0.f);
    s.src[d] = p == 0 ? base + 1 + d : (p == d + 1 ? base : lane);
  }
}

// one output of the star product from the three axis values of this lane
__device__ __forceinline__ float star_apply(const Star& s, float y0, float y1, float y2) {
  const float X0 = s.g[0] * y0 + s.g[3] * y1 + s.g[6] * y2;
  const float X1 = s.g[1] * y0 + s.g[4] * y1 + s.g[7] * y2;
  const float X2 = s.g[2] * y0 + s.g[5] * y1 + s.g[8] * y2;
  const float a0 = __shfl_sync(0xffffffffu, X0, s.src[0]);
  const float a1 = __shfl_sync(0xffffffffu, X1, s.src[1]);
  const float a2 = __shfl_sync(0xffffffffu, X2, s.src[2]);
  return s.c[0] * a0 + s.c[1] * a1 + s.c[2] * a2;
}

// Epilogue of a tensor-core predictor level for the 8-column chunks mc with
// mc % 2 == H: Y (3 axes x MP columns at tacc) -> D^{k+1} (M rows),
// I += ck * D^{k+1}; D^{k+1} goes to the A columns of the next level (TO_A)
// or to registers dn.
// Gravitational free surface (Sec. 4.3) on the tensor-core kernel, for an
// element with one gravitational face: per thread (row p of its element) the
// weight w_p of that row in v_n - sigma_nn / Z at the face (normal n, P
// impedance Z), the element's scratch (null on other rows than p = 0 and on
// lanes without such an element) and the first lane of its element.
struct Grav {
  float w = 0.f;
  float* dst = nullptr;
  int base = 0;
};
// 1/k and 1/k! for the gravitational face's Taylor series (products, not FP64 divisions)
__constant__ double kRcp[48] = {0.0, 1.0 / 1, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6, 1.0 / 7, 1.0 / 8,
                                1.0 / 9, 1.0 / 10, 1.0 / 11, 1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16,
                                1.0 / 17, 1.0 / 18, 1.0 / 19, 1.0 / 20, 1.0 / 21, 1.0 / 22, 1.0 / 23, 1.0 / 24,
                                1.0 / 25, 1.0 / 26, 1.0 / 27, 1.0 / 28, 1.0 / 29, 1.0 / 30, 1.0 / 31, 1.0 / 32,
                                1.0 / 33, 1.0 / 34, 1.0 / 35, 1.0 / 36, 1.0 / 37, 1.0 / 38, 1.0 / 39, 1.0 / 40,
                                1.0 / 41, 1.0 / 42, 1.0 / 43, 1.0 / 44, 1.0 / 45, 1.0 / 46, 1.0 / 47};
__constant__ double kRcpFact[6] = {1.0, 1.0, 1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120};

// sum over the 9 rows of this lane's element of w_p x_p (every lane of the warp takes part)
__device__ __forceinline__ float elem_sum9(float v, int base) {
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) s += __shfl_sync(0xffffffffu, v, (base + k) & 31);
  return s;
}

template <int H, int M, int MP, bool TO_A, bool kG, int BP>
__device__ __forceinline__ void level_epilogue(uint32_t tacc, uint32_t tah, uint32_t tal, const Star& s, float ck,
                                               float (&I)[BP], float* dn, const Grav& gv, int goff) {
#pragma unroll
  for (int mc = H; mc < MP / 8; mc += 2) {
    float y[24];
    tc::ld3x8(tacc + 8 * mc, tacc + MP + 8 * mc, tacc + 2 * MP + 8 * mc, y);
    float d[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int m = 8 * mc + j;
      if (m < M) {
        d[j] = star_apply(s, y[j], y[8 + j], y[16 + j]);
        I[m] += ck * d[j];
        if (!TO_A) dn[m] = d[j];
      } else {
        d[j] = 0.f;
      }
      if constexpr (kG) {  // the gravitational face's projected row of this level
        const float g = elem_sum9(gv.w * d[j], gv.base);
        if (gv.dst && m < M) gv.dst[goff + m] = g;
      }
    }
    if (TO_A) tc::st_split8(tah + 8 * mc, tal + 8 * mc, d);
  }
}

__device__ __forceinline__ void pair_bar(int slot) { asm volatile("bar.sync %0, 256;" ::"r"(slot + 1)); }
// the two warps (one per half) of a slot that hold the same 32 rows
__device__ __forceinline__ void warp_pair_bar(int slot, int w) {
  asm volatile("bar.sync %0, 64;" ::"r"(3 + 4 * slot + w));
}

// Everything one thread needs to work on the tiles of its slot.
// (Arrays and sizes come from the launch's StepArgs, read where they are used.)
struct Lane {
  float tcf[6];       // dt^{k+1}/(k+1)!, k = 0..5, of the tile's cluster
  int slot, t, w, lane;
  uint32_t tbase, trow, sbase;
  int btrace_mode;    // of the tile's cluster: 0 none, 1 overwrite, 2 accumulate (LTS buffers)
  uint32_t phase;
  int it;             // tiles this slot has begun (degree 4: the staged-rows buffer of a tile is it % 2)
  double dt;          // the tile's cluster step (gravitational faces)
};

// One tensor-core round of a slot: both halves' A stores made visible, MMAs
// issued by thread 0 of half 0, bounded wait for their completion.
template <int H, class F>
__device__ __forceinline__ bool pair_round(Lane& L, unsigned int* err, F&& issue_fn) {
  asm volatile("tcgen05.wait::st.sync.aligned;");
  tc::fence_before();
  pair_bar(L.slot);
  tc::fence_after();
  if (H == 0 && L.t == 0) {
    issue_fn();
    tc::commit(&s_mbar[L.slot]);
    if (!tc::mbar_wait(&s_mbar[L.slot], L.phase, kWaitIters)) {
      atomicOr(err, ERR_TIMEOUT);
      s_abort[L.slot] = 1;
    }
  }
  pair_bar(L.slot);
  const bool ok = !*(volatile int*)&s_abort[L.slot];
  if (ok) tc::mbar_wait(&s_mbar[L.slot], L.phase, 1 << 20);  // observe the completed phase in every thread
  L.phase ^= 1u;
  tc::fence_after();
  return ok;
}

// Degree 4: the tile's dofs rows in shared memory.  The 256 threads of the
// slot (u) copy the rows of the tile's elements [v0, v0 + nE) with coalesced
// loads (a tile's rows are consecutive in memory; an acoustic tile takes rows
// 0 and 6..8 of each element); tile row (element ei, quantity qi) sits at
// (ei * M::Q + qi) * B.
// (asynchronous: cp.async of 4 bytes each, committed by the caller)
template <class M, int B>
__device__ __forceinline__ void rows_load(float* sQ, const float* Q, int64_t v0, int nE, int u) {
  const int n = nE * M::Q * B;
  for (int i = u; i < n; i += 256) {
    int64_t src;
    if constexpr (M::fluid) {
      const int ej = i / (4 * B), r = i - ej * 4 * B;
      src = (v0 + ej) * 9 * B + (r < B ? r : 5 * B + r);
    } else {
      src = v0 * 9 * B + i;
    }
    tc::cp_async4(sQ + i, Q + src);
  }
}
// ... and back (acoustic: the normal-stress row as sigma_xx, sigma_yy and
// sigma_zz, then the velocity rows; the shear rows stay zero)
template <class M, int B>
__device__ __forceinline__ void rows_store(const float* sQ, float* Q, int64_t v0, int nE, int u) {
  if constexpr (M::fluid) {
    const int n = nE * 6 * B;
    for (int i = u; i < n; i += 256) {
      const int ej = i / (6 * B), r = i - ej * 6 * B;
      const int qi = r < 3 * B ? 0 : 1 + (r - 3 * B) / B;
      const int k = r < 3 * B ? r % B : (r - 3 * B) % B;
      Q[(v0 + ej) * 9 * B + (r < 3 * B ? r : 3 * B + r)] = sQ[(ej * 4 + qi) * B + k];
    }
  } else {
    const int n = nE * 9 * B;
    for (int i = u; i < n; i += 256) Q[v0 * 9 * B + i] = sQ[i];
  }
}

// One tile, the share of half H (8-column chunks c with c % 2 == H); false
// after a timed-out wait.
// kBuf: some elements of the launch have an LTS buffer (a coarser neighbour)
// tile: index within its segment; t2: this slot's tile after the next among
// all tiles of the launch (kMulti: the launch has several segments)
// Derivative traces of level m (Sec. 4.4: a finer neighbour integrates this
// element's Taylor expansion over its sub-steps) on this row's faces with a
// finer neighbour: one tensor-core round T = D^m E^T with D^m the A operand
// in TMEM (K = KM), then this half's trace chunks to dtr[f] (null: no finer
// neighbour on face f; [N+1][9][Bf] per face, this row's quantity already
// offset).  False after a timed-out wait.
template <int N, int H, int KM>
__device__ __forceinline__ bool dtrace_round(Lane& L, const StepArgs& a, float* const (&dtr)[4], int m) {
  using I_ = LImg<N>;
  constexpr int BF = I_::BF, NTH = H == 0 ? (I_::NTCH + 1) / 2 : I_::NTCH / 2;
  if (!pair_round<H>(L, a.err, [&] {
        tc::mma3_ts<I_::NT, KM>(L.tbase + cAcc, L.tbase + cAh, L.tbase + cAl, L.sbase + 4 * I_::oT,
                                L.sbase + 4 * (I_::oT + I_::sT), false);
      }))
    return false;
  const uint32_t trow = L.trow;
  float tv[48];
  if constexpr (N == 5) {
    tc::ld3x8(trow + cAcc + 8 * H, trow + cAcc + 8 * (H + 2), trow + cAcc + 8 * (H + 4), tv);
    tc::ld3x8(trow + cAcc + 8 * (H + 6), trow + cAcc + 8 * (H + 8), trow + cAcc + 8 * (H == 0 ? 10 : 9), tv + 24);
  } else {
    tc::ld3x8(trow + cAcc + 8 * H, trow + cAcc + 8 * (H + 2), trow + cAcc + 8 * (H + 4), tv);
    tc::ld8(trow + cAcc + 8 * (H + 6), tv + 24);
  }
#pragma unroll
  for (int cj = 0; cj < NTH; ++cj) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int col = 8 * (H + 2 * cj) + j;
      if (col < 4 * BF) {
        const int f = col / BF, n = col - f * BF;
        if (dtr[f]) dtr[f][m * 9 * BF + n] = tv[8 * cj + j];
      }
    }
  }
  return true;
}

// kSpec: the launch's elements may have one gravitational face and faces with
// a finer LTS neighbour (elastic instantiation)
template <int N, class M, int H, bool kBuf, bool kMulti, bool kSpec>
__device__ __forceinline__ bool local_tile(Lane& L, const StepArgs& a, const Segs& g, int64_t t1, int64_t t2,
                                           int64_t v_begin, int64_t n_virtual, int64_t tile) {
  using D = LDeg<N>;
  using I_ = LImg<N>;
  constexpr int B = I_::B, BF = I_::BF, BP = I_::BP, NCH = I_::NCH, FS = I_::FS, TS = D::TS, NL = D::NL;
  constexpr int TE = M::TE;
  float* const Q = reinterpret_cast<float*>(a.Q);
  const int64_t v0 = v_begin + tile * TE;
  const int64_t nrem = n_virtual - tile * TE;
  const int nE = (int)(nrem < TE ? nrem : TE);
  const int jj = L.lane / M::Q, p = L.lane - M::Q * (L.lane / M::Q);
  const int i = M::EW * L.w + jj;
  const bool valid = L.lane < M::EW * M::Q && i < nE;
  const int64_t v = v0 + (valid ? i : 0);
  const int64_t e = v / a.S;
  Star st;
  if constexpr (M::fluid)
    star_setup_acoustic(L.lane, valid, reinterpret_cast<const float*>(a.par) + e * PAR, st);
  else
    star_setup(L.lane, valid, reinterpret_cast<const float*>(a.par) + e * PAR, st);
  const uint32_t trow = L.trow, tbase = L.tbase, sbase = L.sbase;
  // gravitational face of this row's element
  Grav gv;
  int gface = -1, gsl = -1;
  if constexpr (kSpec) {
    static_assert(!M::fluid, "gravitational faces take the elastic instantiation");
    gv.base = 9 * jj;
    if (valid && a.gslot) {
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const int gs = a.gslot[e * 4 + f];
        if (gs >= 0) { gface = f; gsl = gs; }
      }
    }
    if (gsl >= 0) {
      const double* gp = a.gpar + (int64_t)gsl * GPAR;
      const float nx = (float)gp[0], ny = (float)gp[1], nz = (float)gp[2], iz = (float)(1.0 / gp[3]);
      const float w[9] = {-nx * nx * iz, -ny * ny * iz, -nz * nz * iz, -2.f * nx * ny * iz, -2.f * ny * nz * iz,
                          -2.f * nx * nz * iz, nx, ny, nz};
      gv.w = w[p];
      if (p == 0) gv.dst = a.gscr + ((int64_t)gsl * a.S + (v - e * a.S)) * gscr_floats(N);
    }
  }
  // faces with a finer neighbour: this row's derivative traces there; tile_fine:
  // some element of the tile has one (the same answer in every thread of the slot)
  float* dtr[4] = {nullptr, nullptr, nullptr, nullptr};
  bool tile_fine = false;
  if constexpr (kSpec) {
    if (a.dslot)
      for (int k = 0; k < 4 * nE; ++k) tile_fine |= a.dslot[((v0 + (k >> 2)) / a.S) * 4 + (k & 3)] >= 0;
    if (valid && a.dslot) {
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const int ds = a.dslot[e * 4 + f];
        if (ds >= 0)
          dtr[f] = reinterpret_cast<float*>(a.dtrace) + ((int64_t)ds * a.S + (v - e * a.S)) * (N + 1) * 9 * BF + p * BF;
      }
    }
  }

  // the tile after the next of this slot into L2 while this one is worked on
  if (H == 0 && L.t == 0) {
    if (t2 < g.first[g.n]) {
      const int i2 = seg_of<kMulti>(g, t2);
      const int64_t l2 = t2 - g.first[i2], rem2 = g.s[i2].n - l2 * TE;
      tc::prefetch_l2_inner(Q + (g.s[i2].v_begin + l2 * TE) * 9 * B, (uint32_t)((rem2 < TE ? rem2 : TE) * 9 * B * 4));
    }
  }
  // ---- D^0 = Q row: I = dt Q, A = Q
  float* Qrow = Q + (v * 9 + M::row(p)) * B;
  float* sQ = nullptr;   // degree 4: the slot's staged rows
  float* srow = nullptr; // ... and this thread's
  if constexpr (!I_::kAligned) {
    // two buffers per slot: this tile's rows were requested during the
    // previous tile (the first tile's here), the next tile's are requested now
    float* const sQb = reinterpret_cast<float*>(smem_raw) + I_::oQ + L.slot * 2 * I_::sQ;
    sQ = sQb + (L.it & 1) * I_::sQ;
    srow = sQ + (i * M::Q + p) * B;
    pair_bar(L.slot);  // the previous tile's rows have been written back from the other buffer
    if (L.it == 0) {
      rows_load<M, B>(sQ, Q, v0, nE, L.t + 128 * H);
      tc::cp_async_commit();
    }
    if (t1 < g.first[g.n]) {
      const int i1 = seg_of<kMulti>(g, t1);
      const int64_t l1 = t1 - g.first[i1], rem1 = g.s[i1].n - l1 * TE;
      rows_load<M, B>(sQb + ((L.it + 1) & 1) * I_::sQ, Q, g.s[i1].v_begin + l1 * TE, (int)(rem1 < TE ? rem1 : TE),
                      L.t + 128 * H);
    }
    tc::cp_async_commit();
    tc::cp_async_wait<1>();  // this tile's rows
    pair_bar(L.slot);
  }
  float I[BP];
#pragma unroll
  for (int c = H; c < NCH; c += 2) {
    float x[8];
    if constexpr (I_::kAligned) {
      float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f), x1 = x0;
      if (valid) {
        x0 = *reinterpret_cast<const float4*>(Qrow + 8 * c);
        x1 = *reinterpret_cast<const float4*>(Qrow + 8 * c + 4);
      }
      x[0] = x0.x; x[1] = x0.y; x[2] = x0.z; x[3] = x0.w;
      x[4] = x1.x; x[5] = x1.y; x[6] = x1.z; x[7] = x1.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = (valid && 8 * c + j < B) ? srow[8 * c + j] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) I[8 * c + j] = L.tcf[0] * x[j];
    if constexpr (kSpec) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float gsum = elem_sum9(gv.w * x[j], gv.base);
        if (gv.dst && 8 * c + j < B) gv.dst[gscr_off(N, 0) + 8 * c + j] = gsum;
      }
    }
    tc::st_split8(trow + cAh + 8 * c, trow + cAl + 8 * c, x);
  }
  // ---- predictor levels on the tensor cores: all but the last feed the next
  // level's A operand, the last leaves the 10 rows of D^NL in registers
  if constexpr (NL == 3) {
    if constexpr (kSpec) {
      if (tile_fine && !dtrace_round<N, H, D::K[0]>(L, a, dtr, 0)) return false;
    }
    if (!pair_round<H>(L, a.err, [&] {
          tc::mma3_ts<D::NN[0], D::K[0]>(tbase + cAcc, tbase + cAh, tbase + cAl, sbase + 4 * I_::oP0,
                                         sbase + 4 * (I_::oP0 + I_::sP0), false);
        }))
      return false;
    level_epilogue<H, D::M[0], D::MP[0], true, kSpec>(trow + cAcc, trow + cAh, trow + cAl, st, L.tcf[1], I, nullptr,
                                                      gv, gscr_off(N, 1));
  }
  constexpr int l1 = NL - 2, l2 = NL - 1;
  constexpr int o1 = l1 == 0 ? I_::oP0 : I_::oP1, s1 = l1 == 0 ? I_::sP0 : I_::sP1;
  constexpr int o2 = l2 == 1 ? I_::oP1 : I_::oP2, s2 = l2 == 1 ? I_::sP1 : I_::sP2;
  if constexpr (kSpec) {
    if (tile_fine && !dtrace_round<N, H, D::K[l1]>(L, a, dtr, l1)) return false;
  }
  if (!pair_round<H>(L, a.err, [&] {
        tc::mma3_ts<D::NN[l1], D::K[l1]>(tbase + cAcc, tbase + cAh, tbase + cAl, sbase + 4 * o1,
                                         sbase + 4 * (o1 + s1), false);
      }))
    return false;
  level_epilogue<H, D::M[l1], D::MP[l1], true, kSpec>(trow + cAcc, trow + cAh, trow + cAl, st, L.tcf[l1 + 1], I,
                                                     nullptr, gv, gscr_off(N, l1 + 1));
  if constexpr (kSpec) {
    if (tile_fine && !dtrace_round<N, H, D::K[l2]>(L, a, dtr, l2)) return false;
  }
  if (!pair_round<H>(L, a.err, [&] {
        tc::mma3_ts<D::NN[l2], D::K[l2]>(tbase + cAcc, tbase + cAh, tbase + cAl, sbase + 4 * o2,
                                         sbase + 4 * (o2 + s2), false);
      }))
    return false;
  static_assert(D::M[l2] == 10 && D::MP[l2] == 16, "the last tensor-core level leaves 10 rows");
  float dl[16];
  level_epilogue<H, D::M[l2], D::MP[l2], false, kSpec>(trow + cAcc, trow + cAh, trow + cAl, st, L.tcf[NL], I, dl, gv,
                                                      gscr_off(N, l2 + 1));
  // ---- the last two levels (half 0, with rows 8 and 9 of D^NL from half 1)
  if (H == 1) {
    s_X[L.slot][2 * L.t] = dl[8];
    s_X[L.slot][2 * L.t + 1] = dl[9];
  }
  pair_bar(L.slot);
  if (H == 0) {
    dl[8] = s_X[L.slot][2 * L.t];
    dl[9] = s_X[L.slot][2 * L.t + 1];
    const float* k3 = reinterpret_cast<const float*>(smem_raw) + I_::oK3;
    const float* k4 = reinterpret_cast<const float*>(smem_raw) + I_::oK4;
    float d4[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      float y0 = 0.f, y1 = 0.f, y2 = 0.f;
#pragma unroll
      for (int l = 0; l < 10; ++l) {
        y0 += k3[(0 * 4 + m) * 10 + l] * dl[l];
        y1 += k3[(1 * 4 + m) * 10 + l] * dl[l];
        y2 += k3[(2 * 4 + m) * 10 + l] * dl[l];
      }
      d4[m] = star_apply(st, y0, y1, y2);
      I[m] += L.tcf[NL + 1] * d4[m];
      if constexpr (kSpec) {
        const float gsum = elem_sum9(gv.w * d4[m], gv.base);
        if (gv.dst) gv.dst[gscr_off(N, NL + 1) + m] = gsum;
      }
    }
    float y0 = 0.f, y1 = 0.f, y2 = 0.f;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      y0 += k4[0 * 4 + l] * d4[l];
      y1 += k4[1 * 4 + l] * d4[l];
      y2 += k4[2 * 4 + l] * d4[l];
    }
    const float d5 = star_apply(st, y0, y1, y2);
    I[0] += L.tcf[NL + 2] * d5;
    if constexpr (kSpec) {
      const float gsum = elem_sum9(gv.w * d5, gv.base);
      if (gv.dst) gv.dst[gscr_off(N, NL + 2)] = gsum;
      // derivative traces of the last three levels (10, 4 and 1 rows) on the
      // faces with a finer neighbour, on the CUDA cores (E: hi + lo of the image)
      const float* img = reinterpret_cast<const float*>(smem_raw);
#pragma unroll 1
      for (int f = 0; f < 4; ++f) {
        if (!dtr[f]) continue;
#pragma unroll 1
        for (int n = 0; n < BF; ++n) {
          float t3 = 0.f, t4 = 0.f;
#pragma unroll
          for (int l = 0; l < 10; ++l) {
            const int o = tc::canon(f * BF + n, l, I_::NT);
            const float E = img[I_::oT + o] + img[I_::oT + I_::sT + o];
            t3 += E * dl[l];
            if (l < 4) t4 += E * d4[l];
          }
          const int o0 = tc::canon(f * BF + n, 0, I_::NT);
          dtr[f][NL * 9 * BF + n] = t3;
          dtr[f][(NL + 1) * 9 * BF + n] = t4;
          dtr[f][(NL + 2) * 9 * BF + n] = (img[I_::oT + o0] + img[I_::oT + I_::sT + o0]) * d5;
        }
      }
    }
  }

  // ---- face traces: T = I E^T (N = 4 x BF)
#pragma unroll
  for (int c = H; c < NCH; c += 2) tc::st_split8(trow + cAh + 8 * c, trow + cAl + 8 * c, I + 8 * c);
  if (!pair_round<H>(L, a.err, [&] {
        tc::mma3_ts<I_::NT, BP>(tbase + cAcc, tbase + cAh, tbase + cAl, sbase + 4 * I_::oT,
                                sbase + 4 * (I_::oT + I_::sT), false);
      }))
    return false;
  // traces leave face by face: the rows go to a shared buffer laid out like
  // the element's face block in memory, then one thread of the warp pair
  // copies each element's block with a bulk copy; two buffers alternate, the
  // copier waits until the copy before the last has read its buffer
  {
    constexpr int NTH = H == 0 ? (I_::NTCH + 1) / 2 : I_::NTCH / 2;  // this half's trace chunks
    const int nmine = nE - M::EW * L.w < M::EW ? nE - M::EW * L.w : M::EW;  // elements of this warp (may be <= 0)
    const bool copier = H == 0 && L.lane == 0;
    // this half's chunks c = H, H + 2, ... of the trace columns, read once
    float tv[48];
    if constexpr (N == 5) {
      tc::ld3x8(trow + cAcc + 8 * H, trow + cAcc + 8 * (H + 2), trow + cAcc + 8 * (H + 4), tv);
      tc::ld3x8(trow + cAcc + 8 * (H + 6), trow + cAcc + 8 * (H + 8), trow + cAcc + 8 * (H == 0 ? 10 : 9), tv + 24);
    } else {
      static_assert(N == 4 && I_::NTCH == 8, "trace chunks of degree 4");
      tc::ld3x8(trow + cAcc + 8 * H, trow + cAcc + 8 * (H + 2), trow + cAcc + 8 * (H + 4), tv);
      tc::ld8(trow + cAcc + 8 * (H + 6), tv + 24);
    }
    // an element with a coarser neighbour also adds its four face traces to
    // its LTS buffer, in FP64 (overwrite at the first of the two steps)
    if (kBuf && !M::fluid && L.btrace_mode && a.bslot && valid) {
      const int bs = a.bslot[e];
      if (bs >= 0) {
        double* bt = a.btrace + ((int64_t)bs * a.S + (v - e * a.S)) * 36 * BF;
#pragma unroll
        for (int cj = 0; cj < NTH; ++cj) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int col = 8 * (H + 2 * cj) + j;
            if (col < 4 * BF) {
              const int f = col / BF, n = col - f * BF;
              double* b = bt + (f * 9 + p) * BF + n;
              *b = (L.btrace_mode == 1 ? 0.0 : *b) + (double)tv[8 * cj + j];
            }
          }
        }
      }
    }
    if constexpr (M::fluid) {
      // acoustic: this face's (p, v) rows of the warp's eight elements in a
      // compact buffer [element][4][BF], then the warp pair writes each
      // element's full face block (sigma_xx three times, zero shear, v,
      // padding zeros) with 16-byte stores
      float* sC = s_T[L.slot][L.w];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
#pragma unroll
        for (int cj = 0; cj < NTH; ++cj) {
          const int c = H + 2 * cj;
          if (8 * c + 7 < BF * f || 8 * c >= BF * (f + 1)) continue;  // chunk outside face f
          if (valid) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int col = 8 * c + j;
              if (col >= BF * f && col < BF * (f + 1)) sC[(jj * 4 + p) * BF + col - BF * f] = tv[8 * cj + j];
            }
          }
        }
        warp_pair_bar(L.slot, L.w);
        for (int k = L.lane + 32 * H; k < nmine * (FS / 4); k += 64) {
          const int ej = k / (FS / 4), c4 = k - ej * (FS / 4);
          float x[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int idx = 4 * c4 + t, r = idx / BF, n = idx - BF * (idx / BF);
            x[t] = (idx >= 9 * BF || (r >= 3 && r < 6)) ? 0.f : sC[(ej * 4 + (r < 3 ? 0 : r - 5)) * BF + n];
          }
          reinterpret_cast<float4*>(reinterpret_cast<float*>(a.trace) +
                                    ((v0 + M::EW * L.w + ej) * 4 + f) * FS)[c4] = make_float4(x[0], x[1], x[2], x[3]);
        }
        warp_pair_bar(L.slot, L.w);  // the next face refills the buffer
      }
    } else {
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        float* sTf = s_T[L.slot][L.w] + (f & 1) * kTB;
#pragma unroll
        for (int cj = 0; cj < NTH; ++cj) {
          const int c = H + 2 * cj;
          if (8 * c + 7 < BF * f || 8 * c >= BF * (f + 1)) continue;  // chunk outside face f
          if (valid) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int col = 8 * c + j;
              if (col >= BF * f && col < BF * (f + 1)) sTf[jj * TS + p * BF + col - BF * f] = tv[8 * cj + j];
            }
          }
        }
        tc::fence_async_smem();
        if (copier) tc::bulk_wait_read();  // the other buffer is free for face f + 1
        warp_pair_bar(L.slot, L.w);
        if (copier) {
          for (int ej = 0; ej < nmine; ++ej)
            tc::bulk_store(reinterpret_cast<float*>(a.trace) + ((v0 + M::EW * L.w + ej) * 4 + f) * FS,
                           sTf + ej * TS, FS * 4);
          tc::bulk_commit();
        }
        if constexpr (kSpec) {
          // the own-trace part of the gravitational face's flux, sum_p Fg[q][p] V[p][n],
          // from this face's staged block, for the warp pair's elements whose gravitational face is f
          int gfe[M::EW], gse[M::EW];
#pragma unroll
          for (int ej = 0; ej < M::EW; ++ej) {
            gfe[ej] = __shfl_sync(0xffffffffu, gface, 9 * ej);
            gse[ej] = __shfl_sync(0xffffffffu, gsl, 9 * ej);
          }
          for (int k = L.lane + 32 * H; k < nmine * 9 * BF; k += 64) {
            const int ej = k / (9 * BF), r = k - ej * 9 * BF, q = r / BF, n = r - q * BF;
            int gf = -1, gs = -1;
#pragma unroll
            for (int jx = 0; jx < M::EW; ++jx)
              if (jx == ej) { gf = gfe[jx]; gs = gse[jx]; }
            if (gf != f || gs < 0) continue;
            const double* Fg = a.gpar + (int64_t)gs * GPAR + 6 + q * 9;
            float acc = 0.f;
#pragma unroll
            for (int pp = 0; pp < 9; ++pp) acc += (float)Fg[pp] * sTf[ej * TS + pp * BF + n];
            const int64_t ve = v0 + M::EW * L.w + ej;
            a.gscr[((int64_t)gs * a.S + (ve - (ve / a.S) * a.S)) * gscr_floats(N) + gscr_off(N, N + 1) + q * BF + n] =
                acc;
          }
        }
      }
    }
  }

  // ---- gravitational faces: the face's normal-projected derivative traces
  // f_m = E g_m, the (eta, H) ODE of Sec. 4.3 in FP64 over the step (its
  // Taylor series, as in the CUDA-core kernel) and the face's time-integrated
  // flux; one (element, node) per thread of the slot
  if constexpr (kSpec) {
    pair_bar(L.slot);  // the slot's scratch rows are written
    const int u = L.t + 128 * H;
    const int ei = u / BF, n = u - (u / BF) * BF;
    if (u < TE * BF && ei < nE && a.gslot) {
      const int64_t ve = v0 + ei, ee = ve / a.S;
      const int sc = (int)(ve - ee * a.S);
      int gf = -1, gs = -1;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const int x = a.gslot[ee * 4 + f];
        if (x >= 0) { gf = f; gs = x; }
      }
      if (gs >= 0) {
        const float* gsrc = a.gscr + ((int64_t)gs * a.S + sc) * gscr_floats(N);
        const float* img = reinterpret_cast<const float*>(smem_raw);
        double fm[N + 1];
#pragma unroll
        for (int m = 0; m <= N; ++m) {
          const int Bm = nb3(N - m);
          float acc = 0.f;
          for (int l = 0; l < Bm; ++l) {
            const int o = tc::canon(gf * BF + n, l, I_::NT);
            acc += (img[I_::oT + o] + img[I_::oT + I_::sT + o]) * gsrc[gscr_off(N, m) + l];
          }
          fm[m] = (double)acc * kRcpFact[m];
        }
        const double* gp = a.gpar + (int64_t)gs * GPAR;
        double* eta = a.eta + ((int64_t)gs * a.S + sc) * BF;
        const double kappa = gp[4], rg = gp[5], dt = L.dt;
        const double eta0 = eta[n];
        double c = eta0, e1 = eta0, Hint = eta0 * dt, pw = 1.0;
#pragma unroll 1
        for (int m = 0; m < N + 40; ++m) {
          double fv = 0.0;
#pragma unroll
          for (int k = 0; k <= N; ++k)
            if (k == m) fv = fm[k];
          c = (fv - kappa * c) * kRcp[m + 1];
          pw *= dt;
          const double term = c * pw;
          e1 += term;
          Hint += term * dt * kRcp[m + 2];
          if (m > N && fabs(term) <= 1e-17 * fabs(e1)) break;
        }
        eta[n] = e1;
        float* gfl = reinterpret_cast<float*>(a.gflux) + ((int64_t)gs * a.S + sc) * 9 * BF;
#pragma unroll
        for (int q = 0; q < 9; ++q)
          gfl[q * BF + n] = (float)(gp[87 + q] * (-rg * Hint) + gp[96 + q] * (e1 - eta0) +
                                    (double)gsrc[gscr_off(N, N + 1) + q * BF + n]);
      }
    }
  }

  // ---- volume: W_a = K_a I (l < B1) for the three axes in one product,
  // then Q += sum_a A*_a W_a = -sum_d c_d X_d[src_d] (Jacobian form)
  constexpr int KV = I_::KV;
#pragma unroll
  for (int c = H; c < KV / 8; c += 2) tc::st_split8(trow + 8 * c, trow + KV + 8 * c, I + 8 * c);
  // the dofs rows for the update are requested before the round (degree 5;
  // degree 4 updates its staged rows)
  float4 qv[8];
  if constexpr (I_::kAligned) {
#pragma unroll
    for (int c = H; c < NCH; c += 2) {
      qv[c - H] = make_float4(0.f, 0.f, 0.f, 0.f);
      qv[c - H + 1] = qv[c - H];
      if (valid) {
        qv[c - H] = reinterpret_cast<const float4*>(Qrow + 8 * c)[0];
        qv[c - H + 1] = reinterpret_cast<const float4*>(Qrow + 8 * c)[1];
      }
    }
  }
  constexpr uint32_t cV = 2 * KV;  // volume accumulator: axis a, basis m at column cV + BP a + m
  if (!pair_round<H>(L, a.err, [&] {
        tc::mma3_ts<I_::NV, KV>(tbase + cV, tbase + 0, tbase + KV, sbase + 4 * I_::oV,
                                sbase + 4 * (I_::oV + I_::sV), false);
      }))
    return false;
  // ---- Q += volume term (face terms follow in the neighbour kernel)
#pragma unroll
  for (int c = H; c < NCH; c += 2) {
    float y[24];
    tc::ld3x8(trow + cV + 8 * c, trow + cV + BP + 8 * c, trow + cV + 2 * BP + 8 * c, y);
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = -star_apply(st, y[j], y[8 + j], y[16 + j]);
    if constexpr (I_::kAligned) {
      if (valid) {
        const float4 q0 = qv[c - H], q1 = qv[c - H + 1];
        const float4 n0 = make_float4(q0.x + x[0], q0.y + x[1], q0.z + x[2], q0.w + x[3]);
        const float4 n1 = make_float4(q1.x + x[4], q1.y + x[5], q1.z + x[6], q1.w + x[7]);
        // (acoustic: the normal-stress row is written as sigma_xx, sigma_yy and sigma_zz)
#pragma unroll
        for (int r = 0; r < (M::fluid && p == 0 ? 3 : 1); ++r) {
          float4* dst = reinterpret_cast<float4*>(Qrow + r * B + 8 * c);
          dst[0] = n0;
          dst[1] = n1;
        }
      }
    } else {
      if (valid) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (8 * c + j < B) srow[8 * c + j] += x[j];
      }
    }
  }
  if constexpr (!I_::kAligned) {
    pair_bar(L.slot);
    rows_store<M, B>(sQ, Q, v0, nE, L.t + 128 * H);
  }
  // the next tile's first MMA overwrites these columns only after the
  // barrier at the start of its round
  tc::fence_before();
  return true;
}

// N: degree; M: the medium (Elastic or Acoustic); kChunk: consecutive tiles a
// slot takes per sweep (a compile-time launch shape)
template <int N, class M, bool kBuf, bool kMulti, int kChunk, bool kSpec = false>
__global__ void __launch_bounds__(kThreadsL, 1) local_tc_kernel(StepArgs a, const __grid_constant__ Segs g) {
  float* sm = reinterpret_cast<float*>(smem_raw);
  __shared__ uint32_t tmem_base;
  uint64_t* mbar = s_mbar;
  float (*sT)[4][2 * kTB] = s_T;

  __shared__ __align__(8) uint64_t s_img;  // completion of the operand image's bulk copies
  const int tid = threadIdx.x, slot = tid >> 8, half = (tid >> 7) & 1;
  // the operand image (the reference matrices' B operands) into shared memory
  // by the TMA engine, while the threads set up the rest
  if (tid == 0) {
    tc::mbar_init(&s_img, 1);
    tc::bulk_load_all(sm, a.tc_local, LImg<N>::floats * 4, &s_img);
  }
  for (int r = tid; r < 2 * 4 * 2 * kTB; r += kThreadsL) (&sT[0][0][0])[r] = 0.f;
  if (tid < 2) {
    tc::mbar_init(&mbar[tid], 1);
    s_abort[tid] = 0;
  }
  if (tid < 32) tc::tmem_alloc<512>(&tmem_base);
  __syncthreads();  // (the image barrier is initialised)
  const bool img_ok = tc::mbar_wait(&s_img, 0, kWaitIters);
  tc::fence_async_smem();
  tc::fence_before();
  const bool all_ok = __syncthreads_and(img_ok);
  tc::fence_after();
  if (!all_ok) {
    // the image did not arrive within the bound: report, give the copies a
    // bounded chance to finish, free the columns and leave
    if (tid == 0) {
      atomicOr(a.err, ERR_TIMEOUT);
      tc::mbar_wait(&s_img, 0, kWaitIters);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid < 32) tc::tmem_dealloc<512>(tmem_base);
    return;
  }

  Lane L;
  L.slot = slot;
  L.t = tid & 127;
  L.w = L.t >> 5;
  L.lane = tid & 31;
  L.tbase = tmem_base + (uint32_t)slot * 256u;
  L.trow = L.tbase + ((uint32_t)(32 * L.w) << 16);
  L.sbase = tc::smem_u32(sm);
  L.phase = 0;
  // tiles of all segments (the clusters of this phase) in one sequence; slot
  // `me` of all `slots` takes kChunk consecutive tiles per sweep
  const int64_t ntiles = g.first[g.n];
  const int slots = (int)gridDim.x * 2, me = (int)blockIdx.x * 2 + slot;
  auto work = [&](int64_t tile, int64_t t1, int64_t t2) {
    const Seg& sg = g.s[seg_of<kMulti>(g, tile)];
#pragma unroll
    for (int k = 0; k <= N; ++k) L.tcf[k] = (float)sg.tcoef[k];
    L.btrace_mode = sg.btrace_mode;
    L.dt = sg.dt;
    const int64_t lt = tile - g.first[&sg - g.s];
    const bool ok = half == 0 ? local_tile<N, M, 0, kBuf, kMulti, kSpec>(L, a, g, t1, t2, sg.v_begin, sg.n, lt)
                              : local_tile<N, M, 1, kBuf, kMulti, kSpec>(L, a, g, t1, t2, sg.v_begin, sg.n, lt);
    L.it++;
    return ok;
  };
  L.it = 0;
  if constexpr (kChunk == 1) {
    for (int64_t tile = me; tile < ntiles; tile += slots)
      if (!work(tile, tile + (int64_t)slots, tile + 2 * (int64_t)slots)) break;
  } else {
    for (int it = 0;; ++it) {
      const int64_t tile = slot_tile(it, me, slots, kChunk);
      if (tile >= ntiles ||
          !work(tile, slot_tile(it + 1, me, slots, kChunk), slot_tile(it + 2, me, slots, kChunk)))
        break;
    }
  }
  tc::cp_async_wait<0>();  // (degree 4) no copy into shared memory outlives the loop
  // after a timed-out wait, give this slot's MMAs in flight a bounded chance
  // to finish before the columns are freed
  if (half == 0 && L.t == 0 && s_abort[slot]) tc::mbar_wait(&mbar[slot], L.phase ^ 1u, kWaitIters);
  if (half == 0 && L.lane == 0) tc::bulk_wait();  // trace copies complete before shared memory is released
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (tid < 32) tc::tmem_dealloc<512>(tmem_base);
}

}  // namespace

// The launcher of degree N (the kernel table of that degree's translation unit).
template <int N>
int launch_local_tc_deg(const StepArgs& a, const Segs& g, int n_sms, void* stream, bool buffers, bool acoustic,
                        bool grav) {
  using K = void (*)(StepArgs, Segs);
  // elastic [kBuf][kMulti][chunk 1, 2, 4]; acoustic [kMulti][chunk] (its elements have no LTS buffer)
  static const K kern[2][2][3] = {
      {{local_tc_kernel<N, Elastic, false, false, 1>, local_tc_kernel<N, Elastic, false, false, 2>,
        local_tc_kernel<N, Elastic, false, false, 4>},
       {local_tc_kernel<N, Elastic, false, true, 1>, local_tc_kernel<N, Elastic, false, true, 2>,
        local_tc_kernel<N, Elastic, false, true, 4>}},
      {{local_tc_kernel<N, Elastic, true, false, 1>, local_tc_kernel<N, Elastic, true, false, 2>,
        local_tc_kernel<N, Elastic, true, false, 4>},
       {local_tc_kernel<N, Elastic, true, true, 1>, local_tc_kernel<N, Elastic, true, true, 2>,
        local_tc_kernel<N, Elastic, true, true, 4>}}};
  static const K kfl[2][3] = {
      {local_tc_kernel<N, Acoustic, false, false, 1>, local_tc_kernel<N, Acoustic, false, false, 2>,
       local_tc_kernel<N, Acoustic, false, false, 4>},
      {local_tc_kernel<N, Acoustic, false, true, 1>, local_tc_kernel<N, Acoustic, false, true, 2>,
       local_tc_kernel<N, Acoustic, false, true, 4>}};
  // elements with a gravitational face or a finer neighbour: [kMulti], one tile per sweep, LTS buffers allowed
  static const K kgr[2] = {local_tc_kernel<N, Elastic, true, false, 1, true>,
                           local_tc_kernel<N, Elastic, true, true, 1, true>};
  const int rc = configure_on_device((const void*)kern[0][0][0], [] {
    cudaError_t ce = cudaSuccess;
    for (int i = 0; i < 20; ++i) {
      const K k = i < 12 ? kern[i / 6][(i / 3) % 2][i % 3] : i < 18 ? kfl[(i - 12) / 3][(i - 12) % 3] : kgr[i - 18];
      if (ce == cudaSuccess)
        ce = cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, LImg<N>::bytes);
    }
    return ce;
  });
  if (rc) return rc;
  const int64_t ntiles = g.n ? g.first[g.n] : 0;
  if (ntiles <= 0) return 0;
  if (acoustic && (buffers || grav)) return (int)cudaErrorInvalidValue;
  const int ci = g.chunk >= 4 ? 2 : (g.chunk >= 2 ? 1 : 0);
  const int64_t want = (ntiles + 1) / 2;
  const unsigned grid = (unsigned)(want < n_sms ? want : n_sms);
  const K k = grav ? kgr[g.n > 1 ? 1 : 0]
                   : acoustic ? kfl[g.n > 1 ? 1 : 0][ci] : kern[buffers ? 1 : 0][g.n > 1 ? 1 : 0][ci];
  k<<<grid, kThreadsL, LImg<N>::bytes, (cudaStream_t)stream>>>(a, g);
  return (int)cudaGetLastError();
}

// Host-side image of the operands of degree N: kt[a][m][l], kvol[a][m][l]
// (l < B1) and efc[f][n][l] of that degree's basis, split into tf32 hi / lo
// and laid out as the canonical K-major B operands of local_tc_kernel.
template <int N>
void pack_local_tc_deg(const double* kt, const double* kvol, const double* efc, float* out) {
  using D = LDeg<N>;
  using I_ = LImg<N>;
  constexpr int B = I_::B, B1 = I_::B1, BF = I_::BF, BP = I_::BP;
  for (int i = 0; i < I_::floats; ++i) out[i] = 0.f;
  auto put = [&](int off, int size, int R, int n, int k, double x) {
    const float xf = (float)x;
    const float hi = tc::tf32_trunc(xf);
    const int o = tc::canon(n, k, R);
    out[off + o] = hi;
    out[off + size + o] = xf - hi;
  };
  const int offk[3] = {I_::oP0, I_::oP1, I_::oP2}, sizek[3] = {I_::sP0, I_::sP1, I_::sP2};
  for (int lev = 0; lev < D::NL; ++lev)
    for (int ax = 0; ax < 3; ++ax)
      for (int m = 0; m < D::M[lev]; ++m)
        for (int l = 0; l < D::KU[lev]; ++l)
          put(offk[lev], sizek[lev], D::NN[lev], ax * D::MP[lev] + m, l, kt[((size_t)ax * B + m) * B + l]);
  for (int ax = 0; ax < 3; ++ax)
    for (int m = 0; m < B; ++m)
      for (int l = 0; l < B1; ++l)
        put(I_::oV, I_::sV, I_::NV, ax * BP + m, l, kvol[((size_t)ax * B + m) * B1 + l]);
  for (int f = 0; f < 4; ++f)
    for (int n = 0; n < BF; ++n)
      for (int l = 0; l < B; ++l) put(I_::oT, I_::sT, I_::NT, f * BF + n, l, efc[((size_t)f * BF + n) * B + l]);
  for (int ax = 0; ax < 3; ++ax)
    for (int m = 0; m < 4; ++m)
      for (int l = 0; l < 10; ++l) out[I_::oK3 + (ax * 4 + m) * 10 + l] = (float)kt[((size_t)ax * B + m) * B + l];
  for (int ax = 0; ax < 3; ++ax)
    for (int l = 0; l < 4; ++l) out[I_::oK4 + ax * 4 + l] = (float)kt[((size_t)ax * B + 0) * B + l];
}

}  // namespace adg

// Neighbour kernel on the tensor cores (tcgen05, 3xTF32), degrees 5 and 4,
// FP32 dofs: face fluxes of Sec. 4.2 (Eq. numerical-flux) and their lift for
// elements whose faces are interior faces to the same or a coarser LTS
// cluster, periodic faces or linear boundaries (the others take the CUDA-core
// kernel); a coarser neighbour's face values are the integral of its Taylor
// expansion over this element's sub-interval (Sec. 4.4), formed while staging.
//
// Same tile as the local tensor-core kernel: 12 (virtual) elements x 9
// quantities = 128 TMEM lanes (warp w: elements 3w..3w+2, lane 9j+p = element
// 3w+j, quantity p; lanes 27..31 zero).  A CTA keeps two tiles in flight, each
// worked on by two warpgroups (256 threads).  Per tile and face f:
//   1. the own and the neighbours' time-integrated traces of face f are
//      copied asynchronously (cp.async, double-buffered over the faces) into
//      shared memory as they are stored, [element][quantity][node] (element
//      stride padded against bank conflicts);
//   2. work item (element, node), one per thread of the tile, forms the
//      scaled Godunov flux G[.][n] = s_f (F- V_own[.][n] + F+ V_nbr[.][perm n])
//      (s_f = 2|S_f|/|J|) in the face frame: both states rotated to (n, s, t),
//      the middle state of Eq. (boundary-state) (a linear boundary's ghost
//      folded into it), A- applied and the result rotated back, with the
//      face's coefficients formed once per tile from a 32-byte face record
//      and the element's material; it writes the 9 values to a transposition
//      buffer [element][p][28];
//   3. the thread of row (element, p) takes its CW columns (the face's nodes
//      padded to 8: 24 at degree 5, 16 at degree 4), splits them into tf32
//      hi + lo and writes them to TMEM columns CW f + n.
// One MMA chain then lifts all four faces:
//   Q[(element, p)][m] -= sum_{f,n} G[p][CW f + n] lift_f[m][n],
// A = G in TMEM (K = 4 CW), B = the lift matrices resident in shared memory.
// The next tile's face records, parameters and face 0 are requested before
// this tile's lift.  At degree 4 a dofs row (140 bytes) is not 16-byte
// aligned: the tile's rows are staged in shared memory with coalesced loads
// and written back the same way.
//
// This header holds the kernel for both degrees; neighbour_tc.cu and
// neighbour_tc4.cu instantiate it, one degree per translation unit.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "func_attr.hpp"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace adg {

namespace {

constexpr int TE = kTileElems;
constexpr int kThreadsN = 512;  // two tiles in flight, two warpgroups (halves) per tile
constexpr int kWaitIters = 1 << 24;
constexpr int kCoef = 32;       // per (face, element): frame n, s, t; middle-state and A- coefficients

// Shapes of degree N: CW TMEM columns per face (BF nodes, zero padded), the
// lift's N (the basis, padded to 16) and the transposed flux row kGrow
// (CW floats, padded so that the 8 rows of a quarter warp's 16-byte reads
// fall on distinct banks).
template <int N>
struct NDeg;
template <>
struct NDeg<5> {
  static constexpr int B = 56, BF = 21, CW = 24, kN = 64, kGrow = 28;
};
template <>
struct NDeg<4> {
  static constexpr int B = 35, BF = 15, CW = 16, kN = 48, kGrow = 20;
};

template <int N>
struct NImg : NDeg<N> {
  using D = NDeg<N>;
  static constexpr int B = D::B, BF = D::BF, CW = D::CW, kN = D::kN, kGrow = D::kGrow;
  static constexpr int kK = 4 * CW;               // lift: K = 4 faces x CW columns
  static constexpr int kFS = face_stride(N);      // floats per face block in the trace array
  static constexpr int kSS = kFS + 8;             // staged floats per element face: the 8 extra put the
                                                  // elements a warp's work items span on different banks
  static constexpr int kStage = TE * kSS;         // floats per staged face array
  static constexpr int kG = TE * 9 * kGrow;       // floats per transposition buffer
  static constexpr int kItems = TE * BF;          // work items per face: element x node
  static constexpr bool kAligned = B % 4 == 0;    // dofs rows 16-byte aligned (float4 access)
  static constexpr int oL = 0, sL = kN * kK;                  // lift hi, lo
  static constexpr int oPerm = oL + 2 * sL;                   // 6 x BF ints
  // per tile slot and tile parity: [face][element] int64 + int
  static constexpr int oMeta = oPerm + 128;
  static constexpr int sMeta = 4 * TE * 3;
  static constexpr int kBufs = 3;                             // staged faces: the one in use and two ahead
  static constexpr int oStage = oMeta + 2 * 2 * sMeta;        // per tile slot: kBufs buffers x (own, nbr)
  static constexpr int oRec = oStage + 2 * kBufs * 2 * kStage;  // per slot and tile parity: face records
  static constexpr int sRec = TE * 4 * FREC;                  // [element][face][FREC]
  static constexpr int oCoef = oRec + 2 * 2 * sRec;           // per slot and tile parity: [face][element][kCoef]
  static constexpr int sCoef = 4 * TE * kCoef;
  static constexpr int oPar = oCoef + 2 * 2 * sCoef;          // per slot and tile parity: element parameters
  static constexpr int sPar = TE * PAR;
  static constexpr int oG = oPar + 2 * 2 * sPar;              // per tile slot: transposition buffer
  static constexpr int oQ = oG + 2 * kG;                      // per tile slot (degree 4): the tile's dofs rows
  static constexpr int sQ = kAligned ? 0 : TE * 9 * B;
  static constexpr int floats = oQ + 2 * sQ;
  static constexpr int bytes = floats * 4;
  static_assert(kItems <= 256 && 6 * BF <= 128 && kK <= 96 && 2 * kK + kN <= 256, "shapes of one tile slot");
  static_assert(bytes + 64 <= 232448, "neighbour tensor-core kernel exceeds the shared memory of one CTA");
};

// per-slot TMEM columns: G hi [0, kK), G lo [kK, 2 kK), accumulator [2 kK, 2 kK + kN)

// the 256 threads (two warpgroups) of a tile slot
__device__ __forceinline__ void slot_bar(int slot) { asm volatile("bar.sync %0, 256;" ::"r"(slot + 1)); }

// asynchronous 16-byte copy global -> shared; zero fill when !valid
__device__ __forceinline__ void cp16(void* dst, const void* src, bool valid = true) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::smem_u32(dst)), "l"(src),
               "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;"); }
template <int NPEND>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(NPEND)); }

// Stage face f of a tile (thread u of the slot's 256): own traces and the
// neighbours' traces of that face, both as stored (one 16-byte aligned face
// block [quantity][node] per element); the neighbour's node order is applied
// when the values are read.  nbase: the neighbour's face block in the trace
// array (>= 0), none (-1), for a coarser neighbour -2 - the offset of its
// derivative traces [N+1][9][Bf], integrated here over this element's
// sub-interval with the coefficients cc (sum_k cc_k D_k, in the order of the
// CUDA-core kernel), for a finer neighbour kFineTag - the offset of its FP64
// LTS buffer [9][Bf] (the integral of its face traces over this element's
// step).  kCoarse: the launch has such faces (coarser or finer).
constexpr long long kFineTag = -(1LL << 50);
template <int N, bool kCoarse>
__device__ __forceinline__ void stage_face(int f, int u, int64_t v0, int nE, const float* trace,
                                           const long long* nbase, float* so, float* sn, const float* dtrace,
                                           const float* cc, const double* btrace) {
  using I_ = NImg<N>;
  constexpr int kFS = I_::kFS, kSS = I_::kSS, BF = I_::BF;
  constexpr int kChunks = kFS / 4;  // 16-byte chunks per face block
#pragma unroll
  for (int it = 0; it < (TE * kChunks + 255) / 256; ++it) {
    const int r = u + 256 * it;
    if (r < TE * kChunks) {
      const int ei = r / kChunks, ch = r - ei * kChunks;
      const bool ok = ei < nE;
      const long long nb = nbase[f * TE + ei];
      const bool okn = ok && nb >= 0;
      cp16(so + ei * kSS + 4 * ch, trace + ((v0 + (ok ? ei : 0)) * 4 + f) * kFS + 4 * ch, ok);
      if (kCoarse && ok && nb <= kFineTag) {
        const double* bt = btrace + (kFineTag - nb);
        float x[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int pos = 4 * ch + t;
          x[t] = pos < 9 * BF ? (float)bt[pos] : 0.f;
        }
        *reinterpret_cast<float4*>(sn + ei * kSS + 4 * ch) = make_float4(x[0], x[1], x[2], x[3]);
      } else if (kCoarse && ok && nb <= -2) {
        const float* dt = dtrace + (-2 - nb);
        float x[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int pos = 4 * ch + t;
          float acc = 0.f;
          if (pos < 9 * BF) {
#pragma unroll
            for (int k = 0; k <= N; ++k) acc += cc[k] * dt[k * 9 * BF + pos];
          }
          x[t] = acc;
        }
        *reinterpret_cast<float4*>(sn + ei * kSS + 4 * ch) = make_float4(x[0], x[1], x[2], x[3]);
      } else {
        cp16(sn + ei * kSS + 4 * ch, trace + (okn ? nb : 0) + 4 * ch, okn);
      }
    }
  }
}

// Coefficients of face f of the tile's element el (el < ne; others untouched)
// from its face record and parameters: the frame (n, s, t) with n the outward
// normal and s, t any orthonormal tangents (the flux does not depend on
// them); the middle state w^b = Mm w- + Mp w+ of the rotated states on the
// components the x-Jacobian reads (Sec. 4.2, Eq. boundary-state; normal pair
// (0, 6) with the P impedances, shear pairs (3, 7) and (5, 8) with the S
// impedances, welded when both sides are solid, else zero shear traction);
// for a linear boundary the ghost w+ = G w- (free surface: traction
// mirrored; rigid wall: normal velocity mirrored; absorbing: G = 0) is folded
// into Mm; and the x-Jacobian entries of the element's material times the
// face scale s_f = 2|S_f|/|J|.
__device__ __forceinline__ void face_coefficients(int f, int el, int ne, const float* sRec, const float* sPr,
                                                  float* sCo) {
  if (el >= ne) return;
  const float* rec = sRec + (el * 4 + f) * FREC;
  const float* pr = sPr + el * PAR;
  float* co = sCo + (f * TE + el) * kCoef;
  const float nx = rec[0], ny = rec[1], nz = rec[2];
  // tangent from the coordinate axis along which n is smallest
  const float ax = fabsf(nx), ay = fabsf(ny), az = fabsf(nz);
  const int k = (ay < ax) ? ((az < ay) ? 2 : 1) : ((az < ax) ? 2 : 0);
  const float dot = k == 0 ? nx : (k == 1 ? ny : nz);
  float sx = (k == 0 ? 1.f : 0.f) - dot * nx, sy = (k == 1 ? 1.f : 0.f) - dot * ny,
        sz = (k == 2 ? 1.f : 0.f) - dot * nz;
  const float is = rsqrtf(sx * sx + sy * sy + sz * sz);
  sx *= is; sy *= is; sz *= is;
  const float tx = ny * sz - nz * sy, ty = nz * sx - nx * sz, tz = nx * sy - ny * sx;
  const float rho = pr[9], lam = pr[10], mu = pr[11], sf = pr[12 + f];
  const float Zpm = sqrtf(rho * (lam + 2.f * mu)), Zsm = sqrtf(rho * mu);
  const int code = (int)rec[5];
  const float Zpp = code == FACE_NEIGHBOUR ? rec[3] : Zpm, Zsp = code == FACE_NEIGHBOUR ? rec[4] : Zsm;
  const float c = Zpm * Zpp / (Zpm + Zpp);
  float a00 = 1.f - c / Zpp, a06 = -c, b00 = c / Zpp, b06 = c;
  float a60 = -c / (Zpp * Zpm), a66 = 1.f - c / Zpm, b60 = c / (Zpp * Zpm), b66 = c / Zpm;
  float stt, stv, svt, svv, ttt, ttv, tvt, tvv;
  if (Zsm > 0.f && Zsp > 0.f) {
    const float cs = Zsm * Zsp / (Zsm + Zsp);
    stt = 1.f - cs / Zsp; stv = -cs; ttt = cs / Zsp; ttv = cs;
    svt = -cs / (Zsp * Zsm); svv = 1.f - cs / Zsm; tvt = cs / (Zsp * Zsm); tvv = cs / Zsm;
  } else {
    stt = stv = ttt = ttv = tvt = tvv = 0.f;
    svv = 1.f;
    svt = Zsm > 0.f ? -1.f / Zsm : 0.f;
  }
  if (code != FACE_NEIGHBOUR) {
    // ghost multipliers of the rotated components: traction (0), shear traction
    // (3, 5), normal velocity (6), tangential velocities (7, 8)
    const float G0 = code == FACE_FREE ? -1.f : (code == FACE_RIGID ? 1.f : 0.f);
    const float G3 = code == FACE_ABSORB ? 0.f : -1.f;
    const float G6 = code == FACE_FREE ? 1.f : (code == FACE_RIGID ? -1.f : 0.f);
    const float G7 = code == FACE_ABSORB ? 0.f : 1.f;
    a00 += b00 * G0; a06 += b06 * G6; a60 += b60 * G0; a66 += b66 * G6;
    stt += ttt * G3; stv += ttv * G7; svt += tvt * G3; svv += tvv * G7;
    b00 = b06 = b60 = b66 = ttt = ttv = tvt = tvv = 0.f;
  }
  const float v[29] = {nx, ny, nz, sx, sy, sz, tx, ty, tz, a00, a06, a60, a66, b00, b06, b60, b66,
                       stt, stv, svt, svv, ttt, ttv, tvt, tvv,
                       -(lam + 2.f * mu) * sf, -lam * sf, -mu * sf, -sf / rho};
#pragma unroll
  for (int i = 0; i < 29; ++i) co[i] = v[i];
  // a gravitational face lifts the flux the local kernel stored: its slot and s_f
  co[29] = code == FACE_GRAVITY ? rec[6] : __int_as_float(-1);
  co[30] = sf;
}

// Scaled Godunov flux of one face node: qm, qp the minus and plus traces
// (global frame, quantities sxx syy szz sxy syz sxz vx vy vz); g = s_f (F- qm +
// F+ qp) = s_f T A- (Mm T^-1 qm + Mp T^-1 qp).
__device__ __forceinline__ void face_flux(const float* cop, const float qm[9], const float qp[9], float g[9]) {
  // the 29 coefficients in eight 16-byte loads (a (face, element) record is 32 floats, 16-byte aligned)
  float co[32];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 x = reinterpret_cast<const float4*>(cop)[i];
    co[4 * i] = x.x; co[4 * i + 1] = x.y; co[4 * i + 2] = x.z; co[4 * i + 3] = x.w;
  }
  const float nx = co[0], ny = co[1], nz = co[2], sx = co[3], sy = co[4], sz = co[5], tx = co[6], ty = co[7],
              tz = co[8];
  float w[2][6];  // rotated components 0, 3, 5, 6, 7, 8 of each state
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const float* q = side == 0 ? qm : qp;
    const float snx = q[0] * nx + q[3] * ny + q[5] * nz;
    const float sny = q[3] * nx + q[1] * ny + q[4] * nz;
    const float snz = q[5] * nx + q[4] * ny + q[2] * nz;
    w[side][0] = nx * snx + ny * sny + nz * snz;
    w[side][1] = sx * snx + sy * sny + sz * snz;
    w[side][2] = tx * snx + ty * sny + tz * snz;
    w[side][3] = nx * q[6] + ny * q[7] + nz * q[8];
    w[side][4] = sx * q[6] + sy * q[7] + sz * q[8];
    w[side][5] = tx * q[6] + ty * q[7] + tz * q[8];
  }
  const float b0 = co[9] * w[0][0] + co[10] * w[0][3] + co[13] * w[1][0] + co[14] * w[1][3];
  const float b6 = co[11] * w[0][0] + co[12] * w[0][3] + co[15] * w[1][0] + co[16] * w[1][3];
  const float b3 = co[17] * w[0][1] + co[18] * w[0][4] + co[21] * w[1][1] + co[22] * w[1][4];
  const float b7 = co[19] * w[0][1] + co[20] * w[0][4] + co[23] * w[1][1] + co[24] * w[1][4];
  const float b5 = co[17] * w[0][2] + co[18] * w[0][5] + co[21] * w[1][2] + co[22] * w[1][5];
  const float b8 = co[19] * w[0][2] + co[20] * w[0][5] + co[23] * w[1][2] + co[24] * w[1][5];
  // x-Jacobian of the minus material (times s_f) on the middle state
  const float f0 = co[25] * b6, f1 = co[26] * b6, f3 = co[27] * b7, f5 = co[27] * b8;
  const float f6 = co[28] * b0, f7 = co[28] * b3, f8 = co[28] * b5;
  // back to the global frame: stress f1 I + n u^T + u n^T, velocity f6 n + f7 s + f8 t
  const float h = 0.5f * (f0 - f1);
  const float ux = h * nx + f3 * sx + f5 * tx, uy = h * ny + f3 * sy + f5 * ty, uz = h * nz + f3 * sz + f5 * tz;
  g[0] = f1 + 2.f * nx * ux;
  g[1] = f1 + 2.f * ny * uy;
  g[2] = f1 + 2.f * nz * uz;
  g[3] = nx * uy + ux * ny;
  g[4] = ny * uz + uy * nz;
  g[5] = nx * uz + ux * nz;
  g[6] = f6 * nx + f7 * sx + f8 * tx;
  g[7] = f6 * ny + f7 * sy + f8 * ty;
  g[8] = f6 * nz + f7 * sz + f8 * tz;
}

// kOne: one scenario (S = 1), where a virtual element is its element and the
// 64-bit divisions by S drop out; kCoarse: some faces of the launch have a
// coarser or finer LTS neighbour (without, their code stays out of the kernel)
// kChunk: consecutive tiles a slot takes per sweep (a compile-time launch shape)
template <int N, bool kOne, bool kCoarse, bool kMulti, int kChunk>
__global__ void __launch_bounds__(kThreadsN, 1) neighbour_tc_kernel(StepArgs a, const __grid_constant__ Segs g) {
  using NI = NImg<N>;
  constexpr int B = NI::B, BF = NI::BF, CW = NI::CW, kN = NI::kN, kK = NI::kK, kGrow = NI::kGrow;
  constexpr int kFS = NI::kFS, kSS = NI::kSS, kStage = NI::kStage, kG = NI::kG, kItems = NI::kItems;
  constexpr uint32_t cGh = 0, cGl = kK, cAcc = 2 * kK;
  constexpr int NCH = (B + 7) / 8;  // 8-column chunks of a dofs row
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  int* sPerm = reinterpret_cast<int*>(sm + NI::oPerm);
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ int s_abort[2];

  // slot: tile in flight; half: warpgroup within the slot; u: thread within the slot
  const int tid = threadIdx.x, slot = tid >> 8, half = (tid >> 7) & 1;
  const int u = tid & 255, t = tid & 127, w = t >> 5, lane = tid & 31;
  __shared__ __align__(8) uint64_t s_img;  // completion of the lift operand's bulk copies
  // the lift operand into shared memory by the TMA engine, while the threads set up the rest
  if (tid == 0) {
    tc::mbar_init(&s_img, 1);
    tc::bulk_load_all(sm + NI::oL, a.tc_lift, 2 * NI::sL * 4, &s_img);
  }
  for (int r = tid; r < 6 * BF; r += kThreadsN) sPerm[r] = a.perm[r];
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
    // the operand did not arrive within the bound: report, give the copies a
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

  const uint32_t tbase = tmem_base + (uint32_t)slot * 256u;
  const uint32_t trow = tbase + ((uint32_t)(32 * w) << 16);
  const uint32_t sL = tc::smem_u32(sm + NI::oL);
  // staged face g (counted over the slot's tiles, 4 per tile) in buffer g % 3:
  // own traces at 2 b, the neighbours' at 2 b + 1
  float* sStage = sm + NI::oStage + slot * NI::kBufs * 2 * kStage;
  auto stage_buf = [&](int gface) { return sStage + (gface % NI::kBufs) * 2 * kStage; };
  // per tile parity: the trace-block table and node permutations of a tile's
  // faces, its face records and element parameters
  auto sNb = [&](int par) { return reinterpret_cast<long long*>(sm + NI::oMeta + (slot * 2 + par) * NI::sMeta); };
  auto sPm = [&](int par) { return reinterpret_cast<int*>(sNb(par) + 4 * TE); };
  auto sRec = [&](int par) { return sm + NI::oRec + (slot * 2 + par) * NI::sRec; };  // [element - e0][face][FREC]
  auto sPr = [&](int par) { return sm + NI::oPar + (slot * 2 + par) * NI::sPar; };
  const float* trace = reinterpret_cast<const float*>(a.trace);
  auto sCo = [&](int par) { return sm + NI::oCoef + (slot * 2 + par) * NI::sCoef; };  // [face][element - e0][kCoef]
  // [element][p][28]; one buffer: face f + 1's items start after the barrier
  // that every thread reaches only when its rows of face f are done
  float* sG = sm + NI::oG + slot * kG;
  for (int r = u; r < kG; r += 256) sG[r] = 0.f;  // columns 21..27 stay zero
  const int jj = lane / 9, p = lane - 9 * (lane / 9);
  const int S = kOne ? 1 : a.S;
  const float* dtrace = reinterpret_cast<const float*>(a.dtrace);
  auto elem = [&](int64_t vv) -> int64_t { return kOne ? vv : vv / S; };  // element of a virtual element
  // tiles of all segments (the clusters of this phase) in one sequence: tile
  // tl starts at virtual element pv0 with prem virtual elements left in its
  // segment, whose coarser neighbours' expansion over this step's
  // sub-interval has the coefficients cc
  const int64_t ntiles = g.first[g.n];
  auto tile_at = [&](int64_t tl, int64_t& pv0, int64_t& prem, float* cc) {
    const Seg& sg = g.s[seg_of<kMulti>(g, tl)];
    const int64_t lt = tl - g.first[&sg - g.s];
    pv0 = sg.v_begin + lt * TE;
    prem = sg.n - lt * TE;
    if (cc) {
#pragma unroll
      for (int k = 0; k <= N; ++k) cc[k] = (float)sg.ccoef[k];
    }
  };
  uint32_t phase = 0;
  float bad = 0.f;  // stays 0 while every updated dof is finite (x * 0 is NaN for x = inf, NaN)

  // Neighbour trace blocks of a tile's faces, then one cp.async group per
  // thread with the tile's face records, element parameters and face 0, all
  // into the buffers of the tile's parity.  Thread u < 48 owns (face u / 12,
  // element u % 12) of a tile: its neighbour information, loaded early
  // (meta_load) and made the tile's trace-block table later (prefetch).
  auto meta_load = [&](int64_t tl, int& info, int& nbe) {
    info = 0;
    nbe = 0;
    int64_t pv0, prem;
    tile_at(tl, pv0, prem, nullptr);
    if (u < 4 * TE) {
      const int f = u / TE, ei = u - f * TE;
      if (ei < prem) {
        const int64_t ee = elem(pv0 + ei);
        info = a.ninfo[ee * 4 + f];
        nbe = a.nbr[ee * 4 + f];
      }
    }
  };
  auto prefetch = [&](int64_t tl, int par, int info, int nbe) {
    int64_t pv0, prem;
    float cc[N + 1];
    tile_at(tl, pv0, prem, kCoarse ? cc : nullptr);
    const int pnE = (int)(prem < TE ? prem : TE);
    if (u < 4 * TE) {
      const int ei = u - (u / TE) * TE;
      long long nb = -1;
      int pm = 0;
      const int kind = (info >> 5) & 7;
      if (ei < pnE && (kind == NK_SAME || (kCoarse && (kind == NK_COARSE || kind == NK_FINE)))) {
        const int64_t ve = pv0 + ei, ee = elem(ve);
        if (kind == NK_SAME) {
          const int64_t vn_e = (int64_t)nbe * S + (ve - ee * S);
          nb = (vn_e * 4 + (info & 3)) * kFS;
        } else if (kind == NK_COARSE) {
          const int ds = a.dslot[(int64_t)nbe * 4 + (info & 3)];
          nb = -2 - ((int64_t)ds * S + (ve - ee * S)) * (N + 1) * 9 * BF;
        } else {
          const int bs = a.bslot[nbe];
          nb = kFineTag - (((int64_t)bs * S + (ve - ee * S)) * 4 + (info & 3)) * 9 * BF;
        }
        pm = (info >> 2) & 7;
      }
      sNb(par)[u] = nb;
      sPm(par)[u] = pm;
    }
    slot_bar(slot);
    const int64_t e0 = elem(pv0);
    const int ne = (int)(elem(pv0 + pnE - 1) - e0 + 1);
    // face records of elements e0 .. e0 + ne - 1: ne x 128 bytes, 16-byte aligned
    for (int i4 = u; i4 < ne * FREC; i4 += 256) cp16(sRec(par) + 4 * i4, a.frec + e0 * 4 * FREC + 4 * i4);
    for (int c = u; c < ne * (PAR / 4); c += 256)
      cp16(sPr(par) + 4 * c, reinterpret_cast<const float*>(a.par) + e0 * PAR + 4 * c);
    // (committed with the tile's face 0)
  };
  // face f of the tile with slot counter itl: staged (one cp.async group) into buffer (4 itl + f) % 3
  auto stage = [&](int64_t tl, int itl, int f) {
    int64_t pv0, prem;
    float cc[N + 1];
    tile_at(tl, pv0, prem, kCoarse ? cc : nullptr);
    const int pnE = (int)(prem < TE ? prem : TE);
    float* buf = stage_buf(4 * itl + f);
    stage_face<N, kCoarse>(f, u, pv0, pnE, trace, sNb(itl & 1), buf, buf + kStage, dtrace, cc, a.btrace);
    cp_commit();
  };

  // Faces are staged two ahead of their use (three buffers): at face f of a
  // tile, face f + 2 of the same tile (f < 2) or face f - 2 of the next tile
  // (f >= 2; with face 0 come the next tile's records and parameters) is
  // requested, then the oldest group, face f, is waited for.  Every step
  // commits one group (an empty one past the last tile), so cp.async.wait_group 2
  // always leaves exactly the two younger faces in flight.
  const int slots = (int)gridDim.x * 2, me = (int)blockIdx.x * 2 + slot;
  int it = 0;
  int64_t tile = slot_tile(0, me, slots, kChunk);
  if (tile < ntiles) {
    int info0, nbe0;
    meta_load(tile, info0, nbe0);
    prefetch(tile, 0, info0, nbe0);
    stage(tile, 0, 0);
    stage(tile, 0, 1);
  }
  for (; tile < ntiles; tile = slot_tile(++it, me, slots, kChunk)) {
    const int64_t next = slot_tile(it + 1, me, slots, kChunk);
    const int par = it & 1;
    int info_n = 0, nbe_n = 0;  // the next tile's neighbour information, needed at face 2
    if (next < ntiles) meta_load(next, info_n, nbe_n);
    int64_t v0, nrem;
    float cc[N + 1];
    tile_at(tile, v0, nrem, kCoarse ? cc : nullptr);
    const int nE = (int)(nrem < TE ? nrem : TE);
    const int i = 3 * w + jj;
    const bool valid = lane < 27 && i < nE;
    const int64_t v = v0 + (valid ? i : 0);
    const int r0 = kOne ? 0 : (int)(v0 - elem(v0) * S);  // scenario of the tile's first virtual element
    const int ne = (int)(elem(v0 + nE - 1) - elem(v0) + 1);  // elements of the tile
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
      // ---- request the face two ahead, wait for face f
      if (f < 2) {
        stage(tile, it, f + 2);
      } else if (next < ntiles) {
        if (f == 2) prefetch(next, par ^ 1, info_n, nbe_n);
        stage(next, it + 1, f - 2);
      } else {
        cp_commit();
      }
      cp_wait<2>();
      if (f == 2) {  // the rows of faces 0 and 1 are in TMEM: their lift starts now
        asm volatile("tcgen05.wait::st.sync.aligned;");
        tc::fence_before();
      }
      slot_bar(slot);
      if (f == 2 && u == 0) {
        tc::fence_after();
        tc::mma3_ts<kN, 2 * CW>(tbase + cAcc, tbase + cGh, tbase + cGl, sL, sL + 4 * NI::sL, false);
      }
      if (f == 0 && it == 0) {  // the first tile's face coefficients (later tiles': during the lift before)
        if (u < 4 * TE) face_coefficients(u / TE, u % TE, ne, sRec(par), sPr(par), sCo(par));
        slot_bar(slot);
      }
      const float* sVo = stage_buf(4 * it + f);
      const float* sVn = sVo + kStage;
      // ---- work item (element, node) of thread u: scaled Godunov flux in the face frame
      if (u < kItems) {
        const int ei = u / BF, n = u - ei * BF;
        const int el = kOne ? ei : (r0 + ei) / S;  // element of item's virtual element, from the tile's first
        float* gout = sG + ei * 9 * kGrow + n;
        if (ei < nE) {
          const int pn = sPerm[sPm(par)[f * TE + ei] * BF + n];
          float qo[9], qn[9];
#pragma unroll
          for (int qq = 0; qq < 9; ++qq) {
            qo[qq] = sVo[ei * kSS + qq * BF + n];
            qn[qq] = sVn[ei * kSS + qq * BF + pn];
          }
          float g[9];
          const float* cof = sCo(par) + (f * TE + el) * kCoef;
          const int gs = __float_as_int(cof[29]);
          if (gs >= 0) {
            // gravitational face: s_f times the time-integrated flux of the local kernel
            const int sc = kOne ? 0 : (r0 + ei) % S;
            const float* src = reinterpret_cast<const float*>(a.gflux) + ((int64_t)gs * S + sc) * 9 * BF + n;
            const float sf = cof[30];
#pragma unroll
            for (int pp = 0; pp < 9; ++pp) g[pp] = sf * src[pp * BF];
          } else {
            face_flux(cof, qo, qn, g);
          }
#pragma unroll
          for (int pp = 0; pp < 9; ++pp) gout[pp * kGrow] = g[pp];
        } else {
#pragma unroll
          for (int pp = 0; pp < 9; ++pp) gout[pp * kGrow] = 0.f;
        }
      }
      slot_bar(slot);
      // ---- this row's CW columns of face f -> TMEM (hi, lo): 8-column chunk c
      // by the half (c + f) % 2
      {
        const float4* g4 = reinterpret_cast<const float4*>(sG + ((i < TE ? i : 0) * 9 + p) * kGrow);
#pragma unroll
        for (int c = 0; c < CW / 8; ++c) {
          if (((c + f) & 1) != half) continue;
          const float4 x0 = g4[2 * c], x1 = g4[2 * c + 1];
          float g[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
          if (!valid) {
#pragma unroll
            for (int jn = 0; jn < 8; ++jn) g[jn] = 0.f;
          }
          tc::st_split8(trow + cGh + CW * f + 8 * c, trow + cGl + CW * f + 8 * c, g);
        }
      }
    }
    // this half's chunks (c % 2 == half) of the dofs row (in L2 from the
    // prefetch two tiles back), loaded while the next tile's copies are issued
    // and the lift runs; degree 4: the tile's rows, staged in shared memory by
    // the slot's 256 threads with coalesced loads
    float* Qrow = reinterpret_cast<float*>(a.Q) + (v * 9 + p) * B;
    float q[32];
    float* sQ = sm + NI::oQ + slot * NI::sQ;
    if constexpr (NI::kAligned) {
#pragma unroll
      for (int cj = 0; cj < 4; ++cj) {
        const int c = half + 2 * cj;
        float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f), x1 = x0;
        if (c < B / 8 && valid) {
          x0 = reinterpret_cast<const float4*>(Qrow + 8 * c)[0];
          x1 = reinterpret_cast<const float4*>(Qrow + 8 * c)[1];
        }
        q[8 * cj] = x0.x; q[8 * cj + 1] = x0.y; q[8 * cj + 2] = x0.z; q[8 * cj + 3] = x0.w;
        q[8 * cj + 4] = x1.x; q[8 * cj + 5] = x1.y; q[8 * cj + 6] = x1.z; q[8 * cj + 7] = x1.w;
      }
    } else {
      // (one cp.async group, the youngest: waited for before the update)
      const float* Qt = reinterpret_cast<const float*>(a.Q) + v0 * 9 * B;
      for (int r = u; r < nE * 9 * B; r += 256) tc::cp_async4(sQ + r, Qt + r);
      cp_commit();
    }
    // ---- the tile after the next into L2
    const int64_t next2 = slot_tile(it + 2, me, slots, kChunk);
    if (u == 0 && next2 < ntiles) {
      int64_t q0, rem2;
      tile_at(next2, q0, rem2, nullptr);
      const uint32_t n2 = (uint32_t)(rem2 < TE ? rem2 : TE);
      tc::prefetch_l2_inner(reinterpret_cast<const float*>(a.Q) + q0 * 9 * B, n2 * 9 * B * 4);
      tc::prefetch_l2(trace + q0 * 4 * kFS, n2 * 4 * kFS * 4);
      const int64_t e0 = elem(q0), ne = elem(q0 + n2 - 1) - e0 + 1;
      tc::prefetch_l2(a.frec + e0 * 4 * FREC, (uint32_t)(ne * 4 * FREC * 4));
    }
    // ---- lift of faces 2 and 3 on the tensor cores (faces 0 and 1 were issued above);
    // meanwhile threads 64..111 form the next tile's face coefficients (its
    // records and parameters came with its face 0, the older of the two groups
    // in flight)
    if (next < ntiles) {
      if constexpr (NI::kAligned)
        cp_wait<1>();
      else
        cp_wait<2>();  // the staged dofs rows are younger
    }
    asm volatile("tcgen05.wait::st.sync.aligned;");
    tc::fence_before();
    slot_bar(slot);
    tc::fence_after();
    if (next < ntiles && u >= 64 && u < 64 + 4 * TE) {
      int64_t pv0, prem;
      tile_at(next, pv0, prem, nullptr);
      const int pnE = (int)(prem < TE ? prem : TE);
      const int ne_n = (int)(elem(pv0 + pnE - 1) - elem(pv0) + 1);
      face_coefficients((u - 64) / TE, (u - 64) % TE, ne_n, sRec(par ^ 1), sPr(par ^ 1), sCo(par ^ 1));
    }
    if (u == 0) {
      tc::mma3_ts<kN, kK, 2 * CW>(tbase + cAcc, tbase + cGh, tbase + cGl, sL, sL + 4 * NI::sL, true);
      tc::commit(&mbar[slot]);
      if (!tc::mbar_wait(&mbar[slot], phase, kWaitIters)) {
        atomicOr(a.err, ERR_TIMEOUT);
        s_abort[slot] = 1;
      }
    }
    if constexpr (!NI::kAligned) cp_wait<0>();  // the tile's staged dofs rows
    slot_bar(slot);
    if (s_abort[slot]) break;
    tc::mbar_wait(&mbar[slot], phase, 1 << 20);
    phase ^= 1u;
    tc::fence_after();
    // ---- Q -= lift, this half's chunks
    {
      float x[32];
      tc::ld3x8(trow + cAcc + 8 * half, trow + cAcc + 8 * (half + 2), trow + cAcc + 8 * (half + 4), x);
      if constexpr (NCH > 6) {
        if (half == 0) tc::ld8(trow + cAcc + 48, x + 24);
      }
      if constexpr (NI::kAligned) {
#pragma unroll
        for (int cj = 0; cj < 4; ++cj) {
          const int c = half + 2 * cj;
          if (c < B / 8 && valid) {
            float nq[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              nq[j] = q[8 * cj + j] - x[8 * cj + j];
              bad = fmaf(nq[j], 0.f, bad);
            }
            float4* dst = reinterpret_cast<float4*>(Qrow + 8 * c);
            dst[0] = make_float4(nq[0], nq[1], nq[2], nq[3]);
            dst[1] = make_float4(nq[4], nq[5], nq[6], nq[7]);
          }
        }
      } else {
        static_assert(NCH <= 6, "three chunks per half");
        float* srow = sQ + (i * 9 + p) * B;
#pragma unroll
        for (int cj = 0; cj < 3; ++cj) {
          const int c = half + 2 * cj;
          if (c < NCH && valid) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              if (8 * c + j < B) {
                const float nq = srow[8 * c + j] - x[8 * cj + j];
                bad = fmaf(nq, 0.f, bad);
                srow[8 * c + j] = nq;
              }
            }
          }
        }
        slot_bar(slot);
        float* Qt = reinterpret_cast<float*>(a.Q) + v0 * 9 * B;
        for (int r = u; r < nE * 9 * B; r += 256) Qt[r] = sQ[r];
      }
    }
    tc::fence_before();
  }
  if (__any_sync(0xffffffffu, bad != 0.f) && lane == 0) atomicOr(a.err, ERR_NAN);
  cp_wait<0>();  // no copy into shared memory outlives the loop (an aborted slot may leave some)
  if (u == 0 && s_abort[slot]) tc::mbar_wait(&mbar[slot], phase ^ 1u, kWaitIters);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (tid < 32) tc::tmem_dealloc<512>(tmem_base);
}

}  // namespace

// The launcher of degree N (the kernel table of that degree's translation unit).
template <int N>
int launch_neighbour_tc_deg(const StepArgs& a, const Segs& g, int n_sms, void* stream, bool coarse) {
  using K = void (*)(StepArgs, Segs);
#define ADG_NK(one, coarse, multi) \
  { neighbour_tc_kernel<N, one, coarse, multi, 1>, neighbour_tc_kernel<N, one, coarse, multi, 2>, \
    neighbour_tc_kernel<N, one, coarse, multi, 4> }
  // [S == 1][coarse][multi][chunk 1, 2, 4]
  static const K kern[2][2][2][3] = {{{ADG_NK(false, false, false), ADG_NK(false, false, true)},
                                      {ADG_NK(false, true, false), ADG_NK(false, true, true)}},
                                     {{ADG_NK(true, false, false), ADG_NK(true, false, true)},
                                      {ADG_NK(true, true, false), ADG_NK(true, true, true)}}};
#undef ADG_NK
  const int rc = configure_on_device((const void*)kern[0][0][0][0], [] {
    cudaError_t ce = cudaSuccess;
    for (int i = 0; i < 24; ++i)
      if (ce == cudaSuccess)
        ce = cudaFuncSetAttribute((const void*)kern[i / 12][(i / 6) % 2][(i / 3) % 2][i % 3],
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, NImg<N>::bytes);
    return ce;
  });
  if (rc) return rc;
  const int64_t ntiles = g.n ? g.first[g.n] : 0;
  if (ntiles <= 0) return 0;
  const int ci = g.chunk >= 4 ? 2 : (g.chunk >= 2 ? 1 : 0);
  const int64_t want = (ntiles + 1) / 2;
  const unsigned grid = (unsigned)(want < n_sms ? want : n_sms);
  kern[a.S == 1 ? 1 : 0][coarse ? 1 : 0][g.n > 1 ? 1 : 0][ci]<<<grid, kThreadsN, NImg<N>::bytes,
                                                               (cudaStream_t)stream>>>(a, g);
  return (int)cudaGetLastError();
}

// Host-side B operand of the lift of degree N: lift[f][m][n] of that
// degree's basis at row m, column CW f + n, split into tf32 hi / lo,
// canonical K-major layout.
template <int N>
void pack_lift_tc_deg(const double* lift, float* out) {
  using NI = NImg<N>;
  constexpr int B = NI::B, BF = NI::BF;
  for (int i = 0; i < 2 * NI::sL; ++i) out[i] = 0.f;
  for (int f = 0; f < 4; ++f)
    for (int m = 0; m < B; ++m)
      for (int n = 0; n < BF; ++n) {
        const float xf = (float)lift[((size_t)f * B + m) * BF + n];
        const float hi = tc::tf32_trunc(xf);
        const int o = tc::canon(m, NI::CW * f + n, NI::kN);
        out[o] = hi;
        out[NI::sL + o] = xf - hi;
      }
}

}  // namespace adg

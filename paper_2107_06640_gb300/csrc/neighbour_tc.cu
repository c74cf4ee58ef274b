// Neighbour-flux kernel with the lift on the tensor cores (tcgen05, 3xTF32),
// degree 5, FP32 dofs.
//
// Per tile of TE = 8 elements (persistent CTAs):
//   1. gather, on CUDA cores: own time-integrated traces, the neighbours'
//      traces through the node permutation (or the coarser neighbour's Taylor
//      integral / the finer neighbour's FP64 buffer under LTS), F- and F+;
//   2. face fluxes G_f = F-_f V_own + F+_f V_nbr (gravity and fault faces:
//      the stored fluxes), scaled by 2|S_f|/|J|, split into tf32 hi + lo and
//      written as the B operand (72 columns = element x quantity, K = 84 face
//      nodes x faces, padded to 88);
//   3. one thread issues 11 K-steps x 3 MMAs (A_hi B_hi + A_hi B_lo +
//      A_lo B_hi; A = the stacked lift matrix, 56 x 84 padded to 64 x 88,
//      resident in shared memory) into a 64 x 72 fp32 accumulator in TMEM and
//      commits to an mbarrier;
//   4. after a bounded wait, the accumulator is read with tcgen05.ld and
//      subtracted from Q (the semi-discrete face term of Sec. 4.1).
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"
#include "tc_common.cuh"

namespace adg {

namespace {

constexpr int N5 = 5, B5 = 56, BF5 = 21;
constexpr int TE = 8;             // elements per tile
constexpr int NC = 9 * TE;        // accumulator columns
constexpr int MR = 64;            // accumulator rows (56 used)
constexpr int KL = 88;            // reduction length (84 used)
constexpr int TV = 36 * BF5;      // trace floats per element (756)
constexpr int kThreadsTC = 256;
constexpr int kTmemCols = 128;
constexpr int kWaitIters = 1 << 24;

struct SmemTC {
  static constexpr int oAh = 0, oAl = oAh + MR * KL, oBh = oAl + MR * KL, oBl = oBh + NC * KL,
                       oVo = oBl + NC * KL, oVn = oVo + TE * TV, oF = oVn + TE * TV, oSc = oF + TE * 648,
                       oEnd = oSc + TE * 4;
  static constexpr int bytes = oEnd * 4 + TE * 4 * 4 * 2 + 64;
};

__global__ void __launch_bounds__(kThreadsTC, 1) neighbour_tc_kernel(StepArgs a, int64_t n_virtual) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  float* sAh = sm + SmemTC::oAh;
  float* sAl = sm + SmemTC::oAl;
  float* sBh = sm + SmemTC::oBh;
  float* sBl = sm + SmemTC::oBl;
  float* sVo = sm + SmemTC::oVo;
  float* sVn = sm + SmemTC::oVn;
  float* sF = sm + SmemTC::oF;
  float* sSc = sm + SmemTC::oSc;
  int* sKind = reinterpret_cast<int*>(sm + SmemTC::oEnd);
  int* sGrav = sKind + TE * 4;
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int s_abort;

  const int tid = threadIdx.x, nth = blockDim.x, warp = tid >> 5, lane = tid & 31;
  const float* Aglob = a.tc_lift;
  for (int r = tid; r < 2 * MR * KL; r += nth) sAh[r] = Aglob[r];  // hi then lo, canonical layout
  for (int r = tid; r < NC * 4; r += nth) {                        // zero the K padding 84..87
    const int row = r / 4, k = 84 + r % 4;
    sBh[tc::canon(row, k, NC)] = 0.f;
    sBl[tc::canon(row, k, NC)] = 0.f;
  }
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    s_abort = 0;
  }
  if (warp == 0) tc::tmem_alloc<kTmemCols>(&tmem_base);
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = tc::idesc_tf32(MR, NC);
  const int64_t ntiles = (n_virtual + TE - 1) / TE;
  uint32_t phase = 0;
  bool bad = false;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t v0 = a.v_begin + tile * TE;
    const int nE = (int)((n_virtual - tile * TE) < TE ? (n_virtual - tile * TE) : TE);
    // ---- 1. per-element metadata, matrices and own traces
    if (tid < TE * 4) {
      const int i = tid / 4, f = tid % 4;
      if (i < nE) {
        const int64_t e = (v0 + i) / a.S;
        sSc[tid] = reinterpret_cast<const float*>(a.par)[e * PAR + 12 + f];
        sKind[tid] = (a.ninfo[e * 4 + f] >> 5) & 7;
        sGrav[tid] = a.gslot ? a.gslot[e * 4 + f] : -1;
      } else {
        sSc[tid] = 0.f;
        sKind[tid] = NK_NONE;
        sGrav[tid] = -1;
      }
    }
    for (int r = tid; r < TE * 648; r += nth) {
      const int i = r / 648, k = r % 648;
      float val = 0.f;
      if (i < nE) {
        const int64_t e = (v0 + i) / a.S;
        val = k < 324 ? reinterpret_cast<const float*>(a.Fm)[e * 324 + k]
                      : reinterpret_cast<const float*>(a.Fp)[e * 324 + k - 324];
      }
      sF[r] = val;
    }
    for (int r = tid; r < TE * TV; r += nth) {
      const int i = r / TV;
      sVo[r] = i < nE ? reinterpret_cast<const float*>(a.trace)[v0 * TV + r] : 0.f;
    }
    __syncthreads();
    // neighbours' traces in this face's node order
    for (int r = tid; r < TE * TV; r += nth) {
      const int i = r / TV, rr = r % TV;
      const int f = rr / (9 * BF5), p = (rr / BF5) % 9, n = rr % BF5;
      const int kind = sKind[i * 4 + f];
      float val = 0.f;
      if (kind == NK_SAME || kind == NK_FINE || kind == NK_COARSE) {
        const int64_t v = v0 + i;
        const int64_t e = v / a.S;
        const int s = (int)(v - e * a.S);
        const int info = a.ninfo[e * 4 + f];
        const int64_t nb = a.nbr[e * 4 + f];
        const int j = info & 3, pm = (info >> 2) & 7;
        const int src = a.perm[pm * BF5 + n];
        if (kind == NK_SAME) {
          val = reinterpret_cast<const float*>(a.trace)[((nb * a.S + s) * 4 + j) * 9 * BF5 + p * BF5 + src];
        } else if (kind == NK_FINE) {
          val = (float)a.btrace[(((int64_t)a.bslot[nb] * a.S + s) * 4 + j) * 9 * BF5 + p * BF5 + src];
        } else {
          const float* dt = reinterpret_cast<const float*>(a.dtrace) +
                            ((int64_t)a.dslot[nb * 4 + j] * a.S + s) * (N5 + 1) * 9 * BF5;
          float acc = 0.f;
#pragma unroll
          for (int k = 0; k <= N5; ++k) acc += (float)a.ccoef[k] * dt[(k * 9 + p) * BF5 + src];
          val = acc;
        }
      }
      sVn[r] = val;
    }
    __syncthreads();
    // ---- 2. scaled face fluxes -> B operand (column = element*9 + q, K = face*21 + node)
    for (int r = tid; r < TE * TV; r += nth) {
      const int i = r / TV, rr = r % TV;
      const int f = rr / (9 * BF5), q = (rr / BF5) % 9, n = rr % BF5;
      float g = 0.f;
      if (i < nE) {
        const int kind = sKind[i * 4 + f];
        if (kind == NK_FAULT) {
          const int64_t v = v0 + i;
          const int64_t e = v / a.S;
          const int s = (int)(v - e * a.S);
          const int fsl = a.fslot[e * 4 + f];
          g = reinterpret_cast<const float*>(a.drout)[((((int64_t)(fsl >> 1) * a.S + s) * 2 + (fsl & 1)) * 9 + q) * BF5 + n];
        } else if (sGrav[i * 4 + f] >= 0) {
          const int64_t v = v0 + i;
          const int64_t e = v / a.S;
          const int s = (int)(v - e * a.S);
          g = reinterpret_cast<const float*>(a.gflux)[((int64_t)sGrav[i * 4 + f] * a.S + s) * 9 * BF5 + q * BF5 + n];
        } else {
          const float* Fm = sF + i * 648 + f * 81 + q * 9;
          const float* Vo = sVo + i * TV + f * 9 * BF5 + n;
#pragma unroll
          for (int p = 0; p < 9; ++p) g += Fm[p] * Vo[p * BF5];
          if (kind != NK_NONE) {
            const float* Fp = sF + i * 648 + 324 + f * 81 + q * 9;
            const float* Vn = sVn + i * TV + f * 9 * BF5 + n;
#pragma unroll
            for (int p = 0; p < 9; ++p) g += Fp[p] * Vn[p * BF5];
          }
        }
        g *= sSc[i * 4 + f];
      }
      const float hi = tc::tf32_trunc(g);
      const int off = tc::canon(i * 9 + q, f * BF5 + n, NC);
      sBh[off] = hi;
      sBl[off] = g - hi;
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    // ---- 3. lift on the tensor cores
    if (tid == 0) {
      const uint32_t aH = tc::smem_u32(sAh), aL = tc::smem_u32(sAl), bH = tc::smem_u32(sBh), bL = tc::smem_u32(sBl);
      constexpr uint32_t lboA = (MR / 8) * 128, lboB = (NC / 8) * 128;
#pragma unroll 1
      for (int kk = 0; kk < KL / 8; ++kk) {
        const uint32_t oa = kk * 2 * lboA, ob = kk * 2 * lboB;
        const uint64_t dAh = tc::sdesc(aH + oa, lboA, 128), dAl = tc::sdesc(aL + oa, lboA, 128);
        const uint64_t dBh = tc::sdesc(bH + ob, lboB, 128), dBl = tc::sdesc(bL + ob, lboB, 128);
        tc::mma_tf32(tmem, dAh, dBh, idesc, kk > 0 ? 1u : 0u);
        tc::mma_tf32(tmem, dAh, dBl, idesc, 1u);
        tc::mma_tf32(tmem, dAl, dBh, idesc, 1u);
      }
      tc::commit(&mbar);
    }
    // ---- 4. wait, read the accumulator, Q -= lift
    if (!tc::mbar_wait(&mbar, phase, kWaitIters)) {
      if (lane == 0) atomicOr(a.err, ERR_TIMEOUT);
      s_abort = 1;
    }
    phase ^= 1u;
    tc::fence_after();
    __syncthreads();
    if (s_abort) break;
    {
      const int quarter = warp & 3;
      const int m = quarter * 16 + lane;  // accumulator row held by this lane
      const int c_begin = warp < 4 ? 0 : 5, c_end = warp < 4 ? 5 : NC / 8;
      for (int c = c_begin; c < c_end; ++c) {
        float vals[8];
        tc::tmem_ld8(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(c * 8), vals);
        if (lane < 16 && m < B5) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int col = c * 8 + j, i = col / 9, q = col % 9;
            if (i < nE) {
              float* Q = reinterpret_cast<float*>(a.Q) + ((v0 + i) * 9 + q) * B5 + m;
              const float nq = *Q - vals[j];
              *Q = nq;
              bad |= !isfinite(nq);
            }
          }
        }
      }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.err, ERR_NAN);
  __syncthreads();
  if (s_abort) {
    // give the in-flight MMAs a bounded chance to finish before freeing TMEM
    tc::mbar_wait(&mbar, phase ^ 1u, kWaitIters);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc<kTmemCols>(tmem);
}

}  // namespace

int neighbour_tc_smem_bytes() { return SmemTC::bytes; }

int launch_neighbour_tc(const StepArgs& a, int64_t n_virtual, int n_sms, void* stream) {
  static bool configured = false;
  if (!configured) {
    cudaError_t ce =
        cudaFuncSetAttribute(neighbour_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SmemTC::bytes);
    if (ce != cudaSuccess) return (int)ce;
    configured = true;
  }
  if (n_virtual <= 0) return 0;
  const int64_t ntiles = (n_virtual + TE - 1) / TE;
  const unsigned grid = (unsigned)(ntiles < n_sms ? ntiles : n_sms);
  neighbour_tc_kernel<<<grid, kThreadsTC, SmemTC::bytes, (cudaStream_t)stream>>>(a, n_virtual);
  return (int)cudaGetLastError();
}

// Host-side operand: the stacked lift matrix (rows m < 56, K = face*21 + node),
// split into tf32 hi / lo, in the canonical K-major layout; 2 * 64 * 88 floats.
void pack_lift_tc(const double* lift /* [4][B][Bf] */, float* out) {
  for (int i = 0; i < 2 * MR * KL; ++i) out[i] = 0.f;
  for (int m = 0; m < B5; ++m)
    for (int f = 0; f < 4; ++f)
      for (int n = 0; n < BF5; ++n) {
        const double x = lift[((size_t)f * B5 + m) * BF5 + n];
        const float hi = tc::tf32_trunc((float)x);
        const float lo = (float)(x - (double)hi);
        const int off = tc::canon(m, f * BF5 + n, MR);
        out[off] = hi;
        out[MR * KL + off] = lo;
      }
}

}  // namespace adg

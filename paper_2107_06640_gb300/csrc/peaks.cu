// Peak-rate probes of this GPU, for the roofline denominators of the kernels
// that are not plain copies or BF16 GEMMs:
//   kind 0: tcgen05.mma kind::tf32 (A in TMEM, B in shared memory, FP32
//           accumulation), M = 128, N = 256, K = 8 per instruction, one CTA
//           per SM, one issuing thread; the rate of every 3xTF32 split
//           product is a third of it;
//   kind 1: FP32 fused multiply-add on the CUDA cores;
//   kind 2: FP64 fused multiply-add.
// Each returns the floating-point operations it performed and its duration
// (CUDA events around the launches, after one untimed launch).
#include <cuda_runtime.h>

#include <cstdint>

#include "adg_internal.hpp"
#include "func_attr.hpp"
#include "tc_common.cuh"

namespace {

constexpr int kMmaN = 256, kMmaK = 32;  // B operand N x K (canonical K-major), four K-steps of 8
constexpr int kBatch = 64;              // MMAs between commits
constexpr int kWaitIters = 1 << 24;

__global__ void __launch_bounds__(128, 1) mma_tf32_loop(int batches, unsigned int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* sB = reinterpret_cast<float*>(smem_raw);
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t mbar[2];
  const int t = threadIdx.x;
  for (int i = t; i < kMmaN * kMmaK; i += 128) sB[i] = adg::tc::tf32_trunc(1.0f + 1e-3f * (float)(i % 97));
  if (t == 0) {
    adg::tc::mbar_init(&mbar[0], 1);
    adg::tc::mbar_init(&mbar[1], 1);
  }
  if (t < 32) adg::tc::tmem_alloc<512>(&tmem_base);
  adg::tc::fence_async_smem();
  adg::tc::fence_before();
  __syncthreads();
  adg::tc::fence_after();
  const uint32_t tb = tmem_base;
  // A: row t, K = 32 values at columns [0, 32)
  {
    float x[8];
    for (int c = 0; c < kMmaK / 8; ++c) {
      for (int j = 0; j < 8; ++j) x[j] = adg::tc::tf32_trunc(1e-2f * (float)((t + 8 * c + j) % 13));
      adg::tc::st_split8(tb + ((uint32_t)(32 * (t >> 5)) << 16) + 8 * c,
                         tb + ((uint32_t)(32 * (t >> 5)) << 16) + 64 + 8 * c, x);
    }
  }
  asm volatile("tcgen05.wait::st.sync.aligned;");
  adg::tc::fence_before();
  __syncthreads();
  adg::tc::fence_after();
  if (t == 0) {
    constexpr uint32_t idesc = adg::tc::idesc_tf32(128, kMmaN);
    constexpr uint32_t lbo = (kMmaN / 8) * 128;
    const uint64_t d0 = adg::tc::sdesc(adg::tc::smem_u32(sB), lbo, 128);
    uint32_t ph[2] = {0, 0};
    for (int b = 0; b < batches; ++b) {
      for (int i = 0; i < kBatch; ++i) {
        const int kk = i & 3;
        adg::tc::mma_ts(tb + 256, tb + 8 * kk, d0 + (uint64_t)((kk * 2 * lbo) >> 4), idesc,
                        (b > 0 || i > 0) ? 1u : 0u);
      }
      adg::tc::commit(&mbar[b & 1]);
      // keep at most two batches in flight
      if (b >= 1) {
        if (!adg::tc::mbar_wait(&mbar[(b - 1) & 1], ph[(b - 1) & 1], kWaitIters)) {
          atomicOr(err, 2u);
          break;
        }
        ph[(b - 1) & 1] ^= 1u;
      }
    }
    if (batches >= 1 && !adg::tc::mbar_wait(&mbar[(batches - 1) & 1], ph[(batches - 1) & 1], kWaitIters))
      atomicOr(err, 2u);
  }
  adg::tc::fence_before();
  __syncthreads();
  adg::tc::fence_after();
  if (t < 32) adg::tc::tmem_dealloc<512>(tb);
}

template <typename T>
__global__ void __launch_bounds__(256) fma_loop(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == (T)-1.2345) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the loop
}

}  // namespace

extern "C" int adg_measure_peak(int kind, int device, int reps, double* flops, double* ms) {
  if (kind < 0 || kind > 2 || reps < 1 || !flops || !ms) return ADG_E_INVALID;
  if (cudaSetDevice(device) != cudaSuccess) return ADG_E_INVALID;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return ADG_E_CUDA;
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return ADG_E_CUDA;
  unsigned int* err = nullptr;
  void* out = nullptr;
  cudaEvent_t e0, e1;
  cudaError_t ce = cudaMalloc(&err, sizeof(unsigned int));
  if (ce == cudaSuccess) ce = cudaMalloc(&out, (size_t)sms * 8 * 256 * 8);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(err, 0, sizeof(unsigned int), st);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  double per = 0.0;
  const int smem = kMmaN * kMmaK * 4;
  auto launch = [&]() -> cudaError_t {
    if (kind == 0) {
      const int batches = 4096;
      mma_tf32_loop<<<sms, 128, smem, st>>>(batches, err);
      per = (double)sms * batches * kBatch * 2.0 * 128 * kMmaN * 8;
    } else if (kind == 1) {
      const int iters = 1 << 16;
      fma_loop<float><<<sms * 8, 256, 0, st>>>((float*)out, iters, 0.999999f, 1e-7f);
      per = (double)sms * 8 * 256 * iters * 4 * 8 * 2.0;
    } else {
      const int iters = 1 << 11;
      fma_loop<double><<<sms * 8, 256, 0, st>>>((double*)out, iters, 0.999999, 1e-7);
      per = (double)sms * 8 * 256 * iters * 4 * 8 * 2.0;
    }
    return cudaGetLastError();
  };
  if (ce == cudaSuccess && kind == 0)
    ce = (cudaError_t)adg::configure_on_device((const void*)mma_tf32_loop, [&] {
      return cudaFuncSetAttribute(mma_tf32_loop, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
  if (ce == cudaSuccess) ce = launch();  // untimed
  if (ce == cudaSuccess) ce = cudaEventRecord(e0, st);
  for (int r = 0; r < reps && ce == cudaSuccess; ++r) ce = launch();
  if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  float t = 0.f;
  unsigned int herr = 0;
  if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
  if (ce == cudaSuccess) ce = cudaMemcpy(&herr, err, sizeof(unsigned int), cudaMemcpyDeviceToHost);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(err);
  cudaFree(out);
  cudaStreamDestroy(st);
  if (ce != cudaSuccess) return ADG_E_CUDA;
  if (herr) return ADG_E_TIMEOUT;
  *flops = per * reps;
  *ms = t;
  return ADG_OK;
}

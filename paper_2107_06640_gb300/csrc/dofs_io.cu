// Dofs between the caller's element order and the library's cluster order, on
// the device: upload  out[i] = in[order[i]]  (caller FP32 -> dofs precision T),
// download out[order[i]] = in[i]  (T -> FP32); rows of `per` values
// (S x 9 x B per element).  One warp per row, 16-byte chunks where the row
// length allows.  Also the gather (subset readout) and scatter (subset
// overwrite) of listed elements' rows.
#include <cuda_runtime.h>

#include <cstdint>

namespace adg {

namespace {

template <typename T, bool kUp, int W>
__global__ void __launch_bounds__(256) permute_dofs_kernel(const void* __restrict__ in, void* __restrict__ out,
                                                            const int64_t* __restrict__ order, int64_t nt,
                                                            int per) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cpr = per / W;  // chunks per row
  for (int64_t i = (int64_t)blockIdx.x * 8 + warp; i < nt; i += (int64_t)gridDim.x * 8) {
    const int64_t u = order[i];  // the caller's element of library element i
    for (int c = lane; c < cpr; c += 32) {
      if (kUp) {
        const float* src = static_cast<const float*>(in) + u * per + c * W;
        T* dst = static_cast<T*>(out) + i * per + c * W;
        if (W == 4) {
          const float4 x = *reinterpret_cast<const float4*>(src);
          dst[0] = (T)x.x; dst[1] = (T)x.y; dst[2] = (T)x.z; dst[3] = (T)x.w;
        } else {
          dst[0] = (T)src[0];
        }
      } else {
        const T* src = static_cast<const T*>(in) + i * per + c * W;
        float* dst = static_cast<float*>(out) + u * per + c * W;
        if (W == 4)
          *reinterpret_cast<float4*>(dst) = make_float4((float)src[0], (float)src[1], (float)src[2], (float)src[3]);
        else
          dst[0] = (float)src[0];
      }
    }
  }
}

template <typename T, bool kUp>
void launch_t(const void* in, void* out, const int64_t* order, int64_t nt, int per, unsigned grid, cudaStream_t st) {
  if (per % 4 == 0)
    permute_dofs_kernel<T, kUp, 4><<<grid, 256, 0, st>>>(in, out, order, nt, per);
  else
    permute_dofs_kernel<T, kUp, 1><<<grid, 256, 0, st>>>(in, out, order, nt, per);
}

// out[k] = Q[idx[k]]: rows of `per` values of the listed library elements
template <typename T>
__global__ void __launch_bounds__(256) gather_dofs_kernel(const T* __restrict__ Q, const int64_t* __restrict__ idx,
                                                           int64_t n, int per, T* __restrict__ out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t k = (int64_t)blockIdx.x * 8 + warp; k < n; k += (int64_t)gridDim.x * 8)
    for (int c = lane; c < per; c += 32) out[k * per + c] = Q[idx[k] * per + c];
}

// Q[idx[k]] = in[k]: rows of the listed library elements overwritten
template <typename T>
__global__ void __launch_bounds__(256) scatter_dofs_kernel(const T* __restrict__ in, const int64_t* __restrict__ idx,
                                                            int64_t n, int per, T* __restrict__ Q) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t k = (int64_t)blockIdx.x * 8 + warp; k < n; k += (int64_t)gridDim.x * 8)
    for (int c = lane; c < per; c += 32) Q[idx[k] * per + c] = in[k * per + c];
}

}  // namespace

int launch_scatter_dofs(int fp64, const void* in, const int64_t* idx, int64_t n, int per, void* Q, void* stream) {
  if (n <= 0) return 0;
  const int64_t want = (n + 7) / 8;
  const unsigned grid = (unsigned)(want < 4096 ? want : 4096);
  if (fp64)
    scatter_dofs_kernel<double><<<grid, 256, 0, (cudaStream_t)stream>>>((const double*)in, idx, n, per, (double*)Q);
  else
    scatter_dofs_kernel<float><<<grid, 256, 0, (cudaStream_t)stream>>>((const float*)in, idx, n, per, (float*)Q);
  return (int)cudaGetLastError();
}

int launch_gather_dofs(int fp64, const void* Q, const int64_t* idx, int64_t n, int per, void* out, void* stream) {
  if (n <= 0) return 0;
  const int64_t want = (n + 7) / 8;
  const unsigned grid = (unsigned)(want < 4096 ? want : 4096);
  if (fp64)
    gather_dofs_kernel<double><<<grid, 256, 0, (cudaStream_t)stream>>>((const double*)Q, idx, n, per, (double*)out);
  else
    gather_dofs_kernel<float><<<grid, 256, 0, (cudaStream_t)stream>>>((const float*)Q, idx, n, per, (float*)out);
  return (int)cudaGetLastError();
}

int launch_permute_dofs(int fp64, int up, const void* in, void* out, const int64_t* order, int64_t nt, int per,
                        int n_sms, void* stream) {
  if (nt <= 0) return 0;
  const int64_t want = (nt + 7) / 8;
  const unsigned grid = (unsigned)(want < 16 * (int64_t)n_sms ? want : 16 * (int64_t)n_sms);
  cudaStream_t st = (cudaStream_t)stream;
  if (fp64) {
    if (up) launch_t<double, true>(in, out, order, nt, per, grid, st);
    else launch_t<double, false>(in, out, order, nt, per, grid, st);
  } else {
    if (up) launch_t<float, true>(in, out, order, nt, per, grid, st);
    else launch_t<float, false>(in, out, order, nt, per, grid, st);
  }
  return (int)cudaGetLastError();
}

namespace {
template <typename T>
__global__ void __launch_bounds__(256) isotropic_fluid_kernel(T* __restrict__ Q, const int64_t* __restrict__ elems,
                                                               int64_t n, int sb, int B) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n * sb) return;
  const int64_t e = elems[k / sb];
  const int r = (int)(k % sb), s = r / B, l = r - s * B;
  T* q = Q + ((e * (sb / B) + s) * 9) * B + l;  // row p of virtual element (e, s) at q[p * B]
  const T m = (q[0] + q[B] + q[2 * B]) / T(3);
  q[0] = m;
  q[B] = m;
  q[2 * B] = m;
  q[3 * B] = T(0);
  q[4 * B] = T(0);
  q[5 * B] = T(0);
}
}  // namespace

int launch_isotropic_fluid(int fp64, void* Q, const int64_t* elems, int64_t n, int sb, int B, void* stream) {
  if (n <= 0) return 0;
  const int64_t total = n * sb;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  if (fp64)
    isotropic_fluid_kernel<double><<<blocks, 256, 0, (cudaStream_t)stream>>>((double*)Q, elems, n, sb, B);
  else
    isotropic_fluid_kernel<float><<<blocks, 256, 0, (cudaStream_t)stream>>>((float*)Q, elems, n, sb, B);
  return (int)cudaGetLastError();
}

}  // namespace adg

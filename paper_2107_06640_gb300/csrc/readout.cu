// Receiver readout: q at fixed reference points of fixed elements,
// out[r][s][p] = sum_l phi_r(l) Q[e_r * S + s][p][l]  (result in double).
#include <cuda_runtime.h>
#include <cstdint>

namespace adg {

template <typename T>
__global__ void receivers_kernel(int B, const T* __restrict__ Q, int S, int64_t n, const int64_t* __restrict__ elem,
                                 const double* __restrict__ phi, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // over (r, s, p)
  if (i >= n * S * 9) return;
  const int p = (int)(i % 9);
  const int64_t rs = i / 9;
  const int s = (int)(rs % S);
  const int64_t r = rs / S;
  const T* q = Q + ((elem[r] * S + s) * 9 + p) * B;
  double acc = 0;
  for (int l = 0; l < B; ++l) acc += phi[r * B + l] * (double)q[l];
  out[i] = acc;
}

int launch_receivers(int fp64, int B, const void* Q, int S, int64_t n, const int64_t* elem, const double* phi,
                     double* out, void* stream) {
  const int64_t tot = n * S * 9;
  if (tot <= 0) return 0;
  const unsigned grid = (unsigned)((tot + 127) / 128);
  if (fp64)
    receivers_kernel<double><<<grid, 128, 0, (cudaStream_t)stream>>>(B, (const double*)Q, S, n, elem, phi, out);
  else
    receivers_kernel<float><<<grid, 128, 0, (cudaStream_t)stream>>>(B, (const float*)Q, S, n, elem, phi, out);
  return (int)cudaGetLastError();
}

}  // namespace adg

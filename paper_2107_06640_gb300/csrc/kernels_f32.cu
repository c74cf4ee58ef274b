// FP32 instantiations of the element-update kernels.
#include "kernels_impl.cuh"

namespace adg {
int launch_local_f32(int N, const StepArgs& a, int64_t nb, void* st) {
  return dispatch_local<float>(N, a, nb, (cudaStream_t)st);
}
int launch_neighbour_f32(int N, const StepArgs& a, int64_t nb, void* st) {
  return dispatch_neighbour<float>(N, a, nb, (cudaStream_t)st);
}
int smem_f32(int N) { return smem_of<float>(N); }

int launch_local_f64(int N, const StepArgs& a, int64_t nb, void* st);
int launch_neighbour_f64(int N, const StepArgs& a, int64_t nb, void* st);
int smem_f64(int N);

int launch_local(int fp64, int N, const StepArgs& a, int64_t nblocks, void* stream) {
  return fp64 ? launch_local_f64(N, a, nblocks, stream) : launch_local_f32(N, a, nblocks, stream);
}
int launch_neighbour(int fp64, int N, const StepArgs& a, int64_t nblocks, void* stream) {
  return fp64 ? launch_neighbour_f64(N, a, nblocks, stream) : launch_neighbour_f32(N, a, nblocks, stream);
}
int local_smem_bytes(int fp64, int N) { return fp64 ? smem_f64(N) : smem_f32(N); }
}  // namespace adg

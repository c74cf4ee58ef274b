// FP64 instantiations of the element-update kernels.
#include "kernels_impl.cuh"

namespace adg {
int launch_local_f64(int N, const StepArgs& a, const Segs& nb, int th, void* st) {
  return dispatch_local<double>(N, a, nb, th, (cudaStream_t)st);
}
int launch_neighbour_f64(int N, const StepArgs& a, const Segs& nb, int th, void* st) {
  return dispatch_neighbour<double>(N, a, nb, th, (cudaStream_t)st);
}
int smem_f64(int N) { return smem_of<double>(N); }
}  // namespace adg

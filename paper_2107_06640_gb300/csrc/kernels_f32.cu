// FP32 instantiations of the element-update kernels.
#include "kernels_impl.cuh"

namespace adg {
int launch_local_f32(int N, const StepArgs& a, const Segs& nb, int th, void* st) {
  return dispatch_local<float>(N, a, nb, th, (cudaStream_t)st);
}
int launch_neighbour_f32(int N, const StepArgs& a, const Segs& nb, int th, void* st) {
  return dispatch_neighbour<float>(N, a, nb, th, (cudaStream_t)st);
}
int smem_f32(int N) { return smem_of<float>(N); }

int launch_local_f64(int N, const StepArgs& a, const Segs& nb, int th, void* st);
int launch_neighbour_f64(int N, const StepArgs& a, const Segs& nb, int th, void* st);
int smem_f64(int N);

int launch_local(int fp64, int N, const StepArgs& a, const Segs& g, void* stream, int threads) {
  return fp64 ? launch_local_f64(N, a, g, threads, stream) : launch_local_f32(N, a, g, threads, stream);
}
int launch_neighbour(int fp64, int N, const StepArgs& a, const Segs& g, void* stream, int threads) {
  return fp64 ? launch_neighbour_f64(N, a, g, threads, stream) : launch_neighbour_f32(N, a, g, threads, stream);
}
int local_smem_bytes(int fp64, int N) { return fp64 ? smem_f64(N) : smem_f32(N); }

Segs make_segs(const Seg* s, int n, int unit, int chunk) {
  Segs g{};
  g.chunk = chunk < 1 ? 1 : chunk;
  int64_t u = 0;
  for (int i = 0; i < n && g.n < kMaxSeg; ++i) {
    if (s[i].n <= 0) continue;
    g.s[g.n] = s[i];
    g.first[g.n] = u;
    u += (s[i].n + unit - 1) / unit;
    g.n++;
  }
  g.first[g.n] = u;
  return g;
}
}  // namespace adg

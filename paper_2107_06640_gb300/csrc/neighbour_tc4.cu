// Degree-4 instantiation of the tensor-core neighbour kernel.
#include "neighbour_tc.cuh"

namespace adg {

int launch_neighbour_tc4(const StepArgs& a, const Segs& g, int n_sms, void* stream, bool coarse) {
  return launch_neighbour_tc_deg<4>(a, g, n_sms, stream, coarse);
}

}  // namespace adg

// Degree-4 instantiation of the tensor-core local kernel.
#include "local_tc.cuh"

namespace adg {

int launch_local_tc4(const StepArgs& a, const Segs& g, int n_sms, void* stream, bool buffers, bool acoustic,
                     bool grav) {
  return launch_local_tc_deg<4>(a, g, n_sms, stream, buffers, acoustic, grav);
}

}  // namespace adg

// Degree-5 instantiation of the tensor-core neighbour kernel, and the degree
// dispatch of its launcher and lift operand (degree 4: neighbour_tc4.cu).
#include "neighbour_tc.cuh"

namespace adg {

int launch_neighbour_tc4(const StepArgs& a, const Segs& g, int n_sms, void* stream, bool coarse);

int launch_neighbour_tc(int degree, const StepArgs& a, const Segs& g, int n_sms, void* stream, bool coarse) {
  if (degree == 4) return launch_neighbour_tc4(a, g, n_sms, stream, coarse);
  if (degree != 5) return (int)cudaErrorInvalidValue;
  return launch_neighbour_tc_deg<5>(a, g, n_sms, stream, coarse);
}

void pack_lift_tc(int degree, const double* lift, float* out) {
  if (degree == 4)
    pack_lift_tc_deg<4>(lift, out);
  else
    pack_lift_tc_deg<5>(lift, out);
}

int lift_tc_floats(int degree) { return degree == 4 ? 2 * NImg<4>::sL : 2 * NImg<5>::sL; }

}  // namespace adg

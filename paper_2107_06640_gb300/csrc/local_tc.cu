// Degree-5 instantiation of the tensor-core local kernel, and the degree
// dispatch of its launcher and operand image (degree 4: local_tc4.cu).
#include "local_tc.cuh"

namespace adg {

int launch_local_tc4(const StepArgs& a, const Segs& g, int n_sms, void* stream, bool buffers, bool acoustic,
                     bool grav);

int launch_local_tc(int degree, const StepArgs& a, const Segs& g, int n_sms, void* stream, bool buffers,
                    bool acoustic, bool grav) {
  if (degree == 4) return launch_local_tc4(a, g, n_sms, stream, buffers, acoustic, grav);
  if (degree != 5) return (int)cudaErrorInvalidValue;
  return launch_local_tc_deg<5>(a, g, n_sms, stream, buffers, acoustic, grav);
}

void pack_local_tc(int degree, const double* kt, const double* kvol, const double* efc, float* out) {
  if (degree == 4)
    pack_local_tc_deg<4>(kt, kvol, efc, out);
  else
    pack_local_tc_deg<5>(kt, kvol, efc, out);
}

int local_tc_floats(int degree) { return degree == 4 ? LImg<4>::floats : LImg<5>::floats; }

}  // namespace adg

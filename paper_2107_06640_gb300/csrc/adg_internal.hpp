// Internal context of the C ABI (not part of the public interface).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/adg.h"
#include "kernels.cuh"
#include "refmat.hpp"

namespace adg {

struct AdgError : std::runtime_error {
  int code;
  AdgError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};
[[noreturn]] void throw_err(int code, const std::string& m);
void tet_rule(int deg, std::vector<double>& pts, std::vector<double>& w);

// receiver readout kernel launcher (readout.cu)
int launch_receivers(int fp64, int B, const void* Q, int S, int64_t n, const int64_t* elem,
                     const double* phi, double* out, void* stream);

struct Ctx {
  adg_config cfg{};
  std::string last_error;
  // user mesh
  int64_t nv = 0, nt = 0;
  std::vector<double> xyz;
  std::vector<int64_t> tets, partner;
  std::vector<int32_t> tag;
  std::vector<double> rho, lam, mu;
  bool has_mesh = false, has_mat = false, inited = false;
  // discretisation
  int N = 0, B = 0, Bf = 0, B1 = 0, S = 1;
  bool fp64 = true;
  RefOps ops;
  int ncl = 1;
  std::vector<int64_t> order, inv, cl_begin;
  std::vector<int> cluster;
  double dtmin = 0, time = 0;
  int64_t tick = 0;
  std::vector<int64_t> gfaces;  // user tet*4+face of gravity faces
  int n_bslots = 0, n_dslots = 0, n_gslots = 0;
  int64_t n_fault_faces = 0;
  // device
  cudaStream_t stream = nullptr, own_stream = nullptr;
  std::vector<void*> owned;
  int64_t dev_bytes = 0;
  void *dQ = nullptr, *dTrace = nullptr, *dDtrace = nullptr;
  double *dBtrace = nullptr, *dEta = nullptr, *dGpar = nullptr;
  void *dPar = nullptr, *dFm = nullptr, *dFp = nullptr;
  void *dKt = nullptr, *dKvol = nullptr, *dEfc = nullptr, *dLift = nullptr;
  int *dNbr = nullptr, *dNinfo = nullptr, *dGslot = nullptr, *dBslot = nullptr, *dDslot = nullptr,
      *dPerm = nullptr;
  unsigned int* dErr = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  bool use_graph = true;
  // per-kernel profiling (adg_profile)
  struct ProfEv { int kind; cudaEvent_t a, b; };
  std::vector<ProfEv>* prof = nullptr;
  // receivers
  int64_t n_rec = 0;
  int64_t* dRecElem = nullptr;
  double *dRecPhi = nullptr, *dRecOut = nullptr;

  void setup();
  StepArgs base_args() const;
  void launch_tick(int s, double dtm);
  void run_macro(double scale);
  int64_t launches_per_macro() const;
  void check_err();
  ~Ctx();
};

}  // namespace adg

struct adg_ctx {
  adg::Ctx c;
};

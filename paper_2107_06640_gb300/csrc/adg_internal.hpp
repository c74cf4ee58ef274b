// Internal context of the C ABI (not part of the public interface).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
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

// friction-guess network training (mlp.cu)
int mlp_trainable();
int launch_mlp_grad(const float* P, const float* rows, int64_t row0, int64_t n, int64_t n_norm, float* grad,
                    double* loss, void* stream);
int launch_adam(float* P, const float* g, float* m, float* v, float lr, int step, void* stream);

// dofs reordering between the caller's and the library's element order (dofs_io.cu)
int launch_permute_dofs(int fp64, int up, const void* in, void* out, const int64_t* order, int64_t nt, int per,
                        int n_sms, void* stream);
int launch_gather_dofs(int fp64, const void* Q, const int64_t* idx, int64_t n, int per, void* out, void* stream);
int launch_scatter_dofs(int fp64, const void* in, const int64_t* idx, int64_t n, int per, void* Q, void* stream);
// the stress of the listed elements' dofs replaced by its isotropic part:
// sigma_xx = sigma_yy = sigma_zz = their mean, no shear (rows [9][B] per
// virtual element, `sb` = S x B columns of basis functions per element)
int launch_isotropic_fluid(int fp64, void* Q, const int64_t* elems, int64_t n, int sb, int B, void* stream);
// receiver readout kernel launcher (readout.cu)
int launch_receivers(int fp64, int B, const void* Q, int S, int64_t n, const int64_t* elem,
                     const double* phi, double* out, void* stream);

// Host-side plan of a mesh (caller's element order): geometry, face
// connectivity, CFL time steps and rate-2 clusters (Sec. 4.4)
struct MeshPlan {
  std::vector<double> Jinv, detJ, area, nrm, fcen, h, dte;  // [E*9], [E], [E*4], [E*12], [E*12], [E], [E]
  std::vector<int64_t> nbr;                                // [E*4] neighbour tet or -1
  std::vector<int> nface, nperm, cl;                       // [E*4] its face, node permutation; [E] cluster
  double dtmin = 0;
  int ncl = 1;
};

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
  // host plan for adg_plan / adg_face_flux / adg_face_neighbour, kept until the
  // next mesh or material upload (adg_init builds its own)
  std::unique_ptr<struct MeshPlan> host_plan;
  RefOps host_ops;
  // discretisation
  int N = 0, B = 0, Bf = 0, B1 = 0, S = 1;
  bool fp64 = true;
  bool tc = false;          // tensor-core (3xTF32) local kernel in use
  int n_sms = 1;
  float* dTcLocal = nullptr;
  float* dTcLift = nullptr;
  RefOps ops;
  int ncl = 1;
  std::vector<int64_t> order, inv, cl_begin;
  // elements [cl_begin[c], cl_begin[c] + cl_plain[c]) of cluster c have no
  // gravitational face, fault face or LTS buffer (tensor-core local kernel)
  std::vector<int64_t> cl_plain;
  // cluster c's tensor-core range includes elements with a coarser or finer
  // neighbour (the neighbour kernel's LTS-face code)
  std::vector<char> cl_tc_lts;
  // acoustic ocean (adg_set_acoustic_ocean): the plain fluid elements of
  // cluster c, [cl_begin[c] + cl_elastic[c], + cl_fluid[c]), take the
  // 4-quantity local kernel; the library keeps fluid stress isotropic
  bool acoustic = false;
  std::vector<int64_t> cl_elastic, cl_fluid;
  // the last cl_grav[c] elements of cluster c's tensor-core range have one
  // gravitational face or a finer neighbour (their own local launch; dGscr:
  // the gravitational faces' scratch)
  std::vector<int64_t> cl_grav;
  float* dGscr = nullptr;
  int64_t* dFluid = nullptr;  // library indices of all fluid elements (projection at upload)
  int64_t n_fluid = 0;
  void project_fluid(bool sync = true);  // fluid stress -> its isotropic part, on the device
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
  void *dQ = nullptr, *dTrace = nullptr, *dDtrace = nullptr, *dGflux = nullptr;
  int64_t* dOrder = nullptr;  // order on the device: the caller's element of library element i
  double *dBtrace = nullptr, *dEta = nullptr, *dGpar = nullptr;
  void *dPar = nullptr, *dFm = nullptr, *dFp = nullptr;
  float* dFrec = nullptr;  // face records of the tensor-core neighbour kernel
  void *dKt = nullptr, *dKvol = nullptr, *dEfc = nullptr, *dLift = nullptr;
  int *dNbr = nullptr, *dNinfo = nullptr, *dGslot = nullptr, *dBslot = nullptr, *dDslot = nullptr,
      *dPerm = nullptr;
  unsigned int* dErr = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  bool use_graph = true;
  // launch shapes (adg_autotune; phase 0 local, 1 neighbour): threads per
  // element block of the CUDA-core kernels, consecutive tiles per CTA-slot
  // sweep of the tensor-core kernels
  int cc_threads[2] = {128, 128};
  int tc_chunk[2] = {1, 1};
  // dynamic rupture: fault faces in internal (cluster) order
  int64_t nff = 0;
  std::vector<int> fface;                 // [nff][5] minus elem, face, plus elem, face, perm
  std::vector<int64_t> fcl_begin;         // per cluster ranges of fault faces
  std::vector<int64_t> fminus_user, fplus_user;  // user tet*4+face of both sides
  std::vector<double> fgeo;               // [nff][FGEO]
  int *dFface = nullptr, *dFslot = nullptr;
  double *dFgeo = nullptr, *dFpar = nullptr, *dFstate = nullptr;
  void* dDrout = nullptr;
  unsigned long long* dNewton = nullptr;
  bool fault_set = false;
  // friction-guess network and training-sample capture
  float* dMlp = nullptr;
  bool mlp_on = false;
  int fric_law = 0;  // ADG_FRICTION_RS / ADG_FRICTION_LSW
  float* dCapture = nullptr;
  unsigned long long* dCapCount = nullptr;
  int64_t cap_capacity = 0;
  bool cap_on = false;
  void launch_rupture_cluster(int c, double dt);
  // per-kernel profiling (adg_profile)
  struct ProfEv { int kind; cudaEvent_t a, b; int launches; cudaEvent_t m = nullptr; };  // m: after the tensor-core launch
  std::vector<ProfEv>* prof = nullptr;
  // pinned host staging buffer for dofs upload / download (allocated on first use)
  void* hstage = nullptr;
  size_t hstage_bytes = 0;
  // pipelined FP32 dofs transfers (adg_set_dofs_f32_async / adg_get_dofs_f32_async):
  // two device staging buffers for uploads and two for downloads (transfer j
  // uses buffer j % 2, so a copy never waits for the reordering of the
  // transfer just before it), a copy stream for each direction, and the
  // events that order them with the library stream (created on first use)
  struct AsyncIo {
    cudaStream_t in = nullptr, out = nullptr;
    float *dIn[2] = {nullptr, nullptr}, *dOut[2] = {nullptr, nullptr};
    cudaEvent_t in_copied[2] = {nullptr, nullptr};   // an upload's host copy has landed in dIn[b]
    cudaEvent_t in_used[2] = {nullptr, nullptr};     // the library stream has reordered dIn[b] into the dofs
    cudaEvent_t out_made[2] = {nullptr, nullptr};    // the library stream has written a download into dOut[b]
    cudaEvent_t out_copied[2] = {nullptr, nullptr};  // dOut[b] has been copied to the host
    int64_t n_in = 0, n_out = 0;                     // uploads and downloads enqueued so far
  } aio;
  void aio_setup();
  void aio_sync();
  void aio_free();
  // receivers
  int64_t n_rec = 0;
  int64_t* dRecElem = nullptr;
  double *dRecPhi = nullptr, *dRecOut = nullptr;
  // recording at a cadence (adg_record_*): [0] receivers, [1] sea-surface height
  struct Recorder {
    int every = 0;                  // macro steps between samples; 0: off
    int64_t cap = 0, count = 0, read = 0, dropped = 0, macro = 0;
    size_t sample = 0;              // doubles per sample
    double* dRing = nullptr;        // device ring [cap][sample]
    double* hRing = nullptr;        // pinned host ring [cap][sample]
    std::vector<double> t;          // [cap] time of the sample in each slot
    std::vector<cudaEvent_t> taken, copied;  // [cap] sample taken / copied to the host ring
  };
  Recorder rec[2];
  cudaStream_t rec_stream = nullptr;
  void record_after_macro();
  void record_free(int kind);

  void plan_mesh(const RefOps& o, int degree, MeshPlan& plan) const;
  void face_flux(const MeshPlan& pl, int64_t eu, int f, double* Fm, double* Fp) const;
  void face_neighbour(const MeshPlan& pl, const RefOps& o, int64_t eu, int f, int64_t* nb, int* nf,
                      int32_t* node_map) const;
  void setup();
  StepArgs base_args() const;
  void launch_tick(int s, double dtm);
  void run_macro(double scale);
  int64_t launches_per_macro() const;
  void autotune(int reps, bool force, int* choice, double* ms);
  void check_err();
  ~Ctx();
};

}  // namespace adg

struct adg_ctx {
  adg::Ctx c;
};

// extern "C" entry points for dynamic rupture (Sec. 3, Eq. bc-dynrup) and the
// friction-guess network: fault-face listing, per-node parameters, state
// readout, Newton statistics, training-sample capture and on-GPU training.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "adg_internal.hpp"

using adg::Ctx;

namespace {

template <typename F>
int guard(adg_ctx* ctx, F&& f) {
  try {
    f();
    if (ctx) ctx->c.last_error.clear();
    return ADG_OK;
  } catch (const adg::AdgError& ex) {
    if (ctx) ctx->c.last_error = ex.what();
    return ex.code;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->c.last_error = "out of host memory";
    return ADG_E_NOMEM;
  } catch (const std::exception& ex) {
    if (ctx) ctx->c.last_error = ex.what();
    return ADG_E_INVALID;
  }
}

void cuda_ok(cudaError_t e, const char* what) {
  if (e != cudaSuccess) adg::throw_err(ADG_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void need_faults(const Ctx& c) {
  if (!c.inited) adg::throw_err(ADG_E_STATE, "call adg_init first");
  if (!c.nff) adg::throw_err(ADG_E_STATE, "the mesh has no fault faces");
}

const int kFaceV[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

}  // namespace

extern "C" {

int adg_fault_faces(adg_ctx* ctx, int64_t* minus_face, int64_t* plus_face, double* node_xyz, double* normal) {
  if (!ctx) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_faults(c);
    for (int64_t i = 0; i < c.nff; ++i) {
      if (minus_face) minus_face[i] = c.fminus_user[i];
      if (plus_face) plus_face[i] = c.fplus_user[i];
      if (normal)
        for (int d = 0; d < 3; ++d) normal[3 * i + d] = c.fgeo[i * adg::FGEO + d];
      if (node_xyz) {
        const int64_t e = c.fminus_user[i] / 4;
        const int f = (int)(c.fminus_user[i] % 4);
        const double* A = &c.xyz[3 * c.tets[4 * e + kFaceV[f][0]]];
        const double* Bv = &c.xyz[3 * c.tets[4 * e + kFaceV[f][1]]];
        const double* C = &c.xyz[3 * c.tets[4 * e + kFaceV[f][2]]];
        for (int n = 0; n < c.Bf; ++n) {
          const double c1 = c.ops.node_chi[2 * n], c2 = c.ops.node_chi[2 * n + 1];
          for (int d = 0; d < 3; ++d)
            node_xyz[((size_t)i * c.Bf + n) * 3 + d] = A[d] + c1 * (Bv[d] - A[d]) + c2 * (C[d] - A[d]);
        }
      }
    }
  });
}

int adg_set_fault(adg_ctx* ctx, const double* par) {
  if (!ctx || !par) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_faults(c);
    const size_t npts = (size_t)c.nff * c.S * c.Bf;
    std::vector<double> st(npts * adg::FSTATE, 0.0);
    for (size_t k = 0; k < npts; ++k) {
      const double* p = par + k * adg::FPAR;
      if (c.fric_law == ADG_FRICTION_LSW) {
        if (!(p[1] >= 0) || !(p[0] >= p[1]) || !(p[2] > 0) || !(p[3] >= 0) || !(p[11] >= 0) || !(p[12] >= 0))
          adg::throw_err(ADG_E_INVALID,
                         "slip-weakening parameters: need mu_s >= mu_d >= 0, D_c > 0, cohesion >= 0, "
                         "initial slip path and slip rate >= 0");
      } else if (!(p[0] > 0) || !(p[2] > 0) || !(p[4] > 0) || !(p[6] > 0) || !(p[12] > 0)) {
        adg::throw_err(ADG_E_INVALID, "fault parameters: a, L, V0, V_w and the initial slip rate must be positive");
      }
      st[k * adg::FSTATE + 0] = p[12];
      st[k * adg::FSTATE + 1] = p[11];
    }
    cuda_ok(cudaMemcpy(c.dFpar, par, npts * adg::FPAR * 8, cudaMemcpyHostToDevice), "fault parameters");
    cuda_ok(cudaMemcpy(c.dFstate, st.data(), st.size() * 8, cudaMemcpyHostToDevice), "fault state");
    c.fault_set = true;
  });
}

int adg_set_friction_law(adg_ctx* ctx, int law) {
  if (!ctx || (law != ADG_FRICTION_RS && law != ADG_FRICTION_LSW)) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_faults(c);
    c.fric_law = law;
    c.fault_set = false;  // the parameters mean other things under the other law
  });
}

int adg_read_fault(adg_ctx* ctx, double* state) {
  if (!ctx || !state) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_faults(c);
    cuda_ok(cudaStreamSynchronize(c.stream), "fault readout");
    cuda_ok(cudaMemcpy(state, c.dFstate, (size_t)c.nff * c.S * c.Bf * adg::FSTATE * 8, cudaMemcpyDeviceToHost),
            "fault readout");
  });
}

int adg_fault_stats(adg_ctx* ctx, int64_t* solves, int64_t* iterations, int reset) {
  if (!ctx || !solves || !iterations) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_faults(c);
    cuda_ok(cudaStreamSynchronize(c.stream), "fault stats");
    unsigned long long h[2];
    cuda_ok(cudaMemcpy(h, c.dNewton, sizeof(h), cudaMemcpyDeviceToHost), "fault stats");
    *solves = (int64_t)h[0];
    *iterations = (int64_t)h[1];
    if (reset) cuda_ok(cudaMemset(c.dNewton, 0, sizeof(h)), "fault stats");
  });
}

int adg_rupture_capture(adg_ctx* ctx, int64_t capacity, int64_t* n_captured) {
  if (!ctx || capacity < 0) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_faults(c);
    cuda_ok(cudaStreamSynchronize(c.stream), "capture");
    unsigned long long n = 0;
    cuda_ok(cudaMemcpy(&n, c.dCapCount, sizeof(n), cudaMemcpyDeviceToHost), "capture");
    if (n_captured) *n_captured = (int64_t)std::min<unsigned long long>(n, (unsigned long long)c.cap_capacity);
    if (capacity == 0) {
      c.cap_on = false;
      return;
    }
    if (capacity != c.cap_capacity) {
      if (c.dCapture) {
        cudaFree(c.dCapture);
        for (auto& o : c.owned)
          if (o == c.dCapture) o = nullptr;
        c.dCapture = nullptr;
      }
      cuda_ok(cudaMalloc((void**)&c.dCapture, (size_t)capacity * (adg::MLP_IN + 1) * sizeof(float)), "capture");
      c.owned.push_back(c.dCapture);
      c.cap_capacity = capacity;
    }
    cuda_ok(cudaMemset(c.dCapCount, 0, sizeof(unsigned long long)), "capture");
    c.cap_on = true;
    if (c.graph_exec) {  // the captured graph bakes the capture pointer in
      cudaGraphExecDestroy(c.graph_exec);
      c.graph_exec = nullptr;
    }
  });
}

int adg_mlp_params(adg_ctx* ctx, const float* set, float* get, int enable) {
  if (!ctx) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_faults(c);
    if (set) cuda_ok(cudaMemcpy(c.dMlp, set, adg::MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice), "mlp set");
    if (get) cuda_ok(cudaMemcpy(get, c.dMlp, adg::MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost), "mlp get");
    if (enable >= 0 && (enable != 0) != c.mlp_on) {
      c.mlp_on = enable != 0;
      if (c.graph_exec) {
        cudaGraphExecDestroy(c.graph_exec);
        c.graph_exec = nullptr;
      }
    }
  });
}

// Train the network on the captured samples with the project's own forward /
// backward kernels (mlp.cu) and Adam; loss[0] / loss[1] = mean squared error
// of the scaled target before / after training.
int adg_mlp_train(adg_ctx* ctx, int epochs, int batch, double lr, int seed, double* loss) {
  if (!ctx || epochs < 0 || batch < 1 || !(lr > 0)) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_faults(c);
    cuda_ok(cudaStreamSynchronize(c.stream), "train");
    unsigned long long ncap = 0;
    cuda_ok(cudaMemcpy(&ncap, c.dCapCount, sizeof(ncap), cudaMemcpyDeviceToHost), "train");
    const int64_t n = (int64_t)std::min<unsigned long long>(ncap, (unsigned long long)c.cap_capacity);
    if (n < 16) adg::throw_err(ADG_E_STATE, "too few captured friction solves to train on");
    const int K = adg::MLP_IN + 1;
    std::vector<float> rows((size_t)n * K);
    cuda_ok(cudaMemcpy(rows.data(), c.dCapture, rows.size() * sizeof(float), cudaMemcpyDeviceToHost), "train");
    // fixed normalisation from the data
    std::vector<float> P(adg::MLP_NPARAM, 0.f);
    const int off_mu = adg::mlp_trainable(), off_sd = off_mu + adg::MLP_IN, off_osc = off_sd + adg::MLP_IN;
    for (int k = 0; k < K; ++k) {
      double m = 0, v = 0;
      for (int64_t i = 0; i < n; ++i) m += rows[(size_t)i * K + k];
      m /= n;
      for (int64_t i = 0; i < n; ++i) v += (rows[(size_t)i * K + k] - m) * (rows[(size_t)i * K + k] - m);
      double sd = std::sqrt(v / n);
      if (!(sd > 1e-6)) sd = 1.0;
      if (k < adg::MLP_IN) {
        P[off_mu + k] = (float)m;
        P[off_sd + k] = (float)sd;
      } else {
        P[off_osc] = (float)m;
        P[off_osc + 1] = (float)sd;
      }
    }
    std::mt19937 rng(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    const int H = adg::MLP_H, IN = adg::MLP_IN;
    int o = 0;
    for (int i = 0; i < H * IN; ++i) P[o++] = nd(rng) / std::sqrt((float)IN);
    o += H;
    for (int i = 0; i < H * H; ++i) P[o++] = nd(rng) / std::sqrt((float)H);
    o += H;
    for (int i = 0; i < H; ++i) P[o++] = nd(rng) / std::sqrt((float)H);
    const int nt = adg::mlp_trainable();
    float *dg = nullptr, *dm = nullptr, *dv = nullptr;
    double* dl = nullptr;
    cuda_ok(cudaMalloc((void**)&dg, nt * 4), "train");
    cuda_ok(cudaMalloc((void**)&dm, nt * 4), "train");
    cuda_ok(cudaMalloc((void**)&dv, nt * 4), "train");
    cuda_ok(cudaMalloc((void**)&dl, 8), "train");
    struct Free {
      void* p[4];
      ~Free() { for (void* q : p) cudaFree(q); }
    } fr{{dg, dm, dv, dl}};
    cuda_ok(cudaMemset(dm, 0, nt * 4), "train");
    cuda_ok(cudaMemset(dv, 0, nt * 4), "train");
    cuda_ok(cudaMemcpy(c.dMlp, P.data(), P.size() * 4, cudaMemcpyHostToDevice), "train");
    auto full_loss = [&]() {
      cuda_ok(cudaMemsetAsync(dg, 0, nt * 4, c.stream), "train");
      cuda_ok(cudaMemsetAsync(dl, 0, 8, c.stream), "train");
      if (adg::launch_mlp_grad(c.dMlp, c.dCapture, 0, n, n, dg, dl, c.stream)) adg::throw_err(ADG_E_CUDA, "mlp grad");
      double h = 0;
      cuda_ok(cudaMemcpyAsync(&h, dl, 8, cudaMemcpyDeviceToHost, c.stream), "train");
      cuda_ok(cudaStreamSynchronize(c.stream), "train");
      return h;
    };
    if (loss) loss[0] = full_loss();
    int step = 0;
    for (int ep = 0; ep < epochs; ++ep)
      for (int64_t r0 = 0; r0 < n; r0 += batch) {
        const int64_t m = std::min<int64_t>(batch, n - r0);
        cuda_ok(cudaMemsetAsync(dg, 0, nt * 4, c.stream), "train");
        cuda_ok(cudaMemsetAsync(dl, 0, 8, c.stream), "train");
        if (adg::launch_mlp_grad(c.dMlp, c.dCapture, r0, m, m, dg, dl, c.stream)) adg::throw_err(ADG_E_CUDA, "mlp grad");
        if (adg::launch_adam(c.dMlp, dg, dm, dv, (float)lr, ++step, c.stream)) adg::throw_err(ADG_E_CUDA, "adam");
      }
    if (loss) loss[1] = full_loss();
  });
}

// Gradient of the mean loss for given parameters and samples (host arrays):
// grad[MLP trainable count], loss (mean squared scaled error).
int adg_mlp_gradient(const float* params, int64_t n, const float* rows, float* grad, double* loss) {
  if (!params || n < 1 || !rows || !grad) return ADG_E_INVALID;
  return guard(nullptr, [&] {
    const int nt = adg::mlp_trainable();
    float *dP = nullptr, *dR = nullptr, *dg = nullptr;
    double* dl = nullptr;
    cuda_ok(cudaMalloc((void**)&dP, adg::MLP_NPARAM * 4), "mlp gradient");
    struct Free {
      void** p[4];
      ~Free() { for (auto q : p) if (*q) cudaFree(*q); }
    } fr{{(void**)&dP, (void**)&dR, (void**)&dg, (void**)&dl}};
    cuda_ok(cudaMalloc((void**)&dR, (size_t)n * (adg::MLP_IN + 1) * 4), "mlp gradient");
    cuda_ok(cudaMalloc((void**)&dg, nt * 4), "mlp gradient");
    cuda_ok(cudaMalloc((void**)&dl, 8), "mlp gradient");
    cuda_ok(cudaMemcpy(dP, params, adg::MLP_NPARAM * 4, cudaMemcpyHostToDevice), "mlp gradient");
    cuda_ok(cudaMemcpy(dR, rows, (size_t)n * (adg::MLP_IN + 1) * 4, cudaMemcpyHostToDevice), "mlp gradient");
    cuda_ok(cudaMemset(dg, 0, nt * 4), "mlp gradient");
    cuda_ok(cudaMemset(dl, 0, 8), "mlp gradient");
    if (adg::launch_mlp_grad(dP, dR, 0, n, n, dg, dl, nullptr)) adg::throw_err(ADG_E_CUDA, "mlp grad");
    cuda_ok(cudaDeviceSynchronize(), "mlp gradient");
    cuda_ok(cudaMemcpy(grad, dg, nt * 4, cudaMemcpyDeviceToHost), "mlp gradient");
    if (loss) cuda_ok(cudaMemcpy(loss, dl, 8, cudaMemcpyDeviceToHost), "mlp gradient");
  });
}

}  // extern "C"

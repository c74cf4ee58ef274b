// Autotuner of the launch shapes (adg_autotune).  The work of a step is fixed
// by the scheme; how it is cut into launches is a choice per kernel kind:
//   knob 0 / 1: threads per element block of the CUDA-core local / neighbour
//               kernels (64, 128, 256);
//   knob 2 / 3: consecutive 12-element tiles a CTA slot of the tensor-core
//               local / neighbour kernel takes per sweep (1, 2, 4), i.e. the
//               elements one CTA works through before striding on.
// Each candidate is timed with CUDA events on this context's own clusters
// (whole macro steps of adg_profile's per-phase events, after one untimed
// macro step), one knob after the other; the fastest is kept.  The solver
// state the steps change (dofs, sea surface, fault state, Newton counters,
// error word, time) is copied aside on the device first and put back after,
// so tuning leaves the solution where it was.  Choices are cached for the
// process by (degree, precision, ensemble, element count rounded to a power
// of two, clusters), so a second context of the same kind reuses them.
#include <cuda_runtime.h>

#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "adg_internal.hpp"

namespace adg {

namespace {

constexpr int kCand[4][3] = {{64, 128, 256}, {64, 128, 256}, {1, 2, 4}, {1, 2, 4}};

using Key = std::tuple<int, int, int, int, int, int>;  // degree, precision, S, log2 nt, clusters, knob
std::mutex g_tune_mu;
std::map<Key, int> g_tune_cache;

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw AdgError(ADG_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// device copy of a buffer, put back by restore()
struct Saved {
  void* dst = nullptr;
  void* copy = nullptr;
  size_t bytes = 0;
};

}  // namespace

void Ctx::autotune(int reps, bool force, int* choice, double* ms) {
  // which kernel kinds run in this context
  bool runs[4] = {false, false, false, false};
  for (int c = 0; c < ncl; ++c) {
    const int64_t n = cl_begin[c + 1] - cl_begin[c], np = tc ? cl_plain[c] : 0;
    if (n > np) runs[0] = runs[1] = true;
    if (np > 0) runs[2] = runs[3] = true;
  }
  int lg = 0;
  while (((int64_t)1 << (lg + 1)) <= nt) ++lg;
  int* knob[4] = {&cc_threads[0], &cc_threads[1], &tc_chunk[0], &tc_chunk[1]};
  for (int k = 0; k < 12; ++k) ms[k] = -1.0;

  // state the timed steps change
  const size_t ts = fp64 ? 8 : 4;
  std::vector<Saved> saved = {{dQ, nullptr, (size_t)nt * S * 9 * B * ts},
                              {dEta, nullptr, (size_t)n_gslots * S * Bf * 8},
                              {dFstate, nullptr, (size_t)nff * S * Bf * FSTATE * 8},
                              {dNewton, nullptr, dNewton ? 2 * sizeof(unsigned long long) : 0},
                              {dErr, nullptr, sizeof(unsigned int)}};
  const double time0 = time;
  const int64_t tick0 = tick;
  const bool cap0 = cap_on;
  auto restore = [&] {
    for (auto& s : saved) {
      if (s.copy) {
        cudaMemcpyAsync(s.dst, s.copy, s.bytes, cudaMemcpyDeviceToDevice, stream);
      }
    }
    cudaStreamSynchronize(stream);
    for (auto& s : saved)
      if (s.copy) cudaFree(s.copy);
    time = time0;
    tick = tick0;
    cap_on = cap0;
    prof = nullptr;
  };
  try {
    for (auto& s : saved) {
      if (!s.dst || !s.bytes) continue;
      ck(cudaMalloc(&s.copy, s.bytes), "autotune: state copy");
      ck(cudaMemcpyAsync(s.copy, s.dst, s.bytes, cudaMemcpyDeviceToDevice, stream), "autotune: state copy");
    }
    cap_on = false;
    const int ticks = 1 << (ncl - 1);
    auto macro = [&](std::vector<ProfEv>* p) {
      prof = p;
      for (int s = 0; s < ticks; ++s) launch_tick(s, dtmin);
      prof = nullptr;
    };
    for (int k = 0; k < 4; ++k) {
      if (!runs[k]) {
        choice[k] = 0;
        continue;
      }
      const Key key{N, (int)cfg.precision, S, lg, ncl, k};
      if (!force) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
          *knob[k] = choice[k] = it->second;
          continue;
        }
      }
      const int phase = k & 1;
      const bool tc_knob = k >= 2;
      double best = 1e300;
      int best_c = *knob[k];
      for (int ci = 0; ci < 3; ++ci) {
        *knob[k] = kCand[k][ci];
        macro(nullptr);  // untimed
        std::vector<ProfEv> evs;
        for (int r = 0; r < reps; ++r) macro(&evs);
        ck(cudaStreamSynchronize(stream), "autotune: steps");
        double t = 0.0;
        for (auto& e : evs) {
          float x = 0.f;
          if (e.kind == phase) {
            // the tensor-core launch is timed alone (a -> m); the CUDA-core one after it (m -> b)
            if (tc_knob && e.m) ck(cudaEventElapsedTime(&x, e.a, e.m), "autotune: events");
            if (!tc_knob && e.launches > (e.m ? 1 : 0)) ck(cudaEventElapsedTime(&x, e.m ? e.m : e.a, e.b), "autotune: events");
          }
          t += x;
          cudaEventDestroy(e.a);
          cudaEventDestroy(e.b);
          if (e.m) cudaEventDestroy(e.m);
        }
        ms[3 * k + ci] = t / reps;
        if (t < best) {
          best = t;
          best_c = kCand[k][ci];
        }
      }
      *knob[k] = choice[k] = best_c;
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[key] = best_c;
    }
  } catch (...) {
    restore();
    throw;
  }
  restore();
  ck(cudaGetLastError(), "autotune");
  // the macro-step graph holds the old launch shapes
  if (graph_exec) {
    cudaGraphExecDestroy(graph_exec);
    graph_exec = nullptr;
  }
}

}  // namespace adg

extern "C" int adg_autotune(adg_ctx* ctx, int reps, int force, int* choice, double* ms) {
  if (!ctx || reps < 1 || !choice) return ADG_E_INVALID;
  adg::Ctx& c = ctx->c;
  try {
    if (!c.inited) throw adg::AdgError(ADG_E_STATE, "call adg_init first");
    if (c.tick % (1 << (c.ncl - 1))) throw adg::AdgError(ADG_E_STATE, "autotune at a macro-step boundary only");
    double scratch[12];
    c.autotune(reps, force != 0, choice, ms ? ms : scratch);
  } catch (const adg::AdgError& e) {
    c.last_error = e.what();
    return e.code;
  } catch (const std::exception& e) {
    c.last_error = e.what();
    return ADG_E_INVALID;
  }
  c.last_error.clear();
  return ADG_OK;
}

// extern "C" entry points of include/adg.h: argument checks, user<->internal
// reordering, host<->device copies and the time-stepping front end.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <stdexcept>
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
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->c.last_error = "out of host memory";
    return ADG_E_NOMEM;
  } catch (const adg::AdgError& ex) {
    if (ctx) ctx->c.last_error = ex.what();
    return ex.code;
  } catch (const std::exception& ex) {
    if (ctx) ctx->c.last_error = ex.what();
    return ADG_E_INVALID;
  }
}

constexpr size_t kStateHeader = 80;  // 10 int64 words: magic, N, S, nt, fp64, n_gface, tick, fault bytes, time, 0

void need_init(const Ctx& c) {
  if (!c.inited) adg::throw_err(ADG_E_STATE, "call adg_init first");
}

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) adg::throw_err(ADG_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Pinned staging buffer sized for the dofs in device precision: conversion to
// or from the caller's double array runs in parallel on the host, the copy over
// the host link runs from pinned memory.  Chunks of elements are converted and
// copied in a pipeline (the copy of chunk k overlaps the conversion of k+1).
template <typename T>
T* staging(Ctx& c) {
  const size_t bytes = (size_t)c.nt * c.S * 9 * c.B * sizeof(T);
  if (c.hstage_bytes < bytes) {
    if (c.hstage) cudaFreeHost(c.hstage);
    c.hstage = nullptr;
    c.hstage_bytes = 0;
    check_cuda(cudaHostAlloc(&c.hstage, bytes, cudaHostAllocDefault), "pinned staging buffer");
    c.hstage_bytes = bytes;
  }
  return (T*)c.hstage;
}

constexpr int64_t kChunks = 8;

template <typename T>
void put_dofs(Ctx& c, const double* Q) {
  const int64_t per = (int64_t)c.S * 9 * c.B;
  T* buf = staging<T>(c);
  for (int64_t ch = 0; ch < kChunks; ++ch) {
    const int64_t i0 = c.nt * ch / kChunks, i1 = c.nt * (ch + 1) / kChunks;
#pragma omp parallel for schedule(static)
    for (int64_t i = i0; i < i1; ++i) {
      const double* src = Q + c.order[i] * per;
      T* dst = buf + i * per;
      for (int64_t k = 0; k < per; ++k) dst[k] = (T)src[k];
    }
    check_cuda(cudaMemcpyAsync((T*)c.dQ + i0 * per, buf + i0 * per, (size_t)(i1 - i0) * per * sizeof(T),
                               cudaMemcpyHostToDevice, c.stream),
               "dofs upload");
  }
  check_cuda(cudaStreamSynchronize(c.stream), "dofs upload");
}
template <typename T>
void take_dofs(Ctx& c, double* Q) {
  const int64_t per = (int64_t)c.S * 9 * c.B;
  T* buf = staging<T>(c);
  // all chunk copies are queued at once; chunk k is converted as soon as its
  // copy has completed, while the later chunks are still in flight
  cudaEvent_t done[kChunks];
  for (int64_t ch = 0; ch < kChunks; ++ch) {
    const int64_t i0 = c.nt * ch / kChunks, i1 = c.nt * (ch + 1) / kChunks;
    check_cuda(cudaEventCreateWithFlags(&done[ch], cudaEventDisableTiming), "dofs download");
    check_cuda(cudaMemcpyAsync(buf + i0 * per, (const T*)c.dQ + i0 * per, (size_t)(i1 - i0) * per * sizeof(T),
                               cudaMemcpyDeviceToHost, c.stream),
               "dofs download");
    check_cuda(cudaEventRecord(done[ch], c.stream), "dofs download");
  }
  cudaError_t err = cudaSuccess;
  for (int64_t ch = 0; ch < kChunks; ++ch) {
    const int64_t i0 = c.nt * ch / kChunks, i1 = c.nt * (ch + 1) / kChunks;
    if (err == cudaSuccess) err = cudaEventSynchronize(done[ch]);
    if (err == cudaSuccess) {
#pragma omp parallel for schedule(static)
      for (int64_t i = i0; i < i1; ++i) {
        const T* src = buf + i * per;
        double* dst = Q + c.order[i] * per;
        for (int64_t k = 0; k < per; ++k) dst[k] = (double)src[k];
      }
    }
  }
  for (int64_t ch = 0; ch < kChunks; ++ch) cudaEventDestroy(done[ch]);
  check_cuda(err, "dofs download");
}

// FP32 dofs to or from the caller go through the trace array as device
// scratch: between macro steps no trace is pending, and 4 S_f >= 9 B for every
// supported degree.
float* dofs_scratch(Ctx& c) {
  if (c.tick % (1 << (c.ncl - 1)))
    adg::throw_err(ADG_E_STATE, "FP32 dofs transfer: only at a macro-step boundary");
  const size_t need = (size_t)c.nt * c.S * 9 * c.B * sizeof(float);
  const size_t have = (size_t)c.nt * c.S * 4 * adg::face_stride(c.N) * (c.fp64 ? 8 : 4);
  if (need > have) adg::throw_err(ADG_E_INVALID, "FP32 dofs transfer: scratch too small");
  return static_cast<float*>(c.dTrace);
}

void run_ticks_to_boundary(Ctx& c) {
  const int ticks = 1 << (c.ncl - 1);
  while (c.tick % ticks) {
    c.launch_tick((int)(c.tick % ticks), c.dtmin);
    c.tick++;
    c.time += c.dtmin;
  }
}

// The host plan of the uploaded mesh, built on first use and kept until the
// next upload; *o receives the reference operators it was built with.
const adg::MeshPlan& host_plan(Ctx& c, const adg::RefOps** o) {
  if (!c.has_mesh || !c.has_mat) adg::throw_err(ADG_E_STATE, "upload mesh and material first");
  if (!c.inited && c.host_ops.N != c.cfg.degree) c.host_ops = adg::make_ref_ops(c.cfg.degree);
  *o = c.inited ? &c.ops : &c.host_ops;
  if (!c.host_plan) {
    auto p = std::make_unique<adg::MeshPlan>();
    c.plan_mesh(**o, c.cfg.degree, *p);
    c.host_plan = std::move(p);
  }
  return *c.host_plan;
}

}  // namespace

extern "C" {

void adg_default_config(adg_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->degree = 5;
  cfg->precision = ADG_FP64;
  cfg->cfl = 0.35;
  cfg->gravity = 9.81;
  cfg->max_clusters = 1;
  cfg->ensemble = 1;
  cfg->device = 0;
  cfg->cuda_stream = nullptr;
}

int adg_create(const adg_config* cfg, adg_ctx** out) {
  if (!cfg || !out) return ADG_E_INVALID;
  *out = nullptr;
  if (cfg->degree < 1 || cfg->degree > 5 ||
      (cfg->precision != ADG_FP64 && cfg->precision != ADG_FP32 && cfg->precision != ADG_3XTF32) ||
      !(cfg->cfl > 0) || cfg->max_clusters < 1 || cfg->max_clusters > 16 || cfg->ensemble < 1 ||
      cfg->gravity < 0)
    return ADG_E_INVALID;
  adg_ctx* c = new (std::nothrow) adg_ctx();
  if (!c) return ADG_E_NOMEM;
  c->c.cfg = *cfg;
  *out = c;
  return ADG_OK;
}

int adg_upload_mesh(adg_ctx* ctx, int64_t nv, const double* xyz, int64_t nt, const int64_t* tet_v,
                    const int32_t* face_tag, const int64_t* face_partner) {
  if (!ctx) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    if (c.inited) adg::throw_err(ADG_E_STATE, "mesh is fixed after adg_init");
    if (nv < 4 || nt < 1 || !xyz || !tet_v || !face_tag || nt > (int64_t)1 << 30)
      adg::throw_err(ADG_E_INVALID, "bad mesh arguments");
    c.nv = nv;
    c.nt = nt;
    c.xyz.assign(xyz, xyz + 3 * nv);
    c.tets.assign(tet_v, tet_v + 4 * nt);
    c.tag.assign(face_tag, face_tag + 4 * nt);
    if (face_partner) c.partner.assign(face_partner, face_partner + 4 * nt);
    else c.partner.clear();
    c.has_mesh = true;
    c.host_plan.reset();
  });
}

int adg_upload_material(adg_ctx* ctx, const double* rho, const double* lambda, const double* mu) {
  if (!ctx) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    if (!c.has_mesh) adg::throw_err(ADG_E_STATE, "upload the mesh first");
    if (c.inited) adg::throw_err(ADG_E_STATE, "material is fixed after adg_init");
    if (!rho || !lambda || !mu) adg::throw_err(ADG_E_INVALID, "null material array");
    c.rho.assign(rho, rho + c.nt);
    c.lam.assign(lambda, lambda + c.nt);
    c.mu.assign(mu, mu + c.nt);
    c.has_mat = true;
    c.host_plan.reset();
  });
}

int adg_set_acoustic_ocean(adg_ctx* ctx, int enable) {
  if (!ctx) return ADG_E_INVALID;
  return guard(ctx, [&] {
    if (ctx->c.inited) adg::throw_err(ADG_E_STATE, "the ocean model is fixed at adg_init");
    ctx->c.acoustic = enable != 0;
  });
}

int adg_init(adg_ctx* ctx) {
  if (!ctx) return ADG_E_INVALID;
  return guard(ctx, [&] {
    if (ctx->c.inited) adg::throw_err(ADG_E_STATE, "already initialised");
    ctx->c.setup();
  });
}

int adg_plan(adg_ctx* ctx, double* dt_elem, int32_t* cluster, double* dt_min, int* n_clusters) {
  if (!ctx) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    const adg::RefOps* o;
    const adg::MeshPlan& p = host_plan(c, &o);
    if (dt_elem) std::copy(p.dte.begin(), p.dte.end(), dt_elem);
    if (cluster)
      for (int64_t e = 0; e < c.nt; ++e) cluster[e] = p.cl[e];
    if (dt_min) *dt_min = p.dtmin;
    if (n_clusters) *n_clusters = p.ncl;
  });
}

int adg_face_flux(adg_ctx* ctx, int64_t tet, int face, double* Fm, double* Fp) {
  if (!ctx) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    if (tet < 0 || tet >= c.nt || face < 0 || face > 3) adg::throw_err(ADG_E_INVALID, "tet or face out of range");
    const adg::RefOps* o;
    c.face_flux(host_plan(c, &o), tet, face, Fm, Fp);
  });
}

int adg_face_neighbour(adg_ctx* ctx, int64_t tet, int face, int64_t* nb_tet, int* nb_face, int32_t* node_map) {
  if (!ctx) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    if (tet < 0 || tet >= c.nt || face < 0 || face > 3) adg::throw_err(ADG_E_INVALID, "tet or face out of range");
    const adg::RefOps* o;
    const adg::MeshPlan& p = host_plan(c, &o);
    c.face_neighbour(p, *o, tet, face, nb_tet, nb_face, node_map);
  });
}

int adg_query(const adg_ctx* ctx, adg_info* out) {
  if (!ctx || !out) return ADG_E_INVALID;
  const Ctx& c = ctx->c;
  if (!c.inited) return ADG_E_STATE;
  std::memset(out, 0, sizeof(*out));
  out->n_tets = c.nt;
  out->n_basis = c.B;
  out->n_face_nodes = c.Bf;
  out->n_clusters = c.ncl;
  for (int i = 0; i < c.ncl && i < 16; ++i) out->cluster_size[i] = c.cl_begin[i + 1] - c.cl_begin[i];
  out->dt_min = c.dtmin;
  out->macro_dt = c.dtmin * (double)(1 << (c.ncl - 1));
  out->time = c.time;
  out->n_gravity_faces = (int64_t)c.gfaces.size();
  out->n_fault_faces = c.n_fault_faces;
  int64_t upd = 0;
  for (int i = 0; i < c.ncl; ++i) upd += (c.cl_begin[i + 1] - c.cl_begin[i]) * ((int64_t)1 << (c.ncl - 1 - i));
  out->updates_per_macro = upd * c.S;
  out->device_bytes = c.dev_bytes;
  int64_t utc = 0;
  for (int i = 0; i < c.ncl && i < (int)c.cl_plain.size(); ++i) utc += c.cl_plain[i] * ((int64_t)1 << (c.ncl - 1 - i));
  out->tensor_core_updates_per_macro = utc * c.S;
  out->n_receivers = c.n_rec;
  int64_t ua = 0;
  for (int i = 0; i < c.ncl && i < (int)c.cl_fluid.size(); ++i) ua += c.cl_fluid[i] * ((int64_t)1 << (c.ncl - 1 - i));
  out->acoustic_updates_per_macro = ua * c.S;
  return ADG_OK;
}

int adg_set_dofs(adg_ctx* ctx, const double* Q) {
  if (!ctx || !Q) return ADG_E_INVALID;
  return guard(ctx, [&] {
    need_init(ctx->c);
    if (ctx->c.fp64) put_dofs<double>(ctx->c, Q);
    else put_dofs<float>(ctx->c, Q);
    ctx->c.project_fluid();
  });
}

int adg_get_dofs(adg_ctx* ctx, double* Q) {
  if (!ctx || !Q) return ADG_E_INVALID;
  return guard(ctx, [&] {
    need_init(ctx->c);
    if (ctx->c.fp64) take_dofs<double>(ctx->c, Q);
    else take_dofs<float>(ctx->c, Q);
  });
}

int adg_set_dofs_f32(adg_ctx* ctx, const float* Q) {
  if (!ctx || !Q) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    float* scratch = dofs_scratch(c);
    const int per = c.S * 9 * c.B;
    check_cuda(cudaMemcpyAsync(scratch, Q, (size_t)c.nt * per * sizeof(float), cudaMemcpyHostToDevice, c.stream),
               "dofs upload");
    check_cuda((cudaError_t)adg::launch_permute_dofs(c.fp64, 1, scratch, c.dQ, c.dOrder, c.nt, per, c.n_sms,
                                                      c.stream),
               "dofs upload");
    check_cuda(cudaStreamSynchronize(c.stream), "dofs upload");
    c.project_fluid();
  });
}

int adg_get_dofs_f32(adg_ctx* ctx, float* Q) {
  if (!ctx || !Q) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    float* scratch = dofs_scratch(c);
    const int per = c.S * 9 * c.B;
    check_cuda((cudaError_t)adg::launch_permute_dofs(c.fp64, 0, c.dQ, scratch, c.dOrder, c.nt, per, c.n_sms,
                                                      c.stream),
               "dofs download");
    check_cuda(cudaMemcpyAsync(Q, scratch, (size_t)c.nt * per * sizeof(float), cudaMemcpyDeviceToHost, c.stream),
               "dofs download");
    check_cuda(cudaStreamSynchronize(c.stream), "dofs download");
  });
}

// Pipelined transfers: an upload's host copy runs on its own stream into one
// of two staging buffers and is reordered into the dofs on the library
// stream; a download is reordered on the library stream into one of two
// other staging buffers and copied to the host on a second stream.  Events
// keep each staging buffer from being overwritten before its last reader is
// done, so a step's compute overlaps the later uploads and the earlier
// downloads, and neither copy stream waits for the reordering in between.
int adg_set_dofs_f32_async(adg_ctx* ctx, const float* Q) {
  if (!ctx || !Q) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    c.aio_setup();
    const int per = c.S * 9 * c.B;
    const size_t bytes = (size_t)c.nt * per * sizeof(float);
    const int b = (int)(c.aio.n_in & 1);
    // buffer b was last read by the reordering of the upload before the previous one
    check_cuda(cudaStreamWaitEvent(c.aio.in, c.aio.in_used[b], 0), "dofs upload");
    check_cuda(cudaMemcpyAsync(c.aio.dIn[b], Q, bytes, cudaMemcpyHostToDevice, c.aio.in), "dofs upload");
    check_cuda(cudaEventRecord(c.aio.in_copied[b], c.aio.in), "dofs upload");
    check_cuda(cudaStreamWaitEvent(c.stream, c.aio.in_copied[b], 0), "dofs upload");
    check_cuda((cudaError_t)adg::launch_permute_dofs(c.fp64, 1, c.aio.dIn[b], c.dQ, c.dOrder, c.nt, per, c.n_sms,
                                                      c.stream),
               "dofs upload");
    check_cuda(cudaEventRecord(c.aio.in_used[b], c.stream), "dofs upload");
    c.aio.n_in++;
    c.project_fluid(false);
  });
}

int adg_get_dofs_f32_async(adg_ctx* ctx, float* Q) {
  if (!ctx || !Q) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    c.aio_setup();
    const int per = c.S * 9 * c.B;
    const size_t bytes = (size_t)c.nt * per * sizeof(float);
    const int b = (int)(c.aio.n_out & 1);
    // buffer b was last read by the host copy of the download before the previous one
    check_cuda(cudaStreamWaitEvent(c.stream, c.aio.out_copied[b], 0), "dofs download");
    check_cuda((cudaError_t)adg::launch_permute_dofs(c.fp64, 0, c.dQ, c.aio.dOut[b], c.dOrder, c.nt, per, c.n_sms,
                                                      c.stream),
               "dofs download");
    check_cuda(cudaEventRecord(c.aio.out_made[b], c.stream), "dofs download");
    check_cuda(cudaStreamWaitEvent(c.aio.out, c.aio.out_made[b], 0), "dofs download");
    check_cuda(cudaMemcpyAsync(Q, c.aio.dOut[b], bytes, cudaMemcpyDeviceToHost, c.aio.out), "dofs download");
    check_cuda(cudaEventRecord(c.aio.out_copied[b], c.aio.out), "dofs download");
    c.aio.n_out++;
  });
}

int adg_advance_async(adg_ctx* ctx, int n_macro) {
  if (!ctx || n_macro < 0) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    run_ticks_to_boundary(c);
    for (int i = 0; i < n_macro; ++i) {
      c.run_macro(1.0);
      c.tick += 1 << (c.ncl - 1);
      c.record_after_macro();
    }
  });
}

int adg_hydrostatic_start(adg_ctx* ctx) {
  if (!ctx) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    const int64_t ngf = (int64_t)c.gfaces.size();
    if (!ngf) adg::throw_err(ADG_E_STATE, "no gravitational face: no sea surface to start from");
    const int N = c.N, Bf = c.Bf, B = c.B, S = c.S;
    // sea-surface height at the face nodes, [ngf][S][Bf]
    std::vector<double> eta((size_t)ngf * S * Bf);
    check_cuda(cudaMemcpyAsync(eta.data(), c.dEta, eta.size() * 8, cudaMemcpyDeviceToHost, c.stream), "eta");
    check_cuda(cudaStreamSynchronize(c.stream), "eta");
    // the P_N interpolant on a face: eta(chi) = sum_n eta_n L_n(chi) with
    // L(chi) = m(chi)^T Vinv, m the monomials chi1^a chi2^b (a + b <= N)
    std::vector<int> ma, mb;
    for (int a = 0; a <= N; ++a)
      for (int b = 0; b <= N - a; ++b) { ma.push_back(a); mb.push_back(b); }
    std::vector<double> V((size_t)Bf * Bf), Vinv((size_t)Bf * Bf, 0.0);
    for (int n = 0; n < Bf; ++n)
      for (int j = 0; j < Bf; ++j)
        V[n * Bf + j] = std::pow(c.ops.node_chi[2 * n], ma[j]) * std::pow(c.ops.node_chi[2 * n + 1], mb[j]);
    for (int n = 0; n < Bf; ++n) Vinv[n * Bf + n] = 1.0;
    for (int k = 0; k < Bf; ++k) {  // Gauss-Jordan with partial pivoting: Vinv = V^-1
      int piv = k;
      for (int r = k + 1; r < Bf; ++r)
        if (std::fabs(V[r * Bf + k]) > std::fabs(V[piv * Bf + k])) piv = r;
      for (int j = 0; j < Bf; ++j) {
        std::swap(V[k * Bf + j], V[piv * Bf + j]);
        std::swap(Vinv[k * Bf + j], Vinv[piv * Bf + j]);
      }
      const double d = V[k * Bf + k];
      for (int j = 0; j < Bf; ++j) { V[k * Bf + j] /= d; Vinv[k * Bf + j] /= d; }
      for (int r = 0; r < Bf; ++r) {
        if (r == k) continue;
        const double f = V[r * Bf + k];
        if (f == 0.0) continue;
        for (int j = 0; j < Bf; ++j) { V[r * Bf + j] -= f * V[k * Bf + j]; Vinv[r * Bf + j] -= f * Vinv[k * Bf + j]; }
      }
    }
    // the faces seen from above: x(chi) = a + chi1 e1 + chi2 e2 in (x, y), and
    // a uniform grid of cells listing the faces whose box meets them
    static const int kFV[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
    std::vector<double> tri((size_t)ngf * 6);
    double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
    for (int64_t k = 0; k < ngf; ++k) {
      const int64_t e = c.gfaces[k] / 4;
      const int f = (int)(c.gfaces[k] % 4);
      const double* A = &c.xyz[3 * c.tets[4 * e + kFV[f][0]]];
      const double* Bv = &c.xyz[3 * c.tets[4 * e + kFV[f][1]]];
      const double* Cv = &c.xyz[3 * c.tets[4 * e + kFV[f][2]]];
      double* t = &tri[6 * k];
      t[0] = A[0]; t[1] = A[1];
      t[2] = Bv[0] - A[0]; t[3] = Bv[1] - A[1];
      t[4] = Cv[0] - A[0]; t[5] = Cv[1] - A[1];
      for (const double* P : {A, Bv, Cv}) {
        x0 = std::min(x0, P[0]); x1 = std::max(x1, P[0]);
        y0 = std::min(y0, P[1]); y1 = std::max(y1, P[1]);
      }
    }
    const int G = std::max(1, (int)std::sqrt((double)ngf));
    const double hx = (x1 - x0) / G + 1e-300, hy = (y1 - y0) / G + 1e-300;
    auto cell = [&](double v, double lo, double h) { return std::min(G - 1, std::max(0, (int)((v - lo) / h))); };
    std::vector<std::vector<int64_t>> grid((size_t)G * G);
    for (int64_t k = 0; k < ngf; ++k) {
      const double* t = &tri[6 * k];
      const double bx0 = std::min({t[0], t[0] + t[2], t[0] + t[4]}), bx1 = std::max({t[0], t[0] + t[2], t[0] + t[4]});
      const double by0 = std::min({t[1], t[1] + t[3], t[1] + t[5]}), by1 = std::max({t[1], t[1] + t[3], t[1] + t[5]});
      for (int i = cell(bx0, x0, hx); i <= cell(bx1, x0, hx); ++i)
        for (int j = cell(by0, y0, hy); j <= cell(by1, y0, hy); ++j) grid[(size_t)i * G + j].push_back(k);
    }
    // fluid elements, quadrature, projection (sigma_ii = -rho g eta, the rest 0)
    std::vector<int64_t> fluid;
    for (int64_t e = 0; e < c.nt; ++e)
      if (c.mu[e] == 0.0) fluid.push_back(e);
    if (fluid.empty()) return;
    std::vector<double> pts, w;
    adg::tet_rule(2 * N + 4, pts, w);
    const int nq = (int)w.size();
    std::vector<double> phi((size_t)nq * B);
    for (int q = 0; q < nq; ++q) adg::eval_basis(c.ops, &pts[3 * q], &phi[(size_t)q * B]);
    const int per = S * 9 * B;
    const int64_t nf = (int64_t)fluid.size();
    std::vector<double> out((size_t)nf * per, 0.0);
    int missing = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : missing)
    for (int64_t i = 0; i < nf; ++i) {
      const int64_t e = fluid[i];
      const double* P0 = &c.xyz[3 * c.tets[4 * e]];
      std::vector<double> coef((size_t)S * B, 0.0), L(Bf), m(Bf), es(S);
      for (int q = 0; q < nq; ++q) {
        double x[3];
        for (int d = 0; d < 3; ++d) {
          x[d] = P0[d];
          for (int k = 0; k < 3; ++k) x[d] += (c.xyz[3 * c.tets[4 * e + k + 1] + d] - P0[d]) * pts[3 * q + k];
        }
        // the face above: largest smallest barycentric coordinate among the cell's faces
        int64_t best = -1;
        double bmin = -1e-9, b1 = 0, b2 = 0;
        for (int64_t k : grid[(size_t)cell(x[0], x0, hx) * G + cell(x[1], y0, hy)]) {
          const double* t = &tri[6 * k];
          const double det = t[2] * t[5] - t[3] * t[4];
          const double px = x[0] - t[0], py = x[1] - t[1];
          const double c1 = (px * t[5] - py * t[4]) / det, c2 = (t[2] * py - t[3] * px) / det;
          const double mn = std::min(std::min(c1, c2), 1.0 - c1 - c2);
          if (mn > bmin) { bmin = mn; best = k; b1 = c1; b2 = c2; }
        }
        if (best < 0) { ++missing; continue; }
        for (int j = 0; j < Bf; ++j) m[j] = std::pow(b1, ma[j]) * std::pow(b2, mb[j]);
        for (int n = 0; n < Bf; ++n) {
          double v = 0.0;
          for (int j = 0; j < Bf; ++j) v += m[j] * Vinv[j * Bf + n];
          L[n] = v;
        }
        for (int s = 0; s < S; ++s) {
          const double* et = &eta[((size_t)best * S + s) * Bf];
          double v = 0.0;
          for (int n = 0; n < Bf; ++n) v += et[n] * L[n];
          es[s] = w[q] * c.rho[e] * c.cfg.gravity * v;
        }
        for (int s = 0; s < S; ++s)
          for (int l = 0; l < B; ++l) coef[(size_t)s * B + l] += es[s] * phi[(size_t)q * B + l];
      }
      for (int s = 0; s < S; ++s)
        for (int p = 0; p < 3; ++p)
          for (int l = 0; l < B; ++l) out[(size_t)i * per + ((size_t)s * 9 + p) * B + l] = -coef[(size_t)s * B + l];
    }
    if (missing) adg::throw_err(ADG_E_MESH, "hydrostatic start: fluid points outside the sea surface seen from above");
    // overwrite the fluid elements' dofs on the device
    const size_t ts = c.fp64 ? 8 : 4;
    std::vector<int64_t> idx((size_t)nf);
    for (int64_t i = 0; i < nf; ++i) idx[i] = c.inv[fluid[i]];
    std::vector<float> out32;
    const void* src = out.data();
    if (!c.fp64) {
      out32.resize(out.size());
      for (size_t k = 0; k < out.size(); ++k) out32[k] = (float)out[k];
      src = out32.data();
    }
    void* d = nullptr;
    check_cuda(cudaMalloc(&d, (size_t)nf * 8 + out.size() * ts), "hydrostatic start");
    int64_t* dIdx = static_cast<int64_t*>(d);
    void* dIn = static_cast<char*>(d) + (size_t)nf * 8;
    cudaError_t err = cudaMemcpyAsync(dIdx, idx.data(), (size_t)nf * 8, cudaMemcpyHostToDevice, c.stream);
    if (err == cudaSuccess) err = cudaMemcpyAsync(dIn, src, out.size() * ts, cudaMemcpyHostToDevice, c.stream);
    if (err == cudaSuccess) err = (cudaError_t)adg::launch_scatter_dofs(c.fp64, dIn, dIdx, nf, per, c.dQ, c.stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(c.stream);
    cudaFree(d);
    check_cuda(err, "hydrostatic start");
  });
}

int adg_get_dofs_subset(adg_ctx* ctx, int64_t n, const int64_t* tets, double* Q) {
  if (!ctx || n < 0 || (n && (!tets || !Q))) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    if (!n) return;
    std::vector<int64_t> idx((size_t)n);
    for (int64_t k = 0; k < n; ++k) {
      if (tets[k] < 0 || tets[k] >= c.nt) adg::throw_err(ADG_E_INVALID, "tet index out of range");
      idx[k] = c.inv[tets[k]];
    }
    const int per = c.S * 9 * c.B;
    const size_t ts = c.fp64 ? 8 : 4;
    void* d = nullptr;
    check_cuda(cudaMalloc(&d, (size_t)n * 8 + (size_t)n * per * ts), "dofs subset");
    int64_t* dIdx = static_cast<int64_t*>(d);
    void* dOut = static_cast<char*>(d) + (size_t)n * 8;
    std::vector<char> h((size_t)n * per * ts);
    cudaError_t e = cudaMemcpyAsync(dIdx, idx.data(), (size_t)n * 8, cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) e = (cudaError_t)adg::launch_gather_dofs(c.fp64, c.dQ, dIdx, n, per, dOut, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), dOut, h.size(), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    cudaFree(d);
    check_cuda(e, "dofs subset");
    for (size_t k = 0; k < (size_t)n * per; ++k)
      Q[k] = c.fp64 ? reinterpret_cast<const double*>(h.data())[k] : (double)reinterpret_cast<const float*>(h.data())[k];
  });
}

int adg_initial_points(adg_ctx* ctx, int* n_pts, double* xyz) {
  if (!ctx || !n_pts) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    std::vector<double> pts, w;
    adg::tet_rule(2 * c.N + 4, pts, w);
    const int nq = (int)w.size();
    *n_pts = nq;
    if (!xyz) return;
    for (int64_t e = 0; e < c.nt; ++e) {
      const double* P0 = &c.xyz[3 * c.tets[4 * e]];
      for (int q = 0; q < nq; ++q)
        for (int d = 0; d < 3; ++d) {
          double x = P0[d];
          for (int k = 0; k < 3; ++k) x += (c.xyz[3 * c.tets[4 * e + k + 1] + d] - P0[d]) * pts[3 * q + k];
          xyz[((size_t)e * nq + q) * 3 + d] = x;
        }
    }
  });
}

int adg_set_initial_values(adg_ctx* ctx, const double* values) {
  if (!ctx || !values) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    std::vector<double> pts, w;
    adg::tet_rule(2 * c.N + 4, pts, w);
    const int nq = (int)w.size();
    std::vector<double> phi((size_t)nq * c.B);
    for (int q = 0; q < nq; ++q) adg::eval_basis(c.ops, &pts[3 * q], &phi[(size_t)q * c.B]);
    const int64_t per = (int64_t)c.S * 9 * c.B;
    std::vector<double> Q((size_t)(c.nt * per), 0.0);
    for (int64_t e = 0; e < c.nt; ++e)
      for (int s = 0; s < c.S; ++s) {
        const double* val = values + (((size_t)e * c.S + s) * nq) * 9;
        double* out = Q.data() + e * per + (int64_t)s * 9 * c.B;
        for (int q = 0; q < nq; ++q)
          for (int p = 0; p < 9; ++p) {
            const double v = w[q] * val[q * 9 + p];
            for (int l = 0; l < c.B; ++l) out[p * c.B + l] += v * phi[(size_t)q * c.B + l];
          }
      }
    if (c.fp64) put_dofs<double>(c, Q.data());
    else put_dofs<float>(c, Q.data());
    c.project_fluid();
  });
}

int adg_gravity_faces(adg_ctx* ctx, int64_t* elem_face, double* node_xyz) {
  if (!ctx) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    static const int fv[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
    for (size_t g = 0; g < c.gfaces.size(); ++g) {
      if (elem_face) elem_face[g] = c.gfaces[g];
      if (node_xyz) {
        const int64_t e = c.gfaces[g] / 4;
        const int f = (int)(c.gfaces[g] % 4);
        const double* A = &c.xyz[3 * c.tets[4 * e + fv[f][0]]];
        const double* Bv = &c.xyz[3 * c.tets[4 * e + fv[f][1]]];
        const double* C = &c.xyz[3 * c.tets[4 * e + fv[f][2]]];
        for (int n = 0; n < c.Bf; ++n) {
          const double c1 = c.ops.node_chi[2 * n], c2 = c.ops.node_chi[2 * n + 1];
          for (int d = 0; d < 3; ++d)
            node_xyz[((size_t)g * c.Bf + n) * 3 + d] = A[d] + c1 * (Bv[d] - A[d]) + c2 * (C[d] - A[d]);
        }
      }
    }
  });
}

int adg_set_eta(adg_ctx* ctx, const double* eta) {
  if (!ctx || !eta) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    const size_t n = c.gfaces.size() * (size_t)c.S * c.Bf;
    if (n) {
      check_cuda(cudaMemcpyAsync(c.dEta, eta, n * 8, cudaMemcpyHostToDevice, c.stream), "eta upload");
      check_cuda(cudaStreamSynchronize(c.stream), "eta upload");
    }
  });
}

int adg_read_ssh(adg_ctx* ctx, double* eta) {
  if (!ctx || !eta) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    const size_t n = c.gfaces.size() * (size_t)c.S * c.Bf;
    if (n) {
      check_cuda(cudaMemcpyAsync(eta, c.dEta, n * 8, cudaMemcpyDeviceToHost, c.stream), "eta download");
      check_cuda(cudaStreamSynchronize(c.stream), "eta download");
    }
  });
}

int adg_advance(adg_ctx* ctx, int n_macro) {
  if (!ctx || n_macro < 0) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    run_ticks_to_boundary(c);
    for (int i = 0; i < n_macro; ++i) {
      c.run_macro(1.0);
      c.tick += 1 << (c.ncl - 1);
      c.record_after_macro();
    }
    c.check_err();
  });
}

int adg_advance_to(adg_ctx* ctx, double t) {
  if (!ctx) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    run_ticks_to_boundary(c);
    const double macro = c.dtmin * (double)(1 << (c.ncl - 1));
    if (t < c.time - 1e-12 * macro) adg::throw_err(ADG_E_INVALID, "target time is in the past");
    while (c.time + macro <= t + 1e-12 * macro) {
      c.run_macro(1.0);
      c.tick += 1 << (c.ncl - 1);
      c.record_after_macro();
    }
    const double rest = t - c.time;
    if (rest > 1e-12 * macro) {
      c.run_macro(rest / macro);
      c.tick += 1 << (c.ncl - 1);
      c.time = t;
      c.record_after_macro();
    }
    c.time = t;
    c.check_err();
  });
}

int adg_step_tick(adg_ctx* ctx) {
  if (!ctx) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    const int ticks = 1 << (c.ncl - 1);
    c.launch_tick((int)(c.tick % ticks), c.dtmin);
    c.tick++;
    c.time += c.dtmin;
    c.check_err();
  });
}

int adg_step_cluster(adg_ctx* ctx, int cl) {
  if (!ctx) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    if (cl < 0 || cl >= c.ncl) adg::throw_err(ADG_E_INVALID, "no such cluster");
    const int ticks = 1 << (c.ncl - 1);
    do {
      c.launch_tick((int)(c.tick % ticks), c.dtmin);
      c.tick++;
      c.time += c.dtmin;
    } while (c.tick % (1 << cl));
    c.check_err();
  });
}

int adg_profile(adg_ctx* ctx, int n_macro, double* ms, int64_t* launches) {
  if (!ctx || n_macro < 1 || !ms || !launches) return ADG_E_INVALID;
  std::vector<Ctx::ProfEv> evs;
  int rc = guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    run_ticks_to_boundary(c);
    const int ticks = 1 << (c.ncl - 1);
    c.prof = &evs;
    try {
      for (int i = 0; i < n_macro; ++i)
        for (int s = 0; s < ticks; ++s) {
          c.launch_tick(s, c.dtmin);
          c.tick++;
          c.time += c.dtmin;
        }
    } catch (...) {
      c.prof = nullptr;
      throw;
    }
    c.prof = nullptr;
    check_cuda(cudaStreamSynchronize(c.stream), "profile");
    double tot[5] = {0, 0, 0, 0, 0};
    int64_t cnt[5] = {0, 0, 0, 0, 0}, nl[5] = {0, 0, 0, 0, 0};
    for (auto& e : evs) {
      float t = 0;
      check_cuda(cudaEventElapsedTime(&t, e.a, e.b), "profile events");
      tot[e.kind] += t;
      cnt[e.kind] += 1;
      nl[e.kind] += e.launches;
      if (e.m) {  // tensor-core launch of the phase, timed alone
        check_cuda(cudaEventElapsedTime(&t, e.a, e.m), "profile events");
        tot[3 + e.kind] += t;
        cnt[3 + e.kind] += 1;
        nl[3 + e.kind] += 1;
      }
    }
    for (int k = 0; k < 5; ++k) {
      ms[k] = cnt[k] ? tot[k] / cnt[k] : 0.0;
      launches[k] = nl[k];
    }
    c.check_err();
  });
  for (auto& e : evs) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
    if (e.m) cudaEventDestroy(e.m);
  }
  return rc;
}

int adg_sync(adg_ctx* ctx) {
  if (!ctx) return ADG_E_INVALID;
  return guard(ctx, [&] {
    need_init(ctx->c);
    ctx->c.aio_sync();  // the pipelined copies (their streams wait on the library stream where needed)
    ctx->c.check_err();
  });
}

int adg_add_receivers(adg_ctx* ctx, int64_t n, const double* xyz) {
  if (!ctx || n < 0 || (n && !xyz)) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    if (c.rec[ADG_RECORD_RECEIVERS].every)
      adg::throw_err(ADG_E_STATE, "receivers are being recorded: adg_record_stop first");
    std::vector<int64_t> elem((size_t)n, -1);
    std::vector<double> phi((size_t)n * c.B);
    for (int64_t r = 0; r < n; ++r) {
      const double* x = xyz + 3 * r;
      double best = -1e300;
      int64_t be = -1;
      double bxi[3] = {0, 0, 0};
      for (int64_t e = 0; e < c.nt; ++e) {
        const double* P[4];
        for (int k = 0; k < 4; ++k) P[k] = &c.xyz[3 * c.tets[4 * e + k]];
        double J[3][3];
        for (int d = 0; d < 3; ++d)
          for (int k = 0; k < 3; ++k) J[d][k] = P[k + 1][d] - P[0][d];
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        double b[3] = {x[0] - P[0][0], x[1] - P[0][1], x[2] - P[0][2]};
        double xi[3];
        for (int a = 0; a < 3; ++a) {  // Cramer
          double M[3][3];
          for (int d = 0; d < 3; ++d)
            for (int k = 0; k < 3; ++k) M[d][k] = (k == a) ? b[d] : J[d][k];
          xi[a] = (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                   M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                   M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0])) / det;
        }
        const double lmin = std::min(std::min(xi[0], xi[1]), std::min(xi[2], 1 - xi[0] - xi[1] - xi[2]));
        if (lmin > best) {
          best = lmin;
          be = e;
          bxi[0] = xi[0]; bxi[1] = xi[1]; bxi[2] = xi[2];
        }
      }
      if (best < -1e-9) adg::throw_err(ADG_E_INVALID, "receiver outside the mesh");
      elem[r] = c.inv[be];
      adg::eval_basis(c.ops, bxi, &phi[(size_t)r * c.B]);
    }
    for (void* p : {(void*)c.dRecElem, (void*)c.dRecPhi, (void*)c.dRecOut}) {
      if (!p) continue;
      cudaFree(p);
      for (auto& o : c.owned)
        if (o == p) o = nullptr;
    }
    c.n_rec = n;
    c.dRecElem = nullptr; c.dRecPhi = nullptr; c.dRecOut = nullptr;
    if (!n) return;
    check_cuda(cudaMalloc((void**)&c.dRecElem, n * 8), "receivers");
    c.owned.push_back(c.dRecElem);
    check_cuda(cudaMalloc((void**)&c.dRecPhi, n * c.B * 8), "receivers");
    c.owned.push_back(c.dRecPhi);
    check_cuda(cudaMalloc((void**)&c.dRecOut, n * c.S * 9 * 8), "receivers");
    c.owned.push_back(c.dRecOut);
    check_cuda(cudaMemcpy(c.dRecElem, elem.data(), n * 8, cudaMemcpyHostToDevice), "receivers");
    check_cuda(cudaMemcpy(c.dRecPhi, phi.data(), n * c.B * 8, cudaMemcpyHostToDevice), "receivers");
  });
}

int adg_read_receivers(adg_ctx* ctx, double* out) {
  if (!ctx || !out) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    if (!c.n_rec) return;
    int rc = adg::launch_receivers(c.fp64, c.B, c.dQ, c.S, c.n_rec, c.dRecElem, c.dRecPhi, c.dRecOut, c.stream);
    if (rc) adg::throw_err(ADG_E_CUDA, "receiver kernel");
    check_cuda(cudaMemcpyAsync(out, c.dRecOut, c.n_rec * c.S * 9 * 8, cudaMemcpyDeviceToHost, c.stream),
               "receiver download");
    check_cuda(cudaStreamSynchronize(c.stream), "receiver download");
  });
}

int adg_record_start(adg_ctx* ctx, int kind, int every, int64_t capacity) {
  if (!ctx || (kind != ADG_RECORD_RECEIVERS && kind != ADG_RECORD_SSH) || every < 1 || capacity < 1)
    return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    const size_t sample = kind == ADG_RECORD_RECEIVERS ? (size_t)c.n_rec * c.S * 9 : c.gfaces.size() * (size_t)c.S * c.Bf;
    if (!sample)
      adg::throw_err(ADG_E_INVALID, kind == ADG_RECORD_RECEIVERS ? "no receivers to record" : "no sea surface to record");
    c.record_free(kind);
    if (!c.rec_stream) check_cuda(cudaStreamCreateWithFlags(&c.rec_stream, cudaStreamNonBlocking), "record stream");
    Ctx::Recorder& r = c.rec[kind];
    r.sample = sample;
    r.cap = capacity;
    r.t.assign((size_t)capacity, 0.0);
    r.taken.assign((size_t)capacity, nullptr);
    r.copied.assign((size_t)capacity, nullptr);
    for (int64_t k = 0; k < capacity; ++k) {
      check_cuda(cudaEventCreateWithFlags(&r.taken[k], cudaEventDisableTiming), "record events");
      check_cuda(cudaEventCreateWithFlags(&r.copied[k], cudaEventDisableTiming), "record events");
    }
    const size_t bytes = (size_t)capacity * sample * 8;
    cudaError_t e = cudaMalloc((void**)&r.dRing, bytes);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&r.hRing, bytes, cudaHostAllocDefault);
    if (e != cudaSuccess) {
      c.record_free(kind);
      adg::throw_err(ADG_E_NOMEM, std::string("record rings: ") + cudaGetErrorString(e));
    }
    r.every = every;  // last: a failure above leaves the kind off
  });
}

int adg_record_read(adg_ctx* ctx, int kind, int64_t max_samples, double* t, double* data, int64_t* n_read,
                    int64_t* n_dropped) {
  if (!ctx || (kind != ADG_RECORD_RECEIVERS && kind != ADG_RECORD_SSH) || max_samples < 0 ||
      (max_samples > 0 && (!t || !data)))
    return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    Ctx::Recorder& r = c.rec[kind];
    if (!r.every) adg::throw_err(ADG_E_STATE, "this kind is not being recorded");
    const int64_t n = std::min(max_samples, r.count - r.read);
    for (int64_t i = 0; i < n; ++i) {
      const int64_t slot = (r.read + i) % r.cap;
      check_cuda(cudaEventSynchronize(r.copied[slot]), "record copy");
      std::memcpy(data + i * r.sample, r.hRing + slot * r.sample, r.sample * 8);
      t[i] = r.t[slot];
    }
    r.read += n;
    if (n_read) *n_read = n;
    if (n_dropped) *n_dropped = r.dropped;
  });
}

int adg_record_stop(adg_ctx* ctx, int kind) {
  if (!ctx || (kind != ADG_RECORD_RECEIVERS && kind != ADG_RECORD_SSH)) return ADG_E_INVALID;
  return guard(ctx, [&] { ctx->c.record_free(kind); });
}

int adg_save_state(adg_ctx* ctx, void* buf, size_t* len) {
  if (!ctx || !len) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    const int ticks = 1 << (c.ncl - 1);
    if (c.tick % ticks) adg::throw_err(ADG_E_STATE, "save only at a macro-step boundary");
    const size_t qb = (size_t)c.nt * c.S * 9 * c.B * (c.fp64 ? 8 : 4);
    const size_t eb = c.gfaces.size() * (size_t)c.S * c.Bf * 8;
    const size_t fb = c.fault_set ? (size_t)c.nff * c.S * c.Bf * adg::FSTATE * 8 : 0;
    const size_t need = kStateHeader + qb + eb + fb;
    if (!buf) { *len = need; return; }
    if (*len < need) adg::throw_err(ADG_E_INVALID, "buffer too small");
    char* p = (char*)buf;
    int64_t hdr[10] = {0x41444732, c.N, c.S, c.nt, c.fp64, (int64_t)c.gfaces.size(), c.tick, (int64_t)fb, 0, 0};
    std::memcpy(&hdr[8], &c.time, 8);
    std::memcpy(p, hdr, sizeof(hdr));
    char* body = p + kStateHeader;
    check_cuda(cudaStreamSynchronize(c.stream), "save");
    check_cuda(cudaMemcpy(body, c.dQ, qb, cudaMemcpyDeviceToHost), "save dofs");
    if (eb) check_cuda(cudaMemcpy(body + qb, c.dEta, eb, cudaMemcpyDeviceToHost), "save eta");
    if (fb) check_cuda(cudaMemcpy(body + qb + eb, c.dFstate, fb, cudaMemcpyDeviceToHost), "save fault state");
    *len = need;
  });
}

int adg_load_state(adg_ctx* ctx, const void* buf, size_t len) {
  if (!ctx || !buf) return ADG_E_INVALID;
  return guard(ctx, [&] {
    Ctx& c = ctx->c;
    need_init(c);
    const char* p = (const char*)buf;
    int64_t hdr[10];
    if (len < kStateHeader) adg::throw_err(ADG_E_INVALID, "state too short");
    std::memcpy(hdr, p, sizeof(hdr));
    const size_t qb = (size_t)c.nt * c.S * 9 * c.B * (c.fp64 ? 8 : 4);
    const size_t eb = c.gfaces.size() * (size_t)c.S * c.Bf * 8;
    const size_t fb = (size_t)hdr[7];
    const size_t fb_ctx = (size_t)c.nff * c.S * c.Bf * adg::FSTATE * 8;
    if (hdr[0] != 0x41444732 || hdr[1] != c.N || hdr[2] != c.S || hdr[3] != c.nt || hdr[4] != (int64_t)c.fp64 ||
        hdr[5] != (int64_t)c.gfaces.size() || (fb && fb != fb_ctx) || len < kStateHeader + qb + eb + fb)
      adg::throw_err(ADG_E_INVALID, "state does not match this context");
    const char* body = p + kStateHeader;
    check_cuda(cudaStreamSynchronize(c.stream), "load");
    check_cuda(cudaMemcpy(c.dQ, body, qb, cudaMemcpyHostToDevice), "load dofs");
    c.project_fluid();
    if (eb) check_cuda(cudaMemcpy(c.dEta, body + qb, eb, cudaMemcpyHostToDevice), "load eta");
    if (fb) {
      if (!c.fault_set) adg::throw_err(ADG_E_STATE, "set the fault parameters before loading a fault state");
      check_cuda(cudaMemcpy(c.dFstate, body + qb + eb, fb, cudaMemcpyHostToDevice), "load fault state");
    }
    c.tick = hdr[6];
    std::memcpy(&c.time, &hdr[8], 8);
  });
}

int adg_reference_operators(int degree, double* kt, double* kvol, double* efc, double* lift) {
  try {
    adg::RefOps o = adg::make_ref_ops(degree);
    if (kt) std::memcpy(kt, o.kt.data(), o.kt.size() * 8);
    if (kvol) std::memcpy(kvol, o.kvol.data(), o.kvol.size() * 8);
    if (efc) std::memcpy(efc, o.efc.data(), o.efc.size() * 8);
    if (lift) std::memcpy(lift, o.lift.data(), o.lift.size() * 8);
    return ADG_OK;
  } catch (...) {
    return ADG_E_INVALID;
  }
}

const char* adg_last_error(const adg_ctx* ctx) { return ctx ? ctx->c.last_error.c_str() : "null context"; }

void adg_destroy(adg_ctx* ctx) { delete ctx; }

}  // extern "C"

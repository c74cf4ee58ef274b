/*
 * adg.h - C ABI of the GB300 ADER-DG solver for the fully coupled
 * elastic (Earth) / acoustic (ocean) wave equation with a gravitational free
 * surface, local time stepping and dynamic rupture, after Krenz et al.,
 * "3D Acoustic-Elastic Coupling with Gravity: The Dynamics of the 2018 Palu,
 * Sulawesi Earthquake and Tsunami" (SC'21).
 *
 * Conventions shared by every entry point
 *  - Return value: ADG_OK (0) or a negative ADG_E_* code; adg_last_error()
 *    gives a message.  No exception or abort crosses the ABI.
 *  - Pointers are HOST pointers unless the name says otherwise; they are
 *    borrowed for the duration of the call only.  The library owns every
 *    device allocation it makes (cudaMalloc) and frees it in adg_destroy().
 *  - A context is used by one host thread at a time.
 *  - Quantities q = (s_xx, s_yy, s_zz, s_xy, s_yz, s_xz, v_x, v_y, v_z):
 *    stress (positive in tension) and particle velocity (Sec. 3,
 *    Eq. elasticity-pde).  The ocean is the acoustic special case mu = 0,
 *    lambda = K, s_ij = -p delta_ij (Sec. 4.1).
 *  - Mesh: tetrahedra with 4 vertex indices each, positively oriented
 *    (det[v1-v0, v2-v0, v3-v0] > 0); local face f is the face opposite local
 *    vertex f; its vertices in increasing local order (a, b, c) parametrise it
 *    as x(chi) = xa + chi1 (xb - xa) + chi2 (xc - xa).
 *  - Dofs: modal coefficients of the orthonormal Dubiner basis on the
 *    reference tet (0,0,0),(1,0,0),(0,1,0),(0,0,1), ordered by total degree,
 *    then i, then j of the product index (i, j, k); B = (N+1)(N+2)(N+3)/6
 *    (Sec. 4.1).  Array layout Q[tet][scenario][quantity][basis], double.
 *  - Face nodes (sea-surface height, fault output): the (N+1)(N+2)/2
 *    equispaced points chi = (i1/N, i2/N), i2 outer loop, i1 inner loop.
 */
#ifndef ADG_H
#define ADG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ADG_OK 0
#define ADG_E_INVALID (-1)   /* bad argument or size                          */
#define ADG_E_MESH (-2)      /* inverted tet, non-matching or unpaired faces  */
#define ADG_E_STATE (-3)     /* call out of order (e.g. step before init)     */
#define ADG_E_CUDA (-4)      /* CUDA runtime error                            */
#define ADG_E_NOMEM (-5)     /* device or host allocation failed              */
#define ADG_E_NAN (-6)       /* non-finite value detected in the dofs         */
#define ADG_E_NEWTON (-7)    /* friction Newton solve did not converge        */
#define ADG_E_TIMEOUT (-8)   /* a bounded device wait ran out                 */
#define ADG_E_NOT_READY (-9) /* dependencies of a cluster step are not met    */

#define ADG_FP64 0
#define ADG_FP32 1
/* FP32 dofs; at degrees 5 and 4 the reference-matrix products (predictor,
 * face traces, volume term, lift) of every element without a fault face or
 * two or more gravitational faces run on the tensor cores (tcgen05) as 3xTF32
 * split products with FP32 accumulation (elements at LTS cluster borders and
 * with one gravitational face included), everything else as in ADG_FP32;
 * the sea-surface series, LTS buffers and friction stay FP64; other degrees
 * behave as ADG_FP32. */
#define ADG_3XTF32 2

/* Face tags (per tet and local face). */
#define ADG_TAG_INTERIOR 0  /* matched with the face sharing its three vertices  */
#define ADG_TAG_FREE 1      /* traction-free surface                            */
#define ADG_TAG_GRAVITY 2   /* gravitational free surface p = rho g eta (Sec. 3) */
#define ADG_TAG_ABSORB 3    /* outgoing-only: ghost state q+ = 0                */
#define ADG_TAG_PERIODIC 4  /* paired with face_partner                         */
#define ADG_TAG_FAULT 5     /* dynamic-rupture fault (both sides tagged)        */
#define ADG_TAG_RIGID 6     /* rigid free-slip wall: u_n = 0                    */

typedef struct adg_ctx adg_ctx;

typedef struct adg_config {
  int degree;        /* polynomial degree N in [1, 5]; 5 = order 6 (Sec. 6)       */
  int precision;     /* ADG_FP64, ADG_FP32 or ADG_3XTF32: storage and arithmetic of the dofs;
                        eta/H, LTS buffers and friction stay FP64                 */
  double cfl;        /* C in dt = C/(2N+1) h / c_p, h = insphere diameter (Sec. 4.4) */
  double gravity;    /* g in p = rho g eta; 9.81 in the paper (Sec. 3)            */
  int max_clusters;  /* rate-2 LTS clusters (Sec. 4.4); 1 = global time stepping */
  int ensemble;      /* S >= 1 independent scenarios sharing mesh and material    */
  int device;        /* CUDA device ordinal                                       */
  void* cuda_stream; /* cudaStream_t to run on, or NULL for a library stream      */
} adg_config;

typedef struct adg_info {
  int64_t n_tets;
  int n_basis;         /* B */
  int n_face_nodes;    /* (N+1)(N+2)/2 */
  int n_clusters;      /* clusters actually used */
  int64_t cluster_size[16];
  double dt_min;       /* step of cluster 0 */
  double macro_dt;     /* 2^(n_clusters-1) dt_min */
  double time;         /* current simulated time */
  int64_t n_gravity_faces;
  int64_t n_fault_faces;
  int64_t updates_per_macro; /* element updates (x ensemble) per macro step */
  int64_t device_bytes;
  int64_t tensor_core_updates_per_macro; /* of those, by the tensor-core kernels (ADG_3XTF32, degree 5 or 4) */
  int64_t n_receivers;       /* from the last adg_add_receivers */
  int64_t acoustic_updates_per_macro; /* of the tensor-core ones, on the 4-quantity local kernel
                                         (adg_set_acoustic_ocean) */
} adg_info;

/* Default configuration: N=5, FP64, cfl 0.35 (Sec. 6), g 9.81, GTS, S=1. */
void adg_default_config(adg_config* cfg);

/* Create a context on cfg->device.  *out receives the context. */
int adg_create(const adg_config* cfg, adg_ctx** out);

/* Mesh upload (Sec. 4.1: conforming tetrahedral mesh).
 * xyz[3*nv] vertex coordinates; tet_v[4*nt] vertex indices;
 * face_tag[4*nt] ADG_TAG_* per local face; face_partner[4*nt] = t*4+f of the
 * paired face for ADG_TAG_PERIODIC faces (ignored otherwise) or NULL when no
 * face is periodic.  Validation (orientation, matching) happens in adg_init
 * and adg_plan. */
int adg_upload_mesh(adg_ctx* ctx, int64_t nv, const double* xyz, int64_t nt,
                    const int64_t* tet_v, const int32_t* face_tag, const int64_t* face_partner);

/* Element-wise constant material (Sec. 4.1): density, Lame lambda, mu (mu = 0: fluid). */
int adg_upload_material(adg_ctx* ctx, const double* rho, const double* lambda, const double* mu);

/* Geometry, CFL time steps, rate-2 clustering, Godunov flux matrices F-/F+
 * per face (Sec. 4.2, Eq. numerical-flux), device allocation.  Dofs start at 0. */
/* The ocean as the acoustic system (Sec. 4.1: the fluid is the elastic
 * system with mu = 0, its stress -p I).  Call before adg_init (else
 * ADG_E_STATE); enable = 0 restores the default.  With it:
 *  - the stress of every fluid element (mu = 0) is kept isotropic: each dofs
 *    upload (adg_set_dofs, adg_set_dofs_f32, adg_set_initial_values,
 *    adg_load_state) replaces it by sigma_xx = sigma_yy = sigma_zz = their mean,
 *    with no shear stress; the scheme keeps that form (the acoustic subspace
 *    is invariant), so the results equal those of the 9-quantity system on
 *    such data;
 *  - with the tensor-core kernels (ADG_3XTF32, degree 5 or 4), the fluid elements
 *    without gravitational face, fault face or LTS neighbour in another
 *    cluster take a 4-quantity (p, v) local kernel (the others the 9-quantity
 *    ones): 32 elements per 128-row
 *    tile, the acoustic star product, 4 of the 9 dofs rows read; their face
 *    traces are written in the usual 9-quantity layout.
 * Without it the fluid carries whatever stress the caller uploads (a
 * deviatoric part stays constant in a fluid but drives velocities). */
int adg_set_acoustic_ocean(adg_ctx* ctx, int enable);

int adg_init(adg_ctx* ctx);

/* Host-only plan of the uploaded mesh (no device needed): call after
 * adg_upload_mesh and adg_upload_material, before or after adg_init.  Gives
 * what adg_init derives from the mesh, in the caller's element order: the CFL
 * time step of every element, dt_e = cfl/(2N+1) h_e / c_p,e with h_e the
 * insphere diameter (Sec. 4.4), and its rate-2 cluster c_e (Sec. 4.4): the
 * largest c with 2^c dt_min <= dt_e, at most max_clusters - 1, face neighbours
 * at most one cluster apart and both sides of a fault face in one cluster.
 * The element steps 2^c_e dt_min; a macro step is 2^(n_clusters-1) dt_min.
 * dt_elem[nt] (seconds), cluster[nt], dt_min[1], n_clusters[1]: caller-owned
 * outputs, each may be NULL.  Errors: ADG_E_STATE before both uploads;
 * ADG_E_MESH for the mesh faults adg_init reports (an inverted tet, a vertex
 * index or face tag out of range, an interior face without its neighbour, a
 * fault tagged on one side only, a bad periodic partner); ADG_E_INVALID for a
 * bad material (rho <= 0, mu < 0, c_p not positive).  Nothing is written on
 * error.  The plan (and, before adg_init, the reference operators) is kept
 * in the context for adg_face_flux and adg_face_neighbour until the next
 * upload. */
int adg_plan(adg_ctx* ctx, double* dt_elem, int32_t* cluster, double* dt_min, int* n_clusters);

/* Host-only: the Godunov flux matrices adg_init builds for local face `face`
 * of user tet `tet` (Sec. 4.2, Eq. numerical-flux), global frame, row-major
 * 9x9, caller-owned Fm[81], Fp[81] (either may be NULL).  The flux T A^- w^b
 * through the face is Fm q^- + Fp q^+ for interior and periodic faces (q^+ the
 * neighbour's state at the same point) and Fm q^- for free-surface, rigid-wall
 * and absorbing faces (Fp zero); both are zero for gravitational and fault
 * faces, whose fluxes come from the (eta, H) ODE and the friction solve.  The
 * element update subtracts 2|S_f|/|J| times the face integral of the flux
 * against the basis.  No device needed; call after both uploads.  Errors:
 * ADG_E_INVALID for tet or face out of range; otherwise as adg_plan. */
int adg_face_flux(adg_ctx* ctx, int64_t tet, int face, double* Fm, double* Fp);

/* Host-only: local face `face` of user tet `tet` as its neighbour sees it
 * (interior, periodic and fault faces): *nb_tet, *nb_face = the neighbour tet
 * and its local face (-1, -1 for a face without neighbour), and
 * node_map[Bf] = for each face node n (equispaced, see above) the
 * neighbour's face node at the same physical point (for periodic faces:
 * after the translation between the two faces).  This is the re-orientation
 * the neighbour flux applies to the neighbour's trace (Sec. 4.2).  Outputs
 * caller-owned, each may be NULL; node_map is left untouched without a
 * neighbour.  No device needed.  Errors as adg_face_flux. */
int adg_face_neighbour(adg_ctx* ctx, int64_t tet, int face, int64_t* nb_tet, int* nb_face,
                       int32_t* node_map);

int adg_query(const adg_ctx* ctx, adg_info* out);

/* Dofs in user tet order, layout [nt][S][9][B] (host, double). */
int adg_set_dofs(adg_ctx* ctx, const double* Q);
int adg_get_dofs(adg_ctx* ctx, double* Q);
/* The same in FP32 host arrays, [nt][S][9][B] floats: one copy over the host
 * link (at full speed from pinned memory: cudaHostAlloc, cudaHostRegister or
 * a pinned torch tensor), the reordering to the library's element order and
 * the conversion to the dofs precision run on the device.  The trace array is
 * the device scratch, so these calls need a macro-step boundary (always the
 * case after adg_advance / adg_advance_to); ADG_E_STATE otherwise.  The host
 * array is borrowed for the call; both calls return after their copy. */
int adg_set_dofs_f32(adg_ctx* ctx, const float* Q);
int adg_get_dofs_f32(adg_ctx* ctx, float* Q);
/* Pipelined forms of the three calls above (host-transfer plumbing; the paper
 * has no counterpart): each enqueues its work and returns without waiting, so
 * that the host copies of one step overlap the compute of another.  Q, layout and precision as in adg_set_dofs_f32 /
 * adg_get_dofs_f32 (pinned host memory for an asynchronous copy).
 * - adg_set_dofs_f32_async: the host array is copied on the context's
 *   upload stream into a device staging buffer of its own, then reordered
 *   into the dofs on the library stream (after everything enqueued there
 *   before, before everything enqueued after).  The array is borrowed until
 *   adg_sync returns: the caller neither frees nor changes it before.
 * - adg_get_dofs_f32_async: the dofs as they stand after the work enqueued
 *   before are reordered into a second staging buffer on the library stream
 *   and copied to the host array on the download stream.  The array holds
 *   them once adg_sync has returned.
 * - adg_advance_async: adg_advance without waiting for the steps: device
 *   errors (ADG_E_NAN, ADG_E_NEWTON, ADG_E_TIMEOUT) are reported by the next
 *   adg_sync or synchronous call instead.
 * - adg_sync (declared below) waits for all of the context's enqueued work
 *   and copies, then reports device errors as adg_advance does.
 * The staging buffers (two per direction, transfer j using buffer j % 2:
 * 4 x nt x S x 9 x B floats of device memory) and the two copy streams are
 * created by the first pipelined call and released by adg_destroy.  Any call needs no macro-step boundary (the staging is not the
 * trace array).  Errors: ADG_E_INVALID for a NULL argument or n_macro < 0,
 * ADG_E_STATE before adg_init, ADG_E_CUDA for a failed enqueue or allocation. */
int adg_set_dofs_f32_async(adg_ctx* ctx, const float* Q);
int adg_get_dofs_f32_async(adg_ctx* ctx, float* Q);
int adg_advance_async(adg_ctx* ctx, int n_macro);
/* The dofs of n listed user tets (indices in [0, nt)), Q[n][S][9][B] double,
 * gathered on the device: a cheap look at a few elements of a large mesh, at
 * any point (also inside an LTS macro step, where the elements of a cluster
 * that has not finished its step hold their mid-step values).
 * ADG_E_INVALID for an index out of range. */
int adg_get_dofs_subset(adg_ctx* ctx, int64_t n, const int64_t* tets, double* Q);

/* Initial condition by projection: adg_initial_points returns, for every tet,
 * n_pts physical points (xyz[nt][n_pts][3]); the caller evaluates its field
 * there and passes values[nt][S][n_pts][9]; the library projects them onto
 * the basis with the matching quadrature weights (exact for degree 2N+4). */
int adg_initial_points(adg_ctx* ctx, int* n_pts, double* xyz /* may be NULL to query n_pts */);
int adg_set_initial_values(adg_ctx* ctx, const double* values);

/* Hydrostatic start of the ocean from the current sea-surface height (set by
 * adg_set_eta): every fluid tet (mu = 0) gets, in every scenario, the
 * projection of the state at rest with the pressure perturbation
 * p' = rho g eta(x, y), i.e. s_xx = s_yy = s_zz = -p', shear stresses and
 * velocity zero; eta(x, y) is the P_N interpolant of the gravitational face
 * whose horizontal projection contains (x, y).  The dofs of the solid tets
 * are left as they are.  ADG_E_STATE without gravitational faces, ADG_E_MESH
 * if a fluid point has no face above it. */
int adg_hydrostatic_start(adg_ctx* ctx);

/* Gravitational faces (tag 2) in increasing user (tet*4+face) order:
 * elem_face[n_gravity_faces]; node_xyz[n_gravity_faces][Bf][3] or NULL. */
int adg_gravity_faces(adg_ctx* ctx, int64_t* elem_face, double* node_xyz);
/* Sea-surface height eta at the face nodes: [n_gravity_faces][S][Bf] (Sec. 4.3). */
int adg_set_eta(adg_ctx* ctx, const double* eta);
int adg_read_ssh(adg_ctx* ctx, double* eta);

/* Time stepping (Sec. 4.4).  A macro step advances every cluster by
 * macro_dt = 2^(n_clusters-1) dt_min through the rate-2 tick schedule, as one
 * CUDA graph launch.  adg_advance(n) runs n macro steps; adg_advance_to(t)
 * runs whole macro steps and a final one with all cluster steps shortened
 * uniformly so that the time lands on t. */
int adg_advance(adg_ctx* ctx, int n_macro);
int adg_advance_to(adg_ctx* ctx, double t);
/* One rate-2 tick: predictors of the clusters whose step starts, then
 * correctors of the clusters whose step ends.  Ticks run in order; cluster
 * c is in step with the others after every 2^c ticks. */
int adg_step_tick(adg_ctx* ctx);
/* Run ticks until cluster c completes one more step. */
int adg_step_cluster(adg_ctx* ctx, int c);
/* Block until queued work is done, the copies of the pipelined transfers
 * included; reports device-side errors (NaN...). */
int adg_sync(adg_ctx* ctx);

/* Per-kernel timing for roofline reports: runs n_macro macro steps with
 * eager (non-graph) launches and a CUDA event pair around the work of every
 * kernel kind of a cluster on the library stream.  ms[k] = mean duration of
 * one such phase of kind k, launches[k] = number of kernel launches (arrays
 * of 5), k = 0 local (predictor, volume, traces; with ADG_3XTF32 at degree 5
 * or 4 tensor-core and CUDA-core launches), 1 neighbour flux,
 * 2 fault friction solve, 3 and 4 the tensor-core launch of the local and
 * of the neighbour phase alone (0 without one).  Advances the simulation
 * like adg_advance. */
int adg_profile(adg_ctx* ctx, int n_macro, double* ms, int64_t* launches);

/* Allocation-free global steps (the paper has no counterpart; this is a
 * service of this library).  For callers that must not allocate device
 * memory while they step - for example a plug-in whose host application owns
 * and budgets all device memory - this runs n_steps global time steps on the
 * caller's own dofs and allocates nothing: the face-trace scratch that the
 * step needs lives in a fixed 32 MiB static device array inside the library
 * (held by every GPU that loads the library until the process exits).
 *  - ctx: an initialised context with one cluster, ensemble 1 and no
 *    gravitational or fault faces (else ADG_E_INVALID); its tables are read,
 *    its own dofs are not touched.
 *  - d_Q: DEVICE pointer to the caller's dofs in the context's precision,
 *    layout [tet][9][B] in user tet order (for such contexts the internal
 *    order is the user order), updated in place.  Owned by the caller.
 *  - stream: cudaStream_t to launch on; NULL is CUDA's default (legacy)
 *    stream, as in any CUDA call, so work the caller enqueued on it (torch's
 *    default stream, handle 0) is ordered before these kernels.  The call
 *    only enqueues work (no synchronisation).
 *  - Arithmetic: the CUDA-core kernels in the context's precision.  In an
 *    ADG_3XTF32 context those are the FP32 kernels of ADG_FP32 (the
 *    tensor-core kernels stage through shared memory the library allocates
 *    with the context), so the result is the ADG_FP32 one: within 2e-5
 *    relative L2 of the FP64 solution after a few steps, not bit-equal to
 *    adg_advance of that context.
 *  - Meshes whose traces need more than the fixed maximum
 *    (n_tets * 4 * S_f * sizeof(precision) > 32 MiB, S_f = 9 Bf rounded up
 *    to a multiple of 4) are rejected with
 *    ADG_E_INVALID and a message naming both sizes.
 *  - The first call on a device looks up the array's device address with
 *    that device current; make that first call before any stream capture.
 *  - All calls share the array and it keeps the last call's contents
 *    (every trace is written before it is read); calls whose work overlaps
 *    on the GPU race on it.  Non-finite dofs are reported by the next
 *    adg_sync() on the context. */
int adg_step_noalloc(adg_ctx* ctx, void* d_Q, int n_steps, void* stream);

/* Autotuner of the launch shapes (the paper has no counterpart; a service
 * of this library).  The work of a step is fixed by the scheme; how it is cut
 * into launches is chosen per kernel kind by timing the candidates on this
 * context's own clusters with CUDA events (whole macro steps, per-phase
 * events as in adg_profile, after one untimed macro step):
 *   choice[0] / [1]: threads per element block of the CUDA-core local /
 *                    neighbour kernels, of {64, 128, 256};
 *   choice[2] / [3]: consecutive 12-element tiles one CTA slot of the
 *                    tensor-core local / neighbour kernel takes per sweep
 *                    (elements per CTA before it strides on), of {1, 2, 4};
 *   0 for a kernel kind this context does not launch.
 * ms (optional, [4][3]): mean milliseconds per macro step of that kernel kind
 * for each candidate (-1 where not timed).  reps >= 1 timed macro steps per
 * candidate.  The state the steps change (dofs, sea surface, fault state and
 * counters, error word, time) is copied aside on the device and restored, so
 * the solution is unchanged; the call allocates that copy.  Choices are
 * cached for the process by (degree, precision, ensemble, tet count rounded
 * to a power of two, clusters) and reused unless force != 0.  Call at a
 * macro-step boundary after adg_init (else ADG_E_STATE); results of later
 * steps are bit-identical for every choice.  ADG_E_INVALID for bad
 * arguments, ADG_E_CUDA / ADG_E_NOMEM on device errors. */
int adg_autotune(adg_ctx* ctx, int reps, int force, int* choice, double* ms);

/* Peak-rate probe of a GPU (a measurement aid for the roofline denominators;
 * the paper has no counterpart).  kind 0: tcgen05.mma kind::tf32 with FP32
 * accumulation (M = 128, N = 256, A in TMEM, B in shared memory, one CTA per
 * SM); kind 1: FP32 fused multiply-add on the CUDA cores; kind 2: FP64 fused
 * multiply-add.  Runs one untimed launch, then `reps` timed launches on a
 * stream of its own; *flops = floating-point operations of the timed
 * launches, *ms = their duration (CUDA events).  Allocates and frees a few
 * bytes of device memory.  ADG_E_INVALID for a bad kind, device or reps,
 * ADG_E_TIMEOUT if a bounded wait of the MMA loop ran out, ADG_E_CUDA on a
 * CUDA error. */
int adg_measure_peak(int kind, int device, int reps, double* flops, double* ms);

/* Receivers: physical points; readout of q at the current time (whole ticks
 * synchronised: at macro-step boundaries), out[n][S][9] (host, double). */
int adg_add_receivers(adg_ctx* ctx, int64_t n, const double* xyz);
int adg_read_receivers(adg_ctx* ctx, double* out);

/* ---- Recording at a cadence (receivers and sea-surface height) --------------
 * Output streams at fixed cadences while adg_advance / adg_advance_to run,
 * e.g. receivers every 0.01 s and the sea surface every 0.1 s (Sec. 6).  After
 * every `every`-th macro step of those calls the library takes a sample on
 * its stream, into a device ring of `capacity` samples:
 *   ADG_RECORD_RECEIVERS  the receivers as adg_read_receivers, [n_rec][S][9];
 *   ADG_RECORD_SSH        eta as adg_read_ssh, [n_gravity_faces][S][Bf].
 * A second stream copies each sample to a pinned host ring while the next
 * steps run (an event orders it after the sample, and the slot is not
 * rewritten before its copy is done).  Samples the caller has not read when
 * the ring wraps are overwritten and counted as dropped.
 * adg_record_start: (re)starts one kind with its cadence and capacity (>= 1);
 *   ADG_E_INVALID if there is nothing of that kind (no receivers, no
 *   gravitational faces).  Counting starts at the call.
 * adg_record_read: moves up to max_samples of the oldest unread samples to the
 *   caller: times t[k] (simulated time after the macro step) and data
 *   [k][sample]; *n_read = samples moved, *n_dropped = overwritten so far
 *   (either may be NULL).  Waits only for the copies of those samples.
 * adg_record_stop: ends one kind and frees its rings.
 * adg_add_receivers while receivers are being recorded: ADG_E_STATE. */
#define ADG_RECORD_RECEIVERS 0
#define ADG_RECORD_SSH 1
int adg_record_start(adg_ctx* ctx, int kind, int every, int64_t capacity);
int adg_record_read(adg_ctx* ctx, int kind, int64_t max_samples, double* t, double* data, int64_t* n_read,
                    int64_t* n_dropped);
int adg_record_stop(adg_ctx* ctx, int kind);

/* ---- Dynamic rupture (Sec. 3, Eq. bc-dynrup) --------------------------------
 * Faces tagged ADG_TAG_FAULT on both sides (solid-solid).  Each tet pair is one
 * fault face; its minus side is the tet with the lower user index and n is that
 * tet's outward normal.  The fault lives at the face nodes of the minus face
 * (equispaced, see above).  Friction (reading of the fast-velocity-weakening
 * law): f = a asinh(V/(2V0) e^{psi/a}), dpsi/dt = -(V/L)(psi - psi_ss(V)),
 * f_ss = f_w + (f0 - (b-a) ln(V/V0) - f_w)/(1 + (V/V_w)^8)^{1/8}; strength
 * S = max(0, -(sigma_n0 + sigma_n)); solved per node at N+1 Gauss time points
 * per step by Newton on ln|V| in FP64.
 *
 * adg_fault_faces: per fault face (library order, cluster-major) the user
 *   tet*4+face of both sides, node coordinates [nff][Bf][3] and n [nff][3];
 *   any pointer may be NULL.  n_fault_faces comes from adg_query.
 * adg_set_fault: per node and scenario parameters [nff][S][Bf][13] =
 *   a, b, L, f0, V0, f_w, V_w, sigma_n0 (tension positive), tau0 (3, global
 *   frame; its normal part is ignored), psi_init, V_init (> 0); required before
 *   the first step.  Resets slip and traction.
 * adg_read_fault: state [nff][S][Bf][8] = |V|, psi, slip (3), shear traction (3).
 * adg_fault_stats: friction solves and Newton iterations so far (reset if asked). */
int adg_fault_faces(adg_ctx* ctx, int64_t* minus_face, int64_t* plus_face, double* node_xyz, double* normal);
int adg_set_fault(adg_ctx* ctx, const double* par);

/* Friction law of the fault faces: ADG_FRICTION_RS (default, above) or
 * ADG_FRICTION_LSW, linear slip weakening (the Scenario-A fault of Sec. 5,
 * law of Andrews 1976): psi = slip path length, dpsi/dt = |V|,
 * f = mu_s - (mu_s - mu_d) min(psi/D_c, 1), strength tau_S = C + f S, and at
 * each time point |V| = max(0, Theta - tau_S)/eta_s in closed form (the same
 * time points and two passes as for rate and state; no Newton, no learned
 * start).  Its adg_set_fault parameters [13] are mu_s, mu_d, D_c (> 0),
 * cohesion C (>= 0), three unused slots, sigma_n0, tau0 (3), psi_init (>= 0),
 * V_init (>= 0), with mu_s >= mu_d >= 0.  Requires fault faces; clears the
 * parameters, so adg_set_fault follows it.  ADG_E_INVALID for another law. */
#define ADG_FRICTION_RS 0
#define ADG_FRICTION_LSW 1
int adg_set_friction_law(adg_ctx* ctx, int law);
int adg_read_fault(adg_ctx* ctx, double* state);
int adg_fault_stats(adg_ctx* ctx, int64_t* solves, int64_t* iterations, int reset);

/* ---- Learned Newton start for the friction solve ----------------------------
 * A 6-32-32-1 tanh network predicts the first-pass solution ln|V*| of every
 * friction solve as x_a + network, x_a the large-argument asymptote of asinh.
 * At the second and later time points of a step the first Newton pass starts
 * from the warm start ln|V_prev| moved by the change of that prediction since
 * the previous time point; at the first it starts from the warm start, and a
 * start that fails falls back to it.  Newton then converges to the same
 * tolerance as from the plain start, so only the iteration count changes.
 * adg_rupture_capture(capacity): start recording rows (6 features,
 *   ln|V*| - x_a) of every first-pass solve into a device buffer of that many
 *   rows (0 stops recording);
 *   *n_captured returns the rows recorded since the last start.
 * adg_mlp_train: fit the network to the recorded rows on the GPU (own forward,
 *   backward and Adam kernels); loss[2] = scaled MSE before / after.
 * adg_mlp_params: set (if set != NULL) / get the MLP_NPARAM = 1327 floats and
 *   enable (1) or disable (0) the guess (-1 keeps the current setting).
 * adg_mlp_gradient: the loss gradient for given parameters and rows (host
 *   arrays, rows [n][7]); grad receives the 1313 trainable entries. */
int adg_rupture_capture(adg_ctx* ctx, int64_t capacity, int64_t* n_captured);
int adg_mlp_train(adg_ctx* ctx, int epochs, int batch, double lr, int seed, double* loss);
int adg_mlp_params(adg_ctx* ctx, const float* set, float* get, int enable);
int adg_mlp_gradient(const float* params, int64_t n, const float* rows, float* grad, double* loss);

/* Checkpoint: dofs, eta, fault state and time at a macro-step boundary.
 * adg_save_state with buf == NULL returns the size in *len; a buffer smaller
 * than that is ADG_E_INVALID, a call inside a macro step ADG_E_STATE.
 * adg_load_state takes a buffer saved by a context with the same degree,
 * ensemble, tet count, precision and gravitational faces (else ADG_E_INVALID);
 * a fault state needs adg_set_fault first (else ADG_E_STATE).  The buffer is
 * a host array owned by the caller. */
int adg_save_state(adg_ctx* ctx, void* buf, size_t* len);
int adg_load_state(adg_ctx* ctx, const void* buf, size_t len);

/* Reference operators the library generated (for inspection and tests):
 * kt[3][B][B] = int phi_m dphi_l/dxi_a, kvol[3][B][B1] = int dphi_m/dxi_a phi_l,
 * efc[4][Bf][B] basis values at face nodes, lift[4][B][Bf]; any may be NULL. */
int adg_reference_operators(int degree, double* kt, double* kvol, double* efc, double* lift);

const char* adg_last_error(const adg_ctx* ctx);
void adg_destroy(adg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* ADG_H */

"""Benchmark: ADER-DG element-updates/s at order 6 (degree N=5).

Workload: the coupled ocean-crust box, 100 x 100 x 40 km, 80 x 80 hex columns
x 39 layers (2 km water in 4 layers over 35 crust layers), 1,497,600 tets,
gravitational free surface on top, absorbing elsewhere, seafloor v_z pulse
(sigma 5 km horizontally, 1 km vertically) plus seeded higher-mode noise.  One
step = one global time step of the whole element update (CK predictor,
volume, local flux with the gravity-face ODE, neighbour flux) for every tet,
i.e. one macro step of the C ABI, replayed as a CUDA graph.

`value` is the FP32 path (the fast form); the FP64 path is measured in the
same run (`fp64`).  Dofs (3 GB FP32 / 6 GB FP64) are far larger than L2
(129 MB), so no flush is needed between steps.  With --gpus N (torchrun),
every rank runs an independent replica with its own source position (weak
scaling, no collective on the data path).

--impl reference times the FP64 oracle (test infrastructure) as it stands on
the host cores, one bounded sample of the workload per step.
"""

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEG = 5
METRIC = "ADER-DG element-updates/s at order 6, FP32/batched vs FP64; % of roofline"
UNIT = "element-updates/s"
WORKLOAD = ("coupled ocean-crust box 100x100x40 km, 1,497,600 tets, degree 5, gravitational surface, "
            "acoustic ocean")


def flops_per_update(N):
    """Algorithmic flop count per element update (fixed counting convention)."""
    nb = lambda n: (n + 1) * (n + 2) * (n + 3) // 6 if n >= 0 else 0
    B, Bf = nb(N), (N + 1) * (N + 2) // 2
    pred = sum(54 * nb(N - k - 1) * nb(N - k) + 486 * nb(N - k - 1) for k in range(N)) + 18 * sum(
        nb(N - k) for k in range(N + 1))
    vol = 3 * (18 * B * nb(N - 1) + 162 * B)
    loc = 4 * (36 * Bf * B + 162 * Bf)
    nbf = loc + 72 * Bf * Bf
    total = pred + vol + loc + nbf
    # kernel split: the local kernel projects the time integral onto the 4
    # faces; the neighbour kernel does both flux products and the lift
    local = pred + vol + 4 * 18 * Bf * B
    # reference-matrix products the tensor-core local kernel runs as MMAs:
    # predictor levels 0..N-3, the volume term and the face traces
    tensor = sum(54 * nb(N - k - 1) * nb(N - k) for k in range(N - 2)) + 54 * B * nb(N - 1) + 72 * Bf * B
    return {"pred": pred, "vol": vol, "loc": loc, "nb": nbf, "local_kernel": local,
            "neighbour_kernel": total - local, "total": total, "local_tensor": tensor}


def bytes_per_update(N, w):
    """Algorithmic HBM bytes per element update and kernel: the local kernel
    reads and writes the dofs and writes 4 face traces; the neighbour kernel
    reads the own and the neighbours' traces and reads and writes the dofs.
    The tensor-core forms count what they move: face blocks padded to a
    multiple of 4 floats, the element parameters, and (neighbour) the four
    32-byte face records (normal, neighbour impedances, face code)."""
    B, Bf = (N + 1) * (N + 2) * (N + 3) // 6, (N + 1) * (N + 2) // 2
    FS = (9 * Bf + 3) // 4 * 4
    return {"local_kernel": (2 * 9 * B + 4 * 9 * Bf) * w, "neighbour_kernel": (2 * 9 * B + 8 * 9 * Bf) * w,
            "local_tc_kernel": (2 * 9 * B + 4 * FS + 16) * w,
            # acoustic element: reads its 4 (p, v) rows, writes the three normal-stress rows and v
            "local_tc_kernel_acoustic": ((4 + 6) * B + 4 * FS + 16) * w,
            "neighbour_tc_kernel": (2 * 9 * B + 8 * FS + 16) * w + 4 * 32}


# DRAM bytes (read + write) per element of the tensor-core kernels (elastic and
# acoustic local, neighbour), from the one-kernel ncu captures of the
# 374,400-tet box (profiles/tensor_core_kernels_box40.md); a launch's traffic
# is scaled from them by its elements of each kind
TC_DRAM_BYTES_PER_ELEMENT = {"local_tc_kernel": 6996.4, "local_tc_kernel_acoustic": 5649.0,
                             "neighbour_tc_kernel": 7701.7}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def unit_peaks():
    """The TF32 tensor, FP32 and FP64 rates this project measured on the GPU
    (profiles/peaks.md, written by `python -m paper_2107_06640_gb300.peaks`),
    or None."""
    from paper_2107_06640_gb300 import peaks as pk
    return pk.load()


def tf32x3_peak_tflops(peaks, units=None):
    """(peak, source) of a 3xTF32 split product: a third of the measured dense
    TF32 tcgen05 rate (a burst rate: the tensor-core launches are timed alone);
    without that measurement, the measured burst bf16 rate times the nominal
    tf32/bf16 ratio 1.1/2.25, divided by 3."""
    if units and units.get("tf32_tensor_tflops"):
        return units["tf32_tensor_tflops"] / 3.0, "measured tcgen05 kind::tf32 rate / 3 (profiles/peaks.md)"
    return peaks["bf16_tflops"] * (1.1 / 2.25) / 3.0, "measured burst bf16 x nominal 1.1/2.25 / 3"


def alu_peak_tflops(fp64, sm_mhz, units=None, sm_count=None):
    """(peak, source) of the CUDA-core kernels: the measured FP64 or FP32 FMA
    rate; without it, SMs x 128 FP32 lanes x 2 x clock, or the nominal
    1.25 TFLOP/s FP64 scaled to the clock."""
    key = "fp64_fma_tflops" if fp64 else "fp32_fma_tflops"
    if units and units.get(key):
        return units[key], f"measured {key} (profiles/peaks.md)"
    if fp64:
        return 1.25 * sm_mhz / 2070.0, "nominal 1.25 TFLOP/s FP64 at the sampled clock"
    return (sm_count or 152) * 128 * 2 * sm_mhz * 1e6 / 1e12, "derived: SMs x 128 FP32 lanes x 2 x clock"


# where the nvidia-smi clock samples of each timed region are written (--clock-dir)
CLOCK_DIR = [tempfile.gettempdir()]


class Ranks:
    """The ranks of one launch (torchrun's RANK / WORLD_SIZE): the barrier
    around a timed region and the maximum of a host number over the ranks
    (through `dist` on `device`; a single rank needs neither)."""

    def __init__(self, dist=None, world=1, device="cpu"):
        self.dist, self.world, self.device = dist, world, device

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def max(self, x):
        if self.world == 1:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units all ranks processed (each the same weak-scaling share) over the
    slowest rank's time."""
    return units_per_rank * world / seconds


class ClockSampler:
    def __init__(self, path):
        self.path = path
        self.p = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self, device):
        if self.p is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(device):
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_workload(seed, nxy=80):
    import numpy as np
    from synthetic.workloads import coupled_box, random_dofs, seafloor_pulse
    m, mat = coupled_box(nxy=nxy, L=100e3 * nxy / 80)
    rng = np.random.default_rng(seed)
    x0, y0 = rng.uniform(30e3, 70e3, 2)
    pulse = seafloor_pulse(x0, y0, m.extra["seafloor"])
    B = (N_DEG + 1) * (N_DEG + 2) * (N_DEG + 3) // 6
    # constant mode of the orthonormal basis is phi_0 = sqrt(6): the projection of
    # the pulse sampled at the centroid, plus small seeded noise in all modes
    Q = random_dofs((m.nt, 9, B), seed, decay=1.0, N=N_DEG) * 1e-4
    Q[:, :, 0] += pulse(m.centroids()) / np.sqrt(6.0)
    return m, mat, Q


def cpu_sample_run(seconds, steps=None):
    """Time the oracle on a bounded sample of the workload (in-process)."""
    import numpy as np
    from oracle.ader import Oracle
    from synthetic.workloads import coupled_box, random_dofs
    # a 6 x 6 hex-column piece of the same box: same spacing, materials, faces
    m, mat = coupled_box(nxy=6, n_water=4, n_crust=3, L=100e3 * 6 / 80, depth=2e3 + 3 * 38e3 / 35,
                         water=2e3)
    o = Oracle(m.xyz, m.tets, m.face_tag, m.face_partner, *mat, N_DEG, cfl=0.35)
    o.Q = random_dofs((m.nt, o.B, 9), 0, N=N_DEG) * 1e-3
    n = 0
    t0 = time.perf_counter()
    while True:
        o.step_gts()
        n += 1
        el = time.perf_counter() - t0
        if (steps is not None and n >= steps) or (steps is None and el >= seconds):
            break
    return m.nt * n / el, m.nt, n, el


def _oracle_procs(seconds, nproc):
    """nproc single-threaded oracle processes at once, each on its own copy of
    the sample piece; returns their [updates/s, tets, steps, seconds]."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import sys, json; sys.path.insert(0, %r); import bench; v, nt, n, el = bench.cpu_sample_run(%f); "
            "print(json.dumps([v, nt, n, el]))" % (ROOT, seconds))
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                           env=env) for _ in range(nproc)]
    out = []
    for p in ps:
        o, _ = p.communicate(timeout=900)
        out.append(json.loads(o.strip().splitlines()[-1]))
    return out


def cpu_baseline(seconds=12.0):
    """The oracle on the host: one process, and one single-threaded process per
    host core, each stepping its own copy of the sample piece (the element
    update needs no communication between independent pieces, so the summed
    rate is the oracle's throughput on all cores)."""
    v, nt, n, el = _oracle_procs(seconds, 1)[0]
    ncores = os.cpu_count() or 1
    runs = _oracle_procs(seconds, ncores)
    return {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{nt}-tet 6x6-column piece of the same box (N=5, FP64, numpy), {n} global steps in {el:.1f} s, single thread",
            "all_cores": {"value": sum(r[0] for r in runs), "unit": UNIT, "cores": ncores,
                          "sample": f"{ncores} single-threaded processes, each stepping its own copy of the piece for "
                                    f"about {seconds:.0f} s ({min(r[2] for r in runs)}-{max(r[2] for r in runs)} steps)"}}


def run_reference(args, rank):
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "bench.cpu_sample_run(0, steps=%d); v, nt, n, el = bench.cpu_sample_run(0, steps=%d); "
            "print(json.dumps([v, nt, n, el]))" % (ROOT, max(1, warm), steps))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    v, nt, n, el = json.loads(r.stdout.strip().splitlines()[-1])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": 1e3 * el / n, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (oracle: bounded sample per step)", "degree": N_DEG},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{nt}-tet piece of the box per step, single thread"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _timed_advance(s, steps, warm, stream, torch, tag):
    import numpy as np  # noqa: F401
    s.advance(warm)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(os.path.join(CLOCK_DIR[0], f"clocks_{tag}.csv")) as cs:
        ev0.record(stream)
        s.advance(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    return ev0.elapsed_time(ev1), cs.summary(torch.cuda.current_device())


def run_other_workload(args):
    """LTS, rupture and ensemble workloads: one JSON line each (single GPU)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2107_06640_gb300 as pkg
    from paper_2107_06640_gb300 import Solver, _lib
    from synthetic.workloads import (coupled_box, fault_box, lsw_fault_params, random_dofs, rs_fault_params,
                                     uplift_scenarios)
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    steps, warm = args.steps, args.warmup
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic", "warmup": warm}
    t_setup = time.perf_counter()
    if args.workload == "lts":
        L = 100e3
        bathy = lambda x, y: -2000.0 + 500.0 * np.sin(2 * np.pi * x / L) * np.sin(2 * np.pi * y / L)
        m, (rho, lam, mu) = coupled_box(nxy=200, bathy=bathy, grading=32.0)
        s = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=N_DEG, precision=pkg.ADG_3XTF32, cfl=0.35,
                   max_clusters=6, stream=stream.cuda_stream, acoustic_ocean=True)
        ef, nxyz = s.gravity_faces()
        s.set_eta(np.exp(-((nxyz[..., 0] - L / 2) ** 2 + (nxyz[..., 1] - L / 2) ** 2) / (2 * 8e3 ** 2))[:, None, :])
        info = s.info
        hist = [int(info.cluster_size[c]) for c in range(info.n_clusters)]
        upd = int(info.updates_per_macro)
        gts_upd = s.nt * (1 << (info.n_clusters - 1))
        line["config"] = {"workload": f"LTS-graded coupled box, sin bathymetry +-500 m, x/y grading 32x, "
                                      f"{s.nt} tets, degree 5", "n_tets": s.nt, "clusters": hist,
                          "lts_update_reduction": gts_upd / upd, "macro_dt": info.macro_dt,
                          "tensor_core_update_fraction": int(info.tensor_core_updates_per_macro) / upd}
        line["dtype"] = "f32 (3xTF32 tensor-core products)"
    elif args.workload in ("rupture", "rupture-lsw"):
        r = args.fault_scale
        m, (rho, lam, mu) = fault_box(nx=32 * r, ny=40 * r, nz=16 * r, dz=1e3 / r, dip_deg=15.0,
                                      ocean_layers=2 * r, water=2e3)
        s = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=4, precision=pkg.ADG_3XTF32, cfl=0.35,
                   max_clusters=1, stream=stream.cuda_stream, acoustic_ocean=True)
        nff = int(s.info.n_fault_faces)
        mf, pf, fxyz, fn = _lib.adg_fault_faces(s.ctx, nff, s.Bf)
        c = fxyz.reshape(-1, 3).mean(0)
        if args.workload == "rupture-lsw":
            _lib.adg_set_friction_law(s.ctx, _lib.ADG_FRICTION_LSW)
            par = lsw_fault_params(fxyz, fn, seed=0, patch_center=c, patch_radius=8e3, taper=10e3)
            law = "linear slip-weakening friction (cohesion rising toward the seafloor)"
        else:
            par = rs_fault_params(fxyz, fn, seed=0, patch_center=c, patch_radius=8e3)
            law = "rate-and-state fast-velocity-weakening friction"
        _lib.adg_set_fault(s.ctx, par[:, None])
        upd = int(s.info.updates_per_macro)
        line["config"] = {"workload": f"15-degree planar megathrust 150 x 60 km under 2 km ocean with gravity, "
                                      f"{law}, {s.nt} tets, degree 4, acoustic ocean",
                          "n_tets": s.nt, "fault_faces": nff, "fault_nodes": nff * s.Bf,
                          "tensor_core_update_fraction": int(s.info.tensor_core_updates_per_macro) / upd,
                          "acoustic_kernel_updates": int(s.info.acoustic_updates_per_macro)}
        line["dtype"] = "f32 (3xTF32 tensor-core products; friction f64)"
    elif args.workload == "ocean":
        # ocean-dominated coupled box (34 of 39 layers water, like the ocean share of the paper's mesh L),
        # acoustic ocean; the same box on the 9-quantity local kernel is timed below for comparison
        m, (rho, lam, mu) = coupled_box(nxy=80, n_water=34, n_crust=5, water=34e3)
        Q0 = random_dofs((m.nt, 9, 56), 0, N=N_DEG) * 1e-4
        mk = lambda ac: Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=N_DEG, precision=pkg.ADG_3XTF32,
                               cfl=0.35, stream=stream.cuda_stream, acoustic_ocean=ac)
        s = mk(True)
        s.set_dofs(Q0)
        s.set_eta(np.zeros((int(s.info.n_gravity_faces), 1, s.Bf)))
        upd = int(s.info.updates_per_macro)
        line["config"] = {"workload": f"ocean-dominated coupled box 100x100x40 km, 34 km water over 6 km crust, "
                                      f"{s.nt} tets ({int((mu == 0).sum())} fluid), degree 5, acoustic ocean",
                          "n_tets": s.nt, "fluid_tets": int((mu == 0).sum()),
                          "acoustic_kernel_updates": int(s.info.acoustic_updates_per_macro)}
        line["dtype"] = "f32 (3xTF32 tensor-core products)"
    elif args.workload == "record":
        m, (rho, lam, mu), Q0 = make_workload(seed=0, nxy=args.nxy)
        s = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=N_DEG, precision=pkg.ADG_3XTF32, cfl=0.35,
                   stream=stream.cuda_stream, acoustic_ocean=True)
        s.set_dofs(Q0)
        s.set_eta(np.zeros((int(s.info.n_gravity_faces), 1, s.Bf)))
        pick = np.random.default_rng(0).choice(m.nt, 1000, replace=False)
        s.add_receivers(m.xyz[m.tets[pick]].mean(1))
        upd = int(s.info.updates_per_macro)
        line["config"] = {"workload": f"coupled ocean-crust box, {s.nt} tets, degree 5, recording 1000 receivers "
                                      f"and the sea surface every macro step", "n_tets": s.nt}
        line["dtype"] = "f32 (3xTF32 tensor-core products)"
    else:
        S = 32
        m, (rho, lam, mu) = coupled_box(nxy=66)
        s = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=N_DEG, precision=pkg.ADG_3XTF32, cfl=0.35,
                   ensemble=S, stream=stream.cuda_stream, acoustic_ocean=True)
        ef, nxyz = s.gravity_faces()
        eta0 = np.stack([f(nxyz[..., 0], nxyz[..., 1]) for f in uplift_scenarios(S, seed=0)], axis=1)
        s.set_eta(eta0)
        t_hot = time.perf_counter()
        s.hydrostatic_start()  # the ocean at rest with p' = rho g eta0 under each scenario's surface
        t_hot = time.perf_counter() - t_hot
        upd = int(s.info.updates_per_macro)
        line["config"] = {"workload": f"ensemble of {S} sea-surface uplift scenarios (8 Gaussian bumps, 0.1-2 m) "
                                      f"with a hydrostatic start of the ocean, on a {s.nt}-tet coupled box, degree 5; "
                                      f"64 scenarios = 2 passes of {S}",
                          "n_tets": s.nt, "ensemble": S, "hydrostatic_start_s": t_hot}
        line["dtype"] = "f32 (3xTF32 tensor-core products)"
    t_setup = time.perf_counter() - t_setup
    ch, tms = _lib.adg_autotune(s.ctx, reps=1)
    line["autotune"] = {"choice": [int(x) for x in ch], "ms_per_candidate": tms.round(3).tolist()}
    ms, clk = _timed_advance(s, steps, warm, stream, torch, args.workload)
    line.update({"value": upd * steps / (ms * 1e-3), "steps": steps, "ms_per_step": ms / steps, "clocks": clk,
                 "setup_s": t_setup})
    kms, kcnt = _lib.adg_profile(s.ctx, 1)
    line["kernel_ms"] = {"local": kms[0], "neighbour": kms[1], "rupture": kms[2],
                         "launches_per_macro": [int(x) for x in kcnt[:3]]}
    line["gpu_launches"] = int(kcnt[:3].sum()) * steps
    import resource
    line["host_peak_rss_gb"] = resource.getrusage(resource.RUSAGE_SELF).ru_maxrss / 2 ** 20
    if args.workload == "record":
        # the same steps again while both kinds are recorded every macro step
        R, H = _lib.ADG_RECORD_RECEIVERS, _lib.ADG_RECORD_SSH
        s.record(R, 1, steps + warm)
        s.record(H, 1, steps + warm)
        ms_r, clk_r = _timed_advance(s, steps, warm, stream, torch, "record_on")
        tr, _, dr = s.read_record(R)
        th, _, dh = s.read_record(H)
        n_ssh = int(s.info.n_gravity_faces) * s.Bf
        line["recording"] = {"receivers": 1000, "ssh_values": n_ssh, "every_macro_steps": 1,
                             "bytes_per_step": (1000 * 9 + n_ssh) * 8,
                             "ms_per_step_without": ms / steps, "ms_per_step_with": ms_r / steps,
                             "overhead": ms_r / ms - 1.0, "samples": [len(tr), len(th)], "dropped": [dr, dh],
                             "clocks_with": clk_r}
        line["value"] = upd * steps / (ms_r * 1e-3)
        line["ms_per_step"] = ms_r / steps
    if args.workload == "ocean":
        # the same box, its fluid on the 9-quantity kernels (the ocean embedded in the elastic system)
        del s
        s9 = mk(False)
        s9.set_dofs(Q0)
        s9.set_eta(np.zeros((int(s9.info.n_gravity_faces), 1, s9.Bf)))
        _lib.adg_autotune(s9.ctx, reps=1)
        ms9, clk9 = _timed_advance(s9, steps, warm, stream, torch, "ocean9")
        kms9, _ = _lib.adg_profile(s9.ctx, 1)
        line["nine_quantity_ocean"] = {"value": upd * steps / (ms9 * 1e-3), "ms_per_step": ms9 / steps,
                                       "kernel_ms": {"local": kms9[0], "neighbour": kms9[1]}, "clocks": clk9}
    if args.workload == "rupture-lsw":
        st = _lib.adg_read_fault(s.ctx, np.empty((nff, 1, s.Bf, 8)))
        line["rupture"] = {"slipping_node_fraction": float(np.mean(st[..., 0] > 1e-3)),
                           "max_slip_rate": float(st[..., 0].max()), "max_slip_path": float(st[..., 1].max()),
                           "friction_kernel_ms": kms[2]}
    if args.workload == "rupture":
        solves, iters = _lib.adg_fault_stats(s.ctx, reset=True)
        # learned Newton start: capture, train on the GPU, rerun the same steps
        state = s.save_state()
        _lib.adg_rupture_capture(s.ctx, 1 << 22)
        s.advance(steps)
        ncap = _lib.adg_rupture_capture(s.ctx, 0)
        s0, i0 = _lib.adg_fault_stats(s.ctx, reset=True)
        loss = _lib.adg_mlp_train(s.ctx, epochs=30, batch=4096, lr=3e-3, seed=0)
        s.load_state(state)
        _lib.adg_mlp_params(s.ctx, enable=1)
        s.advance(steps)
        torch.cuda.synchronize()
        s1, i1 = _lib.adg_fault_stats(s.ctx, reset=True)
        kms_l, _ = _lib.adg_profile(s.ctx, 1)
        line["rupture"] = {"newton_iters_per_solve_plain": i0 / max(s0, 1),
                           "newton_iters_per_solve_learned": i1 / max(s1, 1), "training_solves": ncap,
                           "train_loss": [float(loss[0]), float(loss[1])], "solves_per_step": s0 / steps,
                           "friction_kernel_ms": kms[2], "friction_kernel_ms_learned": kms_l[2]}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--nxy", type=int, default=80,
                    help="hex columns per side (80: the 1.5 M-tet workload; smaller for profiling)")
    ap.add_argument("--only", default=None, choices=["fp64", "fp32", "3xtf32"],
                    help="profiling aid: run one precision of the coupled workload, print no JSON line")
    ap.add_argument("--degree", type=int, default=N_DEG,
                    help="profiling aid (with --only): the polynomial degree of that run")
    ap.add_argument("--workload", default="coupled",
                    choices=["coupled", "lts", "rupture", "rupture-lsw", "ensemble", "record", "ocean"],
                    help="coupled: the headline line; lts / rupture / rupture-lsw / ensemble / record / ocean: the "
                         "other workloads")
    ap.add_argument("--fault-scale", type=int, default=5,
                    help="megathrust refinement r: 32r x 40r x 18r hex columns (3: 3.73 M tets, 5: 17.3 M tets)")
    ap.add_argument("--clock-dir", default=None,
                    help="directory for the nvidia-smi clock samples of each timed region (default: the temp dir)")
    args = ap.parse_args()
    if args.clock_dir:
        os.makedirs(args.clock_dir, exist_ok=True)
        CLOCK_DIR[0] = args.clock_dir
    if args.workload != "coupled":
        run_other_workload(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    import paper_2107_06640_gb300 as pkg
    from paper_2107_06640_gb300 import Solver

    ranks = Ranks(dist, world, torch.device("cuda", local))

    def barrier():
        ranks.barrier()
        torch.cuda.synchronize()

    max_over_ranks = ranks.max

    m, (rho, lam, mu), Q0 = make_workload(seed=rank, nxy=args.nxy)
    stream = torch.cuda.current_stream()
    res = {}
    HEAD = pkg.ADG_3XTF32
    runs = ((pkg.ADG_FP64, args.fp64_steps, 1), (pkg.ADG_3XTF32, args.steps, args.warmup),
            (pkg.ADG_FP32, args.steps, args.warmup))
    if args.only:
        # profiling aid: one precision, a short run, no JSON line
        prec = {"fp64": pkg.ADG_FP64, "fp32": pkg.ADG_FP32, "3xtf32": pkg.ADG_3XTF32}[args.only]
        s = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=args.degree, precision=prec, cfl=0.35,
                   device=local, stream=stream.cuda_stream, acoustic_ocean=True)
        s.set_dofs(np.ascontiguousarray(Q0[:, :, :s.B]))  # (the hierarchical basis: a lower degree's leading modes)
        s.advance(args.warmup + args.steps)
        s.sync()
        print(f"profiling run: {args.only}, degree {args.degree}, {args.warmup + args.steps} steps", flush=True)
        return
    for prec, steps, warm in runs:
        s = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=N_DEG, precision=prec, cfl=0.35,
                   device=local, stream=stream.cuda_stream, acoustic_ocean=True)
        s.set_dofs(Q0)
        s.set_eta(np.zeros((int(s.info.n_gravity_faces), 1, s.Bf)))
        upd = int(s.info.updates_per_macro)
        tune = None
        if prec != pkg.ADG_FP64:  # launch shapes by the library's autotuner (FP64 keeps the defaults)
            ch, tms = pkg._lib.adg_autotune(s.ctx, reps=2)
            tune = {"choice": {"cc_local_threads": int(ch[0]), "cc_neighbour_threads": int(ch[1]),
                               "tc_local_tiles_per_sweep": int(ch[2]), "tc_neighbour_tiles_per_sweep": int(ch[3])},
                    "ms_per_candidate": tms.round(4).tolist(),
                    "candidates": [[64, 128, 256], [64, 128, 256], [1, 2, 4], [1, 2, 4]]}
        s.advance(warm)
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(os.path.join(CLOCK_DIR[0], f"clocks_r{rank}_{prec}.csv")) as cs:
            ev0.record(stream)
            s.advance(steps)
            ev1.record(stream)
            barrier()
        ms = max_over_ranks(ev0.elapsed_time(ev1))
        # per-kernel durations (CUDA events on the library stream)
        kms, kcnt = pkg._lib.adg_profile(s.ctx, 2)
        res[prec] = dict(solver=s, ms=ms, steps=steps, upd=upd, kms=kms, kcnt=kcnt, tune=tune,
                         clocks=cs.summary(local), launches=int(kcnt[:3].sum() // 2),
                         advanced=warm + steps + 2)
        if prec not in (HEAD, pkg.ADG_FP64):
            del s
            res[prec]["solver"] = None
    r32 = res[HEAD]                # headline: FP32 dofs, reference-matrix products on the tensor cores
    upd = r32["upd"]
    value = whole_job_rate(upd * r32["steps"], world, r32["ms"] * 1e-3)
    ms_step = r32["ms"] / r32["steps"]
    r64 = res[pkg.ADG_FP64]
    value64 = whole_job_rate(upd * r64["steps"], world, r64["ms"] * 1e-3)
    rcc = res[pkg.ADG_FP32]
    value_cc = whole_job_rate(upd * rcc["steps"], world, rcc["ms"] * 1e-3)

    # accuracy of the headline form against FP64 after the same steps from the same input
    s64 = res[pkg.ADG_FP64]["solver"]
    n64 = res[pkg.ADG_FP64]["advanced"]
    sa = Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, degree=N_DEG, precision=HEAD, cfl=0.35,
                device=local, stream=stream.cuda_stream, acoustic_ocean=True)
    sa.set_dofs(Q0)
    sa.set_eta(np.zeros((int(sa.info.n_gravity_faces), 1, sa.Bf)))
    sa.advance(n64)
    q64, qa = s64.get_dofs(), sa.get_dofs()
    h64, ha = s64.read_ssh(), sa.read_ssh()
    accuracy = {"steps": n64, "against": "ADG_FP64 on the same input",
                "dofs_rel_l2": float(np.linalg.norm(qa - q64) / np.linalg.norm(q64)),
                "ssh_rel_l2": float(np.linalg.norm(ha - h64) / max(np.linalg.norm(h64), 1e-300))}
    del q64, qa, sa, s64
    res[pkg.ADG_FP64]["solver"] = None

    # e2e through the public API with host buffers: every step uploads its
    # dofs from pinned host memory, advances one macro step and downloads the
    # result.  Headline: the pipelined calls (adg_set_dofs_f32_async,
    # adg_advance_async, adg_get_dofs_f32_async, then adg_sync), where step k's
    # compute overlaps step k+1's upload and step k-1's download on the two
    # copy engines; also the synchronous calls, one after the other.  One
    # untimed round of each first.
    s = r32["solver"]
    Qp = torch.empty((s.nt, 1, 9, s.B), dtype=torch.float32, pin_memory=True)
    outp = torch.empty((s.nt, 1, 9, s.B), dtype=torch.float32, pin_memory=True)
    Qh32, out32 = Qp.numpy(), outp.numpy()
    Qh32[:, 0] = Q0

    def e2e_pipelined(k):
        for _ in range(k):
            s.set_dofs_f32_async(Qh32)
            s.advance_async(1)
            s.get_dofs_f32_async(out32)
        s.sync()

    def e2e_sync(k):
        for _ in range(k):
            s.set_dofs_f32(Qh32)
            s.advance(1)
            s.get_dofs_f32(out32)

    e2e_pipelined(1)
    barrier()
    t0 = time.perf_counter()
    e2e_pipelined(args.e2e_steps)
    barrier()
    e2e_val = whole_job_rate(upd * args.e2e_steps, world, max_over_ranks(time.perf_counter() - t0))
    e2e_sync(1)
    barrier()
    t0 = time.perf_counter()
    e2e_sync(args.e2e_steps)
    barrier()
    e2e_sync_val = whole_job_rate(upd * args.e2e_steps, world, max_over_ranks(time.perf_counter() - t0))
    bytes_q = s.nt * 9 * s.B * 4
    # the same through the double-array calls (conversion on the host cores)
    Qh = np.ascontiguousarray(Q0)
    out = np.empty((s.nt, 1, 9, s.B))
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        s.set_dofs(Qh)
        s.advance(1)
        pkg._lib.adg_get_dofs(s.ctx, out)
    barrier()
    e2e64_val = whole_job_rate(upd * args.e2e_steps, world, max_over_ranks(time.perf_counter() - t0))

    peaks, src = load_peaks()
    fl = flops_per_update(N_DEG)
    by = bytes_per_update(N_DEG, 4)
    kms = r32["kms"]
    # elements of one launch of the dominant kernel and that launch's own duration:
    # with the tensor-core form the tensor-core launches are timed alone (kms[3], kms[4])
    n_tc = int(s.info.tensor_core_updates_per_macro)
    n_ac = int(s.info.acoustic_updates_per_macro)  # of those, on the 4-quantity local kernel
    tc_form = HEAD == pkg.ADG_3XTF32 and n_tc > 0
    t_k = [kms[3], kms[4]] if tc_form else [kms[0], kms[1]]
    n_k = n_tc if tc_form else s.nt
    dom = 0 if t_k[0] >= t_k[1] else 1
    kname = ["local_tc_kernel", "neighbour_tc_kernel"][dom] if tc_form else ["local_kernel", "neighbour_kernel"][dom]
    clk = r32["clocks"]
    sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    units = unit_peaks()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak, alu_src = alu_peak_tflops(False, peaks.get("sm_max_mhz", 2070.0), units, n_sm)
    achieved_flops = fl[kname.replace("_tc", "")] * n_k / (t_k[dom] * 1e-3) / 1e12
    # an acoustic element's reference-matrix products act on 4 of the 9 quantity rows
    local_bytes = by["local_tc_kernel"] * (n_k - n_ac) + by["local_tc_kernel_acoustic"] * n_ac
    launch_bytes = local_bytes if kname == "local_tc_kernel" else by[kname] * n_k
    achieved_bytes = launch_bytes / (t_k[dom] * 1e-3) / 1e9
    frac_alu = achieved_flops / alu_peak
    frac_hbm = achieved_bytes / peaks["hbm_gbs"]
    tc_peak, tc_src = tf32x3_peak_tflops(peaks, units)
    tensor_flops = fl["local_tensor"] * ((n_k - n_ac) + n_ac * 4.0 / 9.0)
    achieved_tc = tensor_flops / (t_k[0] * 1e-3) / 1e12 if tc_form else None
    if kname == "local_tc_kernel":
        roof = {"bound": "tensor", "achieved": achieved_tc, "peak": tc_peak, "unit": "TFLOP/s",
                "frac": achieved_tc / tc_peak, "traffic": None, "kernel": kname,
                "peak_source": tc_src,
                "flops_counted": "reference-matrix products only (predictor levels 0-2, volume, traces); "
                                 "an acoustic element's count 4/9 of an elastic one's",
                "elements": {"elastic": n_k - n_ac, "acoustic": n_ac}}
    elif kname == "neighbour_tc_kernel":
        # the lift runs on the tensor cores and the fluxes are ~27 kflop per update:
        # HBM (traces, flux matrices, dofs) is the roof
        roof = {"bound": "hbm", "achieved": achieved_bytes, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": frac_hbm, "traffic": None, "kernel": kname, "peak_source": src,
                "bytes_counted": f"{by[kname]} B per update: own and neighbour face blocks, face records, dofs read+write"}
    elif frac_alu >= frac_hbm:
        roof = {"bound": "alu", "achieved": achieved_flops, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": frac_alu, "traffic": None, "kernel": kname,
                "peak_source": alu_src}
    else:
        roof = {"bound": "hbm", "achieved": achieved_bytes, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": frac_hbm, "traffic": None, "kernel": kname, "peak_source": src}
    if kname in TC_DRAM_BYTES_PER_ELEMENT:
        roof["traffic"] = (TC_DRAM_BYTES_PER_ELEMENT[kname] * (n_k - n_ac) +
                           TC_DRAM_BYTES_PER_ELEMENT["local_tc_kernel_acoustic"] * n_ac
                           if kname == "local_tc_kernel" else TC_DRAM_BYTES_PER_ELEMENT[kname] * n_k)
        roof["traffic_note"] = "DRAM bytes per launch, ncu on the 374,400-tet box scaled by elements"
    roof.update({"ms_per_launch": t_k[dom], "elements_per_launch": n_k, "hbm_frac": frac_hbm,
                 # the CUDA-core ALU fraction of a tensor-core kernel's whole flop count means nothing
                 "alu_frac": None if kname.endswith("_tc_kernel") else frac_alu,
                 "kernel_ms": {"local": kms[0], "neighbour": kms[1]}})
    if tc_form:
        roof.update({"tc_kernel_ms": {"local_tc": kms[3], "neighbour_tc": kms[4]},
                     "local_tc_tensor_frac": achieved_tc / tc_peak,
                     "local_tc_hbm_frac": local_bytes / (kms[3] * 1e-3) / 1e9 / peaks["hbm_gbs"],
                     "neighbour_tc_hbm_frac": by["neighbour_tc_kernel"] * n_k / (kms[4] * 1e-3) / 1e9
                     / peaks["hbm_gbs"]})
    r64k = r64["kms"]
    fp64_alu = fl["local_kernel"] * s.nt / (r64k[0] * 1e-3) / 1e12
    fp64_peak, fp64_src = alu_peak_tflops(True, r64["clocks"].get("sm_mhz") or 2070.0, units, n_sm)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": r32["steps"],
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.nxy == 80 else f"{args.nxy}x{args.nxy}-column box", "n_tets": s.nt, "degree": N_DEG, "time_stepping": "global (1 cluster)",
                   "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (3 GB FP32 dofs)"},
        "gflops": value * fl["total"] / 1e9,
        "precision": "FP32 dofs; reference-matrix products of the local kernel as tcgen05 3xTF32 MMAs with "
                     "FP32 accumulation, star and flux products on FP32 CUDA cores (eta, LTS buffers, friction FP64)",
        "fp32_cuda_cores": {"value": value_cc, "unit": UNIT, "ms_per_step": rcc["ms"] / rcc["steps"],
                            "note": "every product on FP32 CUDA cores",
                            "kernel_ms": {"local": rcc["kms"][0], "neighbour": rcc["kms"][1]}},
        "fp64": {"value": value64, "unit": UNIT, "steps": r64["steps"], "ms_per_step": r64["ms"] / r64["steps"],
                 "local_kernel_tflops": fp64_alu, "fp64_peak_tflops": fp64_peak, "fp64_peak_source": fp64_src,
                 "local_kernel_frac": fp64_alu / fp64_peak,
                 "kernel_ms": {"local": r64k[0], "neighbour": r64k[1]}, "clocks": r64["clocks"]},
        "roofline": roof,
        "accuracy": accuracy,
        "clocks": clk,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": bytes_q, "d2h_bytes_per_step": bytes_q,
                "steps": args.e2e_steps,
                "note": "per step adg_set_dofs_f32_async + adg_advance_async(1) + adg_get_dofs_f32_async on "
                        "pinned host float arrays, adg_sync after the last; every copy inside the timed region",
                "synchronous": {"value": e2e_sync_val, "unit": UNIT,
                                "note": "adg_set_dofs_f32 + adg_advance(1) + adg_get_dofs_f32, one after the other"},
                "host_double_arrays": {"value": e2e64_val, "unit": UNIT,
                                       "note": "adg_set_dofs + adg_advance(1) + adg_get_dofs, conversion on the host"}},
        "gpu_launches": r32["launches"] * r32["steps"],
        "autotune": r32["tune"],
    }
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

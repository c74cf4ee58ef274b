"""ctypes binding of the C ABI in include/adg.h (argument marshalling only).

Every function here has the name of the C entry point it wraps, takes numpy
arrays for the pointer arguments and raises AdgError on a negative status.
All computation happens in libadg.so (CUDA kernels + host set-up); there is
no Python or CPU fallback: loading fails loudly if the library is missing.
"""

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libadg.so")

ADG_OK = 0
ADG_FP64, ADG_FP32, ADG_3XTF32 = 0, 1, 2
ADG_FRICTION_RS, ADG_FRICTION_LSW = 0, 1
ADG_RECORD_RECEIVERS, ADG_RECORD_SSH = 0, 1
ERRORS = {-1: "INVALID", -2: "MESH", -3: "STATE", -4: "CUDA", -5: "NOMEM", -6: "NAN",
          -7: "NEWTON", -8: "TIMEOUT", -9: "NOT_READY"}


class AdgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ADG_E_{ERRORS.get(code, code)} ({code}): {msg}")
        self.code = code


class adg_config(C.Structure):
    _fields_ = [("degree", C.c_int), ("precision", C.c_int), ("cfl", C.c_double),
                ("gravity", C.c_double), ("max_clusters", C.c_int), ("ensemble", C.c_int),
                ("device", C.c_int), ("cuda_stream", C.c_void_p)]


class adg_info(C.Structure):
    _fields_ = [("n_tets", C.c_int64), ("n_basis", C.c_int), ("n_face_nodes", C.c_int),
                ("n_clusters", C.c_int), ("cluster_size", C.c_int64 * 16), ("dt_min", C.c_double),
                ("macro_dt", C.c_double), ("time", C.c_double), ("n_gravity_faces", C.c_int64),
                ("n_fault_faces", C.c_int64), ("updates_per_macro", C.c_int64),
                ("device_bytes", C.c_int64), ("tensor_core_updates_per_macro", C.c_int64),
                ("n_receivers", C.c_int64), ("acoustic_updates_per_macro", C.c_int64)]


_P = C.c_void_p
_SIGS = {
    "adg_default_config": (None, [C.POINTER(adg_config)]),
    "adg_create": (C.c_int, [C.POINTER(adg_config), C.POINTER(_P)]),
    "adg_upload_mesh": (C.c_int, [_P, C.c_int64, _P, C.c_int64, _P, _P, _P]),
    "adg_upload_material": (C.c_int, [_P, _P, _P, _P]),
    "adg_init": (C.c_int, [_P]),
    "adg_set_acoustic_ocean": (C.c_int, [_P, C.c_int]),
    "adg_plan": (C.c_int, [_P, _P, _P, C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "adg_face_flux": (C.c_int, [_P, C.c_int64, C.c_int, _P, _P]),
    "adg_face_neighbour": (C.c_int, [_P, C.c_int64, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int), _P]),
    "adg_query": (C.c_int, [_P, C.POINTER(adg_info)]),
    "adg_set_dofs": (C.c_int, [_P, _P]),
    "adg_get_dofs": (C.c_int, [_P, _P]),
    "adg_set_dofs_f32": (C.c_int, [_P, _P]),
    "adg_get_dofs_subset": (C.c_int, [_P, C.c_int64, _P, _P]),
    "adg_hydrostatic_start": (C.c_int, [_P]),
    "adg_record_start": (C.c_int, [_P, C.c_int, C.c_int, C.c_int64]),
    "adg_record_read": (C.c_int, [_P, C.c_int, C.c_int64, _P, _P, _P, _P]),
    "adg_record_stop": (C.c_int, [_P, C.c_int]),
    "adg_get_dofs_f32": (C.c_int, [_P, _P]),
    "adg_set_dofs_f32_async": (C.c_int, [_P, _P]),
    "adg_get_dofs_f32_async": (C.c_int, [_P, _P]),
    "adg_advance_async": (C.c_int, [_P, C.c_int]),
    "adg_initial_points": (C.c_int, [_P, C.POINTER(C.c_int), _P]),
    "adg_set_initial_values": (C.c_int, [_P, _P]),
    "adg_gravity_faces": (C.c_int, [_P, _P, _P]),
    "adg_set_eta": (C.c_int, [_P, _P]),
    "adg_read_ssh": (C.c_int, [_P, _P]),
    "adg_advance": (C.c_int, [_P, C.c_int]),
    "adg_advance_to": (C.c_int, [_P, C.c_double]),
    "adg_step_tick": (C.c_int, [_P]),
    "adg_step_cluster": (C.c_int, [_P, C.c_int]),
    "adg_sync": (C.c_int, [_P]),
    "adg_profile": (C.c_int, [_P, C.c_int, _P, _P]),
    "adg_step_noalloc": (C.c_int, [_P, _P, C.c_int, _P]),
    "adg_autotune": (C.c_int, [_P, C.c_int, C.c_int, _P, _P]),
    "adg_measure_peak": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "adg_fault_faces": (C.c_int, [_P, _P, _P, _P, _P]),
    "adg_set_fault": (C.c_int, [_P, _P]),
    "adg_set_friction_law": (C.c_int, [_P, C.c_int]),
    "adg_read_fault": (C.c_int, [_P, _P]),
    "adg_fault_stats": (C.c_int, [_P, _P, _P, C.c_int]),
    "adg_rupture_capture": (C.c_int, [_P, C.c_int64, _P]),
    "adg_mlp_train": (C.c_int, [_P, C.c_int, C.c_int, C.c_double, C.c_int, _P]),
    "adg_mlp_params": (C.c_int, [_P, _P, _P, C.c_int]),
    "adg_mlp_gradient": (C.c_int, [_P, C.c_int64, _P, _P, _P]),
    "adg_add_receivers": (C.c_int, [_P, C.c_int64, _P]),
    "adg_read_receivers": (C.c_int, [_P, _P]),
    "adg_save_state": (C.c_int, [_P, _P, C.POINTER(C.c_size_t)]),
    "adg_load_state": (C.c_int, [_P, _P, C.c_size_t]),
    "adg_reference_operators": (C.c_int, [C.c_int, _P, _P, _P, _P]),
    "adg_last_error": (C.c_char_p, [_P]),
    "adg_destroy": (None, [_P]),
}

_lib = None


def load():
    """Load libadg.so (built by paper_2107_06640_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2107_06640_gb300.build`"
                              " (the solver has no CPU fallback)")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(ctx, rc):
    if rc != ADG_OK:
        msg = load().adg_last_error(ctx).decode() if ctx else ""
        raise AdgError(rc, msg)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# Host arrays cross the ABI as plain pointers: the library reads or writes as
# many values as the context's sizes say, so every array is checked here.
_NT = {}  # tets of each context's uploaded mesh (for the material upload)


def _dims(ctx):
    """(n_tets, S, B, Bf, n_gravity_faces, n_fault_faces, n_receivers) of an initialised context."""
    i = adg_query(ctx)
    ncl = int(i.n_clusters)
    w = sum(int(i.cluster_size[c]) << (ncl - 1 - c) for c in range(ncl))
    S = int(i.updates_per_macro) // w if w else 1
    return (int(i.n_tets), S, int(i.n_basis), int(i.n_face_nodes), int(i.n_gravity_faces), int(i.n_fault_faces),
            int(i.n_receivers))


def _host(a, dtype, count, what, out=False):
    """`a` as the library sees it: `count` values of `dtype`, C-contiguous.  An
    input is converted; an output must already be such an array."""
    if out:
        if not (isinstance(a, np.ndarray) and a.dtype == np.dtype(dtype) and a.flags.c_contiguous):
            raise ValueError(f"{what}: needs a C-contiguous {np.dtype(dtype).name} array")
    else:
        a = np.ascontiguousarray(a, dtype=dtype)
    if a.size != count:
        raise ValueError(f"{what}: {a.size} values given, the library uses {count}")
    return a


def adg_default_config():
    cfg = adg_config()
    load().adg_default_config(C.byref(cfg))
    return cfg


def adg_create(cfg):
    h = C.c_void_p()
    _check(None, load().adg_create(C.byref(cfg), C.byref(h)))
    return h


def adg_upload_mesh(ctx, xyz, tets, face_tag, face_partner=None):
    xyz = _f64(xyz)
    tets = np.ascontiguousarray(tets, dtype=np.int64)
    if xyz.ndim != 2 or xyz.shape[1] != 3 or tets.ndim != 2 or tets.shape[1] != 4:
        raise ValueError("mesh: xyz [nv][3] and tets [nt][4] expected")
    nt = tets.shape[0]
    face_tag = _host(face_tag, np.int32, 4 * nt, "face_tag [nt][4]")
    fp = None if face_partner is None else _host(face_partner, np.int64, 4 * nt, "face_partner [nt][4]")
    _check(ctx, load().adg_upload_mesh(ctx, xyz.shape[0], _ptr(xyz), nt, _ptr(tets), _ptr(face_tag), _ptr(fp)))
    _NT[ctx.value] = nt


def adg_upload_material(ctx, rho, lam, mu):
    nt = _NT.get(ctx.value)
    if nt is None:
        raise ValueError("material: upload the mesh first")
    rho, lam, mu = (_host(a, np.float64, nt, name) for a, name in ((rho, "rho"), (lam, "lambda"), (mu, "mu")))
    _check(ctx, load().adg_upload_material(ctx, _ptr(rho), _ptr(lam), _ptr(mu)))


def adg_init(ctx):
    _check(ctx, load().adg_init(ctx))


def adg_set_acoustic_ocean(ctx, enable=True):
    _check(ctx, load().adg_set_acoustic_ocean(ctx, int(bool(enable))))


def adg_plan(ctx):
    """(dt_elem [nt], cluster [nt], dt_min, n_clusters) of the uploaded mesh,
    computed on the host (no device needed)."""
    nt = _NT.get(ctx.value)
    if nt is None:
        raise ValueError("plan: upload the mesh first")
    dt = np.empty(nt, np.float64)
    cl = np.empty(nt, np.int32)
    dtmin, ncl = C.c_double(), C.c_int()
    _check(ctx, load().adg_plan(ctx, _ptr(dt), _ptr(cl), C.byref(dtmin), C.byref(ncl)))
    return dt, cl, dtmin.value, ncl.value


def adg_face_flux(ctx, tet, face):
    """(Fm, Fp), each [9][9], of local face `face` of user tet `tet` (host only)."""
    Fm = np.empty((9, 9), np.float64)
    Fp = np.empty((9, 9), np.float64)
    _check(ctx, load().adg_face_flux(ctx, int(tet), int(face), _ptr(Fm), _ptr(Fp)))
    return Fm, Fp


def adg_face_neighbour(ctx, tet, face, n_face_nodes):
    """(neighbour tet, its local face, node_map [Bf]) of local face `face` of
    user tet `tet` (host only); (-1, -1, None) without a neighbour."""
    nb, nf = C.c_int64(), C.c_int()
    node_map = np.full(int(n_face_nodes), -1, np.int32)
    _check(ctx, load().adg_face_neighbour(ctx, int(tet), int(face), C.byref(nb), C.byref(nf), _ptr(node_map)))
    return (nb.value, nf.value, node_map) if nb.value >= 0 else (-1, -1, None)


def adg_query(ctx):
    info = adg_info()
    _check(ctx, load().adg_query(ctx, C.byref(info)))
    return info


def _ndofs(ctx):
    nt, S, B = _dims(ctx)[:3]
    return nt * S * 9 * B


def adg_set_dofs(ctx, Q):
    Q = _host(Q, np.float64, _ndofs(ctx), "dofs [nt][S][9][B]")
    _check(ctx, load().adg_set_dofs(ctx, _ptr(Q)))


def adg_get_dofs(ctx, out):
    _host(out, np.float64, _ndofs(ctx), "dofs [nt][S][9][B]", out=True)
    _check(ctx, load().adg_get_dofs(ctx, _ptr(out)))
    return out


def adg_set_dofs_f32(ctx, Q):
    """Q: float32 [tet][S][9][B] (pinned host memory for full speed)."""
    Q = _host(Q, np.float32, _ndofs(ctx), "dofs [nt][S][9][B]")
    _check(ctx, load().adg_set_dofs_f32(ctx, _ptr(Q)))


def adg_get_dofs_f32(ctx, out):
    _host(out, np.float32, _ndofs(ctx), "dofs [nt][S][9][B]", out=True)
    _check(ctx, load().adg_get_dofs_f32(ctx, _ptr(out)))
    return out


def adg_set_dofs_f32_async(ctx, Q):
    """Enqueue the upload of Q (C-contiguous float32 [tet][S][9][B], pinned host
    memory; never a converted copy, since Q is borrowed until adg_sync returns)."""
    _host(Q, np.float32, _ndofs(ctx), "dofs [nt][S][9][B]", out=True)
    _check(ctx, load().adg_set_dofs_f32_async(ctx, _ptr(Q)))
    return Q


def adg_get_dofs_f32_async(ctx, out):
    """Enqueue the download into out (float32, pinned); complete after adg_sync."""
    _host(out, np.float32, _ndofs(ctx), "dofs [nt][S][9][B]", out=True)
    _check(ctx, load().adg_get_dofs_f32_async(ctx, _ptr(out)))
    return out


def adg_advance_async(ctx, n):
    _check(ctx, load().adg_advance_async(ctx, int(n)))


def adg_record_start(ctx, kind, every, capacity):
    _check(ctx, load().adg_record_start(ctx, int(kind), int(every), int(capacity)))


def adg_record_read(ctx, kind, max_samples, sample):
    """Up to max_samples unread samples of `sample` doubles each: (t, data[k][sample], dropped)."""
    t = np.empty(max(int(max_samples), 0))
    data = np.empty((max(int(max_samples), 0), int(sample)))
    n, dropped = C.c_int64(0), C.c_int64(0)
    _check(ctx, load().adg_record_read(ctx, int(kind), int(max_samples), _ptr(t), _ptr(data), C.byref(n),
                                       C.byref(dropped)))
    return t[: n.value], data[: n.value], dropped.value


def adg_record_stop(ctx, kind):
    _check(ctx, load().adg_record_stop(ctx, int(kind)))


def adg_hydrostatic_start(ctx):
    _check(ctx, load().adg_hydrostatic_start(ctx))


def adg_get_dofs_subset(ctx, tets, out):
    tets = np.ascontiguousarray(tets, dtype=np.int64).ravel()
    nt, S, B = _dims(ctx)[:3]
    _host(out, np.float64, tets.size * S * 9 * B, "dofs [n][S][9][B]", out=True)
    _check(ctx, load().adg_get_dofs_subset(ctx, tets.size, _ptr(tets), _ptr(out)))
    return out


def adg_initial_points(ctx, n_tets):
    if int(n_tets) != _dims(ctx)[0]:
        raise ValueError("initial points: n_tets differs from the mesh")
    n = C.c_int()
    _check(ctx, load().adg_initial_points(ctx, C.byref(n), None))
    xyz = np.empty((n_tets, n.value, 3))
    _check(ctx, load().adg_initial_points(ctx, C.byref(n), _ptr(xyz)))
    return xyz


def adg_set_initial_values(ctx, values):
    nt, S = _dims(ctx)[:2]
    nq = C.c_int()
    _check(ctx, load().adg_initial_points(ctx, C.byref(nq), None))
    values = _host(values, np.float64, nt * S * nq.value * 9, "values [nt][S][n_pts][9]")
    _check(ctx, load().adg_set_initial_values(ctx, _ptr(values)))


def adg_gravity_faces(ctx, n, Bf):
    d = _dims(ctx)
    if int(n) != d[4] or int(Bf) != d[3]:
        raise ValueError("gravity faces: n or Bf differs from the context")
    ef = np.empty(n, np.int64)
    xyz = np.empty((n, Bf, 3))
    if n:
        _check(ctx, load().adg_gravity_faces(ctx, _ptr(ef), _ptr(xyz)))
    return ef, xyz


def _neta(ctx):
    nt, S, B, Bf, ngf = _dims(ctx)[:5]
    return ngf * S * Bf


def adg_set_eta(ctx, eta):
    eta = _host(eta, np.float64, _neta(ctx), "eta [n_gravity_faces][S][Bf]")
    _check(ctx, load().adg_set_eta(ctx, _ptr(eta)))


def adg_read_ssh(ctx, out):
    _host(out, np.float64, _neta(ctx), "eta [n_gravity_faces][S][Bf]", out=True)
    _check(ctx, load().adg_read_ssh(ctx, _ptr(out)))
    return out


def adg_advance(ctx, n):
    _check(ctx, load().adg_advance(ctx, int(n)))


def adg_advance_to(ctx, t):
    _check(ctx, load().adg_advance_to(ctx, float(t)))


def adg_step_tick(ctx):
    _check(ctx, load().adg_step_tick(ctx))


def adg_step_cluster(ctx, c):
    _check(ctx, load().adg_step_cluster(ctx, int(c)))


def adg_sync(ctx):
    _check(ctx, load().adg_sync(ctx))


def adg_profile(ctx, n_macro):
    ms = np.zeros(5)
    cnt = np.zeros(5, np.int64)
    _check(ctx, load().adg_profile(ctx, int(n_macro), _ptr(ms), _ptr(cnt)))
    return ms, cnt


def adg_step_noalloc(ctx, d_Q_ptr, n_steps, stream_ptr=None):
    """d_Q_ptr: integer device address of the caller's dofs (see include/adg.h)."""
    _check(ctx, load().adg_step_noalloc(ctx, C.c_void_p(d_Q_ptr), int(n_steps),
                                        None if stream_ptr is None else C.c_void_p(stream_ptr)))


def adg_autotune(ctx, reps=2, force=False):
    """Launch shapes chosen by the library's autotuner: (choice [4] =
    CUDA-core local / neighbour threads per block, tensor-core local /
    neighbour tiles per CTA sweep; ms [4][3] per candidate)."""
    choice = np.zeros(4, np.int32)
    ms = np.zeros((4, 3))
    _check(ctx, load().adg_autotune(ctx, int(reps), int(bool(force)), _ptr(choice), _ptr(ms)))
    return choice, ms


def adg_measure_peak(kind, device=0, reps=20):
    """(flops, ms) of `reps` timed launches of peak probe `kind` (0: tcgen05
    kind::tf32 MMA, 1: FP32 FMA, 2: FP64 FMA) on `device`."""
    f, ms = C.c_double(), C.c_double()
    _check(None, load().adg_measure_peak(int(kind), int(device), int(reps), C.byref(f), C.byref(ms)))
    return f.value, ms.value


FPAR, FSTATE, MLP_NPARAM, MLP_TRAINABLE = 13, 8, 1327, 1313


def adg_fault_faces(ctx, nff, Bf):
    d = _dims(ctx)
    if int(nff) != d[5] or int(Bf) != d[3]:
        raise ValueError("fault faces: nff or Bf differs from the context")
    mf = np.empty(nff, np.int64)
    pf = np.empty(nff, np.int64)
    xyz = np.empty((nff, Bf, 3))
    nrm = np.empty((nff, 3))
    _check(ctx, load().adg_fault_faces(ctx, _ptr(mf), _ptr(pf), _ptr(xyz), _ptr(nrm)))
    return mf, pf, xyz, nrm


def _nfault(ctx):
    nt, S, B, Bf, ngf, nff = _dims(ctx)[:6]
    return nff * S * Bf


def adg_set_fault(ctx, par):
    par = _host(par, np.float64, _nfault(ctx) * FPAR, "fault parameters [nff][S][Bf][13]")
    _check(ctx, load().adg_set_fault(ctx, _ptr(par)))


def adg_set_friction_law(ctx, law):
    _check(ctx, load().adg_set_friction_law(ctx, int(law)))


def adg_read_fault(ctx, out):
    _host(out, np.float64, _nfault(ctx) * FSTATE, "fault state [nff][S][Bf][8]", out=True)
    _check(ctx, load().adg_read_fault(ctx, _ptr(out)))
    return out


def adg_fault_stats(ctx, reset=False):
    s = C.c_int64()
    it = C.c_int64()
    _check(ctx, load().adg_fault_stats(ctx, C.byref(s), C.byref(it), int(reset)))
    return s.value, it.value


def adg_rupture_capture(ctx, capacity):
    n = C.c_int64()
    _check(ctx, load().adg_rupture_capture(ctx, int(capacity), C.byref(n)))
    return n.value


def adg_mlp_train(ctx, epochs, batch, lr, seed=0):
    loss = np.zeros(2)
    _check(ctx, load().adg_mlp_train(ctx, int(epochs), int(batch), float(lr), int(seed), _ptr(loss)))
    return loss


def adg_mlp_params(ctx, set_params=None, enable=-1):
    get = np.empty(MLP_NPARAM, np.float32)
    sp = None if set_params is None else _host(set_params, np.float32, MLP_NPARAM, "network parameters")
    _check(ctx, load().adg_mlp_params(ctx, _ptr(sp), _ptr(get), int(enable)))
    return get


def adg_mlp_gradient(params, rows):
    params = _host(params, np.float32, MLP_NPARAM, "network parameters")
    rows = np.ascontiguousarray(rows, dtype=np.float32)
    if rows.ndim != 2 or rows.shape[1] != 7:
        raise ValueError("rows: [n][7] expected (6 features, target)")
    grad = np.empty(MLP_TRAINABLE, np.float32)
    loss = np.zeros(1)
    _check(None, load().adg_mlp_gradient(_ptr(params), rows.shape[0], _ptr(rows), _ptr(grad), _ptr(loss)))
    return grad, loss[0]


def adg_add_receivers(ctx, xyz):
    xyz = _f64(xyz)
    if xyz.ndim != 2 or xyz.shape[1] != 3:
        raise ValueError("receivers: xyz [n][3] expected")
    _check(ctx, load().adg_add_receivers(ctx, xyz.shape[0], _ptr(xyz)))


def adg_read_receivers(ctx, out):
    d = _dims(ctx)
    _host(out, np.float64, d[6] * d[1] * 9, "receivers [n][S][9]", out=True)
    _check(ctx, load().adg_read_receivers(ctx, _ptr(out)))
    return out


def adg_save_state(ctx):
    n = C.c_size_t(0)
    _check(ctx, load().adg_save_state(ctx, None, C.byref(n)))
    buf = np.empty(n.value, np.uint8)
    _check(ctx, load().adg_save_state(ctx, _ptr(buf), C.byref(n)))
    return buf


def adg_load_state(ctx, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(ctx, load().adg_load_state(ctx, _ptr(buf), buf.size))


def adg_reference_operators(N):
    B = (N + 1) * (N + 2) * (N + 3) // 6
    Bf = (N + 1) * (N + 2) // 2
    B1 = N * (N + 1) * (N + 2) // 6
    kt = np.empty((3, B, B))
    kvol = np.empty((3, B, B1))
    efc = np.empty((4, Bf, B))
    lift = np.empty((4, B, Bf))
    _check(None, load().adg_reference_operators(N, _ptr(kt), _ptr(kvol), _ptr(efc), _ptr(lift)))
    return kt, kvol, efc, lift


def adg_last_error(ctx):
    return load().adg_last_error(ctx).decode()


def adg_destroy(ctx):
    if ctx is not None:
        _NT.pop(ctx.value, None)
    load().adg_destroy(ctx)

"""Convenience wrapper around one adg_ctx (marshalling only; see _lib)."""

import numpy as np

from . import _lib as L


def plan(xyz, tets, face_tag, rho, lam, mu, face_partner=None, degree=5, cfl=0.35, max_clusters=1):
    """The element time steps and rate-2 clusters a Solver on this mesh would
    use, computed on the host without a device (adg_plan): returns
    (dt_elem [nt], cluster [nt], dt_min, n_clusters)."""
    cfg = L.adg_default_config()
    cfg.degree = degree
    cfg.cfl = cfl
    cfg.max_clusters = max_clusters
    ctx = L.adg_create(cfg)
    try:
        L.adg_upload_mesh(ctx, xyz, tets, face_tag, face_partner)
        L.adg_upload_material(ctx, rho, lam, mu)
        return L.adg_plan(ctx)
    finally:
        L.adg_destroy(ctx)


class Solver:
    def __init__(self, xyz, tets, face_tag, rho, lam, mu, face_partner=None, degree=5,
                 precision=L.ADG_FP64, cfl=0.35, gravity=9.81, max_clusters=1, ensemble=1,
                 device=0, stream=None, acoustic_ocean=False):
        cfg = L.adg_default_config()
        cfg.degree = degree
        cfg.precision = precision
        cfg.cfl = cfl
        cfg.gravity = gravity
        cfg.max_clusters = max_clusters
        cfg.ensemble = ensemble
        cfg.device = device
        cfg.cuda_stream = stream
        self.ctx = L.adg_create(cfg)
        try:
            L.adg_upload_mesh(self.ctx, xyz, tets, face_tag, face_partner)
            L.adg_upload_material(self.ctx, rho, lam, mu)
            if acoustic_ocean:
                L.adg_set_acoustic_ocean(self.ctx, True)
            L.adg_init(self.ctx)
        except Exception:
            L.adg_destroy(self.ctx)
            self.ctx = None
            raise
        self.info = L.adg_query(self.ctx)
        self.nt = int(self.info.n_tets)
        self.B = self.info.n_basis
        self.Bf = self.info.n_face_nodes
        self.S = ensemble

    def __del__(self):
        if getattr(self, "ctx", None) is not None:
            L.adg_destroy(self.ctx)
            self.ctx = None

    def plan(self):
        """(dt_elem, cluster, dt_min, n_clusters) in the caller's element order."""
        return L.adg_plan(self.ctx)

    def query(self):
        self.info = L.adg_query(self.ctx)
        return self.info

    @property
    def time(self):
        return L.adg_query(self.ctx).time

    def set_dofs(self, Q):
        """Q[tet][S][9][B] (or [tet][9][B] when S == 1)."""
        L.adg_set_dofs(self.ctx, Q)

    def get_dofs(self):
        out = np.empty((self.nt, self.S, 9, self.B))
        L.adg_get_dofs(self.ctx, out)
        return out[:, 0] if self.S == 1 else out

    def hydrostatic_start(self):
        """Ocean at rest with p' = rho g eta under the current sea surface (after set_eta)."""
        L.adg_hydrostatic_start(self.ctx)

    def get_dofs_subset(self, tets):
        """Dofs of the listed tets, [n][S][9][B] (or [n][9][B] when S == 1)."""
        tets = np.asarray(tets, dtype=np.int64).ravel()
        out = np.empty((tets.size, self.S, 9, self.B))
        L.adg_get_dofs_subset(self.ctx, tets, out)
        return out[:, 0] if self.S == 1 else out

    def set_dofs_f32(self, Q):
        """Q: float32 [tet][S][9][B] (or [tet][9][B] when S == 1); at a macro-step boundary."""
        L.adg_set_dofs_f32(self.ctx, Q)

    def get_dofs_f32(self, out=None):
        """Into out (float32 [tet][S][9][B], e.g. pinned) or a new array; at a macro-step boundary."""
        if out is None:
            out = np.empty((self.nt, self.S, 9, self.B), np.float32)
        L.adg_get_dofs_f32(self.ctx, out)
        return out

    def set_dofs_f32_async(self, Q):
        """Enqueue the upload of Q (C-contiguous float32 [tet][S][9][B], pinned);
        Q stays borrowed until sync() returns."""
        L.adg_set_dofs_f32_async(self.ctx, Q)

    def get_dofs_f32_async(self, out):
        """Enqueue the download of the dofs into out (float32, pinned); complete after sync()."""
        L.adg_get_dofs_f32_async(self.ctx, out)
        return out

    def advance_async(self, n=1):
        """Enqueue n macro steps; device errors surface at the next sync()."""
        L.adg_advance_async(self.ctx, n)

    def initial_points(self):
        return L.adg_initial_points(self.ctx, self.nt)

    def set_initial_values(self, values):
        L.adg_set_initial_values(self.ctx, values)

    def gravity_faces(self):
        return L.adg_gravity_faces(self.ctx, int(self.info.n_gravity_faces), self.Bf)

    def set_eta(self, eta):
        L.adg_set_eta(self.ctx, eta)

    def read_ssh(self):
        out = np.empty((int(self.info.n_gravity_faces), self.S, self.Bf))
        return L.adg_read_ssh(self.ctx, out)

    def advance(self, n=1):
        L.adg_advance(self.ctx, n)

    def advance_to(self, t):
        L.adg_advance_to(self.ctx, t)

    def step_tick(self):
        L.adg_step_tick(self.ctx)

    def step_cluster(self, c):
        L.adg_step_cluster(self.ctx, c)

    def sync(self):
        L.adg_sync(self.ctx)

    def add_receivers(self, xyz):
        self._nrec = len(xyz)
        L.adg_add_receivers(self.ctx, xyz)

    def read_receivers(self):
        out = np.empty((self._nrec, self.S, 9))
        return L.adg_read_receivers(self.ctx, out)

    def record(self, kind, every, capacity):
        """Start recording receivers (L.ADG_RECORD_RECEIVERS) or the sea surface
        (L.ADG_RECORD_SSH) every `every` macro steps of advance / advance_to."""
        L.adg_record_start(self.ctx, kind, every, capacity)
        self._rec_cap = getattr(self, "_rec_cap", {})
        self._rec_cap[kind] = int(capacity)

    def read_record(self, kind, max_samples=None):
        """Unread samples, oldest first (at most max_samples, default the ring
        capacity): (t[k], samples[k] shaped as read_receivers / read_ssh,
        dropped so far)."""
        if kind == L.ADG_RECORD_RECEIVERS:
            shape = (self._nrec, self.S, 9)
        else:
            shape = (int(self.info.n_gravity_faces), self.S, self.Bf)
        cap = getattr(self, "_rec_cap", {}).get(kind, 0) if max_samples is None else int(max_samples)
        t, data, dropped = L.adg_record_read(self.ctx, kind, cap, int(np.prod(shape)))
        return t, data.reshape((len(t),) + shape), dropped

    def stop_record(self, kind):
        L.adg_record_stop(self.ctx, kind)

    def save_state(self):
        return L.adg_save_state(self.ctx)

    def load_state(self, buf):
        L.adg_load_state(self.ctx, buf)

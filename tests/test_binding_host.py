"""Host side of the Python binding (no GPU): every wrapper that hands a host
array to the C ABI checks it against the context's sizes (from adg_query)
and refuses a wrong size, dtype or layout with ValueError before the call;
correct arrays reach the library.  A fake library stands in for libadg.so."""

import ctypes as C

import numpy as np
import pytest

from paper_2107_06640_gb300 import _lib as L

NT, S, B, BF, NGF, NFF, NREC, NQ = 10, 2, 20, 10, 3, 2, 4, 7


class FakeLib:
    """Records the calls; adg_query reports two clusters (4 + 6 tets), S = 2."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*args):
            self.calls.append(name)
            if name == "adg_query":
                info = args[1]._obj
                info.n_tets, info.n_basis, info.n_face_nodes, info.n_clusters = NT, B, BF, 2
                info.cluster_size[0], info.cluster_size[1] = 4, 6
                info.updates_per_macro = (4 * 2 + 6) * S
                info.n_gravity_faces, info.n_fault_faces, info.n_receivers = NGF, NFF, NREC
            elif name == "adg_initial_points":
                args[1]._obj.value = NQ
            elif name == "adg_last_error":
                return b""
            return 0
        return call


@pytest.fixture
def fake():
    saved = L._lib
    L._lib = FakeLib()
    ctx = C.c_void_p(0x1234)
    L.adg_upload_mesh(ctx, np.zeros((5, 3)), np.zeros((NT, 4)), np.zeros((NT, 4)))
    yield ctx, L._lib
    L.adg_destroy(ctx)
    L._lib = saved


def test_sizes_from_the_context(fake):
    ctx, _ = fake
    assert L._dims(ctx) == (NT, S, B, BF, NGF, NFF, NREC)


def test_correct_arrays_reach_the_library(fake):
    ctx, lib = fake
    L.adg_upload_material(ctx, np.ones(NT), np.ones(NT), np.ones(NT))
    L.adg_set_dofs(ctx, np.zeros((NT, S, 9, B)))
    L.adg_get_dofs(ctx, np.zeros((NT, S, 9, B)))
    L.adg_set_dofs_f32(ctx, np.zeros((NT, S, 9, B), np.float32))
    L.adg_get_dofs_f32(ctx, np.zeros((NT, S, 9, B), np.float32))
    L.adg_get_dofs_subset(ctx, [1, 2, 3], np.zeros((3, S, 9, B)))
    L.adg_set_initial_values(ctx, np.zeros((NT, S, NQ, 9)))
    L.adg_set_eta(ctx, np.zeros((NGF, S, BF)))
    L.adg_read_ssh(ctx, np.zeros((NGF, S, BF)))
    L.adg_set_fault(ctx, np.zeros((NFF, S, BF, L.FPAR)))
    L.adg_read_fault(ctx, np.zeros((NFF, S, BF, L.FSTATE)))
    L.adg_read_receivers(ctx, np.zeros((NREC, S, 9)))
    for name in ("adg_upload_material", "adg_set_dofs", "adg_get_dofs", "adg_set_dofs_f32", "adg_get_dofs_f32",
                 "adg_get_dofs_subset", "adg_set_initial_values", "adg_set_eta", "adg_read_ssh", "adg_set_fault",
                 "adg_read_fault", "adg_read_receivers"):
        assert name in lib.calls


@pytest.mark.parametrize("bad", [
    lambda c: L.adg_set_dofs(c, np.zeros((NT, S, 9, B - 1))),
    lambda c: L.adg_get_dofs(c, np.zeros((NT, S, 9, B), np.float32)),          # dtype
    lambda c: L.adg_get_dofs(c, np.zeros((NT, S, 9, 2 * B))[..., ::2]),        # not contiguous
    lambda c: L.adg_set_dofs_f32(c, np.zeros((NT, 1, 9, B), np.float32)),      # one scenario short
    lambda c: L.adg_get_dofs_subset(c, [1, 2], np.zeros((3, S, 9, B))),
    lambda c: L.adg_set_initial_values(c, np.zeros((NT, S, NQ - 1, 9))),
    lambda c: L.adg_set_eta(c, np.zeros((NGF, BF))),
    lambda c: L.adg_read_fault(c, np.zeros((NFF, S, BF, L.FSTATE - 1))),
    lambda c: L.adg_read_receivers(c, np.zeros((NREC + 1, S, 9))),
    lambda c: L.adg_gravity_faces(c, NGF + 1, BF),
    lambda c: L.adg_fault_faces(c, NFF, BF + 1),
    lambda c: L.adg_initial_points(c, NT + 1),
    lambda c: L.adg_upload_material(c, np.ones(NT - 1), np.ones(NT), np.ones(NT)),
    lambda c: L.adg_upload_mesh(c, np.zeros((5, 2)), np.zeros((NT, 4)), np.zeros((NT, 4))),
    lambda c: L.adg_add_receivers(c, np.zeros((NREC, 2))),
    lambda c: L.adg_mlp_params(c, np.zeros(L.MLP_NPARAM - 1, np.float32)),
])
def test_wrong_arrays_are_refused_before_the_call(fake, bad):
    ctx, lib = fake
    n = len(lib.calls)
    with pytest.raises(ValueError):
        bad(ctx)
    assert all(c in ("adg_query", "adg_initial_points") for c in lib.calls[n:])

"""CPU-only checks of the C-ABI library: it loads, exports every entry point
declared in include/adg.h, and its host-generated reference operators agree
with the oracle's independent construction (exact monomial integrals in C++
versus Jacobi-polynomial quadrature in numpy)."""

import os
import re

import numpy as np
import pytest

from oracle import basis as ob
from oracle.quadrature import tri_rule


@pytest.fixture(scope="module")
def lib():
    from paper_2107_06640_gb300 import build
    build.build()
    from paper_2107_06640_gb300 import _lib
    return _lib


def test_exports_every_declared_symbol(lib, root):
    hdr = open(os.path.join(root, "include", "adg.h")).read()
    declared = set(re.findall(r"\b(adg_[a-z0-9_]+)\s*\(", hdr))
    declared -= {"adg_ctx"}
    L = lib.load()
    for name in declared:
        assert hasattr(L, name), name
    assert declared == set(lib.exported_symbols())


def _oracle_ops(N):
    B, Bf = ob.n_basis(N), ob.n_face_basis(N)
    K = ob.stiffness(N)                       # K[a][k,l] = int dphi_k/dxi_a phi_l
    kt = np.transpose(K, (0, 2, 1))          # kt[a][m][l] = int phi_m dphi_l/dxi_a
    kvol = K[:, :, : ob.n_basis(N - 1)]
    nodes = np.array([[i1 / N, i2 / N] for i2 in range(N + 1) for i1 in range(N + 1 - i2)])
    efc = np.stack([ob.eval_basis(N, ob.face_to_ref(f, nodes)) for f in range(4)])
    # Lagrange basis on the nodes, integrated against the face traces
    mono = [(a, b) for a in range(N + 1) for b in range(N + 1 - a)]
    V = np.array([[x ** a * y ** b for (a, b) in mono] for x, y in nodes])
    chi, w = tri_rule(2 * N)
    Vq = np.array([[x ** a * y ** b for (a, b) in mono] for x, y in chi])
    ell = Vq @ np.linalg.inv(V)              # ell[q, n]
    lift = np.stack([np.einsum("q,qm,qn->mn", w, ob.eval_basis(N, ob.face_to_ref(f, chi)), ell)
                     for f in range(4)])
    assert lift.shape == (4, B, Bf)
    return kt, kvol, efc, lift


@pytest.mark.parametrize("N", [1, 3, 5])
def test_reference_operators_match_oracle(lib, N):
    got = lib.adg_reference_operators(N)
    want = _oracle_ops(N)
    for g, w, name in zip(got, want, ("kt", "kvol", "efc", "lift")):
        assert g.shape == w.shape, name
        assert np.abs(g - w).max() < 1e-11 * max(1.0, np.abs(w).max()), (name, np.abs(g - w).max())


def test_context_errors_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("checks the no-GPU failure mode")
    cfg = lib.adg_default_config()
    cfg.degree = 9
    with pytest.raises(lib.AdgError):
        lib.adg_create(cfg)
    cfg = lib.adg_default_config()
    cfg.degree = 2
    ctx = lib.adg_create(cfg)
    try:
        with pytest.raises(lib.AdgError) as ei:
            lib.adg_init(ctx)  # nothing uploaded
        assert ei.value.code == -3
        import synthetic as syn
        m = syn.unit_cube_periodic(1)
        lib.adg_upload_mesh(ctx, m.xyz, m.tets, m.face_tag, m.face_partner)
        lib.adg_upload_material(ctx, *syn.elastic_uniform(m.nt))
        with pytest.raises(lib.AdgError) as ei:
            lib.adg_init(ctx)  # no device here: a loud CUDA error, never a CPU fallback
        assert ei.value.code == -4
    finally:
        lib.adg_destroy(ctx)

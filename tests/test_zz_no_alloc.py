"""The allocation-free step entry point (adg_step_noalloc).

Callers that must not allocate device memory while they step (a plug-in
whose host application owns all device memory, for instance) keep their dofs
in memory they already own; adg_step_noalloc steps them in place and uses a
fixed static device array inside the library for its face-trace scratch.
This file runs last so that a failure here never hides another test.  The
test itself allocates the caller's buffer with torch, as such a caller would
have done ahead of time.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2107_06640_gb300 import build
    build.build()
    from paper_2107_06640_gb300 import _lib
    return _lib


def _periodic_context(n, N, precision=0):
    from paper_2107_06640_gb300 import Solver
    from synthetic.workloads import plane_wave_case
    m, (rho, lam, mu) = plane_wave_case(n)
    return m, Solver(m.xyz, m.tets, m.face_tag, rho, lam, mu, face_partner=m.face_partner,
                     degree=N, cfl=0.5, precision=precision)


def test_noalloc_steps_match_the_context_path(lib):
    import torch
    from synthetic.workloads import random_dofs
    m, s = _periodic_context(8, 3)          # 3072 tets: 8.8 MB of FP64 traces
    Q0 = random_dofs((m.nt, 9, s.B), 21, N=3)
    d = torch.tensor(Q0, dtype=torch.float64, device="cuda").contiguous()
    stream = torch.cuda.current_stream()
    out = []
    for _ in range(2):                       # two calls in a row on the same buffer
        lib.adg_step_noalloc(s.ctx, d.data_ptr(), 1, stream.cuda_stream)
        torch.cuda.synchronize()
        out.append(d.cpu().numpy().copy())
    assert np.all(s.get_dofs() == 0.0)       # the context's own dofs were not touched
    s.sync()
    s.set_dofs(Q0)
    for k in range(2):
        s.advance(1)
        ref = s.get_dofs()
        err = np.linalg.norm(out[k] - ref) / np.linalg.norm(ref)
        assert err <= 1e-10, (k, err)


@pytest.mark.parametrize("precision,tol", [(1, 1e-6), (2, 2e-5)])
def test_noalloc_fp32_contexts(lib, precision, tol):
    """FP32 contexts: ADG_FP32 steps with the same CUDA-core kernels as
    adg_advance (equal up to FP32 rounding order); in an ADG_3XTF32 context the
    call also runs the FP32 CUDA-core kernels (its tensor-core path stages
    through shared memory the context allocated), so it is held to the FP32
    tolerance against that context's own steps.  Two calls in a row."""
    import torch
    from synthetic.workloads import random_dofs
    m, s = _periodic_context(4, 5, precision)   # 384 tets at N=5
    Q0 = random_dofs((m.nt, 9, s.B), 22, N=5)
    d = torch.tensor(Q0, dtype=torch.float32, device="cuda").contiguous()
    out = []
    for _ in range(2):
        lib.adg_step_noalloc(s.ctx, d.data_ptr(), 1, torch.cuda.current_stream().cuda_stream)
        out.append(d.cpu().numpy().astype(np.float64))
    s.set_dofs(Q0)
    for k in range(2):
        s.advance(1)
        ref = s.get_dofs()
        err = np.linalg.norm(out[k] - ref) / np.linalg.norm(ref)
        assert err <= tol, (k, err)


def test_noalloc_is_ordered_on_the_callers_streams(lib):
    """The caller writes its dofs on a stream, steps on it and reads back on
    it, with no device-wide synchronisation: once on a side stream of its own,
    once on torch's default stream passed as handle 0 (CUDA's default
    stream) and once with no stream (NULL: the same default stream)."""
    import torch
    from synthetic.workloads import random_dofs
    m, s = _periodic_context(4, 3)
    Q0 = torch.tensor(random_dofs((m.nt, 9, s.B), 23, N=3), dtype=torch.float64).pin_memory()
    s.set_dofs(Q0.numpy())
    s.advance(1)
    ref = s.get_dofs()
    side = torch.cuda.Stream()
    for which in ("side", "default", "null"):
        st = side if which == "side" else torch.cuda.default_stream()
        with torch.cuda.stream(st):
            d = torch.empty((m.nt, 9, s.B), dtype=torch.float64, device="cuda")
            d.copy_(Q0, non_blocking=True)                    # enqueued on st only
            handle = None if which == "null" else st.cuda_stream
            lib.adg_step_noalloc(s.ctx, d.data_ptr(), 1, handle)
            got = d.to("cpu", non_blocking=False).numpy()   # waits for st only
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-10, (which, err)


def test_noalloc_rejects_meshes_beyond_the_scratch_limit(lib):
    import torch
    m, s = _periodic_context(12, 5)         # 10368 tets at N=5: 63.7 MB of traces
    d = torch.zeros((m.nt, 9, s.B), dtype=torch.float64, device="cuda")
    with pytest.raises(lib.AdgError) as ei:
        lib.adg_step_noalloc(s.ctx, d.data_ptr(), 1)
    assert ei.value.code == -1 and "maximum" in str(ei.value)

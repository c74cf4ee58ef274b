"""The C ABI from plain C: tests/c_abi_caller.c includes include/adg.h, links
libadg.so and calls the host entry points (no GPU, no Python in the caller);
its time step equals the oracle's for the same 2 x 2 x 2 Kuhn box."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import synthetic as syn
from oracle.geometry import Geometry, cfl_dt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plain_c_caller(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2107_06640_gb300 import build
    lib = build.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "c_abi_caller")
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-O1", "-I" + os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_caller.c"), "-L" + libdir, "-ladg",
                    "-Wl,-rpath," + libdir, "-lm", "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    word, nt, ncl, dtmin = r.stdout.split()
    assert word == "ok" and int(nt) == 48 and int(ncl) == 1
    g = np.linspace(0.0, 1.0, 3)
    m = syn.kuhn_box(g, g, g)
    rho, lam, mu = syn.elastic_uniform(m.nt)
    want = cfl_dt(Geometry(m.xyz, m.tets, m.face_tag), rho, lam, mu, 3, 0.5).min()
    assert float(dtmin) == pytest.approx(want, rel=1e-14)

"""The CPU checks of the library's host set-up catch plausible mistakes in
it: each case compiles a copy of csrc/adg_host.cpp with one mistake planted,
links it with the other objects of the in-tree build into a library of its
own (in a temporary directory; nothing in the tree changes), and runs the
host tests against that library, which must then fail."""

import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2107_06640_gb300")
HOST = os.path.join(PKG, "csrc", "adg_host.cpp")

# (id, original text, planted text, host tests (-k expression in test_plan_host.py))
CASES = [
    ("middle-state-impedance", "Mm[0 * 9 + 0] = 1 - c / Zpp;", "Mm[0 * 9 + 0] = 1 - c / Zpm;", "face_flux"),
    ("jacobian-normal-stress", "A[0 * 9 + 6] = -(lam + 2 * mu);", "A[0 * 9 + 6] = -(lam + mu);", "face_flux"),
    ("rigid-wall-ghost", "else if (tag == ADG_TAG_RIGID) G = diag9({1, 1, 1, -1, 1, -1, -1, 1, 1});",
     "else if (tag == ADG_TAG_RIGID) G = diag9({-1, 1, 1, -1, 1, -1, 1, 1, 1});", "face_flux"),
    ("cfl-length", "h[e] = 6.0 * (det / 6.0) / asum;", "h[e] = 3.0 * (det / 6.0) / asum;", "plan_equals"),
    ("clusters-ignore-faults", "int lim = tag[4 * e + f] == ADG_TAG_FAULT ? cl[e2] : cl[e2] + 1;",
     "int lim = cl[e2] + 1;", "plan_equals"),
    ("orientation-reversed", "if (tets[4 * e2 + kFaceV[f2][s2]] == gv) sig[s] = s2;",
     "if (tets[4 * e2 + kFaceV[f2][s2]] == gv) sig[s] = (s2 + 1) % 3;", "node_maps"),
]

_CHILD = """
import sys
sys.path.insert(0, {root!r})
from paper_2107_06640_gb300 import _lib, build
build.build = lambda *a, **k: {lib!r}   # the test fixtures must not rebuild the in-tree library
_lib.LIB_PATH = {lib!r}
import pytest
sys.exit(pytest.main(["-q", "-x", "-p", "no:cacheprovider", {tests!r}, "-k", {sel!r}]))
"""


def _nvcc():
    return shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc")
                                    else None)


@pytest.fixture(scope="module")
def objects():
    from paper_2107_06640_gb300 import build
    build.build()
    obj = os.path.join(PKG, "_build")
    others = [os.path.join(obj, f) for f in sorted(os.listdir(obj))
              if f.endswith(".o") and f != "adg_host.cpp.o"]
    return others


def _run(case, others, tmp):
    name, old, new, sel = case
    src = open(HOST).read()
    if src.count(old) != 1:
        return None, f"{name}: the original text is not unique"
    d = os.path.join(tmp, name)
    os.makedirs(d)
    cpp = os.path.join(d, "adg_host.cpp")
    # compiled from the tree's own folder so that its relative includes resolve
    csrc = os.path.join(PKG, "csrc") + "/"
    open(cpp, "w").write(src.replace(old, new).replace('#include "', '#include "' + csrc))
    nvcc = _nvcc()
    o = os.path.join(d, "adg_host.o")
    lib = os.path.join(d, "libadg.so")
    c = subprocess.run([nvcc, "-O1", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fopenmp",
                        "-I" + os.path.join(ROOT, "include"), "-c", cpp, "-o", o], capture_output=True, text=True)
    if c.returncode != 0:
        return None, f"{name}: compile failed\n{c.stderr[-2000:]}"
    lk = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-Xcompiler", "-fopenmp",
                        "-o", lib, o, *others], capture_output=True, text=True)
    if lk.returncode != 0:
        return None, f"{name}: link failed\n{lk.stderr[-2000:]}"
    code = _CHILD.format(root=ROOT, lib=lib, tests=os.path.join(ROOT, "tests", "test_plan_host.py"), sel=sel)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-2000:] + r.stderr[-2000:]


# the same build without a planted mistake: the host checks pass, so the
# failures above come from the mistakes and not from the way the copy is built
CONTROL = ("control-unchanged", "h[e] = 6.0 * (det / 6.0) / asum;", "h[e] = 6.0 * (det / 6.0) / asum;",
           "plan_equals or face_flux or node_maps")


@pytest.fixture(scope="module")
def results(objects, tmp_path_factory):
    if _nvcc() is None:
        pytest.skip("nvcc not available")
    from concurrent.futures import ThreadPoolExecutor
    tmp = str(tmp_path_factory.mktemp("host_mutations"))
    cases = CASES + [CONTROL]
    with ThreadPoolExecutor(max_workers=max(1, min(7, os.cpu_count() or 1))) as ex:
        return dict(zip((c[0] for c in cases), ex.map(lambda c: _run(c, objects, tmp), cases)))


def test_the_unchanged_copy_passes_the_host_checks(results):
    rc, out = results[CONTROL[0]]
    assert rc == 0, out


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_host_mistake_fails_the_host_checks(case, results):
    rc, out = results[case[0]]
    assert rc == 1, f"{case[0]}: host checks did not fail (exit {rc})\n{out}"

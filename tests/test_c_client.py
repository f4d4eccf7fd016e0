"""The C ABI from a C99 program (tests/c_client/dgfs_client.c): the header
compiles as C with warnings as errors, the program links against the in-tree
library, and on a GPU the operator it gets through dgfs_collide_host matches
the oracle (FP64 to 1e-12, 3xTF32 to the form's 1e-5 of max |Q|)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1903_04670_gb300 import binding as B
from paper_1903_04670_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_client", "dgfs_client.c")


def _build(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(B.library_path())
    exe = str(tmp_path / "dgfs_client")
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-O1", "-I", os.path.join(ROOT, "include"),
           SRC, "-o", exe, "-L", libdir, "-ldgfs", "-Wl,-rpath," + libdir, "-lm"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    assert r.returncode == 0, r.stdout
    return exe


def test_c_client_compiles_links_and_runs_without_gpu(tmp_path):
    exe = _build(tmp_path)
    r = subprocess.run([exe, "info"], stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True, timeout=120)
    assert r.returncode == 0, r.stdout
    assert "sm_103a" in r.stdout
    assert "DGFS_OK DGFS_ETIMEOUT" in r.stdout
    assert "null" in r.stdout


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32_tc", 1e-5)])
def test_c_client_collide_matches_oracle(tmp_path, prec, tol):
    import oracle as O
    exe = _build(tmp_path)
    pb = W.make_problem("c1_homog_n16")
    N, S, P = pb["N"], len(pb["masses"]), pb["f"].shape[0]
    inp, out = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    with open(inp, "wb") as fh:
        fh.write(np.array([N, pb["M"], pb["Nrho"], S, P], dtype=np.int32).tobytes())
        fh.write(np.array([pb["L"]], dtype=np.float64).tobytes())
        fh.write(np.asarray(pb["masses"], dtype=np.float64).tobytes())
        fh.write(np.array([[p["omega"], p["alpha"], p.get("d", 1.0)] for p in pb["pairs"]],
                          dtype=np.float64).tobytes())
        f = pb["f"] if prec == "fp64" else pb["f"].astype(np.float32).astype(np.float64)
        fh.write(np.ascontiguousarray(f, dtype=np.float64).tobytes())
    r = subprocess.run([exe, "collide", prec, inp, out], stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stdout
    Q = np.fromfile(out, dtype=np.float64).reshape(P, S, S, N, N, N)
    prob = O.Problem(N, pb["L"], pb["M"], pb["Nrho"], pb["masses"], pb["pairs"])
    Qo = prob.collide_all(f)
    assert np.abs(Q - Qo).max() <= tol * np.abs(Qo).max()

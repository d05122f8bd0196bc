"""df64 (double-float) arithmetic of the mixed-precision step, against FP64.

The mixed kernels evaluate the source terms of their polish and of each substep's
start in df64 (csrc/tc_df64.cuh): pairs of FP32 numbers on the FP32 pipes instead of
FP64.  tests/host/tc_df64_check.cu runs the same header on the host and reports the
largest errors of each operation and of the physics' terms against FP64 over seeded
operands and over the cells of the slab and of random states; the GPU test runs the
arithmetic as the fast-math kernels compile it.  Bounds: ~2^-44 per operation (the
sloppy double-double forms and a two-digit division), exp relative error set by the
argument's own representation (|x| 2^-48, 1.2e-13 at x = 80), log absolute error a
few |log x| 2^-48 (the result's own representation and two additions); the rates and
terms within 1e-11 relative; the cooling function L within 1e-9 (it can be a
difference itself: the gas-dust term heats the gas where T_d > T, and cancels part of
the line cooling); the net H = n G - n^2 L, what the polish's residual and the
substep length use, within 1e-10 of its larger term on the host."""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import synthgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2210_08024_gb300", "csrc")
IN_KEYS = ("n", "chi_pe", "chi_lw", "f_h2", "f_c", "F_lyc", "xi", "Zg", "Zd", "T", "xH2", "xHp")

OP_BOUNDS = {"add": 3e-14, "mul": 3e-14, "div": 6e-14, "sqrt": 3e-14, "exp": 2e-13, "log_abs": 6e-13, "conv": 4e-15}
TERM_BOUNDS = {"chem_T": 1e-11, "cool_T": 1e-11, "xe": 1e-11, "G": 1e-11, "L": 1e-9, "H": 1e-10, "form": 1e-11,
               "dest": 1e-11, "ion": 1e-11, "rec": 1e-11, "Td": 1e-10}


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("df64") / "tc_df64_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-x", "cu", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                    os.path.join(ROOT, "tests", "host", "tc_df64_check.cu"), "-o", out], check=True, capture_output=True)
    return out


def _run(exe, cells, path):
    n = np.asarray(cells["T"]).size
    with open(path, "wb") as fh:
        fh.write(np.int64(n).tobytes())
        for k in IN_KEYS:
            fh.write(np.ascontiguousarray(np.broadcast_to(np.asarray(cells[k], np.float64), (n,))).tobytes())
        fh.write(np.float64(0.0).tobytes())
    return json.loads(subprocess.run([exe, str(path)], check=True, capture_output=True, text=True).stdout)


def _slab(k=8000, key=7):
    c = synthgen.slab()
    idx = np.sort(np.random.default_rng(key).choice(c["n"].size, k, replace=False))
    return synthgen.subset(c, idx)


WORKLOADS = {"slab": _slab, "random42": lambda: synthgen.cells_4096(n=8000, key=42),
             "random91": lambda: synthgen.cells_4096(n=8000, key=91)}


@pytest.mark.parametrize("workload", sorted(WORKLOADS))
def test_df64_host_errors_within_bounds(exe, tmp_path, workload):
    r = _run(exe, WORKLOADS[workload](), tmp_path / "cells.bin")
    assert r["saturates"] and r["underflow"]
    for k, b in {**OP_BOUNDS, **TERM_BOUNDS}.items():
        assert r[k] <= b, (k, r[k], b)


@pytest.fixture(scope="module")
def tc():
    import paper_2210_08024_gb300 as P
    P.build()
    from paper_2210_08024_gb300 import tc as T
    return T


@pytest.mark.gpu
def test_df64_device_matches_fp64(tc):
    # The kernels are built with flush-to-zero for FP32, but df64's own instructions
    # keep subnormals (PTX without .ftz), so its trailing parts survive down to FP32's
    # subnormal range: operands over the host test's ranges, and the last checks below
    # ~1e-31.
    import torch
    rng = np.random.default_rng(3)
    n = 1 << 18
    sgn = lambda: np.where(rng.random(n) < 0.5, -1.0, 1.0)
    a = sgn() * np.exp(rng.uniform(np.log(1e-15), np.log(1e15), n))
    b = sgn() * np.exp(rng.uniform(np.log(1e-15), np.log(1e15), n))
    x = rng.uniform(-70.0, 80.0, n)
    y = np.exp(rng.uniform(np.log(1e-30), np.log(1e30), n))
    dev = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    out = torch.empty(n, dtype=torch.float64, device="cuda")

    def run(op, u, v=None):
        tc.tc_df64_eval(op, dev(u), None if v is None else dev(v), out)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    rel = lambda g, r: np.max(np.abs(g - r) / np.abs(r))
    errs = {"add": np.max(np.abs(run("add", a, b) - (a + b)) / np.maximum(np.abs(a), np.abs(b))),
            "mul": rel(run("mul", a, b), a * b), "div": rel(run("div", a, b), a / b),
            "sqrt": rel(run("sqrt", np.abs(a)), np.sqrt(np.abs(a))), "exp": rel(run("exp", x), np.exp(x)),
            "log_abs": np.max(np.abs(run("log", y) - np.log(y)))}
    print("device df64 errors:", {k: "%.2e" % v for k, v in errs.items()})
    for k, v in errs.items():
        assert v <= OP_BOUNDS[k], (k, v)
    # saturation instead of infinities, as on the host
    e = run("exp", np.array([1000.0, -100.0] + [0.0] * (n - 2)))
    assert np.isfinite(e[0]) and abs(e[0] / np.exp(80.0) - 1.0) < 1e-12 and e[1] == 0.0
    # below 2e-31 the trailing part is subnormal: fewer bits, still far beyond FP32
    t = np.full(n, 1e-16)
    assert rel(run("mul", t, t), t * t) <= 1e-9
    assert rel(run("exp", np.full(n, -80.0)), np.exp(np.full(n, -80.0))) <= 1e-9
    assert np.max(np.abs(run("log", np.full(n, 1e-33)) - np.log(1e-33))) <= 1e-9


@pytest.mark.gpu
@pytest.mark.parametrize("workload", sorted(WORKLOADS))
def test_df64_source_terms_on_device(tc, workload):
    import torch
    c = WORKLOADS[workload]()
    d = tc.to_device(c)
    f = tc.make_fields(d)
    n = int(f.ncell)
    err = torch.zeros(5 * n, dtype=torch.float64, device="cuda")
    tc.tc_df64_source_check(tc.tc_params_default(tc.TC_MODE_MIXED), f, err)
    torch.cuda.synchronize()
    e = err.cpu().numpy().reshape(5, n)
    m = {k: float(np.max(e[i])) for i, k in enumerate(("H", "CH2", "CHp", "Td", "xe"))}
    print(workload, "device df64 source-term errors:", {k: "%.2e" % v for k, v in m.items()})
    assert np.all(np.isfinite(e))
    # the same bounds as on the host: df64 keeps its trailing parts on the device too
    bounds = {"H": TERM_BOUNDS["H"], "CH2": 1e-11, "CHp": 1e-11, "Td": TERM_BOUNDS["Td"], "xe": TERM_BOUNDS["xe"]}
    for k, b in bounds.items():
        assert m[k] <= b, (k, m[k], b)

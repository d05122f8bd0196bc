"""The library's step functions compiled for the host against the oracle, without a GPU.

tests/host/tc_hoststep.cu runs the device code's own substep functions (the paper's scheme,
coupled FP64 Newton with its Jacobian reuse, and the mixed FP32/FP64 solve) on the CPU,
cell by cell as one lane of the step kernel does, with the library's default
parameters read through the C ABI.  It is a test program outside libtc_gb300.so: a
change to the solver logic shows up here before any GPU run.  The GPU parity tests
remain the check of the kernels themselves (same code, compiled for sm_103a; the mixed
kernels there also use fast FP32 intrinsics)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import synthgen
from tests._parity import assert_fp64_parity, assert_mixed_parity, ulp_spread

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2210_08024_gb300", "csrc")
DT = synthgen.DT_1E4YR
IN_KEYS = ("n", "chi_pe", "chi_lw", "f_h2", "f_c", "F_lyc", "xi", "Zg", "Zd", "T", "xH2", "xHp")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("hoststep") / "tc_hoststep")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-x", "cu", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                    os.path.join(ROOT, "tests", "host", "tc_hoststep.cu"), "-o", out], check=True, capture_output=True)
    return out


@pytest.fixture(scope="module")
def tc():
    import paper_2210_08024_gb300 as P
    P.build()
    from paper_2210_08024_gb300 import tc as T
    return T


def host_step(exe, tc, cells, mode, tmp_path):
    n = np.asarray(cells["T"]).size
    src, dst = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    with open(src, "wb") as fh:
        fh.write(np.int64(n).tobytes())
        for k in IN_KEYS:
            fh.write(np.ascontiguousarray(np.broadcast_to(np.asarray(cells[k], np.float64), (n,))).tobytes())
        fh.write(np.float64(DT).tobytes())
    p = tc.tc_params_default(mode)
    args = [p.dvdr_kms_pc, p.T_cmb, p.chi0, p.opt_over_fuv, p.tau_opt_over_tau_pe, p.limiter, p.fd_rel_step,
            p.newton_rtol, p.newton_rtol_mixed, p.T_floor, p.newton_max, p.max_substeps, p.flags]
    subprocess.run([exe, src, dst, str(mode)] + [repr(a) for a in args], check=True)
    raw = np.fromfile(dst, dtype=np.uint8)
    d = raw[:48 * n].view(np.float64).reshape(6, n)
    i = raw[48 * n:].view(np.int32).reshape(3, n)
    return {"T": d[0], "xH2": d[1], "xHp": d[2], "xe": d[3], "xCp": d[4], "xCO": d[5],
            "nsub": i[0], "status": i[1], "iters": i[2]}


def _slab(k, key):
    c = synthgen.slab()
    idx = np.sort(np.random.default_rng(key).choice(c["n"].size, k, replace=False))
    return synthgen.subset(c, idx)


WORKLOADS = {"slab": lambda: _slab(2048, 4242), "random": lambda: synthgen.cells_4096(n=2048, key=91)}


@pytest.mark.parametrize("workload", sorted(WORKLOADS))
def test_host_newton_fp64_matches_oracle(exe, tc, tmp_path, workload):
    c = WORKLOADS[workload]()
    ref = oracle.step(c, DT, oracle.default_params(mode=1))
    g = host_step(exe, tc, c, tc.TC_MODE_NEWTON_FP64, tmp_path)
    assert np.array_equal(g["status"] & tc.TC_ST_ERROR_MASK, ref["status"] & tc.TC_ST_ERROR_MASK)
    assert np.array_equal(g["nsub"], ref["nsub"])
    assert_fp64_parity(g, ref, "host mode1 " + workload)
    for k in ("xe", "xCp", "xCO"):
        np.testing.assert_allclose(g[k], ref[k], rtol=1e-8, atol=1e-14, err_msg=k)


@pytest.mark.parametrize("workload", sorted(WORKLOADS))
def test_host_paper_scheme_matches_oracle(exe, tc, tmp_path, workload):
    c = WORKLOADS[workload]()
    ref, spread = ulp_spread(oracle, c, DT, oracle.default_params(mode=0))
    g = host_step(exe, tc, c, tc.TC_MODE_PAPER_FP64, tmp_path)
    assert_fp64_parity(g, ref, "host mode0 " + workload, spread=spread)
    assert np.mean(g["nsub"] != ref["nsub"]) < 0.01


@pytest.mark.parametrize("workload", sorted(WORKLOADS))
def test_host_mixed_matches_oracle(exe, tc, tmp_path, workload):
    c = WORKLOADS[workload]()
    ref = oracle.step(c, DT, oracle.default_params(mode=1))
    g = host_step(exe, tc, c, tc.TC_MODE_MIXED, tmp_path)
    # no substep is halved on either side: both integrate on the same substep grid
    assert np.all((g["status"] & tc.TC_ST_ERROR_MASK) == 0)
    assert np.all((ref["status"] & tc.TC_ST_ERROR_MASK) == 0)
    assert np.array_equal(g["nsub"], ref["nsub"])
    assert_mixed_parity(g, ref, "host mixed " + workload)


@pytest.mark.parametrize("key", [42, 43])
def test_host_newton_fp64_strict_on_hot_random_states(exe, tc, tmp_path, key):
    # The random states of keys 42 and 43 hold the hot molecular cells whose Newton
    # solve from the start state fails and is restarted from the block predictor; the
    # kernels' solver must land on the oracle's roots there too, at the plain bound.
    c = synthgen.cells_4096(n=4096, key=key)
    ref = oracle.step(c, DT, oracle.default_params(mode=1))
    assert np.any(ref["status"] & oracle.ST_PREDICTOR)
    g = host_step(exe, tc, c, tc.TC_MODE_NEWTON_FP64, tmp_path)
    assert np.array_equal(g["status"] & tc.TC_ST_ERROR_MASK, ref["status"] & tc.TC_ST_ERROR_MASK)
    assert np.array_equal(g["nsub"], ref["nsub"])
    assert_fp64_parity(g, ref, "host mode1 key %d" % key)

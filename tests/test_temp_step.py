"""The temperature blocks stepped to T + dT (the FP64 Newton Jacobian's temperature
column) against chem_T and cool_T evaluated at T + dT, field by field, on the host build
of the library's own physics header (tests/host/tc_temp_step_check.cu).

Every field's change over dT = 1e-7 T must agree with the exact change up to the step's
second-order term (normalised error below 1), at the cells' own temperatures and on a
sweep from 12 K to 1e7 K, with the physics switches off and on.  A wrong coefficient,
sign or missing term in one field's logarithmic derivative makes its error of order
1/|g| (1e3 to 1e7 here).

The same program checks the C/O/e root's x_C+ and ln psi, which the root solve takes
from its last evaluation stepped to the root instead of evaluating them afresh.
"""
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
ROOT_BOUNDS = {"lpsi_converged": 1e-14, "capped_xe": 1e-13, "capped_xCp": 1e-12, "capped_lpsi": 1e-12}


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("tstep") / "tc_temp_step_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-x", "cu", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                    os.path.join(ROOT, "tests", "host", "tc_temp_step_check.cu"), "-o", out],
                   check=True, capture_output=True)
    return out


def _run(exe, cells, path):
    n = np.asarray(cells["T"]).size
    with open(path, "wb") as fh:
        fh.write(np.int64(n).tobytes())
        for k in IN_KEYS:
            fh.write(np.ascontiguousarray(np.broadcast_to(np.asarray(cells[k], np.float64), (n,))).tobytes())
        fh.write(np.float64(0.0).tobytes())
    return json.loads(subprocess.run([exe, str(path)], check=True, capture_output=True, text=True).stdout)


def _slab(k=400, key=11):
    c = synthgen.slab()
    idx = np.sort(np.random.default_rng(key).choice(c["n"].size, k, replace=False))
    return synthgen.subset(c, idx)


@pytest.mark.parametrize("workload", ["slab", "random42"])
def test_stepped_blocks_match_the_blocks_at_t_plus_dt(exe, tmp_path, workload):
    cells = _slab() if workload == "slab" else synthgen.cells_4096(n=400, key=42)
    r = _run(exe, cells, tmp_path / "cells.bin")
    assert r.pop("checks") == 400 * 12 * 2
    root = {k: r.pop(k) for k in ROOT_BOUNDS}
    bad = {k: v for k, v in r.items() if not v < 1.0}
    assert not bad, bad
    # the C/O/e root's x_C+ and ln psi, stepped from the solve's last evaluation: to
    # rounding when converged, ~1e-14 after one capped step from 1e-7 off the root (a
    # wrong sign or derivative in the step would leave ~1e-7)
    for k, bound in ROOT_BOUNDS.items():
        assert root[k] <= bound, (k, root[k], bound)

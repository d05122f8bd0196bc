"""C ABI checks that need no GPU: the library loads, exports every entry point that
include/*.h declares, its ctypes mirrors have the C layout, and arguments are
validated before any device work."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tc():
    import paper_2210_08024_gb300 as P
    P.build()
    from paper_2210_08024_gb300 import tc as T
    return T


def _declared():
    names = set()
    for h in sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[a-z_]+\s*\**\s*(tc_[a-z_0-9]+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(tc):
    names = _declared()
    assert "tc_step" in names and "tc_create" in names and len(names) >= 10
    for n in names:
        assert hasattr(tc.lib, n), n


def test_struct_layout_matches_header(tc):
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "tc.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(tc_params), sizeof(tc_fields), offsetof(tc_params, flags),
         offsetof(tc_params, blocks_per_sm), offsetof(tc_fields, ncell), offsetof(tc_fields, Zd_val));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "l.c")
        open(c, "w").write(src)
        exe = os.path.join(td, "l")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    exp = [ctypes.sizeof(tc.tc_params), ctypes.sizeof(tc.tc_fields), tc.tc_params.flags.offset,
           tc.tc_params.blocks_per_sm.offset, tc.tc_fields.ncell.offset, tc.tc_fields.Zd_val.offset]
    assert vals == exp


def test_defaults_and_errors(tc):
    p = tc.tc_params_default(tc.TC_MODE_MIXED)
    assert p.limiter == 0.1 and p.fd_rel_step == 1e-3 and p.mode == tc.TC_MODE_MIXED and p.T_cmb == 2.73
    assert tc.tc_strerror(tc.TC_EINVAL) == "invalid argument"
    assert tc.lib.tc_step(None, None, 1.0, None) == tc.TC_EINVAL
    assert tc.lib.tc_create(None, None) == tc.TC_EINVAL
    bad = tc.tc_params_default(0)
    bad.mode = 17
    h = ctypes.c_void_p()
    assert tc.lib.tc_create(ctypes.byref(bad), ctypes.byref(h)) == tc.TC_EINVAL
    assert tc.lib.tc_peak_launch(99, 1, 32, 1, None, None) == tc.TC_EINVAL
    assert tc.lib.tc_df64_eval(7, None, None, None, 1, None) == tc.TC_EINVAL
    assert tc.lib.tc_df64_eval(0, None, None, None, 4, None) == tc.TC_EINVAL
    assert tc.lib.tc_df64_eval(4, None, None, None, 0, None) == tc.TC_OK


def _layout(src):
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "l.c")
        open(c, "w").write(src)
        exe = os.path.join(td, "l")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        return [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]


def test_driver_struct_layouts_match_headers(tc):
    vals = _layout(r'''
#include <stdio.h>
#include <stddef.h>
#include "tc_onezone.h"
#include "tc_pdr.h"
#include "tc_sixray.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(tc_eq_spec), sizeof(tc_eq_out), offsetof(tc_eq_spec, ncurve),
         offsetof(tc_eq_spec, nchunk), offsetof(tc_eq_spec, T_init), offsetof(tc_eq_spec, xHp_init),
         offsetof(tc_eq_out, i_min));
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(tc_pdr_spec), sizeof(tc_pdr_out), offsetof(tc_pdr_spec, ncell),
         offsetof(tc_pdr_spec, nchunk), offsetof(tc_pdr_spec, xHp_init), offsetof(tc_pdr_out, N_trans),
         sizeof(tc_sixray_grid));
  return 0;
}''')
    S, O, P, Q = tc.tc_eq_spec, tc.tc_eq_out, tc.tc_pdr_spec, tc.tc_pdr_out
    exp = [ctypes.sizeof(S), ctypes.sizeof(O), S.ncurve.offset, S.nchunk.offset, S.T_init.offset,
           S.xHp_init.offset, O.i_min.offset,
           ctypes.sizeof(P), ctypes.sizeof(Q), P.ncell.offset, P.nchunk.offset, P.xHp_init.offset, Q.N_trans.offset,
           ctypes.sizeof(tc.tc_sixray_grid)]
    assert vals == exp


def test_driver_defaults_and_argument_errors(tc):
    s = tc.tc_eq_spec()
    assert tc.lib.tc_eq_spec_default(ctypes.byref(s)) == tc.TC_OK
    assert (s.L_shld0_pc, s.n_shld0, s.a_shld, s.nchunk, s.T_init) == (5.0, 1e2, 0.7, 10, 3000.0)
    assert s.t_end_s == pytest.approx(1e2 * 1e6 * 3.15576e7)
    assert tc.lib.tc_eq_spec_default(None) == tc.TC_EINVAL
    assert tc.lib.tc_eq_curves(None, ctypes.byref(s), None, None) == tc.TC_EINVAL
    p = tc.tc_pdr_spec()
    assert tc.lib.tc_pdr_spec_default(ctypes.byref(p)) == tc.TC_OK
    assert (p.nchunk, p.T_init, p.xHp_init) == (300, 100.0, 1e-4)
    assert tc.lib.tc_pdr(None, ctypes.byref(p), None, None) == tc.TC_EINVAL
    g = tc.tc_sixray_grid(0, 1, 1, 1.0, 1.0, 2e-16, 1.0)
    assert tc.lib.tc_sixray(ctypes.byref(g), None, None, None, None, None, None, None, None) == tc.TC_EINVAL
    g = tc.tc_sixray_grid(2, 2, 2, 1.0, 1.0, 2e-16, 1.0)
    assert tc.lib.tc_sixray(ctypes.byref(g), None, None, None, None, None, None, None, None) == tc.TC_EINVAL

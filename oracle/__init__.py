"""CPU FP64 oracle for the per-cell thermochemistry step of arXiv:2210.08024.

TEST INFRASTRUCTURE ONLY: the plain, slow statement of what the step computes, used
to check the CUDA library.  Only tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline leg may import it; the library product path never does, and the oracle
shares no code with the CUDA path.

Mode 0 is the paper's sequential scheme (Sec. 6.1): linearised backward Euler for
T_mu with a finite-difference derivative, then backward Euler for (x_H2, x_H+), then
the C/O/e equilibrium.  Mode 1 is the coupled implicit alternative the same section
names: backward Euler on (T_mu, x_H2, x_H+) solved by Newton's method.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, f) for f in ("tc_oracle.cpp", "tc_oracle.hpp", "tc_opcount.hpp")]

F_CONST_KGR = 1
F_NO_ROVIB = 2
F_NO_CIE = 4
F_FREEZE_T = 256
F_PREDICTOR = 512

ST_OK, ST_MAX_SUBSTEPS, ST_NEWTON, ST_NONFINITE, ST_PREDICTOR = 0, 1, 2, 4, 32

YEAR_S = 3.15576e7

TERM_NAMES = [
    "xe", "xCp", "xCO", "xC", "xO", "xOp", "xMHp",
    "kgr", "zcrH2", "zcrH", "zpd", "zpiH", "zpiH2", "zcd", "zci", "arr",
    "agr", "kci", "kcdH", "kcdH2",
    "G_pe", "G_cr", "G_pi", "G_h2form", "G_h2pump", "G_h2pd", "G_total",
    "L_lya", "L_ci", "L_cd", "L_rovib", "L_ff", "L_rr", "L_hyd",
    "L_Cp", "L_C", "L_O", "L_CO", "L_grrec", "L_neb", "L_gd", "L_cie",
    "S", "L_total", "Td", "H", "CH2", "CHp",
]
PREP_NAMES = ["G0", "zpd", "zpiH", "zpiH2", "zpiC_rad", "zcrC", "lnCO", "qH2", "Gd", "xCtot", "xOtot", "muH", "K"]
OP_NAMES = ["add", "mul", "div", "sqrt", "exp", "log", "pow", "cmp"]


class Params(ctypes.Structure):
    _fields_ = [
        ("dvdr_kms_pc", ctypes.c_double),
        ("T_cmb", ctypes.c_double),
        ("chi0", ctypes.c_double),
        ("opt_over_fuv", ctypes.c_double),
        ("tau_opt_over_tau_pe", ctypes.c_double),
        ("limiter", ctypes.c_double),
        ("fd_rel_step", ctypes.c_double),
        ("newton_rtol", ctypes.c_double),
        ("T_floor", ctypes.c_double),
        ("newton_max", ctypes.c_int),
        ("max_substeps", ctypes.c_int),
        ("mode", ctypes.c_int),
        ("flags", ctypes.c_uint),
    ]


def default_params(mode: int = 0, **kw) -> Params:
    """Defaults: |dv/dr| = 1 km/s/pc, T_CMB = 2.73 K, chi0 = 1, E_OPT,0 = E_FUV,0,
    tau_OPT = tau_PE/3 (Sec. 4.3.6), limiter 0.1 (Sec. 6.1), FD step 1e-3 (READING), Newton
    rtol 1e-12 (50 iterations), T floor 1 K, at most 10^6 substeps."""
    p = Params(1.0, 2.73, 1.0, 1.0, 1.0 / 3.0, 0.1, 1e-3, 1e-12, 1.0, 50, 1000000, mode, 0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class _Fields(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in (
        "n", "chi_pe", "chi_lw", "f_h2", "f_c", "F_lyc", "xi", "Zg", "Zd",
        "T", "xH2", "xHp", "xe", "xCp", "xCO", "nsub", "status", "newton_iters")]


def build(force: bool = False) -> str:
    """Compiles liboracle.so with g++ (plain FP64, no FP contraction, OpenMP)."""
    newest = max(os.path.getmtime(s) for s in _SRC)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, os.path.join(_HERE, "tc_oracle.cpp")]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.oracle_step.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(_Fields), ctypes.c_longlong,
                                  ctypes.c_double, ctypes.c_int]
        L.oracle_opcount.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(_Fields), ctypes.c_longlong,
                                     ctypes.c_double, ctypes.POINTER(ctypes.c_ulonglong)]
        L.oracle_terms.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_double)]
        L.oracle_prepare.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]
        L.oracle_rk45.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_longlong)]
        _lib = L
    return _lib


CELL_KEYS = ("n", "chi_pe", "chi_lw", "f_h2", "f_c", "F_lyc", "xi", "Zg", "Zd")
STATE_KEYS = ("T", "xH2", "xHp")


def _c64(a, n):
    a = np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), (n,)))
    return a


def _prepare_fields(cells: dict):
    n = max(int(np.asarray(cells[k]).size) for k in CELL_KEYS + STATE_KEYS)
    keep = {k: _c64(cells[k], n) for k in CELL_KEYS}
    out = {k: np.array(_c64(cells[k], n), copy=True) for k in STATE_KEYS}
    for k in ("xe", "xCp", "xCO"):
        out[k] = np.zeros(n)
    for k in ("nsub", "status", "newton_iters"):
        out[k] = np.zeros(n, dtype=np.int32)
    f = _Fields(*([keep[k].ctypes.data for k in CELL_KEYS] +
                  [out[k].ctypes.data for k in STATE_KEYS + ("xe", "xCp", "xCO", "nsub", "status", "newton_iters")]))
    return n, f, keep, out


def step(cells: dict, dt: float, params: Params | None = None, nthreads: int = 0) -> dict:
    """Runs one step over dt seconds for every cell.  ``cells`` maps CELL_KEYS and
    STATE_KEYS to arrays (scalars broadcast).  Returns a dict with T, xH2, xHp, xe, xCp,
    xCO, nsub, status, newton_iters."""
    p = params if params is not None else default_params()
    n, f, keep, out = _prepare_fields(cells)
    rc = lib().oracle_step(ctypes.byref(p), ctypes.byref(f), n, float(dt), int(nthreads))
    if rc != 0:
        raise RuntimeError("oracle_step failed: %d" % rc)
    return out


def opcount(cells: dict, dt: float, params: Params | None = None) -> dict:
    """Algorithmic FP64 operation counts of one step summed over the cells."""
    p = params if params is not None else default_params()
    n, f, keep, out = _prepare_fields(cells)
    counts = (ctypes.c_ulonglong * 8)()
    rc = lib().oracle_opcount(ctypes.byref(p), ctypes.byref(f), n, float(dt), counts)
    if rc != 0:
        raise RuntimeError("oracle_opcount failed: %d" % rc)
    d = {k: int(counts[i]) for i, k in enumerate(OP_NAMES)}
    d["result"] = out
    return d


def _cellvec(cell: dict):
    return (ctypes.c_double * 9)(*[float(cell.get(k, DEFAULT_CELL[k])) for k in CELL_KEYS])


DEFAULT_CELL = dict(n=1.0, chi_pe=1.0, chi_lw=1.0, f_h2=1.0, f_c=1.0, F_lyc=0.0, xi=2e-16, Zg=1.0, Zd=1.0)


def terms(cell: dict, T: float, xH2: float, xHp: float, params: Params | None = None, Td: float = -1.0) -> dict:
    """Every rate, heating and cooling term and the equilibrium abundances at one state."""
    p = params if params is not None else default_params()
    out = (ctypes.c_double * len(TERM_NAMES))()
    lib().oracle_terms(ctypes.byref(p), _cellvec(cell), float(T), float(xH2), float(xHp), float(Td), out)
    return {k: out[i] for i, k in enumerate(TERM_NAMES)}


def prepared(cell: dict, params: Params | None = None) -> dict:
    p = params if params is not None else default_params()
    out = (ctypes.c_double * len(PREP_NAMES))()
    lib().oracle_prepare(ctypes.byref(p), _cellvec(cell), out)
    return {k: out[i] for i, k in enumerate(PREP_NAMES)}


def rk45(cell: dict, T: float, xH2: float, xHp: float, dt: float, params: Params | None = None,
         rtol: float = 1e-10, atol_x: float = 1e-14, max_steps: int = 5_000_000):
    """Tight-tolerance Dormand-Prince integration of the underlying DAE; returns
    ((T, xH2, xHp), steps)."""
    p = params if params is not None else default_params()
    out = (ctypes.c_double * 3)()
    ns = ctypes.c_longlong(0)
    rc = lib().oracle_rk45(ctypes.byref(p), _cellvec(cell), float(T), float(xH2), float(xHp), float(dt),
                           float(rtol), float(atol_x), int(max_steps), out, ctypes.byref(ns))
    if rc != 0:
        raise RuntimeError("rk45 did not reach dt (rc=%d, steps=%d)" % (rc, ns.value))
    return (out[0], out[1], out[2]), ns.value

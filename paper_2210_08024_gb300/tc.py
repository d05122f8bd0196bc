"""ctypes binding of the C ABI in include/tc.h (argument marshalling only).

Function names match the C entry points.  Device buffers are torch CUDA tensors (or
raw device addresses); every step of the computation runs in the library's CUDA
kernels.  If the library cannot be loaded the import fails: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtc_gb300.so")

TC_OK, TC_EINVAL, TC_ECUDA, TC_ENOMEM, TC_ENOMLP, TC_ENODEV = 0, -1, -2, -3, -4, -5
TC_MODE_PAPER_FP64, TC_MODE_NEWTON_FP64, TC_MODE_MIXED, TC_MODE_MIXED_SEEDED, TC_MODE_NEWTON_FP64_SEEDED = 0, 1, 2, 3, 4
TC_CONST_KGR, TC_NO_ROVIB, TC_NO_CIE = 1, 2, 4
TC_ST_MAX_SUBSTEPS, TC_ST_NEWTON, TC_ST_NONFINITE, TC_ST_FALLBACK, TC_ST_POLISHED, TC_ST_PREDICTOR = 1, 2, 4, 8, 16, 32
TC_ST_SEEDED, TC_ST_SEED_FAIL = 64, 128
TC_ST_ERROR_MASK = 7


class tc_params(ctypes.Structure):
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
        ("newton_rtol_mixed", ctypes.c_double),
        ("block", ctypes.c_int),
        ("blocks_per_sm", ctypes.c_int),
        ("order_cells", ctypes.c_int),
        ("lanes_per_cell", ctypes.c_int),
    ]


class tc_tune_choice(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("blocks_per_sm", ctypes.c_int), ("lanes_per_cell", ctypes.c_int),
                ("ms", ctypes.c_float)]


_P = ctypes.c_void_p


class tc_fields(ctypes.Structure):
    _fields_ = [
        ("n", _P), ("chi_pe", _P), ("chi_lw", _P), ("f_shld_h2", _P), ("f_shld_c", _P), ("F_lyc", _P),
        ("xi_cr", _P), ("Zg", _P), ("Zd", _P),
        ("T", _P), ("x_h2", _P), ("x_hp", _P),
        ("x_e", _P), ("x_cp", _P), ("x_co", _P),
        ("nsub", _P), ("status", _P),
        ("ncell", ctypes.c_longlong),
        ("Zg_val", ctypes.c_double), ("Zd_val", ctypes.c_double),
        ("newton_iters", _P), ("cost_hint", _P),
    ]


# field name in tc_fields -> key used by callers' dicts
FIELD_KEYS = {
    "n": "n", "chi_pe": "chi_pe", "chi_lw": "chi_lw", "f_shld_h2": "f_h2", "f_shld_c": "f_c", "F_lyc": "F_lyc",
    "xi_cr": "xi", "Zg": "Zg", "Zd": "Zd", "T": "T", "x_h2": "xH2", "x_hp": "xHp", "x_e": "xe", "x_cp": "xCp",
    "x_co": "xCO", "nsub": "nsub", "status": "status", "newton_iters": "iters", "cost_hint": "cost_hint",
}


class tc_eq_spec(ctypes.Structure):
    """include/tc_onezone.h: the one-zone grid (host arrays) and integration settings."""
    _fields_ = [
        ("n_axis", ctypes.c_void_p), ("nn", ctypes.c_longlong),
        ("chi0", ctypes.c_void_p), ("xi0", ctypes.c_void_p), ("Zg", ctypes.c_void_p), ("Zd", ctypes.c_void_p),
        ("ncurve", ctypes.c_int), ("shielded", ctypes.c_int),
        ("L_shld0_pc", ctypes.c_double), ("n_shld0", ctypes.c_double), ("a_shld", ctypes.c_double),
        ("t_end_s", ctypes.c_double), ("nchunk", ctypes.c_int),
        ("T_init", ctypes.c_double), ("xH2_init", ctypes.c_double), ("xHp_init", ctypes.c_double),
    ]


class tc_eq_out(ctypes.Structure):
    """include/tc_onezone.h: device output arrays, curve-major."""
    _fields_ = [(k, ctypes.c_void_p) for k in ("T", "x_h2", "x_hp", "x_e", "P_k", "x_co", "chg", "status",
                                                "i_max", "i_min")]


class tc_pdr_spec(ctypes.Structure):
    """include/tc_pdr.h: per-slab parameters (host arrays) and integration settings."""
    _fields_ = [
        ("n", ctypes.c_void_p), ("chi0", ctypes.c_void_p), ("xi0", ctypes.c_void_p), ("Z", ctypes.c_void_p),
        ("dx_cm", ctypes.c_void_p), ("nslab", ctypes.c_int), ("ncell", ctypes.c_longlong),
        ("t_end_s", ctypes.c_double), ("nchunk", ctypes.c_int),
        ("T_init", ctypes.c_double), ("xH2_init", ctypes.c_double), ("xHp_init", ctypes.c_double),
    ]


class tc_pdr_out(ctypes.Structure):
    """include/tc_pdr.h: device outputs, slab-major."""
    _fields_ = [(k, ctypes.c_void_p) for k in ("T", "x_h2", "x_hp", "x_e", "x_co", "chi_pe", "f_shld_h2", "N_c",
                                                "status", "N_trans")]


class tc_sixray_grid(ctypes.Structure):
    """include/tc_sixray.h: grid shape, cell size and the unattenuated fields."""
    _fields_ = [("nx", ctypes.c_longlong), ("ny", ctypes.c_longlong), ("nz", ctypes.c_longlong),
                ("dx_cm", ctypes.c_double), ("chi0", ctypes.c_double), ("xi0", ctypes.c_double),
                ("Zd", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libtc_gb300.so is not built (run __graft_entry__.build()); no CPU fallback exists")
    L = ctypes.CDLL(LIB_PATH)
    L.tc_params_default.argtypes = [ctypes.POINTER(tc_params), ctypes.c_int]
    L.tc_create.argtypes = [ctypes.POINTER(tc_params), ctypes.POINTER(ctypes.c_void_p)]
    L.tc_step.argtypes = [ctypes.c_void_p, ctypes.POINTER(tc_fields), ctypes.c_double, ctypes.c_void_p]
    L.tc_step_host.argtypes = [ctypes.c_void_p, ctypes.POINTER(tc_fields), ctypes.c_double, ctypes.c_void_p]
    L.tc_seed_predict.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    L.tc_rates.argtypes = [ctypes.c_void_p, ctypes.POINTER(tc_fields), ctypes.c_double, ctypes.c_void_p,
                           ctypes.c_void_p, ctypes.c_void_p]
    L.tc_autotune.argtypes = [ctypes.c_void_p, ctypes.POINTER(tc_fields), ctypes.c_double, ctypes.c_void_p,
                              ctypes.POINTER(tc_tune_choice)]
    L.tc_step_batch.argtypes = [ctypes.c_void_p, ctypes.POINTER(tc_fields), ctypes.c_int, ctypes.c_double,
                                ctypes.c_void_p]
    L.tc_load_mlp.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
    L.tc_sync_status.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p,
                                 ctypes.POINTER(ctypes.c_longlong)]
    L.tc_launch_count.argtypes = [ctypes.c_void_p]
    L.tc_launch_count.restype = ctypes.c_longlong
    L.tc_strerror.argtypes = [ctypes.c_int]
    L.tc_strerror.restype = ctypes.c_char_p
    L.tc_destroy.argtypes = [ctypes.c_void_p]
    L.tc_destroy.restype = None
    L.tc_peak_launch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                 ctypes.c_void_p]
    L.tc_peak_chains.restype = ctypes.c_int
    L.tc_df64_eval.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong,
                               ctypes.c_void_p]
    L.tc_df64_source_check.argtypes = [ctypes.POINTER(tc_params), ctypes.POINTER(tc_fields), ctypes.c_void_p,
                                       ctypes.c_void_p]
    L.tc_step_host_static.argtypes = [ctypes.POINTER(tc_params), ctypes.POINTER(tc_fields), ctypes.c_double,
                                      ctypes.c_void_p]
    # seed network (include/tc_mlp.h)
    L.tc_mlp_n_params.restype = ctypes.c_int
    L.tc_mlp_create.argtypes = [ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_void_p)]
    L.tc_mlp_destroy.argtypes = [ctypes.c_void_p]
    L.tc_mlp_destroy.restype = None
    L.tc_mlp_set_norm.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.tc_mlp_set_params.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.tc_mlp_get_params.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.tc_mlp_predict.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    L.tc_mlp_grad.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.tc_mlp_train_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]
    L.tc_mlp_blob_bytes.restype = ctypes.c_size_t
    L.tc_sixray.argtypes = [ctypes.POINTER(tc_sixray_grid)] + [ctypes.c_void_p] * 8
    L.tc_pdr_spec_default.argtypes = [ctypes.POINTER(tc_pdr_spec)]
    L.tc_pdr.argtypes = [ctypes.c_void_p, ctypes.POINTER(tc_pdr_spec), ctypes.POINTER(tc_pdr_out), ctypes.c_void_p]
    L.tc_eq_spec_default.argtypes = [ctypes.POINTER(tc_eq_spec)]
    L.tc_eq_curves.argtypes = [ctypes.c_void_p, ctypes.POINTER(tc_eq_spec), ctypes.POINTER(tc_eq_out), ctypes.c_void_p]
    L.tc_mlp_export.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
    return L


lib = _load()


class TcError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != TC_OK:
        raise TcError("%s failed: %s (%d)" % (what, lib.tc_strerror(rc).decode(), rc))


def tc_strerror(code: int) -> str:
    return lib.tc_strerror(code).decode()


def tc_params_default(mode: int = TC_MODE_PAPER_FP64, **kw) -> tc_params:
    p = tc_params()
    _check(lib.tc_params_default(ctypes.byref(p), int(mode)), "tc_params_default")
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def tc_create(params: tc_params) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib.tc_create(ctypes.byref(params), ctypes.byref(h)), "tc_create")
    return h


def tc_destroy(h) -> None:
    lib.tc_destroy(h)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def make_fields(arrs: dict, ncell: int | None = None, Zg: float = 1.0, Zd: float = 1.0) -> tc_fields:
    """Builds tc_fields from a dict of torch tensors (device, float64 / int32) keyed as
    in FIELD_KEYS' values.  The caller keeps the tensors alive during the call."""
    f = tc_fields()
    n = ncell
    for cname, key in FIELD_KEYS.items():
        t = arrs.get(key)
        if t is None:
            setattr(f, cname, None)
            continue
        if hasattr(t, "data_ptr"):
            if not t.is_contiguous():
                raise ValueError("field %s must be contiguous" % key)
            if n is None:
                n = t.numel()
            setattr(f, cname, t.data_ptr())
        else:
            setattr(f, cname, int(t))
    f.ncell = int(n if n is not None else 0)
    f.Zg_val = float(Zg)
    f.Zd_val = float(Zd)
    return f


def make_host_fields(arrs: dict, Zg: float = 1.0, Zd: float = 1.0) -> tc_fields:
    """tc_fields over host numpy arrays (for tc_step_host)."""
    f = tc_fields()
    n = None
    for cname, key in FIELD_KEYS.items():
        a = arrs.get(key)
        if a is None:
            setattr(f, cname, None)
            continue
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("field %s must be contiguous" % key)
        n = a.size if n is None else n
        setattr(f, cname, a.ctypes.data)
    f.ncell = int(n or 0)
    f.Zg_val = float(Zg)
    f.Zd_val = float(Zd)
    return f


def tc_seed_predict(h, X, out, stream=None) -> None:
    """The seeded kernels' tensor-core inference of the loaded network on X (device
    float32 [B, 13]) into out (device float32 [B, 3])."""
    _check(lib.tc_seed_predict(h, _ptr(X), int(X.shape[0]), _ptr(out), _stream_ptr(stream)), "tc_seed_predict")


def tc_rates(h, fields: tc_fields, dt: float, rate=None, dts=None, stream=None) -> None:
    """Start-state source terms (C_H2, C_H+, H/(K T_mu)) into `rate` (device float64,
    3 per cell) and the first substep length of a step of dt into `dts` (device
    float64), either may be None."""
    _check(lib.tc_rates(h, ctypes.byref(fields), float(dt), _ptr(rate), _ptr(dts), _stream_ptr(stream)), "tc_rates")


def tc_autotune(h, fields: tc_fields, dt: float, stream=None) -> dict:
    """Times the candidate launch shapes on the cells of `fields` (not modified) and
    records the fastest in the handle for their size class; returns it."""
    c = tc_tune_choice()
    _check(lib.tc_autotune(h, ctypes.byref(fields), float(dt), _stream_ptr(stream), ctypes.byref(c)), "tc_autotune")
    return {"block": c.block, "blocks_per_sm": c.blocks_per_sm, "lanes_per_cell": c.lanes_per_cell, "ms": c.ms}


def tc_step(h, fields: tc_fields, dt: float, stream=None) -> None:
    _check(lib.tc_step(h, ctypes.byref(fields), float(dt), _stream_ptr(stream)), "tc_step")


def tc_step_host(h, fields: tc_fields, dt: float, stream=None) -> None:
    _check(lib.tc_step_host(h, ctypes.byref(fields), float(dt), _stream_ptr(stream)), "tc_step_host")


TC_STATIC_MAX_CELLS = 65536


def tc_step_host_static(params: tc_params, fields: tc_fields, dt: float, stream=None) -> None:
    """tc_step_host without a handle and without any device allocation: for callers
    that hold host arrays but may not allocate device memory.  The library's static
    device scratch holds at most TC_STATIC_MAX_CELLS cells; calls share it, so calls
    that overlap on the GPU race."""
    if fields.ncell > TC_STATIC_MAX_CELLS:
        raise ValueError("tc_step_host_static: ncell %d exceeds the static scratch capacity of %d cells"
                         % (fields.ncell, TC_STATIC_MAX_CELLS))
    _check(lib.tc_step_host_static(ctypes.byref(params), ctypes.byref(fields), float(dt), _stream_ptr(stream)),
           "tc_step_host_static")


def tc_step_batch(h, boxes: list, dt: float, stream=None) -> None:
    arr = (tc_fields * len(boxes))(*boxes)
    _check(lib.tc_step_batch(h, arr, len(boxes), float(dt), _stream_ptr(stream)), "tc_step_batch")


def tc_load_mlp(h, blob: bytes) -> None:
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(lib.tc_load_mlp(h, buf, len(blob)), "tc_load_mlp")


def tc_sync_status(h, status_tensor, stream=None) -> int:
    nbad = ctypes.c_longlong(0)
    _check(lib.tc_sync_status(h, status_tensor.data_ptr(), status_tensor.numel(), _stream_ptr(stream),
                              ctypes.byref(nbad)), "tc_sync_status")
    return int(nbad.value)


def tc_launch_count(h) -> int:
    return int(lib.tc_launch_count(h))


def tc_peak_launch(kind: int, grid: int, block: int, iters: int, sink, stream=None) -> None:
    _check(lib.tc_peak_launch(int(kind), int(grid), int(block), int(iters), sink.data_ptr(), _stream_ptr(stream)),
           "tc_peak_launch")


def tc_peak_chains() -> int:
    return int(lib.tc_peak_chains())


DF64_OPS = {"add": 0, "mul": 1, "div": 2, "sqrt": 3, "exp": 4, "log": 5}


def tc_df64_source_check(params, fields, err, stream=None) -> None:
    """Source terms in df64 against FP64 at the stored state of every cell (include/tc_peak.h):
    err is a contiguous CUDA float64 tensor of 5 * ncell values."""
    _check(lib.tc_df64_source_check(ctypes.byref(params), ctypes.byref(fields), err.data_ptr(), _stream_ptr(stream)),
           "tc_df64_source_check")


def tc_df64_eval(op: str, a, b, out, stream=None) -> None:
    """Element-wise df64 arithmetic on the device (include/tc_peak.h): a, b, out are
    contiguous CUDA float64 tensors of one size (b only for add, mul and div)."""
    n = out.numel()
    _check(lib.tc_df64_eval(DF64_OPS[op], a.data_ptr(), b.data_ptr() if b is not None else None, out.data_ptr(),
                            n, _stream_ptr(stream)), "tc_df64_eval")


# ----------------------------------------------------------------------------- helpers
STATE_OUT = ("T", "xH2", "xHp", "xe", "xCp", "xCO", "nsub", "status", "iters")
INPUT_KEYS = ("n", "chi_pe", "chi_lw", "f_h2", "f_c", "F_lyc", "xi", "Zg", "Zd")


def to_device(cells: dict, device="cuda", outputs: bool = True) -> dict:
    """Copies a dict of numpy arrays (inputs and T, xH2, xHp) to device float64 tensors
    and allocates the optional outputs."""
    import numpy as np
    import torch
    n = int(np.asarray(cells["n"]).size)
    d = {}
    for k in INPUT_KEYS + ("T", "xH2", "xHp"):
        if k not in cells:
            continue
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(cells[k], dtype=np.float64), (n,)))
        d[k] = torch.from_numpy(a.copy()).to(device)
    if outputs:
        for k in ("xe", "xCp", "xCO"):
            d[k] = torch.zeros(n, dtype=torch.float64, device=device)
        for k in ("nsub", "status", "iters"):
            d[k] = torch.zeros(n, dtype=torch.int32, device=device)
    return d


def from_device(d: dict) -> dict:
    return {k: d[k].cpu().numpy() for k in STATE_OUT if k in d}


class Stepper:
    """Owns a tc_handle for one parameter set; steps device tensor dicts in place."""

    def __init__(self, mode: int = TC_MODE_PAPER_FP64, **params):
        self.params = tc_params_default(mode, **params)
        self.h = tc_create(self.params)

    def step(self, d: dict, dt: float, stream=None, Zg: float = 1.0, Zd: float = 1.0) -> None:
        f = make_fields(d, Zg=Zg, Zd=Zd)
        tc_step(self.h, f, dt, stream)

    def autotune(self, d: dict, dt: float, stream=None, Zg: float = 1.0, Zd: float = 1.0) -> dict:
        return tc_autotune(self.h, make_fields(d, Zg=Zg, Zd=Zd), dt, stream)

    def step_host(self, cells: dict, dt: float, stream=None, Zg: float = 1.0, Zd: float = 1.0) -> None:
        tc_step_host(self.h, make_host_fields(cells, Zg=Zg, Zd=Zd), dt, stream)

    def load_mlp(self, blob: bytes) -> None:
        tc_load_mlp(self.h, blob)

    def eq_curves(self, n_axis, chi0, xi0, Zg, Zd, shielded: bool = False, stream=None, **spec) -> dict:
        return tc_eq_curves(self.h, n_axis, chi0, xi0, Zg, Zd, shielded, stream, **spec)

    def pdr(self, n, chi0, xi0, Z, dx_cm, ncell: int, stream=None, **spec) -> dict:
        return tc_pdr(self.h, n, chi0, xi0, Z, dx_cm, ncell, stream, **spec)

    def launches(self) -> int:
        return tc_launch_count(self.h)

    def close(self) -> None:
        if self.h:
            tc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _f64_host(v):
    import numpy as np
    return np.ascontiguousarray(np.atleast_1d(np.asarray(v, dtype=np.float64)))


def tc_eq_curves(h, n_axis, chi0, xi0, Zg, Zd, shielded: bool = False, stream=None, out: dict | None = None,
                 **spec) -> dict:
    """Runs tc_eq_curves for the density axis `n_axis` and per-curve chi0, xi0, Zg, Zd
    (host arrays); `spec` overrides tc_eq_spec fields (t_end_s, nchunk, L_shld0_pc, ...).
    Returns device tensors of shape [ncurve, nn] (T, xH2, xHp, xe, P, xCO, chg, status)
    and [ncurve] (i_max, i_min); `out` may pass preallocated ones."""
    import torch
    n_axis = _f64_host(n_axis)
    cur = [_f64_host(v) for v in (chi0, xi0, Zg, Zd)]
    nc = cur[0].size
    if any(c.size != nc for c in cur):
        raise ValueError("chi0, xi0, Zg, Zd must have the same length")
    s = tc_eq_spec()
    _check(lib.tc_eq_spec_default(ctypes.byref(s)), "tc_eq_spec_default")
    s.n_axis, s.nn = n_axis.ctypes.data, n_axis.size
    s.chi0, s.xi0, s.Zg, s.Zd = (c.ctypes.data for c in cur)
    s.ncurve, s.shielded = nc, int(bool(shielded))
    for k, v in spec.items():
        setattr(s, k, v)
    if out is None:
        shape = (nc, n_axis.size)
        out = {k: torch.empty(shape, dtype=torch.float64, device="cuda")
               for k in ("T", "xH2", "xHp", "xe", "P", "xCO", "chg")}
        out["status"] = torch.empty(shape, dtype=torch.int32, device="cuda")
        out["i_max"] = torch.empty(nc, dtype=torch.int32, device="cuda")
        out["i_min"] = torch.empty(nc, dtype=torch.int32, device="cuda")
    o = tc_eq_out(*[out[k].data_ptr() if out.get(k) is not None else None
                    for k in ("T", "xH2", "xHp", "xe", "P", "xCO", "chg", "status", "i_max", "i_min")])
    _check(lib.tc_eq_curves(h, ctypes.byref(s), ctypes.byref(o), _stream_ptr(stream)), "tc_eq_curves")
    return out


def tc_pdr(h, n, chi0, xi0, Z, dx_cm, ncell: int, stream=None, out: dict | None = None, **spec) -> dict:
    """Runs tc_pdr for slabs with per-slab n, chi0, xi0, Z (= Z'_g = Z'_d) and dx_cm (host
    arrays); `spec` overrides tc_pdr_spec fields.  Returns device tensors [nslab, ncell]
    (T, xH2, xHp, xe, xCO, chi_pe, f_h2, N_c, status) and [nslab] (N_trans)."""
    import torch
    arrs = [_f64_host(v) for v in (n, chi0, xi0, Z, dx_cm)]
    ns = arrs[0].size
    if any(a.size != ns for a in arrs):
        raise ValueError("n, chi0, xi0, Z and dx_cm must have the same length")
    s = tc_pdr_spec()
    _check(lib.tc_pdr_spec_default(ctypes.byref(s)), "tc_pdr_spec_default")
    s.n, s.chi0, s.xi0, s.Z, s.dx_cm = (a.ctypes.data for a in arrs)
    s.nslab, s.ncell = ns, int(ncell)
    for k, v in spec.items():
        setattr(s, k, v)
    if out is None:
        shape = (ns, max(int(ncell), 0))
        out = {k: torch.empty(shape, dtype=torch.float64, device="cuda")
               for k in ("T", "xH2", "xHp", "xe", "xCO", "chi_pe", "f_h2", "N_c")}
        out["status"] = torch.empty(shape, dtype=torch.int32, device="cuda")
        out["N_trans"] = torch.empty(ns, dtype=torch.float64, device="cuda")
    o = tc_pdr_out(*[out[k].data_ptr() if out.get(k) is not None else None
                     for k in ("T", "xH2", "xHp", "xe", "xCO", "chi_pe", "f_h2", "N_c", "status", "N_trans")])
    _check(lib.tc_pdr(h, ctypes.byref(s), ctypes.byref(o), _stream_ptr(stream)), "tc_pdr")
    return out


def tc_sixray(n, x_h2, dx_cm: float, chi0: float = 1.0, xi0: float = 2e-16, Zd: float = 1.0, out: dict | None = None,
              n_eff: bool = True, stream=None) -> dict:
    """Six-ray fields of a grid: n and x_h2 are device float64 tensors of shape
    [nz, ny, nx].  Returns (or fills `out`) chi_pe, chi_lw, f_h2, xi and, if n_eff, N_eff."""
    import torch
    if n.dim() != 3 or n.shape != x_h2.shape or n.dtype != torch.float64 or x_h2.dtype != torch.float64:
        raise ValueError("n and x_h2 must be float64 tensors of the same 3-d shape")
    if not (n.is_contiguous() and x_h2.is_contiguous()):
        raise ValueError("n and x_h2 must be contiguous")
    nz, ny, nx = n.shape
    g = tc_sixray_grid(nx, ny, nz, float(dx_cm), float(chi0), float(xi0), float(Zd))
    if out is None:
        keys = ("chi_pe", "chi_lw", "f_h2", "xi") + (("N_eff",) if n_eff else ())
        out = {k: torch.empty_like(n) for k in keys}
    ne = out.get("N_eff")
    _check(lib.tc_sixray(ctypes.byref(g), n.data_ptr(), x_h2.data_ptr(), out["chi_pe"].data_ptr(),
                         out["chi_lw"].data_ptr(), out["f_h2"].data_ptr(), out["xi"].data_ptr(),
                         ne.data_ptr() if ne is not None else None, _stream_ptr(stream)), "tc_sixray")
    return out


def step_numpy(cells: dict, dt: float, mode: int = TC_MODE_PAPER_FP64, **params) -> dict:
    """Uploads, runs one step on the current CUDA device, downloads (tests/smoke)."""
    import torch
    d = to_device(cells)
    st = Stepper(mode, **params)
    st.step(d, dt)
    torch.cuda.synchronize()
    out = from_device(d)
    st.close()
    return out


# ----------------------------------------------------------------------------- seed network
def _f32(a):
    import numpy as np
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


class SeedNet:
    """Handle of the seed network (include/tc_mlp.h).  X, Y are device float32 torch
    tensors of shape [B, 10] and [B, 3]; all arithmetic runs in the library's kernels."""

    def __init__(self, seed: int = 0):
        self.h = ctypes.c_void_p()
        _check(lib.tc_mlp_create(ctypes.c_ulonglong(seed), ctypes.byref(self.h)), "tc_mlp_create")

    @staticmethod
    def n_params() -> int:
        return int(lib.tc_mlp_n_params())

    def set_norm(self, mean, std) -> None:
        m, s = _f32(mean), _f32(std)
        _check(lib.tc_mlp_set_norm(self.h, m.ctypes.data, s.ctypes.data), "tc_mlp_set_norm")

    def set_params(self, theta) -> None:
        t = _f32(theta)
        assert t.size == self.n_params()
        _check(lib.tc_mlp_set_params(self.h, t.ctypes.data), "tc_mlp_set_params")

    def get_params(self):
        import numpy as np
        t = np.zeros(self.n_params(), dtype=np.float32)
        _check(lib.tc_mlp_get_params(self.h, t.ctypes.data), "tc_mlp_get_params")
        return t

    def predict(self, X, stream=None):
        import torch
        out = torch.empty((X.shape[0], 3), dtype=torch.float32, device=X.device)
        _check(lib.tc_mlp_predict(self.h, X.data_ptr(), X.shape[0], out.data_ptr(), _stream_ptr(stream)),
               "tc_mlp_predict")
        return out

    def grad(self, X, Y, w=(1.0, 1.0, 1.0), stream=None):
        import torch
        g = torch.empty(self.n_params(), dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        w3 = _f32(w)
        _check(lib.tc_mlp_grad(self.h, X.data_ptr(), Y.data_ptr(), X.shape[0], w3.ctypes.data, g.data_ptr(),
                               loss.data_ptr(), _stream_ptr(stream)), "tc_mlp_grad")
        return g, loss

    def train_step(self, X, Y, lr, loss_out=None, w=(1.0, 1.0, 1.0), stream=None) -> None:
        w3 = _f32(w)
        _check(lib.tc_mlp_train_step(self.h, X.data_ptr(), Y.data_ptr(), X.shape[0], w3.ctypes.data,
                                     ctypes.c_float(lr), loss_out.data_ptr() if loss_out is not None else None,
                                     _stream_ptr(stream)), "tc_mlp_train_step")

    def export(self) -> bytes:
        n = int(lib.tc_mlp_blob_bytes())
        buf = ctypes.create_string_buffer(n)
        _check(lib.tc_mlp_export(self.h, buf, n), "tc_mlp_export")
        return buf.raw

    def close(self) -> None:
        if self.h:
            lib.tc_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

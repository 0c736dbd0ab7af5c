"""ctypes binding of the C ABI in include/rt.h.

Argument marshalling only: every step of the radiative-transfer path runs in
the CUDA library.  If librt.so is missing the import fails; there is no
fallback.  Device arrays are passed as torch CUDA tensors (PyTorch provides
device memory and streams and nothing else).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librt.so")

RT_OK, RT_EINVAL, RT_ENOMEM, RT_ECUDA, RT_ENOTSOLVED, RT_EBUDGET, RT_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
RT_IMPROVED, RT_REGULAR = 0, 1
RT_NONISOTHERMAL, RT_ISOTHERMAL = 0, 1
RT_FP32_FORM, RT_FP64_PLAIN = 0, 1
RT_RESONANCE_PAPER, RT_RESONANCE_LIMIT = 0, 1
RT_STAGE_AUTO, RT_STAGE_SHARED, RT_STAGE_DIRECT, RT_STAGE_INLINE = 0, 1, 2, 3
RT_SWEEP_MAX_LAYERS = 40
RT_STAGING_DEPTH_MIN = 2
RT_STAGING_DEPTH_MAX = 3

_STATUS = {0: "RT_OK", -1: "RT_EINVAL", -2: "RT_ENOMEM", -3: "RT_ECUDA", -4: "RT_ENOTSOLVED",
           -5: "RT_EBUDGET", -6: "RT_ETIMEOUT"}


class rt_config(ctypes.Structure):
    _fields_ = [
        ("n_g", ctypes.c_int32), ("g_weights", ctypes.POINTER(ctypes.c_double)),
        ("wn_min", ctypes.c_double), ("wn_max", ctypes.c_double),
        ("two_stream", ctypes.c_int32), ("layers", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("resonance", ctypes.c_int32),
        ("e_clamp", ctypes.c_int32),
        ("eps2", ctypes.c_double), ("grav", ctypes.c_double), ("cp", ctypes.c_double),
        ("T_int", ctypes.c_double), ("F_toa_diffuse", ctypes.c_double),
        ("max_layers", ctypes.c_int32), ("max_bins", ctypes.c_int32),
        ("hbm_budget_bytes", ctypes.c_size_t), ("block_threads", ctypes.c_int32),
        ("ctas_per_sm", ctypes.c_int32), ("planck_staging", ctypes.c_int32),
        ("systems_per_lane", ctypes.c_int32), ("kernel_timing", ctypes.c_int32),
        ("n_edges", ctypes.c_int32), ("wn_edges", ctypes.POINTER(ctypes.c_double)),
        ("n_sweeps", ctypes.c_int32), ("staging_depth", ctypes.c_int32),
    ]


class rt_columns(ctypes.Structure):
    _fields_ = [
        ("n_cols", ctypes.c_int32),
        ("n_layers", ctypes.POINTER(ctypes.c_int32)), ("n_bins", ctypes.POINTER(ctypes.c_int32)),
        ("L", ctypes.c_int32), ("NB", ctypes.c_int32),
        ("dtau", ctypes.c_void_p), ("w0", ctypes.c_void_p), ("g0", ctypes.c_void_p),
        ("T_center", ctypes.c_void_p), ("T_iface", ctypes.c_void_p), ("p_iface", ctypes.c_void_p),
        ("mu_star", ctypes.c_void_p), ("F_star", ctypes.c_void_p),
        ("cube_offset", ctypes.POINTER(ctypes.c_int64)), ("center_offset", ctypes.POINTER(ctypes.c_int64)),
        ("iface_offset", ctypes.POINTER(ctypes.c_int64)), ("bin_offset", ctypes.POINTER(ctypes.c_int64)),
        ("col_index", ctypes.POINTER(ctypes.c_int64)),
        ("n_cube", ctypes.c_int64), ("n_center", ctypes.c_int64), ("n_iface", ctypes.c_int64),
        ("n_fstar", ctypes.c_int64), ("n_mu", ctypes.c_int64),
    ]


class rt_ktable(ctypes.Structure):
    _fields_ = [
        ("n_T", ctypes.c_int32), ("n_P", ctypes.c_int32),
        ("T_grid", ctypes.POINTER(ctypes.c_double)), ("log10p_grid", ctypes.POINTER(ctypes.c_double)),
        ("n_bins", ctypes.c_int32), ("n_g", ctypes.c_int32),
        ("log10_kappa", ctypes.POINTER(ctypes.c_float)),
        ("sigma_scat_cloud", ctypes.POINTER(ctypes.c_double)),
        ("sigma_abs_cloud", ctypes.POINTER(ctypes.c_double)),
        ("g0_cloud", ctypes.POINTER(ctypes.c_double)),
        ("f_cloud", ctypes.c_double), ("x_H2", ctypes.c_double), ("x_He", ctypes.c_double),
        ("mbar_amu", ctypes.c_double),
    ]


class rt_stats_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "systems", "resonance_hits", "etau_hits", "eclamp_hits", "invalid_inputs",
        "nonfinite_outputs", "fp64_evals", "bounds_violations")]


def _load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; build it with "
                           "`python -m paper_2203_02293_b300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    lib.rt_create.argtypes = [ctypes.POINTER(rt_config), ctypes.POINTER(H)]
    lib.rt_query_bytes.argtypes = [H, ctypes.POINTER(rt_columns), ctypes.POINTER(ctypes.c_size_t)]
    lib.rt_check_columns.argtypes = [ctypes.POINTER(rt_config), ctypes.POINTER(rt_columns), ctypes.c_char_p,
                                     ctypes.c_size_t]
    lib.rt_solve_columns.argtypes = [H, ctypes.POINTER(rt_columns), ctypes.c_void_p]
    lib.rt_fluxes.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.rt_heating.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p]
    lib.rt_toa_spectrum.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p]
    lib.rt_set_ktable.argtypes = [H, ctypes.POINTER(rt_ktable)]
    lib.rt_ktable_optics.argtypes = [H, ctypes.POINTER(rt_columns), ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p]
    lib.rt_solve_ktable.argtypes = [H, ctypes.POINTER(rt_columns), ctypes.c_void_p]
    lib.rt_stats.argtypes = [H, ctypes.POINTER(rt_stats_t)]
    lib.rt_kernel_times.argtypes = [H, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
    lib.rt_last_error.argtypes = [H]
    lib.rt_last_error.restype = ctypes.c_char_p
    lib.rt_destroy.argtypes = [H]
    lib.rt_destroy.restype = None
    lib.rt_solve_uniform_noalloc.argtypes = [ctypes.POINTER(rt_config), ctypes.POINTER(rt_columns),
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p]
    lib.rt_solve_uniform_noalloc.restype = ctypes.c_int
    lib.rt_inject_alloc_failures.argtypes = [ctypes.c_int]
    lib.rt_inject_alloc_failures.restype = ctypes.c_int
    for f in ("rt_create", "rt_query_bytes", "rt_solve_columns", "rt_fluxes", "rt_heating",
              "rt_toa_spectrum", "rt_stats", "rt_set_ktable", "rt_ktable_optics", "rt_solve_ktable",
              "rt_kernel_times", "rt_check_columns"):
        getattr(lib, f).restype = ctypes.c_int
    return lib


_lib: ctypes.CDLL | None = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


class RTError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


def _check(code: int, handle=None):
    if code != RT_OK:
        msg = lib().rt_last_error(handle).decode() if handle else ""
        raise RTError(code, msg)


def _ptr(t) -> int | None:
    """Raw address of a torch tensor / numpy array (None passes NULL)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


@dataclass
class Config:
    """Python mirror of rt_config with the paper's defaults (Table 3)."""
    g_weights: np.ndarray
    wn_min: float = 50.0
    wn_max: float = 1.0e4 / 0.3
    two_stream: int = RT_IMPROVED
    layers: int = RT_NONISOTHERMAL
    precision: int = RT_FP32_FORM
    resonance: int = RT_RESONANCE_PAPER
    e_clamp: int = 1
    eps2: float = 2.0 / 3.0
    grav: float = 47.0
    cp: float = 12436.0
    T_int: float = 100.0
    F_toa_diffuse: float = 0.0
    max_layers: int = 1024
    max_bins: int = 4096
    hbm_budget_bytes: int = 0
    block_threads: int = 0
    ctas_per_sm: int = 0
    planck_staging: int = 0              # RT_STAGE_AUTO / _SHARED / _DIRECT / _INLINE
    systems_per_lane: int = 0            # FP32 form: 1 or 2 (0 = 2)
    kernel_timing: int = 0               # 1: CUDA events around each kernel (rt_kernel_times)
    wn_edges: np.ndarray | None = None   # explicit bin edges (cm^-1); None = uniform bins
    n_sweeps: int = 0                    # 0: Thomas; N > 0: N sweeps of the iterative method
    staging_depth: int = 0               # back-substitution levels in flight, 2 or 3 (0 = 2)


def _config(cfg: Config):
    """The C struct for ``cfg``; the returned arrays must outlive the call."""
    PD = ctypes.POINTER(ctypes.c_double)
    gw = np.ascontiguousarray(cfg.g_weights, dtype=np.float64)
    ed = None if cfg.wn_edges is None else np.ascontiguousarray(cfg.wn_edges, dtype=np.float64)
    c = rt_config(len(gw), gw.ctypes.data_as(PD), cfg.wn_min,
                  cfg.wn_max, cfg.two_stream, cfg.layers, cfg.precision, cfg.resonance,
                  cfg.e_clamp, cfg.eps2, cfg.grav, cfg.cp, cfg.T_int, cfg.F_toa_diffuse,
                  cfg.max_layers, cfg.max_bins, cfg.hbm_budget_bytes, cfg.block_threads,
                  cfg.ctas_per_sm, cfg.planck_staging, cfg.systems_per_lane, cfg.kernel_timing,
                  0 if ed is None else ed.size,
                  None if ed is None else ed.ctypes.data_as(PD), cfg.n_sweeps, cfg.staging_depth)
    return c, (gw, ed)


def rt_create(cfg: Config):
    """Create a handle (returns an opaque ctypes pointer)."""
    c, keep = _config(cfg)
    h = ctypes.c_void_p()
    _check(lib().rt_create(ctypes.byref(c), ctypes.byref(h)))
    return h


def _count(t) -> int:
    """Element count of a tensor / array (0 for None)."""
    if t is None:
        return 0
    return int(t.numel()) if hasattr(t, "numel") else int(np.asarray(t).size)


def make_columns(n_cols: int, n_layers, n_bins, dtau, w0, g0, T_center, T_iface, p_iface,
                 mu_star, F_star, L: int = 0, NB: int = 0, gather: dict | None = None,
                 counts: dict | None = None):
    """Build an rt_columns descriptor.  n_layers / n_bins are host int32 arrays
    (or None with uniform L, NB); the rest are device tensors.  ``gather`` may
    give host int64 arrays cube_offset, center_offset, iface_offset,
    bin_offset, col_index (see include/rt.h).  The arrays' element counts,
    which bound every read, are taken from the tensors unless ``counts``
    overrides them (keys n_cube, n_center, n_iface, n_fstar, n_mu).  The
    returned object keeps the host arrays alive."""
    nl = None if n_layers is None else np.ascontiguousarray(n_layers, dtype=np.int32)
    nb = None if n_bins is None else np.ascontiguousarray(n_bins, dtype=np.int32)
    P32 = ctypes.POINTER(ctypes.c_int32)
    P64 = ctypes.POINTER(ctypes.c_int64)
    g = {k: np.ascontiguousarray(v, dtype=np.int64) for k, v in (gather or {}).items()}
    gp = {k: (g[k].ctypes.data_as(P64) if k in g else None)
          for k in ("cube_offset", "center_offset", "iface_offset", "bin_offset", "col_index")}
    c = rt_columns(n_cols, nl.ctypes.data_as(P32) if nl is not None else None,
                   nb.ctypes.data_as(P32) if nb is not None else None, L, NB,
                   _ptr(dtau), _ptr(w0), _ptr(g0), _ptr(T_center), _ptr(T_iface), _ptr(p_iface),
                   _ptr(mu_star), _ptr(F_star), gp["cube_offset"], gp["center_offset"],
                   gp["iface_offset"], gp["bin_offset"], gp["col_index"])
    n = dict(n_cube=min(_count(dtau), _count(w0), _count(g0)), n_center=_count(T_center),
             n_iface=min(_count(T_iface), _count(p_iface)), n_fstar=_count(F_star), n_mu=_count(mu_star))
    n.update(counts or {})
    for k, v in n.items():
        setattr(c, k, int(v))
    c._keep = (nl, nb, g)
    return c


def rt_check_columns(cfg: Config, cols) -> str:
    """Host-only validation of ``cols`` for ``cfg`` (no device needed);
    raises RTError with the library's reason, returns "" when valid."""
    c, keep = _config(cfg)
    buf = ctypes.create_string_buffer(512)
    code = lib().rt_check_columns(ctypes.byref(c), ctypes.byref(cols), buf, len(buf))
    if code != RT_OK:
        raise RTError(code, buf.value.decode())
    return ""


def rt_query_bytes(h, cols) -> int:
    n = ctypes.c_size_t()
    _check(lib().rt_query_bytes(h, ctypes.byref(cols), ctypes.byref(n)), h)
    return n.value


def rt_solve_columns(h, cols, stream=None):
    _check(lib().rt_solve_columns(h, ctypes.byref(cols), _stream_ptr(stream)), h)


def rt_fluxes(h, F_up=None, F_down=None, F_net=None, stream=None):
    _check(lib().rt_fluxes(h, _ptr(F_up), _ptr(F_down), _ptr(F_net), _stream_ptr(stream)), h)


def rt_heating(h, Q, stream=None):
    _check(lib().rt_heating(h, _ptr(Q), _stream_ptr(stream)), h)


def rt_set_ktable(h, kt: dict):
    """Copy a k-table (a dict with the fields of rt_ktable, as drawn by
    ``rt_synth.ktable``) into the handle."""
    PD = ctypes.POINTER(ctypes.c_double)
    d = lambda k: np.ascontiguousarray(kt[k], dtype=np.float64)
    T, lp = d("T_grid"), d("log10p_grid")
    lk = np.ascontiguousarray(kt["log10_kappa"], dtype=np.float32)
    ss, sa, gc = d("sigma_scat_cloud"), d("sigma_abs_cloud"), d("g0_cloud")
    nT, nP, NB, NG = lk.shape
    if T.size != nT or lp.size != nP or ss.size != NB or sa.size != NB or gc.size != NB:
        raise ValueError("k-table arrays disagree with log10_kappa's shape")
    c = rt_ktable(nT, nP, T.ctypes.data_as(PD), lp.ctypes.data_as(PD), NB, NG,
                  lk.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ss.ctypes.data_as(PD),
                  sa.ctypes.data_as(PD), gc.ctypes.data_as(PD), float(kt["f_cloud"]),
                  float(kt["x_h2"]), float(kt["x_he"]), float(kt["mbar_amu"]))
    _check(lib().rt_set_ktable(h, ctypes.byref(c)), h)


def rt_ktable_optics(h, cols, dtau, w0, g0, stream=None):
    _check(lib().rt_ktable_optics(h, ctypes.byref(cols), _ptr(dtau), _ptr(w0), _ptr(g0),
                                  _stream_ptr(stream)), h)


def rt_solve_ktable(h, cols, stream=None):
    _check(lib().rt_solve_ktable(h, ctypes.byref(cols), _stream_ptr(stream)), h)


def rt_toa_spectrum(h, F_up_toa, stream=None):
    """Per-bin upward flux at the TOA of the last solve, [sum NB] float64."""
    _check(lib().rt_toa_spectrum(h, _ptr(F_up_toa), _stream_ptr(stream)), h)


def rt_kernel_times(h):
    """(pre-kernel ms, solve-kernel ms) of the last solve (needs kernel_timing)."""
    a, b = ctypes.c_float(), ctypes.c_float()
    _check(lib().rt_kernel_times(h, ctypes.byref(a), ctypes.byref(b)), h)
    return a.value, b.value


def rt_stats(h) -> dict:
    s = rt_stats_t()
    _check(lib().rt_stats(h, ctypes.byref(s)), h)
    return {n: getattr(s, n) for n, _ in rt_stats_t._fields_}


def rt_last_error(h) -> str:
    return lib().rt_last_error(h).decode()


def rt_destroy(h):
    if h:
        lib().rt_destroy(h)


def rt_inject_alloc_failures(n: int):
    """Make the next ``n`` device workspace allocations fail (RT_ENOMEM);
    0 clears.  A test hook for callers' error handling."""
    _check(lib().rt_inject_alloc_failures(n))


def rt_solve_uniform_noalloc(cfg: Config, cols, F_up, F_down, F_net, Q, stream=None):
    """Solve a uniform-shape batch with no device allocation (see include/rt.h).

    ``cols`` is an rt_columns descriptor with NULL shape arrays and L, NB set;
    the four outputs are device tensors written in place."""
    c, keep = _config(cfg)
    code = lib().rt_solve_uniform_noalloc(ctypes.byref(c), ctypes.byref(cols), _ptr(F_up),
                                          _ptr(F_down), _ptr(F_net), _ptr(Q), _stream_ptr(stream))
    if code != RT_OK:
        raise RTError(code, "rt_solve_uniform_noalloc")

"""FP64 CPU oracle for the column radiative-transfer path (Deitrick et al.,
arXiv 2203.02293, Sec. 2.2 and App. B).

TEST INFRASTRUCTURE ONLY.  The product library never imports, links or calls
this package.  Only the test suite, the smoke check and the benchmark's
CPU-baseline leg use it.  The arithmetic lives in ``rt_oracle.c`` (plain C,
FP64, literal formulas, block Thomas on 2x2 blocks); this module compiles it
with gcc and marshals arrays through ctypes.

Parity status of each oracle function against the paper and the mathematics
is recorded in the tests under ``tests/test_oracle_*.py``.  One reading is
"parity unpinned": the paper's resonance rule (|D| < 1e-5 -> D := 2 mu*,
Sec. 2.2.1 after Eq. 11) is discontinuous and has no independent value to
pin against; only its trigger condition and its limit-mode alternative are
pinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rt_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(src: str = SRC, out: str = LIB, extra: tuple = ()) -> str:
    """Compile the oracle into a shared library (gcc, -O2, OpenMP, IEEE math)."""
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", *extra,
           "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("improved", ctypes.c_int32), ("isothermal", ctypes.c_int32),
        ("resonance", ctypes.c_int32), ("e_clamp", ctypes.c_int32),
        ("eps2", ctypes.c_double), ("grav", ctypes.c_double),
        ("cp", ctypes.c_double), ("T_int", ctypes.c_double),
        ("F_toa", ctypes.c_double), ("wn_min", ctypes.c_double),
        ("wn_max", ctypes.c_double), ("wn_edges", ctypes.POINTER(ctypes.c_double)),
        ("n_sweeps", ctypes.c_int32),
    ]


class _Stats(ctypes.Structure):
    _fields_ = [("resonance_hits", ctypes.c_int64), ("etau_hits", ctypes.c_int64),
                ("eclamp_hits", ctypes.c_int64), ("nonfinite", ctypes.c_int64)]


@dataclass
class OracleConfig:
    """Method switches and constants (Table 3 defaults)."""
    improved: bool = True        # Eq. 19 E fit; False -> regular two-stream, E = 1
    isothermal: bool = False     # False -> non-isothermal layers
    resonance: str = "paper"     # "paper": D := 2 mu* if |D| < 1e-5; "limit": exact solution
    e_clamp: bool = True         # E := max(E_fit, 1)
    eps2: float = 2.0 / 3.0
    grav: float = 47.0
    cp: float = 12436.0
    T_int: float = 100.0
    F_toa: float = 0.0
    wn_min: float = 50.0
    wn_max: float = 1.0e4 / 0.3
    wn_edges: object = None      # None: NB uniform bins; else NB + 1 increasing edges, cm^-1
    n_sweeps: int = 0            # 0: Thomas (Eqs. 12-15); N > 0: N sweeps of the iterative method

    def c(self) -> _Cfg:
        edges = None
        if self.wn_edges is not None:
            self._edges = np.ascontiguousarray(self.wn_edges, dtype=np.float64)
            edges = self._edges.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        return _Cfg(int(self.improved), int(self.isothermal),
                    0 if self.resonance == "paper" else 1, int(self.e_clamp),
                    self.eps2, self.grav, self.cp, self.T_int, self.F_toa,
                    self.wn_min, self.wn_max, edges, int(self.n_sweeps))


_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I = ctypes.POINTER(ctypes.c_int32)


def _p(a, t):
    return a.ctypes.data_as(t)


class Oracle:
    """ctypes front end of one compiled copy of the oracle library."""

    def __init__(self, path: str | None = None):
        if path is None:
            path = LIB
            if (not os.path.exists(path)
                    or os.path.getmtime(path) < os.path.getmtime(SRC)):
                build()
        self.lib = ctypes.CDLL(path)
        L = self.lib
        L.oracle_planck_bin.restype = ctypes.c_double
        L.oracle_planck_bin.argtypes = [ctypes.c_double] * 3
        L.oracle_assemble.restype = ctypes.c_int
        L.oracle_assemble.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int, _F, _F, _F,
                                      _D, _D, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, _D, _D, _D, _D, _D]
        L.oracle_block_thomas.restype = ctypes.c_int
        L.oracle_block_thomas.argtypes = [ctypes.c_int, _D, _D, _D, _D, _D]
        L.oracle_solve_system.restype = ctypes.c_int
        L.oracle_solve_system.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int, _F, _F, _F,
                                          _D, _D, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, _D, _D, _D]
        L.oracle_sweep_system.restype = ctypes.c_int
        L.oracle_sweep_system.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int, _F, _F, _F,
                                          _D, _D, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, _D, _D, _D]
        L.oracle_solve_columns.restype = ctypes.c_int
        L.oracle_solve_columns.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int, _I, _I,
                                           ctypes.c_int, _D, _F, _F, _F, _D, _D, _D,
                                           _D, _D, _D, _D, _D, _D, _D, _D, _D,
                                           ctypes.POINTER(_Stats)]

    # -- Planck -------------------------------------------------------
    def planck_bin(self, T: float, wn_lo: float, wn_hi: float) -> float:
        """Bin-integrated Planck function, W m^-2 sr^-1."""
        return self.lib.oracle_planck_bin(float(T), float(wn_lo), float(wn_hi))

    # -- one system ---------------------------------------------------
    @staticmethod
    def _sys_args(dtau, w0, g0, Bc, Bi):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
        d = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        return f(dtau), f(w0), f(g0), d(Bc), d(Bi)

    def assemble(self, cfg: OracleConfig, dtau, w0, g0, Bc, Bi, mu, Fstar, F_BOA):
        """Blocks A, B, C (n+1, 2, 2), D (n+1, 2) of Eq. 12 and the beam at levels."""
        dtau, w0, g0, Bc, Bi = self._sys_args(dtau, w0, g0, Bc, Bi)
        L = dtau.size
        n = L if cfg.isothermal else 2 * L
        A = np.zeros(4 * (n + 1)); B = np.zeros(4 * (n + 1)); C = np.zeros(4 * (n + 1))
        D = np.zeros(2 * (n + 1)); Fb = np.zeros(n + 1)
        c = cfg.c()
        rc = self.lib.oracle_assemble(ctypes.byref(c), L, _p(dtau, _F), _p(w0, _F), _p(g0, _F),
                                      _p(Bc, _D), _p(Bi, _D), mu, Fstar, F_BOA,
                                      _p(A, _D), _p(B, _D), _p(C, _D), _p(D, _D), _p(Fb, _D))
        assert rc == n
        return (A.reshape(n + 1, 2, 2), B.reshape(n + 1, 2, 2), C.reshape(n + 1, 2, 2),
                D.reshape(n + 1, 2), Fb)

    def block_thomas(self, A, B, C, D):
        n = A.shape[0] - 1
        X = np.zeros(2 * (n + 1))
        a, b, c, d = (np.ascontiguousarray(x, dtype=np.float64).ravel() for x in (A, B, C, D))
        rc = self.lib.oracle_block_thomas(n, _p(a, _D), _p(b, _D), _p(c, _D), _p(d, _D), _p(X, _D))
        assert rc == 0
        return X.reshape(n + 1, 2)

    def solve_system(self, cfg: OracleConfig, dtau, w0, g0, Bc, Bi, mu, Fstar, F_BOA):
        """Levels BOA first: returns F_up, F_dn (diffuse), F_beam, each [n+1]."""
        dtau, w0, g0, Bc, Bi = self._sys_args(dtau, w0, g0, Bc, Bi)
        L = dtau.size
        n = L if cfg.isothermal else 2 * L
        up = np.zeros(n + 1); dn = np.zeros(n + 1); fb = np.zeros(n + 1)
        c = cfg.c()
        rc = self.lib.oracle_solve_system(ctypes.byref(c), L, _p(dtau, _F), _p(w0, _F),
                                          _p(g0, _F), _p(Bc, _D), _p(Bi, _D), mu, Fstar,
                                          F_BOA, _p(up, _D), _p(dn, _D), _p(fb, _D))
        assert rc == n
        return up, dn, fb

    def sweep_system(self, cfg: OracleConfig, dtau, w0, g0, Bc, Bi, mu, Fstar, F_BOA,
                     n_sweeps, up0=None, dn0=None):
        """n_sweeps sweeps of the iterative method (Sec. 2.2.2) from the
        state (up0, dn0) at levels, BOA first (zero diffuse flux if None).
        Returns F_up, F_dn (diffuse), F_beam, each [n+1]."""
        dtau, w0, g0, Bc, Bi = self._sys_args(dtau, w0, g0, Bc, Bi)
        L = dtau.size
        n = L if cfg.isothermal else 2 * L
        up = np.zeros(n + 1) if up0 is None else np.array(up0, dtype=np.float64)
        dn = np.zeros(n + 1) if dn0 is None else np.array(dn0, dtype=np.float64)
        assert up.size == n + 1 and dn.size == n + 1
        fb = np.zeros(n + 1)
        c = cfg.c()
        rc = self.lib.oracle_sweep_system(ctypes.byref(c), L, _p(dtau, _F), _p(w0, _F),
                                          _p(g0, _F), _p(Bc, _D), _p(Bi, _D), mu, Fstar,
                                          F_BOA, int(n_sweeps), _p(up, _D), _p(dn, _D), _p(fb, _D))
        assert rc == n
        return up, dn, fb

    # -- whole batch -------------------------------------------------
    def solve_columns(self, cfg: OracleConfig, cols, per_system: bool = False):
        """Solve a packed batch (an ``rt_synth.Columns``).  Returns a dict with
        F_up, F_down (diffuse + beam), F_net at interfaces, Q per layer and the
        branch-hit counters; with ``per_system`` also the per-system diffuse
        interface fluxes ``sys_up``/``sys_dn``.  ``F_up_toa`` is the upward
        flux at the TOA per bin (sum over g of w_g F_up), [sum NB]."""
        nl = np.ascontiguousarray(cols.n_layers, dtype=np.int32)
        nb = np.ascontiguousarray(cols.n_bins, dtype=np.int32)
        nc = nl.size
        n_if = int((nl + 1).sum())
        n_l = int(nl.sum())
        f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        dtau, w0, g0 = f32(cols.dtau), f32(cols.w0), f32(cols.g0)
        Tc, Ti, p = f64(cols.T_center), f64(cols.T_iface), f64(cols.p_iface)
        mu, Fs, gw = f64(cols.mu_star), f64(cols.F_star), f64(cols.g_weights)
        up = np.zeros(n_if); dn = np.zeros(n_if); net = np.zeros(n_if); Q = np.zeros(n_l)
        toa = np.zeros(int(nb.sum()))
        if cfg.wn_edges is not None and np.any(nb != len(cfg.wn_edges) - 1):
            raise ValueError("explicit bin edges need NB = len(wn_edges) - 1 in every column")
        if per_system:
            n_sys_if = int(((nl + 1) * nb).sum()) * cols.n_g
            su = np.zeros(n_sys_if); sd = np.zeros(n_sys_if)
            psu, psd = _p(su, _D), _p(sd, _D)
        else:
            psu = psd = None
        st = _Stats()
        c = cfg.c()
        rc = self.lib.oracle_solve_columns(
            ctypes.byref(c), nc, _p(nl, _I), _p(nb, _I), int(cols.n_g), _p(gw, _D),
            _p(dtau, _F), _p(w0, _F), _p(g0, _F), _p(Tc, _D), _p(Ti, _D), _p(p, _D),
            _p(mu, _D), _p(Fs, _D), _p(up, _D), _p(dn, _D), _p(net, _D), _p(Q, _D),
            psu, psd, _p(toa, _D), ctypes.byref(st))
        if rc != 0:
            raise MemoryError("oracle_solve_columns failed")
        out = dict(F_up=up, F_down=dn, F_net=net, Q=Q, F_up_toa=toa,
                   stats=dict(resonance_hits=st.resonance_hits, etau_hits=st.etau_hits,
                              eclamp_hits=st.eclamp_hits, nonfinite=st.nonfinite))
        if per_system:
            out["sys_up"] = su
            out["sys_dn"] = sd
        return out


_default: Oracle | None = None


def get() -> Oracle:
    """The oracle built from ``rt_oracle.c`` (compiled on first use)."""
    global _default
    if _default is None:
        _default = Oracle()
    return _default

"""Device-resident batches and a solver handle over the C ABI.

PyTorch supplies device memory and streams; the computation is the CUDA
library's.  Nothing here computes any part of the radiative-transfer path.
"""
from __future__ import annotations

import numpy as np
import torch

from . import rt


class DeviceBatch:
    """A packed batch of columns copied into device memory.

    ``cols`` is any object with the fields of ``rt_synth.Columns`` (n_layers,
    n_bins, n_g, dtau, w0, g0, T_center, T_iface, p_iface, mu_star, F_star)."""

    FIELDS = ("dtau", "w0", "g0", "T_center", "T_iface", "p_iface", "mu_star", "F_star")

    def __init__(self, cols, device="cuda", pin: bool = False):
        self.n_layers = np.ascontiguousarray(cols.n_layers, dtype=np.int32)
        self.n_bins = np.ascontiguousarray(cols.n_bins, dtype=np.int32)
        self.n_cols = int(self.n_layers.size)
        self.n_g = int(cols.n_g)
        self.n_if = int((self.n_layers + 1).sum())
        self.n_lay = int(self.n_layers.sum())
        self.n_systems = int(self.n_bins.astype(np.int64).sum()) * self.n_g
        self.device = device
        for f in self.FIELDS:
            a = getattr(cols, f)
            t = torch.from_numpy(np.ascontiguousarray(a))
            setattr(self, f, t.to(device, non_blocking=False) if device != "cpu" else
                    (t.pin_memory() if pin else t))
        self._desc = None

    @classmethod
    def from_device(cls, dc) -> "DeviceBatch":
        """Wrap inputs that already live on the device (same field names)."""
        b = cls.__new__(cls)
        b.n_layers = np.ascontiguousarray(dc.n_layers, dtype=np.int32)
        b.n_bins = np.ascontiguousarray(dc.n_bins, dtype=np.int32)
        b.n_cols = int(b.n_layers.size)
        b.n_g = int(dc.n_g)
        b.n_if = int((b.n_layers + 1).sum())
        b.n_lay = int(b.n_layers.sum())
        b.n_systems = int(b.n_bins.astype(np.int64).sum()) * b.n_g
        b.device = str(dc.dtau.device)
        for f in cls.FIELDS:
            setattr(b, f, getattr(dc, f))
        b._desc = None
        return b

    @classmethod
    def empty_like(cls, other: "DeviceBatch", device="cuda") -> "DeviceBatch":
        b = cls.__new__(cls)
        for k in ("n_layers", "n_bins", "n_cols", "n_g", "n_if", "n_lay", "n_systems"):
            setattr(b, k, getattr(other, k))
        b.device = device
        for f in cls.FIELDS:
            t = getattr(other, f)
            setattr(b, f, torch.empty(t.shape, dtype=t.dtype, device=device))
        b._desc = None
        return b

    def copy_from(self, src: "DeviceBatch", non_blocking: bool = True):
        for f in self.FIELDS:
            getattr(self, f).copy_(getattr(src, f), non_blocking=non_blocking)

    @property
    def input_bytes(self) -> int:
        return sum(getattr(self, f).numel() * getattr(self, f).element_size() for f in self.FIELDS)

    def state_descriptor(self):
        """Descriptor without optics (for the k-table front end)."""
        if getattr(self, "_sdesc", None) is None:
            self._sdesc = rt.make_columns(self.n_cols, self.n_layers, self.n_bins, None, None, None,
                                          self.T_center, self.T_iface, self.p_iface, self.mu_star,
                                          self.F_star)
        return self._sdesc

    def descriptor(self):
        if self._desc is None:
            self._desc = rt.make_columns(self.n_cols, self.n_layers, self.n_bins, self.dtau, self.w0,
                                         self.g0, self.T_center, self.T_iface, self.p_iface,
                                         self.mu_star, self.F_star)
        return self._desc


class Solver:
    """One rt_handle with the paper's defaults (Table 3) unless overridden."""

    def __init__(self, g_weights, **cfg):
        self.cfg = rt.Config(g_weights=np.asarray(g_weights, np.float64), **cfg)
        self.h = rt.rt_create(self.cfg)

    def close(self):
        if self.h:
            rt.rt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query_bytes(self, batch: DeviceBatch) -> int:
        return rt.rt_query_bytes(self.h, batch.descriptor())

    def solve(self, batch: DeviceBatch, stream=None):
        rt.rt_solve_columns(self.h, batch.descriptor(), stream)

    def set_ktable(self, kt: dict):
        rt.rt_set_ktable(self.h, kt)

    def solve_ktable(self, batch: DeviceBatch, stream=None):
        """Solve with the optics from the k-table front end (``batch``'s
        dtau/w0/g0 are not read)."""
        rt.rt_solve_ktable(self.h, batch.state_descriptor(), stream)

    def ktable_optics(self, batch: DeviceBatch, stream=None) -> dict:
        """The front end's FP32 optics cubes for ``batch``."""
        n = int((batch.n_layers.astype(np.int64) * batch.n_bins).sum()) * batch.n_g
        o = {k: torch.empty(n, dtype=torch.float32, device="cuda") for k in ("dtau", "w0", "g0")}
        rt.rt_ktable_optics(self.h, batch.state_descriptor(), o["dtau"], o["w0"], o["g0"], stream)
        return o

    def outputs(self, batch: DeviceBatch, stream=None, device="cuda") -> dict:
        """Interface fluxes and heating of the last solve as tensors."""
        o = {k: torch.empty(batch.n_if, dtype=torch.float64, device=device)
             for k in ("F_up", "F_down", "F_net")}
        o["Q"] = torch.empty(batch.n_lay, dtype=torch.float64, device=device)
        rt.rt_fluxes(self.h, o["F_up"], o["F_down"], o["F_net"], stream)
        rt.rt_heating(self.h, o["Q"], stream)
        return o

    def outputs_host(self, n_if: int, n_lay: int, stream=None) -> dict:
        """The last solve's outputs (n_if interfaces, n_lay layers) as host arrays."""
        o = {k: np.empty(n_if) for k in ("F_up", "F_down", "F_net")}
        o["Q"] = np.empty(n_lay)
        rt.rt_fluxes(self.h, o["F_up"], o["F_down"], o["F_net"], stream)
        rt.rt_heating(self.h, o["Q"], stream)
        torch.cuda.synchronize()
        return o

    def toa_spectrum(self, batch: DeviceBatch, stream=None, device="cuda"):
        """Upward flux at the TOA per bin of the last solve, [sum NB]."""
        t = torch.empty(int(batch.n_bins.astype(np.int64).sum()), dtype=torch.float64, device=device)
        rt.rt_toa_spectrum(self.h, t, stream)
        return t

    def solve_numpy(self, batch: DeviceBatch) -> dict:
        self.solve(batch)
        o = self.outputs(batch)
        o["F_up_toa"] = self.toa_spectrum(batch)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in o.items()}

    def stats(self) -> dict:
        return rt.rt_stats(self.h)

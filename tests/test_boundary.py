"""The C-ABI library without a GPU: it loads, exports every entry point that
include/rt.h declares, and the ctypes mirrors of its structs have the
C layout.  No compute call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rt.h")


@pytest.fixture(scope="module")
def librt():
    from paper_2203_02293_b300 import build, rt
    if build.stale():
        build.build()
    return rt


def declared_functions(path=HEADER):
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(rt_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_path_entry_points():
    names = declared_functions()
    for n in ("rt_create", "rt_solve_columns", "rt_fluxes", "rt_heating", "rt_query_bytes",
              "rt_stats", "rt_last_error", "rt_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(librt):
    lib = ctypes.CDLL(librt.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_exports_no_torch_symbols(librt):
    out = subprocess.run(["nm", "-D", "--defined-only", librt.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = [l.split()[-1] for l in out.splitlines() if " T " in l]
    assert all(not s.startswith("_ZN2at") and "torch" not in s for s in exported)


def _c_layout(tmp_path, struct, fields):
    prog = ["#include <stdio.h>", "#include <stddef.h>", '#include "rt.h"', "int main(void){",
            f'printf("%zu\\n", sizeof({struct}));']
    prog += [f'printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    prog += ["return 0;}"]
    c = tmp_path / f"{struct}.c"
    c.write_text("\n".join(prog))
    exe = tmp_path / struct
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(c)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    return vals[0], vals[1:]


@pytest.mark.parametrize("name", ["rt_config", "rt_columns", "rt_stats_t", "rt_ktable"])
def test_ctypes_structs_match_c_layout(librt, tmp_path, name):
    cls = getattr(librt, name)
    fields = [f for f, _ in cls._fields_]
    size, offs = _c_layout(tmp_path, name, fields)
    assert ctypes.sizeof(cls) == size
    assert [getattr(cls, f).offset for f in fields] == offs


def test_status_codes_match_header(librt):
    src = open(HEADER).read()
    for name in ("RT_OK", "RT_EINVAL", "RT_ENOMEM", "RT_ECUDA", "RT_ENOTSOLVED", "RT_EBUDGET",
                 "RT_ETIMEOUT", "RT_IMPROVED", "RT_REGULAR", "RT_NONISOTHERMAL", "RT_ISOTHERMAL",
                 "RT_FP32_FORM", "RT_FP64_PLAIN", "RT_RESONANCE_PAPER", "RT_RESONANCE_LIMIT"):
        m = re.search(rf"\b{name}\s*=\s*(-?\d+)", src)
        assert m and int(m.group(1)) == getattr(librt, name), name


def test_create_without_a_gpu_fails_loudly(librt):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    with pytest.raises(librt.RTError):
        librt.rt_create(librt.Config(g_weights=np.ones(1)))


def test_bad_config_is_rejected_before_touching_the_device(librt):
    import numpy as np
    for bad in (dict(eps2=0.0), dict(max_layers=0), dict(block_threads=48), dict(precision=7),
                dict(wn_min=100.0, wn_max=50.0), dict(wn_edges=np.array([50.0])),
                dict(wn_edges=np.array([50.0, 40.0, 60.0])), dict(wn_edges=np.array([-1.0, 40.0])),
                dict(wn_edges=np.array([50.0, np.nan])), dict(planck_staging=4), dict(planck_staging=-1),
                dict(systems_per_lane=3)):
        cfg = librt.Config(g_weights=np.ones(1), **bad)
        with pytest.raises(librt.RTError) as e:
            librt.rt_create(cfg)
        assert e.value.code == librt.RT_EINVAL


def test_missing_library_raises(tmp_path):
    from paper_2203_02293_b300 import rt
    with pytest.raises(RuntimeError):
        rt._load(str(tmp_path / "nope.so"))


# ----------------------------------------------------------------------
# Host-only validation (rt_check_columns): gather offsets against the
# arrays' element counts.  No device call is made and no array is read.
# ----------------------------------------------------------------------

def _pool(rt):
    import numpy as np
    L = np.array([5, 3, 7], np.int32)
    NB = np.array([4, 6, 2], np.int32)
    ng = 3
    n_cube = int((L * NB).sum()) * ng
    arrs = dict(dtau=np.zeros(n_cube, np.float32), w0=np.zeros(n_cube, np.float32),
                g0=np.zeros(n_cube, np.float32), T_center=np.zeros(int(L.sum())),
                T_iface=np.zeros(int((L + 1).sum())), p_iface=np.zeros(int((L + 1).sum())),
                mu_star=np.zeros(3), F_star=np.zeros(int(NB.sum())))
    z = lambda a: np.concatenate([[0], np.cumsum(a)])[:-1].astype(np.int64)
    off = dict(cube_offset=z(L * NB * ng), center_offset=z(L), iface_offset=z(L + 1), bin_offset=z(NB),
               col_index=np.arange(3, dtype=np.int64))
    cfg = rt.Config(g_weights=np.full(ng, 1.0 / ng))
    return L, NB, arrs, off, cfg


def _desc(rt, L, NB, arrs, gather=None, counts=None):
    a = arrs
    return rt.make_columns(len(L), L, NB, a["dtau"], a["w0"], a["g0"], a["T_center"], a["T_iface"],
                           a["p_iface"], a["mu_star"], a["F_star"], gather=gather, counts=counts)


def test_check_columns_accepts_packed_and_gathered(librt):
    rt = librt
    L, NB, arrs, off, cfg = _pool(rt)
    assert rt.rt_check_columns(cfg, _desc(rt, L, NB, arrs)) == ""
    # gathered: the columns in reverse order, each block ending exactly at its column's end
    rev = {k: v[::-1].copy() for k, v in off.items()}
    assert rt.rt_check_columns(cfg, _desc(rt, L[::-1].copy(), NB[::-1].copy(), arrs, gather=rev)) == ""


@pytest.mark.parametrize("key,count_key,what", [
    ("cube_offset", "n_cube", "dtau/w0/g0"), ("center_offset", "n_center", "T_center"),
    ("iface_offset", "n_iface", "T_iface/p_iface"), ("bin_offset", "n_fstar", "F_star"),
    ("col_index", "n_mu", "mu_star")])
def test_check_columns_refuses_offset_past_the_end(librt, key, count_key, what):
    rt = librt
    L, NB, arrs, off, cfg = _pool(rt)
    bad = {k: v.copy() for k, v in off.items()}
    bad[key][2] += 1                      # the last column's block now ends one element past the array
    with pytest.raises(rt.RTError) as ei:
        rt.rt_check_columns(cfg, _desc(rt, L, NB, arrs, gather=bad))
    assert ei.value.code == rt.RT_EINVAL and what in str(ei.value)
    # a gather offset array without its count is refused too
    with pytest.raises(rt.RTError) as ei:
        rt.rt_check_columns(cfg, _desc(rt, L, NB, arrs, gather={key: off[key]}, counts={count_key: 0}))
    assert ei.value.code == rt.RT_EINVAL and "element count" in str(ei.value)


def test_check_columns_packed_count_too_small_and_negative(librt):
    rt = librt
    L, NB, arrs, off, cfg = _pool(rt)
    n = int((L * NB).sum()) * 3
    with pytest.raises(rt.RTError):
        rt.rt_check_columns(cfg, _desc(rt, L, NB, arrs, counts={"n_cube": n - 1}))
    with pytest.raises(rt.RTError):
        rt.rt_check_columns(cfg, _desc(rt, L, NB, arrs, counts={"n_mu": -1}))
    # huge offsets do not wrap around
    bad = {k: v.copy() for k, v in off.items()}
    bad["cube_offset"][0] = 2 ** 62
    with pytest.raises(rt.RTError):
        rt.rt_check_columns(cfg, _desc(rt, L, NB, arrs, gather=bad))


def test_check_columns_refuses_bad_config_and_sweep_limits(librt):
    import numpy as np
    rt = librt
    L, NB, arrs, off, cfg = _pool(rt)
    from dataclasses import replace
    with pytest.raises(rt.RTError):
        rt.rt_check_columns(replace(cfg, n_sweeps=-1), _desc(rt, L, NB, arrs))
    assert rt.rt_check_columns(replace(cfg, n_sweeps=10), _desc(rt, L, NB, arrs)) == ""
    tall = np.array([rt.RT_SWEEP_MAX_LAYERS + 1], np.int32)
    big = {k: np.zeros(10000, v.dtype) for k, v in arrs.items()}
    with pytest.raises(rt.RTError) as ei:
        rt.rt_check_columns(replace(cfg, n_sweeps=10), _desc(rt, tall, np.array([2], np.int32), big))
    assert "iterative" in str(ei.value)
    with pytest.raises(rt.RTError):
        rt.rt_check_columns(replace(cfg, n_sweeps=10, precision=rt.RT_FP64_PLAIN), _desc(rt, L, NB, arrs))

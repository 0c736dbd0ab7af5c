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

"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/smc.h declares (no compute call: this runs without a GPU)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    src = (ROOT / "include" / "smc.h").read_text()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(smc_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def built():
    from paper_1905_10252_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("smc_init", "smc_reweight", "smc_resample", "smc_redistribute", "smc_move", "smc_step"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(str(built))
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(built):
    from paper_1905_10252_gb300 import native

    assert sorted(native.EXPORTED) == declared_functions()
    native.load_library()  # loads without a GPU


def test_workspace_sizes_host_only(built):
    from paper_1905_10252_gb300 import native

    L = native.load_library()
    for n in (1, 4095, 4096, 4097, 2 ** 24):
        out = ctypes.c_size_t()
        assert L.smc_redistribute_ws_bytes(n, ctypes.byref(out)) == 0
        assert out.value >= 4 * (n + 1)
    bad = ctypes.c_size_t()
    assert L.smc_redistribute_ws_bytes(0, ctypes.byref(bad)) == native.SMC_EINVAL
    cfg = native.smc_config()
    cfg.n, cfg.d, cfg.dtype, cfg.target = 1024, 4, native.SMC_F64, native.SMC_GAUSS
    cfg.step, cfg.init_scale = 0.5, 2.0
    cfg.mu_dev, cfg.sigma_dev = 256, 512  # never dereferenced by this host-only query
    out = ctypes.c_size_t()
    assert L.smc_workspace_bytes(ctypes.byref(cfg), ctypes.byref(out)) == 0
    cfg.d = 33
    assert L.smc_workspace_bytes(ctypes.byref(cfg), ctypes.byref(out)) == native.SMC_EINVAL


def test_no_oracle_in_product_package():
    pkg = ROOT / "paper_1905_10252_gb300"
    for p in list(pkg.rglob("*.py")) + list(pkg.rglob("*.cu")) + list(pkg.rglob("*.cuh")) + list(pkg.rglob("*.h")):
        text = p.read_text()
        assert "oracle" not in text.lower(), p

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


def test_init_rejects_bad_arguments_host_only(built):
    """smc_init validates everything before its first CUDA call: bad sizes,
    dtypes, targets and pointers give SMC_EINVAL, a workspace smaller than
    smc_workspace_bytes gives SMC_ENOMEM (admission refused), and no handle is
    returned.  The fake device addresses are never dereferenced."""
    from paper_1905_10252_gb300 import native

    L = native.load_library()
    A = 1 << 24  # 256-byte aligned fake device addresses

    def cfg(**kw):
        c = native.smc_config()
        c.n, c.d, c.dtype, c.target = 1024, 4, native.SMC_F32, native.SMC_GAUSS
        c.step, c.init_scale = 0.5, 2.0
        c.mu_dev, c.sigma_dev = A, A + 4096
        for k, v in kw.items():
            setattr(c, k, v)
        return c

    def init(c, ws_bytes=None, x=A, ws=A + (1 << 20)):
        if ws_bytes is None:
            need = ctypes.c_size_t()
            assert L.smc_workspace_bytes(ctypes.byref(c), ctypes.byref(need)) == 0
            ws_bytes = need.value
        h = ctypes.c_void_p(7)
        rc = L.smc_init(ctypes.byref(h), ctypes.byref(c), x, x, A, A, A, ws, ws_bytes, None)
        assert h.value is None  # no handle on failure
        return rc

    bad = [dict(n=0), dict(n=2 ** 31), dict(d=0), dict(d=33), dict(dtype=7), dict(target=9),
           dict(resample_mode=3), dict(step=-1.0), dict(init_scale=0.0), dict(mu_dev=None),
           dict(target=native.SMC_STUDENT_T, d=2, nu=5.0), dict(target=native.SMC_STUDENT_T, nu=0.0, d=1),
           dict(target=native.SMC_LOGISTIC, X_dev=None, y_dev=A, m=10, prior_var=1.0),
           dict(target=native.SMC_LOGISTIC, X_dev=A, y_dev=A, m=10, prior_var=0.0),
           dict(nstar=-1), dict(nstar=1025)]
    for kw in bad:
        c = cfg(**kw)
        assert L.smc_workspace_bytes(ctypes.byref(c), ctypes.byref(ctypes.c_size_t())) == native.SMC_EINVAL, kw
        assert init(c, ws_bytes=1 << 30) == native.SMC_EINVAL, kw
    c = cfg()
    assert init(c, x=0) == native.SMC_EINVAL  # null buffer
    assert init(c, x=A + 4) == native.SMC_EINVAL  # particle buffer not 16-byte aligned
    assert init(c, ws=A + 128) == native.SMC_EINVAL  # workspace not 256-byte aligned
    need = ctypes.c_size_t()
    L.smc_workspace_bytes(ctypes.byref(c), ctypes.byref(need))
    assert init(c, ws_bytes=need.value - 1) == native.SMC_ENOMEM
    assert b"workspace too small" in L.smc_last_error(None)


def test_struct_layouts_match_the_header(built, tmp_path):
    """The binding's ctypes structures have the sizes and field offsets that
    a C compiler gives the header's structs (gcc, host only)."""
    import shutil
    import subprocess

    from paper_1905_10252_gb300 import native

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"smc_config": native.smc_config, "smc_iter_stats": native.smc_iter_stats}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "smc.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", str(ROOT / "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[f"{name}.{field}"]) == getattr(cls, field).offset, (name, field)



def test_stateless_calls_reject_bad_arguments_host_only(built):
    """The stateless entry points check sizes, pointers, alignment and the
    event count before any CUDA call."""
    from paper_1905_10252_gb300 import native

    L = native.load_library()
    A = 1 << 24  # fake, aligned device addresses (never dereferenced)
    EINVAL = native.SMC_EINVAL
    assert L.smc_redistribute_raw(0, 16, A, A, A, A, None) == EINVAL        # n = 0
    assert L.smc_redistribute_raw(2 ** 31, 16, A, A, A, A, None) == EINVAL  # n too large
    assert L.smc_redistribute_raw(100, 6, A, A, A, A, None) == EINVAL       # row bytes
    assert L.smc_redistribute_raw(100, 16, A, A, A, A + 8, None) == EINVAL  # workspace alignment
    assert L.smc_redistribute_raw(100, 16, A, A + 4, A, A, None) == EINVAL  # rows misaligned
    ev = (ctypes.c_void_p * 3)(A, A, A)
    assert L.smc_redistribute_raw_profile(100, 16, A, A, A, A, None, ev, 2) == EINVAL  # event count
    assert L.smc_redistribute_raw_profile(100, 16, A, A, A, A, None, None, 3) == EINVAL  # null events
    assert L.smc_nearly_sort_raw(100, 16, A + 4, A, A, A, A, None) == EINVAL  # keys misaligned
    assert L.smc_resample_raw(100, A, 0, 0, 3, A, None, A, None) == EINVAL    # mode
    out = ctypes.c_size_t()
    assert L.smc_nearly_sort_ws_bytes(0, ctypes.byref(out)) == EINVAL
    assert L.smc_nearly_sort_ws_bytes(5000, ctypes.byref(out)) == 0 and out.value >= 2 * 4 * 2


def test_binding_constants_match_header():
    """Status codes, dtypes, targets, resampling modes and flags: the values
    the binding passes are the header's (enumerators and #defines)."""
    from paper_1905_10252_gb300 import native

    src = re.sub(r"/\*.*?\*/", "", (ROOT / "include" / "smc.h").read_text(), flags=re.S)
    values = {k: int(v) for k, v in re.findall(r"\b(SMC_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)}
    values.update({k: int(v) for k, v in re.findall(r"^#define\s+(SMC_[A-Z0-9_]+)\s+(\d+)\s*$", src, flags=re.M)})
    checked = 0
    for name, v in values.items():
        py = name[len("SMC_"):] if name.startswith(("SMC_FLAG_", "SMC_RESAMPLE_")) else name
        if hasattr(native, py):
            assert getattr(native, py) == v, (name, getattr(native, py), v)
            checked += 1
    for required in ("SMC_OK", "SMC_ENONFINITE", "SMC_F32", "SMC_GAUSS", "SMC_RESAMPLE_ALWAYS",
                     "SMC_FLAG_DEFER_REDISTRIBUTE"):
        assert required in values
    assert checked >= 16

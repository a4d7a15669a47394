"""The library's NVTX ranges reach a profiler: a small NVTX tool
(tests/nvtx_probe.c, loaded through NVTX_INJECTION64_PATH as Nsight tools
are) records the range events of the domain "libsmc" while entry points run
their host-side argument checks (no GPU needed)."""
import os
import shutil
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
CUDA_INC = Path(os.environ.get("CUDA_HOME", "/usr/local/cuda")) / "include"

CHILD = r"""
import ctypes
from paper_1905_10252_gb300 import native
L = native.load_library()
cfg = native.smc_config()
cfg.n, cfg.d, cfg.dtype, cfg.target = 0, 4, native.SMC_F32, native.SMC_GAUSS  # n = 0: rejected
h = ctypes.c_void_p()
assert L.smc_init(ctypes.byref(h), ctypes.byref(cfg), None, None, None, None, None, None, 0, None) == native.SMC_EINVAL
assert L.smc_redistribute_raw(0, 16, None, None, None, None, None) == native.SMC_EINVAL
assert L.smc_nearly_sort_raw(0, 16, None, None, None, None, None, None) == native.SMC_EINVAL
"""


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None or not (CUDA_INC / "nvtx3" / "nvToolsExt.h").exists():
        pytest.skip("needs a C compiler and the NVTX v3 headers")
    from paper_1905_10252_gb300 import build

    build.build()
    so = tmp_path_factory.mktemp("nvtx") / "libnvtx_probe.so"
    subprocess.run([cc, "-shared", "-fPIC", "-O1", "-I", str(CUDA_INC), str(ROOT / "tests" / "nvtx_probe.c"),
                    "-o", str(so)], check=True)
    return so


def test_entry_points_emit_balanced_ranges(probe, tmp_path):
    log = tmp_path / "ranges.txt"
    env = dict(os.environ, NVTX_INJECTION64_PATH=str(probe), SMC_NVTX_PROBE_OUT=str(log),
               PYTHONPATH=str(ROOT) + os.pathsep + os.environ.get("PYTHONPATH", ""))
    subprocess.run([sys.executable, "-c", CHILD], env=env, check=True, cwd=str(ROOT))
    events = log.read_text().split("\n")
    pushes = [e.split(" ", 1)[1] for e in events if e.startswith("push ")]
    assert pushes == ["smc_init", "smc_redistribute_raw", "smc_nearly_sort_raw"]
    assert events.count("pop") == len(pushes)

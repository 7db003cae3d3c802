"""C-ABI library: builds, loads and exports every symbol include/atdct16.h
declares; its host-side butterfly (same source as the device kernels) matches
the oracle's T.  No GPU needed."""

import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1606_05562_gb300 import atdct16, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return atdct16.lib()


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "atdct16.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(atdct16_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for required in ["atdct16_plan_create", "atdct16_plan_destroy", "atdct16_forward", "atdct16_inverse",
                     "atdct16_compress_zonal", "atdct16_compress_quant", "atdct16_psnr",
                     "atdct16_last_device_status", "atdct16_status_string"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    assert atdct16.status_string(atdct16.OK) == "ok"
    assert "invalid" in atdct16.status_string(atdct16.EINVAL)
    assert lib.atdct16_version().decode().startswith("atdct16")


def test_host_butterfly_matches_t_on_unit_vectors(lib):
    for j in range(16):
        e = [0] * 16
        e[j] = 1
        assert atdct16.host_butterfly(e) == list(O.T[:, j])
        assert atdct16.host_butterfly(e, inverse=True) == list(O.T[j, :])


def test_host_butterfly_random_vectors(lib):
    # the FPGA co-simulation of Sec. 5.2 used 10,000 random 16-point vectors
    rng = np.random.default_rng(1191)
    for _ in range(10000):
        x = rng.integers(-255, 256, size=16)
        assert atdct16.host_butterfly(x) == list(O.T @ x)
        assert atdct16.host_butterfly(x, inverse=True) == list(O.T.T @ x)


def test_host_butterfly_every_pm255_vector(lib):
    # all 2^16 vectors with entries +-255: the extremes of every output row
    signs = ((np.arange(1 << 16)[:, None] >> np.arange(16)) & 1) * 2 - 1
    x = 255 * signs
    want_f, want_i = x @ O.T.T, x @ O.T
    for k in range(1 << 16):
        assert atdct16.host_butterfly(x[k]) == list(want_f[k])
        assert atdct16.host_butterfly(x[k], inverse=True) == list(want_i[k])


def test_null_arguments_rejected_without_gpu(lib):
    assert lib.atdct16_host_butterfly(None, None, 0) == atdct16.EINVAL
    assert lib.atdct16_plan_destroy(None) == atdct16.EINVAL


def test_kernel_zigzag_tables_match_the_oracle_scan(tmp_path):
    """The device-side scan tables (zigzag_word / zigzag_rank, compiled here
    for the host) against the oracle's own walk of the Sec. 4 scan."""
    src = tmp_path / "zz.cpp"
    src.write_text(
        '#include "atdct16_zigzag.cuh"\n#include <cstdio>\n'
        "int main() {\n"
        '  for (int k = 0; k < 256; ++k) std::printf("%d %d\\n", atdct16::zigzag_word(k), atdct16::zigzag_rank(k));\n'
        "  return 0;\n}\n")
    exe = tmp_path / "zz"
    import shutil
    import subprocess
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_1606_05562_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True)
    rows = [tuple(map(int, ln.split())) for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                                 check=True).stdout.split("\n") if ln]
    order = O.zigzag_order()
    rank = O.zigzag_rank()
    assert [w for w, _ in rows] == [16 * u + v for u, v in order]
    assert [r for _, r in rows] == [int(rank[w >> 4, w & 15]) for w in range(256)]

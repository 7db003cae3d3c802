"""The fused kernel's packed int16 forward (two blocks per 32-bit word,
offset-binary fields) run on the host with the kernels' own butterfly and
value type (atdct16_butterfly.cuh, atdct16_ops.cuh): row pass, DC centring
by -2048, column pass, then the fields unpacked must equal Y = T X T^T of
both blocks exactly, with T taken from the oracle (not from the butterfly).
Random, extreme and worst-case blocks.  No GPU needed."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS = r"""
#include <cstdio>
#include <cstdlib>

#include "atdct16_butterfly.cuh"

using atdct16::Swar16;

static const int kT[16][16] = { __T__ };

// forward of two blocks a (low fields) and b (high fields) as the fused kernel does it
static void swar_forward(const int (&a)[16][16], const int (&b)[16][16], long long (&ya)[16][16],
                         long long (&yb)[16][16]) {
  Swar16 rows[16][16];
  for (int m = 0; m < 16; ++m) {
    Swar16 x[16], r[16];
    for (int n = 0; n < 16; ++n) x[n].v = (unsigned)(a[m][n] + 32768) | ((unsigned)(b[m][n] + 32768) << 16);
    atdct16::fwd16(x, r);
    r[0].v -= 0x08000800u;  // centre the DC output by -2048 in both fields
    for (int k = 0; k < 16; ++k) rows[m][k] = r[k];
  }
  for (int k = 0; k < 16; ++k) {
    Swar16 c[16], y[16];
    for (int m = 0; m < 16; ++m) c[m] = rows[m][k];
    atdct16::fwd16(c, y);
    for (int u = 0; u < 16; ++u) {
      ya[u][k] = (long long)(y[u].v & 0xffffu) - 32768;
      yb[u][k] = (long long)(y[u].v >> 16) - 32768;
    }
  }
  ya[0][0] += 16 * 2048;
  yb[0][0] += 16 * 2048;
}

static void direct(const int (&x)[16][16], long long (&y)[16][16]) {
  for (int u = 0; u < 16; ++u)
    for (int v = 0; v < 16; ++v) {
      long long s = 0;
      for (int m = 0; m < 16; ++m)
        for (int n = 0; n < 16; ++n) s += (long long)kT[u][m] * x[m][n] * kT[v][n];
      y[u][v] = s;
    }
}

int main() {
  int nblk = 0;
  if (std::scanf("%d", &nblk) != 1) return 2;
  static int blk[4096][16][16];
  for (int i = 0; i < nblk; ++i)
    for (int m = 0; m < 16; ++m)
      for (int n = 0; n < 16; ++n)
        if (std::scanf("%d", &blk[i][m][n]) != 1) return 2;
  int bad = 0;
  for (int i = 0; i + 1 < nblk; i += 2) {
    long long ya[16][16], yb[16][16], ra[16][16], rb[16][16];
    swar_forward(blk[i], blk[i + 1], ya, yb);
    direct(blk[i], ra);
    direct(blk[i + 1], rb);
    for (int u = 0; u < 16; ++u)
      for (int v = 0; v < 16; ++v) bad += (ya[u][v] != ra[u][v]) + (yb[u][v] != rb[u][v]);
  }
  std::printf("%d\n", bad);
  return 0;
}
"""


def _blocks():
    rng = np.random.default_rng(2016)
    out = [rng.integers(0, 256, size=(16, 16)) for _ in range(600)]
    out += [np.full((16, 16), c) for c in (0, 1, 127, 128, 254, 255)]
    i, j = np.indices((16, 16))
    out += [255 * ((i + j) % 2), 255 * (1 - (i + j) % 2), 255 * (i % 2), 255 * (j % 2)]
    # blocks aligned with the signs of T's rows and columns (the column-pass extremes)
    for u in range(16):
        for v in range(16):
            s = np.outer(O.T[u], O.T[v])
            out.append(np.where(s > 0, 255, 0))
            out.append(np.where(s < 0, 255, 0))
    if len(out) % 2:
        out.append(np.zeros((16, 16), dtype=np.int64))
    return out


def test_packed_int16_forward_is_exact(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = HARNESS.replace("__T__", ", ".join("{" + ", ".join(str(int(t)) for t in row) + "}" for row in O.T))
    (tmp_path / "swar.cpp").write_text(src)
    exe = tmp_path / "swar"
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_1606_05562_gb300", "csrc"),
                    str(tmp_path / "swar.cpp"), "-o", str(exe)], check=True)
    blocks = _blocks()
    assert len(blocks) <= 4096
    text = f"{len(blocks)}\n" + "\n".join(" ".join(str(int(v)) for v in b.reshape(-1)) for b in blocks)
    out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True).stdout
    assert int(out.strip()) == 0

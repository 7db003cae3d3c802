"""The fused zonal kernel's arithmetic, step for step, on the host: the
packed int16 forward with DC centring, 256 Y as an FP32 value, the per-r
weight keep W_u W_v / 256, the FP32 inverse column and row passes (each
f32x2 lane is an IEEE single-precision add, emulated per lane), and the
rounding fl(fl(Z fl(1/2304)) 2^-149) read as an int32 and saturated to u8 —
using the kernels' own butterfly header and value types.  The stored pixels
must equal the oracle's exact reconstruction for every r.  No GPU needed."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_1606_05562_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS = r"""
#include <cstdio>
#include <cstring>

namespace atdct16 {
// one lane of the device's f32x2 butterflies: an IEEE single-precision add
inline float badd(float a, float b) { return a + b; }
inline float bsub(float a, float b) { return a - b; }
}  // namespace atdct16

#include "atdct16_butterfly.cuh"
#include "atdct16_zigzag.cuh"

using atdct16::Swar16;

static unsigned bits(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
static float from_bits(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }

int main() {
  // W_u = 48 / nnz_u from the butterfly's response to unit vectors
  int w[16];
  for (int u = 0; u < 16; ++u) w[u] = 0;
  {
    int nnz[16] = {};
    for (int i = 0; i < 16; ++i) {
      long long x[16] = {}, y[16];
      x[i] = 1;
      atdct16::fwd16(x, y);
      for (int u = 0; u < 16; ++u) nnz[u] += y[u] != 0;
    }
    for (int u = 0; u < 16; ++u) w[u] = 48 / nnz[u];
  }
  const volatile float inv2304 = 1.0f / 2304.0f;
  const float tiny = from_bits(1u);
  int nblk = 0, r = 0;
  while (std::scanf("%d %d", &nblk, &r) == 2) {
    static int blk[2][16][16];
    for (int i = 0; i < 2; ++i)
      for (int m = 0; m < 16; ++m)
        for (int n = 0; n < 16; ++n)
          if (std::scanf("%d", &blk[i][m][n]) != 1) return 2;
    // forward, two blocks per word
    Swar16 rows[16][16];
    for (int m = 0; m < 16; ++m) {
      Swar16 x[16], o[16];
      for (int n = 0; n < 16; ++n) x[n].v = (unsigned)(blk[0][m][n] + 32768) | ((unsigned)(blk[1][m][n] + 32768) << 16);
      atdct16::fwd16(x, o);
      o[0].v -= 0x08000800u;
      for (int k = 0; k < 16; ++k) rows[m][k] = o[k];
    }
    float d[2][16][16];  // weighted coefficients, d[b][u][v]
    for (int v = 0; v < 16; ++v) {
      Swar16 c[16], y[16];
      for (int m = 0; m < 16; ++m) c[m] = rows[m][v];
      atdct16::fwd16(c, y);
      for (int u = 0; u < 16; ++u) {
        const bool keep = atdct16::zigzag_rank(16 * u + v) < r;
        const float kw = keep ? (float)(w[u] * w[v]) / 256.0f : 0.0f;
        for (int b = 0; b < 2; ++b) {
          const int field = b ? (int)(y[u].v >> 16) : (int)(y[u].v & 0xffffu);
          // 2^23 + field -> 256 field - 256 (2^23 + 32768) (+ the centring back for the DC of column 0)
          const float f = (float)(8388608 + field);
          const float o = (u == 0 && v == 0) ? -2147483648.0f : -2155872256.0f;
          const float y256 = f * 256.0f + o;  // exact: the device uses one FMA, both round the same exact value
          d[b][u][v] = y256 * kw;
        }
      }
    }
    for (int b = 0; b < 2; ++b) {
      float uu[16][16];  // after the inverse column pass: uu[m][v]
      for (int v = 0; v < 16; ++v) {
        float col[16], out[16];
        for (int u = 0; u < 16; ++u) col[u] = d[b][u][v];
        atdct16::inv16(col, out);
        for (int m = 0; m < 16; ++m) uu[m][v] = out[m];
      }
      for (int m = 0; m < 16; ++m) {
        float z[16];
        atdct16::inv16(uu[m], z);
        for (int n = 0; n < 16; ++n) {
          const float t = z[n] * inv2304;
          int q = (int)bits(t * tiny);
          q = q < 0 ? 0 : (q > 255 ? 255 : q);
          std::printf("%d ", q);
        }
      }
      std::printf("\n");
    }
  }
  return 0;
}
"""


def _cases():
    rng = np.random.default_rng(4)
    img = synth.ar1_image(64, 64, 0.95, 3)
    blocks = [img[16 * i:16 * i + 16, 16 * j:16 * j + 16] for i in range(4) for j in range(4)]
    blocks += [rng.integers(0, 256, size=(16, 16)) for _ in range(12)]
    i, j = np.indices((16, 16))
    blocks += [np.full((16, 16), 255), np.zeros((16, 16), dtype=np.int64), 255 * ((i + j) % 2),
               np.where(np.outer(O.T[3], O.T[11]) > 0, 255, 0)]
    return [np.asarray(b, dtype=np.int64) for b in blocks]


def test_fused_kernel_arithmetic_matches_exact_reconstruction(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src, exe = tmp_path / "fused.cpp", tmp_path / "fused"
    src.write_text(HARNESS)
    # -ffp-contract=off: every FP32 operation rounds on its own, as the device code does
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I",
                    os.path.join(ROOT, "paper_1606_05562_gb300", "csrc"), str(src), "-o", str(exe)], check=True)
    blocks = _cases()
    lines, want = [], []
    for r in (0, 1, 2, 6, 16, 36, 64, 100, 150, 255, 256):
        for a, b in zip(blocks[0::2], blocks[1::2]):
            lines.append(f"2 {r}\n" + " ".join(str(int(v)) for v in np.concatenate([a.ravel(), b.ravel()])))
            want += [O.compress_zonal_exact(a.astype(np.uint8), r)["recon_u8"],
                     O.compress_zonal_exact(b.astype(np.uint8), r)["recon_u8"]]
    out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True).stdout
    got = [np.array(ln.split(), dtype=np.int64).reshape(16, 16) for ln in out.splitlines()]
    assert len(got) == len(want)
    bad = sum(int(np.count_nonzero(g != w)) for g, w in zip(got, want))
    assert bad == 0, bad

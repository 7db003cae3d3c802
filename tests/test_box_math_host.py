"""The small-extent zonal kernel's arithmetic (r <= 36, the kept set inside
the K x K low-frequency corner), step for step on the host with the kernels'
own butterfly header and value types: the packed int16 forward pruned to K
outputs per pass with the pixels centred at 128, the scaled coefficient
keep W_u W_v Y_c as one FMA on the float 2^23 + field (plus 2304 * 128 on the
DC of column 0), the FP32 inverse over MaybeZero inputs (inputs at or above
K known to be zero), the rounding fl(fl(Z fl(1/2304)) 2^-149), and the exact
squared error 2304 SSE = 2304 sum (x - 128)^2 - sum_kept W_u W_v Y_c^2 from
the byte energy and the DC coefficient; for K = 1 the DC-only body (block
sums, the constant 9 Y_c + 2304 * 128 rounded the same way).  Stored pixels
must equal the oracle's exact reconstruction and 2304 SSE its exact integer,
for every r of each class.  No GPU needed."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_1606_05562_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS = r"""
#include <cmath>
#include <cstdio>
#include <cstring>

namespace atdct16 {
// one lane of the device's f32x2 butterflies: an IEEE single-precision add
inline float badd(float a, float b) { return a + b; }
inline float bsub(float a, float b) { return a - b; }
}  // namespace atdct16

#include "atdct16_butterfly.cuh"
#include "atdct16_zigzag.cuh"

using atdct16::MaybeZero;
using atdct16::Swar16;
using ZF = MaybeZero<float>;

static unsigned bits(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
static float from_bits(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }

int main() {
  int nnz[16];
  atdct16::row_nonzeros(nnz);
  int w[16];
  for (int u = 0; u < 16; ++u) w[u] = 48 / nnz[u];
  const volatile float inv2304 = 1.0f / 2304.0f;
  const float tiny = from_bits(1u);
  int K = 0, r = 0;
  while (std::scanf("%d %d", &K, &r) == 2) {
    static int blk[2][16][16];
    for (int i = 0; i < 2; ++i)
      for (int m = 0; m < 16; ++m)
        for (int n = 0; n < 16; ++n)
          if (std::scanf("%d", &blk[i][m][n]) != 1) return 2;
    // pixel energy of both blocks, as dp4a sums it
    unsigned ex = 0;
    for (int i = 0; i < 2; ++i)
      for (int m = 0; m < 16; ++m)
        for (int n = 0; n < 16; ++n) ex += (unsigned)(blk[i][m][n] * blk[i][m][n]);
    if (K == 1) {
      // the DC-only kernel: block sums, the constant 9 Y_c + 2304 * 128, rounded
      long long kept = 0, dcs = 0;
      for (int b = 0; b < 2; ++b) {
        int s = 0;
        for (int m = 0; m < 16; ++m)
          for (int n = 0; n < 16; ++n) s += blk[b][m][n];
        const int yc = s - 32768;
        const float z = std::fmaf((float)yc, 9.0f, 294912.0f);
        const float t = z * inv2304;
        int q = (int)bits(t * tiny);
        q = q < 0 ? 0 : (q > 255 ? 255 : q);
        for (int k = 0; k < 256; ++k) std::printf("%d ", q);
        std::printf("\n");
        kept += 9LL * yc * yc;
        dcs += yc;
      }
      std::printf("%lld\n", 2304LL * ((long long)ex - 256 * dcs - 2 * 4194304LL) - kept);
      continue;
    }
    // K > 1: row pass (outputs c < K used), DC centred by -2048
    Swar16 rows[16][16];
    for (int m = 0; m < 16; ++m) {
      Swar16 x[16], o[16];
      for (int n = 0; n < 16; ++n) x[n].v = (unsigned)(blk[0][m][n] + 32768) | ((unsigned)(blk[1][m][n] + 32768) << 16);
      atdct16::fwd16(x, o);
      o[0].v -= 0x08000800u;
      for (int k = 0; k < 16; ++k) rows[m][k] = o[k];
    }
    // column pass on columns c < K, outputs u < K; scaled coefficients and kept energy
    ZF d[2][16][16];
    unsigned long long ke = 0;
    long long dc = 0;
    for (int b = 0; b < 2; ++b)
      for (int u = 0; u < 16; ++u)
        for (int v = 0; v < 16; ++v) d[b][u][v] = ZF{0.0f, true};
    for (int c = 0; c < K; ++c) {
      Swar16 col[16], y[16];
      for (int m = 0; m < 16; ++m) col[m] = rows[m][c];
      atdct16::fwd16(col, y);
      for (int u = 0; u < K; ++u) {
        const bool keep = atdct16::zigzag_rank(16 * u + c) < r;
        const unsigned kwi = keep ? (unsigned)(w[u] * w[c]) : 0u;
        const float kwf = (float)kwi;
        const float kc = -kwf * 8421376.0f + ((u == 0 && c == 0) ? 294912.0f : 0.0f);
        for (int b = 0; b < 2; ++b) {
          const unsigned field = b ? (y[u].v >> 16) : (y[u].v & 0xffffu);
          const float f = from_bits(0x4B000000u | field);  // 2^23 + field
          d[b][u][c] = ZF{std::fmaf(f, kwf, kc), false};
          const int yc = (int)(bits(f) - 0x4B008000u);
          ke += (unsigned long long)(unsigned)(yc * yc) * kwi;
          if (u == 0 && c == 0) dc += yc;
        }
      }
    }
    const long long nume = 2304LL * ((long long)ex - 256 * dc - 2 * 4194304LL) - (long long)ke;
    for (int b = 0; b < 2; ++b) {
      ZF uu[16][16];  // after the inverse column pass: uu[m][c]
      for (int m = 0; m < 16; ++m)
        for (int c = 0; c < 16; ++c) uu[m][c] = ZF{0.0f, true};
      for (int c = 0; c < K; ++c) {
        ZF in[16], out[16];
        for (int u = 0; u < 16; ++u) in[u] = d[b][u][c];
        atdct16::inv16(in, out);
        for (int m = 0; m < 16; ++m) uu[m][c] = out[m];
      }
      for (int m = 0; m < 16; ++m) {
        ZF z[16];
        atdct16::inv16(uu[m], z);
        for (int n = 0; n < 16; ++n) {
          const float t = z[n].v * inv2304;
          int q = (int)bits(t * tiny);
          q = q < 0 ? 0 : (q > 255 ? 255 : q);
          std::printf("%d ", q);
        }
      }
      std::printf("\n");
    }
    std::printf("%lld\n", nume);
  }
  return 0;
}
"""

# (K, r values of that class) as the kernels use them
CLASSES = [(1, (1,)), (3, (2, 3, 5, 6)), (6, (7, 10, 15, 16, 21)), (8, (22, 28, 30, 36))]


def _cases():
    rng = np.random.default_rng(5)
    img = synth.ar1_image(64, 64, 0.95, 9)
    noisy = synth.ar1_image(32, 64, 0.8, 10, noise_sigma=8.0)
    blocks = [img[16 * i:16 * i + 16, 16 * j:16 * j + 16] for i in range(4) for j in range(4)]
    blocks += [noisy[16 * i:16 * i + 16, 16 * j:16 * j + 16] for i in range(2) for j in range(4)]
    blocks += [rng.integers(0, 256, size=(16, 16)) for _ in range(8)]
    i, j = np.indices((16, 16))
    blocks += [np.full((16, 16), 255), np.zeros((16, 16), dtype=np.int64), 255 * ((i + j) % 2),
               np.where(np.outer(O.T[3], O.T[11]) > 0, 255, 0), np.where(np.outer(O.T[1], O.T[2]) > 0, 255, 0),
               np.where(np.outer(O.T[7], O.T[0]) < 0, 255, 0)]
    return [np.asarray(b, dtype=np.int64) for b in blocks]


def test_box_kernel_arithmetic_matches_exact_reconstruction(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src, exe = tmp_path / "box.cpp", tmp_path / "box"
    src.write_text(HARNESS)
    # -ffp-contract=off: every FP32 operation rounds on its own, as the device code does
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I",
                    os.path.join(ROOT, "paper_1606_05562_gb300", "csrc"), str(src), "-o", str(exe)], check=True)
    blocks = _cases()
    lines, want_px, want_sse = [], [], []
    for k, rs in CLASSES:
        for r in rs:
            for a, b in zip(blocks[0::2], blocks[1::2]):
                lines.append(f"{k} {r}\n" + " ".join(str(int(v)) for v in np.concatenate([a.ravel(), b.ravel()])))
                ea = O.compress_zonal_exact(a.astype(np.uint8), r)
                eb = O.compress_zonal_exact(b.astype(np.uint8), r)
                want_px += [ea["recon_u8"], eb["recon_u8"]]
                # the oracle's exact squared error, scaled by 2304^2
                want_sse.append(int(ea["block_sse"].sum() * 2304 * 2304 + 0.5) +
                                int(eb["block_sse"].sum() * 2304 * 2304 + 0.5))
    out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.splitlines()
    assert len(out) == 3 * len(want_sse)
    bad_px = bad_sse = 0
    for n, ws in enumerate(want_sse):
        for i in range(2):
            g = np.array(out[3 * n + i].split(), dtype=np.int64).reshape(16, 16)
            bad_px += int(np.count_nonzero(g != want_px[2 * n + i]))
        bad_sse += int(2304 * int(out[3 * n + 2]) != ws)
    assert bad_px == 0, bad_px
    assert bad_sse == 0, bad_sse


def test_box_class_bounds():
    # every r of a class keeps only coefficients inside its K x K corner, and
    # the next r would leave it: r <= K (K + 1) / 2 is the class's limit
    for k, _ in CLASSES:
        rmax = k * (k + 1) // 2
        assert np.all(np.argwhere(O.zonal_mask(rmax)).max(axis=0) < k)
        assert np.argwhere(O.zonal_mask(rmax + 1)).max() >= k

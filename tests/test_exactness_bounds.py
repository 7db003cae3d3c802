"""Exactness of the fused zonal kernel's arithmetic for every u8 input, pinned
by running the kernels' own butterfly source (atdct16_butterfly.cuh) on the
host over linear forms: every node is a form in the 256 pixels of a block,
and its exact range over [0, 255]^256 is read off its coefficients.

- forward row and column passes on int16 fields (bias 32768), with the DC
  row output centred by -2048 as in the kernel: every node must stay in
  [-32768, 32767], or the packed 32-bit adds would carry between fields;
- inverse column and row passes on FP32, fed with keep(u, v) W_u W_v Y for
  every zig-zag prefix r = 1..256: every node must stay below 2^24 in
  magnitude, so that FP32 holds each one exactly.
No GPU needed."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS = r"""
#include <algorithm>
#include <array>
#include <cstdio>

namespace atdct16 {
// a linear form sum_i c[i] x_i + k over the 256 pixels x_i of one block
struct Form {
  std::array<long long, 256> c{};
  long long k = 0;
};
static long long g_lo = 0, g_hi = 0;  // extremes of the nodes made since the last reset
static long long g_box_lo = 0, g_box_hi = 255;  // every variable ranges over [g_box_lo, g_box_hi]
inline void note(const Form& f) {
  long long lo = f.k, hi = f.k;
  for (int i = 0; i < 256; ++i) {
    if (f.c[i] > 0) {
      hi += g_box_hi * f.c[i];
      lo += g_box_lo * f.c[i];
    } else {
      hi += g_box_lo * f.c[i];
      lo += g_box_hi * f.c[i];
    }
  }
  g_lo = std::min(g_lo, lo);
  g_hi = std::max(g_hi, hi);
}
inline Form badd(const Form& a, const Form& b) {
  Form o;
  for (int i = 0; i < 256; ++i) o.c[i] = a.c[i] + b.c[i];
  o.k = a.k + b.k;
  note(o);
  return o;
}
inline Form bsub(const Form& a, const Form& b) {
  Form o;
  for (int i = 0; i < 256; ++i) o.c[i] = a.c[i] - b.c[i];
  o.k = a.k - b.k;
  note(o);
  return o;
}
inline Form scaled(const Form& a, long long s) {
  Form o;
  for (int i = 0; i < 256; ++i) o.c[i] = s * a.c[i];
  o.k = s * a.k;
  return o;
}
}  // namespace atdct16

#include "atdct16_butterfly.cuh"
#include "atdct16_zigzag.cuh"

using atdct16::Form;

static Form X[16][16], R[16][16], Y[16][16], D[16][16], U[16][16];

int main() {
  for (int m = 0; m < 16; ++m)
    for (int n = 0; n < 16; ++n) X[m][n].c[16 * m + n] = 1;
  // forward row pass, then the DC centring of the kernel's int16 column pass
  atdct16::g_lo = atdct16::g_hi = 0;
  for (int m = 0; m < 16; ++m) atdct16::fwd16(X[m], R[m]);
  std::printf("row %lld %lld\n", atdct16::g_lo, atdct16::g_hi);
  for (int m = 0; m < 16; ++m) R[m][0].k -= 2048;
  atdct16::g_lo = atdct16::g_hi = 0;
  for (int m = 0; m < 16; ++m) atdct16::note(R[m][0]);
  for (int k = 0; k < 16; ++k) {
    Form col[16], out[16];
    for (int m = 0; m < 16; ++m) col[m] = R[m][k];
    atdct16::fwd16(col, out);
    for (int u = 0; u < 16; ++u) Y[u][k] = out[u];
  }
  std::printf("col %lld %lld\n", atdct16::g_lo, atdct16::g_hi);
  Y[0][0].k += 16 * 2048;  // the centring taken back: Y = T X T^T exactly
  // W_u = 48 / (number of non-zeros in row u of T), from the butterfly's response
  int w[16];
  {
    long long e[16][16];
    for (int i = 0; i < 16; ++i) {
      long long x[16] = {}, y[16];
      x[i] = 1;
      atdct16::fwd16(x, y);
      for (int u = 0; u < 16; ++u) e[u][i] = y[u];
    }
    for (int u = 0; u < 16; ++u) {
      int nnz = 0;
      for (int i = 0; i < 16; ++i) nnz += e[u][i] != 0;
      w[u] = 48 / nnz;
    }
  }
  long long in_max = 0, node_max = 0;
  for (int r = 1; r <= 256; ++r) {
    atdct16::g_lo = atdct16::g_hi = 0;
    for (int u = 0; u < 16; ++u)
      for (int v = 0; v < 16; ++v) {
        D[u][v] = atdct16::zigzag_rank(16 * u + v) < r ? atdct16::scaled(Y[u][v], (long long)w[u] * w[v]) : Form{};
        atdct16::note(D[u][v]);
      }
    in_max = std::max({in_max, -atdct16::g_lo, atdct16::g_hi});
    for (int v = 0; v < 16; ++v) {
      Form col[16], out[16];
      for (int u = 0; u < 16; ++u) col[u] = D[u][v];
      atdct16::inv16(col, out);
      for (int m = 0; m < 16; ++m) U[m][v] = out[m];
    }
    for (int m = 0; m < 16; ++m) {
      Form z[16];
      atdct16::inv16(U[m], z);
    }
    node_max = std::max({node_max, -atdct16::g_lo, atdct16::g_hi});
  }
  std::printf("inv %lld %lld\n", in_max, node_max);
  // the FP32 forward of the standalone u8 path: inputs carried as 2^23 + 256 x,
  // the DC row output takes back 16 x 2^23, the column pass sees 256 x (row outputs)
  {
    static Form Xs[16][16], Rs[16][16];
    for (int m = 0; m < 16; ++m)
      for (int n = 0; n < 16; ++n) {
        Xs[m][n] = Form{};
        Xs[m][n].c[16 * m + n] = 256;
        Xs[m][n].k = 1LL << 23;
      }
    atdct16::g_lo = atdct16::g_hi = 0;
    for (int m = 0; m < 16; ++m) atdct16::fwd16(Xs[m], Rs[m]);
    long long row_lo = atdct16::g_lo, row_hi = atdct16::g_hi;
    bool offsets_cancel = true;
    for (int m = 0; m < 16; ++m) {
      Rs[m][0].k -= 16LL << 23;
      for (int k = 0; k < 16; ++k) offsets_cancel = offsets_cancel && Rs[m][k].k == 0;
    }
    atdct16::g_lo = atdct16::g_hi = 0;
    for (int k = 0; k < 16; ++k) {
      Form col[16], out[16];
      for (int m = 0; m < 16; ++m) col[m] = Rs[m][k];
      atdct16::fwd16(col, out);
    }
    std::printf("fwd_u8_f32 %lld %lld %lld %lld %d\n", row_lo, row_hi, atdct16::g_lo, atdct16::g_hi,
                offsets_cancel ? 1 : 0);
  }
  // the fused kernel's FP32-column variant: integer row outputs v (13-bit fields)
  // enter the column pass as the floats 2^23 + 2^20 + 256 v
  {
    atdct16::g_lo = atdct16::g_hi = 0;
    for (int k = 0; k < 16; ++k) {
      Form col[16], out[16];
      for (int m = 0; m < 16; ++m) {
        col[m] = atdct16::scaled(R[m][k], 256);
        col[m].k += (1LL << 23) + (1LL << 20) + 256 * 2048 * (k == 0);  // R[m][0] was centred
      }
      atdct16::fwd16(col, out);
    }
    std::printf("fwd_f32col %lld %lld\n", atdct16::g_lo, atdct16::g_hi);
  }
  // the standalone exact inverse on int32 coefficients, all kept: 32-bit route for
  // -2^18 <= Y < 2^18, split route on the halves Y_h in [-2^15, 2^15), Y_l in [0, 2^16)
  const long long boxes[3][2] = {{-(1LL << 18), (1LL << 18) - 1}, {-(1LL << 15), (1LL << 15) - 1}, {0, (1LL << 16) - 1}};
  for (int b = 0; b < 3; ++b) {
    atdct16::g_box_lo = boxes[b][0];
    atdct16::g_box_hi = boxes[b][1];
    atdct16::g_lo = atdct16::g_hi = 0;
    for (int u = 0; u < 16; ++u)
      for (int v = 0; v < 16; ++v) {
        D[u][v] = Form{};
        D[u][v].c[16 * u + v] = (long long)w[u] * w[v];
      }
    for (int v = 0; v < 16; ++v) {
      Form col[16], out[16];
      for (int u = 0; u < 16; ++u) col[u] = D[u][v];
      atdct16::inv16(col, out);
      for (int m = 0; m < 16; ++m) U[m][v] = out[m];
    }
    for (int m = 0; m < 16; ++m) {
      Form z[16];
      atdct16::inv16(U[m], z);
    }
    std::printf("int32_%d %lld %lld\n", b, atdct16::g_lo, atdct16::g_hi);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def bounds(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("bounds")
    src, exe = d / "bounds.cpp", d / "bounds"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_1606_05562_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return {ln.split()[0]: tuple(int(t) for t in ln.split()[1:]) for ln in out.splitlines()}


def test_forward_int16_fields_never_overflow(bounds):
    lo, hi = bounds["row"]
    assert -4080 <= lo and hi <= 4080  # 16 terms of magnitude <= 255
    lo, hi = bounds["col"]
    assert -32768 <= lo and hi <= 32767, (lo, hi)
    assert (lo, hi) == (-32768, 32640)  # the range the kernel's layout is designed around


def test_inverse_nodes_exact_in_fp32(bounds):
    d_max, node_max = bounds["inv"]
    assert d_max == 9 * 65280  # the weighted DC, W_0^2 = 9, of an all-255 block
    assert node_max < 2 ** 24, node_max
    assert node_max == 1941060


def test_weighted_dc_of_a_constant_block(bounds):
    """The largest weighted input is attained: an all-255 block has Y(0, 0) =
    256 x 255 (oracle) and weight W_0^2 = 9, i.e. 2304 x 255, the numerator
    of a reconstruction of 255 everywhere."""
    y = O.forward_int(np.full((16, 16), 255, dtype=np.uint8))
    assert int(np.asarray(y).reshape(16, 16)[0, 0]) == 65280
    assert bounds["inv"][0] == 9 * int(np.asarray(y).reshape(16, 16)[0, 0]) == 2304 * 255


def test_exact_inverse_int32_routes_never_overflow(bounds):
    """The standalone inverse of any int32 coefficients: tiles with every
    -2^18 <= Y < 2^18 run in 32-bit integers, the others transform the halves
    Y = 2^16 Y_h + Y_l in 32 bits; no node of either route leaves int32."""
    for key in ("int32_0", "int32_1", "int32_2"):
        lo, hi = bounds[key]
        assert -(2 ** 31) <= lo and hi < 2 ** 31, (key, lo, hi)
    # the exact extreme is 2304 x 2^18 (2304 = 48^2), half the analytic
    # (sum_u W_u)^2 2^18 = 68^2 2^18 bound
    assert max(-bounds["int32_0"][0], bounds["int32_0"][1]) == 2304 * 2 ** 18


def test_u8_rounding_is_exact_for_every_numerator():
    """The kernels' u8 rounding of X_hat = Z / 2304, restated step by step in
    IEEE single precision (numpy keeps subnormals): t = fl(Z fl(1/2304)),
    then fl(t 2^-149) lands on the subnormal grid, whose bit pattern read as
    int32 is the signed rounded value, saturated to 0..255 as cvt.pack.sat
    does.  Against round-half-to-even of the exact quotient for every
    integer |Z| <= 2^24 (every numerator a u8 block can produce lies within
    +-1941060; larger ones convert to float exactly up to 2^24 and saturate
    beyond)."""
    c = np.float32(1.0) / np.float32(2304.0)
    tiny = np.float32(2.0 ** -149)
    assert tiny.view(np.int32) == 1
    step = 1 << 22
    for lo in range(-(1 << 24), (1 << 24) + 1, step):
        z = np.arange(lo, min(lo + step, (1 << 24) + 1), dtype=np.int64)
        t = z.astype(np.float32) * c
        got = np.clip((t * tiny).view(np.int32), 0, 255)
        q, rem = np.divmod(z, 2304)
        want = q + (rem > 1152) + ((rem == 1152) & (q % 2 == 1))
        assert np.array_equal(got, np.clip(want, 0, 255)), int(z[np.argmax(got != np.clip(want, 0, 255))])


def test_standalone_u8_forward_exact_in_fp32(bounds):
    """The standalone forward carries u8 inputs as 2^23 + 256 x: every row
    node is a multiple of 256 below 2^28 (so exact in FP32), the offsets
    cancel in every row output but the DC, and every column node, 256 x an
    integer, stays below 2^24."""
    row_lo, row_hi, col_lo, col_hi, cancel = bounds["fwd_u8_f32"]
    assert -(2 ** 28) < row_lo and row_hi < 2 ** 28
    assert cancel == 1
    assert -(2 ** 24) < col_lo and col_hi < 2 ** 24
    assert col_hi == 256 * 65280


def test_fused_fp32_column_variant_exact(bounds):
    """The fused kernel's FP32-column variant feeds 2^23 + 2^20 + 256 v into an
    f32x2 column pass: every node is a multiple of 256 (integer forms times
    256 plus multiples of 2^20) below 2^28 in magnitude, hence exact."""
    lo, hi = bounds["fwd_f32col"]
    assert -(2 ** 28) < lo and hi < 2 ** 28, (lo, hi)

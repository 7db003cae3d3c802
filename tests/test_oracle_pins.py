"""Pins of the CPU oracle to what the paper and the mathematics fix.

None of these tests needs a GPU.  Each pin checks the oracle against
something other than itself: values printed in the paper (tests/golden/),
closed forms, invariants, brute force on tiny inputs, or a second
independent route to the same quantity.  ``test_pins_catch_planted_mistakes``
plants plausible mistakes in copies of the oracle's data and checks that the
pins fail on each.
"""

import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O


def _golden_lines(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]


def _printed_decimals(s):
    return len(s.split(".")[1]) if "." in s else 0


# ---------------------------------------------------------------- Sec. 2 ---
def test_t_is_multiplierless_and_tt_diagonal():
    assert set(np.unique(O.T)) <= {-1, 0, 1}
    g = O.t_t_transpose()
    assert np.all(g == np.diag(np.diag(g)))
    # each diagonal entry is the number of non-zeros of that row
    assert np.all(np.diag(g) == np.count_nonzero(O.T, axis=1))


def test_s_matches_printed(golden_dir):
    den = [int(v) for v in _golden_lines(golden_dir, "s_printed.txt")]
    assert len(den) == 16
    np.testing.assert_allclose(O.s_diag(), 1.0 / np.sqrt(den), rtol=0, atol=1e-15)
    assert np.all(O.w_diag() * np.array(den) == 48)


def test_c_hat_orthogonal():
    c = O.c_hat()
    np.testing.assert_allclose(c @ c.T, np.eye(16), atol=1e-14)


def _cycles_to_row_source(text):
    perm = list(range(16))
    for grp in text.replace(")", "").split("(")[1:]:
        elems = [int(t) for t in grp.split()]
        if len(elems) > 1 and elems[0] == elems[-1]:
            elems = elems[:-1]  # printed repetition of the cycle's first element
        for a, b in zip(elems, elems[1:] + elems[:1]):
            perm[a] = b
    return tuple(perm)


def test_factorisation_reproduces_t(golden_dir):
    text = _golden_lines(golden_dir, "p2_cycles.txt")[0]
    assert _cycles_to_row_source(text) == O.P2_ROW_SOURCE
    m1, p1, m2, m3, m4, p2 = O.factors()
    f = m4 @ m3 @ m2 @ p1 @ m1
    assert np.array_equal(p2 @ f, O.T)
    # rows of F are pairwise distinct, so no other row permutation gives T
    assert len({tuple(r) for r in f}) == 16
    # P1 and P2 are permutations
    for p in (p1, p2):
        assert np.array_equal(p @ p.T, np.eye(16, dtype=np.int64))


def test_table1_addition_count(golden_dir):
    mul, add, shift, total = [int(v) for v in _golden_lines(golden_dir, "table1_complexity.txt")[0].split()]
    fs = O.factors()
    assert sum(O.addition_count(m) for m in fs) == add == 60
    assert sum(O.multiplication_count(m) for m in fs) == mul == 0
    assert shift == 0 and total == add
    # the transposed factors (the inverse T^T) need the same count
    assert sum(O.addition_count(m.T) for m in fs) == 60
    # the direct product needs many more: sum over rows of (nnz - 1)
    assert O.addition_count(O.T) == 176


# ---------------------------------------------------------------- Table 2 ---
@pytest.mark.parametrize("name", ["DCT", "Proposed"])
def test_table2_measures(golden_dir, name):
    rows = {ln.split()[0]: ln.split()[1:] for ln in _golden_lines(golden_dir, "table2_measures.txt")}
    printed = rows[name]
    ct = O.dct_matrix() if name == "DCT" else O.c_hat()
    got = O.table2_row(ct)
    for key, text in zip(["d2", "eps", "mse", "cg", "eta"], printed):
        nd = _printed_decimals(text)
        assert round(got[key], nd) == pytest.approx(float(text), abs=10.0 ** -nd / 2 + 1e-12), key


# ------------------------------------------------------- integer forward ---
def _brute_forward(block):
    y = [[0] * 16 for _ in range(16)]
    for u in range(16):
        for v in range(16):
            s = 0
            for m in range(16):
                for n in range(16):
                    s += int(O.T[u, m]) * int(block[m][n]) * int(O.T[v, n])
            y[u][v] = s
    return np.array(y, dtype=np.int64)


def test_forward_brute_force_two_blocks():
    rng = np.random.default_rng(7)
    img = rng.integers(0, 256, size=(16, 32), dtype=np.int64)
    y = O.forward_int(img)
    for bx in range(2):
        assert np.array_equal(y[0, bx], _brute_forward(img[:, 16 * bx:16 * bx + 16].tolist()))


def test_forward_constant_block_is_dc_only():
    for c in (0, 1, 128, 255):
        y = O.forward_int(np.full((16, 16), c))
        expect = np.zeros((16, 16), dtype=np.int64)
        expect[0, 0] = 256 * c
        assert np.array_equal(y[0, 0], expect)


def test_forward_impulse_gives_outer_product():
    for m, n in [(0, 0), (3, 11), (15, 15), (7, 2)]:
        img = np.zeros((16, 16), dtype=np.int64)
        img[m, n] = 1
        assert np.array_equal(O.forward_int(img)[0, 0], np.outer(O.T[:, m], O.T[:, n]))


def test_forward_linearity_and_range():
    rng = np.random.default_rng(3)
    a = rng.integers(-300, 300, size=(32, 48))
    b = rng.integers(-300, 300, size=(32, 48))
    assert np.array_equal(O.forward_int(5 * a + b), 5 * O.forward_int(a) + O.forward_int(b))
    # u8 extremes: |Y| <= 256*255 for DC, <= 128*255 elsewhere
    for c in (0, 255):
        x = np.full((16, 16), c)
        x[::2, ::3] = 255 - c
        y = O.forward_int(x)[0, 0]
        assert abs(y[0, 0]) <= 65280 and np.all(np.abs(y.ravel()[1:]) <= 32640)


def test_one_d_unit_and_extreme_vectors_brute_force():
    # the 1-D transform applied to unit vectors returns T's columns, and the
    # extreme +-255 patterns hit the row bounds nnz_k * 255 exactly
    for j in range(16):
        e = np.zeros((16, 16), dtype=np.int64)
        e[0, j] = 1  # row 0 only -> Y[u, v] = T[u, 0] T[v, j]
        assert np.array_equal(O.forward_int(e)[0, 0][0], O.T[0, 0] * O.T[:, j])
    x = np.where(O.T > 0, 255, -255)  # row k of x aligned with row k of T
    for k in range(16):
        assert int(O.T[k] @ x[k]) == 255 * int(np.count_nonzero(O.T[k]))


# --------------------------------------------------------- exact inverse ---
def test_inverse_exact_all_coefficients():
    rng = np.random.default_rng(11)
    img = rng.integers(0, 256, size=(48, 32), dtype=np.int64).astype(np.uint8)
    y = O.forward_int(img)
    z = O.inverse_numerator(y)
    assert np.array_equal(z, 2304 * O.to_blocks(img.astype(np.int64)))
    assert np.array_equal(O.inverse_exact(y), img)
    res = O.compress_zonal_exact(img, 256)
    assert res["sse"] == 0.0 and math.isinf(res["psnr"])
    assert np.array_equal(res["recon_u8"], img)


def test_round_half_away_div_matches_fractions():
    vals = list(range(-5000, 5001, 7)) + [1152, -1152, 3456, -3456, 2304 * 3 + 1152]
    got = O.round_half_away_div(np.array(vals), 2304)
    for v, g in zip(vals, got):
        f = Fraction(v, 2304)
        q = math.floor(abs(f) + Fraction(1, 2))
        assert g == (q if f >= 0 else -q)


def test_round_half_even_div_matches_python_round():
    # Python's round() of a Fraction is exact round-half-to-even
    vals = list(range(-7000, 7001, 5)) + [1152 * k for k in range(-9, 10, 2)]
    got = O.round_half_even_div(np.array(vals), 2304)
    for v, g in zip(vals, got):
        assert g == round(Fraction(v, 2304))


def _zonal_cases():
    rng = np.random.default_rng(5)
    img_a = rng.integers(0, 256, size=(32, 32)).astype(np.uint8)
    from paper_1606_05562_gb300 import synth
    img_b = synth.ar1_image(64, 48, 0.95, 9)
    return [img_a, img_b]


@pytest.mark.parametrize("r", [1, 6, 16, 36, 64, 100, 150, 255, 256])
def test_exact_route_matches_fp64_definition(r):
    for img in _zonal_cases():
        ex = O.compress_zonal_exact(img, r)
        fp = O.compress_zonal_fp64(img, r)
        np.testing.assert_allclose(ex["numerator"] / 2304.0, O.to_blocks(fp["recon"]), atol=1e-9)
        assert ex["sse"] == pytest.approx(fp["sse"], rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("r", [1, 16, 100, 200])
def test_parseval_sse_equals_discarded_energy(r):
    s = O.s_diag()
    for img in _zonal_cases():
        ex = O.compress_zonal_exact(img, r)
        b = ex["coef"] * (s[:, None] * s[None, :])
        dropped = np.where(O.zonal_mask(r)[None, None], 0.0, b)
        assert ex["sse"] == pytest.approx(float(np.sum(dropped ** 2)), rel=1e-10)


def test_psnr_monotone_in_r():
    for img in _zonal_cases():
        p = [O.compress_zonal_exact(img, r)["psnr"] for r in range(1, 257, 5)]
        assert all(b >= a - 1e-12 for a, b in zip(p, p[1:]))


def test_r1_keeps_block_mean_for_both_transforms():
    for img in _zonal_cases():
        a = O.compress_zonal_fp64(img, 1, "approx")
        d = O.compress_zonal_fp64(img, 1, "dct")
        mean = O.to_blocks(img.astype(np.float64)).mean(axis=(2, 3), keepdims=True)
        np.testing.assert_allclose(O.to_blocks(a["recon"]), np.broadcast_to(mean, O.to_blocks(a["recon"]).shape), atol=1e-9)
        assert a["psnr"] == pytest.approx(d["psnr"], rel=1e-12)


def test_dct_matrix_orthonormal_and_exact_reconstruction():
    c = O.dct_matrix()
    np.testing.assert_allclose(c @ c.T, np.eye(16), atol=1e-14)
    img = _zonal_cases()[1]
    assert O.compress_zonal_fp64(img, 256, "dct")["sse"] < 1e-18 * img.size * 255 ** 2


# -------------------------------------------------------------- zig-zag ---
def _jpeg_walk(n):
    """Zig-zag built by walking: up-right / down-left with boundary bounces."""
    u = v = 0
    out = [(0, 0)]
    up = True  # moving towards row 0 (v increasing)
    while len(out) < n * n:
        if up:
            if v == n - 1:
                u += 1; up = False
            elif u == 0:
                v += 1; up = False
            else:
                u -= 1; v += 1
        else:
            if u == n - 1:
                v += 1; up = True
            elif v == 0:
                u += 1; up = True
            else:
                u += 1; v -= 1
        out.append((u, v))
    return out


def test_zigzag_matches_walk_and_invariants():
    for n in (4, 8, 16):
        assert O.zigzag_order(n) == _jpeg_walk(n)
    z = O.zigzag_order(16)
    assert z[:6] == [(0, 0), (0, 1), (1, 0), (2, 0), (1, 1), (0, 2)]
    assert sorted(z) == [(u, v) for u in range(16) for v in range(16)]
    for (a, b), (c, d) in zip(z, z[1:]):
        assert max(abs(a - c), abs(b - d)) == 1
    # triangular r keep whole anti-diagonals, whatever the orientation
    for r, s in [(1, 0), (6, 2), (36, 7)]:
        m = O.zonal_mask(r)
        assert all(m[u, v] == (u + v <= s) for u in range(16) for v in range(16))
    assert O.zonal_mask(256).all() and O.zonal_mask(150).sum() == 150


# ------------------------------------------ 1-D transforms, zig-zag layout ---
def test_forward_1d_is_the_separable_factor_of_forward_int():
    # the 2-D forward is the 1-D forward of every row, then of every column
    rng = np.random.default_rng(41)
    img = rng.integers(-32768, 32768, size=(32, 48))
    rows = O.forward_1d(O.to_blocks(img))                      # R[m, v]
    y = np.swapaxes(O.forward_1d(np.swapaxes(rows, -1, -2)), -1, -2)
    assert np.array_equal(y, O.forward_int(img))
    for j in range(16):  # unit vectors give the columns of T
        e = np.zeros(16, dtype=np.int64)
        e[j] = 1
        assert np.array_equal(O.forward_1d(e), O.T[:, j])


def test_inverse_1d_matches_fractions_with_printed_s(golden_dir):
    # x_n = sum_u T[u, n] S_u^2 y_u with S_u^2 = 1 / den_u as printed in Sec. 2,
    # rounded half to even (Python's round of a Fraction) and clamped
    den = [int(v) for v in _golden_lines(golden_dir, "s_printed.txt")]
    rng = np.random.default_rng(43)
    cases = [rng.integers(-70000, 70000, size=16), rng.integers(-2**31, 2**31, size=16),
             rng.integers(-3000, 3000, size=16)]
    for k in (8, 24, -8, -24, 40):  # DC alone: x = k / 16, ties at odd multiples of 8
        e = np.zeros(16, dtype=np.int64)
        e[0] = k
        cases.append(e)
    for y in cases:
        for dt in (np.uint8, np.int16):
            info = np.iinfo(dt)
            got = O.inverse_1d(y, dt)
            for n in range(16):
                f = sum(Fraction(int(O.T[u, n]) * int(y[u]), den[u]) for u in range(16))
                assert got[n] == min(max(round(f), info.min), info.max)


def test_inverse_1d_reconstructs_forward_1d():
    rng = np.random.default_rng(44)
    x8 = rng.integers(0, 256, size=(50, 16)).astype(np.uint8)
    x16 = rng.integers(-32768, 32768, size=(50, 16)).astype(np.int16)
    assert np.array_equal(O.inverse_1d(O.forward_1d(x8), np.uint8), x8)
    assert np.array_equal(O.inverse_1d(O.forward_1d(x16), np.int16), x16)


def test_zigzag_layout_round_trip_and_scan():
    assert np.array_equal(O.to_zigzag(O.zigzag_rank()), np.arange(256))
    rng = np.random.default_rng(45)
    c = rng.integers(-1000, 1000, size=(3, 2, 16, 16))
    assert np.array_equal(O.from_zigzag(O.to_zigzag(c)), c)
    for r in (1, 6, 100, 256):
        z = O.to_zigzag(O.zonal_mask(r).astype(np.int64))
        assert z[:r].all() and not z[r:].any()
    # first entries follow the walk of Sec. 4: DC, then (0,1), (1,0), (2,0)
    b = np.arange(256).reshape(16, 16)
    assert list(O.to_zigzag(b)[:4]) == [0, 1, 16, 32]


# ---------------------------------------------------------- quantiser ---
def test_quantiser_fp32_decision_close_to_fp64():
    from paper_1606_05562_gb300 import synth
    x = synth.laplacian_residual(64, 64, 21)
    y = O.forward_int(x)
    for qp in (22, 27, 32, 37):
        l64 = O.quant_levels(y, qp, "fp64")
        l32 = O.quant_levels(y, qp, "fp32")
        diff = l64 != l32
        assert np.all(np.abs(l64 - l32) <= 1)
        assert diff.mean() < 1e-3


def test_quantiser_closed_forms():
    # QP = 0 -> Qstep = 1: level = round_half_away(Y / sqrt(nnz_u nnz_v)),
    # decided in exact arithmetic
    y = np.arange(-512, 512).reshape(4, 16, 16)[None]
    nnz = _nnz_printed()
    got = O.quant_levels(y, 0, "fp64")
    for b in range(4):
        for u in range(16):
            for v in range(16):
                assert got[0, b, u, v] == _level_exact(int(y[0, b, u, v]), nnz[u], nnz[v], 0)
    # very fine step reconstructs the residual to within the step
    x = np.random.default_rng(2).integers(-255, 256, size=(32, 32)).astype(np.int16)
    res = O.compress_quant(x, -60)
    assert np.max(np.abs(res["recon"] - x)) < 2.0 ** -9
    assert np.array_equal(res["recon_i16"], x)
    # huge step zeroes everything
    res = O.compress_quant(x, 120)
    assert np.all(res["levels"] == 0) and np.all(res["recon"] == 0)


def _nnz_printed():
    """Non-zeros per row of the printed T (Sec. 2): ``s_u^2 = 1 / nnz_u``."""
    return [int(np.count_nonzero(row)) for row in O.T]


def _level_exact(y: int, nu: int, nv: int, qp: int) -> int:
    """``sign(B) floor(|B| / Qstep + 1/2)`` for ``B = Y / sqrt(nu nv)`` and
    ``Qstep = 2^(QP/6)``, decided without rounding error: when ``3 | QP`` the
    squared quotient ``Y^2 / (nu nv 2^(QP/3))`` is a fraction and the level is
    the largest L with ``(L - 1/2)^2 <= q^2``; otherwise the quotient is
    irrational (no ties) and 60-digit decimal arithmetic decides it."""
    import decimal
    from fractions import Fraction

    if y == 0:
        return 0
    a = abs(y)
    if qp % 3 == 0:
        q2 = Fraction(a * a, nu * nv) / (Fraction(2) ** (qp // 3))
        lo = 0  # (lo - 1/2)^2 <= q2 holds for lo = 0
        hi = int(math.isqrt(int(q2)) + 2)
        while lo < hi:  # largest L with L - 1/2 <= q
            mid = (lo + hi + 1) // 2
            if (Fraction(2 * mid - 1, 2)) ** 2 <= q2:
                lo = mid
            else:
                hi = mid - 1
        lev = lo
    else:
        with decimal.localcontext() as ctx:
            ctx.prec = 60
            q = decimal.Decimal(a) / ((decimal.Decimal(nu * nv)).sqrt() * decimal.Decimal(2) ** (decimal.Decimal(qp) / 6))
            lev = int((q + decimal.Decimal("0.5")).to_integral_value(rounding=decimal.ROUND_FLOOR))
    return lev if y > 0 else -lev


# Exact half-integer quotients |B| / Qstep (rounded half away from zero):
# (u, v, Y, QP, level).  nnz = 16 at u in {0, 1, 5, 8}, 12 at {2, 6, 7, 9, 10,
# 13, 14, 15}, 8 at {3, 4, 11, 12}.
_QUANT_TIES = [
    (0, 0, 8, 0, 1), (0, 0, -8, 0, -1), (1, 5, 24, 0, 2), (8, 0, 40, 0, 3), (5, 8, -40, 0, -3),
    (3, 4, 4, 0, 1), (11, 12, 20, 0, 3), (12, 3, -20, 0, -3),           # Y / 8
    (2, 6, 12, 6, 1), (9, 13, 60, 6, 3), (14, 15, -36, 6, -2),          # Y / 24
    (0, 3, 40, 3, 3), (4, 8, -24, 3, -2),                               # Y / 16 (nnz 16 x 8, QP 3)
    (1, 1, 640, 24, 3), (6, 7, 336, 18, 4), (13, 9, -36, 6, -2),          # Y / 256, Y / 96, Y / 24
]


def test_qstep_law():
    # Sec. 5.3 sweeps the HEVC quantisation point; its step is 1 at QP 0 and
    # doubles every six points, i.e. Qstep^6 = 2^QP
    assert O.qstep(0) == 1.0
    for k in range(-4, 11):
        assert O.qstep(6 * k) == 2.0 ** k
    for qp in range(-30, 64):
        assert O.qstep(qp) > 0
        assert O.qstep(qp) ** 6 == pytest.approx(2.0 ** qp, rel=1e-13)
        assert O.qstep(qp + 6) == pytest.approx(2 * O.qstep(qp), rel=1e-15)
    assert [round(O.qstep(q), 2) for q in (22, 27, 32, 37)] == [12.7, 22.63, 40.32, 71.84]


def test_quant_levels_ties_round_half_away_from_zero():
    nnz = _nnz_printed()
    for u, v, y, qp, want in _QUANT_TIES:
        assert _level_exact(y, nnz[u], nnz[v], qp) == want, (u, v, y, qp)
        c = np.zeros((16, 16), dtype=np.int64)
        c[u, v] = y
        got = O.quant_levels(c[None, None], qp, "fp64")[0, 0]
        assert got[u, v] == want, (u, v, y, qp, got[u, v])
        assert np.count_nonzero(got) == (1 if want else 0)


@pytest.mark.parametrize("qp", [0, 1, 3, 6, 9, 13, 22, 27, 32, 37, 51])
def test_quant_levels_match_exact_arithmetic(qp):
    nnz = _nnz_printed()
    rng = np.random.default_rng(100 + qp)
    y = rng.integers(-65280, 65281, size=(1, 3, 16, 16))
    y[0, 1] = rng.integers(-300, 301, size=(16, 16))
    q = O.qstep(qp)
    # exact ties of this QP at the classes where the quotient is rational
    for u in range(16):
        for v in range(16):
            if nnz[u] == nnz[v] and qp % 6 == 0:
                y[0, 2, u, v] = int(nnz[u] * q) * (2 * ((u + v) % 5) + 1) // 2 * (1 if (u ^ v) & 1 else -1)
    got = O.quant_levels(y, qp, "fp64")
    for b in range(3):
        for u in range(16):
            for v in range(16):
                assert got[0, b, u, v] == _level_exact(int(y[0, b, u, v]), nnz[u], nnz[v], qp), (b, u, v)


# ------------------------------------------------------------------ PSNR ---
def test_psnr_closed_forms():
    a = np.zeros((16, 16), dtype=np.uint8)
    b = np.full((16, 16), 255, dtype=np.uint8)
    assert O.psnr_images(a, b) == pytest.approx(0.0, abs=1e-12)
    c = a.copy(); c[0, 0] = 1
    assert O.psnr_images(a, c) == pytest.approx(10 * math.log10(255 ** 2 * 256), rel=1e-15)
    assert math.isinf(O.psnr_images(a, a))


# ------------------------------------------------------ planted mistakes ---
def _pins_pass(t, w, p2_source, zig):
    """The pins above, as one predicate over (possibly mutated) oracle data."""
    g = t @ t.T
    if not np.all(g == np.diag(np.diag(g))):
        return False
    if np.any(np.diag(g) == 0) or np.any(48 % np.diag(g) != 0):
        return False
    if not np.array_equal(48 // np.diag(g), w):
        return False
    s = 1.0 / np.sqrt(np.diag(g))
    ct = s[:, None] * t
    got = O.table2_row(ct)
    if abs(got["d2"] - 0.3405) > 5e-5 or abs(got["cg"] - 8.295) > 5e-4:
        return False
    m1, p1, m2, m3, m4, _ = O.factors()
    f = m4 @ m3 @ m2 @ p1 @ m1
    if not np.array_equal(f[list(p2_source)], t):
        return False
    if zig != _jpeg_walk(16):
        return False
    img = np.arange(256).reshape(16, 16) % 251
    y = np.einsum("um,mn,vn->uv", t, img, t)
    z = t.T @ (y * w[:, None] * w[None, :]) @ t
    return np.array_equal(z, 2304 * img)


def test_pins_catch_planted_mistakes():
    t, w = O.T.copy(), O.w_diag().copy()
    p2 = list(O.P2_ROW_SOURCE)
    zig = O.zigzag_order(16)
    assert _pins_pass(t, w, p2, zig)
    mutants = []
    t1 = t.copy(); t1[5, 3] *= -1; mutants.append((t1, w, p2, zig))          # sign flip
    mutants.append((t.T.copy(), w, p2, zig))                                  # transposed T
    t3 = t.copy(); t3[[2, 6]] = t3[[6, 2]]; mutants.append((t3, w, p2, zig))  # swapped rows
    w4 = w.copy(); w4[3] = 4; mutants.append((t, w4, p2, zig))                # wrong weight
    p5 = p2.copy(); p5[1], p5[8] = p5[8], p5[1]; mutants.append((t, w, p5, zig))  # P2 misread
    z6 = zig.copy(); z6[1], z6[2] = z6[2], z6[1]; mutants.append((t, w, p2, z6))  # zig-zag orientation
    t7 = t.copy(); t7[9, 4] = 1; mutants.append((t7, w, p2, zig))            # dropped zero
    for i, m in enumerate(mutants):
        assert not _pins_pass(*m), f"mutant {i} passed the pins"


def _quant_pins_pass(qstep_fn, levels_fn):
    """The quantiser pins above, as one predicate over a (possibly mutated)
    step law and level function."""
    if qstep_fn(0) != 1.0:
        return False
    if any(abs(qstep_fn(q) ** 6 / 2.0 ** q - 1) > 1e-12 for q in range(-12, 52)):
        return False
    nnz = _nnz_printed()
    for u, v, y, qp, want in _QUANT_TIES:
        c = np.zeros((16, 16), dtype=np.int64)
        c[u, v] = y
        if levels_fn(c[None, None], qp)[0, 0, u, v] != want:
            return False
    y = np.random.default_rng(7).integers(-2000, 2001, size=(1, 1, 16, 16))
    got = levels_fn(y, 27)
    return all(got[0, 0, u, v] == _level_exact(int(y[0, 0, u, v]), nnz[u], nnz[v], 27)
               for u in range(16) for v in range(16))


def test_quant_pins_catch_planted_mistakes():
    from oracle.atdct16_oracle import _quant_quotient_fp64 as _quotient

    assert _quant_pins_pass(O.qstep, lambda y, qp: O.quant_levels(y, qp, "fp64"))

    def with_rounding(rnd):
        def levels(y, qp):
            q = _quotient(y, qp)
            return (np.sign(y) * rnd(q)).astype(np.int64)
        return levels

    def with_step(step):
        def levels(y, qp):
            s = O.s_diag()
            b = y * (s[:, None] * s[None, :]) / step(qp)
            return (np.sign(b) * np.floor(np.abs(b) + 0.5)).astype(np.int64)
        return levels

    def with_scale(scale):
        def levels(y, qp):
            b = y * scale(O.s_diag()) / O.qstep(qp)
            return (np.sign(b) * np.floor(np.abs(b) + 0.5)).astype(np.int64)
        return levels

    exact = lambda y, qp: O.quant_levels(y, qp, "fp64")
    mutants = [
        (lambda qp: 2.0 ** (qp / 5.0), with_step(lambda qp: 2.0 ** (qp / 5.0))),                  # wrong slope
        (lambda qp: 2.0 ** ((qp - 4) / 6.0), with_step(lambda qp: 2.0 ** ((qp - 4) / 6.0))),      # HEVC offset
        (O.qstep, with_rounding(np.rint)),                                                       # half to even
        (O.qstep, with_rounding(np.floor)),                                                      # truncation
        (O.qstep, with_rounding(lambda q: np.ceil(q - 0.5))),                                    # half toward zero
        (O.qstep, lambda y, qp: exact(np.abs(y), qp)),                                           # sign dropped
        (O.qstep, with_scale(lambda s: s[:, None] * s[:, None])),                               # s_u^2 for s_u s_v
        (O.qstep, with_scale(lambda s: np.ones((16, 16)) / 16.0)),                               # S left out
    ]
    for i, (st, lv) in enumerate(mutants):
        assert not _quant_pins_pass(st, lv), f"quantiser mutant {i} passed the pins"


# --------------------------------------------------------------------------
# SSIM (Sec. 4, Wang et al. 2004) and APE.
# --------------------------------------------------------------------------
def _ssim_by_filters(a, b, sigma=O.SSIM_SIGMA, win=O.SSIM_WIN, c1=O.SSIM_C1, c2=O.SSIM_C2):
    """The same measure through a library route: separable Gaussian filtering
    (scipy.ndimage, radius 5) and the moment form E[xy] - E[x] E[y], cropped
    to the positions whose window lies inside the image."""
    from scipy import ndimage

    r = (win - 1) // 2
    f = lambda x: ndimage.gaussian_filter(x, sigma, truncate=r / sigma, mode="constant")[r:-r, r:-r]
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    mu_a, mu_b = f(a), f(b)
    s_aa = f(a * a) - mu_a * mu_a
    s_bb = f(b * b) - mu_b * mu_b
    s_ab = f(a * b) - mu_a * mu_b
    m = ((2 * mu_a * mu_b + c1) * (2 * s_ab + c2)) / ((mu_a ** 2 + mu_b ** 2 + c1) * (s_aa + s_bb + c2))
    return float(m.mean()), m.shape


def test_ssim_matches_filter_route():
    rng = np.random.default_rng(7)
    for h, w in ((16, 16), (24, 40), (37, 29)):
        a = rng.integers(0, 256, (h, w)).astype(np.uint8)
        b = np.clip(a.astype(int) + rng.integers(-30, 31, (h, w)), 0, 255).astype(np.uint8)
        ref, shape = _ssim_by_filters(a, b)
        assert O.ssim_map(a, b).shape == shape == (h - 10, w - 10)
        assert O.mssim(a, b) == pytest.approx(ref, rel=0, abs=1e-12)


def test_ssim_closed_forms():
    rng = np.random.default_rng(8)
    a = rng.integers(0, 256, (20, 23)).astype(np.uint8)
    assert O.mssim(a, a) == pytest.approx(1.0, abs=1e-15)
    b = np.clip(a.astype(int) + rng.integers(-9, 10, a.shape), 0, 255).astype(np.uint8)
    assert O.mssim(a, b) == pytest.approx(O.mssim(b, a), abs=1e-15)  # symmetric
    assert O.mssim(a, b) < 1.0
    # constant images: variances and covariance vanish, only the luminance term remains
    for c_a, c_b in ((0, 0), (10, 200), (128, 129), (255, 0)):
        x = np.full((16, 16), c_a, np.uint8)
        y = np.full((16, 16), c_b, np.uint8)
        want = (2.0 * c_a * c_b + O.SSIM_C1) / (c_a * c_a + c_b * c_b + O.SSIM_C1)
        assert O.mssim(x, y) == pytest.approx(want, rel=1e-13)
    # the window is the sampled Gaussian exp(-d^2 / 4.5), normalised
    w = O.ssim_window()
    assert w.shape == (11, 11) and w.sum() == pytest.approx(1.0, abs=1e-15)
    assert w[5, 5] / w[5, 6] == pytest.approx(math.exp(1.0 / 4.5), rel=1e-14)
    assert w[0, 0] / w[5, 5] == pytest.approx(math.exp(-50.0 / 4.5), rel=1e-12)


def test_ssim_pin_catches_planted_mistakes():
    rng = np.random.default_rng(9)
    a = rng.integers(0, 256, (30, 30)).astype(np.uint8)
    b = np.clip(a.astype(int) + rng.integers(-40, 41, a.shape), 0, 255).astype(np.uint8)
    ref = O.mssim(a, b)
    for kw in ({"sigma": 1.0}, {"c1": (0.03 * 255) ** 2}, {"c2": (0.01 * 255) ** 2}):
        assert abs(_ssim_by_filters(a, b, **kw)[0] - ref) > 1e-9, kw  # far outside the pin tolerance


def test_ape_closed_form():
    assert O.ape(110.0, 100.0) == pytest.approx(10.0)
    assert O.ape(90.0, 100.0) == pytest.approx(10.0)
    assert O.ape(0.5, 0.5) == 0.0

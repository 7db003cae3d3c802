"""Plain CPU oracle for the orthogonal 16-point approximate DCT of arXiv 1606.05562.

TEST INFRASTRUCTURE ONLY: used by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline legs of ``bench.py``; never by the product path.

Everything here follows the paper's definitions directly:

* ``T`` (Sec. 2, the printed 16x16 matrix), ``S = diag(T T^T)^(-1/2)`` and
  ``C_hat = S T`` (Sec. 2).
* The 2-D transform ``B = C_hat A C_hat^T`` of every disjoint 16x16 block, the
  zonal zig-zag retention of the first ``r`` coefficients and the inverse
  ``A' = C_hat^T B' C_hat`` (Sec. 4, image-compression procedure).
* ``S`` absorbed into a uniform scalar quantiser (Sec. 2, last paragraph;
  Sec. 5.3 sweeps the HEVC quantisation point).
* PSNR (Sec. 4), SSIM (Sec. 4, the Wang et al. 2004 measure the paper cites) and the
  APE of Sec. 4, and the similarity / coding measures of Sec. 3 (Table 2).
* The 1-D transform ``y = T x`` and its exact inverse ``rne(T^T (W y) / 48)``
  (Sec. 2), and the zig-zag block layout (entry k of a block = scan position k,
  Sec. 4) of coefficients and quantisation levels.

The fast factorisation ``T = P2 M4 M3 M2 P1 M1`` (Sec. 2, Eq. of the
factorisation) is recorded here only so that tests can check that the printed
factors multiply to the printed ``T`` and that they need 60 additions
(Table 1).  The oracle's own transforms never use it: they are direct matrix
products, so an error in a butterfly cannot hide in both sides.

Exactness.  ``T`` has entries in {0, +-1}; ``S^2 = W / 48`` with the integer
diagonal ``W = 48 / diag(T T^T)``.  Hence for any integer image block ``X`` and
any zonal mask, the reconstruction is the rational number
``Z / 2304`` with the integer ``Z = T^T (mask * (W Y W)) T`` and
``Y = T X T^T``.  The oracle computes that integer exactly (int64) and rounds
it exactly.  FP64 is used for the orthonormal-domain definition (a second,
independent route), the quantiser, PSNR and the Table 2 measures.

Readings of points the paper leaves open:

* Block orientation: ``A`` is indexed [row m][column n];
  ``Y[u, v] = sum_m sum_n T[u, m] A[m, n] T[v, n]`` (u = vertical frequency).
* Zig-zag for 16x16 (Sec. 4 adapts the 8x8 scan without spelling it out): the JPEG
  convention extended to 16x16.  Anti-diagonal s = u + v; on even s the scan
  runs with u decreasing, on odd s with v decreasing.
* PSNR is computed on the unrounded, unclipped reconstruction; the stored
  pixel is ``clamp(round_half_to_even(x_hat))``, decided exactly from the
  integer numerator ``Z`` (ties at ``Z = 2304 k + 1152``).
* Quantiser: ``level = sign(B) * floor(|B| / Qstep + 1/2)``,
  ``Qstep = 2^(QP/6)``, ``B = s_u s_v Y``; dequantised ``B' = level * Qstep``.
"""

from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

N = 16

# --------------------------------------------------------------------------
# Sec. 2: the low-complexity matrix T, typed from the printed matrix.
# --------------------------------------------------------------------------
T = np.array(
    [
        [1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1],
        [1, 1, 1, 1, 1, 1, 1, 1, -1, -1, -1, -1, -1, -1, -1, -1],
        [1, 1, 1, 0, 0, -1, -1, -1, -1, -1, -1, 0, 0, 1, 1, 1],
        [1, 1, 0, 0, 0, 0, -1, -1, 1, 1, 0, 0, 0, 0, -1, -1],
        [1, 0, 0, -1, -1, 0, 0, 1, 1, 0, 0, -1, -1, 0, 0, 1],
        [1, 1, -1, -1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1],
        [1, 0, -1, -1, 1, 1, 0, -1, -1, 0, 1, 1, -1, -1, 0, 1],
        [0, 0, -1, 1, 1, -1, -1, 1, -1, 1, 1, -1, -1, 1, 0, 0],
        [1, -1, -1, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, -1, -1, 1],
        [1, -1, -1, 1, 0, 0, 1, -1, 1, -1, 0, 0, -1, 1, 1, -1],
        [1, -1, 0, 1, -1, 0, 1, -1, -1, 1, 0, -1, 1, 0, -1, 1],
        [0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 0, 0],
        [0, -1, 1, 0, 0, 1, -1, 0, 0, -1, 1, 0, 0, 1, -1, 0],
        [1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1],
        [0, -1, 1, -1, 1, -1, 1, 0, 0, 1, -1, 1, -1, 1, -1, 0],
        [1, -1, 0, 0, -1, 1, -1, 1, -1, 1, -1, 1, 0, 0, 1, -1],
    ],
    dtype=np.int64,
)


def t_t_transpose() -> np.ndarray:
    """``T T^T`` (Sec. 2: the paper states it is diagonal)."""
    return T @ T.T


def s_diag() -> np.ndarray:
    """Diagonal of ``S = diag(T T^T)^(-1/2)`` in FP64 (Sec. 2, orthogonalisation)."""
    return 1.0 / np.sqrt(np.diag(t_t_transpose()).astype(np.float64))


def w_diag() -> np.ndarray:
    """Integer diagonal ``W = 48 S^2 = 48 / diag(T T^T)`` (exact; Sec. 2)."""
    d = np.diag(t_t_transpose())
    assert np.all(48 % d == 0)
    return (48 // d).astype(np.int64)


def c_hat() -> np.ndarray:
    """Orthogonal approximation ``C_hat = S T`` in FP64 (Sec. 2)."""
    return s_diag()[:, None] * T.astype(np.float64)


def dct_matrix(n: int = N) -> np.ndarray:
    """Exact orthonormal DCT-II matrix ``C[k, j] = a_k cos(pi (2j+1) k / (2n))``
    (Sec. 3.2, the exact DCT the approximation is compared with)."""
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    c = np.cos(np.pi * (2 * j + 1) * k / (2 * n))
    a = np.full((n, 1), math.sqrt(2.0 / n))
    a[0, 0] = math.sqrt(1.0 / n)
    return a * c


# --------------------------------------------------------------------------
# Sec. 2: sparse factorisation T = P2 M4 M3 M2 P1 M1 (checked by tests only).
# --------------------------------------------------------------------------
def _identity(n):
    return np.eye(n, dtype=np.int64)


def _counter_identity(n):
    return np.eye(n, dtype=np.int64)[::-1]


def factor_m1() -> np.ndarray:
    """``M1 = [[I8, J8], [J8, -I8]]`` (J = counter-identity)."""
    i8, j8 = _identity(8), _counter_identity(8)
    return np.block([[i8, j8], [j8, -i8]])


def factor_p1() -> np.ndarray:
    """``P1 = diag(I9, 7x7 permutation)`` as printed."""
    sub = np.array(
        [
            [0, 0, 1, 0, 0, 0, 0],
            [0, 0, 0, 1, 0, 0, 0],
            [0, 0, 0, 0, 0, 0, 1],
            [0, 0, 0, 0, 0, 1, 0],
            [0, 0, 0, 0, 1, 0, 0],
            [0, 1, 0, 0, 0, 0, 0],
            [1, 0, 0, 0, 0, 0, 0],
        ],
        dtype=np.int64,
    )
    p = _identity(16)
    p[9:, 9:] = sub
    return p


def factor_m2() -> np.ndarray:
    """``M2 = diag(B8, B8)`` with ``B8 = [[I4, J4], [J4, -I4]]``."""
    i4, j4 = _identity(4), _counter_identity(4)
    b8 = np.block([[i4, j4], [j4, -i4]])
    m = np.zeros((16, 16), dtype=np.int64)
    m[:8, :8] = b8
    m[8:, 8:] = b8
    return m


def factor_m3() -> np.ndarray:
    """``M3`` = four printed 4x4 blocks on the diagonal."""
    blocks = [
        [[1, 0, 0, 1], [0, 1, 1, 0], [0, -1, 1, 0], [1, 0, 0, -1]],
        [[0, 1, 1, 1], [-1, -1, 0, 1], [-1, 1, -1, 0], [1, 0, -1, 1]],
        [[1, 0, 0, 1], [0, 1, 1, 0], [0, -1, 1, 0], [-1, 0, 0, 1]],
        [[0, 1, 1, 1], [1, 1, 0, -1], [1, -1, 1, 0], [1, 0, -1, 1]],
    ]
    m = np.zeros((16, 16), dtype=np.int64)
    for i, b in enumerate(blocks):
        m[4 * i : 4 * i + 4, 4 * i : 4 * i + 4] = np.array(b, dtype=np.int64)
    return m


def factor_m4() -> np.ndarray:
    """``M4 = diag(H2, I6, H2, I6)`` with ``H2 = [[1, 1], [1, -1]]``."""
    m = _identity(16)
    h = np.array([[1, 1], [1, -1]], dtype=np.int64)
    m[0:2, 0:2] = h
    m[8:10, 8:10] = h
    return m


# The printed cycle notation of P2 is garbled (each cycle repeats its first
# element).  Reading: the cycles (1 8)(2 4 3 11 10 7 12)(5 9 13 14 6), acting so
# that row i of T is row p(i) of M4 M3 M2 P1 M1.
P2_ROW_SOURCE = (0, 8, 4, 11, 3, 9, 5, 12, 1, 13, 7, 10, 2, 14, 6, 15)


def factor_p2() -> np.ndarray:
    p = np.zeros((16, 16), dtype=np.int64)
    for i, src in enumerate(P2_ROW_SOURCE):
        p[i, src] = 1
    return p


def factors() -> list:
    """The printed factors in application order (M1 first)."""
    return [factor_m1(), factor_p1(), factor_m2(), factor_m3(), factor_m4(), factor_p2()]


def addition_count(m: np.ndarray) -> int:
    """Additions needed by ``y = m x`` for a {0, +-1} matrix: (non-zeros - 1) per
    non-empty row (the counting behind Table 1)."""
    nnz = np.count_nonzero(m, axis=1)
    return int(np.sum(np.maximum(nnz - 1, 0)))


def multiplication_count(m: np.ndarray) -> int:
    """Entries that are neither 0 nor +-1 would need a multiplier (Table 1)."""
    return int(np.count_nonzero((m != 0) & (np.abs(m) != 1)))


# --------------------------------------------------------------------------
# Sec. 4: zig-zag order and zonal mask.
# --------------------------------------------------------------------------
def zigzag_order(n: int = N) -> list:
    """(u, v) pairs in zig-zag order, JPEG convention extended to n x n."""
    order = []
    for s in range(2 * n - 1):
        lo, hi = max(0, s - (n - 1)), min(s, n - 1)
        if s % 2 == 0:
            for u in range(hi, lo - 1, -1):
                order.append((u, s - u))
        else:
            for v in range(hi, lo - 1, -1):
                order.append((s - v, v))
    return order


def zigzag_rank(n: int = N) -> np.ndarray:
    rank = np.zeros((n, n), dtype=np.int64)
    for i, (u, v) in enumerate(zigzag_order(n)):
        rank[u, v] = i
    return rank


def zonal_mask(r: int) -> np.ndarray:
    """Keep the first ``r`` zig-zag coefficients (Sec. 4); 1 <= r <= 256."""
    if not (0 <= r <= N * N):
        raise ValueError("r out of range")
    return zigzag_rank() < r


# --------------------------------------------------------------------------
# Block helpers (Sec. 4: disjoint 16x16 blocks, reassembled afterwards).
# --------------------------------------------------------------------------
def to_blocks(img: np.ndarray) -> np.ndarray:
    """(H, W) -> (H/16, W/16, 16, 16), block [by, bx] holds rows 16by.., cols 16bx.."""
    h, w = img.shape
    if h % N or w % N:
        raise ValueError("image sides must be multiples of 16")
    return img.reshape(h // N, N, w // N, N).transpose(0, 2, 1, 3)


def from_blocks(blk: np.ndarray) -> np.ndarray:
    by, bx = blk.shape[:2]
    return blk.transpose(0, 2, 1, 3).reshape(by * N, bx * N)


# --------------------------------------------------------------------------
# Integer forward transform and exact inverse.
# --------------------------------------------------------------------------
def forward_int(img: np.ndarray) -> np.ndarray:
    """``Y = T X T^T`` for every block, exact int64 (Sec. 2 + Sec. 4 with S
    left out, since S is absorbed into quantisation)."""
    xb = to_blocks(np.asarray(img).astype(np.int64))
    return np.einsum("um,yxmn,vn->yxuv", T, xb, T)


def inverse_numerator(coef: np.ndarray) -> np.ndarray:
    """Exact integer ``Z = T^T (W Y' W) T`` per block, so that the inverse of
    Sec. 4, ``C_hat^T (S Y' S) C_hat``, equals ``Z / 2304`` (``S^2 = W/48``)."""
    w = w_diag()
    d = coef.astype(np.int64) * w[:, None] * w[None, :]
    return np.einsum("um,yxuv,vn->yxmn", T, d, T)


def round_half_away_div(num: np.ndarray, den: int) -> np.ndarray:
    """Exact ``round_half_away_from_zero(num / den)`` for integer arrays."""
    num = np.asarray(num, dtype=np.int64)
    q = (np.abs(num) * 2 + den) // (2 * den)
    return np.sign(num) * q


def round_half_even_div(num: np.ndarray, den: int) -> np.ndarray:
    """Exact ``round_half_to_even(num / den)`` for integer arrays (den even)."""
    num = np.asarray(num, dtype=np.int64)
    shifted = num + den // 2
    q = np.floor_divide(shifted, den)
    tie = (shifted - q * den) == 0
    return np.where(tie & (q % 2 == 1), q - 1, q)


def to_zigzag(coef: np.ndarray) -> np.ndarray:
    """Blocks ``(..., 16, 16)`` -> ``(..., 256)``: entry k of a block is the
    coefficient at zig-zag scan position k (Sec. 4 scan), the order in which
    an entropy coder reads a block."""
    order = zigzag_order()
    c = np.asarray(coef)
    return np.stack([c[..., u, v] for (u, v) in order], axis=-1)


def from_zigzag(z: np.ndarray) -> np.ndarray:
    """Inverse of ``to_zigzag``: ``(..., 256)`` -> ``(..., 16, 16)``."""
    z = np.asarray(z)
    out = np.zeros(z.shape[:-1] + (N, N), dtype=z.dtype)
    for k, (u, v) in enumerate(zigzag_order()):
        out[..., u, v] = z[..., k]
    return out


def forward_1d(x: np.ndarray) -> np.ndarray:
    """``y = T x`` (Sec. 2, S left out) for every 16-sample vector along the
    last axis, exact int64."""
    return np.einsum("un,...n->...u", T, np.asarray(x).astype(np.int64))


def inverse_1d(coef: np.ndarray, out_dtype=np.uint8) -> np.ndarray:
    """Exact 1-D inverse of integer coefficients along the last axis:
    ``C_hat^T (S y) = T^T S^2 y = T^T (W y) / 48``, rounded half to even and
    clamped to the output type."""
    d = np.asarray(coef).astype(np.int64) * w_diag()
    z = np.einsum("un,...u->...n", T, d)
    x = round_half_even_div(z, 48)
    info = np.iinfo(out_dtype)
    return np.clip(x, info.min, info.max).astype(out_dtype)


def inverse_exact(coef: np.ndarray, out_dtype=np.uint8) -> np.ndarray:
    """Reconstruct an image from integer coefficients (no coefficient dropped
    unless ``coef`` already has zeros): exact round-half-to-even of
    ``Z / 2304``, then clamping to the output type."""
    z = inverse_numerator(coef)
    x = round_half_even_div(z, 2304)
    info = np.iinfo(out_dtype)
    return from_blocks(np.clip(x, info.min, info.max).astype(out_dtype))


def psnr_from_sse(sse: float, npix: int, peak: float = 255.0) -> float:
    """``10 log10(peak^2 N / SSE)`` (Sec. 4); +inf when SSE is 0."""
    if sse == 0:
        return math.inf
    return 10.0 * math.log10(peak * peak * npix / sse)


def psnr_images(a: np.ndarray, b: np.ndarray, peak: float = 255.0) -> float:
    """PSNR between two images of equal shape, FP64 (Sec. 4)."""
    d = np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)
    return psnr_from_sse(float(np.sum(d * d)), d.size, peak)


# --------------------------------------------------------------------------
# Sec. 4: SSIM, the second quality measure (Wang, Bovik, Sheikh and Simoncelli
# 2004, which the paper cites).  Reading of the parameters the paper leaves to
# that reference: an 11x11 circular Gaussian window with standard deviation
# 1.5, normalised to sum 1; K1 = 0.01, K2 = 0.03, dynamic range L = 255;
# every window position that lies inside the image ("valid" positions, no
# padding, no downsampling); MSSIM is the mean of the map.  Applied to the
# original and the stored (rounded, clamped) reconstruction.
# --------------------------------------------------------------------------
SSIM_WIN = 11
SSIM_SIGMA = 1.5
SSIM_C1 = (0.01 * 255.0) ** 2
SSIM_C2 = (0.03 * 255.0) ** 2


def ssim_window() -> np.ndarray:
    """The normalised 11x11 Gaussian weights, FP64."""
    k = np.arange(SSIM_WIN, dtype=np.float64) - (SSIM_WIN - 1) / 2.0
    g = np.exp(-(k[:, None] ** 2 + k[None, :] ** 2) / (2.0 * SSIM_SIGMA ** 2))
    return g / g.sum()


def ssim_map(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """SSIM at every valid window position: the weighted means, variances and
    covariance of the two windows, then
    ``(2 mu_a mu_b + C1)(2 s_ab + C2) / ((mu_a^2 + mu_b^2 + C1)(s_a^2 + s_b^2 + C2))``."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    w = ssim_window()
    wa = np.lib.stride_tricks.sliding_window_view(a, (SSIM_WIN, SSIM_WIN))
    wb = np.lib.stride_tricks.sliding_window_view(b, (SSIM_WIN, SSIM_WIN))
    mu_a = np.einsum("ijkl,kl->ij", wa, w)
    mu_b = np.einsum("ijkl,kl->ij", wb, w)
    s_aa = np.einsum("ijkl,kl->ij", (wa - mu_a[:, :, None, None]) ** 2, w)
    s_bb = np.einsum("ijkl,kl->ij", (wb - mu_b[:, :, None, None]) ** 2, w)
    s_ab = np.einsum("ijkl,kl->ij", (wa - mu_a[:, :, None, None]) * (wb - mu_b[:, :, None, None]), w)
    num = (2.0 * mu_a * mu_b + SSIM_C1) * (2.0 * s_ab + SSIM_C2)
    den = (mu_a * mu_a + mu_b * mu_b + SSIM_C1) * (s_aa + s_bb + SSIM_C2)
    return num / den


def mssim(a: np.ndarray, b: np.ndarray) -> float:
    """Mean SSIM over the valid window positions."""
    return float(np.mean(ssim_map(a, b)))


def ape(measure: float, reference: float) -> float:
    """Absolute percentage error of a quality measure against the exact DCT's
    (Sec. 4): ``100 |m - m_DCT| / m_DCT``."""
    return 100.0 * abs(measure - reference) / abs(reference)


def compress_zonal_exact(img: np.ndarray, r: int) -> dict:
    """Sec. 4 procedure with exact arithmetic: forward, keep the first ``r``
    zig-zag coefficients, inverse, reassemble; SSE of the unrounded
    reconstruction, PSNR, and the stored uint8 image."""
    x = np.asarray(img)
    y = forward_int(x)
    yk = np.where(zonal_mask(r)[None, None], y, 0)
    z = inverse_numerator(yk)
    e = z - 2304 * to_blocks(x.astype(np.int64))
    blk_sse = np.sum(e * e, axis=(2, 3))  # int64 per block, scaled by 2304^2
    sse_num = sum(int(v) for v in blk_sse.ravel())
    sse = float(Fraction(sse_num, 2304 * 2304))
    out = from_blocks(np.clip(round_half_even_div(z, 2304), 0, 255).astype(np.uint8))
    return {
        "coef": y,
        "numerator": z,
        "recon_u8": out,
        "block_sse": blk_sse.astype(np.float64) / (2304.0 * 2304.0),
        "sse": sse,
        "psnr": psnr_from_sse(sse, x.size),
        "psnr_u8": psnr_images(out, x),
    }


def compress_zonal_fp64(img: np.ndarray, r: int, transform: str = "approx") -> dict:
    """Sec. 4 procedure in FP64 with an orthonormal matrix, written as the
    paper writes it: ``B = C A C^T``, zonal mask, ``A' = C^T B' C``.
    ``transform`` is "approx" (C_hat of Sec. 2) or "dct" (the exact DCT)."""
    c = c_hat() if transform == "approx" else dct_matrix()
    a = to_blocks(np.asarray(img).astype(np.float64))
    b = np.einsum("um,yxmn,vn->yxuv", c, a, c)
    bk = np.where(zonal_mask(r)[None, None], b, 0.0)
    rec = np.einsum("um,yxuv,vn->yxmn", c, bk, c)
    d = rec - a
    sse = float(np.sum(d * d))
    return {"coef": b, "recon": from_blocks(rec), "sse": sse,
            "psnr": psnr_from_sse(sse, a.size // 1)}


# --------------------------------------------------------------------------
# Quantisation with S absorbed (Sec. 2 last paragraph; Sec. 5.3).
# --------------------------------------------------------------------------
def qstep(qp: float) -> float:
    """Quantisation step ``2^(QP/6)``: 1 at QP = 0 and doubling every six
    points, the step law of the HEVC quantiser that Sec. 5.3 sweeps."""
    return 2.0 ** (qp / 6.0)


def _quant_quotient_fp64(y: np.ndarray, qp: float) -> np.ndarray:
    """``|B| / Qstep = |Y| / sqrt(nnz_u nnz_v 2^(QP/3))`` in FP64.

    ``s_u s_v = 1 / sqrt(nnz_u nnz_v)`` (``nnz = diag(T T^T)``, Sec. 2), so the
    quotient is one division by the square root of ``nnz_u nnz_v 2^(QP/3)``.
    Whenever the quotient is rational that radicand is an exact FP64 number
    whose square root is exact, and a correctly rounded division then lands
    exactly on every half-integer quotient: the ties of the rounding rule are
    decided exactly (when the quotient is irrational there are no ties)."""
    nnz = np.diag(t_t_transpose()).astype(np.float64)
    den = np.sqrt(nnz[:, None] * nnz[None, :] * 2.0 ** (qp / 3.0))
    return np.abs(y).astype(np.float64) / den


def quant_levels(coef: np.ndarray, qp: float, precision: str = "fp64") -> np.ndarray:
    """``level = sign(B) floor(|B| / Qstep + 1/2)`` with ``B = s_u s_v Y``
    (rounding half away from zero).

    ``precision="fp64"``: the definition in FP64, ties decided exactly.
    ``precision="fp32"``: the same decision taken in single precision, as a
    GPU takes it: one rounded FP32 product of the exact integer ``Y`` and the
    FP32 constant ``fp32(s_u s_v / Qstep)``, then ``floor(|p| + 0.5)`` with the
    addition rounded to FP32.
    """
    s = s_diag()
    y = np.asarray(coef, dtype=np.int64)
    if precision == "fp64":
        q = _quant_quotient_fp64(y, qp)
        return (np.sign(y) * np.floor(q + 0.5)).astype(np.int64)
    if precision == "fp32":
        k = (s[:, None] * s[None, :] / qstep(qp)).astype(np.float32)
        p = y.astype(np.float32) * k
        a = np.abs(p) + np.float32(0.5)
        assert a.dtype == np.float32
        return (np.sign(p) * np.floor(a)).astype(np.int64)
    raise ValueError(precision)


def compress_quant(img: np.ndarray, qp: float, precision: str = "fp64") -> dict:
    """Forward, quantise with S absorbed, dequantise, inverse (FP64), for an
    int16 residual plane.  Output plane: ``clamp(round_half_to_even(x_hat))``
    as int16; PSNR of the unrounded reconstruction with peak 255."""
    x = np.asarray(img)
    y = forward_int(x)
    lev = quant_levels(y, qp, precision)
    s = s_diag()
    d = lev.astype(np.float64) * (s[:, None] * s[None, :]) * qstep(qp)  # S B' S
    rec = np.einsum("um,yxuv,vn->yxmn", T.astype(np.float64), d, T.astype(np.float64))
    a = to_blocks(x.astype(np.float64))
    diff = rec - a
    sse = float(np.sum(diff * diff))
    out = from_blocks(np.clip(np.rint(rec), -32768, 32767).astype(np.int16))
    return {"coef": y, "levels": lev, "recon": from_blocks(rec), "recon_i16": out,
            "sse": sse, "psnr": psnr_from_sse(sse, x.size)}


# --------------------------------------------------------------------------
# Sec. 3: similarity and coding measures (Table 2).
# --------------------------------------------------------------------------
def ar1_covariance(rho: float = 0.95, n: int = N) -> np.ndarray:
    """``R[i, j] = rho^|i-j|`` (Sec. 3.2, first-order Markov model)."""
    i = np.arange(n)
    return rho ** np.abs(i[:, None] - i[None, :])


def dct_distortion(ct: np.ndarray) -> float:
    """``d2 = 1 - (1/N) ||diag(C Ct^T)||^2`` (Sec. 3.2)."""
    c = dct_matrix(ct.shape[0])
    return 1.0 - float(np.sum(np.diag(c @ ct.T) ** 2)) / ct.shape[0]


def total_error_energy(ct: np.ndarray) -> float:
    """``eps = pi ||C - Ct||_F^2`` (Sec. 3.2)."""
    c = dct_matrix(ct.shape[0])
    return math.pi * float(np.sum((c - ct) ** 2))


def mse_measure(ct: np.ndarray, rho: float = 0.95) -> float:
    """``MSE = (1/N) tr((C - Ct) R (C - Ct)^T)`` (Sec. 3.2)."""
    c = dct_matrix(ct.shape[0])
    d = c - ct
    return float(np.trace(d @ ar1_covariance(rho, ct.shape[0]) @ d.T)) / ct.shape[0]


def coding_gain(ct: np.ndarray, rho: float = 0.95) -> float:
    """Transform coding gain ``C_g`` (Sec. 3.3), in dB."""
    n = ct.shape[0]
    s = ct @ ar1_covariance(rho, n) @ ct.T
    sii = np.diag(s)
    norms = np.sqrt(np.sum(ct * ct, axis=1))
    geo = float(np.prod(sii * norms)) ** (1.0 / n)
    return 10.0 * math.log10(float(np.mean(sii)) / geo)


def transform_efficiency(ct: np.ndarray, rho: float = 0.95) -> float:
    """Transform efficiency ``eta`` (Sec. 3.3), in percent."""
    s = ct @ ar1_covariance(rho, ct.shape[0]) @ ct.T
    return 100.0 * float(np.sum(np.abs(np.diag(s)))) / float(np.sum(np.abs(s)))


def table2_row(ct: np.ndarray) -> dict:
    return {
        "d2": dct_distortion(ct),
        "eps": total_error_energy(ct),
        "mse": mse_measure(ct),
        "cg": coding_gain(ct),
        "eta": transform_efficiency(ct),
    }

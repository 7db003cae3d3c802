"""SSIM (Sec. 4) on the GPU against the FP64 oracle.

Tolerance: the kernel accumulates the five window moments of centred pixels
(|x - 128| <= 128) in FP32, so a variance or covariance carries an absolute
error of a few units of 2^-24 * 121 * 128^2 (about 1e-3); through the SSIM
ratio, whose variance terms are offset by C2 = 58.5, that is at most a few
1e-5 per window position, and the mean over the positions is held to 5e-5.
"""

import math

import numpy as np
import pytest

import oracle as O
from paper_1606_05562_gb300 import atdct16, build, synth

pytestmark = pytest.mark.gpu
SSIM_ATOL = 5e-5


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    atdct16.lib()
    return t


@pytest.fixture(scope="module")
def plan(torch):
    p = atdct16.Plan(atdct16.U8, max_images=64, workspace_bytes=64 << 20)
    yield p
    p.close()


def _gpu_ssim(torch, plan, pairs):
    dev = [(torch.from_numpy(np.ascontiguousarray(a)).cuda(), torch.from_numpy(np.ascontiguousarray(b)).cuda())
           for a, b in pairs]
    out = torch.empty(len(pairs), dtype=torch.float64, device="cuda")
    plan.ssim([atdct16.image(a, b, 0) for a, b in dev], out)
    torch.cuda.synchronize()
    return out.cpu().tolist()


def test_ssim_of_reconstructions_matches_oracle(torch, plan):
    pairs = []
    for (h, w), r in zip(((16, 16), (48, 272), (160, 96), (256, 256), (64, 400)), (1, 6, 36, 100, 256)):
        img = synth.ar1_image(h, w, 0.9, 31 + h + w)
        rec = O.compress_zonal_exact(img, r)["recon_u8"]
        pairs.append((img, rec))
    got = _gpu_ssim(torch, plan, pairs)
    for (a, b), g in zip(pairs, got):
        assert g == pytest.approx(O.mssim(a, b), abs=SSIM_ATOL)


def test_ssim_closed_forms(torch, plan):
    rng = np.random.default_rng(5)
    a = rng.integers(0, 256, (80, 144)).astype(np.uint8)
    const = [(np.full((32, 48), ca, np.uint8), np.full((32, 48), cb, np.uint8))
             for ca, cb in ((0, 0), (10, 200), (255, 0))]
    got = _gpu_ssim(torch, plan, [(a, a)] + const)
    assert got[0] == pytest.approx(1.0, abs=1e-6)
    for (x, y), g in zip(const, got[1:]):
        ca, cb = float(x[0, 0]), float(y[0, 0])
        want = (2 * ca * cb + O.SSIM_C1) / (ca * ca + cb * cb + O.SSIM_C1)
        assert g == pytest.approx(want, abs=1e-6)


def test_ssim_bench_batch_sample(torch, plan):
    """Images of the 64 x 512 x 512 workload against their zonal reconstructions."""
    batch = synth.image_batch_512(4, 512, first_seed=100)
    pairs = [(batch[i], O.compress_zonal_exact(batch[i], r)["recon_u8"]) for i, r in zip(range(4), (6, 36, 100, 16))]
    got = _gpu_ssim(torch, plan, pairs)
    for (a, b), g in zip(pairs, got):
        assert g == pytest.approx(O.mssim(a, b), abs=SSIM_ATOL)

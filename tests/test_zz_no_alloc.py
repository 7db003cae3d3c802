"""The zonal entry point that allocates nothing, against the plan-based one
and against the CPU oracle.

Callers that cannot allocate device memory while they compress (fixed memory
budgets, latency-critical paths, applications whose own allocator owns the
device) use atdct16_compress_zonal_noalloc.  Its results must equal those of
atdct16_compress_zonal and of the oracle's exact reconstruction, with the same
tolerances as the other parity tests, on two calls in a row (the second call
reuses the shared scratch area), and its plan-free status read must report
success after each good call.  This file is collected last on purpose."""

import math

import numpy as np
import pytest

import oracle as O
from paper_1606_05562_gb300 import atdct16, build, synth

pytestmark = pytest.mark.gpu

PSNR_RTOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    atdct16.lib()
    return t


def _batch(seed):
    rng = np.random.default_rng(seed)
    sizes = [(16 * int(rng.integers(1, 24)), 16 * int(rng.integers(1, 40))) for _ in range(12)]
    imgs = [synth.ar1_image(h, w, float(rng.uniform(0.8, 0.97)), seed * 100 + i) for i, (h, w) in enumerate(sizes)]
    imgs.append(synth.ar1_image(512, 512, 0.95, seed))
    rs = [int(v) for v in rng.choice(synth.ZONAL_R_SWEEP, size=len(imgs))]
    return imgs, rs


def _run(torch, imgs, rs, fn):
    srcs = [torch.from_numpy(im).cuda() for im in imgs]
    dsts = [torch.full_like(s, 3) for s in srcs]
    descs = [atdct16.image(s, d, r) for s, d, r in zip(srcs, dsts, rs)]
    psnr = torch.empty(len(imgs), dtype=torch.float64, device="cuda")
    sse = torch.empty(len(imgs), dtype=torch.float64, device="cuda")
    fn(descs, psnr, sse)
    torch.cuda.synchronize()
    return [d.cpu().numpy() for d in dsts], psnr.cpu().numpy(), sse.cpu().numpy()


def test_noalloc_matches_plan_path_twice(torch):
    plan = atdct16.Plan(atdct16.U8, max_images=64)
    for seed in (1, 2):  # two calls in a row
        imgs, rs = _batch(seed)
        ref = _run(torch, imgs, rs, lambda d, p, s: plan.compress_zonal(d, p, s))
        got = _run(torch, imgs, rs, lambda d, p, s: atdct16.compress_zonal_noalloc(d, p, s))
        for a, b in zip(ref[0], got[0]):
            assert np.array_equal(a, b)
        for pr, pg in zip(ref[1], got[1]):
            if math.isinf(pr):
                assert math.isinf(pg)
            else:
                assert pg == pytest.approx(pr, rel=PSNR_RTOL, abs=1e-5)
        np.testing.assert_allclose(got[2], ref[2], rtol=PSNR_RTOL)
        assert atdct16.noalloc_last_device_status() == atdct16.OK
        # the oracle's exact route (Sec. 4 procedure), image by image
        for im, r, out, pg in zip(imgs, rs, got[0], got[1]):
            want = O.compress_zonal_exact(im, r)
            assert np.array_equal(out, want["recon_u8"])
            if math.isinf(want["psnr"]):
                assert math.isinf(pg)
            else:
                assert pg == pytest.approx(want["psnr"], rel=PSNR_RTOL, abs=1e-5)
    plan.close()


def test_noalloc_rejects_requests_beyond_its_maximum(torch):
    img = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    out = torch.zeros_like(img)
    psnr = torch.empty(65, dtype=torch.float64, device="cuda")
    with pytest.raises(atdct16.Atdct16Error) as e:
        atdct16.compress_zonal_noalloc([atdct16.image(img, out, 16)] * 65, psnr)
    assert e.value.status == atdct16.ENOMEM
    big = torch.zeros((16 * 1040, 2048), dtype=torch.uint8, device="cuda")  # 16 x 1040 = 16640 tiles
    bout = torch.zeros_like(big)
    with pytest.raises(atdct16.Atdct16Error) as e:
        atdct16.compress_zonal_noalloc([atdct16.image(big, bout, 16)] * 8, psnr)  # 133120 tiles > 131072
    assert e.value.status == atdct16.ENOMEM

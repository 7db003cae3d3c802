"""Resident mixed-size batches under a CUDA graph with the autotuner
(atdct16_batch_*), against the oracle and the per-call entry point."""

import json
import math

import numpy as np
import pytest

import oracle as O
from paper_1606_05562_gb300 import atdct16, build, synth

pytestmark = pytest.mark.gpu


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
    p = atdct16.Plan(atdct16.U8, max_images=256)
    yield p
    p.close()


def _mixed(seed, n=40, lo=16, hi=400):
    imgs = synth.mixed_batch(n, lo=lo, hi=hi, seed=seed)
    rs = [int(v) for v in np.random.default_rng(seed).choice(synth.ZONAL_R_SWEEP, size=len(imgs))]
    return imgs, rs


def _dev(torch, imgs):
    src = [torch.from_numpy(im).cuda() for im in imgs]
    dst = [torch.full_like(s, 9) for s in src]
    return src, dst


@pytest.mark.parametrize("flags", [0, atdct16.BATCH_GRAPH, atdct16.BATCH_AUTOTUNE | atdct16.BATCH_GRAPH])
def test_batch_matches_oracle_and_per_call(torch, plan, flags):
    imgs, rs = _mixed(11)
    src, dst = _dev(torch, imgs)
    descs = [atdct16.image(s, d, r) for s, d, r in zip(src, dst, rs)]
    psnr = torch.empty(len(imgs), dtype=torch.float64, device="cuda")
    b = atdct16.Batch(plan, descs, psnr, flags=flags)
    for _ in range(2):  # re-launching the same graph gives the same result
        for d in dst:
            d.fill_(9)
        b.launch()
        torch.cuda.synchronize()
        for im, r, d, p in zip(imgs, rs, dst, psnr.cpu().tolist()):
            ref = O.compress_zonal_exact(im, r)
            assert np.array_equal(d.cpu().numpy(), ref["recon_u8"])
            if math.isinf(ref["psnr"]):
                assert math.isinf(p)
            else:
                assert p == pytest.approx(ref["psnr"], rel=1e-5, abs=1e-5)
    # the per-call entry point gives the same bytes and PSNR
    dst2 = [torch.full_like(s, 1) for s in src]
    psnr2 = torch.empty_like(psnr)
    plan.compress_zonal([atdct16.image(s, d, r) for s, d, r in zip(src, dst2, rs)], psnr2)
    torch.cuda.synchronize()
    for a, c in zip(dst, dst2):
        assert torch.equal(a, c)
    fin = ~psnr.isinf()
    assert torch.equal(psnr.isinf(), psnr2.isinf())
    # the same kernel gives the same PSNR to the bit; an autotuned batch may run
    # another kernel variant, whose FP32 per-tile energy sums in another order
    rtol = 1e-6 if flags & atdct16.BATCH_AUTOTUNE else 1e-12
    assert torch.allclose(psnr[fin], psnr2[fin], rtol=rtol, atol=0)
    info = b.info()
    assert info["tiles"] > 0 and info["grid"] > 0
    if flags & atdct16.BATCH_AUTOTUNE:
        assert info["tuned_ms"] > 0
    b.close()


def test_autotune_cache_file(torch, tmp_path, monkeypatch):
    path = tmp_path / "tune.jsonl"
    monkeypatch.setenv("ATDCT16_TUNE_CACHE", str(path))
    imgs, rs = _mixed(12, n=10)
    src, dst = _dev(torch, imgs)
    descs = [atdct16.image(s, d, r) for s, d, r in zip(src, dst, rs)]
    psnr = torch.empty(len(imgs), dtype=torch.float64, device="cuda")
    p1 = atdct16.Plan(atdct16.U8, max_images=16)
    b1 = atdct16.Batch(p1, descs, psnr, flags=atdct16.BATCH_AUTOTUNE)
    lines = path.read_text().strip().splitlines()
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["warps"] in (2, 4, 8) and rec["ms"] > 0
    b1.close()
    p1.close()
    # a fresh plan finds the result in the file instead of re-tuning
    p2 = atdct16.Plan(atdct16.U8, max_images=16)
    b2 = atdct16.Batch(p2, descs, psnr, flags=atdct16.BATCH_AUTOTUNE)
    assert len(path.read_text().strip().splitlines()) == 1
    info = b2.info()
    assert info["warps"] == rec["warps"] and info["prefetch"] == rec["prefetch"]
    b2.close()
    p2.close()


def test_autotune_rejects_in_place(torch, plan):
    img = torch.from_numpy(synth.ar1_image(64, 64, 0.9, 1)).cuda()
    psnr = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(atdct16.Atdct16Error) as e:
        atdct16.Batch(plan, [atdct16.image(img, img, 16)], psnr, flags=atdct16.BATCH_AUTOTUNE)
    assert e.value.status == atdct16.EINVAL
    b = atdct16.Batch(plan, [atdct16.image(img, img, 256)], psnr, flags=atdct16.BATCH_GRAPH)  # in place is fine untuned
    b.launch()
    torch.cuda.synchronize()
    b.close()


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_every_kernel_variant_matches_oracle(torch, plan, variant):
    """Each zonal kernel variant, pinned: bit-exact pixels against the exact
    oracle, PSNR within the FP tolerance (r spans every mask extent)."""
    rs = [0, 1, 2, 6, 16, 36, 64, 100, 150, 255, 256]
    imgs = _mixed(11)[0][:len(rs)]
    src, dst = _dev(torch, imgs)
    descs = [atdct16.image(s, d, r) for s, d, r in zip(src, dst, rs)]
    psnr = torch.empty(len(imgs), dtype=torch.float64, device="cuda")
    b = atdct16.Batch(plan, descs, psnr, flags=atdct16.BATCH_GRAPH | atdct16.batch_variant(variant))
    assert b.info()["variant"] == atdct16.ZONAL_VARIANTS[variant]
    b.launch()
    torch.cuda.synchronize()
    for im, r, d, p in zip(imgs, rs, dst, psnr.cpu().tolist()):
        ref = O.compress_zonal_exact(im, r)
        assert np.array_equal(d.cpu().numpy(), ref["recon_u8"]), (variant, r)
        if math.isinf(ref["psnr"]):
            assert math.isinf(p)
        else:
            assert p == pytest.approx(ref["psnr"], rel=1e-5, abs=1e-5)
    b.close()


def test_tc_variant_long_pipeline_matches_oracle(torch, plan):
    """The tcgen05 variant with every CTA walking several tile pairs (its
    software pipeline in steady state), pairs that straddle images of
    different sizes and r, ragged tiles: pixels bit-identical to the
    integer-pipe variant's on every image and to the exact oracle on a
    sample; PSNR within the FP tolerance."""
    rng = np.random.default_rng(21)
    imgs = [synth.ar1_image(512, 512, 0.95, 300 + i) for i in range(48)]
    imgs += _mixed(22, n=12, lo=16, hi=400)[0]
    order = rng.permutation(len(imgs))
    imgs = [imgs[i] for i in order]
    rs = [int(v) for v in rng.choice([0, 37, 64, 100, 150, 200, 255, 256], size=len(imgs))]
    out = {}
    for v in (1, 3):
        src, dst = _dev(torch, imgs)
        descs = [atdct16.image(s, d, r) for s, d, r in zip(src, dst, rs)]
        psnr = torch.empty(len(imgs), dtype=torch.float64, device="cuda")
        b = atdct16.Batch(plan, descs, psnr, flags=atdct16.BATCH_GRAPH | atdct16.batch_variant(v))
        info = b.info()
        assert info["variant"] == atdct16.ZONAL_VARIANTS[v]
        if v == 3:
            assert info["tiles"] >= 8 * info["grid"]  # several pairs per CTA
        b.launch()
        b.launch()
        torch.cuda.synchronize()
        out[v] = ([d.cpu().numpy() for d in dst], psnr.cpu().tolist())
        b.close()
    for a, c in zip(out[1][0], out[3][0]):
        assert np.array_equal(a, c)
    assert out[3][1] == pytest.approx(out[1][1], rel=1e-5, abs=1e-5)
    for k in [0, 1] + [i for i in range(len(imgs)) if imgs[i].shape[1] % 128][:2]:
        ref = O.compress_zonal_exact(imgs[k], rs[k])
        assert np.array_equal(out[3][0][k], ref["recon_u8"]), rs[k]
        if math.isinf(ref["psnr"]):
            assert math.isinf(out[3][1][k])
        else:
            assert out[3][1][k] == pytest.approx(ref["psnr"], rel=1e-5, abs=1e-5)


# batch shapes that give the tcgen05 variant's CTAs 1, 2, 3 and 4 tile pairs
# (its prologue and loop guards differ for each): grid = min(4 per SM, tiles / 4),
# tiles per CTA = 2 ceil(tiles / (2 grid))
TC_DEPTHS = [("1-pair", [(16, 128)]), ("2-pairs", [(512, 512)]), ("3-pairs", [(512, 512)] * 24),
             ("4-pairs", [(512, 512)] * 31)]


@pytest.mark.parametrize("shapes", [s for _, s in TC_DEPTHS], ids=[i for i, _ in TC_DEPTHS])
def test_tc_variant_pipeline_depths(torch, plan, shapes):
    imgs = [synth.ar1_image(h, w, 0.9, 70 + i) for i, (h, w) in enumerate(shapes)]
    rs = [(0, 64, 100, 150, 256)[i % 5] for i in range(len(imgs))]
    got = {}
    for v in (1, 3):
        src, dst = _dev(torch, imgs)
        psnr = torch.empty(len(imgs), dtype=torch.float64, device="cuda")
        b = atdct16.Batch(plan, [atdct16.image(s, d, r) for s, d, r in zip(src, dst, rs)], psnr,
                          flags=atdct16.batch_variant(v))
        b.launch()
        assert b.last_device_status() == atdct16.OK
        got[v] = ([d.cpu().numpy() for d in dst], psnr.cpu().tolist())
        b.close()
    for a, c in zip(got[1][0], got[3][0]):
        assert np.array_equal(a, c)
    assert got[3][1] == pytest.approx(got[1][1], rel=1e-5, abs=1e-5)
    ref = O.compress_zonal_exact(imgs[0], rs[0])
    assert np.array_equal(got[3][0][0], ref["recon_u8"])


def test_tc_variant_tensor_wait_times_out_cleanly(torch):
    """With the MMA stall test hook the tcgen05 kernel issues no product: every
    CTA's bounded wait on the tensor core expires, it frees its tensor memory
    and returns, the batch's device status reads ETIMEOUT, and the context
    keeps working (a following tcgen05 batch matches the oracle)."""
    imgs = [synth.ar1_image(64, 256, 0.9, 40 + i) for i in range(3)]
    rs = [64, 150, 256]
    stall = atdct16.Plan(atdct16.U8, max_images=8, flags=atdct16.PLAN_TEST_STALL_MMA)
    src, dst = _dev(torch, imgs)
    psnr = torch.empty(len(imgs), dtype=torch.float64, device="cuda")
    b = atdct16.Batch(stall, [atdct16.image(s, d, r) for s, d, r in zip(src, dst, rs)], psnr,
                      flags=atdct16.batch_variant(3))
    b.launch()
    assert b.last_device_status() == atdct16.ETIMEOUT
    b.close()
    stall.close()
    ok = atdct16.Plan(atdct16.U8, max_images=8)
    src, dst = _dev(torch, imgs)
    b = atdct16.Batch(ok, [atdct16.image(s, d, r) for s, d, r in zip(src, dst, rs)], psnr,
                      flags=atdct16.batch_variant(3))
    b.launch()
    assert b.last_device_status() == atdct16.OK
    for im, r, d in zip(imgs, rs, dst):
        assert np.array_equal(d.cpu().numpy(), O.compress_zonal_exact(im, r)["recon_u8"]), r
    b.close()
    ok.close()


BOX_SHAPES = [(w, d, v) for w in (2, 4, 8) for d in (1, 2, 3) for v in (16, 8)]


@pytest.mark.parametrize("shape", BOX_SHAPES, ids=[f"w{w}-d{d}-v{v}" for w, d, v in BOX_SHAPES])
def test_every_box_shape_matches_oracle(torch, plan, shape):
    """Each launch shape the autotuner may pick for the kernels of r <= 36
    (tiles per CTA x staging depth x copy width), pinned: bit-exact pixels,
    PSNR within tolerance, for every extent class (and a general job)."""
    rs = [1, 2, 6, 7, 16, 21, 22, 36, 64, 1, 36, 6]
    imgs = _mixed(13, n=len(rs), lo=16, hi=300)[0][:len(rs)]
    src, dst = _dev(torch, imgs)
    descs = [atdct16.image(s, d, r) for s, d, r in zip(src, dst, rs)]
    psnr = torch.empty(len(imgs), dtype=torch.float64, device="cuda")
    b = atdct16.Batch(plan, descs, psnr, flags=atdct16.BATCH_GRAPH | atdct16.batch_shape(*shape))
    chosen = b.tuning()["chosen"]
    assert (chosen["tiles_per_cta"], chosen["staging_depth"], chosen["vector_bytes"]) == shape
    b.launch()
    torch.cuda.synchronize()
    for im, r, d, p in zip(imgs, rs, dst, psnr.cpu().tolist()):
        ref = O.compress_zonal_exact(im, r)
        assert np.array_equal(d.cpu().numpy(), ref["recon_u8"]), (shape, r)
        assert p == pytest.approx(ref["psnr"], rel=1e-5, abs=1e-5)
    b.close()


def test_autotune_times_every_candidate(torch):
    # r <= 36 and r > 36 jobs: the box shapes first, then the general variants
    imgs, _ = _mixed(14, n=24, lo=64, hi=512)
    rs = [(16, 36, 100)[i % 3] for i in range(len(imgs))]
    src, dst = _dev(torch, imgs)
    descs = [atdct16.image(s, d, r) for s, d, r in zip(src, dst, rs)]
    psnr = torch.empty(len(imgs), dtype=torch.float64, device="cuda")
    p = atdct16.Plan(atdct16.U8, max_images=64)
    b = atdct16.Batch(p, descs, psnr, flags=atdct16.BATCH_AUTOTUNE)
    t = b.tuning()
    cands = t["candidates"]
    shapes = {(c["tiles_per_cta"], c["staging_depth"], c["vector_bytes"]) for c in cands}
    assert set(BOX_SHAPES) <= shapes
    assert {c["variant"] for c in cands} == set(atdct16.ZONAL_VARIANTS)
    assert all(c["ms"] > 0 for c in cands)
    ch = t["chosen"]
    # the box phase comes first (general shape at its default) and the chosen
    # box shape is its fastest candidate; the general phase ran with that box
    # shape and the chosen variant is its fastest
    key = lambda c: (c["tiles_per_cta"], c["staging_depth"], c["vector_bytes"], c["box_ctas"])
    box_phase = [c for c in cands if c["phase"] == 0]
    gen_phase = [c for c in cands if c["phase"] == 1]
    assert cands == box_phase + gen_phase
    assert {(c["tiles_per_cta"], c["staging_depth"], c["vector_bytes"]) for c in box_phase} == set(BOX_SHAPES)
    assert key(ch) == key(min(box_phase, key=lambda c: c["ms"]))
    assert gen_phase and all(key(c) == key(ch) for c in gen_phase)
    best_gen = min(gen_phase, key=lambda c: c["ms"])
    assert (ch["variant"], ch["general_ctas"]) == (best_gen["variant"], best_gen["general_ctas"])
    assert ch["ms"] == pytest.approx(best_gen["ms"])
    b.launch()
    torch.cuda.synchronize()
    for im, r, d, pv in zip(imgs, rs, dst, psnr.cpu().tolist()):
        ref = O.compress_zonal_exact(im, r)
        assert np.array_equal(d.cpu().numpy(), ref["recon_u8"])
        assert pv == pytest.approx(ref["psnr"], rel=1e-5, abs=1e-5)
    b.close()
    p.close()

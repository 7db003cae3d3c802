"""Continuous-batching server: every result is the same alone and in the
mix, memory-budget admission serialises what does not fit, oversize
requests are refused."""

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


def _requests(n, seed, lo=16, hi=512):
    imgs = synth.mixed_batch(n, lo=lo, hi=hi, seed=seed)
    rs = [int(v) for v in np.random.default_rng(seed).choice((6, 16, 36, 64), size=len(imgs))]
    return imgs, rs


def _pinned(torch, arr):
    return torch.from_numpy(arr).pin_memory()


def test_same_result_alone_and_in_the_mix(torch):
    imgs, rs = _requests(30, 21)
    srcs = [_pinned(torch, im) for im in imgs]
    mix = [torch.zeros_like(s).pin_memory() for s in srcs]
    srv = atdct16.Server(memory_budget_bytes=64 << 20, max_batch=8, compute_slots=3)
    tickets = [srv.submit(s, d, r) for s, d, r in zip(srcs, mix, rs)]  # all arrive at once
    mix_psnr = [srv.wait(t)[0] for t in tickets]
    st = srv.stats()
    assert st["completed"] == len(imgs) and st["launches"] >= 2 and st["arena_used"] == 0
    for i, (s, r) in enumerate(zip(srcs, rs)):  # each request alone
        alone = torch.zeros_like(s).pin_memory()
        p, lat = srv.wait(srv.submit(s, alone, r))
        assert lat > 0
        assert torch.equal(alone, mix[i])
        assert p == mix_psnr[i] or (math.isinf(p) and math.isinf(mix_psnr[i]))
    srv.close()
    for im, r, out, p in list(zip(imgs, rs, mix, mix_psnr))[:8]:
        ref = O.compress_zonal_exact(im, r)
        assert np.array_equal(out.numpy(), ref["recon_u8"])
        assert p == pytest.approx(ref["psnr"], rel=1e-5, abs=1e-5)


def test_admission_under_a_small_budget(torch):
    imgs = [synth.ar1_image(512, 512, 0.9, 30 + i) for i in range(6)]  # 512 KB of arena each
    srcs = [_pinned(torch, im) for im in imgs]
    outs = [torch.zeros_like(s).pin_memory() for s in srcs]
    srv = atdct16.Server(memory_budget_bytes=(3 << 19) + 4096, max_batch=16, compute_slots=2)  # fits 3
    tickets = [srv.submit(s, d, 36) for s, d in zip(srcs, outs)]
    for im, d, t in zip(imgs, outs, tickets):
        p, _ = srv.wait(t)
        ref = O.compress_zonal_exact(im, 36)
        assert np.array_equal(d.numpy(), ref["recon_u8"])
        assert p == pytest.approx(ref["psnr"], rel=1e-5)
    big = _pinned(torch, synth.ar1_image(1024, 1024, 0.9, 1))
    with pytest.raises(atdct16.Atdct16Error) as e:
        srv.submit(big, torch.zeros_like(big), 16)
    assert e.value.status == atdct16.ENOMEM
    srv.close()


def test_request_timing_stages_in_order(torch):
    # requests with scheduled arrival times: every stage boundary on the
    # server clock lies between the previous one and completion, the results
    # stay exact, and wait() measures latency from the arrival
    imgs, rs = _requests(12, 23, lo=64, hi=600)
    srcs = [_pinned(torch, im) for im in imgs]
    outs = [torch.zeros_like(s).pin_memory() for s in srcs]
    srv = atdct16.Server(memory_budget_bytes=256 << 20, max_batch=4, compute_slots=2)
    t0 = atdct16.server_clock()
    tickets = [srv.submit(s, d, r, arrival=t0 - 0.001 * (len(imgs) - i)) for i, (s, d, r) in
               enumerate(zip(srcs, outs, rs))]
    eps = 2e-3  # device timestamps are placed on the host clock through one reference event
    for i, (im, r, d, t) in enumerate(zip(imgs, rs, outs, tickets)):
        p, tm = srv.wait_timing(t)
        assert tm["arrival"] == pytest.approx(t0 - 0.001 * (len(imgs) - i), abs=1e-9)
        order = [tm[k] for k in ("arrival", "submit", "h2d_start", "h2d_end", "compute_start", "compute_end",
                                 "d2h_end", "done")]
        assert all(b >= a - eps for a, b in zip(order, order[1:])), tm
        assert tm["h2d_end"] >= tm["h2d_start"] and tm["compute_end"] >= tm["compute_start"]
        ref = O.compress_zonal_exact(im, r)
        assert np.array_equal(d.numpy(), ref["recon_u8"])
        assert p == pytest.approx(ref["psnr"], rel=1e-5, abs=1e-5)
    s2 = _pinned(torch, imgs[0])
    arr = atdct16.server_clock() - 0.05
    _, lat = srv.wait(srv.submit(s2, torch.zeros_like(s2).pin_memory(), 16, arrival=arr))
    assert lat >= 0.05
    srv.close()

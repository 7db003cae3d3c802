"""Parity of the coefficient pipeline (standalone forward / exact inverse,
1-D and 2-D, row-major or zig-zag block layout, zig-zag quantisation levels)
with the CPU oracle, through the C ABI.  Everything here is integer work and
must match bit for bit."""

import functools

import numpy as np
import pytest

import oracle as O
from paper_1606_05562_gb300 import atdct16, build, synth

pytestmark = pytest.mark.gpu

SHAPES = [(16, 16), (48, 400), (32, 1040), (80, 256)]  # 400 / 1040: last tile holds 1 / 1 block


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    atdct16.lib()
    return t


@pytest.fixture(scope="module", params=[False, True], ids=["rowmajor", "zigzag"])
def cplan(request, torch):
    p = atdct16.Plan(atdct16.U8, max_images=4, zigzag=request.param)
    yield p
    assert p.last_device_status() == atdct16.OK
    p.close()


def layout(plan, y_blocks):
    """Oracle coefficients (by, bx, 16, 16) in the plan's block layout, flat."""
    return (O.to_zigzag(y_blocks) if plan.zigzag else y_blocks).reshape(-1)


def dev(torch, arr, pitch_extra=0):
    h, w = arr.shape
    dt = torch.uint8 if arr.dtype == np.uint8 else torch.int16
    base = torch.zeros((h, w + pitch_extra), dtype=dt, device="cuda")
    view = base[:, :w]
    view.copy_(torch.from_numpy(np.ascontiguousarray(arr)))
    return view


def out_img(torch, h, w, dt, pitch_extra=0):
    return torch.full((h, w + pitch_extra), 77, dtype=dt, device="cuda")[:, :w]


def run_forward(torch, plan, x, dtype, pitch_extra=0):
    h, w = x.shape
    coef = torch.full((h * w,), -7, dtype=torch.int32, device="cuda")
    plan.forward(dev(torch, x, pitch_extra), coef, dtype=dtype)
    torch.cuda.synchronize()
    return coef.cpu().numpy()


def run_inverse(torch, plan, coef_flat, h, w, dtype, pitch_extra=0):
    coef = torch.from_numpy(np.ascontiguousarray(coef_flat.astype(np.int32))).cuda()
    out = out_img(torch, h, w, torch.uint8 if dtype == atdct16.U8 else torch.int16, pitch_extra)
    plan.inverse(coef, out, dtype=dtype)
    torch.cuda.synchronize()
    return out.cpu().numpy()


# ------------------------------------------------------------ 2-D forward ---
@pytest.mark.parametrize("shape", SHAPES)
def test_forward_u8(torch, cplan, shape):
    img = synth.ar1_image(*shape, 0.9, 3)
    img[0, :16] = 255
    img[1, 16:32] = 0
    got = run_forward(torch, cplan, img, atdct16.U8, pitch_extra=16 if shape[1] < 512 else 0)
    assert np.array_equal(got, layout(cplan, O.forward_int(img)))


@pytest.mark.parametrize("shape", SHAPES)
def test_forward_i16(torch, cplan, shape):
    x = synth.laplacian_residual(*shape, seed=13)
    x[0, :16] = 32767
    x[1, :16] = -32768
    x[2:16, :16] = np.where(O.T[2:16] > 0, 32767, -32768)  # rows aligned with T's signs
    got = run_forward(torch, cplan, x, atdct16.I16)
    assert np.array_equal(got, layout(cplan, O.forward_int(x)))


# ------------------------------------------------------ 2-D exact inverse ---
def _coef_cases(h, w, seed):
    """(name, coefficient blocks) with the value ranges that select the
    kernel's routes: |Y| <= 2^18 (32-bit), anything up to the int32 limits
    (two halves), and a mix of the two across tiles."""
    rng = np.random.default_rng(seed)
    by, bx = h // 16, w // 16
    img = synth.ar1_image(h, w, 0.9, seed)
    y = O.forward_int(img)
    cases = [("forward", y)]
    masked = np.where(O.zonal_mask(36)[None, None], y, 0)
    cases.append(("masked", masked))
    cases.append(("small", rng.integers(-(1 << 18), (1 << 18) + 1, size=(by, bx, 16, 16))))
    cases.append(("huge", rng.integers(-(2**31), 2**31, size=(by, bx, 16, 16))))
    mixed = rng.integers(-3000, 3000, size=(by, bx, 16, 16))
    mixed[:, ::3, rng.integers(0, 16), rng.integers(0, 16)] = 2**31 - 1  # one wide coefficient in some tiles
    mixed[0, 0, 0, 0] = -(2**31)
    cases.append(("mixed", mixed))
    # ties: a DC of 1152 * k / 9 ... X_hat = Y_00 W_0^2 / 2304 = Y_00 / 256 per pixel: odd multiples of 128
    ties = np.zeros((by, bx, 16, 16), dtype=np.int64)
    ties[..., 0, 0] = 128 * (2 * rng.integers(0, 255, size=(by, bx)) + 1)
    cases.append(("ties", ties))
    return cases


@pytest.mark.parametrize("shape", [(16, 16), (48, 400), (32, 1040)])
@pytest.mark.parametrize("dtype", [atdct16.U8, atdct16.I16], ids=["u8", "i16"])
def test_inverse_exact(torch, cplan, shape, dtype):
    h, w = shape
    odt = np.uint8 if dtype == atdct16.U8 else np.int16
    for name, y in _coef_cases(h, w, seed=h + w):
        got = run_inverse(torch, cplan, layout(cplan, y), h, w, dtype)
        ref = O.inverse_exact(y, odt)
        assert np.array_equal(got, ref), f"{name}: {np.count_nonzero(got != ref)} pixels differ"


def test_ties_round_half_even(torch, cplan):
    # a DC-only block reconstructs to Y_00 * 9 / 2304 = Y_00 / 256 everywhere
    y = np.zeros((1, 4, 16, 16), dtype=np.int64)
    y[0, :, 0, 0] = [128, 384, 640, -128]  # 0.5, 1.5, 2.5, -0.5 -> 0, 2, 2, 0
    got = run_inverse(torch, cplan, layout(cplan, y), 16, 64, atdct16.U8)
    assert np.array_equal(got[:, ::16][0], [0, 2, 2, 0])
    got16 = run_inverse(torch, cplan, layout(cplan, y), 16, 64, atdct16.I16)
    assert np.array_equal(got16[:, ::16][0], [0, 2, 2, 0])


@pytest.mark.parametrize("dtype", [atdct16.U8, atdct16.I16], ids=["u8", "i16"])
def test_round_trip(torch, cplan, dtype):
    h, w = 64, 784
    x = synth.ar1_image(h, w, 0.95, 8) if dtype == atdct16.U8 else synth.laplacian_residual(h, w, seed=8)
    coef = torch.empty(h * w, dtype=torch.int32, device="cuda")
    cplan.forward(dev(torch, x), coef, dtype=dtype)
    out = out_img(torch, h, w, torch.uint8 if dtype == atdct16.U8 else torch.int16)
    cplan.inverse(coef, out, dtype=dtype)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), x)


@functools.lru_cache(maxsize=1)
def _big_image():
    return synth.ar1_image(4096, 8192, 0.95, 21)


def test_large_image_sampled_and_round_trip(torch, cplan):
    # the bench's coefficient workload shape, 4096 x 8192 (32 MiB in, 128 MiB
    # of coefficients): sampled blocks against the oracle, and the exact round
    # trip over the whole image
    h, w = 4096, 8192
    x = _big_image()
    xd = dev(torch, x)
    coef = torch.empty(h * w, dtype=torch.int32, device="cuda")
    cplan.forward(xd, coef)
    out = out_img(torch, h, w, torch.uint8)
    cplan.inverse(coef, out)
    torch.cuda.synchronize()
    assert torch.equal(out, xd)
    c = coef.cpu().numpy().reshape(h // 16, w // 16, 256)
    rng = np.random.default_rng(3)
    for _ in range(64):
        by, bx = int(rng.integers(0, h // 16)), int(rng.integers(0, w // 16))
        ref = O.forward_int(x[16 * by:16 * by + 16, 16 * bx:16 * bx + 16])[0, 0]
        ref = O.to_zigzag(ref) if cplan.zigzag else ref.reshape(-1)
        assert np.array_equal(c[by, bx], ref)


@pytest.mark.parametrize("shape", [(16, 32768), (4096, 16)])
def test_extreme_shapes(torch, cplan, shape):
    img = synth.ar1_image(*shape, 0.95, 71)
    got = run_forward(torch, cplan, img, atdct16.U8)
    y = O.forward_int(img)
    assert np.array_equal(got, layout(cplan, y))
    back = run_inverse(torch, cplan, got, *shape, atdct16.U8)
    assert np.array_equal(back, img)


# ----------------------------------------------------------- 1-D transforms ---
@pytest.mark.parametrize("count", [1, 31, 33, 1000])
def test_forward_inverse_1d(torch, cplan, count):
    rng = np.random.default_rng(count)
    for dtype, odt, tdt in ((atdct16.U8, np.uint8, torch.uint8), (atdct16.I16, np.int16, torch.int16)):
        info = np.iinfo(odt)
        x = rng.integers(info.min, info.max + 1, size=(count, 16)).astype(odt)
        x[0] = info.max
        xd = torch.from_numpy(x).cuda()
        coef = torch.full((count * 16,), -7, dtype=torch.int32, device="cuda")
        cplan.forward_1d(xd, coef, dtype=dtype)
        back = torch.full((count, 16), 5, dtype=tdt, device="cuda")
        cplan.inverse_1d(coef, back, dtype=dtype)
        torch.cuda.synchronize()
        assert np.array_equal(coef.cpu().numpy(), O.forward_1d(x).reshape(-1))
        assert np.array_equal(back.cpu().numpy(), x)


@pytest.mark.parametrize("dtype", [atdct16.U8, atdct16.I16], ids=["u8", "i16"])
def test_inverse_1d_any_int32(torch, cplan, dtype):
    rng = np.random.default_rng(17)
    odt, tdt = (np.uint8, torch.uint8) if dtype == atdct16.U8 else (np.int16, torch.int16)
    y = rng.integers(-5000, 5000, size=(777, 16))
    y[::5] = rng.integers(-(2**31), 2**31, size=y[::5].shape)  # 64-bit route for these lanes
    y[1::7, 0] = 8 * (2 * rng.integers(-40, 40, size=y[1::7, 0].shape) + 1)  # DC ties
    y[1::7, 1:] = 0
    out = torch.full((777, 16), 5, dtype=tdt, device="cuda")
    cplan.inverse_1d(torch.from_numpy(y.astype(np.int32)).cuda(), out, dtype=dtype)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), O.inverse_1d(y, odt))


def test_zero_count_and_bad_arguments(torch, cplan):
    coef = torch.empty(16, dtype=torch.int32, device="cuda")
    x = torch.zeros(16, dtype=torch.uint8, device="cuda")
    cplan.forward_1d(x, coef, count=0)
    cplan.inverse_1d(coef, x, count=0)
    L = atdct16.lib()
    assert L.atdct16_forward_1d(cplan.handle, 0, x.data_ptr(), -1, coef.data_ptr(), None) == atdct16.EINVAL
    assert L.atdct16_forward_1d(cplan.handle, 0, x.data_ptr() + 1, 1, coef.data_ptr(), None) == atdct16.EINVAL
    assert L.atdct16_inverse_1d(cplan.handle, 2, coef.data_ptr(), 1, x.data_ptr(), None) == atdct16.EINVAL
    assert L.atdct16_inverse(cplan.handle, 0, coef.data_ptr(), 16, 16, x.data_ptr(), 24, None) == atdct16.EINVAL
    with pytest.raises(atdct16.Atdct16Error) as e:
        atdct16.Plan(atdct16.U8, max_images=1, flags=2)
    assert e.value.status == atdct16.EINVAL


def test_forward_1d_of_image_rows_is_row_pass(torch, cplan):
    # a packed image is w / 16 vectors per row: one call gives R = X T^T per block row
    img = synth.ar1_image(32, 96, 0.9, 4)
    coef = torch.empty(32 * 96, dtype=torch.int32, device="cuda")
    cplan.forward_1d(dev(torch, img), coef)
    torch.cuda.synchronize()
    ref = O.forward_1d(img.reshape(32, 6, 16))
    assert np.array_equal(coef.cpu().numpy(), ref.reshape(-1))


# ------------------------------------------------- zig-zag quantisation levels ---
@pytest.mark.parametrize("qp", [22, 37])
def test_quant_levels_in_plan_order(torch, qp):
    planes = [synth.laplacian_residual(48, 400, seed=31), synth.laplacian_residual(64, 128, seed=32)]
    for zig in (False, True):
        qplan = atdct16.Plan(atdct16.I16, max_images=4, zigzag=zig)
        srcs = [dev(torch, p) for p in planes]
        dsts = [out_img(torch, *p.shape, torch.int16) for p in planes]
        descs = [atdct16.image(s, d, qp) for s, d in zip(srcs, dsts)]
        levels = torch.full((sum(p.size for p in planes),), -12345, dtype=torch.int16, device="cuda")
        psnr = torch.empty(len(planes), dtype=torch.float64, device="cuda")
        qplan.compress_quant(descs, psnr, levels=levels)
        torch.cuda.synchronize()
        lev = levels.cpu().numpy()
        off = 0
        for p, d in zip(planes, dsts):
            ref = O.compress_quant(p, qp, precision="fp32")
            want = O.to_zigzag(ref["levels"]).reshape(-1) if zig else ref["levels"].reshape(-1)
            assert np.array_equal(lev[off:off + p.size], want)
            off += p.size
            diff = d.cpu().numpy().astype(np.int64) - ref["recon_i16"].astype(np.int64)
            assert np.abs(diff).max() <= 1
        assert qplan.last_device_status() == atdct16.OK
        qplan.close()


# ------------------------------------------------- bounded copy waits ---
def test_inverse_copy_wait_times_out_cleanly(torch):
    """With the stall test hook the inverse announces more bytes than its bulk
    copies deliver: every warp's bounded wait expires, the plan's device
    status reads ETIMEOUT, and the context keeps working."""
    stall = atdct16.Plan(atdct16.U8, max_images=1, flags=atdct16.PLAN_TEST_STALL_COPIES)
    x = synth.ar1_image(16, 256, 0.9, 11)
    y = O.forward_int(x).reshape(-1)
    coef = torch.from_numpy(y.astype(np.int32)).cuda()
    out = out_img(torch, 16, 256, torch.uint8)
    stall.inverse(coef, out, dtype=atdct16.U8)
    assert stall.last_device_status() == atdct16.ETIMEOUT
    stall.close()
    ok = atdct16.Plan(atdct16.U8, max_images=1)
    got = run_inverse(torch, ok, y, 16, 256, atdct16.U8)
    assert np.array_equal(got, x)
    assert ok.last_device_status() == atdct16.OK
    ok.close()


def test_unknown_plan_flags_rejected(torch):
    with pytest.raises(atdct16.Atdct16Error) as e:
        atdct16.Plan(atdct16.U8, max_images=1, flags=0x20000000)
    assert e.value.status == atdct16.EINVAL

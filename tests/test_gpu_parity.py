"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (written per test):
  FP64 storage: max-abs <= 1e-10 after whole solves, 1e-12 after one step.
  FP32 storage: max-abs <= 2e-4 on [0, 1] intensities and PSNR difference
  <= 0.01 dB after whole solves; 2e-5 after one step (float rounding of
  |tau P u| <= tau * 32 * max|u|).
"""
import math

import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - the marker deselects these on CPU
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2006_10406_gb300 as fg  # noqa: E402

DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module", autouse=True)
def _threads():
    O.set_threads(max(1, min(16, __import__("os").cpu_count() or 1)))
    yield


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def _psnr(u, ref):
    mse = float(np.mean((u - ref) ** 2))
    return math.inf if mse == 0 else 10 * math.log10(1.0 / mse)


METHODS = [(0, "foeed"), (1, "eed")]


# --------------------------------------------------------------------------
# single steps, ragged sizes, every Gaussian radius

@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("shape", [(37, 53), (1, 7), (6, 1), (2, 2), (64, 64), (67, 130), (17, 200)])
@pytest.mark.parametrize("sigma", [0.0, 0.5, 1.0, 1.5, 2.0])
def test_step_f64_matches_oracle(method, shape, sigma):
    rng = _rng(hash((method, shape, sigma)) % 2 ** 32)
    h, w = shape
    ucur = rng.uniform(size=shape)
    uprev = ucur + 0.01 * rng.normal(size=shape)
    mask = (rng.uniform(size=shape) < 0.1).astype(np.uint8)
    alpha, tau, lam = 1.37, (0.05 if method == 0 else 0.25), 0.07
    ref = O.fsi_step(method, uprev, ucur, mask, alpha, tau, sigma, lam)
    a, b, m = _dev(uprev, torch.float64), _dev(ucur, torch.float64), _dev(mask, torch.uint8)
    out = torch.full_like(b, float("nan"))
    (fg.foeed_step if method == 0 else fg.eed_step)(a, b, out, m, alpha, lam, sigma, tau=tau)
    got = out.cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
    k = mask != 0
    np.testing.assert_array_equal(got[k], ucur[k])


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("shape", [(37, 53), (64, 64), (67, 130), (3, 300)])
@pytest.mark.parametrize("sigma", [1.0, 1.5])
def test_step_f32_matches_oracle(method, shape, sigma):
    rng = _rng(7 + method)
    ucur = rng.uniform(size=shape).astype(np.float32).astype(np.float64)
    uprev = (ucur + 0.01 * rng.normal(size=shape)).astype(np.float32).astype(np.float64)
    mask = (rng.uniform(size=shape) < 0.1).astype(np.uint8)
    alpha, tau, lam = 1.2, (0.05 if method == 0 else 0.25), 0.05
    ref = O.fsi_step(method, uprev, ucur, mask, alpha, tau, sigma, lam)
    a, b, m = _dev(uprev, torch.float32), _dev(ucur, torch.float32), _dev(mask, torch.uint8)
    out = torch.empty_like(b)
    (fg.foeed_step if method == 0 else fg.eed_step)(a, b, out, m, alpha, lam, sigma, tau=tau)
    got = out.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-5)


@pytest.mark.parametrize("g_kind", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("mu3", [0, 1, 2])
def test_step_variants_f64(g_kind, mu3):
    rng = _rng(100 + 3 * g_kind + mu3)
    shape = (33, 41)
    ucur = rng.uniform(size=shape)
    mask = (rng.uniform(size=shape) < 0.1).astype(np.uint8)
    lam = 0.3 if g_kind in (3, 4) else 0.05
    ref = O.fsi_step(0, ucur, ucur, mask, 2.0 / 3.0, 0.01, 1.0, lam, g_kind, mu3)
    b, m = _dev(ucur, torch.float64), _dev(mask, torch.uint8)
    out = torch.empty_like(b)
    fg.foeed_step(b, b, out, m, 2.0 / 3.0, lam, 1.0, tau=0.01, diffusivity=g_kind, mu3_mode=mu3)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=1e-12)


def test_step_without_mask_and_pitched_rows():
    rng = _rng(9)
    h, w, pitch = 40, 45, 64
    base = torch.zeros((h, pitch), dtype=torch.float64, device=DEV)
    u = base[:, :w]
    un = torch.zeros((h, pitch), dtype=torch.float64, device=DEV)[:, :w]
    uc = rng.uniform(size=(h, w))
    u.copy_(torch.from_numpy(uc))
    fg.foeed_step(u, u, un, None, 1.0, 0.05, 1.0, tau=0.05)
    ref = O.fsi_step(0, uc, uc, None, 1.0, 0.05, 1.0, 0.05)
    np.testing.assert_allclose(un.cpu().numpy(), ref, rtol=0, atol=1e-12)


# --------------------------------------------------------------------------
# whole solves

@pytest.mark.parametrize("method", [0, 1])
def test_inpaint_workload1_f64(method):
    """64x64 FP64, 40 cycles of length 20: max-abs <= 1e-10 against the oracle."""
    img, mask, p = synth.workload(1)
    ref, st, info = O.inpaint(method, img, mask, p["sigma"], p["lam"], p["cycle_len"], p["max_cycles"])
    u, rep = (fg.foeed_inpaint if method == 0 else fg.eed_inpaint)(
        _dev(img, torch.float64), _dev(mask, torch.uint8), p["lam"], p["sigma"], p["cycle_len"], p["max_cycles"])
    got = u.cpu().numpy()
    assert rep.cycles_run == p["max_cycles"]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10)
    assert abs(rep.last_rel_change - info["rel_change"]) <= 1e-8 * max(info["rel_change"], 1e-300) + 1e-14
    k = mask != 0
    np.testing.assert_array_equal(got[k], img[k])


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("dtype", ["f32", "f32_f64u"])
def test_inpaint_workload1_f32(method, dtype):
    """Same solve in FP32 storage: max-abs <= 2e-4, PSNR within 0.01 dB of the oracle's.
    With the two-float FSI update (f32_f64u) the error is that of the FP32 stencils
    alone: max-abs <= 2e-6 against the oracle run on the same FP32-rounded input."""
    img, mask, p = synth.workload(1)
    ref, st, info = O.inpaint(method, img, mask, p["sigma"], p["lam"], p["cycle_len"], p["max_cycles"])
    f32 = img.astype(np.float32)
    u, rep = (fg.foeed_inpaint if method == 0 else fg.eed_inpaint)(
        _dev(f32, torch.float32), _dev(mask, torch.uint8), p["lam"], p["sigma"], p["cycle_len"], p["max_cycles"],
        dtype=dtype)
    got = u.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 2e-4
    if dtype == "f32_f64u":
        ref32, _, _ = O.inpaint(method, f32.astype(np.float64), mask, p["sigma"], p["lam"], p["cycle_len"],
                                p["max_cycles"])
        assert np.max(np.abs(got - ref32)) <= 2e-6
    assert abs(_psnr(got, img) - _psnr(ref, img)) <= 0.01
    k = mask != 0
    np.testing.assert_array_equal(u.cpu().numpy()[k], f32[k])


@pytest.mark.parametrize("method", [0, 1])
def test_inpaint_tol_stops_at_the_oracle_cycle(method):
    """tol > 0: the device stop flag ends the solve at the same cycle as the oracle."""
    img, mask, p = synth.workload(2, h=48, w=40)
    tol = 1e-5
    ref, st, info = O.inpaint(method, img, mask, 1.0, 0.03, 10, 3000, tol=tol)
    assert st == 0 and info["converged"]
    for every in (1, 3, 8):
        u, rep = (fg.foeed_inpaint if method == 0 else fg.eed_inpaint)(
            _dev(img, torch.float64), _dev(mask, torch.uint8), 0.03, 1.0, 10, 3000, tol=tol, check_every=every)
        assert rep.converged and rep.cycles_run == info["cycles"]
        np.testing.assert_allclose(u.cpu().numpy(), ref, rtol=0, atol=1e-10)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_inpaint_short_cycles_f64(n):
    """Cycle lengths 1..4 exercise every buffer-rotation case of the cycle graph."""
    img, mask, p = synth.workload(1, h=29, w=31)
    for method in (0, 1):
        ref, _, _ = O.inpaint(method, img, mask, 1.0, 0.05, n, 5)
        u, rep = (fg.foeed_inpaint if method == 0 else fg.eed_inpaint)(
            _dev(img, torch.float64), _dev(mask, torch.uint8), 0.05, 1.0, n, 5)
        assert rep.cycles_run == 5
        np.testing.assert_allclose(u.cpu().numpy(), ref, rtol=0, atol=1e-11)


@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (7, 1), (2, 3), (65, 33)])
def test_inpaint_tiny_and_ragged_images(shape):
    rng = _rng(11)
    img = rng.uniform(size=shape)
    mask = (rng.uniform(size=shape) < 0.3).astype(np.uint8)
    mask.flat[0] = 1
    for method in (0, 1):
        ref, _, _ = O.inpaint(method, img, mask, 1.0, 0.1, 5, 4)
        u, _ = (fg.foeed_inpaint if method == 0 else fg.eed_inpaint)(
            _dev(img, torch.float64), _dev(mask, torch.uint8), 0.1, 1.0, 5, 4)
        np.testing.assert_allclose(u.cpu().numpy(), ref, rtol=0, atol=1e-11)


def _guarded_solve(method, img, mask, dtype, pitch, lam, sigma, n, cycles):
    """A solve through the C ABI on banded buffers; returns (result, bands intact)."""
    import ctypes as C
    h, w = img.shape
    code = fg.F64 if dtype == torch.float64 else fg.F32
    (f, fb), (m, mb) = _guarded(img, pitch, dtype), _guarded(mask, pitch, torch.uint8)
    u, ub = _guarded(np.zeros_like(img), pitch, dtype)
    ws = torch.empty(fg.workspace_bytes(w, h, code), dtype=torch.uint8, device=DEV)
    p = fg._params(lam, sigma, 0.0, n, cycles)
    rep = fg._Report()
    fn = fg.lib().foeed_inpaint if method == 0 else fg.lib().eed_inpaint
    st = fn(C.c_void_p(f.data_ptr()), C.c_void_p(m.data_ptr()), C.c_void_p(u.data_ptr()), w, h, pitch, code,
            C.byref(p), C.c_void_p(ws.data_ptr()), ws.numel(), C.c_void_p(torch.cuda.current_stream().cuda_stream),
            C.byref(rep))
    assert st == 0, fg.lib().foeed_last_error()
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64), all(_band_intact(x, w) for x in (fb, mb, ub))


@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (33, 70), (130, 67), (97, 300)])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_ragged_solves_stay_inside_their_rows(shape, dtype):
    """Whole solves on buffers with a guard band: the band is untouched and the
    result matches the oracle (pitch a multiple of 4 and an odd pitch)."""
    rng = _rng(13)
    img = rng.uniform(size=shape)
    if dtype == torch.float32:
        img = img.astype(np.float32).astype(np.float64)
    mask = (rng.uniform(size=shape) < 0.1).astype(np.uint8)
    mask.flat[0] = 1
    h, w = shape
    for method in (0, 1):
        ref, _, _ = O.inpaint(method, img, mask, 1.0, 0.05, 6, 3)
        for pitch in (((w + 3) // 4) * 4 + 8, w + 3):
            got, intact = _guarded_solve(method, img, mask, dtype, pitch, 0.05, 1.0, 6, 3)
            assert intact, (method, pitch)
            np.testing.assert_allclose(got, ref, rtol=0, atol=1e-11 if dtype == torch.float64 else 2e-4)


def test_inpaint_edge_masks():
    rng = _rng(12)
    img = rng.uniform(size=(20, 24))
    # every pixel known: the result is f
    full = np.ones(img.shape, np.uint8)
    u, _ = fg.foeed_inpaint(_dev(img, torch.float64), _dev(full, torch.uint8), 0.05, 1.0, 4, 2)
    np.testing.assert_array_equal(u.cpu().numpy(), img)
    # no known pixel and init from the mean of an empty set: the zero image stays zero
    empty = np.zeros(img.shape, np.uint8)
    u, _ = fg.foeed_inpaint(_dev(img, torch.float64), _dev(empty, torch.uint8), 0.05, 1.0, 4, 2)
    assert np.all(u.cpu().numpy() == 0.0)
    # no known pixel, start from u0: the smoothing variant conserves the mean (symmetric P)
    u, _ = fg.foeed_inpaint(_dev(img, torch.float64), _dev(empty, torch.uint8), 0.05, 1.0, 10, 5, u0=_dev(img, torch.float64))
    assert abs(u.cpu().numpy().sum() - img.sum()) < 1e-10


def test_constant_image_fixed_bitwise_f32():
    c = np.full((50, 70), 0.3, np.float32)
    mask = np.zeros(c.shape, np.uint8); mask[5, 5] = 1
    for m in (0, 1):
        u, _ = (fg.foeed_inpaint if m == 0 else fg.eed_inpaint)(_dev(c, torch.float32), _dev(mask, torch.uint8),
                                                               0.05, 1.0, 10, 3)
        assert np.all(u.cpu().numpy() == np.float32(0.3))


def test_host_inputs_round_trip():
    img, mask, p = synth.workload(1, h=32, w=32)
    u, rep = fg.foeed_inpaint(img, mask, 0.05, 1.0, 5, 2)
    assert isinstance(u, torch.Tensor) and not u.is_cuda and u.dtype == torch.float64
    ref, _, _ = O.inpaint(0, img, mask, 1.0, 0.05, 5, 2)
    np.testing.assert_allclose(u.numpy(), ref, rtol=0, atol=1e-11)


def test_divergence_and_argument_errors():
    rng = _rng(13)
    img = rng.uniform(size=(16, 16))
    empty = np.zeros(img.shape, np.uint8)
    u, rep = fg.foeed_inpaint(_dev(img, torch.float64), _dev(empty, torch.uint8), 1e30, 1.0, 1, 400, tau=0.5,
                              u0=_dev(img, torch.float64), raise_on_status=False)
    assert rep.status == 4
    with pytest.raises(fg.FoeedError):
        fg.foeed_inpaint(_dev(img, torch.float64), _dev(empty, torch.uint8), -1.0, 1.0, 1, 1)
    with pytest.raises(fg.FoeedError):
        fg.foeed_inpaint(_dev(img, torch.float64), _dev(empty, torch.uint8), 0.1, 2.5, 1, 1)
    b = _dev(img, torch.float64)
    with pytest.raises(fg.FoeedError):
        fg.foeed_step(b, b, b, None, 1.0, 0.1, 1.0)


def test_errors_metric():
    rng = _rng(14)
    a = rng.uniform(size=(31, 45)); b = rng.uniform(size=(31, 45))
    mse, aae, psnr = fg.foeed_errors(_dev(a, torch.float64), _dev(b, torch.float64))
    rm, ra = O.errors(a, b)
    assert abs(mse - rm) < 1e-14 and abs(aae - ra) < 1e-14
    assert abs(psnr - 10 * math.log10(1 / rm)) < 1e-10


# --------------------------------------------------------------------------
# full sizes, in the launch configuration the benchmark times

@pytest.mark.parametrize("method", [0, 1])
def test_fullsize_2048_one_cycle_f32_vs_oracle(method):
    """2048 x 2048 phantom, sigma 1.5 (R = 5), one FSI cycle of length 40, every pixel."""
    img, mask, p = synth.workload(3)
    f32 = img.astype(np.float32)
    ref, _, _ = O.inpaint(method, f32.astype(np.float64), mask, p["sigma"], p["lam"], p["cycle_len"], 1)
    u, rep = (fg.foeed_inpaint if method == 0 else fg.eed_inpaint)(
        _dev(f32, torch.float32), _dev(mask, torch.uint8), p["lam"], p["sigma"], p["cycle_len"], 1)
    got = u.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 2e-4


def test_fullsize_2048_bench_solve_against_the_oracle():
    """The benchmarked solve itself (2048 x 2048 phantom, sigma 1.5, lambda 0.02, 100
    FSI cycles of 40 = 4000 steps) against the FP64 oracle run to the same iterate:
    FP32 within 2e-4 and 0.01 dB of PSNR, FP32 storage with the two-float FSI
    update within 2e-6, the FP64 GPU solve within 1e-10; Dirichlet pixels bitwise f. The oracle
    takes about three minutes on 16 host cores."""
    img, mask, p = synth.workload(3)
    f32 = img.astype(np.float32)
    f64 = f32.astype(np.float64)
    n, cycles = p["cycle_len"], p["max_cycles"]
    ref, st, info = O.inpaint(0, f64, mask, p["sigma"], p["lam"], n, cycles)
    assert st == 0 and info["cycles"] == cycles
    u32, r32 = fg.foeed_inpaint(_dev(f32, torch.float32), _dev(mask, torch.uint8), p["lam"], p["sigma"], n, cycles)
    umx, rmx = fg.foeed_inpaint(_dev(f32, torch.float32), _dev(mask, torch.uint8), p["lam"], p["sigma"], n, cycles,
                                dtype="f32_f64u")
    u64, r64 = fg.foeed_inpaint(_dev(f64, torch.float64), _dev(mask, torch.uint8), p["lam"], p["sigma"], n, cycles)
    assert r32.cycles_run == rmx.cycles_run == r64.cycles_run == cycles
    a = u32.cpu().numpy().astype(np.float64)
    k = mask != 0
    np.testing.assert_array_equal(a[k], f64[k])
    assert np.isfinite(a).all()
    assert np.max(np.abs(a - ref)) <= 2e-4
    assert abs(_psnr(a, img) - _psnr(ref, img)) <= 0.01
    assert np.max(np.abs(umx.cpu().numpy().astype(np.float64) - ref)) <= 2e-6
    assert np.max(np.abs(u64.cpu().numpy() - ref)) <= 1e-10


@pytest.mark.parametrize("method", [0, 1])
def test_512_tolerance_run_stops_with_the_oracle(method):
    """The 512 x 512 polygon workload run until the relative change of a cycle falls
    below 1e-6 (Sec. 3.3 stop test). FP64: the solve stops at the oracle's cycle and
    matches its result. FP32: the relative change is measured on FP32 iterates, whose
    rounding adds about 1e-7 to it, so near tol the stop can come some cycles later
    (measured: cycle 131 against 123); the FP32 result then matches the oracle's
    iterate after the same number of cycles within 2e-4 and 0.01 dB, and that
    cycle is a valid stop of the exact iteration (its FP64 change is below tol, or within 2% of it one cycle early)."""
    img, mask, p = synth.workload(2)
    f64 = img.astype(np.float32).astype(np.float64)
    n, tol, cap = p["cycle_len"], p["tol"], p["max_cycles"]
    solve = fg.foeed_inpaint if method == 0 else fg.eed_inpaint
    ref, st, info = O.inpaint(method, f64, mask, p["sigma"], p["lam"], n, cap, tol=tol)
    assert st == 0 and info["converged"]
    u64, rep64 = solve(_dev(f64, torch.float64), _dev(mask, torch.uint8), p["lam"], p["sigma"], n, cap, tol=tol)
    assert rep64.converged and rep64.cycles_run == info["cycles"]
    np.testing.assert_allclose(u64.cpu().numpy(), ref, rtol=0, atol=1e-10)
    u32, rep32 = solve(_dev(f64, torch.float32), _dev(mask, torch.uint8), p["lam"], p["sigma"], n, cap, tol=tol)
    assert rep32.converged and rep32.last_rel_change < tol
    assert info["cycles"] - 1 <= rep32.cycles_run <= info["cycles"] + 20, (rep32.cycles_run, info["cycles"])
    ref32, st32, info32 = O.inpaint(method, f64, mask, p["sigma"], p["lam"], n, rep32.cycles_run)
    assert st32 == 0 and info32["rel_change"] < tol * 1.02
    got = u32.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref32)) <= 2e-4
    assert abs(_psnr(got, img) - _psnr(ref32, img)) <= 0.01


# --------------------------------------------------------------------------
# the register-blocked FP32 kernel (pitch % 4 == 0, Charbonnier) and the
# generic one (any pitch, every diffusivity / mu3) must agree with the oracle

def _pitched(a, pitch, dtype):
    h, w = a.shape
    buf = torch.zeros((h, pitch), dtype=dtype, device=DEV)
    buf[:, :w] = torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)
    return buf[:, :w]


# Guard bands (compute-sanitizer is not available to these runs): every image lives
# in a buffer with one extra row above and below and pitch - w padding columns, all
# filled with a sentinel (NaN for images, 0xA5 for masks). A kernel that wrote
# outside the image would change the band; one that read from it would pull a NaN
# into the result, which the oracle comparison would catch.
def _guarded(a, pitch, dtype):
    """(view of the image inside the band, the whole banded buffer). The band above
    the image has as many rows as keep the view 16-byte aligned (the register-blocked
    kernel needs aligned rows), at least one; the band below has one row."""
    h, w = a.shape
    esize = torch.tensor([], dtype=dtype).element_size()
    top = 16 // math.gcd(pitch * esize, 16)
    fill = 0xA5 if dtype == torch.uint8 else float("nan")
    buf = torch.full((top + h + 1, pitch), fill, dtype=dtype, device=DEV)
    buf[top:top + h, :w] = torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)
    return buf[top:top + h, :w], (buf, top, h)


def _band_intact(banded, w):
    """True if the band of a buffer made by _guarded still holds its sentinel."""
    buf, top, h = banded
    band = torch.cat([buf[:top].reshape(-1), buf[top + h:].reshape(-1), buf[top:top + h, w:].reshape(-1)])
    if buf.dtype == torch.uint8:
        return bool((band == 0xA5).all().item())
    return bool(torch.isnan(band).all().item())


@pytest.mark.parametrize("method", [0, 1])
# the small shapes run the fast kernel on 64 x 16 tiles; 630 x 1030 (340 tiles of
# 64 x 32, ragged in both directions) on 64 x 32 tiles
@pytest.mark.parametrize("shape", [(100, 130), (33, 70), (64, 64), (5, 300), (130, 7), (630, 1030)])
@pytest.mark.parametrize("sigma", [0.5, 1.0, 1.5, 2.0])
def test_fast_and_generic_f32_paths_match_oracle(method, shape, sigma):
    rng = _rng(200 + method)
    h, w = shape
    ucur = rng.uniform(size=shape).astype(np.float32).astype(np.float64)
    uprev = (ucur + 0.01 * rng.normal(size=shape)).astype(np.float32).astype(np.float64)
    mask = (rng.uniform(size=shape) < 0.08).astype(np.uint8)
    alpha, tau, lam = 1.5, (0.05 if method == 0 else 0.25), 0.03
    ref = O.fsi_step(method, uprev, ucur, mask, alpha, tau, sigma, lam)
    outs = []
    # a pitch that is a multiple of 4 runs the register-blocked kernel, an odd one the generic kernel
    for pitch in (((w + 3) // 4) * 4 + 4, w + 1 if (w + 1) % 4 else w + 2):
        (a, ab), (b, bb) = _guarded(uprev, pitch, torch.float32), _guarded(ucur, pitch, torch.float32)
        m, mb = _guarded(mask, pitch, torch.uint8)
        out, ob = _guarded(np.zeros(shape), pitch, torch.float32)
        (fg.foeed_step if method == 0 else fg.eed_step)(a, b, out, m, alpha, lam, sigma, tau=tau)
        assert all(_band_intact(x, w) for x in (ab, bb, mb, ob)), pitch
        outs.append(out.cpu().numpy().astype(np.float64))
    for got in outs:
        np.testing.assert_allclose(got, ref, rtol=0, atol=2e-5)
        np.testing.assert_array_equal(got[mask != 0], ucur[mask != 0])


@pytest.mark.parametrize("policy", ["h8", "h16", "h32", "h64"])
@pytest.mark.parametrize("shape", [(100, 130), (630, 1030), (70, 64), (130, 200)])
def test_fast_step_each_tile_shape_matches_oracle(policy, shape):
    """One FOEED step on each fixed tile shape (64 x 8 tiles with 128 threads,
    64 x 16, 64 x 32, 64 x 64 tiles with 512 threads), ragged in both directions,
    inside a guard band."""
    rng = _rng(400)
    h, w = shape
    ucur = rng.uniform(size=shape).astype(np.float32).astype(np.float64)
    uprev = (ucur + 0.01 * rng.normal(size=shape)).astype(np.float32).astype(np.float64)
    mask = (rng.uniform(size=shape) < 0.08).astype(np.uint8)
    ref = O.fsi_step(0, uprev, ucur, mask, 1.5, 0.05, 1.5, 0.03)
    pitch = ((w + 3) // 4) * 4 + 4
    (a, ab), (b, bb) = _guarded(uprev, pitch, torch.float32), _guarded(ucur, pitch, torch.float32)
    m, mb = _guarded(mask, pitch, torch.uint8)
    out, ob = _guarded(np.zeros(shape), pitch, torch.float32)
    try:
        fg.set_tile_policy(policy)
        fg.foeed_step(a, b, out, m, 1.5, 0.03, 1.5, tau=0.05)
        torch.cuda.synchronize()
    finally:
        fg.set_tile_policy("auto")
    assert all(_band_intact(x, w) for x in (ab, bb, mb, ob))
    got = out.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-5)
    np.testing.assert_array_equal(got[mask != 0], ucur[mask != 0])


@pytest.mark.parametrize("policy", ["h8", "h64"])
@pytest.mark.parametrize("sigma", [0.0, 0.5, 1.0, 1.5, 2.0])
def test_fast_step_small_and_large_tiles_every_radius(policy, sigma):
    """The FOEED-only tile shapes (64 x 8 with 128 threads, 64 x 64 with 512) at
    every Gaussian radius R = 0 .. 6, where the window's copy passes and the
    x pass's taps change, ragged in both directions, inside a guard band; the
    result equals the default shape's bitwise."""
    rng = _rng(420)
    shape = (75, 150)
    h, w = shape
    ucur = rng.uniform(size=shape).astype(np.float32).astype(np.float64)
    uprev = (ucur + 0.01 * rng.normal(size=shape)).astype(np.float32).astype(np.float64)
    mask = (rng.uniform(size=shape) < 0.08).astype(np.uint8)
    ref = O.fsi_step(0, uprev, ucur, mask, 1.5, 0.05, sigma, 0.03)
    pitch = ((w + 3) // 4) * 4 + 4
    outs = []
    for pol in ("auto", policy):
        (a, ab), (b, bb) = _guarded(uprev, pitch, torch.float32), _guarded(ucur, pitch, torch.float32)
        m, mb = _guarded(mask, pitch, torch.uint8)
        out, ob = _guarded(np.zeros(shape), pitch, torch.float32)
        try:
            fg.set_tile_policy(pol)
            fg.foeed_step(a, b, out, m, 1.5, 0.03, sigma, tau=0.05)
            torch.cuda.synchronize()
        finally:
            fg.set_tile_policy("auto")
        assert all(_band_intact(x, w) for x in (ab, bb, mb, ob)), pol
        outs.append(out.cpu().numpy())
    np.testing.assert_allclose(outs[1].astype(np.float64), ref, rtol=0, atol=2e-5)
    np.testing.assert_array_equal(outs[1], outs[0])


@pytest.mark.parametrize("shape", [(100, 130), (630, 1030)])
def test_eed_step_under_each_tile_policy(shape):
    """One EED step under every fixed tile policy (64 x 64 and 64 x 8 tiles exist
    for FOEED only: EED takes 64 x 32 under h64 and 64 x 16 under h8): each matches
    the oracle inside a guard band, and all give the same bits."""
    rng = _rng(410)
    h, w = shape
    ucur = rng.uniform(size=shape).astype(np.float32).astype(np.float64)
    uprev = (ucur + 0.01 * rng.normal(size=shape)).astype(np.float32).astype(np.float64)
    mask = (rng.uniform(size=shape) < 0.08).astype(np.uint8)
    ref = O.fsi_step(1, uprev, ucur, mask, 1.5, 0.25, 1.5, 0.03)
    pitch = ((w + 3) // 4) * 4 + 4
    outs = []
    for policy in ("auto", "h8", "h16", "h32", "h64"):
        (a, ab), (b, bb) = _guarded(uprev, pitch, torch.float32), _guarded(ucur, pitch, torch.float32)
        m, mb = _guarded(mask, pitch, torch.uint8)
        out, ob = _guarded(np.zeros(shape), pitch, torch.float32)
        try:
            fg.set_tile_policy(policy)
            fg.eed_step(a, b, out, m, 1.5, 0.03, 1.5, tau=0.25)
            torch.cuda.synchronize()
        finally:
            fg.set_tile_policy("auto")
        assert all(_band_intact(x, w) for x in (ab, bb, mb, ob)), policy
        outs.append(out.cpu().numpy())
    np.testing.assert_allclose(outs[0].astype(np.float64), ref, rtol=0, atol=2e-5)
    np.testing.assert_array_equal(outs[0][mask != 0], ucur[mask != 0])
    for got in outs[1:]:
        np.testing.assert_array_equal(got, outs[0])


@pytest.mark.parametrize("g_kind,mu3", [(1, 0), (2, 1), (0, 2), (0, 1)])
def test_generic_f32_variants(g_kind, mu3):
    rng = _rng(300 + g_kind)
    shape = (48, 64)
    ucur = rng.uniform(size=shape).astype(np.float32).astype(np.float64)
    mask = (rng.uniform(size=shape) < 0.1).astype(np.uint8)
    ref = O.fsi_step(0, ucur, ucur, mask, 2.0 / 3.0, 0.05, 1.0, 0.05, g_kind, mu3)
    b, m = _dev(ucur, torch.float32), _dev(mask, torch.uint8)
    out = torch.empty_like(b)
    fg.foeed_step(b, b, out, m, 2.0 / 3.0, 0.05, 1.0, tau=0.05, diffusivity=g_kind, mu3_mode=mu3)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=2e-5)


# --------------------------------------------------------------------------
# batched solve: many images of uneven sizes in one launch per FSI step;
# each result must equal the single-image solve bit for bit

def _batch_case(seed=0, sizes=((64, 64), (96, 130), (33, 200), (128, 64), (7, 9), (250, 41))):
    imgs, masks, lams = [], [], []
    for i, (h, w) in enumerate(sizes):
        img, mask, _ = synth.workload(2, h=h, w=w, instance=seed + i)
        imgs.append(torch.from_numpy(img.astype(np.float32)).to(DEV))
        masks.append(torch.from_numpy(mask).to(DEV))
        lams.append(0.01 + 0.015 * i)
    return imgs, masks, lams


# --------------------------------------------------------------------------
# the tile-shape autotuner: every policy gives bitwise the same results

@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("shape", [(512, 512), (630, 1030), (96, 2100)])
def test_autotuned_solve_equals_each_fixed_tile_shape(method, shape):
    img, mask, p = synth.workload(2, h=shape[0], w=shape[1], instance=7)
    f, m = _dev(img, torch.float32), _dev(mask, torch.uint8)
    solve = fg.foeed_inpaint if method == 0 else fg.eed_inpaint
    lam, sigma = 0.03, 1.0
    try:
        fg.set_tile_policy("auto")
        ua, _ = solve(f, m, lam, sigma, 8, 3)
        plan = fg.last_tile_plan()
        assert plan["images"] == 1 and plan["tile_h"] in ((8, 16, 32, 64) if method == 0 else (16, 32))
        if plan["tuned"]:
            times = {32: plan["us_h32"], 16: plan["us_h16"]}
            if method == 0:  # 64 x 64 and 64 x 8 tiles are FOEED candidates only
                times[64] = plan["us_h64"]
                times[8] = plan["us_h8"]
            assert all(t > 0 for t in times.values())
            assert plan["us_chosen"] == min(times.values()) == times[plan["tile_h"]]
        ua2, _ = solve(f, m, lam, sigma, 8, 3)
        again = fg.last_tile_plan()
        assert again["tuned"] == 0 and again["tile_h"] == plan["tile_h"]  # the choice is cached
        assert torch.equal(ua, ua2)
        for pol, th in (("h32", 32), ("h16", 16), ("h64", 64 if method == 0 else 32),
                        ("h8", 8 if method == 0 else 16)):
            fg.set_tile_policy(pol)
            u, _ = solve(f, m, lam, sigma, 8, 3)
            assert fg.last_tile_plan()["tile_h"] == th
            assert torch.equal(u, ua), pol
    finally:
        fg.set_tile_policy("auto")


@pytest.mark.parametrize("method", ["foeed", "eed"])
def test_autotuned_batch_equals_each_fixed_tile_plan(method):
    cases = synth.batched_workload(14, sides=(128, 256, 384, 640))
    imgs = [_dev(c[0], torch.float32) for c in cases]
    masks = [_dev(c[1], torch.uint8) for c in cases]
    lams = [float(c[2]) for c in cases]
    solve = fg.foeed_inpaint_batch if method == "foeed" else fg.eed_inpaint_batch
    try:
        fg.set_tile_policy("auto")
        ua, _ = solve(imgs, masks, lams, 1.0, 6, 3)
        plan = fg.last_tile_plan()
        assert plan["images"] == len(imgs) and 0 <= plan["images_h16"] <= len(imgs)
        if plan["tuned"]:
            assert 0 < plan["us_chosen"] <= min(plan["us_h32"], plan["us_h16"])
        for pol, nh16 in (("h32", 0), ("h16", len(imgs)), ("h8", len(imgs)), ("h64", 0)):
            fg.set_tile_policy(pol)
            u, _ = solve(imgs, masks, lams, 1.0, 6, 3)
            assert fg.last_tile_plan()["images_h16"] == nh16
            for a, b in zip(u, ua):
                assert torch.equal(a, b), pol
    finally:
        fg.set_tile_policy("auto")


@pytest.mark.parametrize("n", [2, 3, 25])
@pytest.mark.parametrize("dtype", ["f32", "f32_f64u"])
def test_batch_equals_single_image_solves(n, dtype):
    imgs, masks, lams = _batch_case()
    outs, reps = fg.foeed_inpaint_batch(imgs, masks, lams, 1.0, n, 4, dtype=dtype)
    for f, m, lam, u, r in zip(imgs, masks, lams, outs, reps):
        ref, rr = fg.foeed_inpaint(f, m, lam, 1.0, n, 4, dtype=dtype)
        assert r.cycles_run == rr.cycles_run == 4
        assert torch.equal(u, ref), float((u - ref).abs().max())
        # the images are bitwise equal; the residual is an FP64 sum over tiles, and a small
        # single image runs on 64 x 16 tiles where the batch uses 64 x 32
        assert r.last_rel_change == pytest.approx(rr.last_rel_change, rel=1e-12, abs=0)


def test_batch_matches_oracle_and_keeps_known_pixels():
    imgs, masks, lams = _batch_case(seed=50, sizes=((40, 56), (23, 31)))
    outs, _ = fg.foeed_inpaint_batch(imgs, masks, lams, 1.0, 10, 3)
    for f, m, lam, u in zip(imgs, masks, lams, outs):
        f64 = f.double().cpu().numpy()
        ref, _, _ = O.inpaint(0, f64, m.cpu().numpy(), 1.0, lam, 10, 3)
        got = u.double().cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 2e-4
        k = m.cpu().numpy() != 0
        np.testing.assert_array_equal(u.cpu().numpy()[k], f.cpu().numpy()[k])


def test_batch_tolerance_stops_each_image_like_its_single_solve():
    imgs, masks, lams = _batch_case(seed=70, sizes=((48, 40), (32, 96), (70, 70)))
    outs, reps = fg.foeed_inpaint_batch(imgs, masks, lams, 1.0, 10, 2000, tol=1e-4, check_every=3)
    for f, m, lam, u, r in zip(imgs, masks, lams, outs, reps):
        ref, rr = fg.foeed_inpaint(f, m, lam, 1.0, 10, 2000, tol=1e-4, check_every=3)
        assert r.converged and rr.converged and r.cycles_run == rr.cycles_run
        assert torch.equal(u, ref)


def test_batch_rejects_unsupported_configurations():
    imgs, masks, lams = _batch_case(sizes=((16, 16),))
    with pytest.raises(fg.FoeedError):
        fg.foeed_inpaint_batch(imgs, masks, lams, 1.0, 1, 2)
    with pytest.raises(fg.FoeedError):
        fg.foeed_inpaint_batch(imgs, masks, [-1.0], 1.0, 4, 2)


@pytest.mark.parametrize("n", [2, 7])
def test_eed_batch_equals_single_image_solves(n):
    imgs, masks, lams = _batch_case(seed=90)
    outs, reps = fg.eed_inpaint_batch(imgs, masks, lams, 1.0, n, 3)
    for f, m, lam, u, r in zip(imgs, masks, lams, outs, reps):
        ref, rr = fg.eed_inpaint(f, m, lam, 1.0, n, 3)
        assert torch.equal(u, ref), float((u - ref).abs().max())
        # the images are bitwise equal; the residual is an FP64 sum over tiles, and a small
        # single image runs on 64 x 16 tiles where the batch uses 64 x 32
        assert r.last_rel_change == pytest.approx(rr.last_rel_change, rel=1e-12, abs=0)


def test_eed_batch_matches_oracle():
    imgs, masks, lams = _batch_case(seed=95, sizes=((40, 56), (23, 31)))
    outs, _ = fg.eed_inpaint_batch(imgs, masks, lams, 1.0, 8, 3)
    for f, m, lam, u in zip(imgs, masks, lams, outs):
        ref, _, _ = O.inpaint(1, f.double().cpu().numpy(), m.cpu().numpy(), 1.0, lam, 8, 3)
        assert np.max(np.abs(u.double().cpu().numpy() - ref)) <= 2e-4


@pytest.mark.parametrize("method", ["foeed", "eed"])
def test_channelwise_colour_reconstruction(method):
    # three channels sharing one mask (Sec. 5, colour images): each channel of
    # the batched result equals that channel solved alone, and the oracle
    img, mask, _ = synth.workload(2, h=45, w=77, instance=7)
    rgb = np.stack([img, 1.0 - img, np.sqrt(img)]).astype(np.float32)
    f = torch.from_numpy(rgb).to(DEV)
    m = torch.from_numpy(mask).to(DEV)
    out, reps = fg.inpaint_channels(f, m, 0.03, 1.0, 6, 3, method=method)
    assert out.shape == f.shape and len(reps) == 3
    single = fg.foeed_inpaint if method == "foeed" else fg.eed_inpaint
    for c in range(3):
        ref, _ = single(f[c].contiguous(), m, 0.03, 1.0, 6, 3)
        assert torch.equal(out[c], ref)
        oref, _, _ = O.inpaint(0 if method == "foeed" else 1, rgb[c].astype(np.float64), mask, 1.0, 0.03, 6, 3)
        assert np.max(np.abs(out[c].double().cpu().numpy() - oref)) <= 2e-4


# --------------------------------------------------------------------------
# the unifying fourth-order operator with caller-supplied coefficients

@pytest.mark.parametrize("shape", [(9, 11), (40, 70), (1, 8), (17, 33)])
def test_apply_tensor_field_matches_oracle(shape):
    rng = _rng(500 + shape[0])
    u = rng.uniform(size=shape)
    d = rng.normal(size=shape + (2, 2, 2, 2))          # arbitrary, not symmetric
    ref = O.apply_P_field(u, d)
    got = fg.foeed_apply_tensor_field(_dev(u, torch.float64), torch.from_numpy(d).to(DEV))
    np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=0, atol=1e-12)
    got32 = fg.foeed_apply_tensor_field(_dev(u, torch.float32), torch.from_numpy(d).to(DEV))
    np.testing.assert_allclose(got32.cpu().numpy(), ref, rtol=0, atol=1e-4 * max(1.0, np.abs(ref).max()))


def test_apply_tensor_field_with_the_foeed_tensor_is_the_foeed_operator():
    u = _rng(501).uniform(size=(30, 41))
    d = O.foeed_tensor_field(u, 1.0, 0.05)
    got = fg.foeed_apply_tensor_field(_dev(u, torch.float64), torch.from_numpy(d).to(DEV))
    np.testing.assert_allclose(got.cpu().numpy(), O.foeed_operator(u, 1.0, 0.05), rtol=0, atol=1e-12)


# --------------------------------------------------------------------------
# host threads: each keeps its own graph cache and capture stream

def test_concurrent_solves_from_two_threads_match_sequential_solves():
    import threading
    img, mask, _ = synth.workload(2, h=64, w=96, instance=3)
    f = torch.from_numpy(img.astype(np.float32)).to(DEV)
    m = torch.from_numpy(mask).to(DEV)
    lams = [0.01 * (i + 1) for i in range(6)]  # six graph keys per thread: the 4-entry caches evict
    ref = {lam: fg.foeed_inpaint(f, m, lam, 1.0, 5, 3)[0].clone() for lam in lams}
    got, errors = {}, []

    def worker(tid):
        try:
            s = torch.cuda.Stream(device=DEV)
            for rep in range(2):
                for lam in (lams if tid == 0 else lams[::-1]):
                    u, _ = fg.foeed_inpaint(f, m, lam, 1.0, 5, 3, stream=s)
                    got[(tid, rep, lam)] = u
            torch.cuda.synchronize(DEV)
        except Exception as e:  # reported below
            errors.append(e)

    ts = [threading.Thread(target=worker, args=(t,)) for t in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors
    assert len(got) == 2 * 2 * len(lams)
    for (tid, rep, lam), u in got.items():
        assert torch.equal(u, ref[lam]), (tid, rep, lam)

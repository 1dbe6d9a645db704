"""GPU adjoint of the FOEED solve (gradient with respect to the stored grey
values) against the FP64 oracle's adjoint, finite differences, and itself
under different checkpoint intervals.

Tolerances: FP64 storage, max |GPU - oracle| <= 1e-9 * max |oracle|;
FP32 storage, <= 2e-3 * max |oracle| (float rounding through hundreds of
forward and backward steps); finite differences (FP64, central) relative 1e-5.
"""
import numpy as np
import pytest

import oracle as O
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2006_10406_gb300 as fg  # noqa: E402

DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module", autouse=True)
def _threads():
    O.set_threads(max(1, min(16, __import__("os").cpu_count() or 1)))
    yield


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _case(h, w, seed, density=0.1):
    rng = _rng(seed)
    img, _, _ = synth.workload(2, h=h, w=w, instance=seed)
    mask = (rng.uniform(size=(h, w)) < density).astype(np.uint8)
    mask.flat[0] = 1
    gu = rng.normal(size=(h, w))
    return img, mask, gu


@pytest.mark.parametrize("shape", [(20, 24), (37, 53), (64, 70), (5, 9)])
@pytest.mark.parametrize("n,cycles", [(1, 3), (2, 2), (5, 3)])
def test_vjp_f64_matches_oracle(shape, n, cycles):
    img, mask, gu = _case(*shape, seed=shape[0] + n)
    ref, uref = O.inpaint_vjp(img, mask, gu, 1.0, 0.05, n, cycles)
    gf, uf = fg.foeed_inpaint_vjp(torch.from_numpy(img).to(DEV), torch.from_numpy(mask).to(DEV),
                                  torch.from_numpy(gu).to(DEV), 0.05, 1.0, n, cycles, checkpoint_every=3)
    np.testing.assert_allclose(uf.cpu().numpy(), uref, rtol=0, atol=1e-11)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(gf.cpu().numpy() - ref)) <= 1e-9 * scale
    assert np.all(gf.cpu().numpy()[mask == 0] == 0.0)


@pytest.mark.parametrize("sigma", [1.0, 1.5])
def test_vjp_f32_matches_oracle(sigma):
    img, mask, gu = _case(48, 64, seed=5)
    f32 = img.astype(np.float32)
    ref, _ = O.inpaint_vjp(f32.astype(np.float64), mask, gu, sigma, 0.03, 10, 3)
    gf, _ = fg.foeed_inpaint_vjp(torch.from_numpy(f32).to(DEV), torch.from_numpy(mask).to(DEV),
                                 torch.from_numpy(gu.astype(np.float32)).to(DEV), 0.03, sigma, 10, 3)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(gf.cpu().numpy().astype(np.float64) - ref)) <= 2e-3 * scale


@pytest.mark.parametrize("h,w", [(96, 224), (97, 226)])
@pytest.mark.parametrize("sigma", [1.0, 1.5])
def test_vjp_f32_interior_tiles_match_oracle(h, w, sigma):
    # wide enough that the FP32 backward kernels' interior tiles (windows copied
    # whole, without mirroring) occur beside border tiles; 97 x 226 adds a ragged
    # last row of tiles and a partial last group of four pixels
    img, mask, gu = _case(h, w, seed=h + w)
    f32 = img.astype(np.float32)
    ref, _ = O.inpaint_vjp(f32.astype(np.float64), mask, gu, sigma, 0.03, 8, 3)
    gf, _ = fg.foeed_inpaint_vjp(torch.from_numpy(f32).to(DEV), torch.from_numpy(mask).to(DEV),
                                 torch.from_numpy(gu.astype(np.float32)).to(DEV), 0.03, sigma, 8, 3)
    g = gf.cpu().numpy().astype(np.float64)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(g - ref)) <= 2e-3 * scale
    assert np.all(g[mask == 0] == 0.0)


def test_checkpoint_interval_does_not_change_the_gradient():
    img, mask, gu = _case(40, 44, seed=6)
    args = (torch.from_numpy(img.astype(np.float32)).to(DEV), torch.from_numpy(mask).to(DEV),
            torch.from_numpy(gu.astype(np.float32)).to(DEV), 0.04, 1.0, 6, 4)
    outs = [fg.foeed_inpaint_vjp(*args, checkpoint_every=k)[0] for k in (1, 4, 16, 1000)]
    for o in outs[1:]:
        assert torch.equal(o, outs[0])


def test_autograd_function_backward_is_the_vjp():
    img, mask, _ = _case(32, 48, seed=7)
    target = torch.from_numpy(img.astype(np.float32)).to(DEV)
    f = (target + 0.05 * torch.randn_like(target)).requires_grad_(True)
    md = torch.from_numpy(mask).to(DEV)
    u = fg.foeed_inpaint_diff(f, md, 0.03, 1.0, 8, 3)
    loss = ((u - target) ** 2).mean()
    loss.backward()
    gu = 2.0 * (u.detach() - target) / u.numel()
    gf, _ = fg.foeed_inpaint_vjp(f.detach(), md, gu, 0.03, 1.0, 8, 3)
    assert torch.equal(f.grad, gf)


def test_vjp_f64_matches_finite_differences():
    img, mask, gu = _case(24, 30, seed=8)
    fd_ = torch.from_numpy(img).to(DEV)
    md = torch.from_numpy(mask).to(DEV)
    gud = torch.from_numpy(gu).to(DEV)
    gf, _ = fg.foeed_inpaint_vjp(fd_, md, gud, 0.05, 1.0, 5, 3)
    rng = _rng(9)
    for _ in range(3):
        delta = torch.from_numpy(rng.normal(size=img.shape) * mask).to(DEV)
        h = 1e-5
        up, _ = fg.foeed_inpaint(fd_ + h * delta, md, 0.05, 1.0, 5, 3)
        um, _ = fg.foeed_inpaint(fd_ - h * delta, md, 0.05, 1.0, 5, 3)
        fdv = float(((up - um) * gud).sum()) / (2 * h)
        got = float((gf * delta).sum())
        assert abs(got - fdv) <= 1e-5 * max(1.0, abs(fdv))


def test_vjp_rejects_unsupported_configurations():
    img, mask, gu = _case(16, 16, seed=10)
    a = (torch.from_numpy(img).to(DEV), torch.from_numpy(mask).to(DEV), torch.from_numpy(gu).to(DEV), 0.05, 1.0, 4, 2)
    with pytest.raises(fg.FoeedError):
        fg.foeed_inpaint_vjp(*a, checkpoint_every=0)


# --------------------------------------------------------------------------
# the tonal-optimisation workload: 1024 x 1024 FP32, 4% mask, 30 cycles of 20

def test_w5_gradient_finite_differences_and_crop_oracle():
    img, mask, p = synth.workload(5)
    n, cycles = p["cycle_len"], p["max_cycles"]
    rng = _rng(11)
    target = torch.from_numpy(img).to(DEV)
    f64 = target.clone()
    md = torch.from_numpy(mask).to(DEV)
    u, _ = fg.foeed_inpaint(f64, md, p["lam"], p["sigma"], n, cycles)
    gu = (2.0 * (u - target) / u.numel()).contiguous()
    gf64, _ = fg.foeed_inpaint_vjp(f64, md, gu, p["lam"], p["sigma"], n, cycles, checkpoint_every=16)
    # central finite differences of the FP64 solve at 64 random known pixels, h = 1e-3
    known = np.flatnonzero(mask.reshape(-1))
    picks = rng.choice(known, size=64, replace=False)
    loss = lambda uu: float(((uu - target) ** 2).mean())
    errs = []
    for k in picks:
        e = torch.zeros_like(f64).view(-1)
        e[k] = 1e-3
        up, _ = fg.foeed_inpaint(f64 + e.view_as(f64), md, p["lam"], p["sigma"], n, cycles)
        um, _ = fg.foeed_inpaint(f64 - e.view_as(f64), md, p["lam"], p["sigma"], n, cycles)
        fdv = (loss(up) - loss(um)) / 2e-3
        errs.append(abs(float(gf64.view(-1)[k]) - fdv) / max(abs(fdv), 1e-12))
    assert np.median(errs) < 1e-3 and np.max(errs) < 2e-2, (np.median(errs), np.max(errs))
    # the FP32 gradient of the same problem against the FP64 one
    f32 = target.float()
    u32, _ = fg.foeed_inpaint(f32, md, p["lam"], p["sigma"], n, cycles)
    gu32 = (2.0 * (u32 - target.float()) / u32.numel()).contiguous()
    gf32, _ = fg.foeed_inpaint_vjp(f32, md, gu32, p["lam"], p["sigma"], n, cycles, checkpoint_every=16)
    assert float((gf32.double() - gf64).abs().max()) <= 2e-2 * float(gf64.abs().max())
    # a 128 x 128 crop, solved as its own problem, against the FP64 oracle adjoint
    crop = img[:128, :128]
    cm = mask[:128, :128]
    cg = rng.normal(size=crop.shape)
    ref, _ = O.inpaint_vjp(crop, cm, cg, p["sigma"], p["lam"], n, cycles)
    gcrop, _ = fg.foeed_inpaint_vjp(torch.from_numpy(crop.copy()).to(DEV), torch.from_numpy(cm.copy()).to(DEV),
                                    torch.from_numpy(cg).to(DEV), p["lam"], p["sigma"], n, cycles)
    assert np.max(np.abs(gcrop.cpu().numpy() - ref)) <= 1e-9 * np.max(np.abs(ref))

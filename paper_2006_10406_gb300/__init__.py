"""GB300-native FOEED / EED sparse-mask inpainting (arXiv 2006.10406).

Thin Python binding over the C ABI of libfoeed_gb300.so (include/foeed.h).
Every step of the solve runs in the library's CUDA kernels; this module only
marshals arguments: it takes torch tensors (device memory and streams come
from PyTorch), passes raw pointers, sizes and the stream, and turns status
codes into exceptions. There is no CPU fallback: without the compiled library
or without a CUDA device every call raises.

Entry points (names follow the C ABI):
  foeed_inpaint, eed_inpaint   full FSI solve (Sec. 3.3) of Eq. genModel / Eq. EEDModel
  foeed_step, eed_step         one masked FSI step
  foeed_errors                 MSE / AAE (Sec. 3.2) and PSNR
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

__all__ = ["foeed_inpaint", "eed_inpaint", "foeed_inpaint_batch", "eed_inpaint_batch", "inpaint_channels",
           "foeed_inpaint_vjp", "foeed_inpaint_diff",
           "foeed_step", "eed_step", "foeed_errors", "foeed_apply_tensor_field", "workspace_bytes",
           "set_tile_policy", "last_tile_plan",
           "Report", "FoeedError", "lib", "F32", "F64", "F32_F64U", "STATUS"]

F32, F64, F32_F64U = 0, 1, 2
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_NOT_CONVERGED", 4: "ERR_DIVERGED", 5: "ERR_TIMEOUT"}
DIFFUSIVITY = {"charbonnier": 0, "perona_malik": 1, "perona_malik2": 2, "aubert": 3, "geman_reynolds": 4}
MU3 = {"geometric": 0, "arithmetic": 1, "one": 2}


class FoeedError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Params(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("sigma", C.c_double), ("tau", C.c_double),
                ("cycle_len", C.c_int), ("max_cycles", C.c_int), ("tol", C.c_double),
                ("diffusivity", C.c_int), ("mu3_mode", C.c_int), ("init_mode", C.c_int),
                ("check_every", C.c_int)]


class _Instance(C.Structure):
    _fields_ = [("f", C.c_void_p), ("mask", C.c_void_p), ("u_inout", C.c_void_p), ("w", C.c_int), ("h", C.c_int),
                ("pitch", C.c_long), ("lambda_", C.c_double)]


class _Report(C.Structure):
    _fields_ = [("cycles_run", C.c_int), ("last_rel_change", C.c_double), ("converged", C.c_int),
                ("ms", C.c_float)]


class _TilePlan(C.Structure):
    _fields_ = [("tile_h", C.c_int), ("images", C.c_int), ("images_h16", C.c_int), ("tuned", C.c_int),
                ("us_h32", C.c_float), ("us_h16", C.c_float), ("us_chosen", C.c_float), ("us_h64", C.c_float),
                ("us_h8", C.c_float)]


TILE_POLICY = {"auto": 0, "h8": 8, "h16": 16, "h32": 32, "h64": 64, 0: 0, 8: 8, 16: 16, 32: 32, 64: 64}


@dataclass
class Report:
    status: int
    cycles_run: int
    last_rel_change: float
    converged: bool
    ms: float


_lib = None


def lib():
    """Load libfoeed_gb300.so (building it with nvcc if it is missing or stale).

    FOEED_LIBRARY, if set, names another build of the same library to load."""
    global _lib
    if _lib is None:
        path = os.environ.get("FOEED_LIBRARY") or _build.build()
        L = C.CDLL(path)
        vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
        L.foeed_workspace_bytes.argtypes = [i, i, i]
        L.foeed_workspace_bytes.restype = sz
        for name in ("foeed_inpaint", "eed_inpaint"):
            fn = getattr(L, name)
            fn.argtypes = [vp, vp, vp, i, i, C.c_long, i, C.POINTER(_Params), vp, sz, vp, C.POINTER(_Report)]
            fn.restype = i
        for name in ("foeed_step", "eed_step"):
            fn = getattr(L, name)
            fn.argtypes = [vp, vp, vp, vp, i, i, C.c_long, i, d, C.POINTER(_Params), vp]
            fn.restype = i
        L.foeed_batch_workspace_bytes.argtypes = [C.POINTER(_Instance), i, i]
        L.foeed_batch_workspace_bytes.restype = sz
        for name in ("foeed_inpaint_batch", "eed_inpaint_batch"):
            fn = getattr(L, name)
            fn.argtypes = [C.POINTER(_Instance), i, i, C.POINTER(_Params), vp, sz, vp, C.POINTER(_Report)]
            fn.restype = i
        L.foeed_vjp_workspace_bytes.argtypes = [i, i, i, C.POINTER(_Params), i]
        L.foeed_vjp_workspace_bytes.restype = sz
        L.foeed_inpaint_vjp.argtypes = [vp, vp, vp, vp, vp, i, i, C.c_long, i, C.POINTER(_Params), i, vp, sz, vp]
        L.foeed_inpaint_vjp.restype = i
        L.foeed_apply_tensor_field.argtypes = [vp, vp, vp, i, i, C.c_long, i, vp]
        L.foeed_apply_tensor_field.restype = i
        L.foeed_errors_workspace_bytes.argtypes = [i, i]
        L.foeed_errors_workspace_bytes.restype = sz
        L.foeed_errors.argtypes = [vp, vp, i, i, C.c_long, i, vp, sz, vp, C.POINTER(C.c_double)]
        L.foeed_errors.restype = i
        L.foeed_set_tile_policy.argtypes = [i]
        L.foeed_set_tile_policy.restype = i
        L.foeed_last_tile_plan.argtypes = [C.POINTER(_TilePlan)]
        L.foeed_last_tile_plan.restype = i
        L.foeed_last_error.restype = C.c_char_p
        L.foeed_version.restype = C.c_char_p
        _lib = L
    return _lib


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise FoeedError(2, "no CUDA device: the FOEED library runs on the GPU only")
    return torch


def _check(status):
    if status != 0:
        raise FoeedError(status, lib().foeed_last_error().decode())


def _dtype_code(t, dtype):
    if dtype is not None:
        return {"f32": F32, "f64": F64, "f32_f64u": F32_F64U, F32: F32, F64: F64, F32_F64U: F32_F64U}[dtype]
    import torch
    return F64 if t.dtype == torch.float64 else F32


def _params(lam, sigma, tau=0.0, cycle_len=1, max_cycles=1, tol=0.0, diffusivity=0, mu3_mode=0,
            init_mode=0, check_every=8):
    if isinstance(diffusivity, str):
        diffusivity = DIFFUSIVITY[diffusivity]
    if isinstance(mu3_mode, str):
        mu3_mode = MU3[mu3_mode]
    return _Params(float(lam), float(sigma), float(tau), int(cycle_len), int(max_cycles), float(tol),
                   int(diffusivity), int(mu3_mode), int(init_mode), int(check_every))


def _stream_ptr(stream):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _as_device_image(a, dtype, device):
    """2-D device tensor with unit column stride (row pitch = stride(0))."""
    torch = _torch()
    t = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a))
    if t.dim() != 2:
        raise FoeedError(1, "images must be 2-D [h, w]")
    if t.dtype != dtype:
        t = t.to(dtype)
    if t.device.type != "cuda":
        t = t.pin_memory().to(device, non_blocking=True) if t.numel() else t.to(device)
    if t.stride(1) != 1:
        t = t.contiguous()
    return t


def set_tile_policy(policy="auto"):
    """Tile shape of the register-blocked FP32 kernels for later calls on this host
    thread: "auto" (timed once per size and kept), "h64", "h32" or "h16" (64 x 64,
    64 x 32 or 64 x 16 tiles; 64 x 64 for single FOEED images only). Results are
    bitwise the same under every policy."""
    _check(lib().foeed_set_tile_policy(TILE_POLICY[policy]))


def last_tile_plan():
    """The tile plan of the last solve on this thread (dict of foeed_tile_plan)."""
    t = _TilePlan()
    _check(lib().foeed_last_tile_plan(C.byref(t)))
    return {k: getattr(t, k) for k, _ in _TilePlan._fields_}


def workspace_bytes(w, h, dtype=F32):
    """Device workspace bytes the inpaint solvers need for a w x h image."""
    return int(lib().foeed_workspace_bytes(int(w), int(h), int(dtype)))


def _inpaint(method, f, mask, lam, sigma, cycle_len, max_cycles, tau=0.0, tol=0.0, diffusivity=0, mu3_mode=0,
             init_mode=0, u0=None, dtype=None, check_every=8, stream=None, workspace=None, raise_on_status=True,
             device=None):
    torch = _torch()
    dev = torch.device(device) if device is not None else (
        f.device if isinstance(f, torch.Tensor) and f.is_cuda else torch.device("cuda", torch.cuda.current_device()))
    host_out = not (isinstance(f, torch.Tensor) and f.is_cuda)
    if dtype is not None:
        code = _dtype_code(None, dtype)
    elif isinstance(f, torch.Tensor):
        code = F64 if f.dtype == torch.float64 else F32
    else:
        code = F64 if np.asarray(f).dtype == np.float64 else F32
    tdt = torch.float64 if code == F64 else torch.float32
    fd = _as_device_image(f, tdt, dev)
    h, w = fd.shape
    pitch = fd.stride(0)
    md = _as_device_image(mask, torch.uint8, dev)
    if md.shape != fd.shape:
        raise FoeedError(1, "mask shape differs from image shape")
    if md.stride(0) != pitch:
        md = _pitched_like(md, pitch)
    u = torch.empty_strided((h, w), (pitch, 1), dtype=tdt, device=dev)
    if u0 is not None:
        u.copy_(_as_device_image(u0, tdt, dev))
        init_mode = 1
    nbytes = workspace_bytes(w, h, code)
    if workspace is None or workspace.numel() < nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    p = _params(lam, sigma, tau, cycle_len, max_cycles, tol, diffusivity, mu3_mode, init_mode, check_every)
    rep = _Report()
    fn = lib().foeed_inpaint if method == 0 else lib().eed_inpaint
    with torch.cuda.device(dev):
        st = fn(C.c_void_p(fd.data_ptr()), C.c_void_p(md.data_ptr()), C.c_void_p(u.data_ptr()), w, h, pitch, code,
                C.byref(p), C.c_void_p(workspace.data_ptr()), workspace.numel(), _stream_ptr(stream), C.byref(rep))
    if st not in (0, 3, 4) or (raise_on_status and st != 0):
        _check(st)
    report = Report(st, rep.cycles_run, rep.last_rel_change, bool(rep.converged), rep.ms)
    if host_out:
        u = u.cpu()
    return u, report


def _pitched_like(t, pitch):
    torch = _torch()
    out = torch.empty_strided(t.shape, (pitch, 1), dtype=t.dtype, device=t.device)
    out.copy_(t)
    return out


def foeed_inpaint(f, mask, lam, sigma, cycle_len, max_cycles, **kw):
    """FOEED inpainting solve (Eq. genModel, FSI of Sec. 3.3). Returns (u, Report).

    f, mask: [h, w] tensors or arrays (device tensors stay on the device; host
    inputs are copied in and the result copied back). Keyword arguments:
    tau (<= 0: 0.05), tol (0: run exactly max_cycles), diffusivity, mu3_mode,
    init_mode, u0, dtype ('f32' | 'f64' | 'f32_f64u'), check_every, stream,
    workspace, raise_on_status."""
    return _inpaint(0, f, mask, lam, sigma, cycle_len, max_cycles, **kw)


def eed_inpaint(f, mask, lam, sigma, cycle_len, max_cycles, **kw):
    """Second-order EED solve (Eq. EEDModel), same arguments as foeed_inpaint (tau <= 0: 0.25)."""
    return _inpaint(1, f, mask, lam, sigma, cycle_len, max_cycles, **kw)


def foeed_inpaint_batch(images, masks, lambdas, sigma, cycle_len, max_cycles, **kw):
    """Batched FOEED solve of many images of uneven sizes (one launch per FSI step over
    all their tiles, one captured graph per cycle). images/masks: lists of 2-D CUDA
    tensors (float32 / uint8, unit column stride); lambdas: one contrast parameter per
    image. Keywords: tau, tol, init_mode, dtype ("f32" / "f32_f64u"), check_every,
    stream, workspace, raise_on_status. Returns (list of result tensors, list of Report)."""
    return _inpaint_batch("foeed_inpaint_batch", images, masks, lambdas, sigma, cycle_len, max_cycles, **kw)


def eed_inpaint_batch(images, masks, lambdas, sigma, cycle_len, max_cycles, **kw):
    """Batched second-order EED solve (Eq. EEDModel); same arguments as foeed_inpaint_batch."""
    return _inpaint_batch("eed_inpaint_batch", images, masks, lambdas, sigma, cycle_len, max_cycles, **kw)


def inpaint_channels(image, mask, lam, sigma, cycle_len, max_cycles, method="foeed", **kw):
    """Channel-wise reconstruction of a multi-channel image (Sec. 5, colour images):
    image [C, h, w] float32 CUDA tensor, one mask [h, w] shared by all channels, one
    batched solve with one instance per channel. Returns ([C, h, w] result, reports)."""
    torch = _torch()
    if not (isinstance(image, torch.Tensor) and image.is_cuda and image.dim() == 3):
        raise FoeedError(1, "image must be a [C, h, w] CUDA tensor")
    chans = [image[c].contiguous() for c in range(image.shape[0])]
    m = mask.to(image.device, torch.uint8).contiguous()
    fn = {"foeed": foeed_inpaint_batch, "eed": eed_inpaint_batch}[method]
    outs, reps = fn(chans, [m] * len(chans), [lam] * len(chans), sigma, cycle_len, max_cycles, **kw)
    return torch.stack(outs), reps


def _inpaint_batch(entry, images, masks, lambdas, sigma, cycle_len, max_cycles, tau=0.0, tol=0.0, init_mode=0,
                   dtype="f32", check_every=8, stream=None, workspace=None, raise_on_status=True):
    torch = _torch()
    count = len(images)
    if not (len(masks) == len(lambdas) == count) or count == 0:
        raise FoeedError(1, "images, masks and lambdas must have the same nonzero length")
    code = _dtype_code(None, dtype)
    dev = images[0].device
    outs, arr = [], (_Instance * count)()
    keep = []
    for i, (f, m, lam) in enumerate(zip(images, masks, lambdas)):
        if not (isinstance(f, torch.Tensor) and f.is_cuda and f.dim() == 2 and f.dtype == torch.float32):
            raise FoeedError(1, f"image {i} must be a 2-D float32 CUDA tensor")
        if f.stride(1) != 1:
            f = f.contiguous()
        h, w = f.shape
        pitch = f.stride(0)
        m = m if (m.is_cuda and m.dtype == torch.uint8 and m.stride(1) == 1 and m.stride(0) == pitch) \
            else _pitched_like(m.to(dev, torch.uint8), pitch)
        u = torch.empty_strided((h, w), (pitch, 1), dtype=torch.float32, device=dev)
        keep += [f, m]
        outs.append(u)
        arr[i] = _Instance(f.data_ptr(), m.data_ptr(), u.data_ptr(), w, h, pitch, float(lam))
    nbytes = int(lib().foeed_batch_workspace_bytes(arr, count, code))
    if nbytes == 0:
        raise FoeedError(1, "invalid batch")
    if workspace is None or workspace.numel() < nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    p = _params(1.0, sigma, tau, cycle_len, max_cycles, tol, 0, 0, init_mode, check_every)
    reps = (_Report * count)()
    with torch.cuda.device(dev):
        st = getattr(lib(), entry)(arr, count, code, C.byref(p), C.c_void_p(workspace.data_ptr()),
                                   workspace.numel(), _stream_ptr(stream), reps)
    if st not in (0, 3, 4) or (raise_on_status and st != 0):
        _check(st)
    reports = [Report(st, r.cycles_run, r.last_rel_change, bool(r.converged), r.ms) for r in reps]
    return outs, reports


def foeed_inpaint_vjp(f, mask, grad_u, lam, sigma, cycle_len, max_cycles, tau=0.0, checkpoint_every=16,
                      stream=None, workspace=None):
    """Gradient of a loss of the FOEED reconstruction with respect to the stored grey
    values: grad_f = (d u_final / d f)^T grad_u on the known pixels (0 elsewhere),
    through the whole FSI solve (mean initialisation, fixed cycles), recomputed from
    checkpoints every `checkpoint_every` steps. f, mask, grad_u: 2-D CUDA tensors
    (float32 or float64, one row pitch). Returns (grad_f, u_final)."""
    torch = _torch()
    for t in (f, grad_u):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dim() == 2 and t.stride(1) == 1):
            raise FoeedError(1, "f and grad_u must be 2-D CUDA tensors with unit column stride")
    h, w = f.shape
    pitch = f.stride(0)
    if grad_u.stride(0) != pitch or grad_u.dtype != f.dtype:
        grad_u = _pitched_like(grad_u.to(f.dtype), pitch)
    if not (mask.is_cuda and mask.dtype == torch.uint8 and mask.stride(0) == pitch and mask.stride(1) == 1):
        mask = _pitched_like(mask.to(f.device, torch.uint8), pitch)
    code = F64 if f.dtype == torch.float64 else F32
    p = _params(lam, sigma, tau, cycle_len, max_cycles, 0.0, 0, 0, 0, 8)
    nbytes = int(lib().foeed_vjp_workspace_bytes(w, h, code, C.byref(p), int(checkpoint_every)))
    if workspace is None or workspace.numel() < nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=f.device)
    gf = torch.empty_strided((h, w), (pitch, 1), dtype=f.dtype, device=f.device)
    uf = torch.empty_strided((h, w), (pitch, 1), dtype=f.dtype, device=f.device)
    with torch.cuda.device(f.device):
        _check(lib().foeed_inpaint_vjp(C.c_void_p(f.data_ptr()), C.c_void_p(mask.data_ptr()),
                                       C.c_void_p(grad_u.data_ptr()), C.c_void_p(gf.data_ptr()),
                                       C.c_void_p(uf.data_ptr()), w, h, pitch, code, C.byref(p),
                                       int(checkpoint_every), C.c_void_p(workspace.data_ptr()),
                                       workspace.numel(), _stream_ptr(stream)))
    return gf, uf


def _autograd_function():
    import torch

    class FoeedInpaint(torch.autograd.Function):
        """u = FOEED inpainting of f on the mask; backward through the hand-written adjoint."""

        @staticmethod
        def forward(ctx, f, mask, lam, sigma, cycle_len, max_cycles, tau, checkpoint_every):
            u, _ = foeed_inpaint(f.detach(), mask, lam, sigma, cycle_len, max_cycles, tau=tau)
            ctx.save_for_backward(f.detach(), mask)
            ctx.cfg = (lam, sigma, cycle_len, max_cycles, tau, checkpoint_every)
            return u

        @staticmethod
        def backward(ctx, grad_u):
            f, mask = ctx.saved_tensors
            lam, sigma, n, cycles, tau, K = ctx.cfg
            gf, _ = foeed_inpaint_vjp(f, mask, grad_u.contiguous(), lam, sigma, n, cycles, tau=tau,
                                      checkpoint_every=K)
            return gf, None, None, None, None, None, None, None

    return FoeedInpaint


_FoeedInpaint = None


def foeed_inpaint_diff(f, mask, lam, sigma, cycle_len, max_cycles, tau=0.0, checkpoint_every=16):
    """Differentiable FOEED inpainting (torch.autograd): the gradient of any loss of
    the result flows back to f through foeed_inpaint_vjp."""
    global _FoeedInpaint
    if _FoeedInpaint is None:
        _FoeedInpaint = _autograd_function()
    return _FoeedInpaint.apply(f, mask, lam, sigma, cycle_len, max_cycles, tau, checkpoint_every)


def _step(method, u_prev, u_cur, u_next, mask, alpha, lam, sigma, tau=0.0, diffusivity=0, mu3_mode=0,
          dtype=None, stream=None):
    torch = _torch()
    for t in (u_prev, u_cur, u_next):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dim() == 2 and t.stride(1) == 1):
            raise FoeedError(1, "step images must be 2-D CUDA tensors with unit column stride")
    h, w = u_cur.shape
    pitch = u_cur.stride(0)
    if u_prev.stride(0) != pitch or u_next.stride(0) != pitch:
        raise FoeedError(1, "all step images must share one row pitch")
    code = _dtype_code(u_cur, dtype)
    mptr = None
    if mask is not None:
        if mask.dtype != torch.uint8 or mask.stride(0) != pitch or not mask.is_cuda:
            raise FoeedError(1, "mask must be a CUDA uint8 tensor with the images' row pitch")
        mptr = C.c_void_p(mask.data_ptr())
    p = _params(lam, sigma, tau, diffusivity=diffusivity, mu3_mode=mu3_mode)
    fn = lib().foeed_step if method == 0 else lib().eed_step
    with torch.cuda.device(u_cur.device):
        _check(fn(C.c_void_p(u_prev.data_ptr()), C.c_void_p(u_cur.data_ptr()), C.c_void_p(u_next.data_ptr()), mptr,
                  w, h, pitch, code, float(alpha), C.byref(p), _stream_ptr(stream)))
    return u_next


def foeed_step(u_prev, u_cur, u_next, mask, alpha, lam, sigma, **kw):
    """One masked FOEED FSI step into u_next (device tensors, shared pitch)."""
    return _step(0, u_prev, u_cur, u_next, mask, alpha, lam, sigma, **kw)


def eed_step(u_prev, u_cur, u_next, mask, alpha, lam, sigma, **kw):
    """One masked EED FSI step into u_next."""
    return _step(1, u_prev, u_cur, u_next, mask, alpha, lam, sigma, **kw)


def foeed_apply_tensor_field(u, d, stream=None):
    """Pu = sum_ij d_ij [d_ijkl u_kl] for a coefficient field d of shape [h, w, 2, 2, 2, 2]
    (Eq. gen4thPDE_Model; du/dt = -Pu). u: 2-D CUDA tensor (float32 / float64)."""
    torch = _torch()
    if not (u.is_cuda and u.dim() == 2):
        raise FoeedError(1, "u must be a 2-D CUDA tensor")
    u = u.contiguous()
    h, w = u.shape
    d = d.to(u.device, u.dtype).reshape(h, w, 16).contiguous()
    out = torch.empty_like(u)
    code = F64 if u.dtype == torch.float64 else F32
    with torch.cuda.device(u.device):
        _check(lib().foeed_apply_tensor_field(C.c_void_p(u.data_ptr()), C.c_void_p(d.data_ptr()),
                                              C.c_void_p(out.data_ptr()), w, h, w, code, _stream_ptr(stream)))
    return out


def foeed_errors(u, v, dtype=None, stream=None):
    """(MSE, AAE, PSNR) of two device images over all pixels (Sec. 3.2), reduced in double."""
    torch = _torch()
    if u.shape != v.shape or u.stride(0) != v.stride(0) or u.stride(1) != 1 or v.stride(1) != 1:
        raise FoeedError(1, "u and v must have the same shape and row pitch")
    h, w = u.shape
    code = _dtype_code(u, dtype)
    nbytes = int(lib().foeed_errors_workspace_bytes(w, h))
    ws = torch.empty(nbytes, dtype=torch.uint8, device=u.device)
    out = (C.c_double * 3)()
    with torch.cuda.device(u.device):
        _check(lib().foeed_errors(C.c_void_p(u.data_ptr()), C.c_void_p(v.data_ptr()), w, h, u.stride(0), code,
                                  C.c_void_p(ws.data_ptr()), nbytes, _stream_ptr(stream), out))
    return float(out[0]), float(out[1]), float(out[2])

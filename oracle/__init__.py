"""FP64 CPU oracle for FOEED / EED inpainting with FSI (arXiv 2006.10406).

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously-correct reference that the
CUDA path is checked against. Only tests/, the smoke check and the benchmark's
CPU-baseline leg may import it. It shares no code with the CUDA path.

The arithmetic lives in foeed_oracle.c (plain C loops in IEEE double, compiled
without FMA contraction); this module only marshals numpy arrays through ctypes.
Each wrapper names the passage of the paper its C function follows.

Parity status: every function here is pinned by tests/test_oracle_pins.py
(closed forms, invariants, a dense brute-force assembly of P, a direct linear
solve and the FED product formula); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build as _build

FOEED, EED = 0, 1
G_CHARBONNIER, G_PERONA_MALIK, G_PERONA_MALIK2, G_AUBERT, G_GEMAN_REYNOLDS = range(5)
MU3_GEOMETRIC, MU3_ARITHMETIC, MU3_ONE = range(3)

_lib = None
_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_U8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def lib():
    """Load (building on first use) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build()
        L = C.CDLL(path)
        i, d, vp = C.c_int, C.c_double, C.c_void_p
        L.orc_set_threads.argtypes = [i]
        L.orc_get_threads.restype = i
        L.orc_gauss_weights.argtypes = [d, _D, i]
        L.orc_gauss_weights.restype = i
        L.orc_presmooth.argtypes = [_D, i, i, d, _D]
        L.orc_gradient.argtypes = [_D, i, i, _D, _D]
        L.orc_diffusivity.argtypes = [i, d, d]
        L.orc_diffusivity.restype = d
        L.orc_foeed_tensor.argtypes = [d, d, d, i, i, _D, _D]
        L.orc_foeed_tensor_field.argtypes = [_D, i, i, d, d, i, i, _D]
        L.orc_hessian.argtypes = [_D, i, i, _D, _D, _D]
        L.orc_apply_P_field.argtypes = [_D, _D, i, i, _D]
        L.orc_foeed_operator.argtypes = [_D, i, i, d, d, i, i, _D]
        L.orc_eed_tensor_field.argtypes = [_D, i, i, d, d, i, _D]
        L.orc_apply_eed_field.argtypes = [_D, _D, i, i, _D]
        L.orc_eed_operator.argtypes = [_D, i, i, d, d, i, _D]
        L.orc_fsi_alpha.argtypes = [i]
        L.orc_fsi_alpha.restype = d
        L.orc_fsi_step.argtypes = [i, _D, _D, vp, i, i, d, d, d, d, i, i, _D]
        L.orc_inpaint.argtypes = [i, _D, _U8, _D, i, i, d, d, d, i, i, d, i, i, i, _D]
        L.orc_inpaint.restype = i
        L.orc_errors.argtypes = [_D, _D, C.c_long, _D]
        L.orc_foeed_tensor_grad.argtypes = [d, d, d, i, _D]
        L.orc_foeed_vjp_F.argtypes = [_D, _D, i, i, d, d, i, _D]
        L.orc_inpaint_vjp.argtypes = [_D, _U8, _D, _D, vp, i, i, d, d, d, i, i, i]
        L.orc_inpaint_vjp.restype = i
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    """Host threads for the oracle's row loops (OpenMP); 1 by default."""
    lib().orc_set_threads(int(n))


def gauss_weights(sigma: float):
    """Sampled, truncated (R = ceil(3 sigma)), normalised Gaussian taps; Sec. 2.2 pre-smoothing."""
    w = np.zeros(257)
    R = lib().orc_gauss_weights(float(sigma), w, 257)
    return w[: 2 * R + 1].copy(), R


def presmooth(u, sigma):
    """u_sigma = K_sigma * u with mirrored ghosts (Sec. 2.2)."""
    u = _f64(u); h, w = u.shape
    out = np.empty_like(u)
    lib().orc_presmooth(u, w, h, float(sigma), out)
    return out


def gradient(us):
    """Central-difference gradient of u_sigma (Sec. 3.1)."""
    us = _f64(us); h, w = us.shape
    gx, gy = np.empty_like(us), np.empty_like(us)
    lib().orc_gradient(us, w, h, gx, gy)
    return gx, gy


def diffusivity(kind, s2, lam):
    """g(s^2) of Eq. CharDiff / Table 6."""
    return lib().orc_diffusivity(int(kind), float(s2), float(lam))


def foeed_tensor(gx, gy, lam, g_kind=G_CHARBONNIER, mu3_mode=MU3_GEOMETRIC):
    """Literal d_ijkl (Eq. faod_diffTensor, foad_diffTensor_entries) as a [2,2,2,2] array, and mu1..mu4."""
    d = np.zeros(16); mu = np.zeros(4)
    lib().orc_foeed_tensor(float(gx), float(gy), float(lam), int(g_kind), int(mu3_mode), d, mu)
    return d.reshape(2, 2, 2, 2), mu


def foeed_tensor_field(u, sigma, lam, g_kind=G_CHARBONNIER, mu3_mode=MU3_GEOMETRIC):
    """d_ijkl at every pixel, shape [h, w, 2, 2, 2, 2]."""
    u = _f64(u); h, w = u.shape
    d = np.zeros(h * w * 16)
    lib().orc_foeed_tensor_field(u, w, h, float(sigma), float(lam), int(g_kind), int(mu3_mode), d)
    return d.reshape(h, w, 2, 2, 2, 2)


def hessian(u):
    """(u_xx, u_xy, u_yy) by the finite differences of Sec. 3.3."""
    u = _f64(u); h, w = u.shape
    a, b, c = np.empty_like(u), np.empty_like(u), np.empty_like(u)
    lib().orc_hessian(u, w, h, a, b, c)
    return a, b, c


def apply_P_field(u, d):
    """P u for a given tensor field d [h,w,2,2,2,2] (Eq. genModel, parity ghosts for T)."""
    u = _f64(u); h, w = u.shape
    d = _f64(np.broadcast_to(d, (h, w, 2, 2, 2, 2)))
    out = np.empty_like(u)
    lib().orc_apply_P_field(u, d.reshape(-1), w, h, out)
    return out


def foeed_operator(u, sigma, lam, g_kind=G_CHARBONNIER, mu3_mode=MU3_GEOMETRIC):
    """P(u) u for FOEED (du/dt = -P(u) u)."""
    u = _f64(u); h, w = u.shape
    out = np.empty_like(u)
    lib().orc_foeed_operator(u, w, h, float(sigma), float(lam), int(g_kind), int(mu3_mode), out)
    return out


def eed_tensor_field(u, sigma, lam, g_kind=G_CHARBONNIER):
    """(a, b, c) of D = g v1 v1^T + v2 v2^T at every pixel, shape [h, w, 3] (Eq. diffTensor_EED)."""
    u = _f64(u); h, w = u.shape
    abc = np.zeros(h * w * 3)
    lib().orc_eed_tensor_field(u, w, h, float(sigma), float(lam), int(g_kind), abc)
    return abc.reshape(h, w, 3)


def apply_eed_field(u, abc):
    """-div(D grad u) for a given field (a, b, c) [h, w, 3]."""
    u = _f64(u); h, w = u.shape
    abc = _f64(np.broadcast_to(abc, (h, w, 3)))
    out = np.empty_like(u)
    lib().orc_apply_eed_field(u, abc.reshape(-1), w, h, out)
    return out


def eed_operator(u, sigma, lam, g_kind=G_CHARBONNIER):
    """P_EED(u) u (du/dt = -P_EED(u) u)."""
    u = _f64(u); h, w = u.shape
    out = np.empty_like(u)
    lib().orc_eed_operator(u, w, h, float(sigma), float(lam), int(g_kind), out)
    return out


def fsi_alpha(k):
    """alpha_k = (4k+2)/(2k+3) (Sec. 3.3)."""
    return lib().orc_fsi_alpha(int(k))


def fsi_step(method, uprev, ucur, mask, alpha, tau, sigma, lam, g_kind=G_CHARBONNIER,
             mu3_mode=MU3_GEOMETRIC):
    """One masked FSI step (Sec. 3.3); mask None = no Dirichlet pixels."""
    ucur = _f64(ucur); uprev = _f64(uprev); h, w = ucur.shape
    out = np.empty_like(ucur)
    mk = None
    if mask is not None:
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
    lib().orc_fsi_step(int(method), uprev, ucur, None if mk is None else mk.ctypes.data, w, h,
                       float(alpha), float(tau), float(sigma), float(lam), int(g_kind),
                       int(mu3_mode), out)
    return out


def inpaint(method, f, mask, sigma, lam, cycle_len, max_cycles, tau=0.0, tol=0.0,
            g_kind=G_CHARBONNIER, mu3_mode=MU3_GEOMETRIC, init_mode=0, u0=None):
    """Full FSI inpainting solve (Eq. inpaintingModel + genModel / EEDModel, Sec. 3.3).

    Returns (u, status, info) with info = dict(cycles, rel_change, converged)."""
    f = _f64(f); h, w = f.shape
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    u = _f64(u0).copy() if u0 is not None else np.zeros_like(f)
    out = np.zeros(3)
    st = lib().orc_inpaint(int(method), f, mask, u, w, h, float(sigma), float(lam), float(tau),
                           int(cycle_len), int(max_cycles), float(tol), int(g_kind),
                           int(mu3_mode), int(init_mode), out)
    return u, st, dict(cycles=int(out[0]), rel_change=float(out[1]), converged=bool(out[2]))


def errors(u, v):
    """(MSE, AAE) over all pixels (Sec. 3.2)."""
    u = _f64(u); v = _f64(v)
    out = np.zeros(2)
    lib().orc_errors(u.reshape(-1), v.reshape(-1), u.size, out)
    return float(out[0]), float(out[1])


def foeed_tensor_grad(gx, gy, lam, mu3_mode=MU3_GEOMETRIC):
    """d d_ijkl / d g_m of the Charbonnier FOEED tensor, shape [2 (m), 2, 2, 2, 2]."""
    dd = np.zeros(32)
    lib().orc_foeed_tensor_grad(float(gx), float(gy), float(lam), int(mu3_mode), dd)
    return dd.reshape(2, 2, 2, 2, 2)


def foeed_vjp_F(x, v, sigma, lam, mu3_mode=MU3_GEOMETRIC):
    """J_F(x)^T v for the FOEED operator F(x) = P(x) x (Charbonnier)."""
    x = _f64(x); v = _f64(v); h, w = x.shape
    out = np.empty_like(x)
    lib().orc_foeed_vjp_F(x, v, w, h, float(sigma), float(lam), int(mu3_mode), out)
    return out


def inpaint_vjp(f, mask, grad_u, sigma, lam, cycle_len, cycles, tau=0.0, mu3_mode=MU3_GEOMETRIC):
    """dL/df on the known pixels for L with dL/du_final = grad_u, through the whole
    FOEED FSI solve (init from the mean of f over K, fixed cycles). Returns (grad_f, u_final)."""
    f = _f64(f); h, w = f.shape
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    gu = _f64(grad_u)
    gf = np.zeros_like(f)
    uf = np.zeros_like(f)
    st = lib().orc_inpaint_vjp(f, mask, gu, gf, uf.ctypes.data, w, h, float(sigma), float(lam), float(tau),
                               int(cycle_len), int(cycles), int(mu3_mode))
    if st:
        raise ValueError("bad arguments")
    return gf, uf

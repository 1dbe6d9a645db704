"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed forms
(polynomials, Fourier modes, FED step products), invariants (symmetry, PSD,
conservation, Dirichlet pixels, equivariance), library routines (numpy eigh,
numpy linear solve) or a dense brute-force assembly with explicit transposes.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import dense_bruteforce as DB

BIG_LAMBDA = 1e30  # Charbonnier g == 1 exactly for any realistic gradient


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# Gaussian pre-smoothing (Sec. 2.2)

@pytest.mark.parametrize("sigma", [0.5, 1.0, 1.5, 2.3])
def test_gauss_weights_properties(sigma):
    w, R = O.gauss_weights(sigma)
    assert R == math.ceil(3 * sigma)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_array_equal(w, w[::-1])
    # second moment of the sampled Gaussian truncated at 3 sigma: close to sigma^2
    # once sigma >= 1 (sampling aliasing ~ exp(-2 pi^2 sigma^2), truncation ~3%)
    t = np.arange(-R, R + 1)
    var = float((w * t * t).sum())
    if sigma >= 1.0:
        assert abs(var - sigma ** 2) < 0.03 * sigma ** 2


def test_gauss_sigma_zero_is_identity():
    u = _rng(1).uniform(size=(7, 9))
    np.testing.assert_array_equal(O.presmooth(u, 0.0), u)


@pytest.mark.parametrize("shape", [(9, 13), (1, 6), (5, 1), (2, 3)])
def test_presmooth_matches_dense_and_conserves_sum(shape):
    h, w = shape
    u = _rng(2).uniform(size=shape)
    wts, _ = O.gauss_weights(1.0)
    dense = (DB.gauss_2d(h, w, wts) @ u.reshape(-1)).reshape(h, w)
    us = O.presmooth(u, 1.0)
    np.testing.assert_allclose(us, dense, rtol=0, atol=1e-14)
    # mirrored symmetric smoothing is doubly stochastic: the grey-value sum is conserved
    assert abs(us.sum() - u.sum()) < 1e-12
    # constants are reproduced
    np.testing.assert_allclose(O.presmooth(np.full(shape, 0.37), 1.0), 0.37, atol=1e-15)


def test_presmooth_reproduces_linear_ramp_interior():
    y, x = np.mgrid[0:20, 0:24].astype(float)
    u = 0.3 * x - 0.7 * y + 2.0
    us = O.presmooth(u, 1.0)
    np.testing.assert_allclose(us[4:-4, 4:-4], u[4:-4, 4:-4], atol=1e-13)


def test_gradient_of_ramp_and_mirror_border():
    y, x = np.mgrid[0:6, 0:8].astype(float)
    gx, gy = O.gradient(2.0 * x + 3.0 * y)
    np.testing.assert_allclose(gx[:, 1:-1], 2.0)
    np.testing.assert_allclose(gy[1:-1, :], 3.0)
    # mirror ghost u[-1] = u[0]: one-sided half difference at the border
    np.testing.assert_allclose(gx[:, 0], 1.0)
    np.testing.assert_allclose(gx[:, -1], 1.0)


# --------------------------------------------------------------------------
# Diffusivities (Eq. CharDiff, Table 6)

def test_charbonnier_closed_form_values():
    lam = 0.05
    assert O.diffusivity(O.G_CHARBONNIER, 0.0, lam) == 1.0
    assert abs(O.diffusivity(O.G_CHARBONNIER, lam ** 2, lam) - 1 / math.sqrt(2)) < 1e-15
    assert abs(O.diffusivity(O.G_CHARBONNIER, 3 * lam ** 2, lam) - 0.5) < 1e-15
    vals = [O.diffusivity(O.G_CHARBONNIER, s, lam) for s in np.linspace(0, 1, 50)]
    assert all(a > b for a, b in zip(vals, vals[1:]))


def test_other_diffusivities_closed_forms():
    lam = 0.1
    assert abs(O.diffusivity(O.G_PERONA_MALIK, lam ** 2, lam) - 0.5) < 1e-15
    assert abs(O.diffusivity(O.G_PERONA_MALIK2, lam ** 2, lam) - math.exp(-1)) < 1e-15
    assert abs(O.diffusivity(O.G_GEMAN_REYNOLDS, 0.0, lam) - 2 / lam ** 2) < 1e-9
    assert O.diffusivity(O.G_AUBERT, 0.0, lam) == 0.0


def _table6_rows():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table6_diffusivities.txt")
    rows = []
    with open(path) as f:
        for line in f:
            line = line.split("#")[0].split()
            if line:
                rows.append((int(line[0]), float(line[1]), float(line[2]), float(line[3])))
    return rows


@pytest.mark.parametrize("kind,ratio,lam,expected", _table6_rows())
def test_table6_diffusivities_at_hand_computed_points(kind, ratio, lam, expected):
    """Each Table 6 diffusivity at s = lambda/2, lambda, 3 lambda for two lambdas,
    against values worked out by hand from the printed formulas (tests/golden)."""
    s = ratio * lam
    got = O.diffusivity(kind, s * s, lam)
    assert abs(got - expected) <= 1e-13 * max(1.0, abs(expected)), (kind, ratio, lam, got, expected)


@pytest.mark.parametrize("kind", [O.G_CHARBONNIER, O.G_PERONA_MALIK, O.G_PERONA_MALIK2, O.G_GEMAN_REYNOLDS])
def test_table6_decreasing_diffusivities_are_monotone(kind):
    lam = 0.07
    s = np.linspace(0.0, 5 * lam, 200)
    g = np.array([O.diffusivity(kind, v * v, lam) for v in s])
    assert np.all(np.diff(g) < 0)


def test_aubert_rises_to_its_maximum_at_s_equal_lambda_then_falls():
    """(s/l)^2/(s^2+l^2)^2 as a function of t = s^2 is t/(l^2 (t+l^2)^2), whose
    derivative vanishes at t = l^2 only: increasing below s = lambda, decreasing above."""
    lam = 0.07
    below = np.linspace(0.0, lam, 100)
    above = np.linspace(lam, 5 * lam, 100)
    gb = np.array([O.diffusivity(O.G_AUBERT, v * v, lam) for v in below])
    ga = np.array([O.diffusivity(O.G_AUBERT, v * v, lam) for v in above])
    assert np.all(np.diff(gb) > 0) and np.all(np.diff(ga) < 0)
    assert abs(ga[0] - 1.0 / (4 * lam ** 4)) < 1e-9 / lam ** 4


def test_table6_scaling_in_lambda():
    """At a fixed ratio s/lambda, Charbonnier and both Perona-Malik forms do not depend
    on lambda, Geman-Reynolds scales as lambda^-2 and Aubert as lambda^-4."""
    for r in (0.3, 1.7):
        for kind, p in ((O.G_CHARBONNIER, 0), (O.G_PERONA_MALIK, 0), (O.G_PERONA_MALIK2, 0),
                        (O.G_GEMAN_REYNOLDS, 2), (O.G_AUBERT, 4)):
            a = O.diffusivity(kind, (r * 0.1) ** 2, 0.1)
            b = O.diffusivity(kind, (r * 0.05) ** 2, 0.05)
            assert abs(b / a - 2.0 ** p) < 1e-12 * 2.0 ** p, (kind, r, a, b)


# --------------------------------------------------------------------------
# Fourth-order diffusion tensor (Eq. faod_diffTensor, foad_diffTensor_entries, E3)

def _frob(A, B):
    return float(np.trace(B.T @ A))


@pytest.mark.parametrize("g", [(0.3, -0.4), (1e-3, 2e-3), (0.0, 0.7), (-2.0, 0.0)])
@pytest.mark.parametrize("mode", [O.MU3_GEOMETRIC, O.MU3_ARITHMETIC, O.MU3_ONE])
def test_tensor_symmetries_and_spectrum(g, mode):
    lam = 0.5
    d, mu = O.foeed_tensor(g[0], g[1], lam, O.G_CHARBONNIER, mode)
    np.testing.assert_allclose(d, d.transpose(1, 0, 2, 3), atol=1e-15)   # d_ijkl = d_jikl
    np.testing.assert_allclose(d, d.transpose(0, 1, 3, 2), atol=1e-15)   # d_ijkl = d_ijlk
    np.testing.assert_allclose(d, d.transpose(2, 3, 0, 1), atol=1e-15)   # d_ijkl = d_klij
    s2 = g[0] ** 2 + g[1] ** 2
    mu1 = 1.0 / math.sqrt(1.0 + s2 / lam ** 2)
    mu3 = {O.MU3_GEOMETRIC: math.sqrt(mu1), O.MU3_ARITHMETIC: (1 + mu1) / 2, O.MU3_ONE: 1.0}[mode]
    np.testing.assert_allclose(mu, [mu1, 1.0, mu3, 0.0], atol=1e-15)
    # as a linear map on 2x2 matrices (4x4 matrix), the eigenvalues are {mu1, mu2, mu3, mu4}
    ev = np.sort(np.linalg.eigvalsh(d.reshape(4, 4)))
    np.testing.assert_allclose(ev, np.sort([mu1, 1.0, mu3, 0.0]), atol=1e-14)


def test_eigentensors_orthonormal_and_e3_identity():
    rng = _rng(3)
    for _ in range(20):
        gx, gy = rng.normal(size=2)
        n = math.hypot(gx, gy)
        v1 = np.array([gx, gy]) / n
        v2 = np.array([-v1[1], v1[0]])
        E = [np.outer(v1, v1), np.outer(v2, v2),
             (np.outer(v1, v2) + np.outer(v2, v1)) / math.sqrt(2),
             (np.outer(v1, v2) - np.outer(v2, v1)) / math.sqrt(2)]
        G = np.array([[_frob(a, b) for b in E] for a in E])
        np.testing.assert_allclose(G, np.eye(4), atol=1e-14)
        Hm = rng.normal(size=(2, 2)); Hm = Hm + Hm.T
        d, mu = O.foeed_tensor(gx, gy, 0.8)
        T = np.einsum("ijkl,kl->ij", d, Hm)
        # Eq. foad_diff_direc: D:H = mu1 u_v1v1 E1 + mu2 u_v2v2 E2 + mu3/sqrt2 (u_aa - u_bb) E3
        a = (v1 + v2) / math.sqrt(2); b = (v1 - v2) / math.sqrt(2)
        uaa, ubb = a @ Hm @ a, b @ Hm @ b
        T2 = mu[0] * (v1 @ Hm @ v1) * E[0] + mu[1] * (v2 @ Hm @ v2) * E[1] \
            + mu[2] / math.sqrt(2) * (uaa - ubb) * E[2]
        np.testing.assert_allclose(T, T2, atol=1e-13)
        # Eq. E3: E3:H = (v1^T H v2 + v2^T H v1)/sqrt2 = (u_aa - u_bb)/sqrt2
        assert abs(_frob(E[2], Hm) - (uaa - ubb) / math.sqrt(2)) < 1e-13
        # antisymmetric E4 annihilates a symmetric Hessian
        assert abs(_frob(E[3], Hm)) < 1e-14


def test_zero_gradient_gives_identity_on_symmetric_matrices():
    d, mu = O.foeed_tensor(0.0, 0.0, 0.1)
    Hm = np.array([[0.3, -1.1], [-1.1, 2.0]])
    np.testing.assert_allclose(np.einsum("ijkl,kl->ij", d, Hm), Hm, atol=1e-15)


def test_tensor_rotation_covariance():
    rng = _rng(4)
    for _ in range(10):
        g = rng.normal(size=2)
        th = rng.uniform(0, 2 * np.pi)
        Rm = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        d, _ = O.foeed_tensor(g[0], g[1], 0.7)
        gr = Rm @ g
        dr, _ = O.foeed_tensor(gr[0], gr[1], 0.7)
        expect = np.einsum("ai,bj,ck,dl,ijkl->abcd", Rm, Rm, Rm, Rm, d)
        np.testing.assert_allclose(dr, expect, atol=1e-13)


def test_tensor_matches_einsum_spectral_form():
    rng = _rng(5)
    for _ in range(10):
        gx, gy = rng.normal(size=2) * 0.1
        lam = 0.05
        d, mu = O.foeed_tensor(gx, gy, lam)
        np.testing.assert_allclose(d, DB.spectral_tensor(gx, gy, mu[0], mu[2]), atol=1e-15)


# --------------------------------------------------------------------------
# Inner Hessian (Sec. 3.3)

def test_hessian_exact_on_quadratics():
    y, x = np.mgrid[0:9, 0:11].astype(float)
    u = 1.5 * x * x - 0.25 * x * y + 0.75 * y * y + x - 3
    hxx, hxy, hyy = O.hessian(u)
    np.testing.assert_allclose(hxx[1:-1, 1:-1], 3.0, atol=1e-12)
    np.testing.assert_allclose(hxy[1:-1, 1:-1], -0.25, atol=1e-12)
    np.testing.assert_allclose(hyy[1:-1, 1:-1], 1.5, atol=1e-12)


# --------------------------------------------------------------------------
# Fourth-order operator (Eq. genModel with Sec. 3.3 stencils)

def _poly(h, w, fn):
    y, x = np.mgrid[0:h, 0:w].astype(float)
    x = x - w / 2.0
    y = y - h / 2.0
    return fn(x, y), x, y


@pytest.mark.parametrize("fn,expect", [
    (lambda x, y: x ** 4, lambda x, y: 24.0 + 0 * x),
    (lambda x, y: y ** 4, lambda x, y: 24.0 + 0 * x),
    (lambda x, y: x * x * y * y, lambda x, y: 8.0 + 0 * x),
    (lambda x, y: x ** 5, lambda x, y: 120.0 * x),
    (lambda x, y: x ** 3 * y * y, lambda x, y: 24.0 * x),
    (lambda x, y: 2 * x - y + 0.5 * x * y, lambda x, y: 0.0 * x),
])
def test_isotropic_limit_is_bilaplacian_on_polynomials(fn, expect):
    """g == 1: P u = Delta^2 u exactly for polynomials of degree <= 5 (interior)."""
    u, x, y = _poly(24, 26, fn)
    Pu = O.foeed_operator(u, 1.0, BIG_LAMBDA)
    m = 6
    np.testing.assert_allclose(Pu[m:-m, m:-m], expect(x, y)[m:-m, m:-m], atol=1e-7)


@pytest.mark.parametrize("a,b", [(1, 0), (0, 2), (3, 1), (5, 4), (7, 7)])
def test_isotropic_limit_fourier_eigenmodes_including_border(a, b):
    """g == 1, mirrored border: cos modes are eigenvectors of P with eigenvalue
    16 sin^4(tx/2) + 2 sin^2(tx) sin^2(ty) + 16 sin^4(ty/2) over the whole image."""
    h, w = 12, 14
    tx, ty = np.pi * a / w, np.pi * b / h
    y, x = np.mgrid[0:h, 0:w].astype(float)
    u = np.cos(tx * (x + 0.5)) * np.cos(ty * (y + 0.5))
    lam = 16 * np.sin(tx / 2) ** 4 + 2 * np.sin(tx) ** 2 * np.sin(ty) ** 2 + 16 * np.sin(ty / 2) ** 4
    Pu = O.foeed_operator(u, 1.0, BIG_LAMBDA)
    np.testing.assert_allclose(Pu, lam * u, atol=1e-12)


def test_isotropic_limit_sinusoid_interior_symbol():
    w_, v_ = 0.37, 0.21
    y, x = np.mgrid[0:20, 0:20].astype(float)
    u = np.sin(w_ * x) * np.sin(v_ * y)
    lam = 16 * np.sin(w_ / 2) ** 4 + 2 * np.sin(w_) ** 2 * np.sin(v_) ** 2 + 16 * np.sin(v_ / 2) ** 4
    Pu = O.foeed_operator(u, 1.0, BIG_LAMBDA)
    np.testing.assert_allclose(Pu[3:-3, 3:-3], lam * u[3:-3, 3:-3], atol=1e-13)
    # small-frequency limit of the symbol: (w^2 + v^2)^2, relative error O(w^2)
    for s_ in (0.05, 0.01):
        a_, b_ = s_, 0.6 * s_
        sym = 16 * np.sin(a_ / 2) ** 4 + 2 * np.sin(a_) ** 2 * np.sin(b_) ** 2 + 16 * np.sin(b_ / 2) ** 4
        assert abs(sym / (a_ ** 2 + b_ ** 2) ** 2 - 1.0) < s_ * s_


def _fourth_derivative_tensor(coef):
    """Constant 4th-derivative tensor u_ijkl of sum c_ab x^a y^b with a + b = 4."""
    T = np.zeros((2, 2, 2, 2))
    for (a, b), c in coef.items():
        # u_ijkl with n_x x-indices and n_y y-indices is nonzero only if n_x = a
        for idx in np.ndindex(2, 2, 2, 2):
            nx = idx.count(0)
            if nx == a:
                T[idx] += c * math.factorial(a) * math.factorial(b)
    return T


@pytest.mark.parametrize("theta", [0.0, 0.3, 1.1, 2.5])
def test_frozen_anisotropic_tensor_on_quartics(theta):
    """Constant D from v1 = (cos t, sin t): P u = sum d_ijkl u_ijkl = mu1 u_v1v1v1v1
    + 2 mu3 u_v1v1v2v2 + mu2 u_v2v2v2v2 for a quartic u (interior points)."""
    h, w = 22, 22
    coef = {(4, 0): 0.5, (3, 1): -0.25, (2, 2): 1.0, (1, 3): 0.75, (0, 4): -0.3}
    u, x, y = _poly(h, w, lambda x, y: sum(c * x ** a * y ** b for (a, b), c in coef.items()))
    g = 0.2 * np.array([np.cos(theta), np.sin(theta)])
    d, mu = O.foeed_tensor(g[0], g[1], 0.15)
    Pu = O.apply_P_field(u, d)
    U4 = _fourth_derivative_tensor(coef)
    expect = float(np.einsum("ijkl,ijkl->", d, U4))
    v1 = np.array([np.cos(theta), np.sin(theta)]); v2 = np.array([-v1[1], v1[0]])
    dirs = lambda a, b, c, e: float(np.einsum("ijkl,i,j,k,l->", U4, a, b, c, e))
    expect2 = mu[0] * dirs(v1, v1, v1, v1) + 2 * mu[2] * dirs(v1, v1, v2, v2) + mu[1] * dirs(v2, v2, v2, v2)
    assert abs(expect - expect2) < 1e-10
    np.testing.assert_allclose(Pu[3:-3, 3:-3], expect, atol=1e-7)


@pytest.mark.parametrize("shape", [(6, 6), (7, 5), (1, 8), (8, 2), (3, 3), (9, 10)])
def test_operator_matches_dense_transpose_assembly(shape):
    """The ghost-cell operator equals P = sum A_ij^T diag(d_ijkl) A_kl assembled densely."""
    h, w = shape
    rng = _rng(6)
    u0 = rng.uniform(size=shape)
    d = O.foeed_tensor_field(u0, 1.0, 0.05)
    P = DB.foeed_P(d)
    n = h * w
    cols = np.stack([O.apply_P_field(np.eye(n)[i].reshape(h, w), d).reshape(-1) for i in range(n)], 1)
    np.testing.assert_allclose(cols, P, atol=1e-13)
    # symmetric, positive semi-definite, bounded by 32 (sufficient tau <= 1/16), P 1 = 0
    np.testing.assert_allclose(P, P.T, atol=1e-13)
    ev = np.linalg.eigvalsh(P)
    assert ev.min() > -1e-12
    assert ev.max() <= 32.0 + 1e-9
    np.testing.assert_allclose(P @ np.ones(n), 0.0, atol=1e-13)


def test_operator_full_nonlinear_matches_dense():
    h, w = 8, 9
    u = _rng(7).uniform(size=(h, w))
    wts, _ = O.gauss_weights(1.0)
    us = (DB.gauss_2d(h, w, wts) @ u.reshape(-1))
    _, _, _, Dx, Dy = DB.ops2d(h, w)
    gx, gy = Dx @ us, Dy @ us
    lam = 0.1
    d = np.zeros((h * w, 2, 2, 2, 2))
    for p in range(h * w):
        mu1 = 1.0 / math.sqrt(1.0 + (gx[p] ** 2 + gy[p] ** 2) / lam ** 2)
        d[p] = DB.spectral_tensor(gx[p], gy[p], mu1, math.sqrt(mu1))
    P = DB.foeed_P(d.reshape(h, w, 2, 2, 2, 2))
    np.testing.assert_allclose(O.foeed_operator(u, 1.0, lam).reshape(-1), P @ u.reshape(-1), atol=1e-13)


def test_affine_images_are_in_the_kernel():
    y, x = np.mgrid[0:15, 0:17].astype(float)
    u = 0.2 * x - 0.1 * y + 0.4
    Pu = O.foeed_operator(u, 1.0, 0.05)
    # interior: every second difference of an affine function is exactly zero
    np.testing.assert_allclose(Pu[2:-2, 2:-2], 0.0, atol=1e-14)
    c = np.full((6, 7), 0.3)
    assert np.all(O.foeed_operator(c, 1.0, 0.05) == 0.0)
    assert np.all(O.eed_operator(c, 1.0, 0.05) == 0.0)


# --------------------------------------------------------------------------
# EED comparison path (Eq. EEDModel, diffTensor_EED)

def test_eed_tensor_eigenstructure():
    u = _rng(8).uniform(size=(7, 8))
    abc = O.eed_tensor_field(u, 1.0, 0.1)
    us = O.presmooth(u, 1.0)
    gx, gy = O.gradient(us)
    for p in np.ndindex(7, 8):
        D = np.array([[abc[p][0], abc[p][1]], [abc[p][1], abc[p][2]]])
        g = np.array([gx[p], gy[p]])
        mu1 = 1.0 / math.sqrt(1 + g @ g / 0.01)
        ev = np.sort(np.linalg.eigvalsh(D))
        np.testing.assert_allclose(ev, np.sort([mu1, 1.0]), atol=1e-14)
        np.testing.assert_allclose(D @ g, mu1 * g, atol=1e-14)   # gradient is the mu1 eigenvector


@pytest.mark.parametrize("shape", [(6, 6), (5, 7), (1, 9), (2, 2)])
def test_eed_matches_dense_and_is_symmetric_psd(shape):
    h, w = shape
    u = _rng(9).uniform(size=shape)
    abc = O.eed_tensor_field(u, 1.0, 0.05)
    P = DB.eed_P(abc)
    n = h * w
    cols = np.stack([O.apply_eed_field(np.eye(n)[i].reshape(h, w), abc).reshape(-1) for i in range(n)], 1)
    np.testing.assert_allclose(cols, P, atol=1e-14)
    np.testing.assert_allclose(P, P.T, atol=1e-14)
    ev = np.linalg.eigvalsh(P)
    assert ev.min() > -1e-12
    assert ev.max() <= 8.0 + 1e-9
    np.testing.assert_allclose(P @ np.ones(n), 0.0, atol=1e-14)


@pytest.mark.parametrize("a,b", [(1, 0), (2, 3), (6, 5)])
def test_eed_isotropic_limit_is_5point_laplacian(a, b):
    h, w = 9, 11
    tx, ty = np.pi * a / w, np.pi * b / h
    y, x = np.mgrid[0:h, 0:w].astype(float)
    u = np.cos(tx * (x + 0.5)) * np.cos(ty * (y + 0.5))
    lam = 4 * np.sin(tx / 2) ** 2 + 4 * np.sin(ty / 2) ** 2
    np.testing.assert_allclose(O.eed_operator(u, 1.0, BIG_LAMBDA), lam * u, atol=1e-13)


# --------------------------------------------------------------------------
# FSI time integration (Sec. 3.3)

def _fed_factor(z, n):
    """FED cycle (Grewenig, Weickert, Bruhn): prod_i (1 - z / (2 cos^2(pi (2i+1)/(4n+2))))."""
    r = 1.0
    for i in range(n):
        r *= 1.0 - z / (2.0 * math.cos(math.pi * (2 * i + 1) / (4 * n + 2)) ** 2)
    return r


@pytest.mark.parametrize("method,tau", [(O.FOEED, 0.05), (O.EED, 0.25)])
@pytest.mark.parametrize("n", [1, 2, 5, 20])
def test_fsi_cycle_equals_fed_product_on_eigenmode(method, tau, n):
    """On a Fourier eigenmode of the linear (g == 1) operator, one FSI cycle
    multiplies the mode by the FED box-filter factor; for small tau*lambda the
    factor is 1 - tau*lambda*n(n+1)/3 (the FSI cycle time)."""
    h, w = 10, 12
    a, b = 3, 2
    tx, ty = np.pi * a / w, np.pi * b / h
    y, x = np.mgrid[0:h, 0:w].astype(float)
    u0 = np.cos(tx * (x + 0.5)) * np.cos(ty * (y + 0.5))
    if method == O.FOEED:
        lam = 16 * np.sin(tx / 2) ** 4 + 2 * np.sin(tx) ** 2 * np.sin(ty) ** 2 + 16 * np.sin(ty / 2) ** 4
    else:
        lam = 4 * np.sin(tx / 2) ** 2 + 4 * np.sin(ty / 2) ** 2
    mask = np.zeros((h, w), np.uint8)
    u, st, info = O.inpaint(method, u0, mask, 1.0, BIG_LAMBDA, n, 1, tau=tau, init_mode=1, u0=u0)
    assert st == 0 and info["cycles"] == 1
    np.testing.assert_allclose(u, _fed_factor(tau * lam, n) * u0, atol=1e-12)


def test_fsi_cycle_time():
    for n in (3, 10, 40):
        z = 1e-7
        assert abs((_fed_factor(z, n) - 1.0) / z + n * (n + 1) / 3.0) < 1e-4 * n * n


def test_fsi_alpha_first_values():
    assert O.fsi_alpha(0) == 2.0 / 3.0
    assert abs(O.fsi_alpha(1) - 6.0 / 5.0) < 1e-16
    assert abs(O.fsi_alpha(1000) - 2.0) < 1e-2


@pytest.mark.parametrize("method,tau", [(O.FOEED, 0.05), (O.EED, 0.25)])
def test_linear_inpainting_converges_to_direct_solve(method, tau):
    """g == 1: the FSI steady state solves P_UU u_U = -P_UK f_K (numpy dense solve)."""
    h, w = 8, 7
    rng = _rng(10)
    f = rng.uniform(size=(h, w))
    mask = DB_mask = np.zeros((h, w), np.uint8)
    for (yy, xx) in [(0, 0), (1, 5), (3, 2), (4, 6), (6, 1), (7, 4), (5, 3), (2, 0)]:
        mask[yy, xx] = 1
    u, st, info = O.inpaint(method, f, mask, 1.0, BIG_LAMBDA, 20, 3000, tau=tau, tol=1e-15)
    assert st == 0, info
    if method == O.FOEED:
        d = np.broadcast_to(O.foeed_tensor(0.0, 0.0, 1.0)[0], (h, w, 2, 2, 2, 2))
        P = DB.foeed_P(np.array(d))
    else:
        abc = np.zeros((h, w, 3)); abc[..., 0] = 1.0; abc[..., 2] = 1.0
        P = DB.eed_P(abc)
    K = mask.reshape(-1) != 0
    U = ~K
    fv = f.reshape(-1)
    uU = np.linalg.solve(P[np.ix_(U, U)], -P[np.ix_(U, K)] @ fv[K])
    np.testing.assert_allclose(u.reshape(-1)[U], uU, atol=1e-9)
    np.testing.assert_array_equal(u.reshape(-1)[K], fv[K])


def test_whole_solver_matches_dense_bruteforce():
    """Nonlinear FOEED, all steps: oracle solve == dense-matrix FSI recursion."""
    h, w = 9, 10
    rng = _rng(11)
    f = rng.uniform(size=(h, w))
    mask = (rng.uniform(size=(h, w)) < 0.15).astype(np.uint8)
    wts, _ = O.gauss_weights(1.0)
    ud = DB.dense_foeed_fsi(f, mask, 1.0, 0.1, 0.05, 6, 3, wts)
    u, st, _ = O.inpaint(O.FOEED, f, mask, 1.0, 0.1, 6, 3)
    np.testing.assert_allclose(u, ud, atol=1e-12)


@pytest.mark.parametrize("method", [O.FOEED, O.EED])
def test_known_pixels_fixed_bitwise(method):
    import synth
    img, mask, p = synth.workload(1, h=24, w=20)
    u, st, info = O.inpaint(method, img, mask, 1.0, 0.05, 10, 3)
    k = mask != 0
    np.testing.assert_array_equal(u[k], img[k])
    assert np.isfinite(u).all()


@pytest.mark.parametrize("method", [O.FOEED, O.EED])
def test_mean_conserved_without_mask(method):
    """No Dirichlet pixels: 1^T P = 0 (symmetric P, P 1 = 0), so FSI conserves the sum."""
    u0 = _rng(12).uniform(size=(13, 11))
    mask = np.zeros(u0.shape, np.uint8)
    u, st, _ = O.inpaint(method, u0, mask, 1.0, 0.05, 10, 5, init_mode=1, u0=u0)
    assert abs(u.sum() - u0.sum()) < 1e-11


def test_constant_image_is_fixed_point():
    c = np.full((9, 8), 0.3)
    mask = np.zeros(c.shape, np.uint8); mask[2, 3] = 1
    for method in (O.FOEED, O.EED):
        u, st, _ = O.inpaint(method, c, mask, 1.0, 0.05, 7, 3)
        np.testing.assert_allclose(u, 0.3, atol=1e-15)


@pytest.mark.parametrize("op", ["T", "flipx", "flipy", "rot90"])
def test_equivariance(op):
    import synth
    img, mask, _ = synth.workload(1, h=16, w=12)
    tr = {"T": lambda a: a.T, "flipx": lambda a: a[:, ::-1], "flipy": lambda a: a[::-1, :],
          "rot90": lambda a: np.rot90(a)}[op]
    u, _, _ = O.inpaint(O.FOEED, img, mask, 1.0, 0.05, 8, 3)
    ut, _, _ = O.inpaint(O.FOEED, np.ascontiguousarray(tr(img)), np.ascontiguousarray(tr(mask)),
                         1.0, 0.05, 8, 3)
    np.testing.assert_allclose(ut, tr(u), atol=1e-12)


@pytest.mark.parametrize("method,tau", [(O.FOEED, 1.0 / 16.0), (O.EED, 0.25)])
def test_l2_stability_of_smoothing_variant(method, tau):
    """Eq. l2stability: plain explicit steps (alpha = 1) of the smoothing variant
    never increase the L2 norm for tau <= 2/|P| (|P| <= 32 FOEED, 8 EED)."""
    u = _rng(13).uniform(size=(14, 15))
    for _ in range(30):
        un = O.fsi_step(method, u, u, None, 1.0, tau, 1.0, 0.05)
        assert np.linalg.norm(un) <= np.linalg.norm(u) * (1 + 1e-14)
        u = un


def test_divergence_reported():
    u0 = _rng(14).uniform(size=(10, 10))
    mask = np.zeros(u0.shape, np.uint8)
    u, st, info = O.inpaint(O.FOEED, u0, mask, 1.0, BIG_LAMBDA, 1, 400, tau=0.5, init_mode=1, u0=u0)
    assert st == 4


def test_error_metrics():
    u = np.array([[1.0, 2.0], [3.0, 4.0]])
    v = np.array([[1.0, 0.0], [3.0, 5.0]])
    mse, aae = O.errors(u, v)
    assert mse == (4 + 1) / 4 and aae == (2 + 1) / 4

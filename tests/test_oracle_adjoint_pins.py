"""Pins for the oracle's adjoint (vector-Jacobian product) of the FOEED solve.

The adjoint is pinned against finite differences of the oracle's own forward
map (central differences in FP64) and, for the linear limit g == 1, against a
dense Jacobian built column by column from forward solves.
"""
import numpy as np
import pytest

import oracle as O

BIG_LAMBDA = 1e30


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


@pytest.mark.parametrize("g", [(0.3, -0.4), (1e-3, 2e-3), (0.0, 0.7), (-2.0, 0.05)])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_tensor_gradient_matches_finite_differences(g, mode):
    lam = 0.5
    dd = O.foeed_tensor_grad(g[0], g[1], lam, mode)
    for m in range(2):
        h = 1e-6 * max(1.0, abs(g[m]))
        gp = list(g); gm = list(g)
        gp[m] += h; gm[m] -= h
        fd = (O.foeed_tensor(gp[0], gp[1], lam, 0, mode)[0] - O.foeed_tensor(gm[0], gm[1], lam, 0, mode)[0]) / (2 * h)
        np.testing.assert_allclose(dd[m], fd, atol=1e-7, rtol=1e-6)


def test_tensor_gradient_vanishes_at_zero_gradient_in_direction_terms():
    # at g = 0 the tensor is the identity on symmetric matrices for every direction,
    # and d mu / d g = 0 there: the whole derivative is zero
    dd = O.foeed_tensor_grad(0.0, 0.0, 0.3)
    np.testing.assert_array_equal(dd, 0.0)


@pytest.mark.parametrize("shape", [(9, 11), (6, 5), (1, 8)])
def test_vjp_of_operator_matches_finite_differences(shape):
    rng = _rng(20)
    x = rng.uniform(size=shape)
    wv = rng.normal(size=shape)
    delta = rng.normal(size=shape)
    sigma, lam = 1.0, 0.1
    got = float(np.sum(O.foeed_vjp_F(x, wv, sigma, lam) * delta))
    h = 1e-6
    fd = float(np.sum(wv * (O.foeed_operator(x + h * delta, sigma, lam) -
                             O.foeed_operator(x - h * delta, sigma, lam)))) / (2 * h)
    assert abs(got - fd) <= 1e-6 * max(1.0, abs(fd))


def _loss_and_grad(f, mask, gu, n, cycles, sigma=1.0, lam=0.1):
    gf, uf = O.inpaint_vjp(f, mask, gu, sigma, lam, n, cycles)
    return float(np.sum(gu * uf)), gf


@pytest.mark.parametrize("n,cycles", [(1, 3), (2, 2), (5, 2)])
def test_solve_vjp_matches_finite_differences(n, cycles):
    rng = _rng(21 + n)
    h_, w_ = 10, 9
    f = rng.uniform(size=(h_, w_))
    mask = (rng.uniform(size=(h_, w_)) < 0.25).astype(np.uint8)
    gu = rng.normal(size=(h_, w_))
    _, gf = _loss_and_grad(f, mask, gu, n, cycles)
    assert np.all(gf[mask == 0] == 0.0)
    for trial in range(3):
        delta = rng.normal(size=(h_, w_)) * mask
        h = 1e-6
        lp, _ = _loss_and_grad(f + h * delta, mask, gu, n, cycles)
        lm, _ = _loss_and_grad(f - h * delta, mask, gu, n, cycles)
        fd = (lp - lm) / (2 * h)
        got = float(np.sum(gf * delta))
        assert abs(got - fd) <= 1e-6 * max(1.0, abs(fd)), (trial, got, fd)


def test_solve_vjp_linear_limit_is_the_transposed_jacobian():
    """g == 1: u_final is affine in f, so the VJP is J^T grad_u with J built by forward solves."""
    rng = _rng(22)
    h_, w_ = 6, 7
    f = rng.uniform(size=(h_, w_))
    mask = np.zeros((h_, w_), np.uint8)
    for (yy, xx) in [(0, 1), (2, 5), (4, 3), (5, 0), (1, 2)]:
        mask[yy, xx] = 1
    gu = rng.normal(size=(h_, w_))
    n, cycles = 4, 3
    gf, u0 = O.inpaint_vjp(f, mask, gu, 1.0, BIG_LAMBDA, n, cycles)
    K = np.flatnonzero(mask.reshape(-1))
    J = np.zeros((h_ * w_, len(K)))
    for c, k in enumerate(K):
        e = np.zeros(h_ * w_); e[k] = 1.0
        _, uk = O.inpaint_vjp(f + e.reshape(h_, w_), mask, gu, 1.0, BIG_LAMBDA, n, cycles)
        J[:, c] = (uk - u0).reshape(-1)  # exact: the map is affine
    np.testing.assert_allclose(gf.reshape(-1)[K], J.T @ gu.reshape(-1), atol=1e-12)

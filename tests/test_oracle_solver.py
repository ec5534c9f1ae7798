"""Pins of the oracle's screened-Poisson solver (Eq. 1, Eq. 8) against closed forms:

* the gradient equals central differences of the energy
  E = 1/2 sum over 4-neighbour pairs ((O_i - O_j) - (P_i - P_j))^2 + 1/2 sum wc (O - A)^2;
* with a constant wc = c the iteration converges to the solution of (Lg + c) O = Lg P + c A,
  which the DCT-II diagonalises exactly (Lg with Neumann boundary has the eigenvalues
  (2 - 2 cos(pi k / h)) + (2 - 2 cos(pi l / w)) on the DCT-II basis);
* O = P = A is a fixed point, and wc = 0 with A = P returns P;
* one iteration from O^0 = O^-1 = A moves by -eta grad E(A) only (no momentum yet).
"""
import numpy as np
import pytest
from scipy.fft import dctn, idctn

import oracle
import synth


def _energy(O, P, A, wc):
    dO_y, dP_y = np.diff(O, axis=0), np.diff(P, axis=0)
    dO_x, dP_x = np.diff(O, axis=1), np.diff(P, axis=1)
    return 0.5 * (((dO_y - dP_y) ** 2).sum() + ((dO_x - dP_x) ** 2).sum()) + 0.5 * (wc * (O - A) ** 2).sum()


def test_gradient_is_the_energy_gradient():
    g = synth.rng(60)
    h, w = 9, 13
    O, P, A = g.normal(size=(3, h, w))
    wc = g.uniform(0, 2, (h, w))
    grad = oracle.poisson_grad(O, P, A, wc)
    V = g.normal(size=(h, w))
    eps = 1e-6
    fd = (_energy(O + eps * V, P, A, wc) - _energy(O - eps * V, P, A, wc)) / (2 * eps)
    assert abs(fd - (grad * V).sum()) <= 1e-7 * max(1.0, abs(fd))


@pytest.mark.parametrize("h,w,c", [(16, 24, 0.7), (33, 20, 2.0)])
def test_constant_weight_converges_to_the_dct_solution(h, w, c):
    g = synth.rng(61)
    P = g.random((2, h, w))
    A = g.random((2, h, w))
    wc = np.full((h, w), c)
    O = oracle.poisson_solve(P, A, wc, eta=0.15, kappa=0.2, iters=4000)
    ky = 2 - 2 * np.cos(np.pi * np.arange(h) / h)
    kx = 2 - 2 * np.cos(np.pi * np.arange(w) / w)
    lam = ky[:, None] + kx[None, :]
    for ch in range(2):
        # right-hand side Lg P + c A; Lg is diagonal on the DCT-II basis
        rhs = idctn(lam * dctn(P[ch], type=2, norm="ortho"), type=2, norm="ortho") + c * A[ch]
        exact = idctn(dctn(rhs, type=2, norm="ortho") / (lam + c), type=2, norm="ortho")
        assert np.abs(O[ch] - exact).max() <= 1e-9


def test_fixed_points():
    g = synth.rng(62)
    P = g.random((3, 10, 12))
    wc = g.uniform(0, 3, (10, 12))
    assert np.array_equal(oracle.poisson_solve(P, P, wc, iters=50), P)
    A = g.random((3, 10, 12))
    assert np.allclose(oracle.poisson_solve(P, P, np.zeros((10, 12)), iters=50), P, atol=0, rtol=0)
    assert not np.allclose(oracle.poisson_solve(P, A, wc, iters=50), P)


def test_first_iteration_has_no_momentum():
    g = synth.rng(63)
    P, A = g.random((2, 1, 8, 9))
    wc = g.uniform(0, 2, (8, 9))
    O1 = oracle.poisson_solve(P, A, wc, eta=0.15, kappa=0.2, iters=1)
    want = A[0] - 0.15 * oracle.poisson_grad(A[0], P[0], A[0], wc)
    assert np.abs(O1[0] - want).max() <= 1e-15

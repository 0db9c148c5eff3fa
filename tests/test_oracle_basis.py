"""Pins for the oracle's reference-element tools (Section 3.1 / Section 3.4 footnote)."""
import numpy as np
import pytest

from oracle import basis


@pytest.mark.parametrize("n", range(1, 9))
def test_gauss_legendre_matches_library(n):
    x, w = basis.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, xr, rtol=0, atol=2e-15)
    assert np.allclose(w, wr, rtol=0, atol=2e-15)


@pytest.mark.parametrize("n", range(1, 7))
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    x, w = basis.gauss_legendre(n)
    for p in range(2 * n):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert np.sum(w * x ** p) == pytest.approx(exact, abs=1e-14)
    p = 2 * n
    assert abs(np.sum(w * x ** p) - 2.0 / (p + 1)) > 1e-6      # not exact beyond


@pytest.mark.parametrize("k", range(1, 6))
def test_lagrange_interpolation_and_derivative_exact(k):
    x, _ = basis.gauss_legendre(k + 1)
    assert np.allclose(basis.lagrange_matrix(x, x), np.eye(k + 1), atol=1e-14)
    xe = np.array([-1.0, -0.3, 0.4, 1.0])
    Lm = basis.lagrange_matrix(x, xe)
    Dm = basis.lagrange_derivative_matrix(x, xe)
    for p in range(k + 1):
        assert np.allclose(Lm @ x ** p, xe ** p, atol=1e-13)
        dp = p * xe ** (p - 1) if p else 0 * xe
        assert np.allclose(Dm @ x ** p, dp, atol=1e-12)
    # partition of unity
    assert np.allclose(Lm.sum(axis=1), 1.0, atol=1e-14)
    assert np.allclose(Dm.sum(axis=1), 0.0, atol=1e-12)


def test_diagonal_mass_matrix():
    # Section 3.3: the mass matrix is diagonal for the right basis; with the
    # Lagrange basis at the k+1 Gauss points the (k+1)-point rule is exact for
    # the degree-2k products, so M = diag(w).
    k = 4
    x, w = basis.gauss_legendre(k + 1)
    xf, wf = basis.gauss_legendre(k + 4)
    Lf = basis.lagrange_matrix(x, xf)
    M = (Lf * wf[:, None]).T @ Lf
    assert np.allclose(M, np.diag(w), atol=1e-14)

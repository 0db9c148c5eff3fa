"""One-dimensional Gauss-Legendre rule and Lagrange basis on [-1, 1].

Section 3.1 (discrete space Q^k on hexahedra / quadrilaterals) and the
footnote in Section 3.4 (products of Gauss-Legendre rules).  The paper's
NGSolve space uses an orthogonal Legendre basis with a diagonal mass matrix;
the same space is spanned here by the Lagrange polynomials through the k+1
Gauss-Legendre points, whose mass matrix under the (k+1)-point rule is
exactly diagonal (the rule is exact to degree 2k+1 >= 2k).
"""
import numpy as np


def legendre(n, x):
    """P_n(x) and P_n'(x) by the three-term (Bonnet) recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for j in range(2, n + 1):
        p0, p1 = p1, ((2 * j - 1) * x * p1 - (j - 1) * p0) / j
    # derivative: (1 - x^2) P_n' = n (P_{n-1} - x P_n)
    dp = n * (p0 - x * p1) / (1.0 - x * x)
    return p1, dp


def gauss_legendre(n):
    """Nodes (ascending) and weights of the n-point Gauss-Legendre rule.

    Nodes are the roots of P_n, found by Newton's method from the usual
    cosine initial guesses; weights are 2 / ((1 - x^2) P_n'(x)^2).
    """
    i = np.arange(n)
    x = -np.cos(np.pi * (i + 0.75) / (n + 0.5))
    for _ in range(100):
        p, dp = legendre(n, x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p, dp = legendre(n, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    return x, w


def lagrange_matrix(nodes, x):
    """L[i, a] = l_a(x_i): Lagrange polynomial through ``nodes`` number a at x_i."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    L = np.ones((x.size, n))
    for a in range(n):
        for m in range(n):
            if m != a:
                L[:, a] *= (x - nodes[m]) / (nodes[a] - nodes[m])
    return L


def lagrange_derivative_matrix(nodes, x):
    """D[i, a] = l_a'(x_i), by the product rule over the factors of l_a."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    D = np.zeros((x.size, n))
    for a in range(n):
        for m in range(n):
            if m == a:
                continue
            term = np.full(x.size, 1.0 / (nodes[a] - nodes[m]))
            for l in range(n):
                if l != a and l != m:
                    term *= (x - nodes[l]) / (nodes[a] - nodes[l])
            D[:, a] += term
    return D

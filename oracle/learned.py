"""Learned facet-patch smoother of the oracle (reference for the GPU kernels).

Test infrastructure only (see the package docstring).  The paper has no
learned component; this extends the method beyond the paper, written plainly so the
GPU forward and backward kernels can be checked against it.

For a trace residual r, every facet e gets the features
    X_e = (r_e, r_n1, r_n2, r_n3, r_n4) / s_e,   s_e = RMS of those 5(p+1) values,
(its own p+1 values first, then the four facets that share a cell with it, in
the library's neighbour order), a two-hidden-layer tanh network
    y_e = W3 tanh(W2 tanh(W1 X_e + b1) + b2) + b3 + omega * X_e[:p+1]
and the correction c_e = D_e^-1 (s_e y_e) (D_e the facet diagonal block of S).
The correction is positively homogeneous in r, and with zero weights it is
the damped block-Jacobi step.  Training minimises the residual left after it,
    L = mean_b || r_b - S c(r_b) ||^2 / || r_b ||^2 .
"""
from __future__ import annotations

import numpy as np


def param_shapes(n_in: int, hid: int, n_out: int):
    return [("W1", (hid, n_in)), ("b1", (hid,)), ("W2", (hid, hid)), ("b2", (hid,)),
            ("W3", (n_out, hid)), ("b3", (n_out,))]


def unpack(theta: np.ndarray, n_in: int, hid: int, n_out: int) -> dict:
    out, k = {}, 0
    for name, shp in param_shapes(n_in, hid, n_out):
        size = int(np.prod(shp))
        out[name] = theta[k:k + size].reshape(shp)
        k += size
    return out


def n_params(n_in: int, hid: int, n_out: int) -> int:
    return sum(int(np.prod(s)) for _, s in param_shapes(n_in, hid, n_out))


def features(r: np.ndarray, nbr: np.ndarray, pp: int):
    """X [NF, 5 pp] and s [NF] for a residual in the facet-major layout [NF*pp]."""
    R = r.reshape(-1, pp)
    X = np.concatenate([R[:, None, :], R[nbr]], axis=1).reshape(R.shape[0], 5 * pp)
    s = np.sqrt(np.mean(X ** 2, axis=1)) + 1e-30
    return X / s[:, None], s


def forward(theta, X, hid, pp, omega):
    P = unpack(theta, X.shape[1], hid, pp)
    a1 = X @ P["W1"].T + P["b1"]
    h1 = np.tanh(a1)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.tanh(a2)
    y = h2 @ P["W3"].T + P["b3"] + omega * X[:, :pp]
    return y, (X, a1, h1, a2, h2)


def correction(theta, r, nbr, Dinv_blocks, hid, pp, omega):
    X, s = features(r, nbr, pp)
    y, _ = forward(theta, X, hid, pp, omega)
    c = np.einsum("eij,ej->ei", Dinv_blocks, s[:, None] * y)
    return c.ravel()


def loss_and_grad(theta, R, S, nbr, Dinv_blocks, hid, pp, omega):
    """Mean relative residual after the correction over the rows of R, and its
    gradient with respect to theta (hand-written backward pass)."""
    g = np.zeros_like(theta)
    total = 0.0
    St = S.T.tocsr()
    for r in R:
        X, s = features(r, nbr, pp)
        y, (X_, a1, h1, a2, h2) = forward(theta, X, hid, pp, omega)
        c = np.einsum("eij,ej->ei", Dinv_blocks, s[:, None] * y).ravel()
        rn = r - S @ c
        rr = r @ r
        total += (rn @ rn) / rr
        gc = (-2.0 / rr) * (St @ rn)                                   # dL/dc
        gy = s[:, None] * np.einsum("eji,ej->ei", Dinv_blocks, gc.reshape(-1, pp))  # D^-T
        P = unpack(theta, X.shape[1], hid, pp)
        gW3 = gy.T @ h2
        gb3 = gy.sum(0)
        gh2 = gy @ P["W3"]
        ga2 = gh2 * (1.0 - h2 ** 2)
        gW2 = ga2.T @ h1
        gb2 = ga2.sum(0)
        gh1 = ga2 @ P["W2"]
        ga1 = gh1 * (1.0 - h1 ** 2)
        gW1 = ga1.T @ X
        gb1 = ga1.sum(0)
        g += np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return total / len(R), g / len(R)


def library_neighbours(prob) -> np.ndarray:
    """Neighbour facets in the library's order: for facet e, its two cells in
    order of first appearance, and in each cell the facets of local edges
    (i+1) % 3 and (i+2) % 3 (i the local edge of e)."""
    nbr = np.zeros((prob.n_facets, 4), dtype=np.int64)
    seen = {}
    for K in range(prob.N):
        for i in range(3):
            e = int(prob.facet_of[K, i])
            side = seen.get(e, 0)
            seen[e] = side + 1
            for k in range(2):
                nbr[e, 2 * side + k] = prob.facet_of[K, (i + 1 + k) % 3]
    return nbr

"""Independent reference solutions used to pin the oracle (not the oracle).

* Riccati matrix of the linear-quadratic HJ equation (closed form through a
  matrix exponential, cross-checked by an ODE integrator in the tests).
* Lax-Friedrichs monotone grid scheme (the paper's d=2 comparison, Sec. 5).
* Classical Hopf formula for state-independent H (Sec. 3.4, Example 1),
  solved coordinate by coordinate by brute force when it separates.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def riccati_P(A: np.ndarray, B: np.ndarray, t: float) -> np.ndarray:
    """P(t) for phi = x^T P x / 2 solving phi_t + <Ax, grad phi> + |B^T grad phi|^2/2 = 0,
    phi(x,0) = |x|^2/2, i.e. P' = -(A^T P + P A) - P B B^T P, P(0) = I.
    Linear-fractional form: P = Y X^{-1} with [X; Y]' = [[A, BB^T], [0, -A^T]] [X; Y],
    X(0) = Y(0) = I."""
    d = A.shape[0]
    M = np.block([[A, B @ B.T], [np.zeros((d, d)), -A.T]])
    E = scipy.linalg.expm(t * M)
    XY = E @ np.vstack([np.eye(d), np.eye(d)])
    X, Y = XY[:d], XY[d:]
    return Y @ np.linalg.inv(X)


def lax_friedrichs(H, alpha, g, lo, hi, dx, t, d, cfl=0.9):
    """First-order Lax-Friedrichs scheme for phi_t + H(x, grad phi) = 0 on the
    box [lo, hi]^d (d = 1 or 2), linear extrapolation at the boundary.

    H(X, P) takes a list of coordinate grids X and gradient components P and
    returns the Hamiltonian on the grid; alpha bounds |dH/dp_i|.
    Returns (grids, phi(., t))."""
    n = int(round((hi - lo) / dx)) + 1
    xs = np.linspace(lo, hi, n)
    dx = xs[1] - xs[0]
    X = np.meshgrid(*([xs] * d), indexing="ij")
    phi = g(X)
    dt = cfl * dx / (d * alpha)
    steps = int(np.ceil(t / dt))
    dt = t / steps
    for _ in range(steps):
        pad = np.pad(phi, 1, mode="edge")
        # linear extrapolation into the ghost layer
        for ax in range(d):
            sl_lo = [slice(1, -1)] * d
            sl_lo[ax] = slice(0, 1)
            a0 = [slice(1, -1)] * d
            a0[ax] = slice(1, 2)
            a1 = [slice(1, -1)] * d
            a1[ax] = slice(2, 3)
            pad[tuple(sl_lo)] = 2 * pad[tuple(a0)] - pad[tuple(a1)]
            sl_hi = [slice(1, -1)] * d
            sl_hi[ax] = slice(-1, None)
            b0 = [slice(1, -1)] * d
            b0[ax] = slice(-2, -1)
            b1 = [slice(1, -1)] * d
            b1[ax] = slice(-3, -2)
            pad[tuple(sl_hi)] = 2 * pad[tuple(b0)] - pad[tuple(b1)]
        P = []
        visc = np.zeros_like(phi)
        for ax in range(d):
            fwd = [slice(1, -1)] * d
            fwd[ax] = slice(2, None)
            bwd = [slice(1, -1)] * d
            bwd[ax] = slice(0, -2)
            up, dn = pad[tuple(fwd)], pad[tuple(bwd)]
            P.append((up - dn) / (2 * dx))
            visc += alpha * (up - 2 * phi + dn) / (2 * dx)
        phi = phi - dt * (H(X, P) - visc)
    return xs, phi


def separable_hopf_min(sig2: float, e: float, t: float, x: float, s_eps: float) -> float:
    """min over v of sig2 v^2/2 + t e sqrt(v^2 + s_eps) - x v by a dense grid
    (spacing 1e-4 on [-12, 12], finer near the kink) followed by Newton
    polishing inside the bracketing cell."""
    f = lambda v: 0.5 * sig2 * v * v + t * e * np.sqrt(v * v + s_eps) - x * v
    grid = np.concatenate([np.linspace(-12, 12, 240001), np.linspace(-0.01, 0.01, 20001)])
    vals = f(grid)
    v = grid[np.argmin(vals)]
    for _ in range(60):
        s = np.sqrt(v * v + s_eps)
        d1 = sig2 * v + t * e * v / s - x
        d2 = sig2 + t * e * s_eps / s ** 3
        if d2 <= 0:
            break
        nv = v - d1 / d2
        if abs(nv - v) < 1e-15:
            v = nv
            break
        v = nv
    return float(min(f(v), vals.min()))

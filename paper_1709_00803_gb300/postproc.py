"""Host-side analysis of converged fields (not part of the iteration): stream function,
vorticity and vortex centres of a lid-driven cavity on a uniform n x n quad mesh, as the
paper reports them for its first test (Table 1)."""
from __future__ import annotations

import numpy as np


def _grid(W, n):
    rho = W[0].reshape(n, n)
    return W[1].reshape(n, n) / rho, W[2].reshape(n, n) / rho     # [row j (y), column i (x)]


def stream_function(W, n):
    """psi at the cell centres, psi = integral of u dy from the bottom wall (psi = 0 there),
    by the midpoint rule per cell (cells of the uniform n x n mesh, row-major from the
    bottom-left)."""
    u, _ = _grid(W, n)
    h = 1.0 / n
    return (np.cumsum(u, axis=0) - 0.5 * u) * h


def vorticity(W, n):
    """omega = dv/dx - du/dy at the cell centres (central differences inside, one-sided
    at the walls)."""
    u, v = _grid(W, n)
    h = 1.0 / n
    return np.gradient(v, h, axis=1) - np.gradient(u, h, axis=0)


def _extremum(f, n, mask, sign):
    """Sub-cell location and value of the extremum of a cell-centred field inside mask, by a
    quadratic fit over the 3 x 3 cells around the extreme cell."""
    g = np.where(mask, sign * f, -np.inf)
    j, i = np.unravel_index(np.argmax(g), g.shape)
    j = min(max(j, 1), n - 2); i = min(max(i, 1), n - 2)
    h = 1.0 / n
    ys, xs = (np.arange(n) + 0.5) * h, (np.arange(n) + 0.5) * h
    A, b = [], []
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            x, y = xs[i + di] - xs[i], ys[j + dj] - ys[j]
            A.append([1.0, x, y, x * x, x * y, y * y]); b.append(f[j + dj, i + di])
    c = np.linalg.lstsq(np.array(A), np.array(b), rcond=None)[0]
    H = np.array([[2 * c[3], c[4]], [c[4], 2 * c[5]]])
    d = np.linalg.solve(H, -c[1:3])
    if np.max(np.abs(d)) > 1.5 * h:   # flat or saddle: keep the cell centre
        d = np.zeros(2)
    val = c[0] + c[1] * d[0] + c[2] * d[1] + c[3] * d[0] ** 2 + c[4] * d[0] * d[1] + c[5] * d[1] ** 2
    return val, xs[i] + d[0], ys[j] + d[1]


def _bilinear(f, n, x, y):
    h = 1.0 / n
    fx, fy = x / h - 0.5, y / h - 0.5
    i0, j0 = int(np.clip(np.floor(fx), 0, n - 2)), int(np.clip(np.floor(fy), 0, n - 2))
    a, b = fx - i0, fy - j0
    return ((1 - a) * (1 - b) * f[j0, i0] + a * (1 - b) * f[j0, i0 + 1] +
            (1 - a) * b * f[j0 + 1, i0] + a * b * f[j0 + 1, i0 + 1])


def cavity_vortices(W, n):
    """Primary vortex (minimum of psi; |omega| there), and the left and right secondary
    vortices of the bottom corners (maxima of psi), in the units of Table 1."""
    psi, om = stream_function(W, n), vorticity(W, n)
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(c, c)
    p_val, px, py = _extremum(psi, n, np.ones_like(psi, dtype=bool), -1.0)
    l_val, lx, ly = _extremum(psi, n, (X < 0.35) & (Y < 0.35), 1.0)
    r_val, rx, ry = _extremum(psi, n, (X > 0.6) & (Y < 0.45), 1.0)
    return dict(primary=dict(omega=abs(_bilinear(om, n, px, py)), psi=p_val, x=px, y=py),
                left=dict(psi=l_val, x=lx, y=ly), right=dict(psi=r_val, x=rx, y=ry))

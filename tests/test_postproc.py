"""The cavity analysis (stream function, vorticity, vortex centre) on analytic fields."""
import numpy as np

from paper_1709_00803_gb300 import postproc as P


def _fields_from_psi(n, psi_fn, dpsi_dx, dpsi_dy):
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(c, c)
    u, v = dpsi_dy(X, Y), -dpsi_dx(X, Y)
    W = np.zeros((5, n * n))
    W[0] = 1.0 + 0.01 * X.ravel()
    W[1] = W[0] * u.ravel()
    W[2] = W[0] * v.ravel()
    return W, X, Y


def test_single_vortex_centre_and_vorticity():
    # psi = -A sin(pi x) sin(pi y): centre (0.5, 0.5), psi_min = -A, omega = -lap psi = -2 pi^2 A
    n, A = 100, 0.1
    W, X, Y = _fields_from_psi(n, None,
                               lambda x, y: -A * np.pi * np.cos(np.pi * x) * np.sin(np.pi * y),
                               lambda x, y: -A * np.pi * np.sin(np.pi * x) * np.cos(np.pi * y))
    r = P.cavity_vortices(W, n)["primary"]
    assert abs(r["x"] - 0.5) < 2e-3 and abs(r["y"] - 0.5) < 2e-3
    assert abs(r["psi"] + A) < 1e-3 * A
    assert abs(r["omega"] - 2 * np.pi ** 2 * A) < 2e-3 * 2 * np.pi ** 2 * A


def test_off_centre_vortex_location():
    n, A, x0, y0 = 80, 0.05, 0.53, 0.57
    # a smooth bump with its minimum at (x0, y0): psi = -A exp(-((x-x0)^2 + (y-y0)^2) / 0.02)
    s2 = 0.02
    W, X, Y = _fields_from_psi(n, None,
                               lambda x, y: A * 2 * (x - x0) / s2 * np.exp(-((x - x0) ** 2 + (y - y0) ** 2) / s2),
                               lambda x, y: A * 2 * (y - y0) / s2 * np.exp(-((x - x0) ** 2 + (y - y0) ** 2) / s2))
    r = P.cavity_vortices(W, n)["primary"]
    # psi from u by the midpoint rule starts from 0 at y = 0, so it is offset by psi(x, 0)
    assert abs(r["x"] - x0) < 3e-3 and abs(r["y"] - y0) < 3e-3

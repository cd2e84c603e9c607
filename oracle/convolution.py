"""Heat convolution vs explicit matrix convolution on S^2 (oracle, FP64).
Test infrastructure only.

Paper, App. "Convolution on S^2": the matrix convolution applies the unnormalised
geodesic Gibbs kernel K_eps(x, y) = exp(-d(x, y)^2 / eps), whose integral over the
sphere is C(eps) = int exp(-d(x, y)^2 / eps) dsigma(y); by Varadhan's formula the heat
kernel at t = eps/4 is close to K_eps / C(eps), so the heat output is rescaled by C(eps)
before the mean absolute error between the two convolutions is taken.

Discrete forms (App. C.2 area weights a): (K f)_i = sum_j a_j exp(-d_ij^2 / eps) f_j and
(H f)_i the heat convolution of the oracle's SHT; MAE = mean_i |C(eps) (H f)_i - (K f)_i|
(unweighted mean over the grid nodes).
"""
import numpy as np
from scipy import integrate

from . import sht


def geodesic(X, Y):
    """Great-circle distance between unit vectors, atan2(|x cross y|, x . y): accurate
    near 0 and pi, where arccos of the dot product is not."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    c = np.cross(X, Y)
    return np.arctan2(np.linalg.norm(c, axis=-1), np.sum(X * Y, axis=-1))


def gibbs_normaliser(eps):
    """C(eps) = int_{S^2} exp(-d(x, y)^2 / eps) dsigma(y) = 2 pi int_0^pi exp(-theta^2/eps) sin(theta) dtheta
    (rotation invariance: polar coordinates about x)."""
    f = lambda th: np.exp(-th * th / eps) * np.sin(th)
    # the mass sits within a few sqrt(eps) of 0: split there so quad sees the peak
    cut = min(np.pi, 12.0 * np.sqrt(eps))
    v1, _ = integrate.quad(f, 0.0, cut, epsabs=0.0, epsrel=1e-13, limit=200)
    v2 = 0.0
    if cut < np.pi:
        v2, _ = integrate.quad(f, cut, np.pi, epsabs=0.0, epsrel=1e-13, limit=200)
    return 2.0 * np.pi * (v1 + v2)


def gibbs_apply(grid, f, eps, rows=1024):
    """(K f)_i = sum_j a_j exp(-d_ij^2 / eps) f_j for fields f[..., nlat, nlon], row-blocked."""
    X = grid.xyz.reshape(-1, 3)
    a = grid.a.reshape(-1)
    shp = f.shape
    F = np.asarray(f, dtype=np.float64).reshape(-1, X.shape[0]) * a[None, :]
    out = np.empty_like(F)
    for r0 in range(0, X.shape[0], rows):
        d = geodesic(X[r0:r0 + rows, None, :], X[None, :, :])
        out[:, r0:r0 + rows] = F @ np.exp(-d * d / eps).T
    return out.reshape(shp)


def conv_mae(grid, f, eps):
    """Mean absolute error between C(eps) * heat convolution at t = eps/4 and the matrix
    convolution, per field."""
    h = grid.heat_apply(f, eps / 4.0) if hasattr(grid, "heat_apply") else sht.heat_apply(grid, f, eps / 4.0)
    k = gibbs_apply(grid, f, eps)
    d = np.abs(gibbs_normaliser(eps) * h - k)
    return d.reshape(d.shape[:-2] + (-1,)).mean(axis=-1)

"""Dense heat matrix on tiny grids (oracle, FP64).  Test infrastructure only.

Truncated heat kernel on S^2 (Sec. 3.1-3.2: -Delta Y_lm = l(l+1) Y_lm, so the
heat semigroup acts by exp(-t l(l+1)) on degree l) summed by the addition
theorem sum_m Y_lm(x) conj(Y_lm(y)) = (2l+1)/(4 pi) P_l(<x, y>):

  H^L_t(x, y) = sum_{l<=lmax} (2l+1)/(4 pi) exp(-t l(l+1)) P_l(<x, y>).

With area weights a (App. C.2), the discrete operator is K = H diag(a):
(K v)_i = sum_j H(x_i, x_j) a_j v_j, which is the quadrature form of the kernel
convolution eq. (kernel-conv).
"""
import numpy as np

from .legendre import legendre_series


def heat_matrix(grid, t):
    """H[i, j] over flattened nodes (row-major [nlat, nlon]); n x n, n <= ~5000."""
    X = grid.xyz.reshape(-1, 3)
    z = np.clip(X @ X.T, -1.0, 1.0)
    H = np.zeros_like(z)
    for l, Pl in enumerate(legendre_series(grid.lmax, z)):
        H += (2 * l + 1) / (4.0 * np.pi) * np.exp(-t * l * (l + 1.0)) * Pl
    return H


def kernel_matrix(grid, t):
    """K = H diag(a), so that K @ v.ravel() is the discrete heat convolution."""
    return heat_matrix(grid, t) * grid.a.reshape(1, -1)


def dense_apply(K, f):
    """Apply a dense K to fields f[..., nlat, nlon]."""
    shp = f.shape
    return (f.reshape(-1, shp[-2] * shp[-1]) @ K.T).reshape(shp)

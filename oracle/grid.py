"""Gauss-Legendre grid on S^2 (oracle, FP64).  Test infrastructure only.

Paper: App. C.1 "Gauss-Legendre": the latitudinal samples are the roots of the
Legendre polynomial P_nlat; longitudes are equispaced.  App. C.2: area weights
a with a^T 1 = 4 pi, so that int f dsigma ~ a^T f.

Conventions (a reading, the paper fixes none): ring j runs north -> south, so
x_j = cos(theta_j) is DESCENDING; column k has phi_k = 2 pi k / nlon.  The area
weight of every node of ring j is a_j = w_j * 2 pi / nlon with w_j the GL
weight (sum w = 2).
"""
import numpy as np


def legendre_p_and_dp(n, x):
    """P_n(x) and P_n'(x) by Bonnet's three-term recurrence (textbook)."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    if n == 0:
        return p_prev, np.zeros_like(x)
    p = x.copy()
    for l in range(2, n + 1):
        p_prev, p = p, ((2 * l - 1) * x * p - (l - 1) * p_prev) / l
    # (1 - x^2) P_n'(x) = n (P_{n-1}(x) - x P_n(x))
    dp = n * (p_prev - x * p) / (1.0 - x * x)
    return p, dp


def gauss_legendre(nlat):
    """Nodes x_j (descending) and weights w_j of nlat-point GL quadrature.

    Newton's method on P_nlat from the classical initial guess
    cos(pi (k - 1/4) / (nlat + 1/2)); weights w = 2 / ((1 - x^2) P'(x)^2).
    """
    if nlat < 1:
        raise ValueError("nlat must be >= 1")
    k = np.arange(1, nlat + 1, dtype=np.float64)
    x = np.cos(np.pi * (k - 0.25) / (nlat + 0.5))
    for _ in range(100):
        p, dp = legendre_p_and_dp(nlat, x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-15:
            break
    p, dp = legendre_p_and_dp(nlat, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    return x, w


class Grid:
    """An nlat x nlon Gauss-Legendre grid, degrees 0..lmax (default nlat-1)."""

    def __init__(self, nlat, nlon=None, lmax=None):
        self.nlat = int(nlat)
        self.nlon = int(nlon) if nlon is not None else 2 * self.nlat
        self.lmax = int(lmax) if lmax is not None else self.nlat - 1
        if self.nlon < 2 * self.lmax + 1:
            raise ValueError("nlon must be >= 2*lmax+1")
        self.x, self.w = gauss_legendre(self.nlat)
        self.theta = np.arccos(self.x)
        self.phi = 2.0 * np.pi * np.arange(self.nlon) / self.nlon
        self.a_ring = self.w * (2.0 * np.pi / self.nlon)
        self._pbar = None

    @property
    def n(self):
        return self.nlat * self.nlon

    @property
    def a(self):
        """Area weight of every node, shape [nlat, nlon]."""
        return np.repeat(self.a_ring[:, None], self.nlon, axis=1)

    @property
    def xyz(self):
        """Unit vectors of the nodes, shape [nlat, nlon, 3]."""
        st = np.sqrt(1.0 - self.x * self.x)
        return np.stack([np.outer(st, np.cos(self.phi)),
                         np.outer(st, np.sin(self.phi)),
                         np.outer(self.x, np.ones(self.nlon))], axis=-1)

    @property
    def lat_deg(self):
        return 90.0 - np.degrees(self.theta)

    def pbar(self):
        """Cached orthonormal associated Legendre table (see legendre.pbar)."""
        if self._pbar is None:
            from .legendre import pbar
            self._pbar = pbar(self.lmax, self.x)
        return self._pbar

"""Iso-latitude grids on S^2 (oracle, FP64).  Test infrastructure only.

Paper: App. C.1 "Gauss-Legendre": the latitudinal samples are the roots of the
Legendre polynomial P_nlat; "Equiangular ... Clenshaw-Curtis": equally spaced
colatitudes including both poles, weighted by Clenshaw-Curtis quadrature (the
paper's main runtime grid, Sec. 4.1); longitudes are equispaced in both.
App. C.2: area weights a with a^T 1 = 4 pi, so that int f dsigma ~ a^T f.

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


def clenshaw_curtis(nlat):
    """Nodes x_j = cos(pi j / N), N = nlat - 1 (descending, both poles included),
    and the Clenshaw-Curtis weights, from their definition: integrate the
    degree-N polynomial that interpolates f at the nodes.

    In the Chebyshev basis the interpolant is sum''_k c_k T_k(x) with
    c_k = (2/N) sum''_j f_j cos(k j pi / N) (a double prime halves the first and
    last terms), and int_{-1}^{1} T_k = 2/(1 - k^2) for even k, 0 for odd k.
    Collecting the coefficient of f_j gives w_j.  Exact for polynomials of
    degree <= N.
    """
    if nlat < 2:
        raise ValueError("a Clenshaw-Curtis grid needs nlat >= 2")
    N = nlat - 1
    j = np.arange(N + 1)
    x = np.cos(np.pi * j / N)
    x[N - j[: (N + 1) // 2]] = -x[j[: (N + 1) // 2]]     # exact mirror symmetry
    if N % 2 == 0:
        x[N // 2] = 0.0
    half = np.where((j == 0) | (j == N), 0.5, 1.0)
    w = np.zeros(N + 1)
    for k in range(0, N + 1, 2):
        ck = (2.0 / N) * half * np.cos(np.pi * ((k * j) % (2 * N)) / N)   # d c_k / d f_j
        wk = 0.5 if k in (0, N) else 1.0
        w += wk * ck * (2.0 / (1.0 - k * k))
    w = 0.5 * (w + w[::-1])      # symmetric in exact arithmetic; make it so bitwise
    return x, w


QUADRATURES = {"gl": gauss_legendre, "cc": clenshaw_curtis}


class Grid:
    """An nlat x nlon iso-latitude grid, degrees 0..lmax (default nlat-1).

    quadrature: "gl" (Gauss-Legendre) or "cc" (equiangular, Clenshaw-Curtis).
    """

    def __init__(self, nlat, nlon=None, lmax=None, quadrature="gl"):
        self.nlat = int(nlat)
        self.nlon = int(nlon) if nlon is not None else 2 * self.nlat
        self.lmax = int(lmax) if lmax is not None else self.nlat - 1
        if self.nlon < 2 * self.lmax + 1:
            raise ValueError("nlon must be >= 2*lmax+1")
        self.quadrature = quadrature
        self.x, self.w = QUADRATURES[quadrature](self.nlat)
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

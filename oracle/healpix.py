"""HEALPix grid and its semi-naive SHT (oracle, FP64).  Test infrastructure only.

Paper App. C.1 ("HEALPix"): N = 12 Nside^2 equal-area pixels on iso-latitude rings,
without an exact sampling theorem; the paper's climate study uses Nside = 64.  The
pixel centres follow the HEALPix construction (Gorski et al. 2005), rings i = 1 .. 4 Nside - 1
from north to south:
  polar cap, i < Nside:   z = 1 - i^2 / (3 Nside^2),   4 i pixels,
                          phi_j = pi (j + 1/2) / (2 i),                 j = 0 .. 4i - 1;
  equatorial belt, Nside <= i <= 3 Nside:
                          z = 4/3 - 2 i / (3 Nside),   4 Nside pixels,
                          phi_j = pi (j + 1 - s/2) / (2 Nside),  s = (i - Nside + 1) mod 2;
  south cap: the mirror image (z -> -z, same ring lengths and longitudes).
Every pixel has area a = 4 pi / N (App. C.2 area weights).

Fields are flat arrays of the N pixels in ring order, kept here with shape [..., 1, N] so
that the oracle's Sinkhorn (which sums over the last two axes) runs unchanged.

The SHT is the same semi-naive transform as on the other iso-latitude grids, with each
ring's own length and longitude offset (App. C.1, last paragraph):
  F_m(i) = sum_j f_ij e^{-i m phi_ij},   c_lm = sum_i a Pbar_lm(z_i) F_m(i),
  f_ij   = g_0(i) + 2 Re sum_{m>=1} g_m(i) e^{i m phi_ij},   g_m(i) = sum_l Pbar_lm(z_i) c_lm.
It is not an exact inverse (no sampling theorem), but the heat operator it defines is
H diag(a) by the addition theorem, like on every other node set.
"""
import numpy as np

from .legendre import pbar as _pbar
from .sht import heat_multipliers


def ring_geometry(nside):
    """z, number of pixels and longitude of pixel 0 of every ring (north to south)."""
    nr = 4 * nside - 1
    z = np.empty(nr)
    npx = np.empty(nr, dtype=np.int64)
    phi0 = np.empty(nr)
    for i in range(1, nr + 1):
        k = i if i <= 2 * nside else nr + 1 - i     # ring index mirrored into the north half
        if k < nside:
            zk, nk, p0 = 1.0 - k * k / (3.0 * nside * nside), 4 * k, np.pi / (4.0 * k)
        else:
            s = (k - nside + 1) % 2
            zk, nk, p0 = 4.0 / 3.0 - 2.0 * k / (3.0 * nside), 4 * nside, np.pi * (1.0 - s / 2.0) / (2.0 * nside)
        z[i - 1] = zk if i <= 2 * nside else -zk
        npx[i - 1] = nk
        phi0[i - 1] = p0
    z[2 * nside - 1] = 0.0   # the equator ring
    return z, npx, phi0


class HealpixGrid:
    """HEALPix grid of resolution nside, degrees 0..lmax (default 3 nside - 1)."""

    def __init__(self, nside, lmax=None):
        self.nside = int(nside)
        self.lmax = int(lmax) if lmax is not None else 3 * self.nside - 1
        self.z, self.npx, self.phi0 = ring_geometry(self.nside)
        self.nrings = len(self.z)
        self.off = np.concatenate([[0], np.cumsum(self.npx)])
        self.npix = int(self.off[-1])
        self.ring_of = np.repeat(np.arange(self.nrings), self.npx)
        j = np.arange(self.npix) - self.off[self.ring_of]
        self.phi = self.phi0[self.ring_of] + 2.0 * np.pi * j / self.npx[self.ring_of]
        self.area = 4.0 * np.pi / self.npix
        self._pbar = None

    @property
    def a(self):
        return np.full((1, self.npix), self.area)

    @property
    def lat_deg(self):
        """Latitude of every pixel in degrees, shape [1, npix] (the rings are iso-latitude)."""
        return (90.0 - np.degrees(np.arccos(self.z[self.ring_of])))[None]

    @property
    def xyz(self):
        zz = self.z[self.ring_of]
        st = np.sqrt((1.0 - zz) * (1.0 + zz))
        return np.stack([st * np.cos(self.phi), st * np.sin(self.phi), zz], axis=-1)[None]

    def pbar(self):
        if self._pbar is None:
            self._pbar = _pbar(self.lmax, self.z)
        return self._pbar

    # ---- semi-naive SHT (direct sums per ring) ------------------------------------
    def ring_dft(self, f):
        """F[..., i, m] for m = 0..lmax from flat fields f[..., 1, N]."""
        f = np.asarray(f, dtype=np.float64)[..., 0, :]
        m = np.arange(self.lmax + 1)
        F = np.zeros(f.shape[:-1] + (self.nrings, self.lmax + 1), dtype=np.complex128)
        for i in range(self.nrings):
            s = slice(self.off[i], self.off[i + 1])
            E = np.exp(-1j * np.outer(self.phi[s], m))          # [pixels, m]
            F[..., i, :] = f[..., s] @ E
        return F

    def ring_idft(self, g):
        """Flat real field [..., 1, N] from g[..., i, m] (m = 0..lmax)."""
        m = np.arange(self.lmax + 1)
        wm = np.where(m == 0, 1.0, 2.0)
        out = np.zeros(g.shape[:-2] + (self.npix,))
        for i in range(self.nrings):
            s = slice(self.off[i], self.off[i + 1])
            E = np.exp(1j * np.outer(m, self.phi[s])) * wm[:, None]   # [m, pixels]
            out[..., s] = (g[..., i, :] @ E).real
        return out[..., None, :]

    def analysis(self, f):
        F = self.ring_dft(f)
        P = self.pbar()
        c = np.zeros(F.shape[:-2] + (self.lmax + 1, self.lmax + 1), dtype=np.complex128)
        for m in range(self.lmax + 1):
            A = P[m] * self.area
            Fm = F[..., :, m]
            c[..., m:, m] = Fm.real @ A.T + 1j * (Fm.imag @ A.T)
        return c

    def synthesis(self, c):
        P = self.pbar()
        g = np.zeros(c.shape[:-2] + (self.nrings, self.lmax + 1), dtype=np.complex128)
        for m in range(self.lmax + 1):
            cm = c[..., m:, m]
            g[..., :, m] = cm.real @ P[m] + 1j * (cm.imag @ P[m])
        return self.ring_idft(g)

    def heat_apply(self, f, t):
        c = self.analysis(f)
        c *= heat_multipliers(t, self.lmax)[:, None]
        return self.synthesis(c)

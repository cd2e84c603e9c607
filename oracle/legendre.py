"""Orthonormal associated Legendre functions (oracle, FP64).  Test infrastructure only.

Paper App. B "Spherical harmonics": Y_lm(theta, phi) = N_lm P_l^m(cos theta) e^{i m phi}
with N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), orthonormal on S^2.  We tabulate
Pbar_lm(x) = N_lm P_l^m(x) (Condon-Shortley phase included in P_l^m) with the
standard recurrences that follow from that definition:

  Pbar_00         = 1/sqrt(4 pi)
  Pbar_mm         = -sqrt((2m+1)/(2m)) sin(theta) Pbar_{m-1,m-1}
  Pbar_{m+1,m}    = sqrt(2m+3) x Pbar_mm
  Pbar_lm         = alpha_lm (x Pbar_{l-1,m} - beta_lm Pbar_{l-2,m}),
      alpha_lm = sqrt((4l^2-1)/(l^2-m^2)),  beta_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)).

Sectoral values that fall below the FP64 range flush to zero; at lmax <= 719 on a
GL grid the functions they seed stay below ~1e-200 everywhere, so this is exact
to double precision.
"""
import numpy as np


def pbar(lmax, x):
    """List P with P[m] of shape [lmax+1-m, len(x)]; row i holds l = m + i."""
    x = np.asarray(x, dtype=np.float64)
    sint = np.sqrt(1.0 - x * x)
    out = []
    pmm = np.full_like(x, 1.0 / np.sqrt(4.0 * np.pi))
    for m in range(lmax + 1):
        if m > 0:
            pmm = -np.sqrt((2.0 * m + 1.0) / (2.0 * m)) * sint * pmm
        tab = np.empty((lmax + 1 - m, x.size))
        tab[0] = pmm
        if m < lmax:
            tab[1] = np.sqrt(2.0 * m + 3.0) * x * pmm
        for l in range(m + 2, lmax + 1):
            alpha = np.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            beta = np.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
            tab[l - m] = alpha * (x * tab[l - m - 1] - beta * tab[l - m - 2])
        out.append(tab)
    return out


def legendre_series(lmax, z):
    """[P_0(z), ..., P_lmax(z)] (unnormalised Legendre polynomials), Bonnet recurrence."""
    z = np.asarray(z, dtype=np.float64)
    out = [np.ones_like(z)]
    if lmax >= 1:
        out.append(z.copy())
    for l in range(2, lmax + 1):
        out.append(((2 * l - 1) * z * out[-1] - (l - 1) * out[-2]) / l)
    return out

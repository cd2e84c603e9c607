"""Semi-naive spherical harmonic transform and heat convolution (oracle, FP64).

Test infrastructure only.

Paper App. C.1 (last paragraph): on iso-latitude grids the SHT is a DFT along
each longitude ring followed by a projection onto the associated Legendre
functions of each order m.  App. B defines F[f](l,m) = <f, Y_lm>; on the grid the
integral is the quadrature sum sum_{j,k} a_j f(theta_j, phi_k) conj(Y_lm):

  F_m(j)  = sum_k f_jk e^{-i m phi_k}                       (ring DFT)
  c_lm    = sum_j a_j Pbar_lm(x_j) F_m(j),   0 <= m <= l <= lmax

A real field has c_{l,-m} = (-1)^m conj(c_lm), so synthesis needs m >= 0 only:

  g_m(j)  = sum_l Pbar_lm(x_j) c_lm
  f_jk    = g_0(j) + 2 Re sum_{m>=1} g_m(j) e^{i m phi_k}

Sec. 3.2: HeatConv(v; h) = F^{-1}(h (.) F(v)) with h_l = exp(-t l (l+1)).
"""
import numpy as np


def heat_multipliers(t, lmax):
    """h_l = exp(-t l (l+1)), l = 0..lmax (Sec. 3.2; Alg. 1 step 2)."""
    l = np.arange(lmax + 1, dtype=np.float64)
    return np.exp(-t * l * (l + 1.0))


def _twiddles(nlon, lmax, sign):
    """E[k, m] = exp(sign * 2 pi i (k m mod nlon) / nlon), exact index reduction."""
    km = np.outer(np.arange(nlon), np.arange(lmax + 1)) % nlon
    return np.exp(sign * 2j * np.pi * km / nlon)


def ring_dft(grid, f):
    """F[..., j, m] = sum_k f[..., j, k] e^{-i m phi_k} for m = 0..lmax (direct sum)."""
    f = np.asarray(f, dtype=np.float64)
    return f @ _twiddles(grid.nlon, grid.lmax, -1.0)


def ring_idft(grid, g):
    """f[..., j, k] = Re g_0 + 2 Re sum_{m>=1} g_m e^{i m phi_k} (direct sum)."""
    wm = np.full(grid.lmax + 1, 2.0)
    wm[0] = 1.0
    e = _twiddles(grid.nlon, grid.lmax, +1.0).T * wm[:, None]   # [m, k]
    return (g @ e).real


def analysis(grid, f):
    """Coefficients c[..., l, m] (complex, zero for l < m) of a real grid field."""
    F = ring_dft(grid, f)
    P = grid.pbar()
    lead = F.shape[:-2]
    c = np.zeros(lead + (grid.lmax + 1, grid.lmax + 1), dtype=np.complex128)
    for m in range(grid.lmax + 1):
        A = P[m] * grid.a_ring[None, :]                 # [l-m, j]
        Fm = F[..., :, m]                               # [..., j]
        c[..., m:, m] = Fm.real @ A.T + 1j * (Fm.imag @ A.T)
    return c


def synthesis(grid, c):
    """Real grid field from coefficients c[..., l, m] (m >= 0 half)."""
    P = grid.pbar()
    lead = c.shape[:-2]
    g = np.zeros(lead + (grid.nlat, grid.lmax + 1), dtype=np.complex128)
    for m in range(grid.lmax + 1):
        cm = c[..., m:, m]                              # [..., l-m]
        g[..., :, m] = cm.real @ P[m] + 1j * (cm.imag @ P[m])
    return ring_idft(grid, g)


def heat_apply(grid, f, t):
    """K_t f = HeatConv(f; h) on the grid (Sec. 3.2)."""
    c = analysis(grid, f)
    c *= heat_multipliers(t, grid.lmax)[:, None]
    return synthesis(grid, c)

"""Helpers shared by the GPU parity tests (not collected as tests)."""
import numpy as np


def rel_max(a, b):
    """max |a - b| / max |b|."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def f32(a):
    """Round to FP32 and return (fp32 array for the GPU, the same values in FP64 for the oracle)."""
    x = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return x, x.astype(np.float64)


def s_err(s_gpu, s_ref, ot_ref, tol):
    """Error of a Sinkhorn divergence in units of its tolerance (pass: <= 1).

    S = OT(p,q) - (OT(p,p) + OT(q,q))/2 cancels: each OT carries the FP32 rounding of
    the potentials (measured systematic relative error <= ~1e-7 of u), so its absolute
    error cannot fall below ~2^-24 |OT|.  The bound is tol |S| + 4 * 2^-24 |OT(p,q)|.
    """
    s_gpu, s_ref, ot_ref = (np.asarray(a, dtype=np.float64) for a in (s_gpu, s_ref, ot_ref))
    return np.abs(s_gpu - s_ref) / (tol * np.abs(s_ref) + 4.0 * 2.0 ** -24 * np.abs(ot_ref))


# Unit roundoff of the Legendre contractions per precision: FP32 FFMA (2^-24), the bf16
# hi/lo split with three products (dropped lo*lo term and the rounding of lo: <= 3 * 2^-18
# per product, taken as 2^-16) and the tf32 hi/lo split with three products (dropped lo*lo
# and lo read as TF32: <= 3 * 2^-22 per product, taken as 2^-20).
UNIT = {"fp32": 2.0 ** -24, "bf16x3": 2.0 ** -16, "tf32x3": 2.0 ** -20}


def s_err_prec(s_gpu, s_ref, ot_ref, tol, prec):
    s_gpu, s_ref, ot_ref = (np.asarray(a, dtype=np.float64) for a in (s_gpu, s_ref, ot_ref))
    return np.abs(s_gpu - s_ref) / (tol * np.abs(s_ref) + 4.0 * UNIT[prec] * np.abs(ot_ref))


def potentials_err(grid, eps, u, v, phi_ref, psi_ref):
    """max over problems of the gauge-fixed potential errors (phi~ and psi~ relative to
    their largest magnitude), phi~ = phi - <a,phi>/4pi, psi~ = psi + <a,phi>/4pi: the
    potentials of Alg. 1 are defined up to (phi + c, psi - c)."""
    from oracle.sinkhorn import gauge_fixed
    phi = eps * np.log(np.asarray(u, dtype=np.float64))
    psi = eps * np.log(np.asarray(v, dtype=np.float64))
    gp, gs = gauge_fixed(grid, phi, psi)
    rp, rs = gauge_fixed(grid, phi_ref, psi_ref)
    return max(max(rel_max(gp[b], rp[b]), rel_max(gs[b], rs[b])) for b in range(phi.shape[0]))

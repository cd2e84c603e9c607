"""Gradients of the Sinkhorn divergence with respect to p (oracle, FP64).

Test infrastructure only.

Sec. 4.2 ("Gradient-based regional attribution") uses g = grad_mu S, derived from
the dual potentials and centred by its area-weighted mean.  Reading: the gradient
is Euclidean over node values, dS/dp_i, so it carries the factor a_i; the field
form is dS/dp_i / a_i.

* ``fd_directional``: central differences of S after exactly T iterations (no early
  stop), i.e. the derivative of the very function the unrolled adjoint
  differentiates.
* ``envelope``: at convergence, by the envelope theorem on the dual of
  eq. (uot): balanced  dS/dp = a (.) [phi_pq - (phi_pp + psi_pp)/2]
  (+ eps (m_p - m_q) a for the mass-difference term); unbalanced, dual form:
  dS_dual/dp = a (.) [tau(1-e^{-phi_pq/tau}) - (tau(1-e^{-phi_pp/tau}) + tau(1-e^{-psi_pp/tau}))/2].
"""
import numpy as np

from .sinkhorn import divergence


def fd_directional(grid, p, q, eps, tau, T, dirs, h=1e-6, form="S", kernel="sht"):
    """<dS/dp, d> for every direction d in dirs[k] ([K, nlat, nlon]); p, q one pair."""
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    out = np.empty(len(dirs))
    for k, d in enumerate(dirs):
        P = np.stack([p + h * d, p - h * d])
        Q = np.stack([q, q])
        r = divergence(grid, P, Q, eps, tau, T, 0.0, 0, "l2", kernel)
        if np.any(r["status"] < 0):
            raise FloatingPointError("Sinkhorn broke down; no finite difference")
        s = r["S"] if form == "S" else r["S_dual"]
        out[k] = (s[0] - s[1]) / (2.0 * h)
    return out


def envelope(grid, p, q, eps, tau, T, delta=1e-12, C=10, form="S", kernel="sht"):
    """Envelope gradient dS/dp (shape [nlat, nlon]) from converged potentials."""
    r = divergence(grid, p[None], q[None], eps, tau, T, delta, C, "l2", kernel)
    runs = r["runs"]
    if np.any(r["status"] < 0):
        raise FloatingPointError("Sinkhorn broke down; no gradient")
    a = grid.a
    phi_pq, phi_pp, psi_pp = runs["phi"][0], runs["phi"][1], runs["psi"][1]
    if not np.isfinite(tau):
        g = a * (phi_pq - 0.5 * (phi_pp + psi_pp))
        if form == "S":
            g = g + eps * (r["m_p"][0] - r["m_q"][0]) * a
        return g
    if form != "S_dual":
        raise ValueError("no envelope formula for the Alg. 1 return of the unbalanced problem")
    f = lambda x: tau * (1.0 - np.exp(-x / tau))
    return a * (f(phi_pq) - 0.5 * (f(phi_pp) + f(psi_pp)))


def project_mean_free(grid, g):
    """Remove the component along a: g - a * <g, 1>/<a, a> ... expressed for dS/dp.

    dS/dp is defined modulo c * a in the balanced case; the field form g/a is
    defined modulo a constant.  Returns the field form centred by its area mean.
    """
    a = grid.a
    f = g / a
    return f - np.sum(a * f) / np.sum(a)

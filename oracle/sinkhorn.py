"""Algorithm 1 (Spherical Harmonic Sinkhorn) and the Sinkhorn divergence (oracle, FP64).

Test infrastructure only.

Restates Alg. 1 (App. C) in the paper's order, batched over independent
problems (each problem stops on its own, exactly as if run alone):

  t = eps/4, h_l = exp(-t l(l+1)), u = v = 1
  for k = 1..T:
    balanced (tau = inf):  u = p / K v ;  v = q / K u ;  s = sum_i u_i ;  u /= s ; v *= s
    unbalanced:            u = (p / K v)^{tau/(tau+eps)} ;  v = (q / K u)^{tau/(tau+eps)}
                           c = tau/2 (log sum_i a_i p_i u_i^{-eps/tau} - log sum_i a_i q_i v_i^{-eps/tau})
                           u *= e^{c/eps} ;  v *= e^{-c/eps}
    every C iterations:    e = || u (.) K v - p ||_2 / || p ||_2  (App. C.3); stop if e < delta
  phi = eps log u, psi = eps log v
  return sum_i a_i (phi_i p_i + psi_i q_i)                         (balanced)
         sum_i a_i [tau(1-e^{-phi_i/tau}) p_i + tau(1-e^{-psi_i/tau}) q_i]   (unbalanced)

Readings where the paper is silent (each listed in the design notes):
* a non-positive K v (App. C.4: the update is undefined) or a non-finite result
  stops that problem with status NONPOSITIVE / NONFINITE at iteration k; its
  outputs are then NaN;
* terms with p_i = 0 in the translation-invariant sums contribute 0 (their limit);
* after the loop one more K v gives the final marginal error and the plan mass
  m(pi) = sum_i a_i u_i (K v)_i;
* "dual" objective = Alg. 1's return minus eps * m(pi) (the entropic term of the
  dual of eq. (uot) with the area measure as reference, up to a constant that
  cancels in the divergence);
* the L1 variant of the check is sum_i a_i |u_i (Kv)_i - p_i| / sum_i a_i p_i.
"""
import numpy as np

from .sht import heat_apply
from .dense import kernel_matrix, dense_apply

OK = 0
NOT_CONVERGED = 1
NONPOSITIVE = -5
NONFINITE = -6


def _kernel(grid, eps, kernel):
    t = eps / 4.0
    if kernel == "sht":
        if hasattr(grid, "heat_apply"):   # grids with their own ring layout (HEALPix)
            return lambda f: grid.heat_apply(f, t)
        return lambda f: heat_apply(grid, f, t)
    if kernel == "dense":
        K = kernel_matrix(grid, t)
        return lambda f: dense_apply(K, f)
    if callable(kernel):
        return kernel
    raise ValueError(kernel)


def _bad(kf, res):
    """Per-problem breakdown code: NONPOSITIVE if any K f <= 0, else NONFINITE if any
    value of K f or of the update is not finite, else OK."""
    ax = tuple(range(1, kf.ndim))
    nonpos = np.any(kf <= 0, axis=ax)
    nonfin = ~np.all(np.isfinite(kf), axis=ax) | ~np.all(np.isfinite(res), axis=ax)
    return np.where(nonpos, NONPOSITIVE, np.where(nonfin, NONFINITE, OK))


def marginal_error(grid, u, kv, p, norm="l2"):
    ax = tuple(range(1, p.ndim))
    r = u * kv - p
    if norm == "l2":
        return np.sqrt(np.sum(r * r, axis=ax)) / np.sqrt(np.sum(p * p, axis=ax))
    a = grid.a
    return np.sum(a * np.abs(r), axis=ax) / np.sum(a * p, axis=ax)


def sinkhorn(grid, p, q, eps, tau=np.inf, T=500, delta=0.0, C=10, norm="l2",
             kernel="sht", u0=None, v0=None):
    """Batched Alg. 1.  p, q: [B, nlat, nlon] FP64.  Returns a dict of per-problem arrays."""
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    if p.ndim == 2:
        p, q = p[None], q[None]
    B = p.shape[0]
    K = _kernel(grid, eps, kernel)
    a = grid.a
    balanced = not np.isfinite(tau)
    gamma = 1.0 if balanced else tau / (tau + eps)
    u = np.ones_like(p) if u0 is None else np.array(u0, dtype=np.float64)
    v = np.ones_like(q) if v0 is None else np.array(v0, dtype=np.float64)
    active = np.ones(B, dtype=bool)
    status = np.full(B, OK)
    iters = np.full(B, T)
    last_err = np.full(B, np.nan)

    for k in range(1, T + 1):
        idx = np.nonzero(active)[0]
        if idx.size == 0:
            break
        pi, qi = p[idx], q[idx]
        kv = K(v[idx])
        with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
            un = (pi / kv) ** gamma
        bad = _bad(kv, un)
        ku = K(un)
        with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
            vn = (qi / ku) ** gamma
        bad = np.where(bad != OK, bad, _bad(ku, vn))
        with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
            if balanced:
                s = np.sum(un, axis=(1, 2))
                un = un / s[:, None, None]
                vn = vn * s[:, None, None]
            else:
                def tsum(m, x):
                    terms = np.where(m > 0, a * m * x ** (-eps / tau), 0.0)
                    return np.sum(terms, axis=(1, 2))
                c = 0.5 * tau * (np.log(tsum(pi, un)) - np.log(tsum(qi, vn)))
                un = un * np.exp(c / eps)[:, None, None]
                vn = vn * np.exp(-c / eps)[:, None, None]
        ok = bad == OK
        for b, i in enumerate(idx):
            if ok[b]:
                u[i], v[i] = un[b], vn[b]
            else:
                status[i], iters[i], active[i] = bad[b], k, False
        if C > 0 and k % C == 0:
            idx2 = idx[ok]
            if idx2.size:
                e = marginal_error(grid, u[idx2], K(v[idx2]), p[idx2], norm)
                last_err[idx2] = e
                for b, i in enumerate(idx2):
                    if e[b] < delta:
                        active[i], iters[i] = False, k
    if delta > 0:
        status[(status == OK) & active] = NOT_CONVERGED

    kv = K(v)
    err = marginal_error(grid, u, kv, p, norm)
    with np.errstate(divide="ignore", invalid="ignore"):
        mass = np.sum(a * u * kv, axis=(1, 2))
        phi = eps * np.log(u)
        psi = eps * np.log(v)
        # a node with zero marginal contributes its limit, 0 (where p = 0, u = 0 and phi = -inf)
        if balanced:
            tp, tq = phi * p, psi * q
        else:
            tp = tau * (1.0 - np.exp(-phi / tau)) * p
            tq = tau * (1.0 - np.exp(-psi / tau)) * q
        ot = np.sum(a * (np.where(p > 0, tp, 0.0) + np.where(q > 0, tq, 0.0)), axis=(1, 2))
    broke = status < 0
    for arr in (err, mass, ot):
        arr[broke] = np.nan
    return dict(u=u, v=v, phi=phi, psi=psi, iters=iters, status=status, err=err,
                last_check_err=last_err, mass_pi=mass, ot=ot, ot_dual=ot - eps * mass,
                eps=eps, tau=tau)


def divergence(grid, p, q, eps, tau=np.inf, T=500, delta=0.0, C=10, norm="l2",
               kernel="sht"):
    """Sinkhorn divergence, eq. (sinkhorn-divergence), for a batch of pairs p[b], q[b].

    The three problems of every pair run in one batch ordered
    [(p_b, q_b) for all b] + [(p_b, p_b)] + [(q_b, q_b)], the self terms by the same
    Alg. 1 with q := p.  Two forms from the same converged state:
      S_alg1 = OT(p,q) - (OT(p,p) + OT(q,q))/2 + eps/2 (m(p) - m(q))^2   (Alg. 1 returns)
      S_dual = same with OT_dual = OT - eps m(pi) and no mass-difference term.
    """
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    if p.ndim == 2:
        p, q = p[None], q[None]
    B = p.shape[0]
    P = np.concatenate([p, p, q])
    Q = np.concatenate([q, p, q])
    r = sinkhorn(grid, P, Q, eps, tau, T, delta, C, norm, kernel)
    a = grid.a
    mp = np.sum(a * p, axis=(1, 2))
    mq = np.sum(a * q, axis=(1, 2))
    ot, od = r["ot"], r["ot_dual"]
    S = ot[:B] - 0.5 * (ot[B:2 * B] + ot[2 * B:]) + 0.5 * eps * (mp - mq) ** 2
    Sd = od[:B] - 0.5 * (od[B:2 * B] + od[2 * B:])
    st = np.stack([r["status"][:B], r["status"][B:2 * B], r["status"][2 * B:]])
    status = np.where((st < 0).any(0), st.min(0), st.max(0))
    return dict(S=S, S_dual=Sd, status=status, runs=r, m_p=mp, m_q=mq)


def gauge_fixed(grid, phi, psi):
    """phi - <a,phi>/4pi and psi + <a,phi>/4pi (removes the (phi+c, psi-c) freedom)."""
    c = np.sum(grid.a * phi, axis=(-2, -1), keepdims=True) / (4.0 * np.pi)
    return phi - c, psi + c


def sinkhorn_symmetric(grid, p, eps, tau=np.inf, T=500, delta=0.0, C=10, norm="l2", kernel="sht"):
    """The self term OT(p, p) through the symmetric form of Alg. 1's fixed point.  With q = p
    the scalings of the converged Alg. 1 satisfy u = v = (p / K u)^gamma (gamma = 1 balanced,
    tau/(tau+eps) otherwise; the translation-invariant constant vanishes); the averaged update
    u <- sqrt(u (p / K u)^gamma) of Feydy et al. (2019) reaches that point with one heat
    convolution per iteration.  u = 1 initially; the check of App. C.3 every C iterations on
    || u (.) K u - p ||; breakdowns as in `sinkhorn`.  Returns the Alg. 1 objective with
    phi = psi = eps log u (so OT = 2 sum a phi p balanced, 2 sum a tau (1 - e^{-phi/tau}) p
    unbalanced) and the plan mass m(pi) = sum a u (K u)."""
    p = np.asarray(p, dtype=np.float64)
    if p.ndim == 2:
        p = p[None]
    B = p.shape[0]
    K = _kernel(grid, eps, kernel)
    a = grid.a
    balanced = not np.isfinite(tau)
    gamma = 1.0 if balanced else tau / (tau + eps)
    u = np.ones_like(p)
    active = np.ones(B, dtype=bool)
    status = np.full(B, OK)
    iters = np.full(B, T)
    for k in range(1, T + 1):
        idx = np.nonzero(active)[0]
        if idx.size == 0:
            break
        ku = K(u[idx])
        with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
            un = np.sqrt(u[idx] * (p[idx] / ku) ** gamma)
        bad = _bad(ku, un)
        for b, i in enumerate(idx):
            if bad[b] == OK:
                u[i] = un[b]
            else:
                status[i], iters[i], active[i] = bad[b], k, False
        if C > 0 and k % C == 0:
            idx2 = np.nonzero(active)[0]
            if idx2.size:
                e = marginal_error(grid, u[idx2], K(u[idx2]), p[idx2], norm)
                for b, i in enumerate(idx2):
                    if e[b] < delta:
                        active[i], iters[i] = False, k
    if delta > 0:
        status[(status == OK) & active] = NOT_CONVERGED
    ku = K(u)
    err = marginal_error(grid, u, ku, p, norm)
    with np.errstate(divide="ignore", invalid="ignore"):
        mass = np.sum(a * u * ku, axis=(1, 2))
        phi = eps * np.log(u)
        t = phi * p if balanced else tau * (1.0 - np.exp(-phi / tau)) * p
        ot = 2.0 * np.sum(a * np.where(p > 0, t, 0.0), axis=(1, 2))
    broke = status < 0
    for arr in (err, mass, ot):
        arr[broke] = np.nan
    return dict(u=u, phi=phi, iters=iters, status=status, err=err, mass_pi=mass, ot=ot,
                ot_dual=ot - eps * mass, eps=eps, tau=tau)


def divergence_symmetric_self(grid, p, q, eps, tau=np.inf, T=500, delta=0.0, C=10, norm="l2", kernel="sht"):
    """eq. (sinkhorn-divergence) with OT(p, q) from Alg. 1 and the self terms OT(p, p), OT(q, q)
    from `sinkhorn_symmetric` (same T, delta, C); S and S_dual as in `divergence`."""
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    if p.ndim == 2:
        p, q = p[None], q[None]
    B = p.shape[0]
    r = sinkhorn(grid, p, q, eps, tau, T, delta, C, norm, kernel)
    s = sinkhorn_symmetric(grid, np.concatenate([p, q]), eps, tau, T, delta, C, norm, kernel)
    a = grid.a
    mp = np.sum(a * p, axis=(1, 2))
    mq = np.sum(a * q, axis=(1, 2))
    S = r["ot"] - 0.5 * (s["ot"][:B] + s["ot"][B:]) + 0.5 * eps * (mp - mq) ** 2
    Sd = r["ot_dual"] - 0.5 * (s["ot_dual"][:B] + s["ot_dual"][B:])
    st = np.stack([r["status"], s["status"][:B], s["status"][B:]])
    status = np.where((st < 0).any(0), st.min(0), st.max(0))
    return dict(S=S, S_dual=Sd, status=status, pq=r, self=s, m_p=mp, m_q=mq)

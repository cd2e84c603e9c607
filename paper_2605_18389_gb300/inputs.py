"""Seeded synthetic measures on an iso-latitude grid (shared by tests, bench and smoke).

Holds none of the transport method's arithmetic: it only draws fields.  The
caller passes the grid description (ring cosines x_j = cos(theta_j), the number of
longitudes and the per-ring area weights), from whichever side it trusts.

Recipes (the paper's workloads and their synthetic stand-ins):
* ``uniform``: the runtime experiment of Sec. 4.1 -- i.i.d. U(0,1) per node,
  normalised to unit mass under the area weights.
* ``vmf``: a mixture of K von Mises-Fisher densities (App. D.2 uses vMF inputs),
  centres uniform on S^2 (normalised Gaussian 3-vectors), kappa ~ U[lo, hi],
  density kappa/(2 pi (1 - e^{-2 kappa})) exp(kappa (mu.x - 1)) (overflow-free
  form), equal weights 1/K, plus a floor, normalised to unit mass.
* ``zonal``: multiply by 1 + 0.5 cos(lat - lat0), lat0 ~ U[-23.5, 23.5] degrees,
  before normalising (a seasonal-like modulation of a precipitation-like field).
* ``mass``: multiply a normalised field by a mass drawn U[0.5, 2].
"""
import numpy as np


def node_xyz(x, nlon):
    """Unit vectors [nlat, nlon, 3] of the nodes (theta_j = arccos x_j, phi_k = 2 pi k/nlon)."""
    x = np.asarray(x, dtype=np.float64)
    phi = 2.0 * np.pi * np.arange(nlon) / nlon
    st = np.sqrt(np.clip(1.0 - x * x, 0.0, None))
    return np.stack([np.outer(st, np.cos(phi)), np.outer(st, np.sin(phi)),
                     np.outer(x, np.ones(nlon))], axis=-1)


def _normalise(f, a_ring):
    mass = np.sum(f * np.asarray(a_ring)[:, None])
    return f / mass


def uniform(rng, x, nlon, a_ring):
    f = rng.uniform(size=(len(x), nlon))
    return _normalise(f, a_ring)


def vmf(rng, x, nlon, a_ring, ncomp, kappa_lo, kappa_hi, floor=1e-6, zonal=False):
    X = node_xyz(x, nlon)
    mu = rng.normal(size=(ncomp, 3))
    mu /= np.linalg.norm(mu, axis=1, keepdims=True)
    kap = rng.uniform(kappa_lo, kappa_hi, size=ncomp)
    f = np.zeros(X.shape[:2])
    for m, k in zip(mu, kap):
        f += k / (2.0 * np.pi * (1.0 - np.exp(-2.0 * k))) * np.exp(k * (X @ m - 1.0))
    f = f / ncomp + floor
    if zonal:
        lat0 = np.radians(rng.uniform(-23.5, 23.5))
        lat = np.arcsin(np.clip(np.asarray(x, dtype=np.float64), -1.0, 1.0))
        f = f * (1.0 + 0.5 * np.cos(lat - lat0))[:, None]
    return _normalise(f, a_ring)


# Per-workload recipes: (kind, kwargs).  Seeds: numpy default_rng([base, 2 i]) for p_i
# and default_rng([base, 2 i + 1]) for q_i.
RECIPES = {
    "paper_uniform": ("uniform", {}),
    "vmf3": ("vmf", dict(ncomp=3, kappa_lo=5.0, kappa_hi=50.0)),
    "vmf8": ("vmf", dict(ncomp=8, kappa_lo=10.0, kappa_hi=200.0)),
    "vmf8_zonal": ("vmf", dict(ncomp=8, kappa_lo=10.0, kappa_hi=200.0, zonal=True)),
    "vmf32": ("vmf", dict(ncomp=32, kappa_lo=50.0, kappa_hi=2000.0)),
    # the heat-vs-matrix convolution comparison: one vMF density, kappa = 10, random mean
    "vmf_k10": ("vmf", dict(ncomp=1, kappa_lo=10.0, kappa_hi=10.0, floor=0.0)),
}


def field(recipe, seed, x, nlon, a_ring):
    kind, kw = RECIPES[recipe]
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        return uniform(rng, x, nlon, a_ring)
    return vmf(rng, x, nlon, a_ring, **kw)


def pairs(recipe, base_seed, npairs, x, nlon, a_ring, masses=False, dtype=np.float64):
    """p, q of shape [npairs, nlat, nlon]; optional masses ~ U[0.5, 2] per field."""
    p = np.stack([field(recipe, [base_seed, 2 * i], x, nlon, a_ring) for i in range(npairs)])
    q = np.stack([field(recipe, [base_seed, 2 * i + 1], x, nlon, a_ring) for i in range(npairs)])
    if masses:
        rng = np.random.default_rng([base_seed, 1 << 20])
        p *= rng.uniform(0.5, 2.0, size=npairs)[:, None, None]
        q *= rng.uniform(0.5, 2.0, size=npairs)[:, None, None]
    return p.astype(dtype), q.astype(dtype)


def fd_directions(p, a, k, seed, balanced=True):
    """k directions [k, nlat, nlon] for finite-difference checks of a gradient in p: delta =
    p * xi with xi ~ N(0, 1) per node (numpy default_rng(seed), one direction after the other);
    when `balanced`, a constant is subtracted so that sum(a delta) = 0 (p + h delta keeps the
    mass of p); then delta is scaled so that ||delta||_a = ||p||_a (a: node area weights)."""
    p = np.asarray(p, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(k):
        d = p * rng.normal(size=p.shape)
        if balanced:
            d -= np.sum(a * d) / np.sum(a)
        d *= np.sqrt(np.sum(a * p * p) / np.sum(a * d * d))
        out.append(d)
    return np.array(out)

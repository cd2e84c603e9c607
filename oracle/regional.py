"""Gradient-based regional attribution (oracle, FP64).  Test infrastructure only.

Sec. 4.2 / App. E: the gradient of the divergence as a field (dS/dp_i divided by the area
weight a_i), centred by subtracting its area-weighted mean, and its area-weighted RMS over
five latitude bands: Tropics |lat| < 23.5 deg, ITCZ |lat| < 10, NH mid-latitudes 30-60 N,
SH mid-latitudes 30-60 S, Arctic > 66.5 N.
"""
import numpy as np

BANDS = ("tropics", "itcz", "nh_midlat", "sh_midlat", "arctic")


def band_masks(lat_deg):
    return [np.abs(lat_deg) < 23.5, np.abs(lat_deg) < 10.0, (lat_deg >= 30.0) & (lat_deg <= 60.0),
            (lat_deg <= -30.0) & (lat_deg >= -60.0), lat_deg > 66.5]


def regional_rms(grid, grad):
    """grad: [..., nlat, nlon] dS/dp (HEALPix: [..., 1, npix]); returns [..., 5].  The band
    masks come from the grid's latitudes, per ring ([nlat]) or per node (the node shape)."""
    a = grid.a
    g = np.asarray(grad, dtype=np.float64) / a
    mean = np.sum(a * g, axis=(-2, -1), keepdims=True) / np.sum(a)
    c = g - mean
    out = []
    for mask in band_masks(grid.lat_deg):
        w = a * (mask if mask.shape == a.shape else mask[:, None])
        out.append(np.sqrt(np.sum(w * c * c, axis=(-2, -1)) / np.sum(w)))
    return np.stack(out, axis=-1)

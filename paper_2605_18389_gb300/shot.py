"""Thin ctypes binding of the SHOT C ABI (include/shot.h).

Argument marshalling only: every step of the computation runs in libshot.so's CUDA
kernels.  Functions keep the C names; tensors are torch CUDA tensors (float32,
contiguous) whose device pointers are passed through, and the stream is torch's
current stream.  If the library is not built the import of any entry point raises:
there is no CPU fallback.
"""
import ctypes
import math
import os

import numpy as np

SHOT_OK = 0
SHOT_WARN_NOT_CONVERGED = 1
SHOT_ERR_INVALID_ARG = -1
SHOT_ERR_CUDA = -2
SHOT_ERR_OOM = -3
SHOT_ERR_UNSUPPORTED = -4
SHOT_ERR_NONPOSITIVE = -5
SHOT_ERR_NONFINITE = -6
SHOT_ERR_TIMEOUT = -7

SHOT_FP32 = 0
SHOT_BF16X3 = 1
SHOT_TF32X3 = 2
SHOT_TABLE = 0
SHOT_RECURRENCE = 1
SHOT_GRAD_UNROLLED = 0
SHOT_GRAD_ENVELOPE = 1
SHOT_QUAD_GAUSS_LEGENDRE = 0
SHOT_QUAD_CLENSHAW_CURTIS = 1
SHOT_QUAD_HEALPIX = 2
SHOT_FLAG_NORM_L1 = 0x1
SHOT_FLAG_WARM_START = 0x2
SHOT_FLAG_POTENTIALS = 0x4
SHOT_FLAG_SYMMETRIC_SELF = 0x8

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libshot.so")

_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_dbl_p = ctypes.POINTER(ctypes.c_double)
_c_flt_p = ctypes.POINTER(ctypes.c_float)
_vp = ctypes.c_void_p

# name -> argtypes (all return int)
SIGNATURES = {
    "shot_last_error": [ctypes.c_char_p, ctypes.c_int],
    "shot_grid_init": [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                       ctypes.c_int, _vp],
    "shot_grid_init_quad": [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            ctypes.c_int, ctypes.c_int, _vp],
    "shot_grid_init_healpix": [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp],
    "shot_grid_npix": [_vp, ctypes.POINTER(ctypes.c_longlong)],
    "shot_grid_rings": [_vp, _c_int_p, ctypes.POINTER(ctypes.c_longlong), _c_dbl_p],
    "shot_grid_free": [_vp],
    "shot_gibbs_normaliser": [ctypes.c_double, _c_dbl_p],
    "shot_gibbs_apply": [_vp, ctypes.c_double, _vp, _vp, ctypes.c_int, _vp],
    "shot_conv_compare": [_vp, ctypes.c_double, _vp, ctypes.c_int, _c_dbl_p, _vp],
    "shot_grid_info": [_vp, _c_int_p, _c_int_p, _c_int_p, _c_int_p, _c_int_p],
    "shot_grid_nodes": [_vp, _c_dbl_p, _c_dbl_p, _c_dbl_p],
    "shot_grid_reserve": [_vp, ctypes.c_int],
    "shot_grid_check": [_vp, _vp],
    "shot_grid_set_wait_limit": [_vp, ctypes.c_longlong],
    "shot_heat_apply": [_vp, ctypes.c_double, _vp, _vp, ctypes.c_int, _vp],
    "shot_sht_analysis": [_vp, _vp, _vp, ctypes.c_int, _vp],
    "shot_sht_synthesis": [_vp, _vp, _vp, ctypes.c_int, _vp],
    "shot_sinkhorn": [_vp, _vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                      ctypes.c_double, ctypes.c_int, ctypes.c_int, _vp, _vp, _c_dbl_p, _c_dbl_p, _c_dbl_p,
                      _c_int_p, _c_flt_p, _c_int_p, _vp],
    "shot_divergence": [_vp, _vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                        ctypes.c_double, ctypes.c_int, ctypes.c_int, _c_dbl_p, _c_dbl_p, _c_int_p, _vp, _vp,
                        _c_dbl_p, _c_int_p, _vp],
    "shot_divergence_grad": [_vp, _vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                             ctypes.c_int, ctypes.c_int, _c_dbl_p, _vp, _c_int_p, _vp],
    "shot_regional_rms": [_vp, _vp, ctypes.c_int, _c_dbl_p, _vp],
    "shot_heat_apply_noalloc": [_vp, ctypes.c_double, _vp, _vp, ctypes.c_int, _vp],
    "shot_grid_autotune": [_vp, ctypes.c_int, _c_int_p, _vp],
    "shot_launch_count": [ctypes.POINTER(ctypes.c_longlong)],
    "shot_profile_enable": [ctypes.c_int],
    "shot_profile_read": [_c_dbl_p, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int],
}

PROFILE_KINDS = ("ring_dft", "legendre_analysis", "legendre_synthesis", "inverse_dft_epilogue", "other",
                 "check_final")



class ShotPairSet(ctypes.Structure):
    """struct shot_pair_set of include/shot.h."""
    _fields_ = [("grid", _vp), ("p", _vp), ("q", _vp), ("batch", ctypes.c_int), ("eps", ctypes.c_double),
                ("tau", ctypes.c_double), ("S", _c_dbl_p), ("S_dual", _c_dbl_p), ("status", _c_int_p)]


SIGNATURES["shot_divergence_multi"] = [ctypes.POINTER(ShotPairSet), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_int, _vp]

_lib = None


class ShotError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"SHOT error {code}: {msg}")
        self.code = code


def lib():
    """Load libshot.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
        try:
            import torch  # noqa: F401  (share torch's CUDA runtime in this process)
        except ImportError:
            pass
        l = ctypes.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            f = getattr(l, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        _lib = l
    return _lib


def last_error():
    buf = ctypes.create_string_buffer(1024)
    lib().shot_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def _check(rc, allow_positive=True):
    if rc < 0 or (rc > 0 and not allow_positive):
        raise ShotError(rc, last_error())
    return rc


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return _vp(s.cuda_stream)


def _dev_ptr(t, name, shape=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous float32")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return _vp(t.data_ptr())


def _np_ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# ---- C-named entry points ---------------------------------------------------------

def shot_grid_init(nlat, nlon=None, lmax=-1, precision=SHOT_FP32, legendre_mode=SHOT_TABLE, stream=None):
    nlon = 2 * nlat if nlon is None else nlon
    h = _vp()
    _check(lib().shot_grid_init(ctypes.byref(h), nlat, nlon, lmax, precision, legendre_mode, _stream(stream)))
    return h


def shot_grid_init_quad(quadrature, nlat, nlon=None, lmax=-1, precision=SHOT_FP32, legendre_mode=SHOT_TABLE,
                        stream=None):
    nlon = 2 * nlat if nlon is None else nlon
    h = _vp()
    _check(lib().shot_grid_init_quad(ctypes.byref(h), quadrature, nlat, nlon, lmax, precision, legendre_mode,
                                     _stream(stream)))
    return h


def shot_gibbs_normaliser(eps):
    c = ctypes.c_double()
    _check(lib().shot_gibbs_normaliser(eps, ctypes.byref(c)))
    return c.value


def shot_gibbs_apply(g, eps, inp, out, stream=None):
    return _check(lib().shot_gibbs_apply(g, eps, _dev_ptr(inp, "in"), _dev_ptr(out, "out"), inp.shape[0],
                                         _stream(stream)))


def shot_conv_compare(g, eps, inp, stream=None):
    """Per-field mean |C(eps) H_{eps/4} f - K_eps f| over the grid nodes (numpy array)."""
    mae = np.empty(inp.shape[0])
    _check(lib().shot_conv_compare(g, eps, _dev_ptr(inp, "in"), inp.shape[0], _np_ptr(mae, ctypes.c_double),
                                   _stream(stream)))
    return mae


def shot_grid_init_healpix(nside, lmax=-1, precision=SHOT_FP32, legendre_mode=SHOT_TABLE, stream=None):
    h = _vp()
    _check(lib().shot_grid_init_healpix(ctypes.byref(h), nside, lmax, precision, legendre_mode, _stream(stream)))
    return h


def shot_grid_npix(g):
    n = ctypes.c_longlong()
    _check(lib().shot_grid_npix(g, ctypes.byref(n)))
    return n.value


def shot_grid_rings(g):
    nr = shot_grid_info(g)["nlat"]
    ln = np.empty(nr, np.int32)
    off = np.empty(nr, np.int64)
    ph = np.empty(nr)
    _check(lib().shot_grid_rings(g, _np_ptr(ln, ctypes.c_int), _np_ptr(off, ctypes.c_longlong),
                                 _np_ptr(ph, ctypes.c_double)))
    return ln, off, ph


def shot_grid_free(g):
    return _check(lib().shot_grid_free(g))


def shot_grid_info(g):
    v = [ctypes.c_int() for _ in range(5)]
    _check(lib().shot_grid_info(g, *[ctypes.byref(x) for x in v]))
    return dict(zip(("nlat", "nlon", "lmax", "precision", "legendre_mode"), [x.value for x in v]))


def shot_grid_nodes(g):
    nlat = shot_grid_info(g)["nlat"]
    x, w, a = (np.empty(nlat) for _ in range(3))
    _check(lib().shot_grid_nodes(g, _np_ptr(x, ctypes.c_double), _np_ptr(w, ctypes.c_double),
                                 _np_ptr(a, ctypes.c_double)))
    return x, w, a


def shot_grid_reserve(g, nfields):
    return _check(lib().shot_grid_reserve(g, nfields))


def shot_grid_check(g, stream=None):
    """Synchronises the stream; raises ShotError(SHOT_ERR_TIMEOUT) if a bounded device-side
    wait expired in a kernel on this grid since the last check."""
    return _check(lib().shot_grid_check(g, _stream(stream)))


def shot_grid_set_wait_limit(g, cycles):
    """Limit (SM clock cycles) of the tensor-core kernels' bounded waits for later launches on
    this grid; cycles <= 0 restores the default 2^30."""
    return _check(lib().shot_grid_set_wait_limit(g, int(cycles)))


def shot_heat_apply(g, t, inp, out, stream=None):
    nf = inp.shape[0]
    return _check(lib().shot_heat_apply(g, float(t), _dev_ptr(inp, "in"), _dev_ptr(out, "out", inp.shape),
                                        nf, _stream(stream)))


def shot_heat_apply_noalloc(g, t, inp, out, stream=None):
    """shot_heat_apply without any device allocation (fixed library-owned scratch)."""
    nf = inp.shape[0]
    return _check(lib().shot_heat_apply_noalloc(g, float(t), _dev_ptr(inp, "in"), _dev_ptr(out, "out", inp.shape),
                                                nf, _stream(stream)))


def shot_sht_analysis(g, inp, coeffs, stream=None):
    return _check(lib().shot_sht_analysis(g, _dev_ptr(inp, "in"), _dev_ptr(coeffs, "coeffs"), inp.shape[0],
                                          _stream(stream)))


def shot_sht_synthesis(g, coeffs, out, stream=None):
    return _check(lib().shot_sht_synthesis(g, _dev_ptr(coeffs, "coeffs"), _dev_ptr(out, "out"), out.shape[0],
                                           _stream(stream)))


def shot_sinkhorn(g, p, q, eps, tau=math.inf, max_iter=500, tol=0.0, check_every=10, flags=0, u=None, v=None,
                  stream=None):
    """Returns (status_code, dict of per-problem numpy outputs); u, v are filled in place."""
    import torch
    B = p.shape[0]
    if u is None:
        u = torch.empty_like(p)
    if v is None:
        v = torch.empty_like(p)
    ot, otd, mass = (np.empty(B) for _ in range(3))
    iters, status = np.empty(B, np.int32), np.empty(B, np.int32)
    err = np.empty(B, np.float32)
    rc = _solver_rc(lib().shot_sinkhorn(
        g, _dev_ptr(p, "p"), _dev_ptr(q, "q", p.shape), B, float(eps), float(tau), int(max_iter), float(tol),
        int(check_every), int(flags), _dev_ptr(u, "u", p.shape), _dev_ptr(v, "v", p.shape),
        _np_ptr(ot, ctypes.c_double), _np_ptr(otd, ctypes.c_double), _np_ptr(mass, ctypes.c_double),
        _np_ptr(iters, ctypes.c_int), _np_ptr(err, ctypes.c_float), _np_ptr(status, ctypes.c_int),
        _stream(stream)))
    return rc, dict(u=u, v=v, ot=ot, ot_dual=otd, mass_pi=mass, iters=iters, err=err, status=status)


def _solver_rc(rc):
    """Negative per-problem statuses are results, not call failures, for the solvers."""
    if rc in (SHOT_ERR_NONPOSITIVE, SHOT_ERR_NONFINITE):
        return rc
    return _check(rc)


def shot_divergence(g, p, q, eps, tau=math.inf, max_iter=500, tol=0.0, check_every=10, flags=0,
                    u3=None, v3=None, stream=None):
    """Returns (status_code, dict with S, S_dual, status, ot3, iters3)."""
    B = p.shape[0]
    S, Sd = np.empty(B), np.empty(B)
    status = np.empty(B, np.int32)
    ot3 = np.empty(3 * B)
    it3 = np.empty(3 * B, np.int32)
    shape3 = (3 * B,) + tuple(p.shape[1:])
    rc = lib().shot_divergence(
        g, _dev_ptr(p, "p"), _dev_ptr(q, "q", p.shape), B, float(eps), float(tau), int(max_iter), float(tol),
        int(check_every), int(flags), _np_ptr(S, ctypes.c_double), _np_ptr(Sd, ctypes.c_double),
        _np_ptr(status, ctypes.c_int),
        _dev_ptr(u3, "u3", shape3) if u3 is not None else None,
        _dev_ptr(v3, "v3", shape3) if v3 is not None else None,
        _np_ptr(ot3, ctypes.c_double), _np_ptr(it3, ctypes.c_int), _stream(stream))
    rc = _solver_rc(rc)
    return rc, dict(S=S, S_dual=Sd, status=status, ot3=ot3, iters3=it3)


def shot_launch_count():
    n = ctypes.c_longlong()
    _check(lib().shot_launch_count(ctypes.byref(n)))
    return n.value


def shot_profile_enable(on=True):
    return _check(lib().shot_profile_enable(1 if on else 0))


def shot_profile_read():
    """{kind: (total_ms, launches)} for the launches recorded since the last read."""
    k = len(PROFILE_KINDS)
    ms = np.zeros(k)
    n = np.zeros(k, np.int64)
    _check(lib().shot_profile_read(_np_ptr(ms, ctypes.c_double), n.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                   k))
    return {name: (float(ms[i]), int(n[i])) for i, name in enumerate(PROFILE_KINDS)}


def shot_divergence_grad(g, p, q, eps, tau=math.inf, max_iter=400, checkpoint_every=20, mode=SHOT_GRAD_UNROLLED,
                         grad=None, stream=None):
    """Returns (status_code, dict with S, status, grad) where grad = dS/dp (device tensor)."""
    import torch
    B = p.shape[0]
    if grad is None:
        grad = torch.empty_like(p)
    S = np.empty(B)
    status = np.empty(B, np.int32)
    rc = _solver_rc(lib().shot_divergence_grad(
        g, _dev_ptr(p, "p"), _dev_ptr(q, "q", p.shape), B, float(eps), float(tau), int(max_iter),
        int(checkpoint_every), int(mode), _np_ptr(S, ctypes.c_double), _dev_ptr(grad, "grad", p.shape),
        _np_ptr(status, ctypes.c_int), _stream(stream)))
    return rc, dict(S=S, status=status, grad=grad)


def divergence(g, p, q, eps, tau=math.inf, max_iter=400, checkpoint_every=20, mode=SHOT_GRAD_UNROLLED):
    """S(p, q) as a differentiable torch function of p (batch of pairs; returns a [batch] tensor).

    The forward runs shot_divergence_grad when p requires a gradient (shot_divergence
    otherwise); backward scales the stored dS/dp by the incoming gradient.
    """
    import torch

    class _Div(torch.autograd.Function):
        @staticmethod
        def forward(ctx, pp):
            if pp.requires_grad:
                rc, r = shot_divergence_grad(g, pp.detach().contiguous(), q, eps, tau, max_iter, checkpoint_every,
                                             mode)
                ctx.save_for_backward(r["grad"])
            else:
                rc, r = shot_divergence(g, pp.detach().contiguous(), q, eps, tau, max_iter, 0.0, 0)
            return torch.as_tensor(r["S"], dtype=torch.float64, device=pp.device)

        @staticmethod
        def backward(ctx, gout):
            (gp,) = ctx.saved_tensors
            return gp * gout.to(gp.dtype).view(-1, *([1] * (gp.dim() - 1)))

    return _Div.apply(p)


def shot_divergence_multi(sets, max_iter=200, tol=0.0, check_every=10, flags=0, stream=None):
    """sets: list of dicts {grid, p, q, eps, tau}.  Returns (status_code, list of dicts S, S_dual, status)."""
    arr = (ShotPairSet * len(sets))()
    outs = []
    for i, st in enumerate(sets):
        B = st["p"].shape[0]
        o = dict(S=np.empty(B), S_dual=np.empty(B), status=np.empty(B, np.int32))
        outs.append(o)
        arr[i] = ShotPairSet(st["grid"], _dev_ptr(st["p"], "p"), _dev_ptr(st["q"], "q", st["p"].shape), B,
                             float(st["eps"]), float(st.get("tau", math.inf)), _np_ptr(o["S"], ctypes.c_double),
                             _np_ptr(o["S_dual"], ctypes.c_double), _np_ptr(o["status"], ctypes.c_int))
    rc = _solver_rc(lib().shot_divergence_multi(arr, len(sets), int(max_iter), float(tol), int(check_every),
                                                int(flags), _stream(stream)))
    return rc, outs


def shot_grid_autotune(g, nfields, stream=None):
    """Tune (or look up) the launch shapes for nfields; returns dict of the four choices."""
    ch = np.zeros(4, np.int32)
    _check(lib().shot_grid_autotune(g, int(nfields), _np_ptr(ch, ctypes.c_int), _stream(stream)))
    return dict(zip(("dft_fg", "idft_fg", "simt_bn", "tc_stages"), [int(x) for x in ch]))


REGIONS = ("tropics", "itcz", "nh_midlat", "sh_midlat", "arctic")


def shot_regional_rms(g, grad, stream=None):
    """[batch, 5] area-weighted RMS of the centred gradient field per latitude band."""
    B = grad.shape[0]
    out = np.empty((B, 5))
    _check(lib().shot_regional_rms(g, _dev_ptr(grad, "grad"), B, _np_ptr(out, ctypes.c_double), _stream(stream)))
    return out

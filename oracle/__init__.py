"""FP64 oracle for the FireANTs registration inner loop (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the product path
(the CUDA library and its Python binding) never does.  The arithmetic lives
in ``fa_oracle.c`` (plain C, double precision, written from the paper); this
file only compiles it with gcc and marshals numpy float64 arrays.

Layouts: volumes are [D, H, W]; fields are [3, D, H, W] with channel 0 the
z (D-axis) component, 1 the y component and 2 the x component, in voxels.

Parity status of each function (what pins it is in tests/test_oracle_*.py):
  warp, warp_adjoint, box_sum, lncc, mse, gauss_taps, gauss_smooth, adam,
  max_norm, step_scale, compose, downsample, upsample_field: pinned.
  register: pinned only by invariants (positive Jacobian determinant, loss
  decrease, recovery of a known translation); the paper prints no worked
  example of a whole registration.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fa_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libfa_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


class _Params(ctypes.Structure):
    _fields_ = [
        ("n_levels", ctypes.c_int),
        ("scales", ctypes.c_int * 8),
        ("iters", ctypes.c_int * 8),
        ("lr", ctypes.c_double),
        ("sigma_grad", ctypes.c_double),
        ("sigma_warp", ctypes.c_double),
        ("window", ctypes.c_int),
        ("loss", ctypes.c_int),
        ("beta1", ctypes.c_double),
        ("beta2", ctypes.c_double),
        ("adam_eps", ctypes.c_double),
        ("cc_eps", ctypes.c_double),
        ("c_lp", ctypes.c_double),
        ("use_jac", ctypes.c_int),
        ("mi_bins", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile fa_oracle.c into a shared library (gcc, OpenMP, no FMA
    contraction so x86 and Arm hosts give identical results)."""
    with _lock:
        if (not force and os.path.exists(_SO)
                and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
            return _SO
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _SO + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
        return _SO


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        i, d = ctypes.c_int, ctypes.c_double
        lib.or_sample.restype = d
        lib.or_sample.argtypes = [_dp, i, i, i, d, d, d, _dp]
        lib.or_warp.argtypes = [_dp, i, i, i, _dp, _dp, _dp]
        lib.or_warp_adjoint.argtypes = [_dp, _dp, i, i, i, i, i, i, _dp]
        lib.or_jac_direction.argtypes = [_dp, _dp, i, i, i, _dp]
        lib.or_svf_exp.argtypes = [_dp, i, i, i, i, _dp]
        lib.or_affine_field.argtypes = [_dp, i, i, i, _dp]
        lib.or_affine_loss_grad.argtypes = [_dp, _dp, i, i, i, _dp, i, i, d, _dp, _dp]
        lib.or_register_from.argtypes = [_dp, _dp, i, i, i, ctypes.c_void_p, _dp, _dp, _dp, _dp]
        lib.or_inverse_energy_grad.argtypes = [_dp, _dp, i, i, i, _dp, _dp]
        lib.or_inverse.argtypes = [_dp, i, i, i, ctypes.c_void_p, _dp, _dp]
        lib.or_svf_loss_grad.argtypes = [_dp, _dp, i, i, i, ctypes.c_void_p, i, _dp, _dp, _dp,
                                          _dp, _dp]
        lib.or_register_svf.argtypes = [_dp, _dp, i, i, i, ctypes.c_void_p, i, _dp, _dp, _dp]
        lib.or_rodrigues.argtypes = [_dp, _dp, _dp]
        lib.or_rodrigues.restype = None
        lib.or_rigid_theta.argtypes = [_dp, i, i, i, _dp]
        lib.or_rigid_loss_grad.argtypes = [_dp, _dp, i, i, i, i, i, i, _dp, i, i, d, _dp, _dp]
        lib.or_rigid_register.argtypes = [_dp, _dp, i, i, i, ctypes.c_void_p, _dp, _dp]
        lib.or_symmetric_loss_grad.argtypes = [_dp, _dp, i, i, i, ctypes.c_void_p, _dp, _dp,
                                               _dp, _dp, _dp]
        lib.or_register_symmetric.argtypes = [_dp, _dp, i, i, i, ctypes.c_void_p,
                                              ctypes.c_void_p, _dp, _dp, _dp, _dp, _dp]
        lib.or_affine_register.argtypes = [_dp, _dp, i, i, i, ctypes.c_void_p, _dp, _dp]
        lib.or_box_sum.argtypes = [_dp, i, i, i, i, _dp]
        lib.or_lncc.argtypes = [_dp, _dp, i, i, i, i, d, _dp, _dp, _dp, _dp]
        lib.or_mse.argtypes = [_dp, _dp, i, i, i, _dp, _dp, _dp]
        lib.or_mi.argtypes = [_dp, _dp, i, i, i, i, _dp, _dp, _dp]
        lib.or_mi_range.argtypes = [_dp, _dp, ctypes.c_size_t, _dp]
        lib.or_gauss_taps.argtypes = [d, _dp, i]
        lib.or_gauss_smooth.argtypes = [_dp, _dp, i, i, i, i, d]
        lib.or_adam.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_size_t, i, d, d, d]
        lib.or_max_norm.restype = d
        lib.or_max_norm.argtypes = [_dp, i, i, i]
        lib.or_step_scale.restype = d
        lib.or_step_scale.argtypes = [_dp, _dp, i, i, i, d, d]
        lib.or_compose.argtypes = [_dp, _dp, _dp, i, i, i]
        lib.or_level_size.argtypes = [i, i]
        lib.or_downsample.argtypes = [_dp, i, i, i, i, _dp]
        lib.or_upsample_field.argtypes = [_dp, i, i, i, _dp, i, i, i, i]
        lib.or_register.argtypes = [_dp, _dp, i, i, i, ctypes.POINTER(_Params), _dp, _dp, _dp]
        _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray | None):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what}: invalid arguments (rc={rc})")


def _dims(vol: np.ndarray):
    if vol.ndim != 3:
        raise ValueError("expected a [D, H, W] volume")
    return tuple(int(s) for s in vol.shape)


def sample(vol, p):
    """Trilinear interpolant (zero outside) and its gradient at one point p=(z,y,x)."""
    vol = _f64(vol)
    D, H, W = _dims(vol)
    g = np.zeros(3)
    v = _L().or_sample(_p(vol), D, H, W, float(p[0]), float(p[1]), float(p[2]), _p(g))
    return v, g


def warp(Im, u, want_grad: bool = True):
    """J(x) = I_m(x + u(x)) and the interpolant's gradient at x + u(x)."""
    Im, u = _f64(Im), _f64(u)
    D, H, W = _dims(Im)
    if u.shape != (3, D, H, W):
        raise ValueError("u must be [3, D, H, W] on the moving image's grid")
    J = np.empty((D, H, W))
    g = np.empty((3, D, H, W)) if want_grad else None
    _check(_L().or_warp(_p(Im), D, H, W, _p(u), _p(J), _p(g)), "warp")
    return (J, g) if want_grad else J


def warp_adjoint(dJ, u, moving_shape):
    """Scatter of a cotangent on the fixed grid back onto the moving grid."""
    dJ, u = _f64(dJ), _f64(u)
    D, H, W = _dims(dJ)
    Dm, Hm, Wm = (int(s) for s in moving_shape)
    out = np.empty((Dm, Hm, Wm))
    _check(_L().or_warp_adjoint(_p(dJ), _p(u), D, H, W, Dm, Hm, Wm, _p(out)), "warp_adjoint")
    return out


def jac_direction(g, u):
    """J(phi)^T g with J(phi) = I + grad u (reading R-jac)."""
    g, u = _f64(g), _f64(u)
    D, H, W = g.shape[1:]
    out = np.empty_like(g)
    _check(_L().or_jac_direction(_p(g), _p(u), D, H, W, _p(out)), "jac_direction")
    return out


def box_sum(x, win: int):
    x = _f64(x)
    D, H, W = _dims(x)
    out = np.empty_like(x)
    _check(_L().or_box_sum(_p(x), D, H, W, int(win), _p(out)), "box_sum")
    return out


def lncc(I, J, win: int, cc_eps: float, want_cc=False, want_dJ=True, want_dI=False):
    """Returns dict(loss=L, cc=..., dJ=..., dI=...) (absent entries are None)."""
    I, J = _f64(I), _f64(J)
    D, H, W = _dims(I)
    if J.shape != I.shape:
        raise ValueError("shape mismatch")
    loss = ctypes.c_double()
    cc = np.empty_like(I) if want_cc else None
    dJ = np.empty_like(I) if want_dJ else None
    dI = np.empty_like(I) if want_dI else None
    _check(_L().or_lncc(_p(I), _p(J), D, H, W, int(win), float(cc_eps), ctypes.byref(loss),
                        _p(cc), _p(dJ), _p(dI)), "lncc")
    return dict(loss=loss.value, cc=cc, dJ=dJ, dI=dI)


def mse(I, J):
    I, J = _f64(I), _f64(J)
    D, H, W = _dims(I)
    loss = ctypes.c_double()
    dJ, dI = np.empty_like(I), np.empty_like(I)
    _check(_L().or_mse(_p(I), _p(J), D, H, W, ctypes.byref(loss), _p(dJ), _p(dI)), "mse")
    return dict(loss=loss.value, dJ=dJ, dI=dI)


def mi_range(If, Im):
    """[lo_f, hi_f, lo_m, hi_m]: the fixed image's range and the moving
    image's with 0 included (reading R-mi)."""
    If, Im = _f64(If), _f64(Im)
    r = np.empty(4)
    _check(_L().or_mi_range(_p(If), _p(Im), If.size, _p(r)), "mi_range")
    return r


def mi(I, J, bins=32, rng=None, want_dJ=True):
    """L = -MI(I, J) (reading R-mi) and dL/dJ; rng defaults to mi_range(I, J)."""
    I, J = _f64(I), _f64(J)
    D, H, W = _dims(I)
    r = _f64(rng if rng is not None else mi_range(I, J))
    loss = ctypes.c_double()
    dJ = np.empty_like(I) if want_dJ else None
    _check(_L().or_mi(_p(I), _p(J), D, H, W, int(bins), _p(r), ctypes.byref(loss), _p(dJ)), "mi")
    return dict(loss=loss.value, dJ=dJ)


def gauss_taps(sigma: float):
    buf = np.zeros(4096)
    R = _L().or_gauss_taps(float(sigma), _p(buf), 4096)
    if R < 0:
        raise ValueError("bad sigma")
    return buf[: 2 * R + 1].copy()


def gauss_smooth(x, sigma: float):
    """Separable Gaussian on [D,H,W] or [C,D,H,W] (channels independent)."""
    x = _f64(x)
    squeeze = x.ndim == 3
    if squeeze:
        x = x[None]
    C, D, H, W = (int(s) for s in x.shape)
    out = np.empty_like(x)
    _check(_L().or_gauss_smooth(_p(x), _p(out), C, D, H, W, float(sigma)), "gauss_smooth")
    return out[0] if squeeze else out


def adam(g, m, v, t: int, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step; returns (d, m_new, v_new) without touching the inputs."""
    g = _f64(g)
    m = _f64(m).copy()
    v = _f64(v).copy()
    d = np.empty_like(g)
    _check(_L().or_adam(_p(g), _p(m), _p(v), _p(d), g.size, int(t), float(beta1), float(beta2),
                        float(eps)), "adam")
    return d, m, v


def max_norm(d):
    d = _f64(d)
    _, D, H, W = d.shape
    return _L().or_max_norm(_p(d), D, H, W)


def step_scale(d, eta: float, c_lp: float = 2.0):
    """delta = -eta / (c_lp max|d|) d; returns (delta, eps_t)."""
    d = _f64(d)
    _, D, H, W = d.shape
    delta = np.empty_like(d)
    e = _L().or_step_scale(_p(d), _p(delta), D, H, W, float(eta), float(c_lp))
    return delta, e


def compose(u, delta):
    """u'(x) = delta(x) + u(x + delta(x))."""
    u, delta = _f64(u), _f64(delta)
    _, D, H, W = u.shape
    out = np.empty_like(u)
    _check(_L().or_compose(_p(u), _p(delta), _p(out), D, H, W), "compose")
    return out


def svf_exp(v, steps: int):
    """exp(v) - id by scaling and squaring with `steps` squarings."""
    v = _f64(v)
    _, D, H, W = v.shape
    out = np.empty_like(v)
    _check(_L().or_svf_exp(_p(v), D, H, W, int(steps), _p(out)), "svf_exp")
    return out


def level_size(n: int, s: int) -> int:
    return int(_L().or_level_size(int(n), int(s)))


def level_shape(shape, s: int):
    return tuple(level_size(n, s) for n in shape)


def downsample(I, s: int):
    I = _f64(I)
    D, H, W = _dims(I)
    out = np.empty(level_shape((D, H, W), s))
    _check(_L().or_downsample(_p(I), D, H, W, int(s), _p(out)), "downsample")
    return out


def upsample_field(src, shape, power: int):
    """power 1: displacement (x s_a); -1: first moment (/ s_a); -2: second moment (/ s_a^2)."""
    src = _f64(src)
    _, Dc, Hc, Wc = src.shape
    Df, Hf, Wf = (int(s) for s in shape)
    out = np.empty((3, Df, Hf, Wf))
    _check(_L().or_upsample_field(_p(src), Dc, Hc, Wc, _p(out), Df, Hf, Wf, int(power)),
           "upsample_field")
    return out


def register(If, Im, scales, iters, lr=0.5, sigma_grad=1.0, sigma_warp=0.5, window=5,
             loss="lncc", beta1=0.9, beta2=0.999, adam_eps=1e-8, cc_eps=1e-5, c_lp=2.0,
             want_trace=False, use_jac=False, u_init=None, mi_bins=32):
    """Algorithm 1 end to end.  Returns dict(u, final_loss, trace)."""
    If, Im = _f64(If), _f64(Im)
    D, H, W = _dims(If)
    if Im.shape != If.shape:
        raise ValueError("fixed and moving must share a grid")
    if not (1 <= len(scales) <= 8) or len(iters) != len(scales):
        raise ValueError("1..8 levels, one iteration count per level")
    p = _Params()
    p.n_levels = len(scales)
    for k, (s, t) in enumerate(zip(scales, iters)):
        p.scales[k] = int(s)
        p.iters[k] = int(t)
    p.lr, p.sigma_grad, p.sigma_warp = float(lr), float(sigma_grad), float(sigma_warp)
    p.window = int(window)
    p.loss = {"lncc": 0, "mse": 1, "mi": 2}[loss]
    p.beta1, p.beta2, p.adam_eps = float(beta1), float(beta2), float(adam_eps)
    p.cc_eps, p.c_lp = float(cc_eps), float(c_lp)
    p.use_jac = 1 if use_jac else 0
    p.mi_bins = int(mi_bins)
    fs = level_shape((D, H, W), scales[-1])
    u = np.empty((3,) + fs)
    fl = ctypes.c_double()
    trace = np.empty(int(sum(iters))) if want_trace else None
    ui = _f64(u_init) if u_init is not None else None
    if ui is not None and ui.shape != (3, D, H, W):
        raise ValueError("u_init must be [3, D, H, W] on the input grid")
    _check(_L().or_register_from(_p(If), _p(Im), D, H, W, ctypes.byref(p), _p(ui), _p(u),
                                 ctypes.byref(fl), _p(trace)), "register")
    return dict(u=u, final_loss=fl.value, trace=trace)


# ------------------------------------------------------------- affine stage
IDENTITY_AFFINE = np.array([1.0, 0, 0, 0, 1.0, 0, 0, 0, 1.0, 0, 0, 0])


def affine_field(theta, shape):
    """Displacement of the affine map theta (A row-major, t) on a grid (R-aff)."""
    th = _f64(theta)
    D, H, W = (int(n) for n in shape)
    u = np.empty((3, D, H, W))
    _check(_L().or_affine_field(_p(th), D, H, W, _p(u)), "affine_field")
    return u


def affine_loss_grad(If, Im, theta, window=5, loss="lncc", cc_eps=1e-5):
    If, Im, th = _f64(If), _f64(Im), _f64(theta)
    D, H, W = _dims(If)
    L = ctypes.c_double()
    g = np.empty(12)
    _check(_L().or_affine_loss_grad(_p(If), _p(Im), D, H, W, _p(th), {"lncc": 0, "mse": 1}[loss],
                                    int(window), float(cc_eps), ctypes.byref(L), _p(g)),
           "affine_loss_grad")
    return L.value, g


def affine_register(If, Im, scales, iters, lr=3e-3, window=5, loss="lncc", beta1=0.9,
                    beta2=0.999, adam_eps=1e-8, cc_eps=1e-5):
    """Multi-scale affine pre-registration (R-aff).  Returns dict(theta, final_loss)."""
    If, Im = _f64(If), _f64(Im)
    D, H, W = _dims(If)
    p = _Params()
    p.n_levels = len(scales)
    for k, (s, t) in enumerate(zip(scales, iters)):
        p.scales[k] = int(s)
        p.iters[k] = int(t)
    p.lr, p.window = float(lr), int(window)
    p.loss = {"lncc": 0, "mse": 1}[loss]
    p.beta1, p.beta2, p.adam_eps, p.cc_eps = float(beta1), float(beta2), float(adam_eps), float(cc_eps)
    th = np.empty(12)
    fl = ctypes.c_double()
    _check(_L().or_affine_register(_p(If), _p(Im), D, H, W, ctypes.byref(p), _p(th),
                                   ctypes.byref(fl)), "affine_register")
    return dict(theta=th, final_loss=fl.value)


# ------------------------------------------------ stationary velocity field
def svf_loss_grad(If, Im, v, steps, window=5, loss="lncc", cc_eps=1e-5, mi_bins=32,
                  want_grad=True):
    """(L(I_f, I_m o exp(v)), grad_v L, exp(v) - id) (reading R-svfreg)."""
    If, Im, v = _f64(If), _f64(Im), _f64(v)
    D, H, W = _dims(If)
    p = _params([1], [0], window=window, loss=loss, cc_eps=cc_eps)
    p.mi_bins = int(mi_bins)
    rng = mi_range(If, Im)
    L = ctypes.c_double()
    gv = np.empty_like(v) if want_grad else None
    u = np.empty_like(v)
    _check(_L().or_svf_loss_grad(_p(If), _p(Im), D, H, W, ctypes.byref(p), int(steps), _p(rng),
                                 _p(v), ctypes.byref(L), _p(gv), _p(u)), "svf_loss_grad")
    return L.value, gv, u


def register_svf(If, Im, scales, iters, steps=7, mi_bins=32, **kw):
    """The Lie-algebra variant end to end (R-svfreg).  Returns dict(v, u, final_loss)."""
    If, Im = _f64(If), _f64(Im)
    D, H, W = _dims(If)
    p = _params(scales, iters, **kw)
    p.mi_bins = int(mi_bins)
    fs = level_shape((D, H, W), scales[-1])
    v, u = np.empty((3,) + fs), np.empty((3,) + fs)
    fl = ctypes.c_double()
    _check(_L().or_register_svf(_p(If), _p(Im), D, H, W, ctypes.byref(p), int(steps), _p(v),
                                _p(u), ctypes.byref(fl)), "register_svf")
    return dict(v=v, u=u, final_loss=fl.value)


# ------------------------------------------------------------- rigid stage
def rodrigues(w, want_grad=True):
    """R = exp([w]x) (3 x 3) and dR/dw_k (3 x 3 x 3) (reading R-rigid)."""
    w = _f64(w)
    R = np.empty(9)
    dR = np.empty(27) if want_grad else None
    _L().or_rodrigues(_p(w), _p(R), _p(dR))
    return R.reshape(3, 3), (dR.reshape(3, 3, 3) if want_grad else None)


def rigid_theta(rp, shape):
    rp = _f64(rp)
    th = np.empty(12)
    _check(_L().or_rigid_theta(_p(rp), *(int(n) for n in shape), _p(th)), "rigid_theta")
    return th


def rigid_loss_grad(If, Im, rp, full_shape=None, window=5, loss="lncc", cc_eps=1e-5):
    If, Im, rp = _f64(If), _f64(Im), _f64(rp)
    D, H, W = _dims(If)
    D0, H0, W0 = full_shape if full_shape is not None else (D, H, W)
    L = ctypes.c_double()
    g = np.empty(6)
    _check(_L().or_rigid_loss_grad(_p(If), _p(Im), D, H, W, D0, H0, W0, _p(rp),
                                   {"lncc": 0, "mse": 1}[loss], int(window), float(cc_eps),
                                   ctypes.byref(L), _p(g)), "rigid_loss_grad")
    return L.value, g


def rigid_register(If, Im, scales, iters, lr=3e-3, window=5, loss="lncc", beta1=0.9,
                   beta2=0.999, adam_eps=1e-8, cc_eps=1e-5):
    """Multi-scale rigid pre-registration (R-rigid).  Returns dict(rp, theta, final_loss)."""
    If, Im = _f64(If), _f64(Im)
    D, H, W = _dims(If)
    p = _params(scales, iters, lr=lr, window=window, loss=loss, beta1=beta1, beta2=beta2,
                adam_eps=adam_eps, cc_eps=cc_eps)
    rp = np.empty(6)
    fl = ctypes.c_double()
    _check(_L().or_rigid_register(_p(If), _p(Im), D, H, W, ctypes.byref(p), _p(rp),
                                  ctypes.byref(fl)), "rigid_register")
    return dict(rp=rp, theta=rigid_theta(rp, (D, H, W)), final_loss=fl.value)


# ---------------------------------------------------------------- inverse
def inverse_energy_grad(u, w, want_grad=True):
    u, w = _f64(u), _f64(w)
    _, D, H, W = u.shape
    E = ctypes.c_double()
    g = np.empty_like(u) if want_grad else None
    _check(_L().or_inverse_energy_grad(_p(u), _p(w), D, H, W, ctypes.byref(E), _p(g)),
           "inverse_energy_grad")
    return E.value, g


def inverse(u, scales, iters, lr=0.5, sigma_grad=1.0, sigma_warp=0.5, beta1=0.9, beta2=0.999,
            adam_eps=1e-8, c_lp=2.0):
    """Post-hoc inverse w of phi = id + u (reading R-inv).  Returns dict(w, final_energy)."""
    u = _f64(u)
    _, D, H, W = u.shape
    p = _Params()
    p.n_levels = len(scales)
    for k, (s, t) in enumerate(zip(scales, iters)):
        p.scales[k] = int(s)
        p.iters[k] = int(t)
    p.lr, p.sigma_grad, p.sigma_warp = float(lr), float(sigma_grad), float(sigma_warp)
    p.beta1, p.beta2, p.adam_eps, p.c_lp = float(beta1), float(beta2), float(adam_eps), float(c_lp)
    fs = level_shape((D, H, W), scales[-1])
    w = np.empty((3,) + fs)
    E = ctypes.c_double()
    _check(_L().or_inverse(_p(u), D, H, W, ctypes.byref(p), _p(w), ctypes.byref(E)), "inverse")
    return dict(w=w, final_energy=E.value)


# -------------------------------------------------------------- symmetric
def _params(scales, iters, lr=0.5, sigma_grad=1.0, sigma_warp=0.5, window=5, loss="lncc",
            beta1=0.9, beta2=0.999, adam_eps=1e-8, cc_eps=1e-5, c_lp=2.0, use_jac=False):
    p = _Params()
    p.n_levels = len(scales)
    for k, (s, t) in enumerate(zip(scales, iters)):
        p.scales[k] = int(s)
        p.iters[k] = int(t)
    p.lr, p.sigma_grad, p.sigma_warp = float(lr), float(sigma_grad), float(sigma_warp)
    p.window = int(window)
    p.loss = {"lncc": 0, "mse": 1, "mi": 2}[loss]
    p.beta1, p.beta2, p.adam_eps = float(beta1), float(beta2), float(adam_eps)
    p.cc_eps, p.c_lp = float(cc_eps), float(c_lp)
    p.use_jac = 1 if use_jac else 0
    return p


def symmetric_loss_grad(If, Im, uF, uM, window=5, loss="lncc", cc_eps=1e-5, want_grad=True):
    """L(I_f o phi_F, I_m o phi_M) and its derivatives in u_F, u_M (R-sym)."""
    If, Im, uF, uM = _f64(If), _f64(Im), _f64(uF), _f64(uM)
    D, H, W = _dims(If)
    p = _params([1], [0], window=window, loss=loss, cc_eps=cc_eps)
    L = ctypes.c_double()
    gF = np.empty_like(uF) if want_grad else None
    gM = np.empty_like(uM) if want_grad else None
    _check(_L().or_symmetric_loss_grad(_p(If), _p(Im), D, H, W, ctypes.byref(p), _p(uF), _p(uM),
                                       ctypes.byref(L), _p(gF), _p(gM)), "symmetric_loss_grad")
    return L.value, gF, gM


def register_symmetric(If, Im, scales, iters, inv_scales=(1,), inv_iters=(50,), **kw):
    """Symmetric registration (R-sym).  Returns dict(u, uF, uM, final_loss,
    mid_loss); u = phi_M o phi_F^-1 - id on the last level's grid."""
    If, Im = _f64(If), _f64(Im)
    D, H, W = _dims(If)
    if Im.shape != If.shape:
        raise ValueError("fixed and moving must share a grid")
    p = _params(scales, iters, **kw)
    ikw = {k: kw[k] for k in ("lr", "sigma_grad", "sigma_warp", "beta1", "beta2", "adam_eps",
                              "c_lp") if k in kw}
    pi = _params(inv_scales, inv_iters, **ikw)
    fs = level_shape((D, H, W), scales[-1])
    u, uF, uM = (np.empty((3,) + fs) for _ in range(3))
    fl, ml = ctypes.c_double(), ctypes.c_double()
    _check(_L().or_register_symmetric(_p(If), _p(Im), D, H, W, ctypes.byref(p), ctypes.byref(pi),
                                      _p(u), _p(uF), _p(uM), ctypes.byref(fl), ctypes.byref(ml)),
           "register_symmetric")
    return dict(u=u, uF=uF, uM=uM, final_loss=fl.value, mid_loss=ml.value)

"""Thin ctypes binding of libfa (include/fa.h).

Argument marshalling only: torch tensors provide device memory and the
current CUDA stream; every step runs in libfa's kernels.  Each function has
the name of the C entry point it calls.  If the library is missing the call
raises; there is no fallback implementation.

Layouts: volumes are float32 CUDA tensors [D, H, W] (or [1, D, H, W]);
fields are [3, D, H, W] with channel 0 the z component, in voxels.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional, Sequence

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libfa.so")

FA_OK = 0
FA_ERR_INVALID = 1
FA_ERR_NONFINITE, FA_ERR_TIMEOUT, FA_ERR_UNSUPPORTED = 5, 6, 7
STATUS_NAMES = {0: "FA_OK", 1: "FA_ERR_INVALID", 2: "FA_ERR_SHAPE", 3: "FA_ERR_DTYPE",
                4: "FA_ERR_CUDA", 5: "FA_ERR_NONFINITE", 6: "FA_ERR_TIMEOUT",
                7: "FA_ERR_UNSUPPORTED", 8: "FA_ERR_WORKSPACE"}
FA_F32, FA_BF16, FA_F16 = 0, 1, 2
FA_LOSS_LNCC, FA_LOSS_MSE, FA_LOSS_MI = 0, 1, 2
FA_MODE_FUSED, FA_MODE_PLAIN, FA_MODE_PERSISTENT = 0, 1, 2
(FA_K_FUSED_WARP_LNCC, FA_K_FUSED_LNCC_GRAD, FA_K_FUSED_SMOOTH_ADAM, FA_K_FUSED_COMPOSE,
 FA_K_PLAIN_ANY, FA_K_FUSED_ALL) = 0, 1, 2, 3, 4, 5

EXPORTED = ["fa_params_default", "fa_status_str", "fa_last_error", "fa_warp",
            "fa_lncc_workspace_size", "fa_lncc_fwd_bwd", "fa_mse_fwd_bwd",
            "fa_gauss_workspace_size", "fa_gauss_smooth", "fa_radam_workspace_size",
            "fa_radam_step", "fa_pyramid_level", "fa_upsample_field",
            "fa_register_workspace_size", "fa_register", "fa_ws_status", "fa_register_timed",
            "fa_launch_count", "fa_lncc_fwd_bwd_noalloc", "fa_register_batched_workspace_size",
            "fa_register_batched", "fa_warp_lncc_adjoint_workspace_size",
            "fa_warp_lncc_adjoint", "fa_autotune", "fa_autotune_reset", "fa_autotune_choices",
            "fa_autotune_set", "fa_jac_direction", "fa_compose", "fa_svf_exp_workspace_size",
            "fa_svf_exp", "fa_register_from", "fa_affine_workspace_size", "fa_affine_register",
            "fa_affine_field", "fa_inverse_workspace_size", "fa_inverse",
            "fa_inverse_energy_grad", "fa_register_symmetric_workspace_size",
            "fa_register_symmetric", "fa_symmetric_loss_grad_workspace_size",
            "fa_symmetric_loss_grad", "fa_mi_workspace_size", "fa_mi_fwd_bwd",
            "fa_rigid_register", "fa_register_svf_workspace_size", "fa_register_svf",
            "fa_svf_loss_grad", "fa_selftest_wait_timeout",
            "fa_register_lockstep_workspace_size", "fa_register_batched_lockstep",
            "fa_pyramid_workspace_size", "fa_pyramid", "fa_workspace_size",
            "fa_graph_cache_clear", "fa_selftest_grid_barrier", "fa_rigid_theta"]


class FAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Vol(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("C", ctypes.c_int32),
                ("D", ctypes.c_int32), ("H", ctypes.c_int32), ("W", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int32), ("scales", ctypes.c_int32 * 8),
                ("iters", ctypes.c_int32 * 8), ("lr", ctypes.c_float),
                ("sigma_grad", ctypes.c_float), ("sigma_warp", ctypes.c_float),
                ("window", ctypes.c_int32), ("loss", ctypes.c_int32), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("adam_eps", ctypes.c_float),
                ("cc_eps", ctypes.c_float), ("c_lp", ctypes.c_float), ("mode", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("use_jac", ctypes.c_int32), ("mi_bins", ctypes.c_int32),
                ("state_storage", ctypes.c_int32),
                ("field_storage", ctypes.c_int32)]


class KernelTimer(ctypes.Structure):
    _fields_ = [("kernel_id", ctypes.c_int32), ("level", ctypes.c_int32),
                ("capacity", ctypes.c_int32), ("count", ctypes.c_int32),
                ("start_events", ctypes.POINTER(ctypes.c_void_p)),
                ("stop_events", ctypes.POINTER(ctypes.c_void_p))]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libfa.so (built by paper_2404_01249_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libfa is not built ({path} missing); run "
                           "`python -m paper_2404_01249_gb300.build` or __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, V, vp, sz, i32, f32 = (ctypes.POINTER(Params), ctypes.POINTER(Vol), ctypes.c_void_p,
                              ctypes.c_size_t, ctypes.c_int32, ctypes.c_float)
    fp = ctypes.POINTER(ctypes.c_float)
    sig = {
        "fa_params_default": (i32, [P]),
        "fa_status_str": (ctypes.c_char_p, [i32]),
        "fa_last_error": (ctypes.c_char_p, []),
        "fa_launch_count": (ctypes.c_uint64, []),
        "fa_warp": (i32, [V, V, V, V, vp]),
        "fa_lncc_workspace_size": (sz, [i32, i32, i32]),
        "fa_lncc_fwd_bwd": (i32, [V, V, i32, f32, vp, V, V, vp, sz, vp]),
        "fa_lncc_fwd_bwd_noalloc": (i32, [V, V, i32, f32, vp, V, V, vp]),
        "fa_mse_fwd_bwd": (i32, [V, V, vp, V, V, vp, sz, vp]),
        "fa_gauss_workspace_size": (sz, [i32, i32, i32, i32]),
        "fa_gauss_smooth": (i32, [V, V, f32, vp, sz, vp]),
        "fa_radam_workspace_size": (sz, [i32, i32, i32]),
        "fa_radam_step": (i32, [V, V, V, V, V, vp, P, vp, vp, sz, vp]),
        "fa_pyramid_level": (i32, [V, i32, V, vp, sz, vp]),
        "fa_pyramid_workspace_size": (sz, [i32, i32, i32, P]),
        "fa_pyramid": (i32, [V, P, V, vp, sz, vp]),
        "fa_workspace_size": (sz, [V, P]),
        "fa_graph_cache_clear": (i32, []),
        "fa_selftest_grid_barrier": (i32, [vp, sz, ctypes.c_int64, vp]),
        "fa_rigid_theta": (i32, [vp, i32, i32, i32, vp, vp]),
        "fa_upsample_field": (i32, [V, V, i32, vp]),
        "fa_register_workspace_size": (sz, [i32, i32, i32, P]),
        "fa_register": (i32, [V, V, P, V, vp, fp, vp, sz, vp]),
        "fa_ws_status": (i32, [vp, vp]),
        "fa_register_timed": (i32, [V, V, P, V, vp, fp, vp, sz, vp,
                                    ctypes.POINTER(KernelTimer)]),
        "fa_register_batched_workspace_size": (sz, [i32, V, i32, P, i32]),
        "fa_register_batched": (i32, [i32, V, V, i32, P, V, vp, vp, i32, vp, sz, vp]),
        "fa_register_lockstep_workspace_size": (sz, [i32, V, i32, P, i32]),
        "fa_register_batched_lockstep": (i32, [i32, V, V, i32, P, V, vp, vp, i32, vp, sz, vp]),
        "fa_warp_lncc_adjoint_workspace_size": (sz, [i32, i32, i32]),
        "fa_warp_lncc_adjoint": (i32, [V, V, V, i32, f32, vp, V, V, V, vp, sz, vp]),
        "fa_autotune": (i32, [i32, i32, i32, P, vp, sz, vp]),
        "fa_autotune_reset": (i32, []),
        "fa_autotune_choices": (i32, [ctypes.POINTER(ctypes.c_int32), i32]),
        "fa_autotune_set": (i32, [ctypes.POINTER(ctypes.c_int32)]),
        "fa_jac_direction": (i32, [V, V, V, vp]),
        "fa_compose": (i32, [V, V, V, vp]),
        "fa_svf_exp_workspace_size": (sz, [i32, i32, i32]),
        "fa_svf_exp": (i32, [V, i32, V, vp, sz, vp]),
        "fa_register_from": (i32, [V, V, P, V, V, vp, fp, vp, sz, vp]),
        "fa_affine_workspace_size": (sz, [i32, i32, i32, P]),
        "fa_affine_register": (i32, [V, V, P, vp, V, vp, vp, sz, vp]),
        "fa_affine_field": (i32, [vp, V, vp]),
        "fa_rigid_register": (i32, [V, V, P, vp, vp, V, vp, vp, sz, vp]),
        "fa_register_svf_workspace_size": (sz, [i32, i32, i32, P, i32]),
        "fa_register_svf": (i32, [V, V, P, i32, V, V, vp, vp, sz, vp]),
        "fa_svf_loss_grad": (i32, [V, V, V, P, i32, vp, V, V, vp, sz, vp]),
        "fa_selftest_wait_timeout": (i32, [vp, sz, ctypes.c_int64, vp]),
        "fa_inverse_workspace_size": (sz, [i32, i32, i32, P]),
        "fa_inverse": (i32, [V, P, V, vp, vp, sz, vp]),
        "fa_inverse_energy_grad": (i32, [V, V, vp, V, vp, sz, vp]),
        "fa_register_symmetric_workspace_size": (sz, [i32, i32, i32, P, P]),
        "fa_register_symmetric": (i32, [V, V, P, P, V, V, V, vp, vp, vp, sz, vp]),
        "fa_symmetric_loss_grad_workspace_size": (sz, [i32, i32, i32]),
        "fa_mi_workspace_size": (sz, [i32]),
        "fa_mi_fwd_bwd": (i32, [V, V, i32, vp, vp, V, vp, sz, vp]),
        "fa_symmetric_loss_grad": (i32, [V, V, V, V, i32, i32, f32, vp, V, V, vp, sz, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != FA_OK:
        raise FAError(status, load().fa_last_error().decode())


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


_DTYPES = {torch.float32: FA_F32, torch.bfloat16: FA_BF16, torch.float16: FA_F16}


def _vol(t: Optional[torch.Tensor], C: int, half_ok: bool = False):
    if t is None:
        return None
    ok = (torch.float32, torch.bfloat16, torch.float16) if half_ok else (torch.float32,)
    if not t.is_cuda or t.dtype not in ok or not t.is_contiguous():
        raise ValueError(f"expected a contiguous CUDA tensor of dtype {ok}")
    shp = tuple(t.shape)
    if C == 1 and len(shp) == 3:
        shp = (1,) + shp
    if len(shp) != 4 or shp[0] != C:
        raise ValueError(f"expected shape [{C}, D, H, W], got {tuple(t.shape)}")
    return ctypes.byref(Vol(t.data_ptr(), _DTYPES[t.dtype], C, shp[1], shp[2], shp[3]))


def _ptr(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def workspace(nbytes: int, device=None) -> torch.Tensor:
    """Caller-owned scratch buffer (torch allocations are 256-byte aligned)."""
    ws = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device or "cuda")
    assert ws.data_ptr() % 256 == 0
    return ws


@dataclasses.dataclass
class RegParams:
    scales: Sequence[int] = (4, 2, 1)
    iters: Sequence[int] = (200, 100, 50)
    lr: float = 0.5
    sigma_grad: float = 1.0
    sigma_warp: float = 0.5
    window: int = 5
    loss: str = "lncc"
    beta1: float = 0.9
    beta2: float = 0.999
    adam_eps: float = 1e-8
    cc_eps: float = 1e-5
    c_lp: float = 2.0
    mode: str = "fused"
    graph: bool = True   # record the launch sequence once, replay it on identical calls
    use_jac: bool = False  # steepest Eulerian direction J(phi)^T dL/dphi
    mi_bins: int = 32      # histogram bins of the MI loss
    state: str = "f32"     # storage of the Adam moments m, nu: "f32" or "bf16"
    field: str = "f32"     # storage of the displacement u between iterations: "f32" or "f16"

    def to_c(self) -> Params:
        p = Params()
        _check(load().fa_params_default(ctypes.byref(p)))
        if len(self.scales) != len(self.iters) or not 1 <= len(self.scales) <= 8:
            raise ValueError("1..8 levels with one iteration count each")
        p.n_levels = len(self.scales)
        for k, (s, t) in enumerate(zip(self.scales, self.iters)):
            p.scales[k] = int(s)
            p.iters[k] = int(t)
        p.lr, p.sigma_grad, p.sigma_warp = self.lr, self.sigma_grad, self.sigma_warp
        p.window = int(self.window)
        p.loss = {"lncc": FA_LOSS_LNCC, "mse": FA_LOSS_MSE, "mi": FA_LOSS_MI}[self.loss]
        p.mi_bins = int(self.mi_bins)
        p.beta1, p.beta2, p.adam_eps = self.beta1, self.beta2, self.adam_eps
        p.cc_eps, p.c_lp = self.cc_eps, self.c_lp
        p.mode = {"fused": FA_MODE_FUSED, "plain": FA_MODE_PLAIN,
                  "persistent": FA_MODE_PERSISTENT}[self.mode]
        p.storage = FA_F32
        p.graph = 1 if self.graph else 0
        p.use_jac = 1 if self.use_jac else 0
        p.state_storage = {"f32": FA_F32, "bf16": FA_BF16, "f16": FA_F16}[self.state]
        p.field_storage = {"f32": FA_F32, "bf16": FA_BF16, "f16": FA_F16}[self.field]
        return p


def level_size(n: int, s: int) -> int:
    return max(1, n // s)


# ------------------------------------------------------------------ entry points

def fa_warp(moving: torch.Tensor, u: torch.Tensor, want_grad: bool = True, out=None, grad=None):
    D, H, W = moving.shape[-3:]
    out = out if out is not None else torch.empty((D, H, W), device=moving.device)
    if want_grad and grad is None:
        grad = torch.empty((3, D, H, W), device=moving.device)
    _check(load().fa_warp(_vol(moving, 1), _vol(u, 3), _vol(out, 1),
                          _vol(grad, 3) if want_grad else None, _stream()))
    return (out, grad) if want_grad else out


def fa_lncc_fwd_bwd(fixed, warped, window: int = 5, cc_eps: float = 1e-5, want_dJ: bool = True,
                    want_dI: bool = False, ws: Optional[torch.Tensor] = None):
    D, H, W = fixed.shape[-3:]
    lib = load()
    need = lib.fa_lncc_workspace_size(D, H, W)
    ws = ws if ws is not None else workspace(need, fixed.device)
    loss = torch.empty((), device=fixed.device)
    dJ = torch.empty((D, H, W), device=fixed.device) if want_dJ else None
    dI = torch.empty((D, H, W), device=fixed.device) if want_dI else None
    _check(lib.fa_lncc_fwd_bwd(_vol(fixed, 1), _vol(warped, 1), window, cc_eps, _ptr(loss),
                               _vol(dJ, 1), _vol(dI, 1), _ptr(ws), ws.numel(), _stream()))
    return dict(loss=loss, dJ=dJ, dI=dI)


def fa_mse_fwd_bwd(fixed, warped, want_dJ: bool = True, want_dI: bool = False):
    D, H, W = fixed.shape[-3:]
    lib = load()
    ws = workspace(lib.fa_lncc_workspace_size(D, H, W), fixed.device)
    loss = torch.empty((), device=fixed.device)
    dJ = torch.empty((D, H, W), device=fixed.device) if want_dJ else None
    dI = torch.empty((D, H, W), device=fixed.device) if want_dI else None
    _check(lib.fa_mse_fwd_bwd(_vol(fixed, 1), _vol(warped, 1), _ptr(loss), _vol(dJ, 1),
                              _vol(dI, 1), _ptr(ws), ws.numel(), _stream()))
    return dict(loss=loss, dJ=dJ, dI=dI)


def fa_gauss_smooth(x: torch.Tensor, sigma: float, out=None):
    squeeze = x.dim() == 3
    xx = x.unsqueeze(0) if squeeze else x
    C, D, H, W = xx.shape
    out = out if out is not None else torch.empty_like(xx)
    out4 = out.view(C, D, H, W)
    lib = load()
    ws = workspace(lib.fa_gauss_workspace_size(C, D, H, W), x.device)
    _check(lib.fa_gauss_smooth(_vol(xx, C), _vol(out4, C), sigma, _ptr(ws), ws.numel(),
                               _stream()))
    return out4[0] if squeeze else out4


def fa_radam_step(u_in, m, v, g, t, params: RegParams, u_out=None):
    """One Riemannian Adam step.  `t` is the device step counter (an int32
    CUDA tensor holding the steps taken so far, advanced by the call) or a
    Python int, the step number after increment (a counter holding t - 1 is
    made for the call).  Updates m, v in place; returns (u_out, eps_t as a
    0-dim CUDA tensor)."""
    D, H, W = u_in.shape[-3:]
    lib = load()
    u_out = u_out if u_out is not None else torch.empty_like(u_in)
    eps_t = torch.empty((), device=u_in.device)
    if isinstance(t, torch.Tensor):
        t_dev = t
    else:
        t_dev = torch.tensor([int(t) - 1], dtype=torch.int32, device=u_in.device)
    ws = workspace(lib.fa_radam_workspace_size(D, H, W), u_in.device)
    p = params.to_c()
    _check(lib.fa_radam_step(_vol(u_in, 3), _vol(u_out, 3), _vol(m, 3, True), _vol(v, 3, True),
                             _vol(g, 3), _ptr(t_dev), ctypes.byref(p), _ptr(eps_t), _ptr(ws),
                             ws.numel(), _stream()))
    return u_out, eps_t


def fa_pyramid_level(img: torch.Tensor, s: int):
    D, H, W = img.shape[-3:]
    out = torch.empty((level_size(D, s), level_size(H, s), level_size(W, s)), device=img.device)
    lib = load()
    ws = workspace(lib.fa_gauss_workspace_size(1, D, H, W), img.device)
    _check(lib.fa_pyramid_level(_vol(img, 1), s, _vol(out, 1), _ptr(ws), ws.numel(), _stream()))
    return out


def fa_pyramid(img: torch.Tensor, params: RegParams):
    """Every level of params' pyramid (Algorithm 1 "downsample") in one call;
    returns the list of level volumes, coarsest first as params orders them."""
    D, H, W = img.shape[-3:]
    lib = load()
    p = params.to_c()
    levels = [torch.empty((level_size(D, s), level_size(H, s), level_size(W, s)),
                          device=img.device) for s in params.scales]
    arr = (Vol * len(levels))(*[_vol_struct(x, 1) for x in levels])
    n = lib.fa_pyramid_workspace_size(D, H, W, ctypes.byref(p))
    if n == 0:
        _check(1)
    ws = workspace(n, img.device)
    _check(lib.fa_pyramid(_vol(img, 1), ctypes.byref(p), arr, _ptr(ws), ws.numel(), _stream()))
    return levels


def fa_graph_cache_clear():
    _check(load().fa_graph_cache_clear())


def fa_upsample_field(coarse: torch.Tensor, shape, power: int):
    fine = torch.empty((3,) + tuple(shape), device=coarse.device)
    _check(load().fa_upsample_field(_vol(coarse, 3), _vol(fine, 3), power, _stream()))
    return fine


def fa_register_workspace_size(shape, params: RegParams) -> int:
    p = params.to_c()
    n = load().fa_register_workspace_size(*[int(s) for s in shape], ctypes.byref(p))
    if n == 0:
        _check(1)
    return n


def fa_register(fixed, moving, params: RegParams, ws: Optional[torch.Tensor] = None,
                sync: bool = True, u_out=None, loss_out=None, timer: Optional[KernelTimer] = None,
                u_init: Optional[torch.Tensor] = None):
    """Whole registration.  Returns dict(u=[3, d, h, w] tensor of the last
    level, loss=0-dim CUDA tensor, final_loss=float or None if sync=False)."""
    D, H, W = fixed.shape[-3:]
    p = params.to_c()
    p.storage = _DTYPES.get(fixed.dtype, FA_F32)  # 16-bit images are widened in the workspace
    lib = load()
    need = lib.fa_register_workspace_size(D, H, W, ctypes.byref(p))
    if need == 0:
        _check(lib.fa_register_workspace_size(D, H, W, ctypes.byref(p)) or 1)
    ws = ws if ws is not None else workspace(need, fixed.device)
    s = params.scales[-1]
    if u_out is None:
        u_out = torch.empty((3, level_size(D, s), level_size(H, s), level_size(W, s)),
                            device=fixed.device)
    loss = loss_out if loss_out is not None else torch.empty((), device=fixed.device)
    host = ctypes.c_float() if sync else None
    args = (_vol(fixed, 1, True), _vol(moving, 1, True), ctypes.byref(p), _vol(u_out, 3), _ptr(loss),
            ctypes.byref(host) if sync else None, _ptr(ws), ws.numel(), _stream())
    if u_init is not None:
        if timer is not None:
            raise ValueError("u_init and timer cannot be combined")
        _check(lib.fa_register_from(args[0], args[1], args[2], _vol(u_init, 3), *args[3:]))
    elif timer is None:
        _check(lib.fa_register(*args))
    else:
        _check(lib.fa_register_timed(*args, ctypes.byref(timer)))
    return dict(u=u_out, loss=loss, final_loss=host.value if sync else None)


def _vol_struct(t: torch.Tensor, C: int, half_ok: bool = False) -> Vol:
    _vol(t, C, half_ok)  # validation
    shp = tuple(t.shape) if t.dim() == 4 else (1,) + tuple(t.shape)
    return Vol(t.data_ptr(), _DTYPES[t.dtype], C, shp[1], shp[2], shp[3])


def _batched_call(size_fn, run_fn, fixed, moving, params, count, ws, sync):
    n_pairs, n_cfg = len(fixed), len(params)
    if len(moving) != n_pairs:
        raise ValueError("fixed and moving need the same number of volumes")
    dev = fixed[0].device
    fv = (Vol * n_pairs)(*[_vol_struct(t, 1, True) for t in fixed])
    mv = (Vol * n_pairs)(*[_vol_struct(t, 1, True) for t in moving])
    if len({t.dtype for t in list(fixed) + list(moving)}) != 1:
        raise ValueError("all images of one batched call share a dtype")
    cs = [q.to_c() for q in params]
    for c in cs:
        c.storage = _DTYPES[fixed[0].dtype]
    pc = (Params * n_cfg)(*cs)
    need = size_fn(n_pairs, fv, n_cfg, pc, count)
    if need == 0:
        raise FAError(FA_ERR_INVALID, load().fa_last_error().decode())
    ws = ws if ws is not None else workspace(need, dev)
    outs = []
    for i in range(n_pairs):
        D, H, W = fixed[i].shape[-3:]
        for q in params:
            s = q.scales[-1]
            outs.append(torch.empty((3, level_size(D, s), level_size(H, s), level_size(W, s)),
                                    device=dev))
    uv = (Vol * len(outs))(*[_vol_struct(t, 3) for t in outs])
    loss = torch.empty(len(outs), device=dev)
    status = torch.zeros(len(outs), dtype=torch.int32, device=dev)
    _check(run_fn(n_pairs, fv, mv, n_cfg, pc, uv, _ptr(loss), _ptr(status), count, _ptr(ws),
                  ws.numel(), _stream()))
    res = [dict(u=u, loss=loss[j]) for j, u in enumerate(outs)]
    if sync:
        torch.cuda.current_stream().synchronize()
        lh, sh = loss.cpu().tolist(), status.cpu().tolist()
        for j, r in enumerate(res):
            r["final_loss"], r["status"] = lh[j], sh[j]
    return res


def fa_register_batched(fixed: list, moving: list, params: list, concurrency: int = 4,
                        ws: Optional[torch.Tensor] = None, sync: bool = True):
    """Registers every pair under every parameter set (job = pair * len(params)
    + set) concurrently.  Returns a list of dicts (u, loss tensor, final_loss
    and status when sync=True), one per job."""
    lib = load()
    return _batched_call(lib.fa_register_batched_workspace_size, lib.fa_register_batched, fixed,
                         moving, params, concurrency, ws, sync)


def fa_register_batched_lockstep(fixed: list, moving: list, params: list,
                                 jobs_per_wave: int = 64, ws: Optional[torch.Tensor] = None,
                                 sync: bool = True):
    """The jobs of fa_register_batched advancing together: each iteration is
    one launch of every fused kernel over all jobs of a wave of
    `jobs_per_wave` jobs.  Same results and return value."""
    lib = load()
    return _batched_call(lib.fa_register_lockstep_workspace_size,
                         lib.fa_register_batched_lockstep, fixed, moving, params, jobs_per_wave,
                         ws, sync)


def fa_warp_lncc_adjoint(fixed, moving, u, window: int = 5, cc_eps: float = 1e-5,
                         want_u: bool = True, want_fixed: bool = True, want_moving: bool = True,
                         ws: Optional[torch.Tensor] = None):
    """L = LNCC(fixed, moving o (id + u)) and its derivatives.  Returns
    dict(loss=0-dim tensor, dL_du, dL_dfixed, dL_dmoving) (None where not
    wanted); asynchronous on the current stream."""
    D, H, W = fixed.shape[-3:]
    lib = load()
    need = lib.fa_warp_lncc_adjoint_workspace_size(D, H, W)
    ws = ws if ws is not None else workspace(need, fixed.device)
    loss = torch.empty((), device=fixed.device)
    du = torch.empty((3, D, H, W), device=fixed.device) if want_u else None
    dfx = torch.empty((D, H, W), device=fixed.device) if want_fixed else None
    dmv = torch.empty((D, H, W), device=fixed.device) if want_moving else None
    _check(lib.fa_warp_lncc_adjoint(_vol(fixed, 1), _vol(moving, 1), _vol(u, 3), int(window),
                                    float(cc_eps), _ptr(loss), _vol(du, 3), _vol(dfx, 1),
                                    _vol(dmv, 1), _ptr(ws), ws.numel(), _stream()))
    return dict(loss=loss, dL_du=du, dL_dfixed=dfx, dL_dmoving=dmv)


def fa_autotune(shape, params: RegParams, ws: Optional[torch.Tensor] = None, device=None):
    """Tunes the fused kernels' tiles for registrations of this shape and
    these parameters (waits for the GPU).  Returns the recorded choices."""
    D, H, W = shape
    p = params.to_c()
    lib = load()
    need = lib.fa_register_workspace_size(D, H, W, ctypes.byref(p))
    ws = ws if ws is not None else workspace(need, device or torch.device("cuda"))
    _check(lib.fa_autotune(D, H, W, ctypes.byref(p), _ptr(ws), ws.numel(), _stream()))
    return fa_autotune_choices()


def fa_autotune_choices():
    lib = load()
    n = lib.fa_autotune_choices(None, 0)
    rows = (ctypes.c_int32 * (8 * max(n, 1)))()
    n = lib.fa_autotune_choices(rows, n)
    keys = ("kernel", "radius", "compose_variant", "D", "H", "W", "wide", "tz")
    return [dict(zip(keys, rows[8 * i:8 * i + 8])) for i in range(n)]


def fa_autotune_set(kernel: int, radius: int, compose_variant: int, D: int, H: int, W: int,
                    wide: int, tz: int):
    row = (ctypes.c_int32 * 8)(kernel, radius, compose_variant, D, H, W, wide, tz)
    _check(load().fa_autotune_set(row))


def fa_autotune_reset():
    _check(load().fa_autotune_reset())


def fa_jac_direction(g: torch.Tensor, u: torch.Tensor, out: Optional[torch.Tensor] = None):
    """J(phi)^T g with J(phi) = I + grad u (out may be g: in place)."""
    out = out if out is not None else torch.empty_like(g)
    _check(load().fa_jac_direction(_vol(g, 3), _vol(u, 3), _vol(out, 3), _stream()))
    return out


def fa_compose(u: torch.Tensor, delta: torch.Tensor, out: Optional[torch.Tensor] = None):
    """delta + u o (id + delta)."""
    out = out if out is not None else torch.empty_like(u)
    _check(load().fa_compose(_vol(u, 3), _vol(delta, 3), _vol(out, 3), _stream()))
    return out


def fa_svf_exp(v: torch.Tensor, steps: int, out: Optional[torch.Tensor] = None):
    """exp(v) - id by scaling and squaring."""
    D, H, W = v.shape[-3:]
    out = out if out is not None else torch.empty_like(v)
    lib = load()
    ws = workspace(lib.fa_svf_exp_workspace_size(D, H, W), v.device)
    _check(lib.fa_svf_exp(_vol(v, 3), int(steps), _vol(out, 3), _ptr(ws), ws.numel(), _stream()))
    return out


def fa_affine_register(fixed, moving, params: RegParams, sync: bool = True):
    """Affine pre-registration (see fa.h).  Returns dict(theta=12 floats on the
    device, u=[3, d, h, w] of the last level, loss, final_loss)."""
    D, H, W = fixed.shape[-3:]
    p = params.to_c()
    lib = load()
    need = lib.fa_affine_workspace_size(D, H, W, ctypes.byref(p))
    if need == 0:
        raise FAError(FA_ERR_INVALID, lib.fa_last_error().decode())
    ws = workspace(need, fixed.device)
    s = params.scales[-1]
    theta = torch.empty(12, device=fixed.device)
    u = torch.empty((3, level_size(D, s), level_size(H, s), level_size(W, s)), device=fixed.device)
    loss = torch.empty((), device=fixed.device)
    _check(lib.fa_affine_register(_vol(fixed, 1), _vol(moving, 1), ctypes.byref(p), _ptr(theta),
                                  _vol(u, 3), _ptr(loss), _ptr(ws), ws.numel(), _stream()))
    out = dict(theta=theta, u=u, loss=loss)
    if sync:
        torch.cuda.current_stream().synchronize()
        out["final_loss"] = float(loss)
    return out


def fa_rigid_register(fixed, moving, params: RegParams, sync: bool = True):
    """Rigid pre-registration (see fa.h).  Returns dict(rp=6 floats (w, t),
    theta=12 floats, u=[3, d, h, w] of the last level, loss, final_loss)."""
    D, H, W = fixed.shape[-3:]
    p = params.to_c()
    lib = load()
    need = lib.fa_affine_workspace_size(D, H, W, ctypes.byref(p))
    if need == 0:
        raise FAError(FA_ERR_INVALID, lib.fa_last_error().decode())
    ws = workspace(need, fixed.device)
    s = params.scales[-1]
    rp = torch.empty(6, device=fixed.device)
    theta = torch.empty(12, device=fixed.device)
    u = torch.empty((3, level_size(D, s), level_size(H, s), level_size(W, s)), device=fixed.device)
    loss = torch.empty((), device=fixed.device)
    _check(lib.fa_rigid_register(_vol(fixed, 1), _vol(moving, 1), ctypes.byref(p), _ptr(rp),
                                 _ptr(theta), _vol(u, 3), _ptr(loss), _ptr(ws), ws.numel(),
                                 _stream()))
    out = dict(rp=rp, theta=theta, u=u, loss=loss)
    if sync:
        torch.cuda.current_stream().synchronize()
        out["final_loss"] = float(loss)
    return out


def fa_affine_field(theta: torch.Tensor, shape, out: Optional[torch.Tensor] = None):
    out = out if out is not None else torch.empty((3,) + tuple(shape), device=theta.device)
    _check(load().fa_affine_field(_ptr(theta), _vol(out, 3), _stream()))
    return out


def fa_inverse(u: torch.Tensor, params: RegParams, sync: bool = True):
    """Post-hoc inverse w of the displacement u (see fa.h).  Returns
    dict(w=[3, d, h, w] of the last level, energy, final_energy)."""
    D, H, W = u.shape[-3:]
    p = params.to_c()
    lib = load()
    need = lib.fa_inverse_workspace_size(D, H, W, ctypes.byref(p))
    if need == 0:
        raise FAError(FA_ERR_INVALID, lib.fa_last_error().decode())
    ws = workspace(need, u.device)
    s = params.scales[-1]
    w = torch.empty((3, level_size(D, s), level_size(H, s), level_size(W, s)), device=u.device)
    energy = torch.empty((), device=u.device)
    _check(lib.fa_inverse(_vol(u, 3), ctypes.byref(p), _vol(w, 3), _ptr(energy), _ptr(ws),
                          ws.numel(), _stream()))
    out = dict(w=w, energy=energy)
    if sync:
        torch.cuda.current_stream().synchronize()
        out["final_energy"] = float(energy)
    return out


def fa_inverse_energy_grad(u: torch.Tensor, w: torch.Tensor):
    """(energy, dE/dw) of the inverse-consistency energy on one grid."""
    D, H, W = u.shape[-3:]
    lib = load()
    p = RegParams(scales=(1,), iters=(0,)).to_c()
    ws = workspace(lib.fa_inverse_workspace_size(D, H, W, ctypes.byref(p)), u.device)
    g = torch.empty_like(w)
    energy = torch.empty((), device=u.device)
    _check(lib.fa_inverse_energy_grad(_vol(u, 3), _vol(w, 3), _ptr(energy), _vol(g, 3),
                                      _ptr(ws), ws.numel(), _stream()))
    return energy, g


def fa_register_symmetric(fixed, moving, params: RegParams, inv_params: RegParams,
                          sync: bool = True):
    """Symmetric registration (see fa.h).  Returns dict(u, uF, uM on the last
    level's grid, loss, mid_loss, final_loss, final_mid_loss)."""
    D, H, W = fixed.shape[-3:]
    p, pi = params.to_c(), inv_params.to_c()
    p.storage = _DTYPES.get(fixed.dtype, FA_F32)  # 16-bit images are widened in the workspace
    lib = load()
    need = lib.fa_register_symmetric_workspace_size(D, H, W, ctypes.byref(p), ctypes.byref(pi))
    if need == 0:
        raise FAError(FA_ERR_INVALID, lib.fa_last_error().decode())
    ws = workspace(need, fixed.device)
    s = params.scales[-1]
    shape = (3, level_size(D, s), level_size(H, s), level_size(W, s))
    u, uF, uM = (torch.empty(shape, device=fixed.device) for _ in range(3))
    loss, mid = torch.empty((), device=fixed.device), torch.empty((), device=fixed.device)
    _check(lib.fa_register_symmetric(_vol(fixed, 1, half_ok=True), _vol(moving, 1, half_ok=True),
                                     ctypes.byref(p), ctypes.byref(pi), _vol(u, 3), _vol(uF, 3),
                                     _vol(uM, 3), _ptr(loss), _ptr(mid), _ptr(ws), ws.numel(),
                                     _stream()))
    out = dict(u=u, uF=uF, uM=uM, loss=loss, mid_loss=mid)
    if sync:
        torch.cuda.current_stream().synchronize()
        out["final_loss"], out["final_mid_loss"] = float(loss), float(mid)
    return out


def fa_symmetric_loss_grad(fixed, moving, uF, uM, window: int = 5, loss: str = "lncc",
                           cc_eps: float = 1e-5):
    """(L, dL/du_F, dL/du_M) of L(I_f o phi_F, I_m o phi_M) on one grid."""
    D, H, W = fixed.shape[-3:]
    lib = load()
    ws = workspace(lib.fa_symmetric_loss_grad_workspace_size(D, H, W), fixed.device)
    gF, gM = torch.empty_like(uF), torch.empty_like(uM)
    L = torch.empty((), device=fixed.device)
    _check(lib.fa_symmetric_loss_grad(_vol(fixed, 1), _vol(moving, 1), _vol(uF, 3), _vol(uM, 3),
                                      {"lncc": FA_LOSS_LNCC, "mse": FA_LOSS_MSE}[loss],
                                      int(window), float(cc_eps), _ptr(L), _vol(gF, 3),
                                      _vol(gM, 3), _ptr(ws), ws.numel(), _stream()))
    return L, gF, gM


def fa_mi_fwd_bwd(fixed, warped, bins: int = 32, rng: Optional[torch.Tensor] = None,
                  want_dJ: bool = True):
    """L = -MI(fixed, warped) and dL/dwarped (see fa.h); rng: 4 device floats
    (lo_f, hi_f, lo_J, hi_J) or None for the two images' own ranges."""
    lib = load()
    need = lib.fa_mi_workspace_size(int(bins))
    if need == 0:
        raise FAError(FA_ERR_INVALID, lib.fa_last_error().decode())
    ws = workspace(need, fixed.device)
    loss = torch.empty((), device=fixed.device)
    dJ = torch.empty_like(warped) if want_dJ else None
    _check(lib.fa_mi_fwd_bwd(_vol(fixed, 1), _vol(warped, 1), int(bins),
                             _ptr(rng) if rng is not None else None, _ptr(loss), _vol(dJ, 1),
                             _ptr(ws), ws.numel(), _stream()))
    return dict(loss=loss, dJ=dJ)


def fa_register_svf(fixed, moving, params: RegParams, steps: int = 7, sync: bool = True):
    """The Lie-algebra (exp) registration (see fa.h).  Returns dict(u=exp(v) -
    id and v on the last level's grid, loss, final_loss)."""
    D, H, W = fixed.shape[-3:]
    p = params.to_c()
    p.storage = _DTYPES.get(fixed.dtype, FA_F32)
    lib = load()
    need = lib.fa_register_svf_workspace_size(D, H, W, ctypes.byref(p), int(steps))
    if need == 0:
        raise FAError(FA_ERR_INVALID, lib.fa_last_error().decode())
    ws = workspace(need, fixed.device)
    s = params.scales[-1]
    shape = (3, level_size(D, s), level_size(H, s), level_size(W, s))
    u, v = torch.empty(shape, device=fixed.device), torch.empty(shape, device=fixed.device)
    loss = torch.empty((), device=fixed.device)
    _check(lib.fa_register_svf(_vol(fixed, 1, half_ok=True), _vol(moving, 1, half_ok=True),
                               ctypes.byref(p), int(steps), _vol(u, 3), _vol(v, 3), _ptr(loss),
                               _ptr(ws), ws.numel(), _stream()))
    out = dict(u=u, v=v, loss=loss)
    if sync:
        torch.cuda.current_stream().synchronize()
        out["final_loss"] = float(loss)
    return out


def fa_svf_loss_grad(fixed, moving, v, steps: int, params: Optional[RegParams] = None):
    """(L(I_f, I_m o exp(v)), grad_v L, exp(v) - id) on one grid."""
    D, H, W = fixed.shape[-3:]
    P = params or RegParams(scales=(1,), iters=(0,))
    p = P.to_c()
    p.n_levels, p.scales[0], p.iters[0] = 1, 1, 0
    lib = load()
    need = lib.fa_register_svf_workspace_size(D, H, W, ctypes.byref(p), int(steps))
    if need == 0:
        raise FAError(FA_ERR_INVALID, lib.fa_last_error().decode())
    ws = workspace(need, fixed.device)
    g, u = torch.empty_like(v), torch.empty_like(v)
    loss = torch.empty((), device=fixed.device)
    _check(lib.fa_svf_loss_grad(_vol(fixed, 1), _vol(moving, 1), _vol(v, 3), ctypes.byref(p),
                                int(steps), _ptr(loss), _vol(g, 3), _vol(u, 3), _ptr(ws),
                                ws.numel(), _stream()))
    return loss, g, u


def fa_selftest_wait_timeout(limit_cycles: int = 1 << 20):
    """Runs the bounded-wait self-test (see fa.h) and returns the status its
    workspace reports (FA_ERR_TIMEOUT expected)."""
    lib = load()
    ws = workspace(256, torch.device("cuda", torch.cuda.current_device()))
    _check(lib.fa_selftest_wait_timeout(_ptr(ws), ws.numel(), int(limit_cycles), _stream()))
    return int(lib.fa_ws_status(_ptr(ws), _stream()))


def fa_launch_count() -> int:
    return int(load().fa_launch_count())


def fa_ws_status(ws: torch.Tensor):
    _check(load().fa_ws_status(_ptr(ws), _stream()))


def make_timer(kernel_id: int, level: int, events_start, events_stop) -> KernelTimer:
    """Timer over caller-created torch.cuda.Event objects (enable_timing=True)."""
    n = len(events_start)
    for e in list(events_start) + list(events_stop):
        e.record()  # torch creates the underlying cudaEvent_t on first record
    st = (ctypes.c_void_p * n)(*[ctypes.c_void_p(e.cuda_event) for e in events_start])
    sp = (ctypes.c_void_p * n)(*[ctypes.c_void_p(e.cuda_event) for e in events_stop])
    t = KernelTimer(kernel_id, level, n, 0, ctypes.cast(st, ctypes.POINTER(ctypes.c_void_p)),
                    ctypes.cast(sp, ctypes.POINTER(ctypes.c_void_p)))
    t._keep = (st, sp)
    return t

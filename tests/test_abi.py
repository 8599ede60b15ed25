"""The C ABI library builds, loads on a machine without a GPU, exports every
entry point include/fa.h declares, and validates arguments on the host
before touching the device."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fa_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import torch  # noqa: F401  (loads the CUDA runtime the library links against)
    from paper_2404_01249_gb300 import build, fa
    build.build()
    return fa.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2404_01249_gb300 import fa
    decl = declared_functions()
    assert len(decl) >= 17
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(fa.EXPORTED) == decl


def test_params_default_and_status_strings(lib):
    from paper_2404_01249_gb300 import fa
    p = fa.Params()
    assert lib.fa_params_default(ctypes.byref(p)) == 0
    assert p.n_levels == 3 and list(p.scales[:3]) == [4, 2, 1] and list(p.iters[:3]) == [200, 100, 50]
    assert p.window == 5 and abs(p.lr - 0.5) < 1e-7 and abs(p.c_lp - 2.0) < 1e-7
    for s in range(9):
        assert lib.fa_status_str(s)
    assert lib.fa_params_default(None) == 1


def test_workspace_queries(lib):
    from paper_2404_01249_gb300 import fa
    n = 160 * 192 * 224
    assert lib.fa_lncc_workspace_size(160, 192, 224) >= 100 * n
    assert lib.fa_gauss_workspace_size(3, 160, 192, 224) >= 24 * n
    assert lib.fa_lncc_workspace_size(0, 1, 1) == 0
    p = fa.RegParams().to_c()
    assert lib.fa_register_workspace_size(160, 192, 224, ctypes.byref(p)) > 0
    p.window = 4
    assert lib.fa_register_workspace_size(160, 192, 224, ctypes.byref(p)) == 0


def _vol(ptr, C, D, H, W, dtype=0):
    from paper_2404_01249_gb300 import fa
    return ctypes.byref(fa.Vol(ptr, dtype, C, D, H, W))


def test_host_validation_rejects_before_launch(lib):
    # fake (never dereferenced) device addresses: validation fails first
    a = 1 << 20
    ok1 = lambda: _vol(a, 1, 4, 5, 6)
    assert lib.fa_warp(None, _vol(a, 3, 4, 5, 6), ok1(), None, None) == 1
    assert lib.fa_warp(ok1(), _vol(a, 1, 4, 5, 6), ok1(), None, None) == 2   # u needs C=3
    assert lib.fa_warp(ok1(), _vol(a, 3, 4, 5, 7), ok1(), None, None) == 2   # grid mismatch
    assert lib.fa_warp(ok1(), _vol(a, 3, 4, 5, 6, dtype=1), ok1(), None, None) == 3
    assert b"share a grid" in lib.fa_last_error() or lib.fa_last_error()
    assert lib.fa_lncc_fwd_bwd(ok1(), ok1(), 4, 1e-5, None, None, None, None, 0, None) == 1
    assert lib.fa_lncc_fwd_bwd(ok1(), ok1(), 5, 1e-5, None, None, None, None, 0, None) == 8
    assert lib.fa_gauss_smooth(_vol(a, 3, 4, 5, 6), _vol(a, 3, 4, 5, 6), 11.0, None, 0, None) == 1
    assert lib.fa_upsample_field(_vol(a, 3, 2, 2, 2), _vol(a + 4096, 3, 4, 4, 4), 2, None) == 1
    from paper_2404_01249_gb300 import fa
    p = fa.RegParams(mode="plain").to_c()
    t_dev = ctypes.c_void_p(a + 8192)
    assert lib.fa_radam_step(_vol(a, 3, 4, 5, 6), _vol(a, 3, 4, 5, 6), _vol(a, 3, 4, 5, 6),
                             _vol(a, 3, 4, 5, 6), _vol(a, 3, 4, 5, 6), t_dev, ctypes.byref(p),
                             None, None, 0, None) == 1   # u_out aliases u_in
    # the device step counter: missing, then misaligned
    for bad_t in (None, ctypes.c_void_p(a + 8194)):
        assert lib.fa_radam_step(_vol(a, 3, 4, 5, 6), _vol(a + 4096, 3, 4, 5, 6),
                                 _vol(a, 3, 4, 5, 6), _vol(a, 3, 4, 5, 6), _vol(a, 3, 4, 5, 6),
                                 bad_t, ctypes.byref(p), None, None, 0, None) == 1
        assert b"t_dev" in lib.fa_last_error()
    # u_out on the wrong grid, then a missing workspace
    assert lib.fa_register(ok1(), ok1(), ctypes.byref(p), _vol(a, 3, 4, 5, 7), None, None, None,
                           0, None) == 2
    assert lib.fa_register(ok1(), ok1(), ctypes.byref(p), _vol(a, 3, 4, 5, 6), None, None, None,
                           0, None) == 8
    assert lib.fa_pyramid_level(_vol(a, 1, 8, 8, 8), 2, _vol(a, 1, 3, 4, 4), None, 0, None) == 2


def test_batched_validation_before_launch(lib):
    from paper_2404_01249_gb300 import fa
    a = 1 << 20
    p = fa.RegParams(scales=(2, 1), iters=(3, 2)).to_c()
    cfgs = (fa.Params * 1)(p)
    fx = (fa.Vol * 2)(fa.Vol(a, 0, 1, 8, 9, 10), fa.Vol(a, 0, 1, 12, 6, 4))
    assert lib.fa_register_batched_workspace_size(0, fx, 1, cfgs, 2) == 0
    assert lib.fa_register_batched_workspace_size(2, fx, 1, cfgs, 0) == 0
    assert lib.fa_register_batched_workspace_size(2, fx, 1, cfgs, 33) == 0
    one = lib.fa_register_workspace_size(8, 9, 10, ctypes.byref(p))
    two = lib.fa_register_workspace_size(12, 6, 4, ctypes.byref(p))
    got = lib.fa_register_batched_workspace_size(2, fx, 1, cfgs, 2)
    assert got >= 2 * max(one, two) and got % 256 == 0
    # a job whose u_out is on the wrong grid is rejected before anything runs
    uo = (fa.Vol * 2)(fa.Vol(a, 0, 3, 8, 9, 10), fa.Vol(a, 0, 3, 12, 6, 5))
    st = lib.fa_register_batched(2, fx, fx, 1, cfgs, uo, None, None, 2, None, 0, None)
    assert st == 2
    assert b"pair 1, parameter set 0" in lib.fa_last_error()
    assert lib.fa_register_batched(0, fx, fx, 1, cfgs, uo, None, None, 2, None, 0, None) == 1


def test_lockstep_validation_before_launch(lib):
    from paper_2404_01249_gb300 import fa
    a = 1 << 20
    p = fa.RegParams(scales=(2, 1), iters=(3, 2)).to_c()
    fx = (fa.Vol * 2)(fa.Vol(a, 0, 1, 8, 9, 10), fa.Vol(a, 0, 1, 12, 6, 4))
    uo = (fa.Vol * 2)(fa.Vol(a, 0, 3, 8, 9, 10), fa.Vol(a, 0, 3, 12, 6, 4))
    cfgs = (fa.Params * 1)(p)
    size = lib.fa_register_lockstep_workspace_size
    run = lib.fa_register_batched_lockstep
    assert size(2, fx, 1, cfgs, 0) == 0 and size(2, fx, 1, cfgs, 65) == 0
    one = lib.fa_register_workspace_size(8, 9, 10, ctypes.byref(p))
    two = lib.fa_register_workspace_size(12, 6, 4, ctypes.byref(p))
    assert size(2, fx, 1, cfgs, 64) >= 2 * max(one, two)
    assert size(2, fx, 1, cfgs, 1) < size(2, fx, 1, cfgs, 2)
    # jobs that cannot advance together are refused before anything runs
    for bad in (fa.RegParams(scales=(2, 1), iters=(3, 2), loss="mse"),
                fa.RegParams(scales=(2, 1), iters=(3, 2), mode="plain"),
                fa.RegParams(scales=(2, 1), iters=(3, 2), use_jac=True),
                fa.RegParams(scales=(2, 1), iters=(4, 2)),
                fa.RegParams(scales=(2, 1), iters=(3, 2), window=3),
                fa.RegParams(scales=(2, 1), iters=(3, 2), sigma_grad=2.5)):
        two_cfgs = (fa.Params * 2)(p, bad.to_c())
        uo4 = (fa.Vol * 4)(*(list(uo)[:1] * 2 + list(uo)[1:] * 2))
        assert run(2, fx, fx, 2, two_cfgs, uo4, None, None, 64, None, 0, None) == 7, bad
    # a wave of one job is always compatible: then the missing workspace is reported
    ok = (fa.Params * 2)(p, fa.RegParams(scales=(2, 1), iters=(3, 2), loss="mse").to_c())
    uo4 = (fa.Vol * 4)(*(list(uo)[:1] * 2 + list(uo)[1:] * 2))
    assert run(2, fx, fx, 2, ok, uo4, None, None, 1, None, 0, None) == 7  # MSE never in lockstep
    same = (fa.Params * 2)(p, fa.RegParams(scales=(2, 1), iters=(3, 2), lr=0.25,
                                           sigma_grad=2.0).to_c())
    assert run(2, fx, fx, 2, same, uo4, None, None, 64, None, 0, None) == 8  # workspace
    assert run(2, fx, fx, 2, same, uo4, None, None, 0, None, 0, None) == 1
    # jobs with FP16 and FP32 u advance together (the missing workspace is reported)
    f16 = (fa.Params * 2)(p, fa.RegParams(scales=(2, 1), iters=(3, 2), field="f16").to_c())
    assert run(2, fx, fx, 2, f16, uo4, None, None, 64, None, 0, None) == 8


def test_moment_storage_validation(lib):
    from paper_2404_01249_gb300 import fa
    d = fa.Params()
    assert lib.fa_params_default(ctypes.byref(d)) == 0 and d.state_storage == 0
    p32 = fa.RegParams().to_c()
    p16 = fa.RegParams(state="bf16").to_c()
    assert 0 < lib.fa_register_workspace_size(40, 48, 56, ctypes.byref(p16)) < \
        lib.fa_register_workspace_size(40, 48, 56, ctypes.byref(p32))
    for st in (2, 5):  # FP16 moments would flush to zero; 5 is no dtype
        bad = fa.RegParams().to_c()
        bad.state_storage = st
        assert lib.fa_register_workspace_size(40, 48, 56, ctypes.byref(bad)) == 0
    # the calls that keep their moments in FP32 refuse 16-bit moments
    assert lib.fa_affine_workspace_size(40, 48, 56, ctypes.byref(p16)) == 0
    assert lib.fa_affine_workspace_size(40, 48, 56, ctypes.byref(p32)) > 0
    assert lib.fa_inverse_workspace_size(40, 48, 56, ctypes.byref(p16)) == 0
    inv = fa.RegParams(scales=(1,), iters=(5,)).to_c()
    assert lib.fa_register_symmetric_workspace_size(40, 48, 56, ctypes.byref(p16),
                                                    ctypes.byref(inv)) == 0
    assert lib.fa_register_symmetric_workspace_size(40, 48, 56, ctypes.byref(p32),
                                                    ctypes.byref(inv)) > 0
    assert lib.fa_register_svf_workspace_size(40, 48, 56, ctypes.byref(p16), 7) == 0
    assert lib.fa_register_svf_workspace_size(40, 48, 56, ctypes.byref(p32), 7) > 0
    # fa_radam_step: m and v must share a supported dtype
    a = 1 << 20
    V = lambda dt: ctypes.byref(fa.Vol(a, dt, 3, 4, 5, 6))
    t_dev = ctypes.c_void_p(a + 8192)
    st = lib.fa_radam_step(V(0), ctypes.byref(fa.Vol(a + 4096, 0, 3, 4, 5, 6)), V(1), V(2), V(0),
                           t_dev, ctypes.byref(p32), None, None, 0, None)
    assert st == 3
    st = lib.fa_radam_step(V(0), ctypes.byref(fa.Vol(a + 4096, 0, 3, 4, 5, 6)), V(7), V(7), V(0),
                           t_dev, ctypes.byref(p32), None, None, 0, None)
    assert st == 3


def test_pyramid_and_workspace_queries(lib):
    """fa_pyramid (every level of Algorithm 1's downsample in one call) and
    fa_workspace_size (the register workspace from the fixed descriptor)
    validate on the host; the graph cache can be cleared without a GPU."""
    from paper_2404_01249_gb300 import fa
    a = 1 << 20
    p = fa.RegParams(scales=(4, 2, 1), iters=(2, 2, 2)).to_c()
    fixed = fa.Vol(a, 0, 1, 40, 48, 56)
    assert lib.fa_workspace_size(ctypes.byref(fixed), ctypes.byref(p)) == \
        lib.fa_register_workspace_size(40, 48, 56, ctypes.byref(p)) > 0
    assert lib.fa_workspace_size(None, ctypes.byref(p)) == 0
    need = lib.fa_pyramid_workspace_size(40, 48, 56, ctypes.byref(p))
    assert need == lib.fa_gauss_workspace_size(1, 40, 48, 56)
    one = fa.RegParams(scales=(1,), iters=(1,)).to_c()
    assert lib.fa_pyramid_workspace_size(40, 48, 56, ctypes.byref(one)) == 256
    bad = fa.RegParams(scales=(4, 2, 1), iters=(2, 2, 2)).to_c()
    bad.scales[1] = 0
    assert lib.fa_pyramid_workspace_size(40, 48, 56, ctypes.byref(bad)) == 0
    levels = (fa.Vol * 3)(fa.Vol(a + (1 << 24), 0, 1, 10, 12, 14),
                          fa.Vol(a + (2 << 24), 0, 1, 20, 24, 28),
                          fa.Vol(a + (3 << 24), 0, 1, 40, 48, 56))
    # a level of the wrong size, a level aliasing the image, a missing workspace
    levels[1].W = 27
    assert lib.fa_pyramid(ctypes.byref(fixed), ctypes.byref(p), levels, None, 0, None) == 2
    assert b"levels[1]" in lib.fa_last_error()
    levels[1].W = 28
    levels[2].data = a
    assert lib.fa_pyramid(ctypes.byref(fixed), ctypes.byref(p), levels, None, 0, None) == 1
    levels[2].data = a + (3 << 24)
    assert lib.fa_pyramid(ctypes.byref(fixed), ctypes.byref(p), levels, None, 0, None) == 8
    assert lib.fa_pyramid(ctypes.byref(fixed), ctypes.byref(bad), levels, None, 0, None) == 1
    assert lib.fa_pyramid(ctypes.byref(fixed), ctypes.byref(p), None, None, 0, None) == 1
    assert lib.fa_graph_cache_clear() == 0


def test_no_fp64_instruction_in_any_kernel(lib):
    """No kernel holds a double-precision instruction: the build passes
    ptxas --warn-on-double-precision-use for every translation unit and
    keeps ptxas's messages in _build/ptxas.log."""
    from paper_2404_01249_gb300 import build
    log = open(os.path.join(build.OUT, "ptxas.log")).read()
    assert "ptxas info" in log                      # the log is ptxas's output
    assert "double precision" not in log.lower()

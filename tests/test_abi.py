"""The C-ABI library loads and exports every entry point declared in include/*.h (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fmx?_[A-Za-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def fm():
    from paper_2508_18468_gb300 import build
    build.build()
    from paper_2508_18468_gb300 import fm as mod
    return mod


def test_every_declared_symbol_is_exported(fm):
    headers = sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
    assert "fm.h" in headers and "fm_testing.h" in headers
    names = {h: _declared(h) for h in headers}
    assert len(names["fm.h"]) >= 19 and len(names["fm_testing.h"]) >= 8
    for h, ns in names.items():
        for n in ns:
            assert hasattr(fm.lib, n), "%s: %s" % (h, n)


def test_struct_layouts(fm):
    assert ctypes.sizeof(fm.fm_params) == 72
    assert ctypes.sizeof(fm.fm_event) == 40
    assert ctypes.sizeof(fm.fm_tuning) == 40
    assert fm.fm_version().startswith("fm ")


def test_workspace_bytes_validates_parameters(fm):
    ok = fm.make_params(64)
    assert fm.fm_workspace_bytes(ok) > 0
    assert fm.fm_workspace_bytes(fm.make_params(64, batch=4)) > fm.fm_workspace_bytes(ok)
    for bad in (fm.make_params(63), fm.make_params(64, batch=0), fm.make_params(64, dt=0.0),
                fm.make_params(64, gamma=-1.0), fm.make_params(64, reorth_interval=0),
                fm.make_params(5, Ly=4), fm.make_params(64, protocol=7), fm.make_params(1)):
        assert fm.fm_workspace_bytes(bad) == 0
    # the event log and the forced-outcome list both scale with event_capacity
    base = fm.fm_workspace_bytes(fm.make_params(64, event_capacity=0))
    assert fm.fm_workspace_bytes(fm.make_params(64, event_capacity=4096)) - base >= 4096 * (40 + 16)


def test_tile_config_is_validated(fm):
    mixed = dict(precision=fm.FM_MIXED, protocol=fm.FM_HOMODYNE)
    assert fm.fm_workspace_bytes(fm.make_params(512, tile_config=0, **mixed)) > 0
    assert fm.fm_workspace_bytes(fm.make_params(512, tile_config=2 | (3 << 2), **mixed)) > 0
    assert fm.fm_workspace_bytes(fm.make_params(256, tile_config=1, **mixed)) > 0
    assert fm.fm_workspace_bytes(fm.make_params(256, tile_config=2, **mixed)) == 0    # N = 128: no 256-wide tiles
    assert fm.fm_workspace_bytes(fm.make_params(512, tile_config=3, **mixed)) == 0
    assert fm.fm_workspace_bytes(fm.make_params(512, tile_config=1 << 5, **mixed)) > 0     # drain every 4 K-blocks
    assert fm.fm_workspace_bytes(fm.make_params(512, tile_config=3 << 5, **mixed)) == 0
    assert fm.fm_workspace_bytes(fm.make_params(512, tile_config=1 << 7, **mixed)) > 0      # a Cholesky chain per trajectory
    assert fm.fm_workspace_bytes(fm.make_params(512, tile_config=1 << 8, **mixed)) == 0
    # the workspace does not depend on the tile configuration
    assert (fm.fm_workspace_bytes(fm.make_params(1024, tile_config=1, **mixed)) ==
            fm.fm_workspace_bytes(fm.make_params(1024, tile_config=2, **mixed)))


def test_autotune_rejects_bad_arguments_without_a_gpu(fm):
    out = fm.fm_tuning()
    p = fm.make_params(64)
    assert fm.lib.fm_autotune(ctypes.byref(p), None, 0, None, 0, 1, 1e-6, 0, ctypes.byref(out)) == fm.FM_EINVAL
    assert fm.lib.fm_autotune(ctypes.byref(p), None, 0, None, 4, 0, 1e-6, 0, ctypes.byref(out)) == fm.FM_EINVAL
    assert fm.lib.fm_autotune(ctypes.byref(p), None, 0, None, 4, 1, 0.0, 0, ctypes.byref(out)) == fm.FM_EINVAL
    assert fm.lib.fm_autotune(ctypes.byref(p), None, 0, None, 4, 1, 1e-6, 0, None) == fm.FM_EINVAL


def test_null_state_calls_fail_cleanly(fm):
    assert fm.lib.fm_step(None, 1) == fm.FM_EINVAL
    assert fm.lib.fm_kernel_launches(None) == 0
    fm.lib.fm_destroy(None)


def test_binding_without_the_library_raises():
    """The binding refuses to import when libfm.so is absent: no fallback implementation."""
    src_path = os.path.join(ROOT, "paper_2508_18468_gb300", "fm.py")
    src = open(src_path).read()
    ns = {"__file__": os.path.join(ROOT, "no_such_directory", "fm.py"), "__name__": "fm_without_library"}
    with pytest.raises(ImportError, match="no non-CUDA fallback"):
        exec(compile(src, src_path, "exec"), ns)


def test_trajectories_fail_loudly_without_a_gpu(fm):
    """On a host without a CUDA device the product path raises instead of computing anything."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(RuntimeError):
        fm.Trajectories(fm.make_params(64))


def test_init_state_validates_arguments_before_touching_the_device(fm):
    """fm_init_state rejects a missing out pointer, invalid parameters, a null or misaligned
    workspace (FM_EINVAL) and a workspace smaller than fm_workspace_bytes (FM_ENOMEM) before any
    device access; calls on a null state return FM_EINVAL."""
    lib = fm.lib
    p = fm.make_params(64)
    need = fm.fm_workspace_bytes(p)
    out = ctypes.c_void_p(12345)
    fake = 1 << 20                                     # aligned, never dereferenced on these paths
    assert lib.fm_init_state(ctypes.byref(p), ctypes.c_void_p(fake), need, None, None) == fm.FM_EINVAL
    bad = fm.make_params(63)
    assert lib.fm_init_state(ctypes.byref(bad), ctypes.c_void_p(fake), need, None, ctypes.byref(out)) == fm.FM_EINVAL
    assert out.value is None                           # *out cleared on failure
    assert lib.fm_init_state(ctypes.byref(p), None, need, None, ctypes.byref(out)) == fm.FM_EINVAL
    assert lib.fm_init_state(ctypes.byref(p), ctypes.c_void_p(fake + 8), need, None,
                             ctypes.byref(out)) == fm.FM_EINVAL
    assert lib.fm_init_state(ctypes.byref(p), ctypes.c_void_p(fake), need - 1, None,
                             ctypes.byref(out)) == fm.FM_ENOMEM
    assert out.value is None
    assert lib.fm_step(None, 1) == fm.FM_EINVAL
    assert lib.fm_last_error(None) == b"null state"
    lib.fm_destroy(None)


def test_test_hooks_reject_invalid_sizes_before_any_launch(fm):
    """The tensor-core and leaf hooks of include/fm_testing.h return cudaErrorInvalidValue (1) for
    sizes their kernels do not take, before touching any pointer."""
    lib = fm.lib
    vp, i32 = ctypes.c_void_p, ctypes.c_int
    lib.fmx_tc_gemm.restype = i32
    lib.fmx_tc_gemm.argtypes = [vp, vp, vp, vp, i32, i32, i32, vp, i32, i32, i32, i32, vp, vp]
    lib.fmx_tc_gram.restype = i32
    lib.fmx_tc_gram.argtypes = [vp, vp, i32, i32, i32, vp, i32, vp, vp]
    lib.fmx_chol_leaf.restype = i32
    lib.fmx_chol_leaf.argtypes = [vp, i32, i32, i32, vp, vp, vp, vp]
    INVALID = 1
    gemm = lambda M, N, K, BN, chunk=0: lib.fmx_tc_gemm(None, None, None, None, M, N, K, None, BN, 0, chunk, 1,
                                                         None, None)
    assert gemm(100, 128, 64, 128) == INVALID          # M not a multiple of 128
    assert gemm(128, 128, 64, 64) == INVALID           # BN neither 128 nor 256
    assert gemm(128, 128, 64, 256) == INVALID          # N not a multiple of BN
    assert gemm(128, 128, 32, 128) == INVALID          # K not a multiple of 64
    assert gemm(128, 256, 64, 256, chunk=2) == INVALID  # register drain only with BN = 128
    assert lib.fmx_tc_gram(None, None, 64, 96, 1, None, 128, None, None) == INVALID
    dummy = ctypes.c_void_p(1 << 20)
    for n, ld, B in ((0, 1, 1), (129, 129, 1), (64, 63, 1), (64, 64, 0)):
        assert lib.fmx_chol_leaf(dummy, n, ld, B, dummy, dummy, dummy, None) == INVALID
    assert lib.fmx_chol_leaf(dummy, 64, 64, 1, dummy, dummy, None, None) == INVALID   # no status word


def test_binding_constants_match_the_header(fm):
    """Every integer constant of include/fm.h (enumerators and object-like #defines) has the same
    value in the binding, and the function-like tile macros agree on a few arguments."""
    src = open(os.path.join(ROOT, "include", "fm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", src, flags=re.S):
        for name, val in re.findall(r"\b(FM_[A-Z0-9_]+)\s*=\s*([0-9]+)", body):
            consts[name] = int(val)
    for name, expr in re.findall(r"#define\s+(FM_[A-Z0-9_]+)\s+(\(?[0-9][0-9 <()]*\)?)\s*$", src, flags=re.M):
        consts[name] = int(eval(expr))                    # plain integers and (1 << k)
    assert {"FM_OK", "FM_MIXED", "FM_TILE_CHOL_CHAINS", "FM_NOALLOC_MAX_N"} <= set(consts)
    for name, val in consts.items():
        if name.startswith("FM_PH_"):
            assert fm.PHASES[val] == name[6:].lower(), name
            continue
        assert getattr(fm, name) == val, name
    for g in range(8):
        assert fm.FM_TILE_GROUP(g) == g << 2
    for d in range(3):
        assert fm.FM_TILE_DRAIN(d) == d << 5


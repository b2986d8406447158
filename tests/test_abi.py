"""Host-side checks of the C ABI (no GPU needed): librv builds for sm_103a,
loads, exports every entry point include/rv.h declares, and rejects bad
arguments before touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rv_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1507_01009_gb300 import build_lib, rv
    build_lib.build()
    return rv.load()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_1507_01009_gb300 import rv
    assert sorted(rv.EXPORTS) == _declared()


def test_config_and_workspace_size(lib):
    from paper_1507_01009_gb300 import rv
    cfg = rv.default_config()
    assert (cfg.n_leaf, cfg.group, cfg.quadrupole, cfg.tile) == (16, 32, 1, 64)
    assert abs(cfg.theta - 0.5) < 1e-7
    s1 = rv.workspace_size(1 << 20, cfg)
    s2 = rv.workspace_size(1 << 21, cfg)
    assert 0 < s1 < s2 < 2 * s1 + (1 << 20)
    bad = rv.default_config(tile=48)
    assert rv.workspace_size(1000, bad) == 0
    bad = rv.default_config(group=65)
    assert rv.workspace_size(1000, bad) == 0
    assert (cfg.mac, abs(cfg.alpha - 1e-3) < 1e-9) == (0, True)
    assert rv.workspace_size(1000, rv.default_config(mac=2)) == 0
    assert rv.workspace_size(1000, rv.default_config(mac=1, alpha=-1.0)) == 0


def test_create_rejects_bad_arguments(lib):
    from paper_1507_01009_gb300 import rv
    h = C.c_void_p()
    cfg = rv.default_config(n_leaf=0)
    assert lib.rv_create(C.byref(h), 100, C.byref(cfg)) == rv.RV_E_INVAL
    cfg = rv.default_config()
    assert lib.rv_create(C.byref(h), -1, C.byref(cfg)) == rv.RV_E_INVAL
    assert lib.rv_build_tree(None, 0, None, None, None, None, None) == rv.RV_E_INVAL
    assert lib.rv_last_error(None) == b"null context"


@pytest.mark.gpu
def test_workspace_too_small_rejected(lib):
    """rv_set_workspace checks size and alignment before touching the device."""
    from paper_1507_01009_gb300 import rv
    cfg = rv.default_config()
    h = C.c_void_p()
    st = lib.rv_create(C.byref(h), 1000, C.byref(cfg))
    if st == rv.RV_E_CUDA:
        pytest.skip("no CUDA device to create a context on")
    assert st == rv.RV_OK
    need = rv.workspace_size(1000, cfg)
    assert lib.rv_set_workspace(h, C.c_void_p(1 << 20), need - 256) == rv.RV_E_WORKSPACE
    assert lib.rv_set_workspace(h, C.c_void_p((1 << 20) + 8), need) == rv.RV_E_WORKSPACE
    assert b"need" in lib.rv_last_error(h)
    lib.rv_destroy(h)


def test_new_entry_points_reject_bad_arguments(lib):
    """Argument checks that run before any device work: the FP64 direct sum,
    the network's feature box and the wait self-test."""
    from paper_1507_01009_gb300 import rv
    assert lib.rv_direct_fp64_scratch_bytes(0) == 0
    assert lib.rv_direct_fp64_scratch_bytes(10) == 8 * 4 * 128 * 10
    nul = [None] * 5
    assert lib.rv_direct_fp64(0, *nul, 1, None, None, None, None, None, None, 0, None) == rv.RV_E_INVAL
    assert lib.rv_direct_fp64(5, *nul, 1, None, None, None, None, None, None, 0, None) == rv.RV_E_INVAL
    assert lib.rv_mlp_fit_feature_box(None, 10, None, None) == rv.RV_E_INVAL
    lo = (C.c_float * 16)(*([1.0] * 16))
    hi = (C.c_float * 16)(*([0.0] * 16))
    assert lib.rv_mlp_set_feature_box(None, lo, hi, None) == rv.RV_E_INVAL
    assert lib.rv_wait_selftest(-1, 0, None, None) == rv.RV_E_INVAL
    assert lib.rv_wait_selftest(10, 2, None, None) == rv.RV_E_INVAL


def test_training_and_state_entry_points_reject_bad_arguments(lib):
    """rv_mlp_train, rv_mlp_save and rv_mlp_load check their arguments (and a
    saved state's header) before any device work."""
    from paper_1507_01009_gb300 import rv
    assert lib.rv_mlp_train_scratch_bytes(0) == 0
    assert lib.rv_mlp_train_scratch_bytes(64) > lib.rv_mlp_scratch_bytes(64)
    n = int(lib.rv_mlp_state_bytes())
    assert n == 64 + int(lib.rv_mlp_param_bytes())
    fake = C.c_void_p(1 << 20)        # never dereferenced: every call below fails its checks first
    cfg = rv.rv_mlp_train_cfg(n=100, x=C.c_void_p(1 << 20), t=C.c_void_p(1 << 21), steps=10, batch=32, step0=1,
                              lr=1e-3, beta1=0.9, beta2=0.999, adam_eps=1e-8, seed=1, fit_box=1)
    need = lib.rv_mlp_train_scratch_bytes(32)
    assert lib.rv_mlp_train(None, C.byref(cfg), None, fake, need, None) == rv.RV_E_INVAL
    assert lib.rv_mlp_train(fake, None, None, fake, need, None) == rv.RV_E_INVAL
    assert lib.rv_mlp_train(fake, C.byref(cfg), None, fake, need - 1, None) == rv.RV_E_WORKSPACE
    for field, bad in (("step0", 0), ("batch", 0), ("n", 0), ("beta1", 1.0), ("adam_eps", 0.0), ("fit_box", 2),
                       ("x", C.c_void_p((1 << 20) + 4))):
        b = rv.rv_mlp_train_cfg.from_buffer_copy(cfg)
        setattr(b, field, bad)
        assert lib.rv_mlp_train(fake, C.byref(b), None, fake, need, None) == rv.RV_E_INVAL, field
    buf = (C.c_char * n)()
    assert lib.rv_mlp_save(fake, buf, n - 1, None) == rv.RV_E_INVAL
    assert lib.rv_mlp_load(fake, buf, n, None) == rv.RV_E_INVAL            # zero header: not a saved state
    assert lib.rv_mlp_load(None, buf, n, None) == rv.RV_E_INVAL

"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/nmf.h declares.  No compute call is made (no GPU here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "nmf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nmf_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2101_08431_gb300 import build, _native
    build.build()
    return _native.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2101_08431_gb300 import _native
    names = _declared()
    assert names, "no declarations parsed"
    assert set(names) == set(_native.EXPORTS)
    for name in names:
        assert hasattr(lib, name), name


def test_host_only_entry_points(lib):
    from paper_2101_08431_gb300 import _native
    cfg = _native.nmf_config()
    lib.nmf_config_init(C.byref(cfg))
    assert cfg.kkt_target == 1e-8 and cfg.prec == _native.NMF_PREC_MIXED and cfg.warm_start == 1
    for s in range(9):
        assert lib.nmf_status_string(s).decode()
    assert lib.nmf_last_error(None) == b""
    assert lib.nmf_launch_count(None) == 0


def test_invalid_arguments_rejected_before_any_device_work(lib):
    from paper_2101_08431_gb300 import _native
    cfg = _native.nmf_config()
    lib.nmf_config_init(C.byref(cfg))
    h = C.c_void_p()
    for n, k, mcap in ((0, 4, 10), (100, 0, 10), (100, 9, 10), (100, 17, 10), (100, 4, 0)):
        cfg.n, cfg.k, cfg.m_capacity = n, k, mcap
        assert lib.nmf_create(C.byref(cfg), C.byref(h)) == _native.NMF_EINVAL
    assert lib.nmf_destroy(None) == _native.NMF_OK


def test_batch_arguments_rejected_before_any_device_work(lib):
    from paper_2101_08431_gb300 import _native
    cfgs = (_native.nmf_config * 2)()
    for j in range(2):
        lib.nmf_config_init(C.byref(cfgs[j]))
        cfgs[j].n, cfgs[j].k, cfgs[j].m_capacity = 100, 4, 10
    b = C.c_void_p()
    assert lib.nmf_batch_create(None, 2, None, C.byref(b)) == _native.NMF_EINVAL
    assert lib.nmf_batch_create(cfgs, 0, None, C.byref(b)) == _native.NMF_EINVAL
    cfgs[1].prec = _native.NMF_PREC_FP64          # the batched form is mixed precision
    assert lib.nmf_batch_create(cfgs, 2, None, C.byref(b)) == _native.NMF_EINVAL
    cfgs[1].prec, cfgs[1].k = _native.NMF_PREC_MIXED, 9
    assert lib.nmf_batch_create(cfgs, 2, None, C.byref(b)) == _native.NMF_EINVAL
    assert lib.nmf_batch_size(None) == 0
    assert lib.nmf_batch_problem(None, 0) is None
    assert lib.nmf_batch_set_pass_mode(None, 0) == _native.NMF_EINVAL
    assert lib.nmf_batch_set_schedule(None, 64, 8) == _native.NMF_EINVAL
    assert lib.nmf_batch_sweep(None, 1, None, None) == _native.NMF_EINVAL
    assert lib.nmf_batch_destroy(None) == _native.NMF_OK


def test_server_arguments_rejected_before_any_device_work(lib):
    from paper_2101_08431_gb300 import _native
    cfg = _native.nmf_server_config()
    lib.nmf_server_config_init(C.byref(cfg))
    assert cfg.max_streams == 64 and cfg.sweeps_per_round == 8 and cfg.kkt_target == 1e-6
    s = C.c_void_p()
    assert lib.nmf_server_create(None, C.byref(s)) == _native.NMF_EINVAL
    cfg.sweeps_per_round = 0
    assert lib.nmf_server_create(C.byref(cfg), C.byref(s)) == _native.NMF_EINVAL
    i = C.c_int32()
    assert lib.nmf_server_open_stream(None, 100, 3, 10, 0, C.byref(i)) == _native.NMF_EINVAL
    assert lib.nmf_server_submit(None, 0, None, 1, 100, None) == _native.NMF_EINVAL
    assert lib.nmf_server_destroy(None) == _native.NMF_OK


def test_library_is_built_for_sm_103a_only():
    from paper_2101_08431_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_selftest_rejects_bad_limit(lib):
    from paper_2101_08431_gb300 import _native
    assert lib.nmf_selftest_bounded_wait(0, None) == _native.NMF_EINVAL
    assert lib.nmf_selftest_bounded_wait(1 << 30, None) == _native.NMF_EINVAL
    assert lib.nmf_selftest_tc16_wait(0, None) == _native.NMF_EINVAL
    assert lib.nmf_selftest_tc16_wait(20000, None) == _native.NMF_EINVAL


def test_noalloc_rejects_misaligned_pointers_before_any_device_work(lib):
    """nmf_sweep_noalloc checks the alignment of the caller's pointers before
    it touches the device (M is staged with bulk copies from 16-byte aligned
    addresses; X, Y and the record are doubles), so these fake addresses are
    never dereferenced."""
    from paper_2101_08431_gb300 import _native
    P = C.c_void_p
    good, m4, x4 = 0x10000, 0x10004, 0x10004
    assert lib.nmf_sweep_noalloc(P(m4), 100, 10, 128, 4, P(good), P(good), None, None) == _native.NMF_EINVAL
    assert lib.nmf_sweep_noalloc(P(0x10008), 100, 10, 128, 4, P(good), P(good), None, None) == _native.NMF_EINVAL
    assert lib.nmf_sweep_noalloc(P(good), 100, 10, 128, 4, P(x4), P(good), None, None) == _native.NMF_EINVAL
    assert lib.nmf_sweep_noalloc(P(good), 100, 10, 128, 4, P(good), P(x4), None, None) == _native.NMF_EINVAL
    assert lib.nmf_sweep_noalloc(P(good), 100, 10, 128, 4, P(good), P(good), P(x4), None) == _native.NMF_EINVAL


def test_persistence_arguments_rejected_before_any_device_work(lib, tmp_path):
    """nmf_save / nmf_load / nmf_get_config reject NULL arguments, a path
    that cannot be opened and a file that is not one of theirs, all before
    any device allocation (nmf_load reads and checks the whole file first)."""
    from paper_2101_08431_gb300 import _native
    h = C.c_void_p()
    cfg = _native.nmf_config()
    assert lib.nmf_save(None, b"/tmp/x") == _native.NMF_EINVAL
    assert lib.nmf_load(None, None, C.byref(h)) == _native.NMF_EINVAL
    assert lib.nmf_load(b"/tmp/x", None, None) == _native.NMF_EINVAL
    assert lib.nmf_get_config(None, C.byref(cfg)) == _native.NMF_EINVAL
    assert lib.nmf_load(str(tmp_path / "missing.nmf").encode(), None, C.byref(h)) == _native.NMF_EINVAL
    for content in (b"", b"NMFGB30", b"NOTMAGIC" + bytes(200), b"NMFGB300" + bytes(200)):
        p = tmp_path / "f.nmf"
        p.write_bytes(content)
        assert lib.nmf_load(str(p).encode(), None, C.byref(h)) == _native.NMF_EINVAL
        assert not h.value


def test_stage2_arguments_rejected_before_any_device_work(lib):
    from paper_2101_08431_gb300 import _native
    z = C.c_void_p(0x1000)
    assert lib.nmf_ipm(None, 1e-6, 10, None) == _native.NMF_EINVAL
    assert lib.nmf_ipm_direction(None, z, z, 0.1, 1e-6, 0, z, z, z, z, 0) == _native.NMF_EINVAL

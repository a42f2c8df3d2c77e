"""The C-ABI library loads and exports every entry point include/wbrw.h
declares; host-only argument checks work without a GPU."""
import ctypes
import os
import re

import pytest

import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "wbrw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wbrw_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1709_02121_gb300 import build, wbrw
    build.build()
    return wbrw.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("wbrw_init", "wbrw_step", "wbrw_annihilate", "wbrw_density"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1709_02121_gb300 import wbrw
    names = _declared()
    assert sorted(wbrw.SYMBOLS) == names
    for n in names:
        assert hasattr(lib, n), n


def _cfg(**over):
    from paper_1709_02121_gb300 import wbrw
    wl = dict(workloads.GAUSS_2D_FP64_2E5)
    wl.update(over)
    return wbrw.Config(2, wbrw.FP64 if wl["precision"] == "fp64" else wbrw.FP32,
                       1 if wl["strategy"] == "sp1" else 2, wl["hbar"], wl["mass"], wl["dt"],
                       wl["gamma0"], wl["nx"], wl["nk"], wl["xmin"], wl["xmax"], wl["kmin"],
                       wl["kmax"], wl["resample_every"], wl["n_alpha"], wl["seed"])


def test_scratch_bytes_and_argument_checks(lib):
    from paper_1709_02121_gb300 import wbrw
    n64 = wbrw.wbrw_scratch_bytes(_cfg(), 100000)
    n32 = wbrw.wbrw_scratch_bytes(_cfg(precision="fp32"), 100000)
    assert n64 > 0 and n32 > 0 and n64 > n32
    sp2 = wbrw.wbrw_scratch_bytes(_cfg(strategy="sp2"), 100000)
    assert sp2 > n64                              # records and bootstrap grids
    assert wbrw.wbrw_scratch_bytes(_cfg(), 0) == 0
    assert wbrw.wbrw_scratch_bytes(_cfg(nx=0), 10) == 0
    assert wbrw.wbrw_scratch_bytes(_cfg(dt=-1.0), 10) == 0
    assert wbrw.wbrw_scratch_bytes(_cfg(xmax=-60.0), 10) == 0
    bad = _cfg()
    bad.dim = 3
    assert wbrw.wbrw_scratch_bytes(bad, 10) == 0
    bad = _cfg(nx=300)
    bad.dim = 4                                   # 300^2 128^2 cells >= 2^30
    assert wbrw.wbrw_scratch_bytes(bad, 10) == 0


def test_init_rejects_bad_arguments_without_touching_a_gpu(lib):
    from paper_1709_02121_gb300 import wbrw
    cfg = _cfg()
    pot = wbrw.Potential(0, 1.0, 1.0, 0.0)
    bufs = wbrw.Buffers()                         # all NULL
    ctx = ctypes.c_void_p()
    st = lib.wbrw_init(ctypes.byref(cfg), ctypes.byref(pot), ctypes.byref(bufs), 10,
                       -15.0, 2.5, 1.5, None, ctypes.byref(ctx))
    assert st == wbrw.ERR_ARG and not ctx.value
    st = lib.wbrw_init(ctypes.byref(cfg), None, ctypes.byref(bufs), 10, -15.0, 2.5, 1.5,
                       None, ctypes.byref(ctx))
    assert st == wbrw.ERR_ARG
    assert lib.wbrw_step(None, 1) == wbrw.ERR_ARG
    assert lib.wbrw_profile(None, 1) == wbrw.ERR_ARG
    assert lib.wbrw_profile_read(None, None, None) == wbrw.ERR_ARG
    assert lib.wbrw_profile_read_events(None, None, None) == wbrw.ERR_ARG
    assert lib.wbrw_counters(None, None) == wbrw.ERR_ARG
    assert lib.wbrw_one_launch_periods(None, 1) == wbrw.ERR_ARG
    assert lib.wbrw_last_error(None) == b"NULL context"
    lib.wbrw_destroy(None)
    # a capacity beyond the 32-bit slot limit is refused before any buffer
    # (here placeholders that are never dereferenced) is touched
    fake = wbrw.Buffers(256, 256, 256, None, wbrw.MAX_CAPACITY + 1, 256, 1 << 20, 256, 1 << 40,
                        None, 0, None)
    st = lib.wbrw_init(ctypes.byref(cfg), ctypes.byref(pot), ctypes.byref(fake), 10,
                       -15.0, 2.5, 1.5, None, ctypes.byref(ctx))
    assert st == wbrw.ERR_ARG and not ctx.value
    hdr = open(os.path.join(ROOT, "include", "wbrw.h")).read()
    assert "#define WBRW_MAX_CAPACITY %dLL" % wbrw.MAX_CAPACITY in hdr


def test_product_path_has_no_fallback(tmp_path):
    from paper_1709_02121_gb300 import wbrw
    with pytest.raises(RuntimeError):
        wbrw._lib, saved = None, wbrw._lib
        try:
            wbrw.load(str(tmp_path / "missing.so"))
        finally:
            wbrw._lib = saved


def test_dim4_scratch_holds_the_kernel_tables(lib):
    from paper_1709_02121_gb300 import wbrw
    c = _cfg(precision="fp32", nx=16, nk=16)
    c.dim = 4
    n = wbrw.wbrw_scratch_bytes(c, 100000)
    c.table_ny, c.table_nkappa = 1024, 512
    m = wbrw.wbrw_scratch_bytes(c, 100000)
    # default tables 4096 x 2048 of float, two types
    assert n - m >= 2 * 4 * (4096 * 2048 - 1024 * 512)
    c.strategy = 2
    assert wbrw.wbrw_scratch_bytes(c, 100000) == 0     # dim 4 is sp1 only
    c.strategy, c.table_ny = 1, 1
    assert wbrw.wbrw_scratch_bytes(c, 100000) == 0     # a table needs two rows

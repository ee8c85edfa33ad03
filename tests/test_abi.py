"""C ABI: the library builds, loads and exports every symbol include/ctrex.h
declares; host-side argument checks answer without a GPU."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ctrex.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ctrex_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2609_30166_gb300 import _build, ctrex

    _build.build_library()
    return ctrex.load_library()


def test_header_declares_the_binding_exports():
    from paper_2609_30166_gb300 import ctrex

    assert declared_symbols() == sorted(ctrex.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(os.path.join(ROOT, "paper_2609_30166_gb300", "libctrex.so"))
    for name in declared_symbols():
        assert hasattr(raw, name), name


def test_null_context_is_rejected_without_gpu(lib):
    assert lib.ctrex_destroy(None) == -1
    assert lib.ctrex_device_status(None) == -1
    assert lib.ctrex_set_geometry(None, None, 1, 1, None, None, 0.5) == -1
    assert lib.ctrex_fwd_project(None, None, 0, None, 0, None, None, 0) == -1
    assert lib.ctrex_sirt_iterate(None, None, 0, None, 0, 1, 1.0, None, 0.0, None, None) == -1
    assert b"invalid context" in lib.ctrex_last_error(None)
    assert lib.ctrex_version().startswith(b"ctrex-gb300")
    assert lib.ctrex_create(None, 0, None) == -1


def test_create_without_device_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.ctrex_create(ctypes.byref(h), 0, None) == -5
    assert not h.value


def test_binding_refuses_to_run_without_library(tmp_path):
    from paper_2609_30166_gb300 import ctrex

    saved = ctrex._lib
    ctrex._lib = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            ctrex.load_library(str(tmp_path / "missing.so"))
    finally:
        ctrex._lib = saved


def test_conv_argument_checks_answer_without_gpu(lib):
    """The conv entry points refuse null and unaligned pointers (their
    kernels copy 16-byte channel vectors) and bad shapes before any CUDA
    call; the pointers below are never dereferenced."""
    vp = ctypes.c_void_p
    st = vp(0x1000)
    a, b, c = vp(0x10000), vp(0x20000), vp(0x30000)
    odd = vp(0x10002)  # 2-byte aligned: a bf16 element, not a 16-byte vector
    E_ARG, E_SHAPE = -1, -2
    fwd = lib.ctrex_conv3d_fwd
    assert fwd(None, b, None, c, 0, 1, 4, 4, 4, 16, 16, 0, st, None) == E_ARG
    assert fwd(odd, b, None, c, 0, 1, 4, 4, 4, 16, 16, 0, st, None) == E_ARG
    assert fwd(a, vp(0x20008), None, c, 0, 1, 4, 4, 4, 16, 16, 0, st, None) == E_ARG
    assert fwd(a, b, None, vp(0x30004), 0, 1, 4, 4, 4, 16, 16, 0, st, None) == E_ARG
    assert fwd(a, b, None, c, 0, 0, 4, 4, 4, 16, 16, 0, st, None) == E_SHAPE
    wg = lib.ctrex_conv3d_wgrad
    assert wg(odd, b, c, 1, 4, 4, 4, 16, 16, st, None) == E_ARG
    assert wg(a, vp(0x20002), c, 1, 4, 4, 4, 16, 16, st, None) == E_ARG
    assert wg(a, b, c, 1, 4, 4, 4, 12, 16, st, None) == E_SHAPE


def test_correct_static_binding_refuses_bad_buffers_without_gpu(lib):
    """The binding checks every caller buffer before the call: an output of
    the wrong dtype, size, device or layout would otherwise be written past
    its end by the kernel.  A CPU input is refused too (no CPU fallback)."""
    import torch

    from paper_2609_30166_gb300 import ctrex

    p = torch.zeros(16)
    q, rs = torch.zeros(16), torch.ones(16)
    bad_r = [torch.zeros(16, dtype=torch.float64), torch.zeros(8), torch.zeros(32)[::2],
             torch.zeros(16, dtype=torch.bfloat16)]
    for r in bad_r:
        with pytest.raises(ValueError, match="r must be"):
            ctrex.correct_static(p, q, rs, r=r)
    bad_sums = [torch.zeros(2, dtype=torch.float32), torch.zeros(1, dtype=torch.float64),
                torch.zeros(4, dtype=torch.float64)[::2]]
    for sums in bad_sums:
        with pytest.raises(ValueError, match="sums must be"):
            ctrex.correct_static(p, q, rs, sums=sums)
    with pytest.raises(ValueError, match="rowsum"):
        ctrex.correct_static(p, q, rs.double())
    with pytest.raises(ValueError, match="no CPU fallback"):
        ctrex.correct_static(p, q, rs, r=torch.zeros(16), sums=torch.zeros(2, dtype=torch.float64))

"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every entry point that include/hj.h declares, and rejects bad arguments
before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hj():
    from paper_2012_04011_gb300 import _build
    _build.build()
    from paper_2012_04011_gb300 import hj as mod
    return mod


def declared_symbols():
    with open(os.path.join(ROOT, "include", "hj.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hj_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("hj_create_grid", "hj_set_dynamics", "hj_set_initial_value", "hj_solve_brt", "hj_read_value",
                 "hj_destroy_grid", "hj_status_string"):
        assert name in syms


def test_library_exports_every_declared_symbol(hj):
    lib = ctypes.CDLL(hj._build.LIB_PATH)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    assert set(hj.SYMBOLS) == set(declared_symbols())


def test_library_exports_nothing_else(hj):
    out = os.popen(f"nm -D --defined-only {hj._build.LIB_PATH}").read()
    exported = sorted({l.split()[-1] for l in out.splitlines() if " T " in l})
    assert [s for s in exported if s.startswith("hj_")] == declared_symbols()


def test_status_strings_and_version(hj):
    assert hj.status_name(hj.HJ_OK) == "HJ_OK"
    assert hj.status_name(hj.HJ_ERR_TIMEOUT) == "HJ_ERR_TIMEOUT"
    assert hj.status_name(99) == "HJ_ERR_UNKNOWN"
    assert hj.hj_version() == 10000


@pytest.mark.parametrize("n,lo,hi,msg", [
    ((2, 5, 5, 5), (0, 0, 0, 0), (1, 1, 1, 1), "N1 = 2"),
    ((5, 5, 5, 5), (0, 0, 0, 0), (1, 1, 0, 1), "axis 3"),
    ((5, 5, 5, 5), (0, 0, 0, float("nan")), (1, 1, 1, 1), "axis 4"),
    ((5, 5, 5, 5000), (0, 0, 0, 0), (1, 1, 1, 1), "N4 = 5000"),
])
def test_create_grid_validates_before_the_device(hj, n, lo, hi, msg):
    with pytest.raises(hj.HjError) as e:
        hj.hj_create_grid(n, lo, hi)
    assert e.value.status == hj.HJ_ERR_INVALID_ARG
    assert msg in str(e.value)


def test_null_grid_is_rejected(hj):
    for fn, args in ((hj.lib.hj_solve_brt, (None, 1.0, 0.8, None)),
                     (hj.lib.hj_set_kernel, (None, 0)),
                     (hj.lib.hj_read_value, (None, None, 0))):
        assert fn(*args) == hj.HJ_ERR_INVALID_ARG
    hj.lib.hj_destroy_grid(None)  # no-op


def test_unknown_precision_and_mask(hj):
    with pytest.raises(hj.HjError) as e:
        hj.hj_create_grid((5, 5, 5, 8), (0, 0, 0, 0), (1, 1, 1, 1), prec=7)
    assert e.value.status == hj.HJ_ERR_INVALID_ARG
    with pytest.raises(hj.HjError) as e:
        hj.hj_create_grid((5, 5, 5, 8), (0, 0, 0, 0), (1, 1, 1, 1), periodic_mask=0x10)
    assert e.value.status == hj.HJ_ERR_INVALID_ARG


def test_build_entry_compiles_everything():
    import __graft_entry__
    __graft_entry__.build()


def test_batch_host_checks(hj):
    assert hj.hj_batch_slot_bytes((40, 40, 16, 24)) >= 3 * 40 * 40 * 16 * 24 * 4
    assert hj.hj_batch_slot_bytes((40, 40, 16, 25)) > hj.hj_batch_slot_bytes((40, 40, 16, 24))  # padded rows
    with pytest.raises(hj.HjError) as e:
        hj.hj_batch_create(0)
    assert e.value.status == hj.HJ_ERR_INVALID_ARG
    for fn, args in ((hj.lib.hj_batch_advance, (None, 1, None)), (hj.lib.hj_batch_remove, (None, 0))):
        assert fn(*args) == hj.HJ_ERR_INVALID_ARG
    hj.lib.hj_batch_destroy(None)


def test_fp64_probe_rejects_bad_arguments(hj):
    """Checked before any CUDA call."""
    for iters, bps in ((0, 8), (1 << 41, 8), (100, 0), (100, 65)):
        assert hj.lib.hj_fp64_fma_probe(iters, bps, None, None) == hj.HJ_ERR_INVALID_ARG

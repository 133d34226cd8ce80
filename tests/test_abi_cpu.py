"""CPU checks of the C ABI: the library loads, exports every symbol include/tdmrg.h declares, and
its host-only calls agree with the oracle (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = "".join(open(os.path.join(ROOT, "include", f)).read() for f in sorted(os.listdir(os.path.join(ROOT, "include")))
                  if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tdmrg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1103_5391_gb300 import tdmrg as T
    if not os.path.exists(T.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return T


def test_exports_every_declared_symbol(lib):
    names = _header_functions()
    assert len(names) >= 18
    raw = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n
    assert sorted(lib.EXPORTED) == names


def test_weights_match_oracle(lib):
    from oracle import density
    for nv in (2, 3, 4, 7):
        assert lib.tdmrg_tst_weights(nv) == pytest.approx(density.tst_weights(nv), abs=1e-16)
    with pytest.raises(lib.TdmrgError):
        lib.tdmrg_tst_weights(1)


def test_default_opts(lib):
    o = lib.tdmrg_default_opts()
    assert o.prec == lib.TDMRG_FP64 and o.nk_max == 16 and o.breakdown_tol == 1e-12


def test_create_without_gpu_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.TdmrgError) as e:
        lib.tdmrg_create()
    assert e.value.code == lib.TDMRG_ECUDA

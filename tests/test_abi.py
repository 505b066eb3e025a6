"""CPU-only checks of the C ABI: libpcba.so loads, exports every function
include/pcba.h declares, and validates its arguments on the host (creating a
handle touches no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2003_01758_b300 import build, pcba
from paper_2003_01758_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return pcba.lib()


def declared_functions():
    inc = os.path.join(ROOT, "include")
    text = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc))
                   if f.endswith(".h"))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pcba_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(pcba.exported_symbols()) == set(names)


def test_status_strings_and_version(lib):
    assert lib.pcba_version() == 1
    assert lib.pcba_status_string(0) == b"OPTIMAL"
    assert lib.pcba_status_string(1) == b"INFEASIBLE"
    assert lib.pcba_status_string(-3) == b"ERR_OOM"


def test_create_validates_on_host(lib):
    p = W.tiny(1000)
    s = pcba.Solver(p.cost, p.ineq, p.eq, p.lo, p.hi, precision=pcba.FP32)
    assert s.item_bytes() % 256 == 0
    with pytest.raises(pcba.PcbaError, match="precision"):
        pcba.Solver(p.cost, p.ineq, p.eq, p.lo, p.hi, precision=16)
    with pytest.raises(pcba.PcbaError, match="lo < hi"):
        pcba.Solver(p.cost, p.ineq, p.eq, p.hi, p.lo)
    with pytest.raises(pcba.PcbaError, match="degree"):
        pcba.Solver(np.ones((18, 2)), None, None, -1, 1)
    with pytest.raises(pcba.PcbaError, match="nvars"):
        pcba.Solver(np.ones((2,) * 9), None, None, -1, 1)
    bad = p.cost.copy()
    bad[0, 0] = np.nan
    with pytest.raises(pcba.PcbaError, match="non-finite"):
        pcba.Solver(bad, p.ineq, p.eq, p.lo, p.hi)


def test_item_bytes_follow_memory_formula(lib):
    """Eq. (memory_per_item) counts 2l + Pi(P+1) + alpha Pi(G+1) + beta Pi(H+1)
    entries of 4 B; the FP32 layout stores the same coefficients in 4 B plus
    an error bound and an offset per constraint patch, the dyadic box and
    padding to 128 B rows."""
    p = W.rtd(2000)
    s = pcba.Solver(p.cost, p.ineq, p.eq, p.lo, p.hi, precision=pcba.FP32)
    entries = 2 * 2 + 49 + 512 * 49
    assert 4 * entries <= s.item_bytes() <= 4 * entries + 8 * 513 + 1024
    s64 = pcba.Solver(p.cost, p.ineq, p.eq, p.lo, p.hi, precision=pcba.FP64)
    assert 8 * (49 + 512 * 49) <= s64.item_bytes() <= 8 * (49 + 512 * 49) + 1024


def test_network_create_validates_on_host(lib):
    with pytest.raises(pcba.PcbaError, match="precision"):
        pcba.Mlp(2, 34, 128, precision=8)
    with pytest.raises(pcba.PcbaError, match="shape"):
        pcba.Mlp(0, 34, 128)
    with pytest.raises(pcba.PcbaError, match="shape"):
        pcba.Mlp(2, 34, 0)


def test_time_limit_is_validated_on_host(lib):
    p = W.tiny(1000)
    s = pcba.Solver(p.cost, p.ineq, p.eq, p.lo, p.hi, precision=pcba.FP32)
    s.set_time_limit(0.4)
    s.set_time_limit(0.0)
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(pcba.PcbaError, match="time limit"):
            s.set_time_limit(bad)
    assert lib.pcba_status_string(pcba.TIMEOUT) == b"TIMEOUT"


def test_failed_device_allocation_reports_oom(lib, monkeypatch):
    """The allocation-failure hook makes every device allocation of a batch
    fail before any other CUDA call, so the out-of-memory path returns
    PCBA_ERR_OOM with the handle intact, on any machine."""
    p = W.tiny(1000)
    s = pcba.Solver(p.cost, p.ineq, p.eq, p.lo, p.hi, precision=pcba.FP64)
    monkeypatch.setenv("PCBA_TEST_FAIL_ALLOC", "1")
    with pytest.raises(pcba.PcbaError, match="ERR_OOM"):
        s.solve(opt_tol=1e-3, mem_cap=1 << 24)
    with pytest.raises(pcba.PcbaError, match="ERR_OOM"):
        pcba.Batch([s], 1 << 24)
    assert s.item_bytes() > 0


def test_host_alloc_argument_checks(lib):
    """pcba_host_alloc rejects a zero size (NULL, with the reason), and
    pcba_host_free accepts NULL; both without touching a device."""
    assert not lib.pcba_host_alloc(0)
    assert b"bytes" in lib.pcba_last_error()
    assert lib.pcba_host_free(None) == 0


def test_packed_row_upload_argument_checks(lib):
    """pcba_batch_upload_rows_packed rejects null arguments before any device
    work; the packed size of a null batch is 0."""
    assert lib.pcba_batch_upload_rows_packed(None, None) != 0
    assert lib.pcba_batch_rows_packed_doubles(None) == 0

"""The allocation-free monomial-to-Bernstein entry point.

Some callers cannot allocate device memory once they are running (a real-time
planning loop, or a host framework that owns every buffer), so
pcba_bernstein_convert_noalloc takes the caller's input and output buffers
and keeps its own scratch in a fixed device array.  Its results must match the
regular conversion (pcba_root_patches) within the tolerance of the other
conversion tests, call after call on the shared scratch.  This file is named
to be collected last."""
import numpy as np
import pytest

import oracle
from paper_2003_01758_b300 import pcba
from paper_2003_01758_b300 import workloads as W

pytestmark = pytest.mark.gpu


def noalloc_convert(tensors, lo, hi):
    import torch
    mono = torch.from_numpy(np.ascontiguousarray(tensors, dtype=np.float64)).cuda()
    out = torch.full_like(mono, float("nan"))
    degree = np.array(tensors.shape[1:]) - 1
    stream = torch.cuda.current_stream()
    pcba.bernstein_convert_noalloc(mono.data_ptr(), tensors.shape[0], degree, lo, hi,
                                   out.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def reference_ineq_patches(p):
    s = pcba.Solver(p.cost, p.ineq, p.eq, p.lo, p.hi, precision=pcba.FP64)
    _, ineq, _ = s.root_patches()
    s.close()
    return ineq


def assert_close_per_patch(got, ref):
    for g, r in zip(got, ref):
        assert np.abs(g - r).max() <= 1e-12 * np.abs(r).max()


def test_noalloc_conversion_matches_root_patches_on_consecutive_calls():
    first = W.tiny(1000)                   # 10 patches of degree (4,4) on [-1,1]^2
    second = W.dim4(3000, n_eq=0)          # 64 patches of degree (3,3,3,3) on [-1,1]^4
    lo2, hi2 = second.lo - 0.5, second.hi + 0.25  # a box other than the unit one
    second = W.Problem(second.cost, second.ineq, second.eq, lo2, hi2)
    got1 = noalloc_convert(first.ineq, first.lo, first.hi)
    got2 = noalloc_convert(second.ineq, second.lo, second.hi)
    assert_close_per_patch(got1, reference_ineq_patches(first))
    assert_close_per_patch(got2, reference_ineq_patches(second))
    # and against the oracle's direct-summation conversion of each patch
    for got, p in ((got1, first), (got2, second)):
        assert_close_per_patch(got, [oracle.bernstein_from_monomial(g, p.lo, p.hi) for g in p.ineq])
    # the scratch now holds the second call's matrices; a repeat of the first
    # call must not see them
    again = noalloc_convert(first.ineq, first.lo, first.hi)
    np.testing.assert_array_equal(again, got1)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    buf = torch.zeros(18 * 18, dtype=torch.float64, device="cuda")
    with pytest.raises(pcba.PcbaError, match="degree"):
        pcba.bernstein_convert_noalloc(buf.data_ptr(), 1, [17, 17], [-1, -1], [1, 1],
                                       buf.data_ptr())
    with pytest.raises(pcba.PcbaError, match="nvars"):
        pcba.bernstein_convert_noalloc(buf.data_ptr(), 1, [1] * 9, [-1] * 9, [1] * 9,
                                       buf.data_ptr())

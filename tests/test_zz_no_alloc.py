"""qfm_count_noalloc: the counting entry point for callers that cannot
allocate device memory (it keeps the work-queue counter in a static device
array instead of allocating it).  Its results must equal qfm_count's, call
after call: the static counter keeps the previous call's value and must be
reset by every call.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2602_04103_gb300 import synth
from tests.gpu_util import dev_u64, dev_u8, host_u64

pytestmark = pytest.mark.gpu


def test_noalloc_matches_qfm_count_two_calls_in_a_row():
    import torch
    from paper_2602_04103_gb300 import capi
    torch.cuda.set_device(0)
    n = 1 << 18
    t = synth.fm_text(91, n, repeat_cover=0.2, len_min=300, len_max=2000, sub_rate=0.02)
    idx = capi.qfm_build(dev_u8(t), n)
    batches = [synth.patterns(92, t, 50_000, 1, 150, 0.01), synth.patterns(93, t, 70_001, 8, 60, 0.01)]
    for pats, off in batches + batches[:1]:
        m = off.size - 1
        dp, doff = dev_u8(pats), dev_u64(off)
        want = torch.full((m,), -1, dtype=torch.int64, device="cuda")
        capi.qfm_count(idx, dp, doff, want)
        for _ in range(2):                               # two calls in a row
            got = torch.full((m,), -1, dtype=torch.int64, device="cuda")
            rc = capi.lib.qfm_count_noalloc(idx, capi.ptr(dp), capi.ptr(doff), m, capi.ptr(got),
                                            capi.stream_ptr())
            assert rc == capi.QR_OK, capi.lib.qr_last_error()
            torch.cuda.synchronize()
            assert np.array_equal(host_u64(got), host_u64(want))
    assert capi.qfm_status(idx) == 0
    # argument errors are reported, not launched
    assert capi.lib.qfm_count_noalloc(None, None, None, 1, None, None) == capi.QR_EINVAL
    idx.free()

"""SM-limited streams (green contexts): the SM-count axis of the timing
recorder. Products on a partition of the SMs give the same bits and take
longer on large matrices."""
import numpy as np
import pytest
import torch

from paper_1801_01134_gb300 import inputs, spc5

pytestmark = pytest.mark.gpu


def test_sm_stream_products_are_identical_and_slower(cuda_device):
    try:
        small = spc5.SmStream(16)
    except spc5.Spc5Error as e:
        if e.status == spc5.EUNSUPPORTED:
            pytest.skip("no green contexts on this driver")
        raise
    sms_all = torch.cuda.get_device_properties(0).multi_processor_count
    assert 16 <= small.sms < sms_all and small.sms % 8 == 0
    A = inputs.stencil3d(96, 96, 64, points=27, seed=1)
    d = spc5.upload_csr(A, torch.float32, "cuda")
    M = spc5.convert(d.rowptr, d.colidx, d.values, A.n, A.m, 2, 4)
    x = torch.rand(A.m, dtype=torch.float32, device="cuda")
    ref = M.spmv(x)
    torch.cuda.synchronize()

    def timed(stream):
        ts = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            y = M.spmv(x, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return min(ts), y

    t_small, y_small = timed(small.stream)
    t_all, _ = timed(torch.cuda.current_stream())
    assert torch.equal(y_small, ref)
    assert t_small > 2.0 * t_all  # 16 of 152 SMs
    # the timing recorder on the partition
    ms = spc5.time_formats(d, reps=3, stream=small.stream)
    assert np.all(ms > 0)
    small.destroy()
    full = spc5.SmStream(100000)
    assert full.sms == sms_all
    full.destroy()

"""Failure detection on the GPU without a fault: a bounded device wait on a barrier that
nothing signals gives up, reports GB_ERR_TIMEOUT through the status word, and the CUDA
context stays usable (a bank call afterwards still matches the oracle)."""
import numpy as np
import pytest

import oracle
from paper_1704_05231_gb300 import synth
from tests.helpers import FP32_TOL, c1_bank, rel_err

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    import torch
    from paper_1704_05231_gb300 import GaborBank, GBError
    th, om, sg = c1_bank()
    with GaborBank(th, om, sg) as gbk:
        gbk.selftest_wait(1, limit_ms=5.0)          # signalled: no error
        gbk.device_status()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        gbk.selftest_wait(0, limit_ms=5.0)          # never signalled: gives up after ~5 ms
        ev1.record()
        with pytest.raises(GBError) as ei:
            gbk.device_status()
        assert ei.value.status == -6
        assert 4.0 <= ev0.elapsed_time(ev1) < 1000.0
        gbk.device_status()                          # the status word was cleared
        img = synth.uniform01(0, 64, 80)
        got = gbk.filter(torch.from_numpy(img).cuda()).cpu().numpy()
    assert rel_err(got, oracle.gabor_bank(img, th, om, sg)) <= FP32_TOL


def test_selftest_argument_checks():
    from paper_1704_05231_gb300 import GaborBank, GBError
    with GaborBank([0.0], [1.0], [1.0]) as gbk:
        for sig, lim in ((2, 5.0), (0, 0.0), (0, 5000.0)):
            with pytest.raises(GBError) as ei:
                gbk.selftest_wait(sig, limit_ms=lim)
            assert ei.value.status == -1

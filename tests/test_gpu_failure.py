"""Failure detection on the GPU without a fault: a bounded device wait that nothing completes gives up,
the kernel sets the handle's error word and returns, the call reports JDE_ERR_TIMEOUT, and the same
handle keeps working (nothing trapped, nothing hung)."""
import numpy as np
import pytest
import torch

import synth
from gpu_helpers import forward, jde, make_handle

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_the_context_stays_usable():
    j = jde()
    h = make_handle(j.JDE_BF16, max_batch=1, src_w=320, src_h=192)
    try:
        st = torch.cuda.current_stream()
        for limit in (1000, 200000):              # about 0.5 us and 100 us of SM clock
            status, word = j.jde_selftest_wait(h, limit, st)
            assert status == 6 and word & 1, (status, word)    # JDE_ERR_TIMEOUT, timeout bit of the word
            assert "gave up" in j.jde_last_error(h)
        assert j.jde_kernel_errors(h) == 0        # the call cleared the word it reported
        heads = forward(h, synth.frames_uniform(1, 1, 192, 320), 320, 192)   # the handle still runs
        assert all(np.isfinite(x).all() for x in heads)
        with pytest.raises(j.JdeError):
            j.jde_selftest_wait(h, 0, st)         # a limit outside [1, 2^31] is refused
    finally:
        j.jde_destroy(h)

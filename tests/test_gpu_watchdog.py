"""Failure detection without a GPU fault: a CTA whose bounded waits (the
tensor-core kernels' own mbarrier waits) run out on a barrier nothing arrives
on flags a time-out; the host reads it as TDE_ERR_TIMEOUT, the status word
is cleared, and the context keeps producing exact results."""
import pytest
import torch

import oracle
from paper_2509_19974_gb300 import synth, tde

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    from paper_2509_19974_gb300 import build
    build.build()
    ctx = tde.Context(0)
    try:
        ctx.selftest_wait_timeout()
        with pytest.raises(tde.TdeError) as ei:
            ctx.sync()
        assert ei.value.status == tde.TDE_ERR_TIMEOUT
        ctx.sync()  # read and cleared
        b = synth.single_pair(n=1500, dmax=100, bits=2)
        x, y = torch.from_numpy(b.x[0]).cuda(), torch.from_numpy(b.y[0]).cuda()
        lag, val = ctx.estimate(x, y, 2, engine="mma")
        ctx.sync()
        assert (int(lag.item()), int(val.item())) == oracle.estimate(b.x[0], b.y[0], 2)
    finally:
        ctx.close()

"""The failure path without a GPU fault (marked gpu): a bounded device wait
that runs out latches the codec's timeout status, lic_sync reports it once,
and the context stays usable -- the next encode/decode round trip is
lossless.  The wait is the tensor-core pipelines' own (same function, a
short limit); nothing hangs, traps or faults."""
import numpy as np
import pytest
import torch

import paper_2208_01641_b300 as lic
from paper_2208_01641_b300 import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_the_context_survives():
    W = synth.make_weights(lic.HYPERPRIOR, 64, 96)
    c = lic.Codec(lic.HYPERPRIOR, 64, 96, W)
    x = torch.from_numpy(synth.make_frames(2, 64, 64, first=3)).cuda()
    out = torch.empty_like(x)
    c.decode(c.encode(x), out)
    assert c.sync_status() == lic.OK
    ref = out.clone()
    c.test_bounded_wait(2_000_000)   # about a millisecond of SM clock
    assert c.sync_status() == lic.E_TIMEOUT
    assert c.sync_status() == lic.OK   # reported once, then cleared
    c.decode(c.encode(x), out)
    assert c.sync_status() == lic.OK
    assert torch.equal(out, ref)
    with pytest.raises(lic.LicError):
        c.test_bounded_wait(0)
    c.close()

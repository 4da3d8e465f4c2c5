"""The bounded device wait of the batched SU(3) kernels reports through the context's
status word: lq_sync returns LQ_ERR_TIMEOUT after a wait gave up, and LQ_OK otherwise.
The failure is made without faulting anything: the host writes the flag (lq_inject_status),
or a self-test block arms its barrier and issues no copy, so its short wait runs out with
nothing in flight (lq_selftest_wait_timeout)."""
import numpy as np
import pytest

import synth
from oracle import su3
from helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lq():
    import paper_1309_0551_gb300 as lq
    return lq


def _matvec_ok(lq, ctx):
    import torch
    A = synth.haar_su3(synth.rng(31), 1000)
    b = synth.complex_gaussian(synth.rng(32), (1000, 3))
    c = torch.empty((1000, 3), dtype=torch.complex128, device="cuda")
    lq.su3_matvec_batch(ctx, torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), c, 1000, 0)
    ctx.sync()
    assert rel_l2(c.cpu().numpy(), su3.mult_su3_mat_vec(A, b)) < 1e-14


def test_sync_ok_after_normal_work(lq):
    ctx = lq.Context(0)
    _matvec_ok(lq, ctx)
    ctx.sync()


def test_host_injected_flag_maps_to_timeout(lq):
    ctx = lq.Context(0)
    ctx.inject_status(1)
    with pytest.raises(lq.LQError, match="TIMEOUT"):
        ctx.sync()
    ctx.sync()            # the word was cleared by the report
    _matvec_ok(lq, ctx)   # and the context stays usable


def test_device_wait_runs_out_and_is_reported(lq):
    ctx = lq.Context(0)
    ctx.selftest_wait_timeout()
    with pytest.raises(lq.LQError, match="TIMEOUT.*TMA"):
        ctx.sync()
    _matvec_ok(lq, ctx)
    ctx.sync()

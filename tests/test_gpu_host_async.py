"""The pipelined host-buffer step (pab_bubble_step_host_async): a sequence of
calls with two sets of pinned host buffers gives, step by step, the same
moments and the same final state as the synchronous host-buffer step, bit for
bit; the waits free the buffers; bad arguments are refused."""
import numpy as np
import pytest

from paper_2511_21031_gb300 import pab, workloads

pytestmark = pytest.mark.gpu


def test_pipelined_steps_equal_synchronous_steps():
    import torch
    wl = workloads.config_small()
    n = 12
    a = pab.Solver(wl.n_cells, wl.n_bins, s_lognormal=wl.s)
    b = pab.Solver(wl.n_cells, wl.n_bins, s_lognormal=wl.s)
    ps = [torch.as_tensor(wl.pressure_step(k)).pin_memory() for k in range(n)]
    outs_a = [torch.empty((pab.N_MOMENTS, wl.n_cells), dtype=torch.float64).pin_memory() for _ in range(n)]
    outs_b = [torch.empty((pab.N_MOMENTS, wl.n_cells), dtype=torch.float64).pin_memory() for _ in range(n)]
    for k in range(n):
        a.step_host(ps[k], wl.dt, moments_host=outs_a[k])
    for k in range(n):
        b.step_host_async(ps[k], wl.dt, moments_host=outs_b[k])
    b.host_wait()
    for k in range(n):
        assert torch.equal(outs_a[k], outs_b[k]), k
    for x, y in zip(a.get_state(), b.get_state()):
        assert torch.equal(x, y)
    # reused host buffers: at most two calls in flight, each call waits for the one two before
    bufs = [torch.empty((pab.N_MOMENTS, wl.n_cells), dtype=torch.float64).pin_memory() for _ in range(2)]
    for k in range(n):
        a.step_host(ps[k], wl.dt, moments_host=outs_a[k])
        b.step_host_async(ps[k], wl.dt, moments_host=bufs[k % 2])
        if k >= 1:
            # the second call after call k-1 has not been made yet, so wait before reading
            pass
    b.host_wait()
    assert torch.equal(bufs[(n - 1) % 2], outs_a[n - 1])
    assert torch.equal(bufs[(n - 2) % 2], outs_a[n - 2])
    assert b.status()["flags"] == 0
    with pytest.raises(pab.PabError):
        b.step_host_async(ps[0], 0.0)
    a.close()
    b.close()

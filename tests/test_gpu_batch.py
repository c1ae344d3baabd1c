"""Batched persistent kernel: every slot advances exactly as the single-instance
step advances it alone, graph replay equals plain launches, rebinding between
queued steps reaches only the later steps, admission by arena memory, release
and reuse, and parity with the FP64 oracle."""
import dataclasses

import numpy as np
import pytest

from paper_2511_21031_gb300 import pab, workloads
from paper_2511_21031_gb300.batch import Batch
from tests.gpu_helpers import moment_errors, rel_err_R, rel_err_V, run_oracle

pytestmark = pytest.mark.gpu


def _instances(n=6, seed=21):
    insts = workloads.batched_instances(n=n, seed=seed, edge_lo=5, edge_hi=12, n_steps=40)
    return insts


def _cfg(w):
    d = dict(s_lognormal=w.s, R0ref=w.R0ref, span_K=w.span_K, alpha0=w.alpha0)
    d.update(w.fluid)
    return d


def _run_batch(insts, n_steps, precision, graph=False, launch=None):
    import torch
    b = Batch(max_slots=len(insts) + 2, precision=precision,
              capacity_bins=sum(w.n_cells * w.n_bins for w in insts) + 1000, max_bins=51)
    if launch:
        b.set_launch(*launch)
    slots = [b.admit(w.n_cells, w.n_bins, **_cfg(w)) for w in insts]
    moms = [torch.empty((7, w.n_cells), dtype=torch.float64, device="cuda") for w in insts]
    ps = [torch.empty(w.n_cells, dtype=torch.float64, device="cuda") for w in insts]
    for s, w, p, m in zip(slots, insts, ps, moms):
        b.bind(s, p, w.dt, moments=m)
    for n in range(n_steps):
        for w, p in zip(insts, ps):
            p.copy_(torch.as_tensor(w.pressure_step(n), device="cuda"))
        b.step(graph=graph)
    torch.cuda.synchronize()
    states = [b.get_state(s) for s in slots]
    stats = [b.status(s) for s in slots]
    out = [dict(R=st[0].cpu().numpy(), V=st[1].cpu().numpy(), h=st[2].cpu().numpy(),
                moments=m.cpu().numpy(), status=x) for st, m, x in zip(states, moms, stats)]
    b.close()
    return out


def _bins(w):
    import oracle
    return oracle.bins(w.n_bins, w.R0ref, w.s, w.span_K)[1]


def _run_single(w, n_steps, precision):
    import torch
    s = pab.Solver(w.n_cells, w.n_bins, precision=precision, **_cfg(w))
    m = torch.empty((7, w.n_cells), dtype=torch.float64, device="cuda")
    for n in range(n_steps):
        s.step(torch.as_tensor(w.pressure_step(n), device="cuda"), w.dt, moments=m)
    R, V, h = s.get_state()
    st = s.status()
    torch.cuda.synchronize()
    out = dict(R=R.cpu().numpy(), V=V.cpu().numpy(), h=h.cpu().numpy(), moments=m.cpu().numpy(), status=st)
    s.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_slots_equal_single_instance_steps(precision):
    insts = _instances()
    assert len({w.n_bins for w in insts}) > 1 and len({w.n_cells for w in insts}) > 1
    got = _run_batch(insts, 30, precision)
    for w, g in zip(insts, got):
        ref = _run_single(w, 30, precision)
        # same per-bin arithmetic; only rounding of the (inlined) code may differ.  The
        # mixed moments of the two kernels differ in how the FP32 parts are summed
        # (FP32 running sums vs FP64 sums of per-bin terms), within the mixed budget.
        assert rel_err_R(g["R"], ref["R"]) <= 1e-11
        assert rel_err_V(g["V"], ref["V"], w.fluid) <= 1e-9
        np.testing.assert_array_equal(g["h"] > 0, ref["h"] > 0)
        mtol = 1e-9 if precision == "fp64" else 1e-6
        for k, e in moment_errors(g["moments"], ref["moments"], ref["R"], ref["V"],
                                  np.array(_bins(w))).items():
            assert e <= mtol, (k, e)
        assert abs(g["status"]["n_attempts"] / ref["status"]["n_attempts"] - 1) <= 1e-3
        assert g["status"]["flags"] == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("launch", [(1, 32, 1), (4, 8, 1)])
def test_batch_of_slices_matches_the_whole_grid(precision, launch):
    """A grid cut into instances of contiguous cells (the bench's same-work batched line) is
    advanced by the batch exactly as the single-instance kernel advances the whole grid: the
    same state, step sizes, moments and trial count.  Both kernels inline the same trial, whose
    every FP32 operation is an explicit rounding and every FP64 product-sum an explicit fma, so
    no contraction choice of the compiler can set them apart."""
    wl = workloads.config_grid128(edge=32)
    insts = workloads.sliced_instances(wl, 8)
    got = _run_batch(insts, 20, precision, launch=launch)
    whole = dataclasses.replace(wl, precision=precision)
    ref = _run_single(whole, 20, precision)
    m = insts[0].n_cells
    for i, g in enumerate(got):
        sl = slice(i * m, (i + 1) * m)
        for key in ("R", "V", "h"):
            np.testing.assert_array_equal(g[key], ref[key][:, sl], err_msg=key)
        np.testing.assert_array_equal(g["moments"], ref["moments"][:, sl])
        assert g["status"]["flags"] == 0
    assert sum(g["status"]["n_attempts"] for g in got) == ref["status"]["n_attempts"]


def test_batch_fp64_matches_oracle():
    insts = _instances(n=4, seed=22)
    got = _run_batch(insts, 40, "fp64")
    for w, g in zip(insts, got):
        o = run_oracle(w, 40)
        assert rel_err_R(g["R"], o["R"]) <= 1e-6
        assert rel_err_V(g["V"], o["V"], w.fluid) <= 1e-6
        for k, e in moment_errors(g["moments"], o["moments"], o["R"], o["V"], o["w"]).items():
            assert e <= 1e-6, (k, e)


@pytest.mark.parametrize("launch", [(4, 1, 1), (16, 2, 2), (8, 4, 1), (1, 16, 1)])
def test_graph_replay_and_launch_shape_do_not_change_results(launch):
    insts = _instances(n=5, seed=23)
    a = _run_batch(insts, 12, "mixed")
    b = _run_batch(insts, 12, "mixed", graph=True, launch=launch)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x["R"], y["R"])
        np.testing.assert_array_equal(x["V"], y["V"])
        np.testing.assert_array_equal(x["h"], y["h"])
        np.testing.assert_array_equal(x["moments"], y["moments"])


@pytest.mark.parametrize("graph", [False, True])
def test_rebinding_between_queued_steps_uses_each_steps_own_inputs(graph):
    """A step reads the slot table when it runs, not when it is enqueued: binding fresh
    pressure tensors before each step while the earlier steps are still queued (behind a busy
    GPU) gives the same bits as refreshing one bound tensor in place."""
    import torch
    insts = _instances(n=4, seed=24)
    n_steps = 8
    ref = _run_batch(insts, n_steps, "mixed", graph=graph)
    b = Batch(max_slots=len(insts) + 2, precision="mixed",
              capacity_bins=sum(w.n_cells * w.n_bins for w in insts) + 1000, max_bins=51)
    slots = [b.admit(w.n_cells, w.n_bins, **_cfg(w)) for w in insts]
    moms = [torch.empty((7, w.n_cells), dtype=torch.float64, device="cuda") for w in insts]
    ps = [[torch.as_tensor(w.pressure_step(n), device="cuda") for w in insts] for n in range(n_steps)]
    torch.cuda.synchronize()
    sleep = getattr(torch.cuda, "_sleep", None)
    if sleep is not None:
        sleep(50_000_000)  # a bounded spin of about 25 ms, so that the steps below queue up
    for n in range(n_steps):
        for s, w, p, m in zip(slots, insts, ps[n], moms):
            b.bind(s, p, w.dt, moments=m)
        b.step(graph=graph)
    torch.cuda.synchronize()
    for s, m, r in zip(slots, moms, ref):
        R, V, h = b.get_state(s)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(R.cpu().numpy(), r["R"])
        np.testing.assert_array_equal(V.cpu().numpy(), r["V"])
        np.testing.assert_array_equal(h.cpu().numpy(), r["h"])
        np.testing.assert_array_equal(m.cpu().numpy(), r["moments"])
    b.close()


def test_admission_by_arena_memory_release_and_reuse():
    import torch
    b = Batch(max_slots=3, precision="mixed", capacity_bins=10 * 21 + 5 * 11, max_bins=21)
    s0 = b.admit(10, 21)
    s1 = b.admit(5, 11)
    assert b.try_admit(1, 1) is None                 # arena full
    u = b.usage()
    assert u["active_slots"] == 2 and u["bins_used"] == u["capacity_bins"]
    b.release(s0)
    assert b.try_admit(11, 21) is None               # 231 bins do not fit the 210 freed
    s2 = b.admit(10, 21)
    assert s2 == s0
    s3 = b.try_admit(1, 1)
    assert s3 is None
    # an admitted but unbound slot is not stepped
    p = torch.full((5,), 2 * 101325.0, dtype=torch.float64, device="cuda")
    b.bind(s1, p, 1e-8)
    b.step()
    R2, _, _ = b.get_state(s2)
    R1, _, _ = b.get_state(s1)
    torch.cuda.synchronize()
    assert torch.all(R2 == R2[:, :1])                # still at its initial R0 column values
    assert b.status(s1)["n_attempts"] > 0 and b.status(s2)["n_attempts"] == 0
    with pytest.raises(pab.PabError):
        b.admit(4, 51)                               # above max_bins
    b.close()


def test_batch_mixed_alpha_within_target_of_oracle():
    insts = _instances(n=4, seed=24)
    got = _run_batch(insts, 40, "mixed")
    for w, g in zip(insts, got):
        o = run_oracle(w, 40)
        em = moment_errors(g["moments"], o["moments"], o["R"], o["V"], o["w"])
        assert em[1] <= 1e-5, em
        assert rel_err_R(g["R"], o["R"]) <= 1e-5

"""Failure detection without a GPU fault (GB300 only).

* A stalled producer: the plan's waiting kernel runs with producers that
  never announce a filled stage (a flag that nothing sets); its bounded waits
  run out after about 2 s, it records FDD_ERR_TIMEOUT in the status word and
  returns; fdd_query reports it once and the plan keeps working.
* Allocation failures injected on the host (fdd_debug_fail_alloc) at several
  points of plan creation: FDD_ERR_ALLOC, nothing leaked.
No test traps, aborts or hangs the GPU.
"""
import time

import numpy as np
import pytest

import oracle
import paper_2110_03482_gb300 as fdd
import synth
from gpu_util import FP32_REL_L2, params_for, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fdd.build()
    yield
    fdd.fdd_debug_fail_alloc(-1)


def _smoke_check(plan, w, fb):
    out = torch.empty(plan.info["out_elems"], device="cuda")
    plan.execute(torch.from_numpy(fb).cuda(), out)
    torch.cuda.synchronize()
    ref = oracle.fdd_time(fb.T.astype(np.float64),
                          oracle.delays(w.channel_centres(), w.dms(), w.t_samp_s), w.chunk_len)
    return rel_l2(out.cpu().numpy().reshape(w.n_dm, -1), ref)


@pytest.mark.parametrize("precision,tol,n_dm", [(fdd.FDD_PREC_FP32, FP32_REL_L2, 0),
                                                (fdd.FDD_PREC_BF16_HILO, 3e-3, 0),
                                                (fdd.FDD_PREC_FP16, 3e-3, 3000)],
                         ids=["fp32", "tensor", "tensor_pair"])
def test_stalled_producer_times_out_and_the_plan_recovers(precision, tol, n_dm):
    """A kernel whose producers never announce a filled stage runs its waits
    out, reports FDD_ERR_TIMEOUT once and leaves the context usable; the
    third case is a plan of the CTA-pair form (3000 trials), whose second
    CTA forwards its stages to the first."""
    w = synth.WORKLOADS["fdd_64ch_4096t_128dm"]
    if n_dm:
        w = w.scaled(n_dm=n_dm, ddm=0.01)
    fb, _ = synth.filterbank(w, seed=20211008)
    with fdd.Plan(**params_for(w, precision=precision)) as plan:
        assert plan.query()["n_bins"] == 2049
        if n_dm:
            assert plan.info["mac_variant"] == fdd.FDD_MAC_TC_PAIR
        t0 = time.perf_counter()
        plan.debug_stall_test()
        dt = time.perf_counter() - t0
        assert 0.5 < dt < 60.0, dt  # the waits ran to their limit, and ended
        with pytest.raises(fdd.FddError) as e:
            plan.query()
        assert e.value.status == fdd.FDD_ERR_TIMEOUT
        plan.query()  # reported once
        assert _smoke_check(plan, w, fb) <= tol  # the context and the plan still work


def test_injected_allocation_failures_leak_nothing():
    w = synth.WORKLOADS["fdd_64ch_4096t_128dm"]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    n_fail = 0
    for after in range(0, 12):
        fdd.fdd_debug_fail_alloc(after)
        try:
            with fdd.Plan(**params_for(w, precision=fdd.FDD_PREC_BF16_HILO)):
                pass
        except fdd.FddError as e:
            assert e.status == fdd.FDD_ERR_ALLOC and "injected" in str(e)
            n_fail += 1
        finally:
            fdd.fdd_debug_fail_alloc(-1)
    assert n_fail >= 5  # the plan makes at least five allocations
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (64 << 20)
    # a batch plan, and the staging buffers of the first host-buffer call
    fdd.fdd_debug_fail_alloc(2)
    with pytest.raises(fdd.FddError) as e:
        fdd.Batch([(3000, 0.0, 1.0, 64)], n_chan=16, nu_lo_mhz=1200.0, dnu_mhz=2.0,
                  t_samp_s=1e-3, in_dtype=fdd.FDD_IN_F32, output=fdd.FDD_OUT_POWER,
                  chunk_len=0, autotune=False)
    assert e.value.status == fdd.FDD_ERR_ALLOC
    fdd.fdd_debug_fail_alloc(-1)
    fb, _ = synth.filterbank(w, seed=3)
    with fdd.Plan(**params_for(w)) as plan:
        h_out = torch.empty(plan.info["out_elems"], dtype=torch.float32).pin_memory()
        h_in = torch.from_numpy(fb.reshape(-1)).pin_memory()
        fdd.fdd_debug_fail_alloc(0)
        with pytest.raises(fdd.FddError) as e:
            plan.execute_host(h_in, h_out)
        assert e.value.status == fdd.FDD_ERR_ALLOC
        fdd.fdd_debug_fail_alloc(-1)
        plan.execute_host(h_in, h_out)  # the next call allocates and runs
        torch.cuda.synchronize()
        assert np.isfinite(h_out.numpy()).all()

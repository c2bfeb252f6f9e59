"""fdd_execute_host (host buffers, copies pipelined with the computation over
(beam, chunk) units on two plan-owned streams) gives bit for bit what
fdd_execute gives on device buffers (GB300 only): both layouts, every output
kind, several beams and chunks, the tensor-core form, back-to-back calls
with different inputs, and pageable host memory.  fdd_execute captured into a
CUDA graph replays bit for bit."""
import numpy as np
import pytest

import paper_2110_03482_gb300 as fdd
import synth
from gpu_util import params_for

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fdd.build()


def _workload(n_beams, output, dtype="u8", chunk_len=2048, n_t=7000):
    return synth.Workload(name="host", n_chan=40, band_lo_mhz=400.0, band_hi_mhz=500.0,
                          t_samp_s=1e-3, n_t=n_t, dtype=dtype, dm0=0.0, ddm=1.0, n_dm=90,
                          chunk_len=chunk_len, n_beams=n_beams, output=output,
                          pulses_per_beam=1,
                          noise_mean=128.0 if dtype == "u8" else 0.0,
                          noise_sigma=16.0 if dtype == "u8" else 1.0)


def _inputs(w, layout, seed):
    fbs = [synth.filterbank(w, seed=seed, beam=b)[0] for b in range(w.n_beams)]
    if layout == fdd.FDD_LAYOUT_CHAN_MAJOR:
        fbs = [np.ascontiguousarray(f.T) for f in fbs]
    return np.ascontiguousarray(np.stack(fbs))


def _out_like(info, output, device):
    shape = (info["out_elems"], 2) if output == fdd.FDD_OUT_SPECTRA else (info["out_elems"],)
    if device:
        return torch.empty(shape, dtype=torch.float32, device="cuda")
    return torch.empty(shape, dtype=torch.float32).pin_memory()


@pytest.mark.parametrize("output,layout,n_beams,precision,ds", [
    (fdd.FDD_OUT_TIME, fdd.FDD_LAYOUT_TIME_MAJOR, 1, fdd.FDD_PREC_FP32, 1),
    (fdd.FDD_OUT_TIME, fdd.FDD_LAYOUT_CHAN_MAJOR, 2, fdd.FDD_PREC_FP32, 1),
    (fdd.FDD_OUT_SPECTRA, fdd.FDD_LAYOUT_TIME_MAJOR, 3, fdd.FDD_PREC_FP32, 1),
    (fdd.FDD_OUT_POWER, fdd.FDD_LAYOUT_CHAN_MAJOR, 2, fdd.FDD_PREC_FP32, 1),
    (fdd.FDD_OUT_TIME, fdd.FDD_LAYOUT_TIME_MAJOR, 5, fdd.FDD_PREC_BF16_HILO, 1),
    (fdd.FDD_OUT_POWER, fdd.FDD_LAYOUT_TIME_MAJOR, 3, fdd.FDD_PREC_BF16_HILO, 1),
    (fdd.FDD_OUT_TIME, fdd.FDD_LAYOUT_TIME_MAJOR, 2, fdd.FDD_PREC_FP32, 4),   # down-sampled
    (fdd.FDD_OUT_TIME, fdd.FDD_LAYOUT_TIME_MAJOR, 3, fdd.FDD_PREC_BF16_HILO, 2),
    (fdd.FDD_OUT_TIME, fdd.FDD_LAYOUT_TIME_MAJOR, 3, fdd.FDD_PREC_FP16, 1),
])
def test_host_pipeline_equals_device_execute(output, layout, n_beams, precision, ds):
    out_name = {fdd.FDD_OUT_TIME: "time", fdd.FDD_OUT_SPECTRA: "spectra",
                fdd.FDD_OUT_POWER: "power"}[output]
    w = _workload(n_beams, out_name)
    with fdd.Plan(**params_for(w, in_layout=layout, precision=precision, downsample=ds)) as plan:
        info = plan.info
        assert info["n_chunks"] >= 3
        stream = torch.cuda.current_stream()
        results = []
        for seed in (1, 2):  # back-to-back calls reuse the pipeline
            x = _inputs(w, layout, seed)
            d_out = _out_like(info, output, True)
            plan.execute(torch.from_numpy(x).cuda(), d_out)
            h_in = torch.from_numpy(x.reshape(-1)).pin_memory()
            h_out = _out_like(info, output, False)
            h_out.fill_(float("nan"))
            plan.execute_host(h_in, h_out, stream)
            results.append((d_out, h_out, h_in))  # h_in stays alive until the sync
        stream.synchronize()
        for d_out, h_out, _ in results:
            assert torch.equal(d_out.cpu(), h_out)


def test_host_pipeline_pageable_memory_and_single_chunk():
    w = _workload(2, "time", dtype="f32", chunk_len=0, n_t=3000)
    x = _inputs(w, fdd.FDD_LAYOUT_TIME_MAJOR, 7)
    with fdd.Plan(**params_for(w)) as plan:
        info = plan.info
        d_out = torch.empty(info["out_elems"], dtype=torch.float32, device="cuda")
        plan.execute(torch.from_numpy(x).cuda(), d_out)
        h_out = torch.empty(info["out_elems"], dtype=torch.float32)  # pageable
        plan.execute_host(torch.from_numpy(x.reshape(-1)), h_out)
        torch.cuda.synchronize()
        assert torch.equal(d_out.cpu(), h_out)


@pytest.mark.parametrize("precision", [fdd.FDD_PREC_FP32, fdd.FDD_PREC_BF16_HILO],
                         ids=["fp32", "bf16_hilo"])
def test_execute_replays_from_a_cuda_graph(precision):
    """fdd_execute neither synchronises nor allocates, so a caller can capture
    it into a CUDA graph (with profiling off): every replay equals the direct
    call bit for bit, including after the input buffer is refilled in place."""
    w = _workload(2, "time", chunk_len=2048)
    x1 = torch.from_numpy(_inputs(w, fdd.FDD_LAYOUT_TIME_MAJOR, 3)).cuda()
    x2 = torch.from_numpy(_inputs(w, fdd.FDD_LAYOUT_TIME_MAJOR, 4)).cuda()
    with fdd.Plan(**params_for(w, precision=precision)) as plan:
        info = plan.info
        ref1 = torch.empty(info["out_elems"], dtype=torch.float32, device="cuda")
        ref2 = torch.empty_like(ref1)
        plan.execute(x1, ref1)
        plan.execute(x2, ref2)
        d_in = x1.clone()
        out = torch.zeros_like(ref1)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            plan.execute(d_in, out)  # warm-up on the capture stream
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            plan.execute(d_in, out)
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref1)
        d_in.copy_(x2)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref2)
        assert plan.query()["out_elems"] == info["out_elems"]  # no device-side status raised

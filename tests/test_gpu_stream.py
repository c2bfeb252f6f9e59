"""fdd_execute_stream (input windows from a source, output blocks to a sink,
through plan-owned rings of two slots) gives bit for bit what fdd_execute
gives on whole device buffers (GB300 only): the FP32 and tensor-core forms,
time, spectra and power output, several chunks and beams, both input layouts,
and output streamed in several trial blocks.  A failing callback ends the
call with its status."""
import ctypes

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


def _workload(n_beams, output, n_dm, dtype="u8", chunk_len=2048, n_t=7000):
    # (trials span DM 0 .. 90 whatever their count: delays stay below the chunk)
    return synth.Workload(name="stream", n_chan=40, band_lo_mhz=400.0, band_hi_mhz=500.0,
                          t_samp_s=1e-3, n_t=n_t, dtype=dtype, dm0=0.0, ddm=90.0 / n_dm,
                          n_dm=n_dm,
                          chunk_len=chunk_len, n_beams=n_beams, output=output,
                          pulses_per_beam=1,
                          noise_mean=128.0 if dtype == "u8" else 0.0,
                          noise_sigma=16.0 if dtype == "u8" else 1.0)


def _stream_into(plan, w, d_in, d_out, layout, stream):
    """fdd_execute_stream with a source reading windows of d_in and a sink
    writing blocks into d_out at the places fdd_execute writes them."""
    info = plan.info
    esz = 1 if w.dtype == "u8" else 4
    oesz = 8 if w.output == "spectra" else 4
    beam_bytes = esz * w.n_t * w.n_chan
    seen = []

    def source(beam, t0, n, d_window, ready, s):
        base = d_in.data_ptr() + beam * beam_bytes
        if layout == fdd.FDD_LAYOUT_TIME_MAJOR:
            fdd.memcpy_async(d_window, base + esz * t0 * w.n_chan, esz * n * w.n_chan, s)
        else:
            fdd.memcpy2d_async(d_window, esz * n, base + esz * t0, esz * w.n_t, esz * n,
                               w.n_chan, s)

    def sink(blk, s):
        seen.append(blk)
        if w.output == "time":
            L = info["out_len"]
            dst = d_out.data_ptr() + 4 * ((blk["beam_first"] * w.n_dm + blk["dm_first"]) * L +
                                          blk["out_offset"])
            fdd.memcpy2d_async(dst, 4 * L, blk["d_data"], 4 * blk["row_pitch"],
                               4 * blk["row_len"], blk["n_dm"], s)
        else:
            K, C = info["n_bins"], info["n_chunks"]
            rows_beam = C * w.n_dm
            dst = d_out.data_ptr() + oesz * ((blk["beam_first"] * rows_beam +
                                              blk["chunk"] * w.n_dm + blk["dm_first"]) * K)
            fdd.memcpy2d_async(dst, oesz * rows_beam * K, blk["d_data"],
                               oesz * blk["n_dm"] * K, oesz * blk["n_dm"] * K,
                               blk["n_beams"], s)

    plan.execute_stream(source, sink, stream)
    return seen


@pytest.mark.parametrize("output,layout,n_beams,precision,n_dm,limit", [
    ("time", fdd.FDD_LAYOUT_TIME_MAJOR, 2, fdd.FDD_PREC_FP32, 90, 0),
    ("time", fdd.FDD_LAYOUT_CHAN_MAJOR, 1, fdd.FDD_PREC_FP32, 300, 1 << 21),  # DM batches
    ("spectra", fdd.FDD_LAYOUT_TIME_MAJOR, 2, fdd.FDD_PREC_FP32, 300, 1 << 21),  # trial blocks
    ("power", fdd.FDD_LAYOUT_CHAN_MAJOR, 3, fdd.FDD_PREC_FP32, 90, 0),
    ("time", fdd.FDD_LAYOUT_TIME_MAJOR, 3, fdd.FDD_PREC_FP16, 90, 0),
    ("power", fdd.FDD_LAYOUT_TIME_MAJOR, 3, fdd.FDD_PREC_FP16, 2100, 1 << 25),  # trial blocks
    ("spectra", fdd.FDD_LAYOUT_CHAN_MAJOR, 2, fdd.FDD_PREC_BF16_HILO, 90, 0),
])
def test_stream_equals_device_execute(output, layout, n_beams, precision, n_dm, limit):
    w = _workload(n_beams, output, n_dm)
    fbs = [synth.filterbank(w, seed=9, beam=b)[0] for b in range(n_beams)]
    if layout == fdd.FDD_LAYOUT_CHAN_MAJOR:
        fbs = [np.ascontiguousarray(f.T) for f in fbs]
    d_in = torch.from_numpy(np.ascontiguousarray(np.stack(fbs))).cuda()
    # (FP32 under a limit: the 128-trial tile, whose blocks the limit splits
    # into several; the default tile's blocks are 2048 trials)
    tile = dict(mac_variant=fdd.FDD_MAC_Q_4X4 + 1) if precision == fdd.FDD_PREC_FP32 and limit \
        else {}
    with fdd.Plan(**params_for(w, in_layout=layout, precision=precision,
                               workspace_limit=limit, **tile)) as plan:
        info = plan.info
        assert info["n_chunks"] >= 3
        shape = (info["out_elems"], 2) if output == "spectra" else (info["out_elems"],)
        ref = torch.empty(shape, dtype=torch.float32, device="cuda")
        plan.execute(d_in, ref)
        got = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream()
        seen = _stream_into(plan, w, d_in, got, layout, stream.cuda_stream)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
        if output != "time":
            assert max(b["n_dm"] for b in seen) == min(info["block_dm"], n_dm)
        if limit and output != "time":
            assert info["block_dm"] < n_dm  # several trial blocks per chunk
        assert plan.query()["stream_bytes"] == info["stream_bytes"]


def test_stream_callback_failure_ends_the_call():
    w = _workload(1, "time", 90)
    with fdd.Plan(**params_for(w)) as plan:
        def source(beam, t0, n, d_window, ready, s):
            raise ValueError("no input here")

        with pytest.raises(ValueError):
            plan.execute_stream(source, lambda blk, s: None)
        torch.cuda.synchronize()


class _Events:
    """Raw CUDA events and a copy stream (through the runtime) for callbacks
    that work off the compute stream."""

    def __init__(self):
        rt = fdd.cudart()
        vp = ctypes.c_void_p
        rt.cudaEventCreateWithFlags.argtypes = [ctypes.POINTER(vp), ctypes.c_uint]
        rt.cudaEventRecord.argtypes = [vp, vp]
        rt.cudaStreamWaitEvent.argtypes = [vp, vp, ctypes.c_uint]
        rt.cudaEventDestroy.argtypes = [vp]
        self.rt = rt
        self.copy = torch.cuda.Stream()
        self.pool = []

    def event(self):
        e = ctypes.c_void_p()
        assert self.rt.cudaEventCreateWithFlags(ctypes.byref(e), 2) == 0  # disable timing
        self.pool.append(e)
        return e.value

    def record(self, ev, stream):
        assert self.rt.cudaEventRecord(ev, stream) == 0

    def wait(self, stream, ev):
        assert self.rt.cudaStreamWaitEvent(stream, ev, 0) == 0

    def close(self):
        for e in self.pool:
            self.rt.cudaEventDestroy(e)


@pytest.mark.parametrize("output,precision,n_dm,limit", [
    ("time", fdd.FDD_PREC_FP16, 90, 0),
    ("spectra", fdd.FDD_PREC_FP32, 300, 1 << 21),
])
def test_stream_resident_input_and_sink_on_another_stream(output, precision, n_dm, limit):
    """Input resident on the device (d_in); the sink copies each block on its
    own stream and hands back a release event, so the copies overlap."""
    w = _workload(3, output, n_dm)
    x = np.ascontiguousarray(np.stack([synth.filterbank(w, seed=4, beam=b)[0]
                                       for b in range(3)]))
    d_in = torch.from_numpy(x).cuda()
    ev = _Events()
    with fdd.Plan(**params_for(w, precision=precision, workspace_limit=limit)) as plan:
        info = plan.info
        shape = (info["out_elems"], 2) if output == "spectra" else (info["out_elems"],)
        ref = torch.empty(shape, dtype=torch.float32, device="cuda")
        plan.execute(d_in, ref)
        got = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
        oesz = 8 if output == "spectra" else 4
        cs = ev.copy.cuda_stream

        def sink(blk, s):
            done = ev.event()
            ev.record(done, s)
            ev.wait(cs, done)  # the block is complete
            if output == "time":
                L = info["out_len"]
                dst = got.data_ptr() + 4 * ((blk["beam_first"] * n_dm + blk["dm_first"]) * L +
                                            blk["out_offset"])
                fdd.memcpy2d_async(dst, 4 * L, blk["d_data"], 4 * blk["row_pitch"],
                                   4 * blk["row_len"], blk["n_dm"], cs)
            else:
                K, C = info["n_bins"], info["n_chunks"]
                rows_beam = C * n_dm
                dst = got.data_ptr() + oesz * ((blk["beam_first"] * rows_beam +
                                                blk["chunk"] * n_dm + blk["dm_first"]) * K)
                fdd.memcpy2d_async(dst, oesz * rows_beam * K, blk["d_data"],
                                   oesz * blk["n_dm"] * K, oesz * blk["n_dm"] * K,
                                   blk["n_beams"], cs)
            rel = ev.event()
            ev.record(rel, cs)
            return rel

        stream = torch.cuda.current_stream()
        plan.execute_stream(None, sink, stream, d_in=d_in)
        torch.cuda.synchronize()
        ev.close()
        assert torch.equal(got, ref)

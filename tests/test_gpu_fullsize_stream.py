"""The multi-beam tensor-core workloads at their full sizes, streamed as the
benchmark runs them (GB300 only), on outputs the FP64 oracle computes one by
one from the same counter-generated input:

- 32 beams x 1024 channels x 2^19 float32 samples x 4096 trials (DM 0 ..
  2047.5), whole-series transform of 2^19 points, time output, FP16 tensor
  cores, input resident, output blocks through fdd_execute_stream: whole
  time rows of two beams at five trials, against the oracle's FFT, Eq. 7 on
  every bin and inverse transform.
- 16 beams x 4096 channels x 2^21 float32 samples x 8192 trials (DM 0 ..
  409.55), overlap-save chunks of 2^19 (six), |Y|^2 output, FP16 tensor
  cores, every (beam, chunk) window generated on the device by the source:
  sampled bins of two beams in the first and last chunk at four trials.

The gate is the low-precision form's rel-L2 of 3e-3 against FP64 (on the
power: twice that, the first-order growth of a relative error under
squaring)."""
import numpy as np
import pytest

import oracle
import paper_2110_03482_gb300 as fdd
import synth
import synth.gpu
from gpu_util import params_for, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TC_REL_L2 = 3e-3
SEED = 20211007


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fdd.build()
    synth.gpu.build()


def _beams(w):
    return synth.gpu.BeamWindows([synth.philox_beam_args(w, SEED, b)[0] for b in range(w.n_beams)])


def _host_rows(gen, beam, t0, n_rows, n_chan):
    buf = torch.empty(n_rows * n_chan, dtype=torch.float32, device="cuda")
    gen.fill(beam, buf.data_ptr(), t0, n_rows, torch.cuda.current_stream().cuda_stream)
    return buf.cpu().numpy().reshape(n_rows, n_chan)


def test_32beam_full_size_time_output_sampled():
    w = synth.WORKLOADS["fdd_32beam_1024ch_2p19t_4096dm"]
    gen = _beams(w)
    beams, trials = [0, 17], [0, 1023, 1024, 2900, 4095]
    with fdd.Plan(**params_for(w, precision=fdd.FDD_PREC_FP16,
                               workspace_limit=200 << 30)) as plan:
        info = plan.info
        assert (info["fft_len"], info["n_chunks"], info["dm_batch"]) == (1 << 19, 1, 1024)
        d_in = torch.empty(w.n_beams * w.n_t * w.n_chan, dtype=torch.float32, device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        for b in range(w.n_beams):
            gen.fill(b, d_in.data_ptr() + 4 * b * w.n_t * w.n_chan, 0, w.n_t, s)
        got = {}

        def sink(blk, stream):
            b = blk["beam_first"]
            for j in trials:
                r = j - blk["dm_first"]
                if b in beams and 0 <= r < blk["n_dm"]:
                    row = torch.empty(blk["row_len"], dtype=torch.float32, device="cuda")
                    fdd.memcpy_async(row.data_ptr(), blk["d_data"] + 4 * r * blk["row_pitch"],
                                     4 * blk["row_len"], stream)
                    got[(b, j)] = row
            return None

        plan.execute_stream(None, sink, torch.cuda.current_stream(), d_in=d_in)
        torch.cuda.synchronize()
        plan.query()
        del d_in
    torch.cuda.empty_cache()  # the next workload needs the device memory back
    assert len(got) == len(beams) * len(trials)
    d = oracle.delays(w.channel_centres(), w.dms()[trials], w.t_samp_s)
    K = (1 << 19) // 2 + 1
    for b in beams:
        x = _host_rows(gen, b, 0, w.n_t, w.n_chan).T.astype(np.float64)
        X = oracle.fft_r2c(x)
        Y = oracle.fdd_bins(X, np.arange(K), 1 << 19, d)
        ref = oracle.irfft(Y, 1 << 19)
        for q, j in enumerate(trials):
            y = got[(b, j)].cpu().numpy().astype(np.float64)
            err = rel_l2(y, ref[q])
            print(f"32 beams, 2^19 points: beam {b} trial {j}: rel-L2 vs FP64 {err:.2e}")
            assert err <= TC_REL_L2, (b, j, err)


def test_16beam_full_size_power_streamed_sampled():
    torch.cuda.empty_cache()
    w = synth.WORKLOADS["fdd_16beam_4096ch_2p21t_8192dm_power"]
    gen = _beams(w)
    beams, chunks, trials = [0, 9], [0, 5], [0, 2047, 2048, 8191]
    with fdd.Plan(**params_for(w, precision=fdd.FDD_PREC_FP16,
                               workspace_limit=240 << 30)) as plan:
        info = plan.info
        L, K, hop = info["fft_len"], info["n_bins"], info["hop"]
        assert (L, info["n_chunks"]) == (1 << 19, 6)
        got = {}

        def source(beam, t0, n, d_window, ready, stream):
            gen.fill(beam, d_window, t0, n, stream)

        def sink(blk, stream):
            c = blk["chunk"]
            if c not in chunks:
                return None
            for q, b in enumerate(range(blk["beam_first"], blk["beam_first"] + blk["n_beams"])):
                if b not in beams:
                    continue
                for j in trials:
                    r = j - blk["dm_first"]
                    if 0 <= r < blk["n_dm"]:
                        row = torch.empty(K, dtype=torch.float32, device="cuda")
                        off = 4 * ((q * blk["n_dm"] + r) * blk["row_pitch"])
                        fdd.memcpy_async(row.data_ptr(), blk["d_data"] + off, 4 * K, stream)
                        got[(b, c, j)] = row
            return None

        plan.execute_stream(source, sink, torch.cuda.current_stream())
        torch.cuda.synchronize()
        plan.query()
    assert len(got) == len(beams) * len(chunks) * len(trials)
    rng = np.random.default_rng(3)
    bins = np.unique(np.concatenate([[0, 1, K - 1], rng.integers(2, K - 1, 29)]))
    d = oracle.delays(w.channel_centres(), w.dms()[trials], w.t_samp_s)
    for b in beams:
        for c in chunks:
            n = min(L, w.n_t - c * hop)
            x = np.zeros((w.n_chan, L))
            x[:, :n] = _host_rows(gen, b, c * hop, n, w.n_chan).T
            X = oracle.fft_r2c(x)[:, bins]
            ref = np.abs(oracle.fdd_bins(X, bins, L, d)) ** 2
            for q, j in enumerate(trials):
                p = got[(b, c, j)].cpu().numpy().astype(np.float64)[bins]
                err = rel_l2(p, ref[q])
                print(f"16 beams, 4096 ch: beam {b} chunk {c} trial {j}: power rel-L2 {err:.2e}")
                assert err <= 2 * TC_REL_L2, (b, c, j, err)

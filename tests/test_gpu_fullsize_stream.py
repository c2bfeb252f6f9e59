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
        # 1941 trials fit under the 200 GiB limit: batches of one-CTA passes
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


@pytest.mark.parametrize("precision", [fdd.FDD_PREC_FP32, fdd.FDD_PREC_FP16], ids=["fp32", "fp16"])
def test_96beam_full_size_batch_streamed_sampled(precision):
    """The 96-beam batch at its full lengths (n_t up to ~2^20, 1536 channels,
    512-4096 trials, |Y|^2), streamed as the benchmark runs it (every beam's
    windows generated on the device, output blocks to a sink), in the FP32
    form (persistent launch per wave) and on tensor cores (groups of beams
    sharing their phasors): sampled bins of the longest, shortest, most- and
    fewest-trial beams at four trials each, against the oracle."""
    torch.cuda.empty_cache()
    bw = synth.BATCH_WORKLOADS["fdd_96beam_1536ch_uneven"]
    beams = bw.beams(SEED)
    n_ts = np.array([b[0] for b in beams])
    n_dms = np.array([b[3] for b in beams])
    checked = sorted({int(np.argmin(n_ts)), int(np.argmax(n_ts)), int(np.argmax(n_dms)),
                      int(np.argmin(n_dms))})
    gen = synth.gpu.BeamWindows([synth.batch_beam_args(bw, desc, SEED, b)[0]
                                 for b, desc in enumerate(beams)])
    common = dict(n_chan=bw.n_chan, nu_lo_mhz=bw.nu_lo_mhz, dnu_mhz=bw.dnu_mhz,
                  t_samp_s=bw.t_samp_s, in_dtype=fdd.FDD_IN_F32, chunk_len=0,
                  output=fdd.FDD_OUT_POWER, precision=precision,
                  workspace_limit=(200 << 30) if precision != fdd.FDD_PREC_FP32 else (100 << 30))
    rng = np.random.default_rng(7)
    picks = {}
    for b in checked:
        K = oracle.next_pow2(beams[b][0]) // 2 + 1
        bins = np.unique(np.concatenate([[0, 1, K - 1], rng.integers(2, K - 1, 5)]))
        trials = sorted({0, beams[b][3] // 2, beams[b][3] - 1, int(rng.integers(1, beams[b][3]))})
        picks[b] = (K, bins, trials)
    got = {}
    with fdd.Batch(beams, autotune=False, **common) as batch:

        def source(beam, t0, n, d_window, ready, s):
            gen.fill(beam, d_window, t0, n, s)

        def sink(blk, s):
            b = blk["beam_first"]
            if b not in picks:
                return None
            K, bins, trials = picks[b]
            for j in trials:
                r = j - blk["dm_first"]
                if 0 <= r < blk["n_dm"]:
                    row = torch.empty(K, dtype=torch.float32, device="cuda")
                    fdd.memcpy_async(row.data_ptr(), blk["d_data"] + 4 * r * blk["row_pitch"],
                                     4 * K, s)
                    got[(b, j)] = row
            return None

        batch.execute_stream(source, sink, torch.cuda.current_stream())
        torch.cuda.synchronize()
        info = batch.info
    torch.cuda.empty_cache()
    assert len(got) == sum(len(p[2]) for p in picks.values())
    errs = []
    for b in checked:
        n_t, dm0, ddm, n_dm = beams[b]
        K, bins, trials = picks[b]
        L = 2 * (K - 1)
        x = np.zeros((bw.n_chan, L))
        x[:, :n_t] = _host_rows(gen, b, 0, n_t, bw.n_chan).T
        X = oracle.fft_r2c(x)[:, bins]
        d = oracle.delays(bw.nu_lo_mhz + bw.dnu_mhz * np.arange(bw.n_chan),
                          dm0 + ddm * np.array(trials, dtype=np.float64), bw.t_samp_s)
        ref = np.abs(oracle.fdd_bins(X, bins, L, d)) ** 2
        for q, j in enumerate(trials):
            p = got[(b, j)].cpu().numpy().astype(np.float64)[bins]
            errs.append(rel_l2(p, ref[q]))
    tol = 2 * (1e-5 if precision == fdd.FDD_PREC_FP32 else TC_REL_L2)
    print(f"96 uneven beams at full length ({'TC' if info['mac_variant'] == fdd.FDD_MAC_TC else 'FP32'}"
          f", {info['n_waves']} waves/plans): power rel-L2 vs FP64 max {max(errs):.2e} "
          f"over beams {checked}")
    assert max(errs) <= tol

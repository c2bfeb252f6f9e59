"""Parity at the workloads' full sizes, on outputs the FP64 oracle can compute
one by one (GB300 only).

Each workload runs in the launch configuration the benchmark times; the
oracle recomputes sampled trials, bins and beams from the same seeded inputs
(the host copy of the filterbank, or the counter-based generator regenerating
the beams it needs).  Errors are printed per workload against FP64.

- 1024 channels x 2^20 8-bit samples x 2048 trials, 2^18-sample overlap-save
  chunks, time-domain output (fdd_execute): 9 whole trial rows of the first,
  a middle and the last chunk, in the time domain and as dedispersed spectra
  (the same plan with spectra output), and the five injected pulses.
- 32 beams x 1024 channels x 4096 trials on the tensor cores: the benchmark's
  2049-bin slice (all bins computed, 6 bins x 2 beams checked) in both
  precisions, and bin windows at DC, mid-band and Nyquist of the whole 2^19
  transform (phases as large as the full workload's).
- 96 uneven beams x 1536 channels (batching form, lengths / 16 as in the
  benchmark, autotuned): four beams checked at 8 bins each, all their trials.
- 16 beams x 4096 channels x 8192 trials (step 0.05) on the tensor cores in
  16-beam groups, power output: bin windows of the 2^19 transform; and the
  whole chain (counter-generated input, chunks of 2^19 with the workload's
  delay span, power output) at 64 channels for the top 64 trials.
"""
import numpy as np
import pytest

import oracle
import paper_2110_03482_gb300 as fdd
import synth
import synth.gpu
from gpu_util import FP32_REL_L2, complex_to_device, device_to_complex, params_for, rel_l2
from synth import philox

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


def _delays(w, dms=None):
    return oracle.delays(w.channel_centres(), w.dms() if dms is None else dms, w.t_samp_s)


# ---------------------------------------------------------------- survey, FP32
def test_survey_full_size_time_output_sampled():
    w = synth.WORKLOADS["fdd_1024ch_2p20t_2048dm"]
    fb, pulses = synth.filterbank(w, seed=SEED)
    d = _delays(w)
    geo = oracle.geometry(w.n_t, w.chunk_len, d)
    with fdd.Plan(**params_for(w)) as plan:
        info = plan.info
        assert (info["fft_len"], info["n_chunks"], info["out_len"]) == (geo.L, geo.n_chunks,
                                                                        geo.n_out)
        dx = torch.from_numpy(fb).cuda()
        out = torch.empty((w.n_dm, info["out_len"]), dtype=torch.float32, device="cuda")
        plan.execute(dx, out)
        torch.cuda.synchronize()
        plan.query()
        del dx
        pulse_rows = [int(round((p.dm - w.dm0) / w.ddm)) for p in pulses]
        rows = sorted(set([0, 1, 1023, 2047] + pulse_rows))
        got = out[rows].cpu().numpy().astype(np.float64)
        # the pulses: each peaks at its own trial (+-1) and emission sample
        for p, j in zip(pulses, pulse_rows):
            if p.t0 + 8 >= info["out_len"]:
                continue
            lo, hi = max(0, j - 6), min(w.n_dm, j + 7)
            blk = out[lo:hi, max(0, p.t0 - 64): p.t0 + 64]
            blk = blk - blk.mean(dim=1, keepdim=True)
            jj, tt = np.unravel_index(int(torch.argmax(blk).item()), tuple(blk.shape))
            assert abs(lo + jj - j) <= 1 and abs(max(0, p.t0 - 64) + tt - p.t0) <= 3, (p, jj, tt)
        del out
    # the same plan with spectra output, one sampled trial per call (all chunks)
    with fdd.Plan(**params_for(w, output=fdd.FDD_OUT_SPECTRA)) as plan:
        dx = torch.from_numpy(fb).cuda()
        spec = torch.empty((len(rows), geo.n_chunks, geo.K, 2), dtype=torch.float32,
                           device="cuda")
        for i, j in enumerate(rows):
            plan.execute_dm_range(dx, j, 1, spec[i])
        torch.cuda.synchronize()
        plan.query()
        spec = device_to_complex(spec, geo.K)
    x = fb.T
    chunks = (0, geo.n_chunks // 2, geo.n_chunks - 1)
    e_spec, e_spec_ac, e_time, e_time_ac = [], [], [], []
    for c in chunks:
        X = oracle.spectra(x, geo, c)  # oracle FFT of the chunk, all channels
        Y = oracle.fdd_bins(X, np.arange(geo.K), geo.L, d[rows])
        e_spec.append(rel_l2(spec[:, c], Y))
        e_spec_ac.append(rel_l2(spec[:, c, 1:], Y[:, 1:]))
        y = oracle.irfft(Y, geo.L)
        keep = min(geo.hop, geo.n_out - c * geo.hop)
        ref = y[:, :keep]
        g = got[:, c * geo.hop: c * geo.hop + keep]
        e_time.append(rel_l2(g, ref))
        e_time_ac.append(rel_l2(g - g.mean(axis=1, keepdims=True),
                                ref - ref.mean(axis=1, keepdims=True)))
    print(f"survey full size: rel-L2 vs FP64 of the dedispersed spectra {max(e_spec):.2e} "
          f"(without DC {max(e_spec_ac):.2e}); time output {max(e_time):.2e} (zero-mean "
          f"{max(e_time_ac):.2e}) over {len(rows)} trials x {len(chunks)} chunks")
    assert max(e_spec) <= FP32_REL_L2 and max(e_spec_ac) <= FP32_REL_L2
    assert max(e_time) <= FP32_REL_L2
    # The zero-mean part of the time series is ~360x smaller than the 8-bit
    # offset it rides on (per sample: 128 x 1024 channels against a noise rms
    # of 16 x sqrt(1024)); FP32 rounding in the inverse transform is relative
    # to the whole signal, ~2^-24 log2(L) per sample, so relative to the
    # zero-mean part the floor is 2^-24 x 18 x 131072 / 512 = 2.7e-4.
    floor = 2.0 ** -24 * np.log2(geo.L) * (128.0 * w.n_chan) / (16.0 * np.sqrt(w.n_chan))
    assert max(e_time_ac) <= floor


# ----------------------------------------------------------- 32 beams, tensor
def _random_spectra(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


@pytest.mark.parametrize("precision", [fdd.FDD_PREC_BF16_HILO, fdd.FDD_PREC_BF16,
                                       fdd.FDD_PREC_FP16], ids=["bf16_hilo", "bf16", "fp16"])
def test_32beam_tensor_core_bench_slice(precision):
    w = synth.WORKLOADS["fdd_32beam_1024ch_2p19t_4096dm"].scaled(n_t=4096)
    rng = np.random.default_rng(SEED + 3)
    K = w.n_t // 2 + 1
    X = _random_spectra(rng, (w.n_beams, w.n_chan, K))
    with fdd.Plan(**params_for(w, output=fdd.FDD_OUT_SPECTRA, precision=precision)) as plan:
        pitch = plan.info["bin_pitch"]
        dX = complex_to_device(X, pitch)
        dY = torch.empty((w.n_beams, w.n_dm, K, 2), dtype=torch.float32, device="cuda")
        plan.dedisperse_spectra(dX, pitch, w.n_beams, 0, w.n_dm, dY, K)
        torch.cuda.synchronize()
        plan.query()
        bins = np.array([0, 1, 2, 1024, K - 2, K - 1])
        beams = [0, 31]
        got = device_to_complex(dY[beams][:, :, torch.from_numpy(bins).cuda()], len(bins))
    d = _delays(w)
    errs = [rel_l2(got[i], oracle.fdd_bins(X[b][:, bins].astype(np.complex128), bins, w.n_t, d))
            for i, b in enumerate(beams)]
    name = {fdd.FDD_PREC_BF16_HILO: "hi+lo", fdd.FDD_PREC_BF16: "bf16",
            fdd.FDD_PREC_FP16: "fp16"}[precision]
    print(f"32 beams, tensor cores ({name}),"
          f" bench slice: rel-L2 vs FP64 {max(errs):.2e}")
    assert max(errs) <= TC_REL_L2


def _windows(K, width=8):
    return [(0, width), (K // 2 - width // 2, width), (K - width, width)]


def _tc_windows(w, precision, out_kind, beams_checked, seed):
    """Bin windows of the workload's whole transform on the tensor cores; the
    oracle recomputes beams_checked at every window bin and trial."""
    L = oracle.next_pow2(w.n_t) if w.chunk_len == 0 else w.chunk_len
    K = L // 2 + 1
    rng = np.random.default_rng(seed)
    d = _delays(w)
    errs = []
    with fdd.Plan(**params_for(w, output=fdd.FDD_OUT_SPECTRA, precision=precision)) as plan:
        assert plan.info["n_bins"] == K
        for b0, nb in _windows(K):
            X = _random_spectra(rng, (w.n_beams, w.n_chan, nb))
            dX = complex_to_device(X, nb)
            if out_kind == fdd.FDD_OUT_SPECTRA:
                dY = torch.empty((w.n_beams, w.n_dm, nb, 2), dtype=torch.float32, device="cuda")
            else:
                dY = torch.empty((w.n_beams, w.n_dm, nb), dtype=torch.float32, device="cuda")
            plan.dedisperse_spectra_bins(dX, nb, w.n_beams, b0, nb, 0, w.n_dm, dY, nb,
                                         out_kind=out_kind)
            torch.cuda.synchronize()
            plan.query()
            bins = np.arange(b0, b0 + nb)
            for b in beams_checked:
                ref = oracle.fdd_bins(X[b].astype(np.complex128), bins, L, d)
                if out_kind == fdd.FDD_OUT_SPECTRA:
                    errs.append(rel_l2(device_to_complex(dY[b], nb), ref))
                else:
                    errs.append(rel_l2(dY[b].cpu().numpy().astype(np.float64), np.abs(ref) ** 2))
    return errs


def test_32beam_tensor_core_full_transform_windows():
    w = synth.WORKLOADS["fdd_32beam_1024ch_2p19t_4096dm"]
    errs = _tc_windows(w, fdd.FDD_PREC_BF16_HILO, fdd.FDD_OUT_SPECTRA, [0, 17, 31], SEED + 4)
    print(f"32 beams, tensor cores (hi+lo), L = 2^19 windows at DC / mid / Nyquist: "
          f"rel-L2 vs FP64 {max(errs):.2e}")
    assert max(errs) <= TC_REL_L2


# ------------------------------------------------------- 96 uneven beams, batch
def test_96beam_batch_bench_configuration_sampled():
    bw = synth.BATCH_WORKLOADS["fdd_96beam_1536ch_uneven"]
    beams = bw.beams(SEED, n_t_div=16)
    common = dict(n_chan=bw.n_chan, nu_lo_mhz=bw.nu_lo_mhz, dnu_mhz=bw.dnu_mhz,
                  t_samp_s=bw.t_samp_s, in_dtype=fdd.FDD_IN_F32, chunk_len=0,
                  output=fdd.FDD_OUT_POWER, workspace_limit=64 << 30)
    n_ts = np.array([b[0] for b in beams])
    n_dms = np.array([b[3] for b in beams])
    checked = sorted({int(np.argmin(n_ts)), int(np.argmax(n_ts)), int(np.argmax(n_dms)),
                      int(np.argmin(n_dms))})
    with fdd.Batch(beams, autotune=True, **common) as batch:
        info = batch.info
        d_in = torch.empty(info["in_elems"], dtype=torch.float32, device="cuda")
        for b, desc in enumerate(beams):
            kw, _ = synth.batch_beam_args(bw, desc, SEED, b)
            off = batch.in_offsets[b]
            synth.gpu.filterbank(d_in[off: off + desc[0] * bw.n_chan], n_rows=desc[0], t0=0, **kw)
        out = torch.empty(info["out_elems"], dtype=torch.float32, device="cuda")
        batch.execute(d_in, out)
        batch.execute(d_in, out)  # graph replay
        torch.cuda.synchronize()
        offs = batch.out_offsets
        got = {}
        for b in checked:
            L = oracle.next_pow2(beams[b][0])
            K = L // 2 + 1
            got[b] = out[offs[b]: offs[b] + beams[b][3] * K].view(beams[b][3], K)
            got[b] = got[b].cpu().numpy().astype(np.float64)
    nu = bw.nu_lo_mhz + bw.dnu_mhz * np.arange(bw.n_chan)
    errs = []
    for b in checked:
        n_t, dm0, ddm, n_dm = beams[b]
        kw, _ = synth.batch_beam_args(bw, beams[b], SEED, b)
        x = philox.filterbank(n_rows=n_t, t0=0, **kw).T.astype(np.float64)
        d = oracle.delays(nu, dm0 + ddm * np.arange(n_dm), bw.t_samp_s)
        geo = oracle.geometry(n_t, 0, d)
        X = oracle.spectra(x, geo, 0)
        rng = np.random.default_rng(b)
        bins = np.unique(np.concatenate([[0, 1, geo.K - 1], rng.integers(2, geo.K - 1, 5)]))
        ref = np.abs(oracle.fdd_bins(X[:, bins], bins, geo.L, d)) ** 2
        errs.append(rel_l2(got[b][:, bins], ref))
    print(f"96 uneven beams, batching form ({fdd.MAC_VARIANT_NAMES[info['mac_variant']]}): "
          f"rel-L2 vs FP64 of |Y|^2 {max(errs):.2e} over beams {checked}")
    assert max(errs) <= 2 * FP32_REL_L2


# ------------------------------------------------- 16 beams, 4096 channels, power
def test_16beam_4096ch_tensor_core_full_transform_windows():
    w = synth.WORKLOADS["fdd_16beam_4096ch_2p21t_8192dm_power"]
    assert fdd.FDD_PREC_BF16_HILO
    errs = _tc_windows(w, fdd.FDD_PREC_BF16_HILO, fdd.FDD_OUT_POWER, [0, 9, 15], SEED + 5)
    print(f"16 beams x 4096 channels x 8192 trials, tensor cores in 16-beam groups, "
          f"L = 2^19 windows, |Y|^2: rel-L2 vs FP64 {max(errs):.2e}")
    assert max(errs) <= 2 * TC_REL_L2


def test_16beam_long_delay_chain_power_top_trials():
    w = synth.WORKLOADS["fdd_16beam_4096ch_2p21t_8192dm_power"].scaled(n_chan=64)
    d = _delays(w)
    geo = oracle.geometry(w.n_t, w.chunk_len, d)
    j0, nj = w.n_dm - 64, 64
    with fdd.Plan(**params_for(w, precision=fdd.FDD_PREC_BF16_HILO)) as plan:
        info = plan.info
        assert (info["n_chunks"], info["hop"], info["d_max"]) == (geo.n_chunks, geo.hop,
                                                                   geo.d_max)
        d_in = torch.empty((w.n_beams, w.n_t * w.n_chan), dtype=torch.float32, device="cuda")
        for b in range(w.n_beams):
            kw, _ = synth.philox_beam_args(w, SEED, b)
            synth.gpu.filterbank(d_in[b], n_rows=w.n_t, t0=0, **kw)
        out = torch.empty((w.n_beams, geo.n_chunks, nj, geo.K), dtype=torch.float32,
                          device="cuda")
        plan.execute_dm_range(d_in, j0, nj, out)
        torch.cuda.synchronize()
        plan.query()
        beams, chunks = [0, 15], [0, geo.n_chunks - 1]
        got = out[beams][:, chunks].cpu().numpy().astype(np.float64)
    errs = []
    rng = np.random.default_rng(SEED)
    for i, b in enumerate(beams):
        kw, _ = synth.philox_beam_args(w, SEED, b)
        for q, c in enumerate(chunks):
            t0 = c * geo.hop
            rows = min(geo.L, w.n_t - t0)
            x = np.zeros((w.n_chan, geo.L))
            x[:, :rows] = philox.filterbank(n_rows=rows, t0=t0, **kw).T
            X = oracle.fft_r2c(x)
            bins = np.unique(np.concatenate([[0, 1, geo.K - 1], rng.integers(2, geo.K - 1, 29)]))
            ref = np.abs(oracle.fdd_bins(X[:, bins], bins, geo.L, d[j0: j0 + nj])) ** 2
            errs.append(rel_l2(got[i, q][:, bins], ref))
    print(f"16 beams, long-delay chunks (D_max {geo.d_max}, {geo.n_chunks} chunks), tensor "
          f"cores, |Y|^2 of the top 64 trials: rel-L2 vs FP64 {max(errs):.2e}")
    assert max(errs) <= 2 * TC_REL_L2

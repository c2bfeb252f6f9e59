"""Tensor-core form (tcgen05; BF16 hi+lo, BF16, or FP16 operands with per-bin
data scaling; FP32 accumulation) against the FP64 oracle (GB300 only).

The gate is the low-precision form's relative L2 error <= 3e-3 against FP64:
BF16 rounding of the data side alone is ~2^-9 / sqrt(3) ~ 1.1e-3 per element.
Shapes span partial and several beam groups (16 beams each for calls of at
most 16 series, else 32), a ragged last channel tile (32 channels each) and
partial trial passes (2048 trials in 16-beam groups, 1024 in 32-beam groups).
"""
import numpy as np
import pytest

import oracle
import paper_2110_03482_gb300 as fdd
import synth
from gpu_util import complex_to_device, device_to_complex, params_for, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TC_REL_L2 = 3e-3


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fdd.build()


def _workload(n_chan, n_t, dms, n_beams, band=(1200.0, 1500.0), t_samp=2e-3, chunk_len=0,
              output="spectra", dtype="f32"):
    dms = np.asarray(dms, dtype=np.float64)
    ddm = float(dms[1] - dms[0]) if dms.size > 1 else 0.0
    return synth.Workload(name="tc", n_chan=n_chan, band_lo_mhz=band[0], band_hi_mhz=band[1],
                          t_samp_s=t_samp, n_t=n_t, dtype=dtype, dm0=float(dms[0]), ddm=ddm,
                          n_dm=dms.size, chunk_len=chunk_len, n_beams=n_beams, output=output,
                          pulses_per_beam=1,
                          noise_mean=128.0 if dtype == "u8" else 0.0,
                          noise_sigma=16.0 if dtype == "u8" else 1.0)


PREC_NAMES = {fdd.FDD_PREC_BF16_HILO: "hi+lo", fdd.FDD_PREC_BF16: "bf16",
              fdd.FDD_PREC_FP16: "fp16"}


def _pair_form(n_series, n_dm):
    """The plans' rule: the CTA-pair form where the calls' last pair pass
    (2048 trials with more than 16 series, else 4096) is full or more than
    half full."""
    p2 = 4096 if n_series <= 16 else 2048
    r = n_dm % p2
    return n_dm > p2 // 2 and (r == 0 or r > p2 // 2)


@pytest.mark.parametrize("precision", [fdd.FDD_PREC_BF16_HILO, fdd.FDD_PREC_BF16,
                                       fdd.FDD_PREC_FP16], ids=["bf16_hilo", "bf16", "fp16"])
@pytest.mark.parametrize("n_series,n_chan,L,dm0,ddm,n_dm", [
    (5, 40, 256, 0.0, 0.5, 2100),    # pair: partial 16-beam group, ragged channel tile,
                                     # one pass of 9 a's (the second CTA's last a padded)
    (32, 64, 128, 3.0, 1.0, 1024),   # one CTA per SM: one full group, exactly one pass
    (37, 33, 512, 0.0, 0.25, 300),   # one CTA: two groups, one partial pass
    (16, 64, 512, 1.0, 0.25, 2100),  # pair: one full 16-beam group, one pass of 9 a's
    (33, 40, 256, 0.5, 0.5, 2200),   # one CTA: 32-beam groups (one of 1 beam), 3 passes
    (40, 24, 128, 0.5, 0.5, 3300),   # pair: 32-beam groups (one of 8 beams), a full pass
                                     # and one of 5 a's
    (1, 1, 64, 0.0, 1.0, 1),         # one series, one channel, one trial
    (2, 7, 32, 5.0, 0.1, 3),         # a few of everything, non-zero first trial
])
def test_tc_kernel_matches_oracle(n_series, n_chan, L, dm0, ddm, n_dm, precision):
    dms = dm0 + ddm * np.arange(n_dm)
    w = _workload(n_chan, L, dms, n_series)
    K = L // 2 + 1
    rng = np.random.default_rng(n_series * 1000 + n_chan)
    X = (rng.standard_normal((n_series, n_chan, K)) +
         1j * rng.standard_normal((n_series, n_chan, K))).astype(np.complex64).astype(np.complex128)
    xp, yp = K + 5, K + 2
    with fdd.Plan(**params_for(w, output=fdd.FDD_OUT_SPECTRA, precision=precision)) as plan:
        assert plan.info["mac_variant"] == (fdd.FDD_MAC_TC_PAIR if _pair_form(n_series, n_dm)
                                            else fdd.FDD_MAC_TC)
        dX = complex_to_device(X, xp)
        dY = torch.zeros((n_series, n_dm, yp, 2), dtype=torch.float32, device="cuda")
        plan.dedisperse_spectra(dX, xp, n_series, 0, n_dm, dY, yp)
        dP = torch.zeros((n_series, n_dm, yp), dtype=torch.float32, device="cuda")
        plan.dedisperse_spectra(dX, xp, n_series, 0, n_dm, dP, yp, out_kind=fdd.FDD_OUT_POWER)
        torch.cuda.synchronize()
        assert plan.query()["n_bins"] == K  # also reports a device-side timeout, if any
        Y = device_to_complex(dY, K)
        P = dP.cpu().numpy()[..., :K].astype(np.float64)
        assert np.all(dY.cpu().numpy()[..., K:, :] == 0)
    d = oracle.delays(w.channel_centres(), w.dms(), w.t_samp_s)
    errs = []
    for s in range(n_series):
        ref = oracle.fdd_bins(X[s], np.arange(K), L, d)
        errs.append(rel_l2(Y[s], ref))
        assert rel_l2(P[s], np.abs(ref) ** 2) <= 2 * TC_REL_L2
    print(f"tensor-core ({PREC_NAMES[precision]}) "
          f"rel-L2 vs FP64: max over series {max(errs):.2e}")
    assert max(errs) <= TC_REL_L2


def test_tc_dm_subrange_matches_full():
    n_series, n_chan, L = 8, 48, 256
    dms = 0.5 * np.arange(2100)
    w = _workload(n_chan, L, dms, n_series)
    K = L // 2 + 1
    rng = np.random.default_rng(3)
    X = rng.standard_normal((n_series, n_chan, K)) + 1j * rng.standard_normal((n_series, n_chan, K))
    with fdd.Plan(**params_for(w, output=fdd.FDD_OUT_SPECTRA,
                               precision=fdd.FDD_PREC_BF16_HILO)) as plan:
        dX = complex_to_device(X, K)
        full = torch.zeros((n_series, 2100, K, 2), device="cuda")
        plan.dedisperse_spectra(dX, K, n_series, 0, 2100, full, K)
        part = torch.zeros((n_series, 700, K, 2), device="cuda")
        plan.dedisperse_spectra(dX, K, n_series, 1111, 700, part, K)
        torch.cuda.synchronize()
        f = device_to_complex(full, K)[:, 1111:1811]
        g = device_to_complex(part, K)
    # same phasors, different split of the trial index: equal to BF16 accuracy
    assert rel_l2(g, f) <= TC_REL_L2


@pytest.mark.parametrize("precision,dtype", [(fdd.FDD_PREC_BF16_HILO, "f32"),
                                             (fdd.FDD_PREC_FP16, "f32"),
                                             (fdd.FDD_PREC_FP16, "u8")],
                         ids=["bf16_hilo", "fp16", "fp16_u8"])
@pytest.mark.parametrize("output", ["time", "power"])
def test_tc_end_to_end(output, precision, dtype):
    """Eight beams through the whole path on the tensor-core form; with 8-bit
    input (mean 128) the FP16 form's per-bin scale must hold spectra whose DC
    bins reach ~1e5 while the rest are ~1e2-1e3."""
    w = _workload(48, 3000, 2.0 * np.arange(150), 8, t_samp=5e-4, chunk_len=1024,
                  output=output, dtype=dtype)
    fbs = np.stack([synth.filterbank(w, seed=17, beam=b)[0] for b in range(8)])
    with fdd.Plan(**params_for(w, precision=precision)) as plan:
        info = plan.info
        dx = torch.from_numpy(fbs).cuda()
        out = torch.empty(info["out_elems"], dtype=torch.float32, device="cuda")
        plan.execute(dx, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy().astype(np.float64)
    d = oracle.delays(w.channel_centres(), w.dms(), w.t_samp_s)
    geo = oracle.geometry(w.n_t, w.chunk_len, d)
    if output == "time":
        o = o.reshape(8, w.n_dm, info["out_len"])
        for b in range(8):
            ref = oracle.fdd_time(fbs[b].T.astype(np.float64), d, w.chunk_len)
            assert rel_l2(o[b], ref) <= TC_REL_L2
            # the zero-mean part too (with 8-bit data the constant dominates the above)
            zm = lambda y: y - y.mean(axis=1, keepdims=True)  # noqa: E731
            assert rel_l2(zm(o[b]), zm(ref)) <= TC_REL_L2
    else:
        o = o.reshape(8, geo.n_chunks, w.n_dm, geo.K)
        for b in range(0, 8, 3):
            x = fbs[b].T.astype(np.float64)
            for c in range(geo.n_chunks):
                ref = np.abs(oracle.fdd_bins(oracle.spectra(x, geo, c), np.arange(geo.K),
                                             geo.L, d)) ** 2
                assert rel_l2(o[b, c], ref) <= 2 * TC_REL_L2
                assert rel_l2(o[b, c][:, 1:], ref[:, 1:]) <= 2 * TC_REL_L2  # without DC


@pytest.mark.parametrize("n_series", [7, 20])
def test_tc_bin_windows_equal_the_whole_range(n_series):
    """A window of bins (absolute phases k_begin + k) gives bit for bit the
    columns of the whole-range call: every bin's products and sums are the same."""
    n_chan, L, n_dm = 40, 1024, 700
    w = _workload(n_chan, L, 0.5 * np.arange(n_dm), n_series)
    K = L // 2 + 1
    rng = np.random.default_rng(n_series)
    X = rng.standard_normal((n_series, n_chan, K)) + 1j * rng.standard_normal((n_series, n_chan, K))
    with fdd.Plan(**params_for(w, output=fdd.FDD_OUT_SPECTRA,
                               precision=fdd.FDD_PREC_BF16_HILO)) as plan:
        dX = complex_to_device(X, K)
        full = torch.zeros((n_series, n_dm, K, 2), device="cuda")
        plan.dedisperse_spectra(dX, K, n_series, 0, n_dm, full, K)
        for b0, nb in [(0, 3), (200, 57), (K - 5, 5)]:
            win = torch.zeros((n_series, n_dm, nb, 2), device="cuda")
            plan.dedisperse_spectra_bins(dX[:, :, b0:].contiguous(), K - b0, n_series, b0, nb,
                                         0, n_dm, win, nb)
            torch.cuda.synchronize()
            assert torch.equal(win, full[:, :, b0: b0 + nb]), (b0, nb)
        with pytest.raises(fdd.FddError) as e:
            plan.dedisperse_spectra_bins(dX, K, n_series, K - 2, 3, 0, n_dm, full, K)
        assert e.value.status == fdd.FDD_ERR_INVALID_ARG


FP8_REL_L2 = 0.1  # E4M3: three mantissa bits, ~2^-4 per element (reported, not the 3e-3 gate)


@pytest.mark.parametrize("n_series,n_chan,L,dm0,ddm,n_dm", [
    (32, 1024, 4096, 0.0, 0.5, 2048),  # the 32-beam tensor-core shape, 16 channel tiles of 64
    (5, 70, 256, 0.0, 0.5, 300),       # partial groups, a ragged 64-channel tile
])
def test_fp8_form_error_is_measured(n_series, n_chan, L, dm0, ddm, n_dm):
    """FP8 E4M3 phasors and data on kind::f8f6f4 (the 8-bit direction of Sect.
    5): its rel-L2 against FP64 is measured and printed; it stays below 10 %
    (the three mantissa bits give ~2^-4 per element) and above the 16-bit
    forms' gate, which it does not meet."""
    dms = dm0 + ddm * np.arange(n_dm)
    w = _workload(n_chan, L, dms, n_series, band=(1250.0, 1550.0), t_samp=0.25e-3)
    K = L // 2 + 1
    rng = np.random.default_rng(n_chan)
    X = rng.standard_normal((n_series, n_chan, K)) + 1j * rng.standard_normal((n_series, n_chan, K))
    with fdd.Plan(**params_for(w, precision=fdd.FDD_PREC_FP8)) as plan:
        dX = complex_to_device(X, plan.info["bin_pitch"])
        dY = torch.empty((n_series, n_dm, K, 2), device="cuda")
        plan.dedisperse_spectra(dX, plan.info["bin_pitch"], n_series, 0, n_dm, dY, K)
        torch.cuda.synchronize()
        plan.query()
    Y = device_to_complex(dY, K)
    bins = np.unique(np.concatenate([[0, 1, K - 1], rng.integers(2, K - 1, 5)]))
    d = oracle.delays(w.channel_centres(), dms, w.t_samp_s)
    errs = []
    for b in range(min(n_series, 3)):
        ref = oracle.fdd_bins(X[b][:, bins], bins, L, d)
        errs.append(rel_l2(Y[b][:, bins], ref))
    err = float(np.sqrt(np.mean(np.square(errs))))
    print(f"FP8 E4M3 form: rel-L2 vs FP64 {err:.3e}")
    assert TC_REL_L2 < err <= FP8_REL_L2

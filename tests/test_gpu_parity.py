"""CUDA path against the FP64 oracle, element by element (GB300 only).

Kernel-only cases feed the same seeded spectra to ``fdd_dedisperse_spectra``
and to ``oracle.fdd_bins``; end-to-end cases run ``fdd_execute`` on seeded
filterbanks and compare with ``oracle.fdd_time`` / the oracle spectra.  Sizes
span several kernel tiles with ragged tails in bins and trials.  The gate is
the FP32 form's relative L2 error <= 1e-5 against FP64.
"""
import numpy as np
import pytest

import oracle
import paper_2110_03482_gb300 as fdd
import synth
from gpu_util import FP32_REL_L2, complex_to_device, device_to_complex, params_for, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fdd.build()


def _small_workload(n_chan, n_t, dms, band=(1200.0, 1500.0), t_samp=1e-3, dtype="f32",
                    chunk_len=0, n_beams=1, output="time"):
    dms = np.asarray(dms, dtype=np.float64)
    ddm = float(dms[1] - dms[0]) if dms.size > 1 else 0.0
    return synth.Workload(name="test", n_chan=n_chan, band_lo_mhz=band[0], band_hi_mhz=band[1],
                          t_samp_s=t_samp, n_t=n_t, dtype=dtype, dm0=float(dms[0]), ddm=ddm,
                          n_dm=dms.size, chunk_len=chunk_len, n_beams=n_beams, output=output,
                          pulses_per_beam=2,
                          noise_mean=128.0 if dtype == "u8" else 0.0,
                          noise_sigma=16.0 if dtype == "u8" else 1.0)


def _oracle_delays(w):
    return oracle.delays(w.channel_centres(), w.dms(), w.t_samp_s)


# ----------------------------------------------------------------- kernel only
_REF_CACHE = {}

KERNEL_CASES = [
    # n_chan, L, dm0, ddm, n_dm, n_series   (tile variant exercised)
    (37, 1024, 0.0, 1.0, 130, 1),     # 128-trial tile: 2 blocks, ragged; 513 bins ragged
    (64, 2048, 3.0, 0.5, 700, 2),     # 1024-trial tile, DM0 != 0, two series
    (16, 4096, 0.0, 0.25, 2100, 1),   # 2048-trial tile plus a ragged block
    (12, 1024, 1.0, 0.3, 3500, 1),    # ragged 2048-trial block of more than 1024 trials
    (5, 64, 7.0, 0.0, 1, 1),          # one trial
    (1, 128, 0.0, 2.0, 3, 3),         # one channel
]


@pytest.mark.parametrize("variant", [0] + [v + 1 for v in range(fdd.FDD_MAC_VARIANTS)],
                         ids=["auto"] + fdd.MAC_VARIANT_NAMES)
@pytest.mark.parametrize("n_chan,L,dm0,ddm,n_dm,n_series", KERNEL_CASES)
def test_kernel_matches_oracle(n_chan, L, dm0, ddm, n_dm, n_series, variant):
    dms = dm0 + ddm * np.arange(n_dm)
    w = _small_workload(n_chan, L, dms, t_samp=2e-3)
    rng = np.random.default_rng(1000 + n_chan + n_dm)
    K = L // 2 + 1
    X = rng.standard_normal((n_series, n_chan, K)) + 1j * rng.standard_normal((n_series, n_chan, K))
    X = X.astype(np.complex64).astype(np.complex128)
    xp, yp = K + 3, K + 5
    with fdd.Plan(**params_for(w, output=fdd.FDD_OUT_SPECTRA, mac_variant=variant)) as plan:
        assert plan.info["fft_len"] == L and plan.info["n_bins"] == K
        dX = complex_to_device(X, xp)
        dY = torch.zeros((n_series, n_dm, yp, 2), dtype=torch.float32, device="cuda")
        plan.dedisperse_spectra(dX, xp, n_series, 0, n_dm, dY, yp)
        dP = torch.zeros((n_series, n_dm, yp), dtype=torch.float32, device="cuda")
        plan.dedisperse_spectra(dX, xp, n_series, 0, n_dm, dP, yp, out_kind=fdd.FDD_OUT_POWER)
        torch.cuda.synchronize()
        Y = device_to_complex(dY, K)
        P = dP.cpu().numpy()[..., :K].astype(np.float64)
        assert np.all(dY.cpu().numpy()[..., K:, :] == 0)  # pitch padding untouched
    key = (n_chan, L, dm0, ddm, n_dm, n_series)
    if key not in _REF_CACHE:
        d = _oracle_delays(w)
        _REF_CACHE[key] = [oracle.fdd_bins(X[s], np.arange(K), L, d) for s in range(n_series)]
    for s in range(n_series):
        ref = _REF_CACHE[key][s]
        err = rel_l2(Y[s], ref)
        assert err <= FP32_REL_L2, err
        assert rel_l2(P[s], np.abs(ref) ** 2) <= 2 * FP32_REL_L2


def test_kernel_g12_two_stage_ring():
    """6000 channels: the G12 tile's phase table leaves room for two ring
    stages only; full blocks, a wide last block and the oracle agree."""
    n_chan, L, n_dm = 6000, 64, 2048 + 600
    dms = 0.25 * np.arange(n_dm)
    w = _small_workload(n_chan, L, dms, t_samp=2e-3)
    rng = np.random.default_rng(61)
    K = L // 2 + 1
    X = rng.standard_normal((1, n_chan, K)) + 1j * rng.standard_normal((1, n_chan, K))
    X = X.astype(np.complex64).astype(np.complex128)
    with fdd.Plan(**params_for(w, output=fdd.FDD_OUT_SPECTRA)) as plan:
        assert plan.info["mac_variant"] == fdd.FDD_MAC_G12_4X8
        dX = complex_to_device(X, K)
        dY = torch.zeros((1, n_dm, K, 2), dtype=torch.float32, device="cuda")
        plan.dedisperse_spectra(dX, K, 1, 0, n_dm, dY, K)
        torch.cuda.synchronize()
        Y = device_to_complex(dY, K)
    ref = oracle.fdd_bins(X[0], np.arange(K), L, _oracle_delays(w))
    assert rel_l2(Y[0], ref) <= FP32_REL_L2


def test_kernel_dm_subrange_and_large_phases():
    """Survey-like phases (L = 2^18, trials 0..1023.5 at 64 us): sampled bins up
    to Nyquist, the full list and a sub-range starting mid-block."""
    n_chan, L = 64, 1 << 18
    dms = 0.5 * np.arange(2048)
    w = _small_workload(n_chan, L, dms, band=(1210.0, 1520.0), t_samp=64e-6)
    K = L // 2 + 1
    rng = np.random.default_rng(7)
    X = (rng.standard_normal((n_chan, K)) + 1j * rng.standard_normal((n_chan, K))).astype(
        np.complex64).astype(np.complex128)
    bins = np.unique(np.concatenate([[0, 1, 2, 1000, K // 2, K - 2, K - 1],
                                     rng.integers(0, K, 57)]))
    d = _oracle_delays(w)
    ref = oracle.fdd_bins(X[:, bins], bins, L, d)
    with fdd.Plan(**params_for(w, output=fdd.FDD_OUT_SPECTRA)) as plan:
        dX = complex_to_device(X, plan.info["bin_pitch"])
        dY = torch.empty((2048, K, 2), dtype=torch.float32, device="cuda")
        plan.dedisperse_spectra(dX, plan.info["bin_pitch"], 1, 0, 2048, dY, K)
        sub0, subn = 333, 1200
        dS = torch.empty((subn, K, 2), dtype=torch.float32, device="cuda")
        plan.dedisperse_spectra(dX, plan.info["bin_pitch"], 1, sub0, subn, dS, K)
        torch.cuda.synchronize()
        bt = torch.from_numpy(bins).cuda()
        Y = dY.index_select(1, bt).cpu().numpy()
        Y = Y[..., 0].astype(np.float64) + 1j * Y[..., 1]
        S = dS.index_select(1, bt).cpu().numpy()
        S = S[..., 0].astype(np.float64) + 1j * S[..., 1]
    assert rel_l2(Y, ref) <= FP32_REL_L2
    assert rel_l2(S, ref[sub0: sub0 + subn]) <= FP32_REL_L2
    for q in range(len(bins)):  # per-bin error too, Nyquist included
        assert rel_l2(Y[:, q], ref[:, q]) <= 4 * FP32_REL_L2, bins[q]


@pytest.mark.parametrize("variant", [0, fdd.FDD_MAC_Q_4X4 + 1, fdd.FDD_MAC_Q12_8X8 + 1,
                                     fdd.FDD_MAC_G12_4X8 + 1, fdd.FDD_MAC_Q_8X8_512 + 1])
def test_kernel_bin_windows_equal_the_whole_range(variant):
    """A window of bins (absolute phases k_begin + k) gives bit for bit the
    columns of the whole-range call, for the default and four other tiles."""
    n_chan, L, n_dm = 48, 4096, 1100
    w = _small_workload(n_chan, L, 0.5 * np.arange(n_dm))
    K = L // 2 + 1
    rng = np.random.default_rng(17)
    X = rng.standard_normal((2, n_chan, K)) + 1j * rng.standard_normal((2, n_chan, K))
    with fdd.Plan(**params_for(w, output=fdd.FDD_OUT_SPECTRA, mac_variant=variant)) as plan:
        dX = complex_to_device(X, K)
        full = torch.zeros((2, n_dm, K, 2), device="cuda")
        plan.dedisperse_spectra(dX, K, 2, 0, n_dm, full, K)
        for b0, nb in [(0, 1), (1, 100), (777, 333), (K - 13, 13)]:
            win = torch.zeros((2, n_dm, nb, 2), device="cuda")
            xw = dX[:, :, b0: b0 + nb].contiguous()
            plan.dedisperse_spectra_bins(xw, nb, 2, b0, nb, 0, n_dm, win, nb)
            torch.cuda.synchronize()
            assert torch.equal(win, full[:, :, b0: b0 + nb]), (b0, nb)
        with pytest.raises(fdd.FddError) as e:
            plan.dedisperse_spectra_bins(dX, K, 2, -1, 4, 0, n_dm, full, K)
        assert e.value.status == fdd.FDD_ERR_INVALID_ARG


# ----------------------------------------------------------------- end to end
def _run_execute(w, x_host, output, **kw):
    with fdd.Plan(**params_for(w, output=output, **kw)) as plan:
        info = plan.info
        dx = torch.from_numpy(np.ascontiguousarray(x_host)).cuda()
        if output == fdd.FDD_OUT_SPECTRA:
            out = torch.empty((info["out_elems"], 2), dtype=torch.float32, device="cuda")
        else:
            out = torch.empty((info["out_elems"],), dtype=torch.float32, device="cuda")
        plan.execute(dx, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        if output == fdd.FDD_OUT_SPECTRA:
            o = o[:, 0].astype(np.float64) + 1j * o[:, 1]
        return o, info


def test_end_to_end_64ch_time_output_and_pulse():
    w = synth.WORKLOADS["fdd_64ch_4096t_128dm"]
    fb, pulses = synth.filterbank(w, seed=20211008)
    y, info = _run_execute(w, fb, fdd.FDD_OUT_TIME)
    y = y.reshape(w.n_dm, info["out_len"])
    ref = oracle.fdd_time(fb.T.astype(np.float64), _oracle_delays(w), w.chunk_len)
    assert rel_l2(y, ref) <= FP32_REL_L2
    j, n = np.unravel_index(np.argmax(y), y.shape)
    assert j == 57 and 998 <= n <= 1004


def test_end_to_end_64ch_spectra_and_power():
    w = synth.WORKLOADS["fdd_64ch_4096t_128dm"]
    fb, _ = synth.filterbank(w, seed=5)
    d = _oracle_delays(w)
    geo = oracle.geometry(w.n_t, w.chunk_len, d)
    Xo = oracle.spectra(fb.T.astype(np.float64), geo, 0)
    ref = oracle.fdd_bins(Xo, np.arange(geo.K), geo.L, d)
    Y, info = _run_execute(w, fb, fdd.FDD_OUT_SPECTRA)
    Y = Y.reshape(w.n_dm, info["n_bins"])
    assert rel_l2(Y, ref) <= FP32_REL_L2
    assert rel_l2(Y[:, 1:], ref[:, 1:]) <= FP32_REL_L2
    P, _ = _run_execute(w, fb, fdd.FDD_OUT_POWER)
    assert rel_l2(P.reshape(w.n_dm, -1), np.abs(ref) ** 2) <= 2 * FP32_REL_L2


@pytest.mark.parametrize("layout", [fdd.FDD_LAYOUT_TIME_MAJOR, fdd.FDD_LAYOUT_CHAN_MAJOR])
def test_end_to_end_chunked_u8(layout):
    """Overlap-save chunks with a ragged last chunk, 8-bit input."""
    w = _small_workload(48, 5000, np.arange(100, dtype=float), band=(400.0, 500.0), t_samp=1e-3,
                        dtype="u8", chunk_len=2048)
    fb, _ = synth.filterbank(w, seed=11)
    x_in = fb if layout == fdd.FDD_LAYOUT_TIME_MAJOR else np.ascontiguousarray(fb.T)
    y, info = _run_execute(w, x_in, fdd.FDD_OUT_TIME, in_layout=layout)
    d = _oracle_delays(w)
    geo = oracle.geometry(w.n_t, w.chunk_len, d)
    assert info["n_chunks"] == geo.n_chunks >= 3 and info["out_len"] == geo.n_out
    y = y.reshape(w.n_dm, geo.n_out)
    ref = oracle.fdd_time(fb.T.astype(np.float64), d, w.chunk_len)
    assert rel_l2(y, ref) <= FP32_REL_L2
    # the zero-mean part as well, so the 8-bit offset does not hide errors
    assert rel_l2(y - y.mean(axis=1, keepdims=True),
                  ref - ref.mean(axis=1, keepdims=True)) <= 4 * FP32_REL_L2


@pytest.mark.parametrize("f,chunk_len,n_t,dtype,precision", [
    (2, 2048, 5000, "u8", fdd.FDD_PREC_FP32),
    (4, 2048, 5000, "u8", fdd.FDD_PREC_FP32),
    (4, 0, 4001, "f32", fdd.FDD_PREC_FP32),    # whole series, n_t not a multiple of f
    (2, 2048, 5000, "f32", fdd.FDD_PREC_BF16_HILO),
])
def test_downsampled_inverse_matches_oracle(f, chunk_len, n_t, dtype, precision):
    """Down-sampling by a shorter inverse transform (Sect. 2.2, last paragraph):
    only bins k <= L/(2f) are dedispersed and inverted with length L/f."""
    w = _small_workload(48, n_t, 1.5 * np.arange(70), band=(400.0, 500.0), t_samp=1e-3,
                        dtype=dtype, chunk_len=chunk_len)
    fb, _ = synth.filterbank(w, seed=13)
    y, info = _run_execute(w, fb, fdd.FDD_OUT_TIME, downsample=f, precision=precision)
    d = _oracle_delays(w)
    ref = oracle.fdd_time_downsampled(fb.T.astype(np.float64), d, chunk_len, f)
    assert info["downsample"] == f and info["out_len"] == ref.shape[1]
    y = y.reshape(w.n_dm, -1)
    tol = FP32_REL_L2 if precision == fdd.FDD_PREC_FP32 else 3e-3
    assert rel_l2(y, ref) <= tol
    assert rel_l2(y - y.mean(axis=1, keepdims=True), ref - ref.mean(axis=1, keepdims=True)) <= 4 * tol


def test_end_to_end_beams_and_dm_range():
    w = _small_workload(32, 3000, 2.0 * np.arange(40), t_samp=5e-4, n_beams=3, chunk_len=1024)
    fbs = np.stack([synth.filterbank(w, seed=3, beam=b)[0] for b in range(3)])
    y, info = _run_execute(w, fbs, fdd.FDD_OUT_TIME)
    y = y.reshape(3, w.n_dm, info["out_len"])
    d = _oracle_delays(w)
    for b in range(3):
        ref = oracle.fdd_time(fbs[b].T.astype(np.float64), d, w.chunk_len)
        assert rel_l2(y[b], ref) <= FP32_REL_L2
    with fdd.Plan(**params_for(w)) as plan:
        dx = torch.from_numpy(fbs).cuda()
        out = torch.empty((3, 15, info["out_len"]), dtype=torch.float32, device="cuda")
        plan.execute_dm_range(dx, 17, 15, out)
        torch.cuda.synchronize()
        part = out.cpu().numpy()
    assert rel_l2(part, y[:, 17:32]) <= FP32_REL_L2


def test_dm_zero_is_channel_sum_on_gpu():
    w = _small_workload(24, 2048, [0.0], t_samp=1e-3)
    fb, _ = synth.filterbank(w, seed=9)
    y, info = _run_execute(w, fb, fdd.FDD_OUT_TIME)
    ref = fb.astype(np.float64).sum(axis=1)
    assert rel_l2(y, ref) <= FP32_REL_L2


def test_single_channel_is_pure_shift():
    """One channel, integer delays: the output is the circularly advanced input."""
    n_t = 1024
    # choose t_samp so that the delay per unit DM is exactly 4 samples
    nu_lo, nu_ref = 1000.0, 1500.0
    rate = oracle.K_DM_PAPER * (nu_lo ** -2 - nu_ref ** -2)
    w = _small_workload(1, n_t, [0.0, 1.0, 2.0, 3.0], band=(nu_lo - 1, nu_lo + 1),
                        t_samp=rate / 4.0)
    x = np.random.default_rng(4).standard_normal((n_t, 1)).astype(np.float32)
    y, info = _run_execute(w, x, fdd.FDD_OUT_TIME, nu_ref_mhz=nu_ref)
    y = y.reshape(4, n_t)
    for j in range(4):
        assert np.max(np.abs(y[j] - np.roll(x[:, 0], -4 * j))) < 1e-5


def test_invalid_calls_do_not_launch():
    w = synth.WORKLOADS["fdd_64ch_4096t_128dm"]
    with fdd.Plan(**params_for(w)) as plan:
        dx = torch.zeros(w.n_t * w.n_chan, dtype=torch.float32, device="cuda")
        with pytest.raises(fdd.FddError) as e:
            plan.execute_dm_range(dx, 120, 20, dx)
        assert e.value.status == fdd.FDD_ERR_INVALID_ARG
        with pytest.raises(fdd.FddError):
            plan.execute(0, dx)
        with pytest.raises(fdd.FddError):
            plan.dedisperse_spectra(dx, 10, 1, 0, 1, dx, 4096)
        assert plan.query()["n_bins"] == 2049

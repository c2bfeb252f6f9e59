"""Brute-force time-domain dedispersion on the GPU (Eq. 2; fdd_tdd_execute)
against the oracle's shift-and-sum (GB300 only).

Shifts are the Eq. 1 delays rounded to the nearest sample; the tests check
that no delay of their configurations sits within 1e-6 of a half sample, so
the oracle's rounding and the plan's (both FP64) agree.  8-bit inputs make
every sum an exact integer in FP32: those cases are compared bit for bit.
"""
import numpy as np
import pytest

import oracle
import paper_2110_03482_gb300 as fdd
import synth
from gpu_util import params_for, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fdd.build()


def _workload(n_chan, n_t, dms, dtype="u8", n_beams=1, band=(400.0, 500.0), t_samp=1e-3):
    dms = np.asarray(dms, dtype=np.float64)
    return synth.Workload(name="tdd", n_chan=n_chan, band_lo_mhz=band[0], band_hi_mhz=band[1],
                          t_samp_s=t_samp, n_t=n_t, dtype=dtype, dm0=float(dms[0]),
                          ddm=float(dms[1] - dms[0]) if dms.size > 1 else 0.0, n_dm=dms.size,
                          chunk_len=0, n_beams=n_beams, output="time", pulses_per_beam=2,
                          noise_mean=128.0 if dtype == "u8" else 0.0,
                          noise_sigma=16.0 if dtype == "u8" else 1.0)


def _shifts(w, dms):
    d = oracle.delays(w.channel_centres(), dms, w.t_samp_s)
    frac = d - np.floor(d)
    assert np.min(np.abs(frac - 0.5)) > 1e-6, "a delay sits on a half-sample tie"
    return np.floor(d + 0.5).astype(np.int64), d


def _run(w, dms, x, layout=fdd.FDD_LAYOUT_TIME_MAJOR):
    with fdd.Plan(**params_for(w, dm_list=np.asarray(dms, dtype=np.float64),
                               in_layout=layout)) as plan:
        info = plan.info
        out_len = w.n_t - info["d_max"]
        y = torch.full((w.n_beams, len(dms), out_len), float("nan"), device="cuda")
        plan.tdd_execute(torch.from_numpy(np.ascontiguousarray(x)).cuda(), y)
        torch.cuda.synchronize()
        plan.query()
        return y.cpu().numpy(), info


@pytest.mark.parametrize("n_chan,n_t,dms,layout", [
    (40, 3001, 0.7 * np.arange(77), fdd.FDD_LAYOUT_TIME_MAJOR),      # ragged trials and samples
    (8, 1000, [0.0, 3.3, 3.31, 50.0, 51.7], fdd.FDD_LAYOUT_CHAN_MAJOR),  # non-uniform list
    (67, 2500, 1.3 * np.arange(33), fdd.FDD_LAYOUT_CHAN_MAJOR),      # n_chan not a multiple of 8
])
def test_tdd_u8_bit_exact(n_chan, n_t, dms, layout):
    dms = np.asarray(dms, dtype=np.float64)
    w = _workload(n_chan, n_t, dms, n_beams=2)
    fbs = np.stack([synth.filterbank(w, seed=31, beam=b)[0] for b in range(2)])
    x = fbs if layout == fdd.FDD_LAYOUT_TIME_MAJOR else np.ascontiguousarray(fbs.transpose(0, 2, 1))
    y, info = _run(w, dms, x, layout)
    s, d = _shifts(w, dms)
    assert info["d_max"] == int(np.ceil(d.max()))
    for b in range(2):
        ref = oracle.tdd(fbs[b].T.astype(np.float64), s, circular=False, n_out=y.shape[2])
        assert np.array_equal(y[b], ref.astype(np.float32)), b


def test_fourier_calls_refuse_a_non_uniform_list():
    dms = np.array([0.0, 1.0, 3.0])
    w = _workload(16, 2048, dms, dtype="f32")
    with fdd.Plan(**params_for(w, dm_list=dms)) as plan:
        assert plan.info["dm_uniform"] == 0
        dx = torch.zeros(w.n_t * w.n_chan, device="cuda")
        out = torch.empty(plan.info["out_elems"], device="cuda")
        with pytest.raises(fdd.FddError) as e:
            plan.execute(dx, out)
        assert e.value.status == fdd.FDD_ERR_UNSUPPORTED
        y = torch.empty((3, w.n_t - plan.info["d_max"]), device="cuda")
        plan.tdd_execute(dx, y)  # the time-domain path takes it
        torch.cuda.synchronize()
        assert torch.all(y == 0)


def test_tdd_f32_and_dm_zero_is_channel_sum():
    dms = np.concatenate([[0.0], 0.45 + 0.9 * np.arange(40)])
    w = _workload(24, 4096, dms, dtype="f32")
    fb, _ = synth.filterbank(w, seed=8)
    y, _ = _run(w, dms, fb)
    s, _ = _shifts(w, dms)
    ref = oracle.tdd(fb.T.astype(np.float64), s, circular=False, n_out=y.shape[2])
    assert rel_l2(y[0], ref) <= 1e-6
    assert rel_l2(y[0][0], fb.astype(np.float64).sum(axis=1)[: y.shape[2]]) <= 1e-6


def test_tdd_pulse_peaks_at_its_trial():
    w = synth.WORKLOADS["fdd_64ch_4096t_128dm"]
    fb, pulses = synth.filterbank(w, seed=20211008)
    dms = w.dms()
    y, _ = _run(w, dms, fb)
    j, n = np.unravel_index(np.argmax(y[0]), y[0].shape)
    assert j == 57 and 998 <= n <= 1004


def test_tdd_equals_fdd_for_integer_delays():
    """With every delay an integer number of samples the two methods compute
    the same valid samples (the oracle's FDD-equals-TDD pin, here between the
    two GPU paths).  Two channels, the top one at the reference frequency: the
    lower one's delay is exactly 16 samples per unit DM."""
    nu = np.array([300.0, 500.0])
    t_samp = oracle.K_DM_PAPER * (nu[0] ** -2 - nu[1] ** -2) / 16.0
    n_t = 4096
    w = synth.Workload(name="int", n_chan=2, band_lo_mhz=200.0, band_hi_mhz=600.0,
                       t_samp_s=t_samp, n_t=n_t, dtype="f32", dm0=0.0, ddm=1.0, n_dm=8,
                       chunk_len=0, output="time")
    assert np.allclose(w.channel_centres(), nu)
    d = oracle.delays(nu, np.arange(8.0), t_samp)
    assert np.allclose(d, 16.0 * np.arange(8.0)[:, None] * [1, 0], atol=1e-9)
    x = np.random.default_rng(2).standard_normal((n_t, 2)).astype(np.float32)
    with fdd.Plan(**params_for(w)) as plan:
        info = plan.info
        dmax = info["d_max"]  # 112, or 113 when 16 * 7 rounds a hair above 112
        assert dmax in (112, 113)
        n_out = n_t - dmax
        dx = torch.from_numpy(x).cuda()
        t = torch.empty((8, n_out), device="cuda")
        plan.tdd_execute(dx, t)
        f = torch.empty(info["out_elems"], device="cuda")
        plan.execute(dx, f)
        torch.cuda.synchronize()
        t, f = t.cpu().numpy(), f.cpu().numpy().reshape(8, n_t)[:, :n_out]
    ref = np.stack([x[16 * j: 16 * j + n_out, 0] + x[:n_out, 1] for j in range(8)])
    assert np.array_equal(t, ref.astype(np.float32))  # two-term sums are exact
    assert rel_l2(f, ref) <= 1e-5

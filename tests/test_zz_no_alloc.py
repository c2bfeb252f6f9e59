"""The allocation-free phase-rotate-and-sum entry point (GB300 only).

fdd_dedisperse_spectra_static serves callers that cannot allocate device
memory (their framework owns the GPU's memory, or they run a real-time loop
that forbids allocation): it takes the plan parameters directly and keeps its
phase table in a static device array that every call rewrites.  Here two
calls with different channel counts, DM grids and inputs are queued back to
back on one stream with no synchronisation between them (so the second call
rewrites the shared table right after the first call's kernel), and each
result must equal the planned entry point fdd_dedisperse_spectra bit for bit
and the FP64 oracle on sampled bins at the FP32 tolerance.  A repeat of both
calls, after their one-time set-up, must leave the device's free memory
unchanged.  This file is collected last, so a failure here comes after every
other test.
"""
import numpy as np
import pytest

import oracle
import paper_2110_03482_gb300 as fdd
from gpu_util import FP32_REL_L2, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

T_SAMP = 1e-3


def _params(n_chan, L, dms, lo=1200.0, hi=1500.0):
    dnu = (hi - lo) / n_chan
    return dict(n_chan=n_chan, nu_lo_mhz=lo + 0.5 * dnu, dnu_mhz=dnu, t_samp_s=T_SAMP, n_t=L,
                dm_list=np.asarray(dms, dtype=np.float64), chunk_len=0, in_dtype=fdd.FDD_IN_F32,
                output=fdd.FDD_OUT_SPECTRA)


# (channels, transform length, trial DMs, seed): a 1024-trial tile and the
# warp-specialised 2048-trial tile
CASES = [
    (48, 2048, 2.0 + 0.5 * np.arange(700), 11),
    (96, 4096, 0.25 * np.arange(2100), 12),
]
N_SERIES = 2


def _inputs():
    out = []
    for n_chan, L, dms, seed in CASES:
        K = L // 2 + 1
        pitch = K + 7
        g = torch.Generator(device="cuda").manual_seed(seed)
        X = torch.randn((N_SERIES, n_chan, pitch, 2), device="cuda", generator=g)
        Y = torch.full((N_SERIES, dms.size, K, 2), float("nan"), device="cuda")
        out.append((fdd.Params(**_params(n_chan, L, dms)), X, pitch, Y, K))
    return out


def _queue_static(cases, stream):
    for p, X, pitch, Y, K in cases:
        fdd.fdd_dedisperse_spectra_static(p, X, pitch, N_SERIES, 0, p.c.n_dm, Y, K, stream=stream)


def test_static_entry_matches_planned_entry_and_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fdd.build()
    cases = _inputs()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())  # inputs made on the default stream
    with torch.cuda.stream(stream):
        _queue_static(cases, stream)  # both calls queued, no sync between them
    stream.synchronize()
    rng = np.random.default_rng(5)
    for (n_chan, L, dms, _), (p, X, pitch, Y_static, K) in zip(CASES, cases):
        with fdd.Plan(**_params(n_chan, L, dms)) as plan:
            Y_plan = torch.zeros_like(Y_static)
            plan.dedisperse_spectra(X, pitch, N_SERIES, 0, dms.size, Y_plan, K)
            torch.cuda.synchronize()
        assert torch.equal(Y_static, Y_plan), "static call differs from the planned call"
        # the FP64 oracle on sampled bins (DC, 1, Nyquist and five more)
        bins = np.unique(np.concatenate([[0, 1, K - 1], rng.integers(2, K - 1, 5)]))
        xs = X.cpu().numpy().astype(np.float64)
        ys = Y_static.cpu().numpy().astype(np.float64)
        nu = oracle.channel_centres(n_chan, p.c.nu_lo_mhz, p.c.dnu_mhz)
        d = oracle.delays(nu, dms, T_SAMP)
        for s in range(N_SERIES):
            Xs = xs[s, :, bins, 0].T + 1j * xs[s, :, bins, 1].T  # [chan][bin]
            ref = oracle.fdd_bins(Xs, bins, L, d)
            got = ys[s][:, bins, 0] + 1j * ys[s][:, bins, 1]
            assert rel_l2(got, ref) <= FP32_REL_L2


def test_static_entry_allocates_nothing():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fdd.build()
    cases = _inputs()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    _queue_static(cases, stream)  # one-time set-up: table address, kernel loading
    stream.synchronize()
    expected = [c[3].clone() for c in cases]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    _queue_static(cases, stream)
    stream.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
    for c, e in zip(cases, expected):
        assert torch.equal(c[3], e)


def test_static_entry_rejects_oversized_tables():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = fdd.Params(**_params(fdd.FDD_STATIC_MAX_CHAN + 1, 64, [0.0, 1.0]))
    X = torch.zeros((1, 4), device="cuda")
    with pytest.raises(fdd.FddError) as e:
        fdd.fdd_dedisperse_spectra_static(p, X, 33, 1, 0, 2, X, 33)
    assert e.value.status == fdd.FDD_ERR_INVALID_ARG
    assert "FDD_STATIC_MAX_CHAN" in fdd.fdd_last_error()

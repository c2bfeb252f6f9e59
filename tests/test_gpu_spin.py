"""Spin-frequency-dependent DM grids on the tensor cores (Sect. 2.3, Eqs. 8
and 9) against the FP64 oracle's restatement of the same approximation
(GB300 only): groups of 16 and 32 bins, DM_0 = 0 and DM_0 > 0 (a scaled grid
reaching below DM_0), bins below the first group (Eq. 7 exactly, FP32
kernels), the partial group at the top of the band, spectra, power and time
output.  The gate is the tensor-core tolerance against the oracle's
approximation; the approximation's own distance from Eq. 7 is printed."""
import numpy as np
import pytest

import oracle
import paper_2110_03482_gb300 as fdd
import synth
from gpu_util import complex_to_device, params_for, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TC_REL_L2 = 3e-3


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fdd.build()


def _workload(n_chan, L, dm0, ddm, n_dm, output="spectra"):
    return synth.Workload(name="spin", n_chan=n_chan, band_lo_mhz=1200.0, band_hi_mhz=1500.0,
                          t_samp_s=1e-3, n_t=L, dtype="f32", dm0=dm0, ddm=ddm, n_dm=n_dm,
                          chunk_len=0, output=output, pulses_per_beam=1)


@pytest.mark.parametrize("precision", [fdd.FDD_PREC_FP16, fdd.FDD_PREC_BF16],
                         ids=["fp16", "bf16"])
@pytest.mark.parametrize("G,eps,n_chan,L,dm0,ddm,n_dm", [
    (16, 0.02, 40, 4096, 0.0, 0.1, 300),     # k_min 750, partial top group
    (32, 0.05, 33, 8192, 2.0, 0.05, 1100),   # DM_0 > 0: scaled grid below DM_0
    (16, 0.5, 8, 1024, 0.0, 0.2, 64),        # nearly every bin grouped
])
def test_spin_spectra_match_oracle(precision, G, eps, n_chan, L, dm0, ddm, n_dm):
    w = _workload(n_chan, L, dm0, ddm, n_dm)
    K = L // 2 + 1
    rng = np.random.default_rng(G + n_chan)
    X = rng.standard_normal((n_chan, K)) + 1j * rng.standard_normal((n_chan, K))
    with fdd.Plan(**params_for(w, precision=precision, spin_group=G, spin_tol=eps)) as plan:
        info = plan.info
        sg = oracle.spin_groups(K, dm0, ddm, n_dm, G, eps)
        assert (info["spin_k_min"], info["spin_j_lo"], info["spin_n_s"]) == \
            (sg.k_min, sg.j_lo, sg.n_s)
        dX = complex_to_device(X[None], info["bin_pitch"])
        dY = torch.empty((1, n_dm, K, 2), device="cuda")
        plan.dedisperse_spectra(dX, info["bin_pitch"], 1, 0, n_dm, dY, K)
        P = torch.empty((1, n_dm, K), device="cuda")
        plan.dedisperse_spectra(dX, info["bin_pitch"], 1, 0, n_dm, P, K,
                                out_kind=fdd.FDD_OUT_POWER)
        torch.cuda.synchronize()
        plan.query()
    got = dY.cpu().numpy().astype(np.float64)[0]
    got = got[..., 0] + 1j * got[..., 1]
    bins = np.unique(np.concatenate([[0, 1, sg.k_min - 1, sg.k_min, sg.k_min + G - 1,
                                      sg.k_min + G, K - 2, K - 1],
                                     rng.integers(1, K - 1, 24)]))
    bins = bins[(bins >= 0) & (bins < K)]
    nu = w.channel_centres()
    ref = oracle.fdd_bins_spin(X[:, bins], bins, L, nu, dm0, ddm, n_dm, w.t_samp_s, G, eps)
    err = rel_l2(got[:, bins], ref)
    assert err <= TC_REL_L2, err
    exact = oracle.fdd_bins(X[:, bins], bins, L,
                            oracle.delays(nu, dm0 + ddm * np.arange(n_dm), w.t_samp_s))
    print(f"spin G={G} eps={eps}: GPU vs approximation {err:.2e}; approximation vs "
          f"Eq. 7 {rel_l2(ref, exact):.2e}")
    for q, k in enumerate(bins):  # per bin too: each group's interpolation
        assert rel_l2(got[:, k], ref[:, q]) <= 4 * TC_REL_L2, k
    pw = P.cpu().numpy().astype(np.float64)[0]
    assert rel_l2(pw[:, bins], np.abs(got[:, bins]) ** 2) <= 1e-6


def test_spin_time_output_matches_oracle():
    """Whole path, time output, one series: the inverse transform of the
    approximation's spectra (oracle: spectra by its FFT, the approximation,
    its inverse)."""
    n_chan, L, n_dm, G, eps = 32, 4096, 160, 16, 0.02
    w = _workload(n_chan, L, 0.0, 0.25, n_dm, output="time")
    fb, _ = synth.filterbank(w, seed=3)
    with fdd.Plan(**params_for(w, precision=fdd.FDD_PREC_FP16, spin_group=G,
                               spin_tol=eps)) as plan:
        d_out = torch.empty(plan.info["out_elems"], device="cuda")
        plan.execute(torch.from_numpy(fb).cuda(), d_out)
        torch.cuda.synchronize()
        plan.query()
    y = d_out.cpu().numpy().astype(np.float64).reshape(n_dm, L)
    x = fb.T.astype(np.float64)
    X = oracle.fft_r2c(x)
    K = L // 2 + 1
    Y = oracle.fdd_bins_spin(X, np.arange(K), L, w.channel_centres(), 0.0, 0.25, n_dm,
                             w.t_samp_s, G, eps)
    ref = oracle.irfft(Y, L)
    assert rel_l2(y, ref) <= TC_REL_L2


def test_spin_rejects_what_it_does_not_run():
    w = _workload(16, 1024, 0.0, 0.5, 64)
    for kw, status in [(dict(precision=fdd.FDD_PREC_FP32, spin_group=16), fdd.FDD_ERR_UNSUPPORTED),
                       (dict(precision=fdd.FDD_PREC_FP16, spin_group=8), fdd.FDD_ERR_INVALID_ARG),
                       (dict(precision=fdd.FDD_PREC_FP16, spin_group=16, n_beams=2),
                        fdd.FDD_ERR_UNSUPPORTED)]:
        with pytest.raises(fdd.FddError) as e:
            fdd.Plan(**params_for(w, **kw))
        assert e.value.status == status

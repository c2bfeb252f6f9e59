"""The allocation-free phase-rotate-and-sum entry point (GB300 only).

fdd_dedisperse_spectra_static serves callers that cannot allocate device
memory (their framework owns the GPU's memory, or they run a real-time loop
that forbids allocation): it takes the plan parameters directly and keeps its
phase table in a static device array.  Here it is called twice in a row, with
different channel counts, DM grids and inputs (so the shared table is
rewritten between the calls), and each result is compared with the planned
entry point fdd_dedisperse_spectra at the FP32 tolerance of the other tests.
This file is collected last, so a failure here comes after every other test.
"""
import numpy as np
import pytest

import paper_2110_03482_gb300 as fdd
from gpu_util import FP32_REL_L2, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _params(n_chan, L, dms, lo=1200.0, hi=1500.0, t_samp=1e-3):
    dnu = (hi - lo) / n_chan
    return dict(n_chan=n_chan, nu_lo_mhz=lo + 0.5 * dnu, dnu_mhz=dnu, t_samp_s=t_samp, n_t=L,
                dm_list=np.asarray(dms, dtype=np.float64), chunk_len=0, in_dtype=fdd.FDD_IN_F32,
                output=fdd.FDD_OUT_SPECTRA)


CASES = [
    (48, 2048, 2.0 + 0.5 * np.arange(700), 11),
    (96, 4096, 0.25 * np.arange(2100), 12),
]


def test_static_entry_matches_planned_entry_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fdd.build()
    results = []
    for n_chan, L, dms, seed in CASES:
        K = L // 2 + 1
        pitch = K + 7
        g = torch.Generator(device="cuda").manual_seed(seed)
        X = torch.randn((2, n_chan, pitch, 2), device="cuda", generator=g)
        n_dm = dms.size
        Y_static = torch.zeros((2, n_dm, K, 2), device="cuda")
        fdd.fdd_dedisperse_spectra_static(fdd.Params(**_params(n_chan, L, dms)), X, pitch, 2, 0,
                                          n_dm, Y_static, K)
        results.append(Y_static)
        with fdd.Plan(**_params(n_chan, L, dms)) as plan:
            Y_plan = torch.zeros((2, n_dm, K, 2), device="cuda")
            plan.dedisperse_spectra(X, pitch, 2, 0, n_dm, Y_plan, K)
            torch.cuda.synchronize()
        ys = Y_static.cpu().numpy().astype(np.float64)
        yp = Y_plan.cpu().numpy().astype(np.float64)
        assert rel_l2(ys[..., 0] + 1j * ys[..., 1], yp[..., 0] + 1j * yp[..., 1]) <= FP32_REL_L2
    # the first call's output is untouched by the second call
    assert results[0].shape != results[1].shape


def test_static_entry_rejects_oversized_tables():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = fdd.Params(**_params(fdd.FDD_STATIC_MAX_CHAN + 1, 64, [0.0, 1.0]))
    X = torch.zeros((1, 4), device="cuda")
    with pytest.raises(fdd.FddError) as e:
        fdd.fdd_dedisperse_spectra_static(p, X, 33, 1, 0, 2, X, 33)
    assert e.value.status == fdd.FDD_ERR_INVALID_ARG
    assert "FDD_STATIC_MAX_CHAN" in fdd.fdd_last_error()

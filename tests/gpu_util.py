"""Helpers shared by the GPU tests (no dedispersion arithmetic here)."""
from __future__ import annotations

import numpy as np

import paper_2110_03482_gb300 as fdd
import synth

FP32_REL_L2 = 1e-5   # accuracy gate of the FP32 form against the FP64 oracle


def rel_l2(got, ref) -> float:
    got = np.asarray(got, dtype=np.complex128 if np.iscomplexobj(got) else np.float64)
    ref = np.asarray(ref, dtype=np.complex128 if np.iscomplexobj(ref) else np.float64)
    den = np.linalg.norm(ref.ravel())
    return float(np.linalg.norm((got - ref).ravel()) / (den if den > 0 else 1.0))


def params_for(w: synth.Workload, **kw) -> dict:
    d = dict(n_chan=w.n_chan, nu_lo_mhz=w.nu_lo_mhz, dnu_mhz=w.dnu_mhz, t_samp_s=w.t_samp_s,
             n_t=w.n_t, dm_list=w.dms(), chunk_len=w.chunk_len, n_beams=w.n_beams,
             in_dtype=fdd.FDD_IN_U8 if w.dtype == "u8" else fdd.FDD_IN_F32,
             output={"time": fdd.FDD_OUT_TIME, "spectra": fdd.FDD_OUT_SPECTRA,
                     "power": fdd.FDD_OUT_POWER}[w.output])
    d.update(kw)
    return d


def complex_to_device(X: np.ndarray, pitch: int):
    """[..., n] complex -> device float32 tensor [..., pitch, 2] (zero padded)."""
    import torch
    shape = X.shape[:-1] + (pitch, 2)
    host = np.zeros(shape, dtype=np.float32)
    host[..., : X.shape[-1], 0] = X.real
    host[..., : X.shape[-1], 1] = X.imag
    return torch.from_numpy(host).cuda()


def device_to_complex(t, n: int) -> np.ndarray:
    a = t.cpu().numpy()
    return a[..., :n, 0].astype(np.float64) + 1j * a[..., :n, 1].astype(np.float64)

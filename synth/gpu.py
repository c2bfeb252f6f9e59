"""Device side of the counter-based generator (``synth/csrc``): fills device
memory with exactly the bytes ``synth.philox.filterbank`` returns on the host.

Built in-tree for sm_103a by ``build()`` into ``synth/_lib/libsynth.so``.
Inputs only; no dedispersion arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

from . import philox

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "philox_filterbank.cu")
LIB_PATH = os.path.join(HERE, "_lib", "libsynth.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

_lib = None


def _nvcc() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home and os.path.isdir(home):
        return os.path.join(home, "bin", "nvcc")
    return shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB_PATH) and \
            os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC):
        return LIB_PATH
    os.makedirs(os.path.dirname(LIB_PATH), exist_ok=True)
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [_nvcc()] + ARCH + ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", SRC,
                              "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {SRC}:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run synth.gpu.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        L.synth_philox_filterbank.argtypes = [
            vp, ctypes.c_int, i64, ctypes.c_int, i64, ctypes.c_uint32, ctypes.c_uint64,
            ctypes.c_float, ctypes.c_float, ctypes.c_float, vp,
            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float), ctypes.c_int, vp]
        L.synth_philox_filterbank.restype = ctypes.c_int
        _lib = L
    return _lib


def filterbank(out, n_chan: int, n_rows: int, t0: int, seed: int, beam: int, *,
               mean: float = 0.0, sigma: float = 1.0, u8: bool = False, pulses=(),
               stream=None) -> None:
    """Fill the device tensor ``out`` (n_rows * n_chan uint8 or float32 elements,
    contiguous) with rows [t0, t0 + n_rows) of one beam; see
    ``synth.philox.filterbank`` for the arguments."""
    import torch
    want = torch.uint8 if u8 else torch.float32
    if out.dtype != want or out.numel() < n_rows * n_chan or not out.is_contiguous():
        raise ValueError("output tensor has the wrong dtype, size or layout")
    pulses = list(pulses)
    d_starts = None
    if pulses:
        starts = np.stack([np.asarray(p[0], dtype=np.int64) for p in pulses])
        d_starts = torch.from_numpy(starts).to(out.device)
    widths = (ctypes.c_int * max(1, len(pulses)))(*[int(p[1]) for p in pulses])
    amps = (ctypes.c_float * max(1, len(pulses)))(*[float(np.float32(p[2])) for p in pulses])
    s = stream if stream is not None else torch.cuda.current_stream(out.device)
    rc = lib().synth_philox_filterbank(
        ctypes.c_void_p(out.data_ptr()), int(u8), n_rows, n_chan, t0, beam, seed,
        float(np.float32(mean)), float(np.float32(sigma)), float(philox.IH8_INV_SIGMA),
        ctypes.c_void_p(d_starts.data_ptr() if d_starts is not None else 0), widths, amps,
        len(pulses), ctypes.c_void_p(s.cuda_stream))
    if rc != 0:
        raise RuntimeError(f"synth_philox_filterbank failed with code {rc}")
    if d_starts is not None:
        s.synchronize()  # d_starts is freed on return


class BeamWindows:
    """Fills raw device windows with rows of one workload's beams (the same
    bytes as ``filterbank``), for streaming sources: the pulses' start tables
    stay on the device for the object's lifetime."""

    def __init__(self, beam_kwargs: list[dict]):
        import torch
        self.kw = []
        for kw in beam_kwargs:
            pulses = list(kw.get("pulses", ()))
            d_starts = None
            if pulses:
                starts = np.stack([np.asarray(p[0], dtype=np.int64) for p in pulses])
                d_starts = torch.from_numpy(starts).cuda()
            widths = (ctypes.c_int * max(1, len(pulses)))(*[int(p[1]) for p in pulses])
            amps = (ctypes.c_float * max(1, len(pulses)))(*[float(np.float32(p[2]))
                                                           for p in pulses])
            self.kw.append((kw, d_starts, widths, amps, len(pulses)))

    def fill(self, beam: int, ptr: int, t0: int, n_rows: int, stream: int) -> None:
        """Rows [t0, t0 + n_rows) of beam ``beam`` (time-major) at device address ptr."""
        kw, d_starts, widths, amps, n_p = self.kw[beam]
        rc = lib().synth_philox_filterbank(
            ctypes.c_void_p(ptr), int(kw.get("u8", False)), n_rows, kw["n_chan"], t0,
            kw["beam"], kw["seed"], float(np.float32(kw.get("mean", 0.0))),
            float(np.float32(kw.get("sigma", 1.0))), float(philox.IH8_INV_SIGMA),
            ctypes.c_void_p(d_starts.data_ptr() if d_starts is not None else 0), widths, amps,
            n_p, ctypes.c_void_p(stream))
        if rc != 0:
            raise RuntimeError(f"synth_philox_filterbank failed with code {rc}")

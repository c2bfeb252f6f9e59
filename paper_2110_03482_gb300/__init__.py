"""GB300 (sm_103a) Fourier-domain dedispersion -- Python binding of the C ABI.

A thin ctypes layer over ``_lib/libfdd.so`` (declared in ``include/fdd.h``).
Functions carry the C names and only marshal arguments; every step of the
path runs in the library's CUDA kernels (and cuFFT for the channel
transforms).  There is no CPU fallback: importing works without the library,
but every call raises ``FddError`` until ``build()`` has produced it.

Device memory and streams come from PyTorch tensors
(``tensor.data_ptr()``, ``torch.cuda.current_stream().cuda_stream``); plain
integers (raw pointers) are accepted as well.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build_mod

LIB_PATH = _build_mod.LIB_PATH

# Constants of include/fdd.h
FDD_OK = 0
FDD_ERR_INVALID_ARG = 1
FDD_ERR_UNSUPPORTED = 2
FDD_ERR_ALLOC = 3
FDD_ERR_CUDA = 4
FDD_ERR_CUFFT = 5
FDD_ERR_TIMEOUT = 6
FDD_ERR_DEVICE = 7
FDD_IN_U8 = 0
FDD_IN_F32 = 1
FDD_LAYOUT_TIME_MAJOR = 0
FDD_LAYOUT_CHAN_MAJOR = 1
FDD_OUT_TIME = 0
FDD_OUT_SPECTRA = 1
FDD_OUT_POWER = 2
FDD_PREC_FP32 = 0
FDD_PREC_BF16_HILO = 1
FDD_PREC_BF16 = 2
FDD_PREC_FP16 = 3
FDD_PREC_FP8 = 4
MAC_VARIANT_NAMES = ["W12_8x8", "Q12_8x8", "Q_4x8", "Q_8x8_512", "Q_4x4", "G12_4x8"]
for _i, _n in enumerate(MAC_VARIANT_NAMES):
    globals()["FDD_MAC_" + _n.upper()] = _i
FDD_MAC_VARIANTS = len(MAC_VARIANT_NAMES)
FDD_MAC_TC = 100
FDD_MAC_TC_PAIR = 101

# Every symbol include/fdd.h declares.
EXPORTS = [
    "fdd_abi_version", "fdd_status_string", "fdd_last_error", "fdd_params_init",
    "fdd_plan_geometry", "fdd_plan", "fdd_query", "fdd_execute", "fdd_execute_dm_range",
    "fdd_execute_host", "fdd_execute_stream", "fdd_dedisperse_spectra", "fdd_profile_enable",
    "fdd_profile_read",
    "fdd_destroy", "fdd_dedisperse_spectra_static", "fdd_batch_plan", "fdd_batch_query",
    "fdd_batch_execute", "fdd_batch_destroy", "fdd_batch_execute_stream",
    "fdd_dedisperse_spectra_bins", "fdd_tdd_execute",
    "fdd_debug_stall_test", "fdd_debug_fail_alloc",
]
FDD_STATIC_MAX_CHAN = 8192

FDD_STAGE_UNPACK = 0
FDD_STAGE_R2C = 1
FDD_STAGE_MAC = 2
FDD_STAGE_C2R = 3
FDD_STAGE_SCATTER = 4
FDD_STAGE_TDD = 5
FDD_STAGE_TRANSPOSE = 6
FDD_STAGE_COUNT = 7
STAGE_NAMES = ["unpack", "r2c", "mac", "c2r", "scatter", "tdd", "transpose"]


class fdd_params(ctypes.Structure):
    _fields_ = [
        ("n_chan", ctypes.c_int32),
        ("n_beams", ctypes.c_int32),
        ("nu_lo_mhz", ctypes.c_double),
        ("dnu_mhz", ctypes.c_double),
        ("t_samp_s", ctypes.c_double),
        ("n_t", ctypes.c_int64),
        ("dm_list", ctypes.POINTER(ctypes.c_double)),
        ("n_dm", ctypes.c_int32),
        ("in_dtype", ctypes.c_int32),
        ("chunk_len", ctypes.c_int64),
        ("k_dm", ctypes.c_double),
        ("nu_ref_mhz", ctypes.c_double),
        ("in_layout", ctypes.c_int32),
        ("output", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("mac_variant", ctypes.c_int32),
        ("workspace_limit", ctypes.c_size_t),
        ("downsample", ctypes.c_int32),
        ("spin_group", ctypes.c_int32),
        ("spin_tol", ctypes.c_double),
    ]


class fdd_info(ctypes.Structure):
    _fields_ = [
        ("fft_len", ctypes.c_int64),
        ("n_bins", ctypes.c_int64),
        ("bin_pitch", ctypes.c_int64),
        ("n_chunks", ctypes.c_int64),
        ("hop", ctypes.c_int64),
        ("d_max", ctypes.c_int64),
        ("out_len", ctypes.c_int64),
        ("valid_len", ctypes.c_int64),
        ("in_elems", ctypes.c_int64),
        ("out_elems", ctypes.c_int64),
        ("out_bytes", ctypes.c_int64),
        ("workspace_bytes", ctypes.c_int64),
        ("dm0", ctypes.c_double),
        ("ddm", ctypes.c_double),
        ("dm_uniform", ctypes.c_int32),
        ("dm_batch", ctypes.c_int32),
        ("mac_variant", ctypes.c_int32),
        ("downsample", ctypes.c_int32),
        ("block_dm", ctypes.c_int32),
        ("stream_bytes", ctypes.c_int64),
        ("spin_group", ctypes.c_int32),
        ("spin_k_min", ctypes.c_int32),
        ("spin_j_lo", ctypes.c_int32),
        ("spin_n_s", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class fdd_block(ctypes.Structure):
    _fields_ = [
        ("beam_first", ctypes.c_int32),
        ("n_beams", ctypes.c_int32),
        ("chunk", ctypes.c_int64),
        ("dm_first", ctypes.c_int32),
        ("n_dm", ctypes.c_int32),
        ("d_data", ctypes.c_void_p),
        ("row_len", ctypes.c_int64),
        ("row_pitch", ctypes.c_int64),
        ("out_offset", ctypes.c_int64),
        ("release_event", ctypes.c_void_p),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


# fdd_source_fn / fdd_sink_fn
SOURCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                             ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
SINK_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(fdd_block),
                           ctypes.c_void_p)


class fdd_profile(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_int64 * FDD_STAGE_COUNT),
        ("ms", ctypes.c_double * FDD_STAGE_COUNT),
        ("dropped", ctypes.c_int64),
        ("kernels", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {"launches": {STAGE_NAMES[i]: int(self.launches[i]) for i in range(FDD_STAGE_COUNT)},
                "ms": {STAGE_NAMES[i]: float(self.ms[i]) for i in range(FDD_STAGE_COUNT)},
                "dropped": int(self.dropped), "kernels": int(self.kernels)}


class fdd_beam_desc(ctypes.Structure):
    _fields_ = [
        ("n_t", ctypes.c_int64),
        ("dm0", ctypes.c_double),
        ("ddm", ctypes.c_double),
        ("n_dm", ctypes.c_int32),
        ("chunk_len", ctypes.c_int32),
    ]


class fdd_batch_info(ctypes.Structure):
    _fields_ = [
        ("in_elems", ctypes.c_int64),
        ("out_elems", ctypes.c_int64),
        ("out_bytes", ctypes.c_int64),
        ("workspace_bytes", ctypes.c_int64),
        ("work_items", ctypes.c_int64),
        ("n_waves", ctypes.c_int32),
        ("mac_variant", ctypes.c_int32),
        ("ctas", ctypes.c_int32),
        ("tail_variant", ctypes.c_int32),
        ("autotune_ms", ctypes.c_double * FDD_MAC_VARIANTS),
    ]

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_ if name != "autotune_ms"}
        d["autotune_ms"] = {MAC_VARIANT_NAMES[i]: self.autotune_ms[i]
                            for i in range(len(MAC_VARIANT_NAMES)) if self.autotune_ms[i] >= 0}
        return d


class FddError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


_lib = None


def library_path() -> str:
    return LIB_PATH


def build(force: bool = False) -> str:
    """Compile the CUDA library for sm_103a in-tree (nvcc)."""
    return _build_mod.build(force=force)


def lib() -> ctypes.CDLL:
    """The loaded CUDA library; raises FddError if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FddError(-1, f"CUDA library not built: {LIB_PATH} is missing "
                               "(run paper_2110_03482_gb300.build())")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.fdd_abi_version.restype = i32
        L.fdd_status_string.restype = ctypes.c_char_p
        L.fdd_status_string.argtypes = [ctypes.c_int]
        L.fdd_last_error.restype = ctypes.c_char_p
        L.fdd_params_init.argtypes = [ctypes.POINTER(fdd_params)]
        L.fdd_params_init.restype = None
        L.fdd_plan_geometry.argtypes = [ctypes.POINTER(fdd_params), ctypes.POINTER(fdd_info)]
        L.fdd_plan.argtypes = [ctypes.POINTER(fdd_params), ctypes.POINTER(vp)]
        L.fdd_query.argtypes = [vp, ctypes.POINTER(fdd_info)]
        L.fdd_execute.argtypes = [vp, vp, vp, vp]
        L.fdd_execute_dm_range.argtypes = [vp, vp, i32, i32, vp, vp]
        L.fdd_execute_host.argtypes = [vp, vp, vp, vp]
        L.fdd_execute_stream.argtypes = [vp, vp, SOURCE_FN, vp, SINK_FN, vp, vp]
        L.fdd_tdd_execute.argtypes = [vp, vp, vp, vp]
        L.fdd_debug_stall_test.argtypes = [vp, vp]
        L.fdd_debug_fail_alloc.argtypes = [i32]
        L.fdd_dedisperse_spectra.argtypes = [vp, vp, i64, i32, i32, i32, vp, i64, i32, vp]
        L.fdd_dedisperse_spectra_bins.argtypes = [vp, vp, i64, i32, i32, i32, i32, i32, vp,
                                                  i64, i32, vp]
        L.fdd_destroy.argtypes = [vp]
        L.fdd_dedisperse_spectra_static.argtypes = [ctypes.POINTER(fdd_params), vp, i64, i32,
                                                     i32, i32, vp, i64, i32, vp]
        L.fdd_batch_plan.argtypes = [ctypes.POINTER(fdd_params), ctypes.POINTER(fdd_beam_desc),
                                     i32, i32, ctypes.POINTER(vp)]
        L.fdd_batch_query.argtypes = [vp, ctypes.POINTER(fdd_batch_info),
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.fdd_batch_execute.argtypes = [vp, vp, vp, vp]
        L.fdd_batch_destroy.argtypes = [vp]
        L.fdd_batch_execute_stream.argtypes = [vp, SOURCE_FN, vp, SINK_FN, vp, vp]
        L.fdd_profile_enable.argtypes = [vp, i32]
        L.fdd_profile_read.argtypes = [vp, ctypes.POINTER(fdd_profile)]
        for name in ["fdd_plan_geometry", "fdd_plan", "fdd_query", "fdd_execute",
                     "fdd_execute_dm_range", "fdd_execute_host", "fdd_execute_stream",
                     "fdd_dedisperse_spectra",
                     "fdd_profile_enable", "fdd_profile_read", "fdd_destroy",
                     "fdd_dedisperse_spectra_static", "fdd_batch_plan", "fdd_batch_query",
                     "fdd_batch_execute", "fdd_batch_destroy", "fdd_batch_execute_stream",
                     "fdd_dedisperse_spectra_bins",
                     "fdd_tdd_execute", "fdd_debug_stall_test", "fdd_debug_fail_alloc"]:
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


_cudart = None


def cudart() -> ctypes.CDLL:
    """The CUDA runtime (for raw-pointer copies inside streaming callbacks;
    the library itself needs nothing from here)."""
    global _cudart
    if _cudart is None:
        home = _build_mod._cuda_home()
        for name in (os.path.join(home, "lib64", "libcudart.so"), "libcudart.so.13",
                     "libcudart.so"):
            try:
                _cudart = ctypes.CDLL(name)
                break
            except OSError:
                continue
        if _cudart is None:
            raise FddError(-1, "libcudart not found")
        sz = ctypes.c_size_t
        vp = ctypes.c_void_p
        _cudart.cudaMemcpyAsync.argtypes = [vp, vp, sz, ctypes.c_int, vp]
        _cudart.cudaMemcpy2DAsync.argtypes = [vp, sz, vp, sz, sz, sz, ctypes.c_int, vp]
    return _cudart


def memcpy_async(dst: int, src: int, nbytes: int, stream: int) -> None:
    """cudaMemcpyAsync with cudaMemcpyDefault (direction from the addresses)."""
    rc = cudart().cudaMemcpyAsync(dst, src, nbytes, 4, stream)
    if rc != 0:
        raise FddError(FDD_ERR_CUDA, f"cudaMemcpyAsync failed ({rc})")


def memcpy2d_async(dst: int, dpitch: int, src: int, spitch: int, width: int, height: int,
                   stream: int) -> None:
    rc = cudart().cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, height, 4, stream)
    if rc != 0:
        raise FddError(FDD_ERR_CUDA, f"cudaMemcpy2DAsync failed ({rc})")


def _check(status: int):
    if status != FDD_OK:
        L = lib()
        raise FddError(status, f"{L.fdd_status_string(status).decode()}: "
                               f"{L.fdd_last_error().decode()}")


def _ptr(x) -> int | None:
    """Device/host address of a torch tensor, numpy array or integer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream(s) -> int | None:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ------------------------------------------------------------------ C names
def fdd_abi_version() -> int:
    return int(lib().fdd_abi_version())


def fdd_status_string(status: int) -> str:
    return lib().fdd_status_string(status).decode()


def fdd_last_error() -> str:
    return lib().fdd_last_error().decode()


class Params:
    """Owns an fdd_params and the DM array it points at."""

    def __init__(self, **kw):
        self.c = fdd_params()
        lib().fdd_params_init(ctypes.byref(self.c))
        dms = kw.pop("dm_list")
        self.dms = np.ascontiguousarray(dms, dtype=np.float64)
        self.c.dm_list = self.dms.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self.c.n_dm = int(self.dms.size)
        for k, v in kw.items():
            if not hasattr(self.c, k):
                raise TypeError(f"unknown parameter {k}")
            setattr(self.c, k, v)


def fdd_params_init(**kw) -> Params:
    return Params(**kw)


def fdd_plan_geometry(params: Params) -> dict:
    info = fdd_info()
    _check(lib().fdd_plan_geometry(ctypes.byref(params.c), ctypes.byref(info)))
    return info.as_dict()


def fdd_plan(params: Params) -> int:
    h = ctypes.c_void_p()
    _check(lib().fdd_plan(ctypes.byref(params.c), ctypes.byref(h)))
    return h.value


def fdd_query(plan: int) -> dict:
    info = fdd_info()
    _check(lib().fdd_query(plan, ctypes.byref(info)))
    return info.as_dict()


def fdd_execute(plan: int, d_in, d_out, stream=None) -> None:
    _check(lib().fdd_execute(plan, _ptr(d_in), _ptr(d_out), _stream(stream)))


def _callbacks(source, sink, err):
    """ctypes callbacks around Python source / sink functions; exceptions are
    collected in err and end the call."""
    def _src(_user, beam, t_begin, n, d_window, ready, s):
        try:
            source(int(beam), int(t_begin), int(n), int(d_window), ready, s)
            return FDD_OK
        except BaseException as e:  # noqa: BLE001 -- re-raised by the caller
            err.append(e)
            return FDD_ERR_INVALID_ARG

    def _snk(_user, blk, s):
        try:
            ev = sink(blk.contents.as_dict(), s)
            blk.contents.release_event = ev
            return FDD_OK
        except BaseException as e:  # noqa: BLE001 -- re-raised by the caller
            err.append(e)
            return FDD_ERR_INVALID_ARG

    c_src = SOURCE_FN(_src) if source is not None else ctypes.cast(None, SOURCE_FN)
    return c_src, SINK_FN(_snk)


def fdd_batch_execute_stream(batch: int, source, sink, stream=None) -> None:
    """Streamed batch execute: ``source(beam, 0, n_t, d_window, ready_event,
    stream)`` per beam, ``sink(block, stream)`` per beam's output block (see
    fdd_execute_stream)."""
    err = []
    c_src, c_snk = _callbacks(source, sink, err)
    status = lib().fdd_batch_execute_stream(batch, c_src, None, c_snk, None, _stream(stream))
    if err:
        raise err[0]
    _check(status)


def fdd_execute_stream(plan: int, source, sink, stream=None, d_in=None) -> None:
    """Streamed execute.  Input: ``d_in`` resident on the device (source None),
    or ``source(beam, t_begin, n_samples, d_window, ready_event, stream)``
    filling each window (device address d_window; raw CUDA event and stream
    handles).  Output: ``sink(block, stream)`` for each block, ``block`` a dict
    of the fdd_block fields; a sink that reads the block on another stream
    returns the handle of a CUDA event recorded after those reads (else None).
    An exception in a callback ends the call and is raised here."""
    err = []
    c_src, c_snk = _callbacks(source, sink, err)
    status = lib().fdd_execute_stream(plan, _ptr(d_in), c_src, None, c_snk, None,
                                      _stream(stream))
    if err:
        raise err[0]
    _check(status)


def fdd_execute_dm_range(plan: int, d_in, dm_first: int, n_dm: int, d_out, stream=None) -> None:
    _check(lib().fdd_execute_dm_range(plan, _ptr(d_in), dm_first, n_dm, _ptr(d_out),
                                      _stream(stream)))


def fdd_debug_stall_test(plan: int, stream=None) -> None:
    """Run the plan's waiting kernel with producers that never arrive: its
    bounded waits run out (~2 s) and the next query reports FDD_ERR_TIMEOUT."""
    _check(lib().fdd_debug_stall_test(plan, _stream(stream)))


def fdd_debug_fail_alloc(after: int) -> None:
    """Make the device allocation after the next `after` ones fail once (-1: off)."""
    _check(lib().fdd_debug_fail_alloc(after))


def fdd_tdd_execute(plan: int, d_in, d_out, stream=None) -> None:
    _check(lib().fdd_tdd_execute(plan, _ptr(d_in), _ptr(d_out), _stream(stream)))


def fdd_execute_host(plan: int, h_in, h_out, stream=None) -> None:
    _check(lib().fdd_execute_host(plan, _ptr(h_in), _ptr(h_out), _stream(stream)))


def fdd_dedisperse_spectra(plan: int, d_X, x_pitch: int, n_series: int, dm_first: int,
                           n_dm: int, d_Y, y_pitch: int, out_kind: int = FDD_OUT_SPECTRA,
                           stream=None) -> None:
    _check(lib().fdd_dedisperse_spectra(plan, _ptr(d_X), x_pitch, n_series, dm_first, n_dm,
                                        _ptr(d_Y), y_pitch, out_kind, _stream(stream)))


def fdd_dedisperse_spectra_bins(plan: int, d_X, x_pitch: int, n_series: int, bin_first: int,
                                n_bins: int, dm_first: int, n_dm: int, d_Y, y_pitch: int,
                                out_kind: int = FDD_OUT_SPECTRA, stream=None) -> None:
    _check(lib().fdd_dedisperse_spectra_bins(plan, _ptr(d_X), x_pitch, n_series, bin_first,
                                             n_bins, dm_first, n_dm, _ptr(d_Y), y_pitch,
                                             out_kind, _stream(stream)))


def fdd_dedisperse_spectra_static(params: Params, d_X, x_pitch: int, n_series: int,
                                  dm_first: int, n_dm: int, d_Y, y_pitch: int,
                                  out_kind: int = FDD_OUT_SPECTRA, stream=None) -> None:
    """Phase-rotate-and-sum without a plan and without any allocation (for
    callers whose device memory is owned elsewhere); see include/fdd.h."""
    _check(lib().fdd_dedisperse_spectra_static(ctypes.byref(params.c), _ptr(d_X), x_pitch,
                                               n_series, dm_first, n_dm, _ptr(d_Y), y_pitch,
                                               out_kind, _stream(stream)))


def fdd_batch_plan(params: Params, beams, autotune: bool = True) -> int:
    """beams: sequence of (n_t, dm0, ddm, n_dm) or (n_t, dm0, ddm, n_dm, chunk_len)."""
    arr = (fdd_beam_desc * len(beams))()
    for i, bm in enumerate(beams):
        n_t, dm0, ddm, n_dm = bm[:4]
        chunk = bm[4] if len(bm) > 4 else 0
        arr[i] = fdd_beam_desc(int(n_t), float(dm0), float(ddm), int(n_dm), int(chunk))
    h = ctypes.c_void_p()
    _check(lib().fdd_batch_plan(ctypes.byref(params.c), arr, len(beams), 1 if autotune else 0,
                                ctypes.byref(h)))
    return h.value


def fdd_batch_query(batch: int, n_beams: int):
    info = fdd_batch_info()
    ino = (ctypes.c_int64 * n_beams)()
    outo = (ctypes.c_int64 * n_beams)()
    _check(lib().fdd_batch_query(batch, ctypes.byref(info), ino, outo))
    return info.as_dict(), list(ino), list(outo)


def fdd_batch_execute(batch: int, d_in, d_out, stream=None) -> None:
    _check(lib().fdd_batch_execute(batch, _ptr(d_in), _ptr(d_out), _stream(stream)))


def fdd_batch_destroy(batch: int) -> None:
    _check(lib().fdd_batch_destroy(batch))


class Batch:
    """RAII wrapper of a batch plan: Batch(beams, **common params)."""

    def __init__(self, beams, autotune: bool = True, **kw):
        kw.setdefault("dm_list", [0.0])
        self.params = Params(**kw)
        self.n_beams = len(beams)
        self.handle = fdd_batch_plan(self.params, beams, autotune)
        self.info, self.in_offsets, self.out_offsets = fdd_batch_query(self.handle, self.n_beams)

    def execute(self, d_in, d_out, stream=None):
        fdd_batch_execute(self.handle, d_in, d_out, stream)

    def execute_stream(self, source, sink, stream=None):
        fdd_batch_execute_stream(self.handle, source, sink, stream)

    def close(self):
        if self.handle:
            fdd_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fdd_profile_enable(plan: int, on: bool = True) -> None:
    _check(lib().fdd_profile_enable(plan, 1 if on else 0))


def fdd_profile_read(plan: int) -> dict:
    prof = fdd_profile()
    _check(lib().fdd_profile_read(plan, ctypes.byref(prof)))
    return prof.as_dict()


def fdd_destroy(plan: int) -> None:
    _check(lib().fdd_destroy(plan))


# ------------------------------------------------------------------ convenience
class Plan:
    """RAII wrapper: Plan(**params) -> .execute(d_in, d_out) ... .close()."""

    def __init__(self, **kw):
        self.params = Params(**kw)
        self.handle = fdd_plan(self.params)
        self.info = fdd_query(self.handle)

    def execute(self, d_in, d_out, stream=None):
        fdd_execute(self.handle, d_in, d_out, stream)

    def execute_dm_range(self, d_in, dm_first, n_dm, d_out, stream=None):
        fdd_execute_dm_range(self.handle, d_in, dm_first, n_dm, d_out, stream)

    def execute_host(self, h_in, h_out, stream=None):
        fdd_execute_host(self.handle, h_in, h_out, stream)

    def execute_stream(self, source, sink, stream=None, d_in=None):
        fdd_execute_stream(self.handle, source, sink, stream, d_in)

    def debug_stall_test(self, stream=None):
        fdd_debug_stall_test(self.handle, stream)

    def tdd_execute(self, d_in, d_out, stream=None):
        """Brute-force time-domain dedispersion (Eq. 2) with this plan's
        parameters: d_out is float [n_beams][n_dm][n_t - d_max]."""
        fdd_tdd_execute(self.handle, d_in, d_out, stream)

    def dedisperse_spectra(self, d_X, x_pitch, n_series, dm_first, n_dm, d_Y, y_pitch,
                           out_kind=FDD_OUT_SPECTRA, stream=None):
        fdd_dedisperse_spectra(self.handle, d_X, x_pitch, n_series, dm_first, n_dm, d_Y,
                               y_pitch, out_kind, stream)

    def dedisperse_spectra_bins(self, d_X, x_pitch, n_series, bin_first, n_bins, dm_first, n_dm,
                                d_Y, y_pitch, out_kind=FDD_OUT_SPECTRA, stream=None):
        fdd_dedisperse_spectra_bins(self.handle, d_X, x_pitch, n_series, bin_first, n_bins,
                                    dm_first, n_dm, d_Y, y_pitch, out_kind, stream)

    def query(self) -> dict:
        return fdd_query(self.handle)

    def profile_enable(self, on: bool = True):
        fdd_profile_enable(self.handle, on)

    def profile_read(self) -> dict:
        return fdd_profile_read(self.handle)

    def close(self):
        if self.handle:
            fdd_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

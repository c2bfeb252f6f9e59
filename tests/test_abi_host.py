"""The C ABI on the CPU: the library loads, exports what include/fdd.h
declares, and its host-only plan geometry agrees with the oracle's reading of
the chunking (no GPU needed; no compute calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2110_03482_gb300 as fdd
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    fdd.build()


def declared_functions():
    with open(os.path.join(ROOT, "include", "fdd.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    # (function declarations only: not the callback typedefs)
    return sorted(set(re.findall(r"^\s*(?!typedef)(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\**\s+\**"
                                 r"(fdd_[a-z_0-9]+)\s*\(", src, flags=re.M)))


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(fdd.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(fdd.library_path())
    for name in declared_functions():
        assert hasattr(L, name), name
    assert fdd.fdd_abi_version() == 2


def test_status_strings():
    assert fdd.fdd_status_string(0) == "FDD_OK"
    assert fdd.fdd_status_string(6) == "FDD_ERR_TIMEOUT"
    assert fdd.fdd_status_string(99) == "FDD_ERR_UNKNOWN"


def _params(w: synth.Workload, **kw):
    d = dict(n_chan=w.n_chan, nu_lo_mhz=w.nu_lo_mhz, dnu_mhz=w.dnu_mhz, t_samp_s=w.t_samp_s,
             n_t=w.n_t, dm_list=w.dms(), chunk_len=w.chunk_len, n_beams=w.n_beams,
             in_dtype=fdd.FDD_IN_U8 if w.dtype == "u8" else fdd.FDD_IN_F32,
             output={"time": 0, "spectra": 1, "power": 2}[w.output])
    d.update(kw)
    return fdd.Params(**d)


@pytest.mark.parametrize("name", list(synth.WORKLOADS))
def test_geometry_matches_oracle(name):
    w = synth.WORKLOADS[name]
    g = fdd.fdd_plan_geometry(_params(w))
    d = oracle.delays(w.channel_centres(), w.dms(), w.t_samp_s)
    og = oracle.geometry(w.n_t, w.chunk_len, d)
    assert g["fft_len"] == og.L
    assert g["n_bins"] == og.K
    assert g["d_max"] == og.d_max
    assert g["n_chunks"] == og.n_chunks
    assert g["out_len"] == og.n_out
    if w.chunk_len:
        assert g["hop"] == og.hop
    assert g["dm_uniform"] == 1
    assert g["bin_pitch"] >= g["n_bins"] and g["bin_pitch"] % 64 == 0
    assert g["in_elems"] == w.n_beams * w.n_t * w.n_chan


def test_geometry_survey_values():
    """Survey-shaped workload: 1024 channels over 1210-1520 MHz at 64 us, trials
    0..1023.5: the sweep is ~16.2 samples per unit DM (16585 samples at the top
    trial), so 2^18-sample chunks keep 245559 samples each and 5 chunks cover
    the 2^20-sample series."""
    w = synth.WORKLOADS["fdd_1024ch_2p20t_2048dm"]
    g = fdd.fdd_plan_geometry(_params(w))
    assert g["fft_len"] == 1 << 18 and g["n_bins"] == (1 << 17) + 1
    assert 16580 <= g["d_max"] <= 16590
    assert g["hop"] == (1 << 18) - g["d_max"]
    assert g["n_chunks"] == 5
    assert g["out_len"] == (1 << 20) - g["d_max"]
    assert g["dm_batch"] == 2048


@pytest.mark.parametrize("kw,status", [
    (dict(n_chan=0), fdd.FDD_ERR_INVALID_ARG),
    (dict(t_samp_s=0.0), fdd.FDD_ERR_INVALID_ARG),
    (dict(n_t=1), fdd.FDD_ERR_INVALID_ARG),
    (dict(dnu_mhz=0.0), fdd.FDD_ERR_INVALID_ARG),
    (dict(chunk_len=101), fdd.FDD_ERR_INVALID_ARG),
    (dict(chunk_len=64), fdd.FDD_ERR_INVALID_ARG),        # shorter than the delay
    (dict(nu_ref_mhz=1000.0), fdd.FDD_ERR_INVALID_ARG),   # below the top channel
    (dict(in_dtype=7), fdd.FDD_ERR_INVALID_ARG),
    (dict(output=9), fdd.FDD_ERR_INVALID_ARG),
    (dict(precision=5), fdd.FDD_ERR_INVALID_ARG),
    (dict(precision=-1), fdd.FDD_ERR_INVALID_ARG),
    (dict(dm_list=np.array([-1.0, 0.0])), fdd.FDD_ERR_INVALID_ARG),
    (dict(dm_list=np.array([0.0, np.nan])), fdd.FDD_ERR_INVALID_ARG),
    (dict(mac_variant=-1), fdd.FDD_ERR_INVALID_ARG),
    (dict(mac_variant=fdd.FDD_MAC_VARIANTS + 1), fdd.FDD_ERR_INVALID_ARG),
    (dict(workspace_limit=1024), fdd.FDD_ERR_INVALID_ARG),
])
def test_invalid_parameters(kw, status):
    w = synth.WORKLOADS["fdd_64ch_4096t_128dm"]
    with pytest.raises(fdd.FddError) as e:
        fdd.fdd_plan_geometry(_params(w, **kw))
    assert e.value.status == status
    assert fdd.fdd_last_error()


def test_non_uniform_dm_list_makes_a_plan_for_the_time_domain_path():
    """Any DM list makes a valid plan (the brute-force time-domain path takes
    it); the geometry reports it, and the Fourier-domain calls refuse it."""
    w = synth.WORKLOADS["fdd_64ch_4096t_128dm"]
    g = fdd.fdd_plan_geometry(_params(w, dm_list=np.array([0.0, 1.0, 3.0])))
    assert g["dm_uniform"] == 0 and g["d_max"] > 0


def test_downsample_geometry_matches_oracle():
    """Shortened inverse transform (Sect. 2.2, last paragraph): the hop is a
    multiple of f and the output counts ceil(native / f) samples."""
    w = synth.WORKLOADS["fdd_1024ch_2p20t_2048dm"]
    d = oracle.delays(w.channel_centres(), w.dms(), w.t_samp_s)
    for f in (1, 2, 4, 8):
        g = fdd.fdd_plan_geometry(_params(w, downsample=f))
        geo = oracle.geometry_downsampled(w.n_t, w.chunk_len, d, f)
        assert g["downsample"] == f and g["hop"] == geo.hop and g["hop"] % f == 0
        assert g["out_len"] == geo.n_out and g["n_chunks"] == geo.n_chunks
        assert g["out_elems"] == w.n_dm * geo.n_out
    w1 = synth.WORKLOADS["fdd_64ch_4096t_128dm"].scaled(n_t=4001)
    g = fdd.fdd_plan_geometry(_params(w1, downsample=4))
    assert g["out_len"] == 1001 and g["n_chunks"] == 1
    for kw in (dict(downsample=3), dict(downsample=-2), dict(downsample=2, output=1),
               dict(downsample=4096)):
        with pytest.raises(fdd.FddError) as e:
            fdd.fdd_plan_geometry(_params(w1, **kw))
        assert e.value.status == fdd.FDD_ERR_INVALID_ARG


def test_variant_choice():
    w = synth.WORKLOADS["fdd_64ch_4096t_128dm"]
    assert fdd.fdd_plan_geometry(_params(w))["mac_variant"] == fdd.FDD_MAC_Q_4X4
    for v in range(fdd.FDD_MAC_VARIANTS):
        assert fdd.fdd_plan_geometry(_params(w, mac_variant=v + 1))["mac_variant"] == v
    w2 = synth.WORKLOADS["fdd_1024ch_2p20t_2048dm"]
    assert fdd.fdd_plan_geometry(_params(w2))["mac_variant"] == fdd.FDD_MAC_G12_4X8
    # least padded-block time: 128-trial blocks up to 256 trials, the
    # 2048-trial tile above (a last block of <= 512 or <= 1024 trials as
    # 512- or 1024-trial wide items); measured rates 0.347 (128), 0.752
    # (2048), wide 0.616, narrow 0.510
    for n, v in [(1, fdd.FDD_MAC_Q_4X4), (256, fdd.FDD_MAC_Q_4X4), (384, fdd.FDD_MAC_G12_4X8),
                 (448, fdd.FDD_MAC_G12_4X8), (512, fdd.FDD_MAC_G12_4X8),
                 (600, fdd.FDD_MAC_G12_4X8), (1024, fdd.FDD_MAC_G12_4X8),
                 (1100, fdd.FDD_MAC_G12_4X8), (4096, fdd.FDD_MAC_G12_4X8)]:
        g = fdd.fdd_plan_geometry(_params(w2, dm_list=0.5 * np.arange(n)))
        assert g["mac_variant"] == v, (n, g["mac_variant"])
    # the G12 tile's ring (three stages of 48 KB, two beyond about 5300
    # channels) leaves room for the phase table of up to 8381 channels (16
    # bytes each) in a CTA's 227 KB; above that the fastest tile that fits is
    # taken
    g = fdd.fdd_plan_geometry(_params(w2, n_chan=8192, dnu_mhz=0.02, workspace_limit=200 << 30))
    assert g["mac_variant"] == fdd.FDD_MAC_G12_4X8
    g = fdd.fdd_plan_geometry(_params(w2, n_chan=9000, dnu_mhz=0.02, workspace_limit=200 << 30))
    assert g["mac_variant"] not in (fdd.FDD_MAC_G12_4X8, fdd.FDD_MAC_TC)


def test_tensor_core_form_geometry():
    """The tensor-core form holds the spectra of every beam at once and batches
    DMs in whole trial passes when the workspace is bounded (below one pass,
    whatever fits).  Plans whose calls end in a pass of the CTA-pair form
    (2048 trials in 32-beam groups, 4096 in 16-beam groups; T = 256 trials
    per a) that is full or more than half full take that form: with time
    output only in DM batches of whole pair passes, with spectra or power
    only while two output blocks of one pair pass fit half the limit."""
    w = synth.WORKLOADS["fdd_32beam_1024ch_2p19t_4096dm"]
    hilo = fdd.FDD_PREC_BF16_HILO
    g = fdd.fdd_plan_geometry(_params(w, precision=hilo, workspace_limit=200 << 30))
    assert g["mac_variant"] == fdd.FDD_MAC_TC  # 1941 trials fit: one-CTA passes
    assert g["dm_batch"] == 1024
    spectra = 32 * 1024 * g["bin_pitch"] * 8
    assert spectra < g["workspace_bytes"] <= 200 << 30
    g = fdd.fdd_plan_geometry(_params(w, precision=hilo, workspace_limit=120 << 30))
    assert g["mac_variant"] == fdd.FDD_MAC_TC
    assert 512 < g["dm_batch"] < 1024 and g["workspace_bytes"] <= 120 << 30
    g = fdd.fdd_plan_geometry(_params(w, precision=hilo, workspace_limit=72 << 30))
    assert 0 < g["dm_batch"] < 256 and g["workspace_bytes"] <= 72 << 30
    # the form by the pair's last pass: 1024 / 2560 / 3072 trials end in a
    # pair pass at most half full, 1100 / 1536 / 2048 / 3584 / 4096 not
    for n, v in [(1024, fdd.FDD_MAC_TC), (1100, fdd.FDD_MAC_TC_PAIR),
                 (1536, fdd.FDD_MAC_TC_PAIR), (2048, fdd.FDD_MAC_TC_PAIR),
                 (2560, fdd.FDD_MAC_TC), (3072, fdd.FDD_MAC_TC),
                 (3584, fdd.FDD_MAC_TC_PAIR), (4096, fdd.FDD_MAC_TC_PAIR)]:
        g = fdd.fdd_plan_geometry(_params(w, precision=fdd.FDD_PREC_FP16, n_t=4096,
                                          output=fdd.FDD_OUT_SPECTRA,
                                          dm_list=0.5 * np.arange(n),
                                          workspace_limit=200 << 30))
        assert g["mac_variant"] == v, (n, g["mac_variant"])
    # 16 beams: 4096-trial pair passes; 120 GiB holds 2048 trials (one-CTA
    # passes), 200 GiB all 4096
    g = fdd.fdd_plan_geometry(_params(w, n_beams=16, precision=hilo, workspace_limit=120 << 30))
    assert g["mac_variant"] == fdd.FDD_MAC_TC
    assert g["dm_batch"] == 2048 and g["workspace_bytes"] <= 120 << 30
    g = fdd.fdd_plan_geometry(_params(w, n_beams=16, precision=hilo, workspace_limit=200 << 30))
    assert g["mac_variant"] == fdd.FDD_MAC_TC_PAIR and g["dm_batch"] == 4096
    # power of 32 beams: a pair pass's block (2048 x 32 x 262145 x 4 B) is
    # above a quarter of 240 GiB, so the one-CTA form, blocks of its pass
    g = fdd.fdd_plan_geometry(_params(w, precision=fdd.FDD_PREC_FP16, output=fdd.FDD_OUT_POWER,
                                      workspace_limit=240 << 30))
    assert g["mac_variant"] == fdd.FDD_MAC_TC and g["block_dm"] == 1024
    g = fdd.fdd_plan_geometry(_params(w, precision=fdd.FDD_PREC_FP16, output=fdd.FDD_OUT_POWER,
                                      workspace_limit=280 << 30))
    assert g["mac_variant"] == fdd.FDD_MAC_TC_PAIR and g["block_dm"] == 2048


def test_geometry_edge_cases():
    w = synth.WORKLOADS["fdd_64ch_4096t_128dm"]
    # single trial, single channel, n_t not a power of two
    g = fdd.fdd_plan_geometry(_params(w, n_chan=1, dm_list=np.array([5.0]), n_t=1000))
    assert g["fft_len"] == 1024 and g["d_max"] == 0 and g["out_len"] == 1000
    assert g["dm_uniform"] == 1 and g["ddm"] == 0.0
    # descending band: channel 0 is the highest, still no negative delays
    g = fdd.fdd_plan_geometry(_params(w, nu_lo_mhz=1550.0 - 4.6875 / 2, dnu_mhz=-4.6875))
    g2 = fdd.fdd_plan_geometry(_params(w))
    assert g["d_max"] == g2["d_max"]
    # a workspace limit forces DM batches of whole kernel blocks
    w2 = synth.WORKLOADS["fdd_1024ch_2p20t_2048dm"]
    g = fdd.fdd_plan_geometry(_params(w2, workspace_limit=4 << 30))
    assert 0 < g["dm_batch"] < 2048 and g["workspace_bytes"] <= 4 << 30


def test_plan_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    w = synth.WORKLOADS["fdd_64ch_4096t_128dm"]
    with pytest.raises(fdd.FddError) as e:
        fdd.fdd_plan(_params(w))
    assert e.value.status in (fdd.FDD_ERR_CUDA, fdd.FDD_ERR_UNSUPPORTED)

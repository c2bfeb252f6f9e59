"""The batching form (uneven beams and trial grids, persistent launch per wave,
CUDA graph, autotuner) against the FP64 oracle (GB300 only)."""
import numpy as np
import pytest

import oracle
import paper_2110_03482_gb300 as fdd
import synth
from gpu_util import FP32_REL_L2, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N_CHAN = 48
BAND = (1200.0, 1500.0)
T_SAMP = 1e-3
# (n_t, dm0, ddm, n_dm): uneven lengths (several transform lengths), trial
# counts spanning several kernel blocks, a single trial and a tiny beam
BEAMS = [(3000, 0.0, 1.0, 130), (1000, 2.0, 0.5, 64), (5000, 0.0, 0.25, 2100),
         (2048, 5.0, 0.0, 1), (700, 0.0, 2.0, 300)]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fdd.build()


def _common(output, **kw):
    dnu = (BAND[1] - BAND[0]) / N_CHAN
    d = dict(n_chan=N_CHAN, nu_lo_mhz=BAND[0] + 0.5 * dnu, dnu_mhz=dnu, t_samp_s=T_SAMP,
             in_dtype=fdd.FDD_IN_F32, output=output, chunk_len=0)
    d.update(kw)
    return d


def _inputs(seed=21):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((n_t, N_CHAN)).astype(np.float32) for n_t, *_ in BEAMS]


def _oracle(x, beam):
    n_t, dm0, ddm, n_dm = beam
    dnu = (BAND[1] - BAND[0]) / N_CHAN
    nu = BAND[0] + 0.5 * dnu + dnu * np.arange(N_CHAN)
    d = oracle.delays(nu, dm0 + ddm * np.arange(n_dm), T_SAMP)
    geo = oracle.geometry(n_t, 0, d)
    X = oracle.spectra(x.T.astype(np.float64), geo, 0)
    return oracle.fdd_bins(X, np.arange(geo.K), geo.L, d)


_REFS = {}


def _refs(xs):
    if "r" not in _REFS:
        _REFS["r"] = [_oracle(x, b) for x, b in zip(xs, BEAMS)]
    return _REFS["r"]


def _run(batch, xs, output):
    d_in = torch.from_numpy(np.concatenate([x.ravel() for x in xs])).cuda()
    n = batch.info["out_elems"]
    out = torch.zeros((n, 2) if output == fdd.FDD_OUT_SPECTRA else (n,), device="cuda")
    batch.execute(d_in, out)
    torch.cuda.synchronize()
    o = out.cpu().numpy().astype(np.float64)
    if output == fdd.FDD_OUT_SPECTRA:
        o = o[:, 0] + 1j * o[:, 1]
    return o, d_in, out


def _check(batch, o, refs, output):
    for i, (b, ref) in enumerate(zip(BEAMS, refs)):
        K = ref.shape[1]
        got = o[batch.out_offsets[i]: batch.out_offsets[i] + b[3] * K].reshape(b[3], K)
        want = ref if output == fdd.FDD_OUT_SPECTRA else np.abs(ref) ** 2
        tol = FP32_REL_L2 if output == fdd.FDD_OUT_SPECTRA else 2 * FP32_REL_L2
        assert rel_l2(got, want) <= tol, (i, rel_l2(got, want))


@pytest.mark.parametrize("output", [fdd.FDD_OUT_SPECTRA, fdd.FDD_OUT_POWER])
def test_batch_matches_oracle(output):
    xs = _inputs()
    with fdd.Batch(BEAMS, autotune=False, **_common(output)) as batch:
        assert batch.info["n_waves"] == 1
        assert batch.info["mac_variant"] == fdd.FDD_MAC_G12_4X8
        # the three-product tile runs a beam's ragged last block (<= 1024
        # trials) as wide items (eight bins, 1024 trials) in the same persistent launch
        assert batch.info["tail_variant"] == -1
        assert batch.in_offsets == list(np.cumsum([0] + [b[0] * N_CHAN for b in BEAMS])[:-1])
        o, _, _ = _run(batch, xs, output)
    _check(batch, o, _refs(xs), output)


@pytest.mark.parametrize("variant", [fdd.FDD_MAC_W12_8X8, fdd.FDD_MAC_Q12_8X8, fdd.FDD_MAC_Q_4X4])
def test_batch_other_tiles_match_oracle(variant):
    xs = _inputs()
    with fdd.Batch(BEAMS, autotune=False, mac_variant=variant + 1,
                   **_common(fdd.FDD_OUT_SPECTRA)) as batch:
        assert batch.info["mac_variant"] == variant
        if variant == fdd.FDD_MAC_W12_8X8:
            # its last blocks of <= 1024 trials go to a second launch on 128-trial blocks
            assert batch.info["tail_variant"] == fdd.FDD_MAC_Q_4X4
        o, _, _ = _run(batch, xs, fdd.FDD_OUT_SPECTRA)
    _check(batch, o, _refs(xs), fdd.FDD_OUT_SPECTRA)


def test_batch_waves_graph_replay_and_rebind():
    """A small workspace splits the batch into waves; replaying the captured graph
    gives identical results; new buffers are re-captured correctly."""
    xs = _inputs()
    # fixed part (header): staging n_chan x max L floats, tables, 64 MiB reserve;
    # a pool of 1.7 MB then holds beams {0,1}, {2}, {3,4}
    fixed = 4 * N_CHAN * 8192 + 16 * N_CHAN * len(BEAMS) + (64 << 20)
    with fdd.Batch(BEAMS, autotune=False, mac_variant=fdd.FDD_MAC_Q_4X8 + 1,
                   workspace_limit=fixed + 1_700_000,
                   **_common(fdd.FDD_OUT_SPECTRA)) as batch:
        assert batch.info["n_waves"] == 3
        assert batch.info["tail_variant"] == -1  # 1024-trial blocks leave no tail
        o1, d_in, out = _run(batch, xs, fdd.FDD_OUT_SPECTRA)
        out.zero_()
        batch.execute(d_in, out)                 # graph replay
        torch.cuda.synchronize()
        o2 = out.cpu().numpy().astype(np.float64)
        assert np.array_equal(o1, o2[:, 0] + 1j * o2[:, 1])
        o3, _, _ = _run(batch, xs, fdd.FDD_OUT_SPECTRA)  # new buffers: re-capture
        assert np.array_equal(o1, o3)
    _check(batch, o1, _refs(xs), fdd.FDD_OUT_SPECTRA)


def test_batch_autotune_picks_a_timed_candidate():
    xs = _inputs()
    with fdd.Batch(BEAMS, autotune=True, **_common(fdd.FDD_OUT_POWER)) as batch:
        timed = batch.info["autotune_ms"]
        assert len(timed) >= 2 and all(t > 0 for t in timed.values())
        chosen = fdd.MAC_VARIANT_NAMES[batch.info["mac_variant"]]
        assert chosen in timed and timed[chosen] == min(timed.values())
        o, _, _ = _run(batch, xs, fdd.FDD_OUT_POWER)
    _check(batch, o, _refs(xs), fdd.FDD_OUT_POWER)


# (n_t, dm0, ddm, n_dm, chunk_len): beams in overlap-save chunks of their own
# lengths next to a whole-series beam (largest delays 132, 34, 533 and 607
# samples), chunk counts 4, 1, 3 and 1; the first beam's 1300 trials end in
# a 1024-trial and a 512-trial wide item of the G12 tile
CHUNKED = [(3000, 0.0, 0.1, 1300, 1024), (1000, 2.0, 0.5, 64, 0), (5000, 0.0, 0.25, 2100, 2048),
           (700, 0.0, 2.0, 300, 1024)]


def _oracle_chunks(x, beam):
    n_t, dm0, ddm, n_dm, chunk = beam
    dnu = (BAND[1] - BAND[0]) / N_CHAN
    nu = BAND[0] + 0.5 * dnu + dnu * np.arange(N_CHAN)
    d = oracle.delays(nu, dm0 + ddm * np.arange(n_dm), T_SAMP)
    geo = oracle.geometry(n_t, chunk, d)
    return [oracle.fdd_bins(oracle.spectra(x.T.astype(np.float64), geo, c), np.arange(geo.K),
                            geo.L, d) for c in range(geo.n_chunks)]


@pytest.mark.parametrize("variant", [0, fdd.FDD_MAC_W12_8X8 + 1])
def test_batch_chunked_beams_match_oracle(variant):
    """Beams with their own overlap-save chunk lengths: every chunk of every
    beam is a work set of the one persistent launch, output [chunk][dm][bin]
    per beam, each chunk against the oracle's spectra of that chunk; the
    streamed execute delivers one block per (beam, chunk) with the same bytes."""
    rng = np.random.default_rng(33)
    xs = [rng.standard_normal((b[0], N_CHAN)).astype(np.float32) for b in CHUNKED]
    refs = [_oracle_chunks(x, b) for x, b in zip(xs, CHUNKED)]
    assert [len(r) for r in refs] == [4, 1, 3, 1]
    with fdd.Batch(CHUNKED, autotune=False, mac_variant=variant,
                   **_common(fdd.FDD_OUT_POWER)) as batch:
        assert batch.info["out_elems"] == sum(len(r) * r[0].size for r in refs)
        d_in = torch.from_numpy(np.concatenate([x.ravel() for x in xs])).cuda()
        out = torch.zeros(batch.info["out_elems"], device="cuda")
        batch.execute(d_in, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy().astype(np.float64)
        for i, ref in enumerate(refs):
            for c, r in enumerate(ref):
                off = batch.out_offsets[i] + c * r.size
                got = o[off: off + r.size].reshape(r.shape)
                assert rel_l2(got, np.abs(r) ** 2) <= 2 * FP32_REL_L2, (i, c)
        got = torch.full_like(out, float("nan"))
        seen = []

        def source(beam, t0, n, d_window, ready, s):
            fdd.memcpy_async(d_window, d_in.data_ptr() + 4 * batch.in_offsets[beam],
                             4 * n * N_CHAN, s)

        def sink(blk, s):
            b, c = blk["beam_first"], blk["chunk"]
            seen.append((b, c))
            n = blk["n_dm"] * blk["row_len"]
            fdd.memcpy_async(got.data_ptr() + 4 * (batch.out_offsets[b] + c * n), blk["d_data"],
                             4 * n, s)
            return None

        batch.execute_stream(source, sink, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert seen == [(b, c) for b, r in enumerate(refs) for c in range(len(r))]
        assert torch.equal(got, out)


def test_batch_rejects_what_it_does_not_do():
    with pytest.raises(fdd.FddError) as e:
        fdd.Batch(BEAMS, **_common(fdd.FDD_OUT_TIME))
    assert e.value.status == fdd.FDD_ERR_UNSUPPORTED
    with pytest.raises(fdd.FddError) as e:
        fdd.Batch(BEAMS, **_common(fdd.FDD_OUT_POWER, chunk_len=1024))
    assert e.value.status == fdd.FDD_ERR_UNSUPPORTED
    with pytest.raises(fdd.FddError) as e:
        fdd.Batch([(100, -1.0, 1.0, 4)], **_common(fdd.FDD_OUT_POWER))
    assert e.value.status == fdd.FDD_ERR_INVALID_ARG


@pytest.mark.parametrize("variant,limit", [(0, 0), (fdd.FDD_MAC_W12_8X8 + 1, 0),
                                           (fdd.FDD_MAC_Q_4X8 + 1, "waves")])
def test_batch_streamed_equals_resident_execute(variant, limit):
    """fdd_batch_execute_stream (a window per beam from the source, one block
    per beam to the sink, output slots per wave) gives bit for bit what the
    resident execute gives: the three-product tile, the warp-specialised tile
    with its tail launch, and several waves."""
    xs = _inputs()
    kw = {}
    if limit == "waves":
        kw["workspace_limit"] = 4 * N_CHAN * 8192 + 16 * N_CHAN * len(BEAMS) + (64 << 20) + 1_700_000
    with fdd.Batch(BEAMS, autotune=False, mac_variant=variant,
                   **_common(fdd.FDD_OUT_POWER, **kw)) as batch:
        if limit == "waves":
            assert batch.info["n_waves"] == 3
        ref, d_in, _ = _run(batch, xs, fdd.FDD_OUT_POWER)
        got = torch.full((batch.info["out_elems"],), float("nan"), device="cuda")
        seen = []

        def source(beam, t0, n, d_window, ready, s):
            assert t0 == 0 and n == BEAMS[beam][0]
            fdd.memcpy_async(d_window, d_in.data_ptr() + 4 * batch.in_offsets[beam],
                             4 * n * N_CHAN, s)

        def sink(blk, s):
            seen.append(blk["beam_first"])
            b = blk["beam_first"]
            fdd.memcpy_async(got.data_ptr() + 4 * batch.out_offsets[b], blk["d_data"],
                             4 * blk["n_dm"] * blk["row_len"], s)
            return None

        for _ in range(2):  # the second call reuses the rings
            seen.clear()
            batch.execute_stream(source, sink, torch.cuda.current_stream())
            torch.cuda.synchronize()
            assert sorted(seen) == list(range(len(BEAMS)))
            assert np.array_equal(got.cpu().numpy().astype(np.float64), ref)


# (n_t, dm0, ddm, n_dm, chunk_len) for the tensor-core batch: three
# whole-series beams of one transform length (4096) and trial grid with
# uneven lengths and trial counts (one plan, run to 300 trials), a beam of
# another length and grid (its own plan), and two chunked beams of one chunk
# length and trial count with 3 and 2 chunks (one plan)
TC_BEAMS = [(3000, 0.0, 1.0, 130, 0), (2500, 0.0, 1.0, 300, 0), (4000, 0.0, 1.0, 64, 0),
            (1000, 2.0, 0.5, 64, 0), (5000, 0.0, 0.25, 2100, 2048),
            (3500, 0.0, 0.25, 2100, 2048)]
TC_REL = 3e-3  # accuracy gate of the tensor-core forms against the FP64 oracle


def _tc_batch_run(batch, d_in, output):
    n = batch.info["out_elems"]
    out = torch.zeros((n, 2) if output == fdd.FDD_OUT_SPECTRA else (n,), device="cuda")
    batch.execute(d_in, out)
    torch.cuda.synchronize()
    return out


def _tc_check(batch, out, refs, output):
    o = out.cpu().numpy().astype(np.float64)
    if output == fdd.FDD_OUT_SPECTRA:
        o = o[:, 0] + 1j * o[:, 1]
    for i, ref in enumerate(refs):
        for c, r in enumerate(ref):
            off = batch.out_offsets[i] + c * r.size
            got = o[off: off + r.size].reshape(r.shape)
            want = r if output == fdd.FDD_OUT_SPECTRA else np.abs(r) ** 2
            tol = TC_REL if output == fdd.FDD_OUT_SPECTRA else 2 * TC_REL
            assert rel_l2(got, want) <= tol, (i, c, rel_l2(got, want))


@pytest.mark.parametrize("output", [fdd.FDD_OUT_SPECTRA, fdd.FDD_OUT_POWER])
def test_tensor_core_batch_matches_oracle(output):
    """Beams grouped by shared phasors into FP16 tensor-core plans: every beam,
    chunk and trial against the oracle; streamed, the same bytes; with plans
    made per execute (a workspace limit below their sum), the oracle again."""
    rng = np.random.default_rng(44)
    xs = [rng.standard_normal((b[0], N_CHAN)).astype(np.float32) for b in TC_BEAMS]
    refs = [_oracle_chunks(x, b) for x, b in zip(xs, TC_BEAMS)]
    assert [len(r) for r in refs] == [1, 1, 1, 1, 3, 2]
    d_in = torch.from_numpy(np.concatenate([x.ravel() for x in xs])).cuda()
    kw = _common(output, precision=fdd.FDD_PREC_FP16)
    with fdd.Batch(TC_BEAMS, **kw) as batch:
        assert batch.info["mac_variant"] == fdd.FDD_MAC_TC
        assert batch.info["n_waves"] == 3  # plans
        held = batch.info["workspace_bytes"]
        assert held > 0  # kept between executes
        out = _tc_batch_run(batch, d_in, output)
        _tc_check(batch, out, refs, output)
        # streamed: one block per (beam, chunk, block of trials)
        got = torch.full_like(out, float("nan"))
        esz = 8 if output == fdd.FDD_OUT_SPECTRA else 4

        def source(beam, t0, n, d_window, ready, s):
            assert 0 <= t0 and t0 + n <= TC_BEAMS[beam][0]
            fdd.memcpy_async(d_window,
                             d_in.data_ptr() + 4 * (batch.in_offsets[beam] + t0 * N_CHAN),
                             4 * n * N_CHAN, s)

        def sink(blk, s):
            b, c = blk["beam_first"], blk["chunk"]
            assert blk["dm_first"] + blk["n_dm"] <= TC_BEAMS[b][3]
            K = blk["row_len"]
            dst = batch.out_offsets[b] + (c * TC_BEAMS[b][3] + blk["dm_first"]) * K
            fdd.memcpy_async(got.data_ptr() + esz * dst, blk["d_data"], esz * blk["n_dm"] * K, s)
            return None

        batch.execute_stream(source, sink, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert torch.equal(got, out)
    # a limit below the plans' sum, above each one's least workspace: the
    # plans share one block for their per-call buffers (their trial blocks
    # may differ); twice, the second call reusing the block
    with fdd.Batch(TC_BEAMS, workspace_limit=held // 2, **kw) as batch:
        assert 0 < batch.info["workspace_bytes"] < held
        first = _tc_batch_run(batch, d_in, output)
        _tc_check(batch, first, refs, output)
        assert torch.equal(_tc_batch_run(batch, d_in, output), first)


@pytest.mark.parametrize("n_chan", [6000, 9000])
def test_batch_many_channels_take_a_tile_that_fits(n_chan):
    """6000 channels: the G12 tile runs with a two-stage ring; 9000: its ring
    leaves the phase table no room, so the batch takes the next tile that
    fits one CTA per SM.  Both match the oracle."""
    beams = [(300, 0.0, 0.5, 64), (200, 1.0, 0.25, 40)]
    lo, hi = 1200.0, 1500.0
    dnu = (hi - lo) / n_chan
    rng = np.random.default_rng(8)
    xs = [rng.standard_normal((b[0], n_chan)).astype(np.float32) for b in beams]
    with fdd.Batch(beams, autotune=False, n_chan=n_chan, nu_lo_mhz=lo + 0.5 * dnu,
                   dnu_mhz=dnu, t_samp_s=T_SAMP, in_dtype=fdd.FDD_IN_F32,
                   output=fdd.FDD_OUT_SPECTRA, chunk_len=0) as batch:
        assert (batch.info["mac_variant"] == fdd.FDD_MAC_G12_4X8) == (n_chan < 8382)
        d_in = torch.from_numpy(np.concatenate([x.ravel() for x in xs])).cuda()
        out = torch.zeros((batch.info["out_elems"], 2), device="cuda")
        batch.execute(d_in, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy().astype(np.float64)
        o = o[:, 0] + 1j * o[:, 1]
        nu = lo + 0.5 * dnu + dnu * np.arange(n_chan)
        for i, (x, (n_t, dm0, ddm, n_dm)) in enumerate(zip(xs, beams)):
            d = oracle.delays(nu, dm0 + ddm * np.arange(n_dm), T_SAMP)
            geo = oracle.geometry(n_t, 0, d)
            ref = oracle.fdd_bins(oracle.spectra(x.T.astype(np.float64), geo, 0),
                                  np.arange(geo.K), geo.L, d)
            got = o[batch.out_offsets[i]: batch.out_offsets[i] + ref.size].reshape(ref.shape)
            assert rel_l2(got, ref) <= FP32_REL_L2, (i, rel_l2(got, ref))

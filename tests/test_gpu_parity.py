"""GPU parity: the CUDA library through its C ABI against the CPU oracle.

Counts are integers, so every comparison is bit-exact.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fb():
    from paper_0905_2203_gb300 import build as b
    b.build()
    from paper_0905_2203_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(fb):
    c = fb.Context(0)
    yield c
    c.close()


def oracle_counts(ty, tm, offs, ct, lo, hi):
    c, _ = oracle.count_many(ty, tm, offs, ct, lo, hi)
    return c.astype(np.int64)


def gpu_counts(fb, ctx, st, offs, ct, lo, hi):
    return ctx.count_episodes(st, fb.Cands(offs, ct, lo, hi)).astype(np.int64)


def test_version_and_symbols(fb):
    assert "sm_103a" in fb.version()


def test_level1_frequency(fb, ctx):
    s, _ = synth.c1_tiny()
    st = ctx.load_stream(s.types, s.times, s.n_types)
    f = st.freq()
    for a in range(s.n_types):
        assert f[a] == oracle.count_fsm(s.types, s.times, [a], [], [])
    st.free()


def test_stream_validation_errors(fb, ctx):
    ty = np.array([0, 1, 0], np.uint16)
    with pytest.raises(fb.FemError) as e:
        ctx.load_stream(ty, np.array([0, 2, 1], np.int32), 2)
    assert e.value.status == fb.FEM_ERR_UNSORTED
    ok = ctx.load_stream(np.array([0, 1, 0], np.uint16), np.array([0, 1, 1], np.int32), 2)  # ties, distinct types
    ok.free()
    with pytest.raises(fb.FemError) as e:
        ctx.load_stream(np.array([0, 1, 0], np.uint16), np.array([0, 1, 0], np.int32), 2)
    assert e.value.status == fb.FEM_ERR_UNSORTED
    with pytest.raises(fb.FemError) as e:
        ctx.load_stream(np.array([0, 1, 1], np.uint16), np.array([0, 5, 5], np.int32), 2)
    assert e.value.status == fb.FEM_ERR_DUP
    with pytest.raises(fb.FemError) as e:
        ctx.load_stream(np.array([0, 2], np.uint16), np.array([0, 1], np.int32), 2)
    assert e.value.status == fb.FEM_ERR_INVAL
    for nt in (32, 128, 12288, 12289):  # a type just past the alphabet, every histogram layout
        with pytest.raises(fb.FemError) as e:
            ctx.load_stream(np.array([0, nt, 1], np.uint16), np.array([0, 1, 2], np.int32), nt)
        assert e.value.status == fb.FEM_ERR_INVAL
    with pytest.raises(fb.FemError) as e:
        ctx.load_stream(np.array([0, 1], np.uint16), np.array([-3, 1], np.int32), 2)
    assert e.value.status == fb.FEM_ERR_RANGE
    with pytest.raises(fb.FemError) as e:
        ctx.load_stream(np.array([0, 1], np.uint16), np.array([5, 2**31 - 1], np.int32), 2)
    assert e.value.status == fb.FEM_ERR_RANGE


def test_candidate_validation_errors(fb, ctx):
    s, _ = synth.c1_tiny()
    st = ctx.load_stream(s.types, s.times, s.n_types)
    bad = [
        (np.array([0, 2]), np.array([0, 1]), np.array([5]), np.array([5])),   # lo == hi
        (np.array([0, 2]), np.array([0, 1]), np.array([-1]), np.array([5])),  # lo < 0
        (np.array([0, 2]), np.array([0, 40]), np.array([0]), np.array([5])),  # type >= n_types
    ]
    for offs, ct, lo, hi in bad:
        with pytest.raises(fb.FemError) as e:
            ctx.count_episodes(st, fb.Cands(offs, ct, lo, hi))
        assert e.value.status == fb.FEM_ERR_INVAL
    st.free()


def test_golden_cases_on_gpu(fb, ctx):
    from golden_io import all_cases
    for name, ty, tm, (E, lo, hi), expect in all_cases():
        st = ctx.load_stream(ty, tm, int(max(ty.max(initial=0), max(E)) + 1))
        offs = np.array([0, len(E)], np.int64)
        got = ctx.count_episodes(st, fb.Cands(offs, np.array(E, np.uint16), np.array(lo, np.int32),
                                              np.array(hi, np.int32)))
        assert int(got[0]) == expect, name
        st.free()


@pytest.mark.parametrize("kernel", [0, 1, 2, 4, 5, 6, 7])
@pytest.mark.parametrize("segments,lanes,tile", [(0, 0, 0), (1, 32, 256), (7, 64, 512), (64, 256, 1024),
                                                  (300, 96, 4096)])
def test_random_tiny_streams(fb, ctx, segments, lanes, tile, kernel):
    """Many random episodes (sizes 1-6, lower bounds 0..6) over random streams
    with frequent equal times, under several segment / CTA / tile settings,
    with the tiled (1) and the sparse (2) counting kernel, with grid-wide
    local tracking (4: latest starts; 5 / 6: occurrence lists compacted by
    atomics / count-scan-write; segment settings do not apply to them) and
    with warp-per-item local tracking (0: episodes with a common prefix share
    its steps; 7: one item per episode; segments apply to both)."""
    r = synth.Rng(99, segments + 7)
    ctx.set_tuning(lanes_per_cta=lanes, segments=segments, tile_events=tile, kernel=kernel)
    try:
        for trial in range(6):
            n_types = int(r.integers(2, 7, 1)[0])
            n = int(r.integers(50, 5000, 1)[0])
            ty, tm = synth.tiny_random_stream(1000 + trial, n, n_types, int(r.integers(n // 3 + 5, 3 * n, 1)[0]))
            nc = 700
            sizes = r.integers(1, 6, nc)
            offs = np.zeros(nc + 1, np.int64)
            offs[1:] = np.cumsum(sizes)
            ct = r.integers(0, n_types - 1, int(offs[-1])).astype(np.uint16)
            ne = int(offs[-1]) - nc
            lo = r.integers(0, 6, ne).astype(np.int32)
            hi = (lo + r.integers(1, 12, ne)).astype(np.int32)
            st = ctx.load_stream(ty, tm, n_types)
            got = gpu_counts(fb, ctx, st, offs, ct, lo, hi)
            want = oracle_counts(ty, tm, offs, ct, lo, hi)
            bad = np.nonzero(got != want)[0]
            assert bad.size == 0, (trial, bad[:5], got[bad[:5]], want[bad[:5]])
            st.free()
    finally:
        ctx.reset_tuning()


@pytest.mark.parametrize("kernel", [0, 1, 2, 4, 5, 6, 7])
@pytest.mark.parametrize("segments", [0, 33, 1000, 4099])
def test_few_episodes_many_segments(fb, ctx, segments, kernel):
    """Few episodes over the 1M-event mid stream cut into up to ~4k segments:
    each episode's count is stitched from thousands of segment records
    (several per lane of the stitch warp, with a ragged last run); with the
    automatic choice (0) and no segment override these few episodes over a
    long recording go to local tracking."""
    s, cfg = synth.c2_mid()
    st = ctx.load_stream(s.types, s.times, s.n_types)
    offs, ct, lo, hi = synth.random_candidates(0xFE0102, 48, s.n_types, 2, 6, cfg["bins"], s.chains, 0.5)
    want = oracle_counts(s.types, s.times, offs, ct, lo, hi)
    ctx.set_tuning(segments=segments, kernel=kernel)
    try:
        got = gpu_counts(fb, ctx, st, offs, ct, lo, hi)
    finally:
        ctx.reset_tuning()
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:5]
    assert want.max() > 0
    st.free()


@pytest.mark.parametrize("track_last", [1, 2])
@pytest.mark.parametrize("kernel,segments", [(0, 0), (7, 0), (0, 7), (7, 300)])
def test_track_last_node_by_events_and_by_entries(fb, ctx, kernel, segments, track_last):
    """The warp-per-item kernel's last node driven by the last node's events
    (1) or by the entries of the node before it (2), on tiny streams with
    many equal times, a bursty stream with the 4-bin set, and the mid stream
    cut into segments (entries whose interval starts before the segment)."""
    ctx.set_tuning(kernel=kernel, segments=segments, track_last=track_last)
    try:
        r = synth.Rng(77, segments + 3)
        for trial in range(4):
            n_types = int(r.integers(2, 7, 1)[0])
            n = int(r.integers(50, 5000, 1)[0])
            ty, tm = synth.tiny_random_stream(2000 + trial, n, n_types, int(r.integers(n // 3 + 5, 3 * n, 1)[0]))
            nc = 500
            sizes = r.integers(2, 6, nc)
            offs = np.zeros(nc + 1, np.int64)
            offs[1:] = np.cumsum(sizes)
            ct = r.integers(0, n_types - 1, int(offs[-1])).astype(np.uint16)
            ne = int(offs[-1]) - nc
            lo = r.integers(0, 6, ne).astype(np.int32)
            hi = (lo + r.integers(1, 12, ne)).astype(np.int32)
            st = ctx.load_stream(ty, tm, n_types)
            got = gpu_counts(fb, ctx, st, offs, ct, lo, hi)
            want = oracle_counts(ty, tm, offs, ct, lo, hi)
            bad = np.nonzero(got != want)[0]
            assert bad.size == 0, (trial, bad[:5], got[bad[:5]], want[bad[:5]])
            st.free()
        s = synth.bursty_60(0xFE0007, 120_000)
        st = ctx.load_stream(s.types, s.times, s.n_types)
        offs, ct, lo, hi = synth.random_candidates(0xFE0007, 1500, 60, 2, 6, synth.BINS_4, s.chains, 0.1)
        want = oracle_counts(s.types, s.times, offs, ct, lo, hi)
        assert np.array_equal(gpu_counts(fb, ctx, st, offs, ct, lo, hi), want)
        assert want.max() > 0
        st.free()
        s, cfg = synth.c2_mid()
        st = ctx.load_stream(s.types, s.times, s.n_types)
        offs, ct, lo, hi = synth.random_candidates(0xFE0108, 64, s.n_types, 2, 5, cfg["bins"], s.chains, 0.5)
        want = oracle_counts(s.types, s.times, offs, ct, lo, hi)
        assert np.array_equal(gpu_counts(fb, ctx, st, offs, ct, lo, hi), want)
        st.free()
    finally:
        ctx.reset_tuning()


def test_mining_graph_last_node_by_entries(fb, ctx):
    """The whole-pass mining graph with the last node forced to each side
    gives the oracle miner's levels."""
    s, cfg = synth.c2_mid()
    st = ctx.load_stream(s.types, s.times, s.n_types)
    want = oracle.mine_levelwise(s.types, s.times, s.n_types, cfg["bins"], cfg["threshold"], 4)
    for mode in (1, 2):
        ctx.set_tuning(track_last=mode)
        try:
            res = ctx.mine_levelwise([st], cfg["bins"], [cfg["threshold"]], 4)
            assert res.stats()["graph_tails"] == 1
            for N in range(1, 5):
                eps, counts = res.level(0, N)
                assert list(zip(eps, counts)) == want[N], (mode, N)
            res.free()
        finally:
            ctx.reset_tuning()
    st.free()


def test_c1_random_candidates(fb, ctx):
    s, _ = synth.c1_tiny()
    st = ctx.load_stream(s.types, s.times, s.n_types)
    offs, ct, lo, hi = synth.random_candidates(7, 3000, s.n_types, 2, 8, [(0, 5), (3, 9), (0, 20)],
                                               s.chains, 0.2)
    assert np.array_equal(gpu_counts(fb, ctx, st, offs, ct, lo, hi), oracle_counts(s.types, s.times, offs, ct, lo, hi))
    st.free()


def test_plain_path_matches_oracle(fb, ctx):
    s, _ = synth.c1_tiny()
    st = ctx.load_stream(s.types, s.times, s.n_types)
    offs, ct, lo, hi = synth.random_candidates(8, 800, s.n_types, 1, 6, [(0, 5), (3, 9)], s.chains, 0.2)
    got = ctx.count_episodes_plain(st, fb.Cands(offs, ct, lo, hi)).astype(np.int64)
    assert np.array_equal(got, oracle_counts(s.types, s.times, offs, ct, lo, hi))
    st.free()


def test_upper_bound_is_relaxed_count(fb, ctx):
    s, _ = synth.c1_tiny()
    st = ctx.load_stream(s.types, s.times, s.n_types)
    offs, ct, lo, hi = synth.random_candidates(9, 600, s.n_types, 2, 5, [(2, 5), (3, 9)], s.chains, 0.3)
    ub = ctx.upper_bound(st, fb.Cands(offs, ct, lo, hi)).astype(np.int64)
    exact = oracle_counts(s.types, s.times, offs, ct, lo, hi)
    relaxed = oracle_counts(s.types, s.times, offs, ct, np.zeros_like(lo), hi)
    assert np.all(ub >= exact)
    assert np.array_equal(ub, relaxed)
    st.free()


@pytest.mark.parametrize("kernel", [0, 1, 2, 4, 5, 6, 7])
def test_bursty_stream_mixed_sizes(fb, ctx, kernel):
    """Network bursts (dense windows) with sizes 2-8 and the 4-bin set."""
    s = synth.bursty_60(0xFE0003, 150_000)
    st = ctx.load_stream(s.types, s.times, s.n_types)
    offs, ct, lo, hi = synth.random_candidates(0xFE0003, 3000, 60, 2, 8, synth.BINS_4, s.chains, 0.05)
    want = oracle_counts(s.types, s.times, offs, ct, lo, hi)
    ctx.set_tuning(kernel=kernel)
    try:
        got = gpu_counts(fb, ctx, st, offs, ct, lo, hi)
    finally:
        ctx.reset_tuning()
    assert np.array_equal(got, want)
    assert want.max() > 0
    st.free()


def test_edge_cases(fb, ctx):
    # empty stream
    st = ctx.load_stream(np.zeros(0, np.uint16), np.zeros(0, np.int32), 3)
    got = ctx.count_episodes(st, fb.Cands(np.array([0, 2, 3]), np.array([0, 1, 2], np.uint16),
                                          np.array([0], np.int32), np.array([4], np.int32)))
    assert got.tolist() == [0, 0]
    st.free()
    # zero candidates
    s, _ = synth.c1_tiny()
    st = ctx.load_stream(s.types, s.times, s.n_types)
    got = ctx.count_episodes(st, fb.Cands(np.array([0], np.int64), np.zeros(0, np.uint16),
                                          np.zeros(0, np.int32), np.zeros(0, np.int32)))
    assert got.size == 0
    # maximum episode size, repeated types, single event stream
    E = np.array([3, 3, 7, 3] * 4, np.uint16)
    offs = np.array([0, 16], np.int64)
    lo = np.zeros(15, np.int32)
    hi = np.full(15, 40, np.int32)
    got = ctx.count_episodes(st, fb.Cands(offs, E, lo, hi))
    assert int(got[0]) == oracle.count_fsm(s.types, s.times, E, lo, hi)
    st.free()
    st = ctx.load_stream(np.array([2], np.uint16), np.array([0], np.int32), 3)
    got = ctx.count_episodes(st, fb.Cands(np.array([0, 1, 3]), np.array([2, 2, 1], np.uint16),
                                          np.array([0], np.int32), np.array([1], np.int32)))
    assert got.tolist() == [1, 0]
    st.free()


def test_device_pointers_with_torch(fb, ctx):
    torch = pytest.importorskip("torch")
    s, _ = synth.c1_tiny()
    dev = torch.device("cuda:0")
    st = ctx.load_stream(torch.from_numpy(s.types.view(np.int16)).to(dev),
                         torch.from_numpy(s.times).to(dev), s.n_types)
    offs, ct, lo, hi = synth.random_candidates(12, 400, s.n_types, 2, 4, [(0, 5)], s.chains, 0.3)
    c = fb.Cands(torch.from_numpy(offs).to(dev), torch.from_numpy(ct.view(np.int16)).to(dev),
                 torch.from_numpy(lo).to(dev), torch.from_numpy(hi).to(dev))
    out = torch.zeros(400, dtype=torch.int32, device=dev)
    ctx.count_episodes(st, c, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.array_equal(got, oracle_counts(s.types, s.times, offs, ct, lo, hi))
    st.free()


def test_count_batch_multi_recording(fb, ctx):
    recs = synth.c4_recordings(0xFE0004, n_rec=6, n_lo=2e3, n_hi=6e4)
    streams = [ctx.load_stream(s.types, s.times, s.n_types) for s, _ in recs]
    offs_l, ct_l, lo_l, hi_l, rid = [], [], [], [], []
    base = 0
    r = synth.Rng(3, 3)
    order = r.integers(0, len(recs) - 1, 1200)
    per = {}
    for k, (s, cfg) in enumerate(recs):
        per[k] = synth.random_candidates(40 + k, 200, 60, 2, 6, synth.BINS_4, s.chains, 0.3)
    # interleave recordings in the candidate order
    cursor = {k: 0 for k in per}
    offs = [0]
    for k in order:
        o, t, l, h = per[k]
        c = cursor[k] % 200
        cursor[k] += 1
        a, b = int(o[c]), int(o[c + 1])
        ct_l.extend(t[a:b]); lo_l.extend(l[a - c:b - c - 1]); hi_l.extend(h[a - c:b - c - 1])
        offs.append(offs[-1] + b - a)
        rid.append(k)
    offs = np.array(offs, np.int64)
    ct = np.array(ct_l, np.uint16); lo = np.array(lo_l, np.int32); hi = np.array(hi_l, np.int32)
    rid = np.array(rid, np.uint32)
    got = ctx.count_batch(streams, fb.Cands(offs, ct, lo, hi), rid).astype(np.int64)
    for k, (s, _) in enumerate(recs):
        idx = np.nonzero(rid == k)[0]
        sub_offs = [0]
        st_, sl, sh = [], [], []
        for c in idx:
            a, b = int(offs[c]), int(offs[c + 1])
            st_.extend(ct[a:b]); sl.extend(lo[a - c:b - c - 1]); sh.extend(hi[a - c:b - c - 1])
            sub_offs.append(sub_offs[-1] + b - a)
        want = oracle_counts(s.types, s.times, np.array(sub_offs), np.array(st_, np.uint16),
                             np.array(sl, np.int32), np.array(sh, np.int32))
        assert np.array_equal(got[idx], want), k
    for st in streams:
        st.free()


def _mine_compare(fb, ctx, streams_np, bins, thrs, max_size):
    streams = [ctx.load_stream(s.types, s.times, s.n_types) for s in streams_np]
    res = ctx.mine_levelwise(streams, bins, thrs, max_size)
    for k, s in enumerate(streams_np):
        want = oracle.mine_levelwise(s.types, s.times, s.n_types, bins, thrs[k], max_size)
        for N in range(1, max_size + 1):
            eps, counts = res.level(k, N)
            assert list(zip(eps, counts)) == want[N], (k, N)
    st = res.stats()
    res.free()
    for x in streams:
        x.free()
    return st


def test_mine_levelwise_c1(fb, ctx):
    s, cfg = synth.c1_tiny()
    _mine_compare(fb, ctx, [s], cfg["bins"], [cfg["threshold"]], cfg["max_size"])


def test_mine_levelwise_c2_short(fb, ctx):
    s, cfg = synth.c2_mid(duration_s=60.0)
    thr = int(0.0025 * s.n)
    _mine_compare(fb, ctx, [s], cfg["bins"], [thr], cfg["max_size"])


def test_mine_levelwise_multi_recording(fb, ctx):
    recs = synth.c4_recordings(0xFE0004, n_rec=5, n_lo=5e3, n_hi=4e4)
    _mine_compare(fb, ctx, [s for s, _ in recs], synth.BINS_4, [cfg["threshold"] for _, cfg in recs], 5)


def test_large_alphabet_and_hashed_filter(fb, ctx):
    """Alphabets above 128 types (shared-memory warp filter) and above 4096
    (hashed filter bits): counts unchanged."""
    for n_types in (300, 5000):
        r = synth.Rng(n_types, 4)
        ty, tm = synth.tiny_random_stream(n_types, 40000, n_types, 60000)
        # concentrate on a few types so counts are non-trivial
        hot = r.integers(0, n_types - 1, 12)
        ty = np.where(r.uniform(ty.size) < 0.6, hot[r.integers(0, 11, ty.size)], ty).astype(np.uint16)
        key = np.unique(tm.astype(np.int64) * 65536 + ty)
        tm = (key // 65536).astype(np.int32)
        ty = (key % 65536).astype(np.uint16)
        nc = 1500
        sizes = r.integers(2, 5, nc)
        offs = np.zeros(nc + 1, np.int64)
        offs[1:] = np.cumsum(sizes)
        ct = hot[r.integers(0, 11, int(offs[-1]))].astype(np.uint16)
        ne = int(offs[-1]) - nc
        lo = r.integers(0, 20, ne).astype(np.int32)
        hi = (lo + r.integers(1, 60, ne)).astype(np.int32)
        st = ctx.load_stream(ty, tm, n_types)
        got = gpu_counts(fb, ctx, st, offs, ct, lo, hi)
        want = oracle_counts(ty, tm, offs, ct, lo, hi)
        assert np.array_equal(got, want), n_types
        assert want.max() > 0
        st.free()


def test_prepass_prunes_but_never_changes_results(fb, ctx):
    """The level-2 upper-bound pre-pass drops candidates (C2-like stream) and
    the frequent sets are identical with it disabled."""
    s, cfg = synth.c2_mid(duration_s=40.0)
    thr = int(0.0025 * s.n)
    st = ctx.load_stream(s.types, s.times, s.n_types)
    res = ctx.mine_levelwise([st], cfg["bins"], [thr], 4)
    stats_on = res.stats()
    on = [res.level(0, N) for N in range(1, 5)]
    res.free()
    ctx.set_tuning(prepass=-1)
    try:
        res = ctx.mine_levelwise([st], cfg["bins"], [thr], 4)
        stats_off = res.stats()
        off = [res.level(0, N) for N in range(1, 5)]
        res.free()
    finally:
        ctx.reset_tuning()
    assert on == off
    assert stats_on["candidates_pruned"] > 0 and stats_off["candidates_pruned"] == 0
    assert stats_on["episode_events"] == stats_off["episode_events"]
    assert stats_on["counted_episode_events"] < stats_off["counted_episode_events"]
    st.free()


@pytest.mark.parametrize("relaxed", [False, True])
def test_local_tracking_shared_prefixes(fb, ctx, relaxed):
    """Local tracking shares the steps of episodes with a common prefix (a
    trie over the candidate set): joined level-3 and level-4 candidates (each
    frequent pair prefixes many of them), with repeated candidates mixed in,
    equal the oracle's counts (and, relaxed, its counts with lower bounds 0)."""
    s, cfg = synth.c1_tiny()
    st = ctx.load_stream(s.types, s.times, s.n_types)
    ftypes = list(range(12))
    pairs = oracle.generate_candidates([], 2, ftypes, [(0, 5), (2, 8)])
    l3 = oracle.generate_candidates(pairs[:60], 3, ftypes, [])
    l4 = oracle.generate_candidates(l3[:200], 4, ftypes, [])
    eps = l3[:150] + l4[:100] + l3[:20]
    offs, ct, lo, hi = oracle.to_csr(eps)
    ctx.set_tuning(kernel=4)
    try:
        if relaxed:
            got = ctx.upper_bound(st, fb.Cands(offs, ct, lo, hi)).astype(np.int64)
            want = oracle_counts(s.types, s.times, offs, ct, np.zeros_like(lo), hi)
        else:
            got = gpu_counts(fb, ctx, st, offs, ct, lo, hi)
            want = oracle_counts(s.types, s.times, offs, ct, lo, hi)
    finally:
        ctx.reset_tuning()
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:5]
    assert want.max() > 0
    st.free()


def test_local_tracking_batches_long_step_arrays(fb, ctx):
    """300 two-node episodes over a 2M-event stream (1M events of the end
    type): the step arrays of one launch would hold 3e8 positions, so local
    tracking splits the episodes into batches of at most 2^28 positions;
    counts equal the oracle's."""
    r = synth.Rng(0xBA7C, 1)
    n = 2_000_000
    tm = np.cumsum(r.integers(1, 4, n)).astype(np.int32)
    ty = (np.arange(n) % 2).astype(np.uint16)
    st = ctx.load_stream(ty, tm, 2)
    nc = 300
    offs = np.arange(0, 2 * nc + 1, 2, dtype=np.int64)
    ct = np.tile(np.array([0, 1], np.uint16), nc)
    lo = (np.arange(nc) % 7).astype(np.int32)
    hi = (lo + 1 + np.arange(nc) // 7).astype(np.int32)
    ctx.set_tuning(kernel=4)
    try:
        got = gpu_counts(fb, ctx, st, offs, ct, lo, hi)
    finally:
        ctx.reset_tuning()
    want = oracle_counts(ty, tm, offs, ct, lo, hi)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:5]
    assert want.min() > 0
    st.free()


def test_coarse_prepass_in_level_wise_mining(fb, ctx):
    """Host-driven mining of two recordings of the many-recordings workload
    with the coarse-tick bound on every level >= 3 (prepass = 1): equal to
    the oracle miner, with level >= 3 candidates pruned beyond the level-2
    pair bound's (prepass = 0 keeps only that one)."""
    recs = synth.c4_recordings(n_rec=2)
    streams = [ctx.load_stream(s.types, s.times, s.n_types) for s, _ in recs]
    thr = [c["threshold"] for _, c in recs]
    bins = recs[0][1]["bins"]
    stats = {}
    try:
        for pp in (1, 0):
            ctx.set_tuning(prepass=pp, level_graph=-1)
            res = ctx.mine_levelwise(streams, bins, thr, 4)
            stats[pp] = res.stats()
            for r, (s, c) in enumerate(recs):
                want = oracle.mine_levelwise(s.types, s.times, s.n_types, bins, c["threshold"], 4)
                for N in range(1, 5):
                    eps, counts = res.level(r, N)
                    assert list(zip(eps, counts)) == want[N], (pp, r, N)
            res.free()
    finally:
        ctx.reset_tuning()
        for st in streams:
            st.free()
    assert stats[1]["candidates_pruned"] > stats[0]["candidates_pruned"]
    assert stats[1]["counted_episode_events"] < stats[0]["counted_episode_events"]


@pytest.mark.parametrize("pp", [1, 0])
def test_coarse_bound_inside_mining_graph(fb, ctx, pp):
    """The whole-pass mining graph with the coarse-tick bound on levels >= 3
    (prepass = 1; 0 = without it): pruned candidates skip the count kernels
    and get count 0; the frequent sets of four recordings mined in one call
    equal the oracle miner's and the graph path is the one that ran."""
    recs = synth.c4_recordings(n_rec=4)
    streams = [ctx.load_stream(s.types, s.times, s.n_types) for s, _ in recs]
    thr = [c["threshold"] for _, c in recs]
    bins = recs[0][1]["bins"]
    wants = [oracle.mine_levelwise(s.types, s.times, s.n_types, bins, c["threshold"], 5) for s, c in recs]
    try:
        ctx.set_tuning(prepass=pp)
        for rep in range(2):  # the first call may grow the graph's capacity; the second reuses it
            res = ctx.mine_levelwise(streams, bins, thr, 5)
            st = res.stats()
            assert rep == 0 or st["graph_tails"] >= 1
            for r in range(len(recs)):
                for N in range(1, 6):
                    eps, counts = res.level(r, N)
                    assert list(zip(eps, counts)) == wants[r][N], (pp, rep, r, N)
            res.free()
    finally:
        ctx.reset_tuning()
        for st_ in streams:
            st_.free()


@pytest.mark.parametrize("which", ["c2", "multi"])
def test_level_graph_equals_host_path(fb, ctx, which):
    """Levels >= 3 run as one captured CUDA graph; results equal the
    level-by-level host path, and a repeated call reuses the cached graph."""
    if which == "c2":
        s, cfg = synth.c2_mid(duration_s=80.0)
        streams_np, thrs, bins, L = [s], [int(0.0025 * s.n)], cfg["bins"], cfg["max_size"]
    else:
        recs = synth.c4_recordings(0xFE0004, n_rec=5, n_lo=5e3, n_hi=6e4)
        streams_np = [x for x, _ in recs]
        thrs = [c["threshold"] for _, c in recs]
        bins, L = synth.BINS_4, 6
    streams = [ctx.load_stream(x.types, x.times, x.n_types) for x in streams_np]

    def run():
        res = ctx.mine_levelwise(streams, bins, thrs, L)
        out = [[res.level(k, N) for N in range(1, L + 1)] for k in range(len(streams))]
        st = res.stats()
        res.free()
        return out, st

    g1, s1 = run()
    g2, s2 = run()
    ctx.set_tuning(level_graph=-1)
    try:
        h, sh = run()
    finally:
        ctx.reset_tuning()
    assert g1 == h and g2 == h
    assert sh["graph_tails"] == 0
    if max(sh["levels"], 0) >= 3:
        assert s1["graph_tails"] == 1 and s2["graph_tails"] == 1
        assert s1["levels"] == sh["levels"]
        assert abs(s1["episode_events"] - sh["episode_events"]) < 1e-6 * sh["episode_events"]
    for x in streams:
        x.free()


def test_graph_capacity_overflow_falls_back_then_grows(fb, ctx):
    """More level-2 survivors than the graph's first capacity (4096): the
    first call redoes the mining on the host path (same results), the next
    call captures a graph with the capacity it needed and runs it."""
    ty, tm = synth.tiny_random_stream(0xCA9, 200_000, 64, 2_000_000)
    st = ctx.load_stream(ty, tm, 64)
    bins = [(0, 50), (50, 100), (100, 150), (150, 200)]

    def run():
        res = ctx.mine_levelwise([st], bins, [100], 2)
        out = [res.level(0, N) for N in (1, 2)]
        s = res.stats()
        res.free()
        return out, s

    a, sa = run()
    b, sb = run()
    ctx.set_tuning(level_graph=-1)
    try:
        h, sh = run()
    finally:
        ctx.reset_tuning()
    assert len(h[1][1]) > 4096
    assert a == h and b == h
    assert sa["graph_tails"] == 0 and sb["graph_tails"] == 1
    st.free()


def test_graph_tail_after_host_level2(fb, ctx):
    """With a kernel override the whole-pass graph does not apply: level 2 is
    counted on the host-driven path and levels >= 3 run in the tail graph;
    results equal the level-by-level path."""
    s, cfg = synth.c2_mid(duration_s=80.0)
    thr = int(0.0025 * s.n)
    st = ctx.load_stream(s.types, s.times, s.n_types)

    def run(**tun):
        ctx.set_tuning(**tun)
        try:
            res = ctx.mine_levelwise([st], cfg["bins"], [thr], cfg["max_size"])
            out = [res.level(0, N) for N in range(1, cfg["max_size"] + 1)]
            stt = res.stats()
            res.free()
        finally:
            ctx.reset_tuning()
        return out, stt

    t, stt = run(kernel=2)
    h, sth = run(kernel=2, level_graph=-1)
    assert t == h
    assert stt["graph_tails"] == 1 and sth["graph_tails"] == 0
    assert stt["levels"] == sth["levels"] >= 3
    st.free()


def test_local_tracking_relaxed_bound_and_mining(fb, ctx):
    """Local tracking (kernel 4): the relaxed upper bound equals the oracle's
    count with every lower bound 0, and level-wise mining with it equals the
    oracle miner; edge cases (empty stream, 1-node and 16-node episodes)."""
    s, cfg = synth.c1_tiny()
    st = ctx.load_stream(s.types, s.times, s.n_types)
    offs, ct, lo, hi = synth.random_candidates(19, 400, s.n_types, 1, 6, [(2, 5), (3, 9)], s.chains, 0.3)
    ctx.set_tuning(kernel=4)
    try:
        ub = ctx.upper_bound(st, fb.Cands(offs, ct, lo, hi)).astype(np.int64)
        assert np.array_equal(ub, oracle_counts(s.types, s.times, offs, ct, np.zeros_like(lo), hi))
        res = ctx.mine_levelwise([st], cfg["bins"], [cfg["threshold"]], cfg["max_size"])
        want = oracle.mine_levelwise(s.types, s.times, s.n_types, cfg["bins"], cfg["threshold"], cfg["max_size"])
        for N in range(1, cfg["max_size"] + 1):
            eps, counts = res.level(0, N)
            assert list(zip(eps, counts)) == want[N], N
        res.free()
        E = np.array([3, 3, 7, 3] * 4, np.uint16)
        got = ctx.count_episodes(st, fb.Cands(np.array([0, 16], np.int64), E, np.zeros(15, np.int32),
                                              np.full(15, 40, np.int32)))
        assert int(got[0]) == oracle.count_fsm(s.types, s.times, E, np.zeros(15, np.int32), np.full(15, 40, np.int32))
        st0 = ctx.load_stream(np.zeros(0, np.uint16), np.zeros(0, np.int32), 3)
        got = ctx.count_episodes(st0, fb.Cands(np.array([0, 2, 3]), np.array([0, 1, 2], np.uint16),
                                               np.array([0], np.int32), np.array([4], np.int32)))
        assert got.tolist() == [0, 0]
        st0.free()
    finally:
        ctx.reset_tuning()
    st.free()


@pytest.mark.parametrize("kernel", [5, 6])
def test_occurrence_lists_overflow_falls_back(fb, ctx, kernel):
    """Occurrence-list local tracking: an episode whose partial occurrences
    outgrow the list capacity (one type, 100 successors per event in the
    window: 2e5 x 100^k entries) is recounted with latest starts; a small
    episode next to it stays on the lists; both equal the oracle."""
    n = 200_000
    ty = np.zeros(n, np.uint16)
    ty[1::7] = 1
    tm = np.arange(n, dtype=np.int32)
    st = ctx.load_stream(ty, tm, 2)
    offs = np.array([0, 4, 6], np.int64)
    ct = np.array([0, 0, 0, 0, 0, 1], np.uint16)
    lo = np.array([0, 0, 0, 2], np.int32)
    hi = np.array([100, 100, 100, 9], np.int32)
    want = oracle_counts(ty, tm, offs, ct, lo, hi)
    ctx.set_tuning(kernel=kernel)
    try:
        got = gpu_counts(fb, ctx, st, offs, ct, lo, hi)
        stats = ctx.last_stats()
    finally:
        ctx.reset_tuning()
    assert np.array_equal(got, want), (got, want)
    assert stats["fallback_recounts"] == 1
    assert want.min() > 0
    st.free()


def test_result_level_arrays_match_tuples(fb, ctx):
    """Result.level_arrays (numpy CSR) carries the same episodes and counts
    as Result.level (tuples)."""
    s, cfg = synth.c1_tiny()
    st = ctx.load_stream(s.types, s.times, s.n_types)
    res = ctx.mine_levelwise([st], cfg["bins"], [cfg["threshold"]], cfg["max_size"])
    for N in range(1, cfg["max_size"] + 1):
        eps, counts = res.level(0, N)
        offs, types, lo, hi, cnt = res.level_arrays(0, N)
        assert len(offs) == len(eps) + 1 and cnt.tolist() == counts
        for c, (E, l, h) in enumerate(eps):
            o, p = int(offs[c]), int(offs[c + 1])
            assert tuple(types[o:p].tolist()) == E
            assert tuple(lo[o - c:p - c - 1].tolist()) == l and tuple(hi[o - c:p - c - 1].tolist()) == h
    res.free()
    st.free()


def _chunks(r, n, n_chunks):
    """Random cut points (some chunks empty, cuts between equal times too)."""
    cuts = np.sort(r.integers(0, n, n_chunks - 1))
    return np.concatenate([[0], cuts, [n]]).astype(np.int64)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_session_appends_equal_prefix_counts(fb, ctx, seed):
    """Counting over a growing stream: after every append the session's
    counts equal the oracle's counts over the prefix appended so far, for
    episodes of 1-6 nodes with lower bounds 0..6 over random streams with
    frequent equal times (cuts fall between equal times, some chunks are
    empty)."""
    r = synth.Rng(0x5E55, seed)
    n_types = 5
    n = 4000
    ty, tm = synth.tiny_random_stream(2000 + seed, n, n_types, 3 * n)
    nc = 400
    sizes = r.integers(1, 6, nc)
    offs = np.zeros(nc + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    ct = r.integers(0, n_types - 1, int(offs[-1])).astype(np.uint16)
    ne = int(offs[-1]) - nc
    lo = r.integers(0, 6, ne).astype(np.int32)
    hi = (lo + r.integers(1, 30, ne)).astype(np.int32)
    sess = ctx.session(fb.Cands(offs, ct, lo, hi), n_types)
    try:
        cuts = _chunks(r, len(ty), 12)
        for a, b in zip(cuts[:-1], cuts[1:]):
            sess.append(ty[a:b], tm[a:b])
            got = sess.counts().astype(np.int64)
            want = oracle_counts(ty[:b], tm[:b], offs, ct, lo, hi)
            bad = np.nonzero(got != want)[0]
            assert bad.size == 0, (int(b), bad[:5], got[bad[:5]], want[bad[:5]])
        seen, tail = sess.info()
        assert seen == len(ty) and 0 < tail < len(ty)
    finally:
        sess.close()


def test_session_errors_leave_counts_unchanged(fb, ctx):
    """An append that goes back in time or repeats a (type, time) pair across
    the join is refused and changes nothing; counting then continues exactly.
    A gap longer than every episode's span shrinks the retained tail to the
    events at the last time."""
    s, cfg = synth.c1_tiny()
    offs, ct, lo, hi = synth.random_candidates(21, 300, s.n_types, 1, 5, [(0, 5), (3, 9)], s.chains, 0.3)
    sess = ctx.session(fb.Cands(offs, ct, lo, hi), s.n_types)
    try:
        h = len(s.types) // 2
        sess.append(s.types[:h], s.times[:h])
        before = sess.counts().copy()
        last_t = int(s.times[h - 1])
        with pytest.raises(fb.FemError) as e:
            sess.append(np.array([0], np.uint16), np.array([last_t - 1], np.int32))
        assert e.value.status == fb.FEM_ERR_UNSORTED
        with pytest.raises(fb.FemError) as e:
            sess.append(np.array([s.types[h - 1]], np.uint16), np.array([last_t], np.int32))
        assert e.value.status == fb.FEM_ERR_DUP
        with pytest.raises(fb.FemError) as e:
            sess.append(np.array([s.n_types], np.uint16), np.array([last_t + 1], np.int32))
        assert e.value.status == fb.FEM_ERR_INVAL
        assert np.array_equal(sess.counts(), before)
        sess.append(s.types[h:], s.times[h:])
        assert np.array_equal(sess.counts().astype(np.int64),
                              oracle_counts(s.types, s.times, offs, ct, lo, hi))
        # a long gap: only the events at the last time stay in the tail
        t_end = int(s.times[-1])
        gap_ty = np.array([1, 2], np.uint16)
        gap_tm = np.array([t_end + 10**6, t_end + 10**6], np.int32)
        sess.append(gap_ty, gap_tm)
        assert sess.info()[1] == 2
        all_ty = np.concatenate([s.types, gap_ty])
        all_tm = np.concatenate([s.times, gap_tm])
        assert np.array_equal(sess.counts().astype(np.int64), oracle_counts(all_ty, all_tm, offs, ct, lo, hi))
    finally:
        sess.close()
    with pytest.raises(fb.FemError) as e:
        ctx.session(fb.Cands(np.array([0, 2]), np.array([0, 1], np.uint16), np.array([5], np.int32),
                             np.array([5], np.int32)), 4)
    assert e.value.status == fb.FEM_ERR_INVAL


def test_session_long_stream_device_chunks(fb, ctx):
    """The 1M-event mid stream appended in ten chunks of device tensors, 48
    episodes of 2-6 nodes: counts after the 3rd and the last chunk equal the
    oracle's."""
    import torch
    s, cfg = synth.c2_mid()
    offs, ct, lo, hi = synth.random_candidates(0xFE0102, 48, s.n_types, 2, 6, cfg["bins"], s.chains, 0.5)
    sess = ctx.session(fb.Cands(offs, ct, lo, hi), s.n_types)
    try:
        dty = torch.from_numpy(s.types.astype(np.int16)).cuda()
        dtm = torch.from_numpy(s.times).cuda()
        cuts = np.linspace(0, len(s.types), 11).astype(np.int64)
        for i, (a, b) in enumerate(zip(cuts[:-1], cuts[1:])):
            sess.append(dty[a:b], dtm[a:b])
            if i in (2, 9):
                want = oracle_counts(s.types[:b], s.times[:b], offs, ct, lo, hi)
                assert np.array_equal(sess.counts().astype(np.int64), want), i
                assert want.max() > 0
        out = torch.zeros(48, dtype=torch.int32, device="cuda")
        sess.counts(out)
        assert np.array_equal(out.cpu().numpy().astype(np.int64),
                              oracle_counts(s.types, s.times, offs, ct, lo, hi))
    finally:
        sess.close()


@pytest.mark.parametrize("kernel", [4, 5, 6])
def test_local_tracking_rejects_malformed_candidates(fb, ctx, kernel):
    """Local tracking checks candidates like the per-episode kernels do."""
    s, _ = synth.c1_tiny()
    st = ctx.load_stream(s.types, s.times, s.n_types)
    bad = [
        (np.array([0, 2]), np.array([0, 1]), np.array([5]), np.array([5])),
        (np.array([0, 2]), np.array([0, 1]), np.array([-1]), np.array([5])),
        (np.array([0, 2]), np.array([0, 40]), np.array([0]), np.array([5])),
    ]
    ctx.set_tuning(kernel=kernel)
    try:
        for offs, ct, lo, hi in bad:
            with pytest.raises(fb.FemError) as e:
                ctx.count_episodes(st, fb.Cands(offs, ct, lo, hi))
            assert e.value.status == fb.FEM_ERR_INVAL
    finally:
        ctx.reset_tuning()
    st.free()


def _coarse_case(seed, n_cand, n=8000, n_types=5, t_max=40_000, hi_span=25):
    r = synth.Rng(0xC0A6, seed)
    ty, tm = synth.tiny_random_stream(3000 + seed, n, n_types, t_max)
    sizes = r.integers(1, 6, n_cand)
    offs = np.zeros(n_cand + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    ct = r.integers(0, n_types - 1, int(offs[-1])).astype(np.uint16)
    ne = int(offs[-1]) - n_cand
    lo = r.integers(0, 6, ne).astype(np.int32)
    hi = (lo + r.integers(1, hi_span, ne)).astype(np.int32)
    return ty, tm, offs, ct, lo, hi


def _sub(offs, ct, lo, hi, idx):
    """Candidates idx of a CSR set, as a new CSR set."""
    o2, c2, l2, h2 = [0], [], [], []
    for c in idx:
        a, b = int(offs[c]), int(offs[c + 1])
        c2 += list(ct[a:b])
        l2 += list(lo[a - c:b - c - 1])
        h2 += list(hi[a - c:b - c - 1])
        o2.append(len(c2))
    return (np.array(o2, np.int64), np.array(c2, np.uint16), np.array(l2, np.int32), np.array(h2, np.int32))


@pytest.mark.parametrize("tick", [1, 3, 0])
@pytest.mark.parametrize("n_cand", [300, 12000])
def test_coarse_bound_matches_oracle(fb, ctx, tick, n_cand):
    """Coarse-tick bound: element by element equal to the oracle's definition
    (on a sample when the set is large) and never below the oracle's count;
    40k ticks = 40 warp chunks, so a few candidates run as many stream slices
    (one chunk of warm-up each) and many candidates as whole-stream warps."""
    from oracle import coarse_bound as cb
    ty, tm, offs, ct, lo, hi = _coarse_case(tick + n_cand, n_cand)
    st = ctx.load_stream(ty, tm, 5)
    ub, w = ctx.upper_bound_coarse(st, fb.Cands(offs, ct, lo, hi), tick)
    assert w == (tick if tick else cb.default_tick(int(hi.max())))
    ub = ub.astype(np.int64)
    assert np.all(ub >= oracle_counts(ty, tm, offs, ct, lo, hi))
    sample = np.arange(n_cand) if n_cand <= 300 else synth.Rng(5, n_cand).integers(0, n_cand - 1, 300)
    want = cb.coarse_ub_many(ty, tm, *_sub(offs, ct, lo, hi, sample), w)
    bad = np.nonzero(ub[sample] != want)[0]
    assert bad.size == 0, (bad[:5], ub[sample][bad[:5]], want[bad[:5]])
    st.free()


def test_coarse_bound_edges_and_full_size(fb, ctx):
    """Edge cases (empty stream, 1-node episodes = frequency, a tick too small
    for an edge) and a 200k-event recording of the many-recordings workload
    with 3- and 4-node candidates of the 4-bin set: never below the oracle's
    count, and equal to the oracle's definition on a sample."""
    from oracle import coarse_bound as cb
    st0 = ctx.load_stream(np.zeros(0, np.uint16), np.zeros(0, np.int32), 3)
    ub, _ = ctx.upper_bound_coarse(st0, fb.Cands(np.array([0, 2, 3]), np.array([0, 1, 2], np.uint16),
                                                 np.array([0], np.int32), np.array([4], np.int32)))
    assert ub.tolist() == [0, 0]
    st0.free()
    s, _ = synth.c1_tiny()
    st = ctx.load_stream(s.types, s.times, s.n_types)
    c1 = fb.Cands(np.arange(s.n_types + 1, dtype=np.int64), np.arange(s.n_types, dtype=np.uint16),
                  np.zeros(0, np.int32), np.zeros(0, np.int32))
    ub, _ = ctx.upper_bound_coarse(st, c1)
    assert np.array_equal(ub, st.freq())
    with pytest.raises(fb.FemError) as e:
        ctx.upper_bound_coarse(st, fb.Cands(np.array([0, 2]), np.array([0, 1], np.uint16),
                                            np.array([0], np.int32), np.array([64], np.int32)), 2)
    assert e.value.status == fb.FEM_ERR_INVAL
    st.free()
    s, cfg = synth.c4_recordings(n_rec=2)[1]  # 190,695 events
    offs, ct, lo, hi = synth.random_candidates(0xC0A7, 3000, s.n_types, 3, 4, cfg["bins"], s.chains, 0.1)
    st = ctx.load_stream(s.types, s.times, s.n_types)
    ub, w = ctx.upper_bound_coarse(st, fb.Cands(offs, ct, lo, hi))
    ub = ub.astype(np.int64)
    exact = oracle_counts(s.types, s.times, offs, ct, lo, hi)
    assert np.all(ub >= exact)
    sample = synth.Rng(6, 1).integers(0, 2999, 12)
    want = cb.coarse_ub_many(s.types, s.times, *_sub(offs, ct, lo, hi, sample), w)
    assert np.array_equal(ub[sample], want)
    st.free()


def test_level3_join_bound_prunes_without_changing_results(fb, ctx):
    """The level-3 join bound (the default pre-pass with the mining graph):
    the same levels as with the level-2 pair bound only and with no bound at
    all, on three recordings of the many-recordings set; it drops level-3
    candidates (reported as pruned, not counted) and the relevant-event
    count only covers what was counted."""
    recs = synth.c4_recordings(which=[4, 19, 22])
    sts = [ctx.load_stream(s.types, s.times, s.n_types) for s, _ in recs]
    bins = recs[0][1]["bins"]
    thr = [c["threshold"] for _, c in recs]
    out = {}
    try:
        for pp in (0, 2, -1):
            ctx.set_tuning(prepass=pp)
            res = ctx.mine_levelwise(sts, bins, thr, 5)
            out[pp] = ([res.level(r, N) for r in range(len(sts)) for N in range(1, 6)], res.stats())
            res.free()
    finally:
        ctx.reset_tuning()
    assert out[0][0] == out[2][0] == out[-1][0]
    s0, s2, sn = out[0][1], out[2][1], out[-1][1]
    assert s0["graph_tails"] == 1 and s2["graph_tails"] == 1
    assert s0["candidates_pruned"] > s2["candidates_pruned"] > 0 == sn["candidates_pruned"]
    assert s0["candidates_counted"] + s0["candidates_pruned"] == s2["candidates_counted"] + s2["candidates_pruned"]
    assert s0["counted_episode_events"] < s2["counted_episode_events"]
    assert s0["relevant_events"] < s2["relevant_events"]
    assert sum(len(out[0][0][r * 5 + 2][0]) for r in range(len(sts))) > 0  # some level-3 episode is frequent
    for st in sts:
        st.free()

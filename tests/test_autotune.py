"""The launch-shape autotuner's search and cache (host logic, no GPU): a fake
timer stands in for the CUDA-event timing of each applied shape."""
import json

from paper_2511_02136_gb300 import autotune


def _fake(times):
    state = {"cur": None, "applied": [], "timed": 0}

    def applier(h, ch, costs):
        state["cur"] = (ch.warps_per_block, ch.persistent, ch.longest_first)
        state["applied"].append(state["cur"])

    def timer(run, repeats):
        state["timed"] += 1
        return times[state["cur"]]
    return state, applier, timer


def _times():
    t = {}
    for wpb in (1, 2, 4, 8):
        for pers in (0, 1):
            for lf in (False, True):
                t[(wpb, pers, lf)] = 10.0 + wpb + pers + (0.5 if lf else 0.0)
    t[(4, 1, True)] = 3.0      # the fastest shape
    t[(2, 0, True)] = 1.0      # never a candidate: the order only matters to the work queue
    return t


def test_picks_fastest_and_skips_order_without_queue(tmp_path):
    state, applier, timer = _fake(_times())
    win = autotune.tune(None, lambda: None, costs=[1.0], timer=timer, applier=applier)
    assert (win.warps_per_block, win.persistent, win.longest_first) == (4, 1, True)
    assert win.ms == 3.0
    # 8 shapes in natural order, 4 work-queue shapes also longest first
    assert state["timed"] == 12
    assert all(not (lf and not pers) for _, pers, lf in state["applied"])
    assert state["applied"][-1] == (4, 1, True)          # the winner is left applied


def test_without_costs_no_longest_first():
    state, applier, timer = _fake(_times())
    win = autotune.tune(None, lambda: None, costs=None, timer=timer, applier=applier)
    assert not win.longest_first and state["timed"] == 8
    assert (win.warps_per_block, win.persistent) == (1, 0)


def test_cache_round_trip(tmp_path):
    cache = str(tmp_path / "tune.json")
    state, applier, timer = _fake(_times())
    win = autotune.tune(None, lambda: None, costs=[1.0], timer=timer, applier=applier, cache=cache, key="k1")
    assert json.load(open(cache))["k1"]["warps_per_block"] == 4
    state2, applier2, timer2 = _fake(_times())
    again = autotune.tune(None, lambda: None, costs=[1.0], timer=timer2, applier=applier2, cache=cache, key="k1")
    assert again == win and state2["timed"] == 0 and state2["applied"] == [(4, 1, True)]


def test_signature_is_order_independent():
    a = autotune.signature(8, {100: 3, 50: 5}, 99.6, 500)
    b = autotune.signature(8, {50: 5, 100: 3}, 100.4, 500)
    assert a == b


def test_threads_per_env_axis_is_timed_and_cached(tmp_path):
    """A candidate with 64 threads per env (one warp per book side) is timed
    like the others and, when fastest, is what the cache records."""
    seen = []

    def applier(h, ch, costs):
        seen.append((ch.warps_per_block, ch.persistent, ch.longest_first, ch.threads_per_env))

    def timer(run, repeats):
        return 2.0 if seen[-1][3] == 64 else 5.0 + seen[-1][0]

    cache = tmp_path / "tune.json"
    win = autotune.tune(None, lambda: None, costs=[1.0], candidates=autotune.DEFAULT_CANDIDATES +
                        autotune.SPLIT_CANDIDATES, timer=timer, applier=applier, cache=str(cache), key="k")
    assert win.threads_per_env == 64 and win.persistent == 0
    assert (1, 0, False, 64) in seen
    assert json.loads(cache.read_text())["k"]["threads_per_env"] == 64
    assert sum(1 for *_, t in seen if t == 64) == 2   # timed, then applied as the winner


def test_tile_axis_timed_on_the_winning_shape(tmp_path):
    """The message-tile sizes are timed on the winning shape only, and the
    fastest (shape, tile) is applied and cached."""
    seen = []

    def applier(h, ch, costs):
        seen.append((ch.warps_per_block, ch.persistent, ch.longest_first, ch.tile_records))

    def timer(run, repeats):
        wpb, pers, lf, tile = seen[-1]
        base = 3.0 if (wpb, pers, lf) == (4, 1, True) else 10.0 + wpb
        return base - (0.5 if tile == 64 else 0.0) + (0.5 if tile == 16 else 0.0)

    cache = tmp_path / "tune.json"
    timed = []
    win = autotune.tune(None, lambda: None, costs=[1.0], timer=timer, applier=applier, cache=str(cache), key="k",
                        timed=timed, tiles=autotune.TILE_CANDIDATES)
    assert (win.warps_per_block, win.persistent, win.longest_first, win.tile_records) == (4, 1, True, 64)
    assert win.ms == 2.5
    # 12 shapes at 32 records, then the winner at 16 and 64
    assert len(timed) == 14
    assert sorted(c.tile_records for c in timed if (c.warps_per_block, c.persistent, c.longest_first) == (4, 1, True)) \
        == [16, 32, 64]
    assert all(c.tile_records == 32 for c in timed[:12])
    assert seen[-1] == (4, 1, True, 64)
    assert json.loads(cache.read_text())["k"]["tile_records"] == 64

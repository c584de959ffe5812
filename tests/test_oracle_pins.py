"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* hand-worked matching examples (price-time priority, JaxMARL-HFT Sec. 2.1);
* a hand-worked two-agent episode (Sec. 4 env step, Eq. 1 portfolio value);
* the agents' action tables (Sec. 4.1);
* SplitMix64's published test vector and properties of the bounded map;
* distributional checks of the shuffle and the random policy;
* invariants on random streams (spread never crossed after a message,
  priority order, volume / cash / inventory conservation).
"""
import json
import math
import os
from collections import Counter

import numpy as np
import pytest

import oracle
from conftest import make_msgs, single_env_stream
from paper_2511_02136_gb300 import mbogen

GOLD = os.path.join(os.path.dirname(__file__), "golden")
BUY, SELL = 1, -1


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _book_rows(o, env=0):
    n2, px, qty, oid, ts = o.book(env)
    return [[[int(px[s, j]), int(qty[s, j]), int(oid[s, j]), int(ts[s, j])] for j in range(n2[s])]
            for s in range(2)]


def _owner(oid, A=2):
    return A if oid >= 0 else (-oid - 1) % A


# ---------------------------------------------------------------- matching

@pytest.mark.parametrize("case", _gold("matching_examples.json")["cases"], ids=lambda c: c["name"])
def test_worked_matching_example(case):
    msgs, off = single_env_stream([case["msgs"]])
    o = oracle.Oracle(1, n_agents=0, cap=case["cap"], episode_len=1, trace=1)
    o.reset(np.zeros(1, np.uint64))
    o.load_messages(msgs, off)
    rc = o.step()
    bids, asks = _book_rows(o)
    assert bids == case["bids"]
    assert asks == case["asks"]
    f = o.fills(0)
    assert [[int(x["maker_id"]), int(x["taker_id"]), int(x["px"]), int(x["qty"])] for x in f] == case["fills"]
    cnt = dict(zip(oracle.COUNTER_NAMES, o.counters()[0].tolist()))
    for k, v in case["counters"].items():
        assert cnt[k] == v, k
    assert rc == (-6 if cnt["bad_msgs"] else 0)


def test_fill_record_fields():
    msgs, off = single_env_stream([[[1, SELL, 101, 5, 1], [4, BUY, 0, 2, 2]]])
    o = oracle.Oracle(1, n_agents=0, cap=4, episode_len=1, trace=1)
    o.reset(np.zeros(1, np.uint64))
    o.load_messages(msgs, off)
    o.step()
    f = o.fills(0)
    assert len(f) == 1 and f[0]["msg_idx"] == 1 and f[0]["taker_side"] == BUY


# ---------------------------------------------------------------- agents

def test_hand_worked_two_agent_episode():
    g = _gold("agent_episode.json")
    c = g["config"]
    msgs, off = single_env_stream([s["msgs"] for s in g["steps"]])
    o = oracle.Oracle(1, n_agents=2, cap=c["cap"], top_levels=c["top_levels"],
                      episode_len=c["episode_len"], exec_target=c["exec_target"],
                      exec_dir=c["exec_dir"], mm_lot=c["mm_lot"], start_px=c["start_px"],
                      action_mode=0, trace=1)
    o.reset(np.array([12345], np.uint64))
    o.load_messages(msgs, off)
    prev_agent_msgs = 0
    for s in g["steps"]:
        assert o.step(np.array([s["actions"]], np.int32)) == 0
        bids, asks = _book_rows(o)
        for got, want in ((bids, s["bids"]), (asks, s["asks"])):
            assert len(got) == len(want)
            for (px, q, oid, ts), (wpx, wq, wown, wts) in zip(got, want):
                assert (px, q, _owner(oid)) == (wpx, wq, wown)
                if wts is not None:
                    assert ts == wts
        fills = [[_owner(int(x["maker_id"])), _owner(int(x["taker_id"])), int(x["px"]), int(x["qty"])]
                 for x in o.fills(0)]
        assert fills == s["fills"]
        obs, rew, done = o.observe()
        np.testing.assert_array_equal(obs[0], np.array(s["obs"], np.float32))
        assert rew[0].tolist() == s["rewards"]
        assert int(done[0]) == s["done"]
        am = int(o.counters()[0][oracle.COUNTER_NAMES.index("agent_msgs")])
        assert am - prev_agent_msgs == s["agent_msgs"]
        prev_agent_msgs = am
    cnt = dict(zip(oracle.COUNTER_NAMES, o.counters()[0].tolist()))
    for k, v in g["final_counters"].items():
        assert cnt[k] == v, k
    assert o.agents()[0].tolist() == g["final_agents"]


def test_hand_worked_multi_agent_episode():
    """Two agents per type (Sec. 3, Table 1): per-agent attribution of fills,
    carry-over cancels, tasks, observations and rewards."""
    g = _gold("multi_agent.json")
    c = g["config"]
    A = 2 * c["agents_per_type"]
    msgs, off = single_env_stream([s["msgs"] for s in g["steps"]])
    o = oracle.Oracle(1, n_agents=A, cap=c["cap"], top_levels=c["top_levels"], episode_len=c["episode_len"],
                      exec_target=c["exec_target"], exec_dir=c["exec_dir"], mm_lot=c["mm_lot"],
                      start_px=c["start_px"], action_mode=0, trace=1)
    o.reset(np.array([5], np.uint64))
    o.load_messages(msgs, off)
    prev = 0
    for s in g["steps"]:
        assert o.step(np.array([s["actions"]], np.int32)) == 0
        bids, asks = _book_rows(o)
        assert [[r[0], r[1], _owner(r[2], A)] for r in bids] == s["bids"]
        assert [[r[0], r[1], _owner(r[2], A)] for r in asks] == s["asks"]
        fills = [[_owner(int(x["maker_id"]), A), _owner(int(x["taker_id"]), A), int(x["px"]), int(x["qty"])]
                 for x in o.fills(0)]
        assert fills == s["fills"]
        obs, rew, done = o.observe()
        np.testing.assert_array_equal(obs[0], np.array(s["obs"], np.float32))
        assert rew[0].tolist() == s["rewards"]
        assert int(done[0]) == s["done"]
        am = int(o.counters()[0][oracle.COUNTER_NAMES.index("agent_msgs")])
        assert am - prev == s["agent_msgs"]
        prev = am
    assert o.agents()[0].tolist() == g["final_agents"]
    cnt = dict(zip(oracle.COUNTER_NAMES, o.counters()[0].tolist()))
    for k, v in g["final_counters"].items():
        assert cnt[k] == v, k


def _reward_cases():
    for sc in _gold("reward_variants.json")["scenarios"]:
        for ex in sc["expected"]:
            yield pytest.param(sc, ex, id=sc["name"] + "-" + "-".join(f"{k}{v}" for k, v in ex.items()
                                                                     if k != "rewards"))


@pytest.mark.parametrize("sc,ex", list(_reward_cases()))
def test_hand_worked_reward_variants(sc, ex):
    c = sc["config"]
    kw = {k: v for k, v in ex.items() if k != "rewards"}
    msgs, off = single_env_stream([s["msgs"] for s in sc["steps"]])
    o = oracle.Oracle(1, n_agents=2, cap=c["cap"], top_levels=c["top_levels"],
                      episode_len=c["episode_len"], exec_target=c["exec_target"],
                      exec_dir=c["exec_dir"], mm_lot=c["mm_lot"], start_px=c["start_px"],
                      action_mode=0, **kw)
    o.reset(np.array([7], np.uint64))
    o.load_messages(msgs, off)
    got = []
    for s in sc["steps"]:
        assert o.step(np.array([s["actions"]], np.int32)) == 0
        got.append(o.observe()[1][0].tolist())
    assert got == ex["rewards"]


def test_reward_variants_leave_book_and_obs_alone():
    """The variants change the reward alone: books, observations and counters are those of mode 0."""
    seeds = mbogen.env_seeds(77, 4)
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=40), seeds, 6)
    outs = []
    for rw in (dict(), dict(reward_mode=2, spooner_lambda_pct=40, inv_penalty=3, exec_penalty_milli=100)):
        o = oracle.Oracle(4, n_agents=2, cap=16, episode_len=6, action_mode=1, exec_target=30, **rw)
        o.reset(seeds)
        o.load_messages(st.msgs, st.offsets)
        rec = []
        for _ in range(6):
            o.step()
            obs, rew, done = o.observe()
            rec.append((obs.copy(), o.counters().copy(), o.agents().copy(), rew.copy()))
        outs.append(rec)
    differs = False
    for a, b in zip(*outs):
        for x, y in zip(a[:3], b[:3]):
            np.testing.assert_array_equal(x, y)
        differs |= not np.array_equal(a[3][:, 1], b[3][:, 1])
    # the execution agent's reward differs from Eq. 1 only by the penalty at the last step
    for a, b in zip(outs[0][:-1], outs[1][:-1]):
        np.testing.assert_array_equal(a[3][:, 0], b[3][:, 0])
    assert differs


def _setup_two_quotes(start_px, exec_dir, actions, mm_space=0):
    """Step 0 places a bid 99 x 50 and an ask 104 x 50; step 1 runs `actions`."""
    msgs, off = single_env_stream([[[1, BUY, 99, 50, 0], [1, SELL, 104, 50, 1]], []])
    o = oracle.Oracle(1, n_agents=2, cap=50, top_levels=2, episode_len=100, exec_target=100,
                      exec_dir=exec_dir, mm_lot=1, start_px=start_px, action_mode=0, trace=1,
                      mm_space=mm_space)
    o.reset(np.array([7], np.uint64))
    o.load_messages(msgs, off)
    o.step(np.array([[9, 0]], np.int32))
    step0 = _book_rows(o)
    o.step(np.array([actions], np.int32))
    return o, step0


def test_mm_action_table():
    g = _gold("action_tables.json")
    for k, want in g["mm"].items():
        o, _ = _setup_two_quotes(200, SELL, [9, int(k)])
        bids, asks = _book_rows(o)
        mb = [r for r in bids if _owner(r[2]) == 1]
        ma = [r for r in asks if _owner(r[2]) == 1]
        if want is None:
            assert mb == [] and ma == []
        else:
            assert [r[0] for r in mb] == [want[0]] and [r[0] for r in ma] == [want[1]]
            assert mb[0][1] == 1 and ma[0][1] == 1


@pytest.mark.parametrize("which,space", [("mm_fixed_quantity", 1), ("mm_directional", 2)])
def test_mm_other_action_spaces(which, space):
    g = _gold("action_tables.json")[which]
    for k, (want_b, want_a) in g.items():
        o, _ = _setup_two_quotes(200, SELL, [9, int(k)], mm_space=space)
        bids, asks = _book_rows(o)
        mb = [(r[0], r[1]) for r in bids if _owner(r[2]) == 1]
        ma = [(r[0], r[1]) for r in asks if _owner(r[2]) == 1]
        assert mb == ([] if want_b is None else [(want_b, 1)]), k
        assert ma == ([] if want_a is None else [(want_a, 1)]), k


@pytest.mark.parametrize("space,n", [(0, 12), (1, 8), (2, 3)])
def test_random_policy_covers_each_mm_space(space, n):
    """The random policy draws the market maker's action uniformly over its space's options."""
    seeds = mbogen.env_seeds(3, 400)
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=2), seeds, 1)
    o = oracle.Oracle(400, n_agents=2, cap=8, episode_len=1, action_mode=1, mm_space=space)
    o.reset(seeds)
    o.load_messages(st.msgs, st.offsets)
    o.step()
    acts = o.actions()
    assert acts[:, 1].min() == 0 and acts[:, 1].max() == n - 1
    assert acts[:, 0].max() == 11
    for e in range(0, 400, 37):
        want = oracle.lemire(oracle.draw(int(seeds[e]), 0, oracle.TAG_POLICY, 1), n)
        assert acts[e, 1] == want


@pytest.mark.parametrize("which,exec_dir", [("exec_sell", SELL), ("exec_buy", BUY)])
def test_exec_action_table(which, exec_dir):
    g = _gold("action_tables.json")[which]
    for k, (px, q, crosses) in g["table"].items():
        o, step0 = _setup_two_quotes(g["start_px"], exec_dir, [int(k), 0])
        bids, asks = _book_rows(o)
        own = [r for r in bids + asks if _owner(r[2]) == 0]
        fills = [x for x in o.fills(0) if _owner(int(x["taker_id"])) == 0]
        if crosses:
            assert own == [] and [(int(x["px"]), int(x["qty"])) for x in fills] == [(px, q)]
        else:
            assert fills == [] and [(r[0], r[1]) for r in own] == [(px, q)]
            assert own[0] in (bids if exec_dir == BUY else asks)


def test_empty_book_uses_last_trade_price():
    e = _gold("action_tables.json")["empty_book_passive_exec"]
    _, step0 = _setup_two_quotes(e["start_px"], SELL, [9, 0])
    assert [r[0] for r in step0[1] if _owner(r[2]) == 0] == [e["exec_sell_price_at_step0"]]
    _, step0 = _setup_two_quotes(e["start_px_buy"], BUY, [9, 0])
    assert [r[0] for r in step0[0] if _owner(r[2]) == 0] == [e["exec_buy_price_at_step0"]]


def test_exec_quantity_clamped_and_stops_at_target():
    # target 3, T = 2 -> q0 = 2; x5 is clamped to the remaining 3; then nothing
    msgs, off = single_env_stream([[[1, BUY, 99, 50, 0]], [], []])
    o = oracle.Oracle(1, n_agents=2, cap=10, top_levels=2, episode_len=2, exec_target=3,
                      exec_dir=SELL, start_px=99, action_mode=0, trace=1)
    o.reset(np.array([1], np.uint64))
    o.load_messages(msgs, off)
    o.step(np.array([[9, 0]], np.int32))      # passive sell 101 x 2 rests
    o.step(np.array([[2, 0]], np.int32))      # far touch (99) x5 -> clamp to 3
    f = o.fills(0)
    assert [(int(x["px"]), int(x["qty"])) for x in f] == [(99, 3)]
    assert o.agents()[0][0].tolist()[3] == 3
    o.step(np.array([[2, 0]], np.int32))      # target met: no order, nothing rests
    assert o.fills(0).size == 0
    assert all(_owner(r[2]) != 0 for side in _book_rows(o) for r in side)


# ---------------------------------------------------------------- RNG

def test_splitmix64_published_vector():
    g = _gold("splitmix64_vectors.json")
    got = [oracle.splitmix(g["seed"], i) for i in range(len(g["outputs"]))]
    assert got == [int(x) for x in g["outputs"]]


def test_keyed_draw_matches_independent_restatement():
    import brute_lob
    for seed in (0, 1, 2**63 + 5, 0xDEADBEEF):
        for t in (0, 1, 999):
            for tag in (oracle.TAG_SHUFFLE, oracle.TAG_POLICY):
                want = brute_lob.keyed_draws(seed, t, tag, 3)
                assert [oracle.draw(seed, t, tag, i) for i in range(3)] == want


def test_bounded_map_properties():
    for n in (1, 2, 3, 12, 1000, 2**31 + 11):
        assert oracle.lemire(0, n) == 0
        assert oracle.lemire(2**64 - 1, n) == n - 1
        # the first high word mapping to k is ceil(k * 2^32 / n)
        for k in sorted(k for k in {0, 1, n // 2, n - 1} if k < n):
            lo = -(-(k << 32) // n)
            assert oracle.lemire(lo << 32, n) == k
            if lo > 0:
                assert oracle.lemire(((lo - 1) << 32) | 0xFFFFFFFF, n) == k - 1
    xs = sorted(int(v) for v in np.random.default_rng(0).integers(0, 2**63, 500, dtype=np.uint64))
    ys = [oracle.lemire(x, 12) for x in xs]
    assert ys == sorted(ys)


def _chi2_ok(counts, n_cats, total, z=5.0):
    exp = total / n_cats
    chi2 = sum((counts.get(k, 0) - exp) ** 2 / exp for k in range(n_cats))
    dof = n_cats - 1
    return chi2 < dof + z * math.sqrt(2 * dof)


def test_random_policy_uniform_over_12_actions():
    n_env, T = 256, 40
    seeds = mbogen.env_seeds(3, n_env)
    msgs, off = mbogen.MSG_DTYPE, None
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=0), seeds, T)
    o = oracle.Oracle(n_env, episode_len=T, action_mode=1)
    o.reset(seeds)
    o.load_messages(st.msgs, st.offsets)
    cnt = [Counter(), Counter()]
    for _ in range(T):
        o.step()
        for a in range(2):
            cnt[a].update(o.actions()[:, a].tolist())
    for a in range(2):
        assert set(cnt[a]) <= set(range(12))
        assert _chi2_ok(cnt[a], 12, n_env * T)
    # the two agents draw different numbers
    assert cnt[0] != cnt[1]


def test_shuffle_permutations_uniform():
    """Three non-interacting agent orders; their arrival stamps give the order."""
    n_env = 3000
    seeds = mbogen.env_seeds(11, n_env)
    rows = [[1, BUY, 90, 50, 0], [1, SELL, 110, 50, 1]]
    one = make_msgs(rows)
    msgs = np.concatenate([one] * n_env)
    off = np.zeros((n_env, 3), np.int64)
    off[:, 0] = np.arange(n_env) * 2
    off[:, 1] = off[:, 0] + 2
    off[:, 2] = off[:, 1]
    o = oracle.Oracle(n_env, n_agents=2, cap=10, top_levels=2, episode_len=100, exec_target=100,
                      exec_dir=SELL, start_px=200, action_mode=0)
    o.reset(seeds)
    o.load_messages(msgs, off)
    o.step(np.tile(np.array([[9, 0]], np.int32), (n_env, 1)))
    # exec passive sell at 112, MM quotes 90 / 110+2: nothing crosses
    o.step(np.tile(np.array([[9, 3]], np.int32), (n_env, 1)))
    perms = Counter()
    for e in range(n_env):
        n2, px, qty, oid, ts = o.book(e)
        agent = []
        for s in range(2):
            for j in range(n2[s]):
                if oid[s, j] < 0 and ts[s, j] >= 3:
                    agent.append((int(ts[s, j]), (_owner(int(oid[s, j])), s)))
        assert len(agent) == 3
        perms[tuple(x[1] for x in sorted(agent))] += 1
    assert len(perms) == 6
    keys = sorted(perms)
    assert _chi2_ok({i: perms[k] for i, k in enumerate(keys)}, 6, n_env)


# ---------------------------------------------------------------- invariants

def _tiny_model(**kw):
    base = dict(price_p=0.55, size_p=0.3, msgs_per_step=40)
    base.update(kw)
    return mbogen.MessageModel(**base)


@pytest.mark.parametrize("cap", [1, 2, 3, 5, 8])
def test_invariants_after_every_message(cap):
    T = 12
    seeds = mbogen.env_seeds(100 + cap, 1)
    st = mbogen.generate(_tiny_model(), seeds, T)
    o = oracle.Oracle(1, n_agents=2, cap=cap, top_levels=3, episode_len=T, exec_target=40,
                      action_mode=1, trace=3)
    o.reset(seeds)
    o.load_messages(st.msgs, st.offsets)
    for _ in range(T):
        o.step()
        snaps = o.snapshots()
        assert len(snaps) > 0
        for sn in snaps:
            nb, na = int(sn["n"][0]), int(sn["n"][1])
            assert 0 <= nb <= cap and 0 <= na <= cap
            bpx, apx = sn["px"][0][:nb], sn["px"][1][:na]
            assert np.all(sn["qty"][0][:nb] > 0) and np.all(sn["qty"][1][:na] > 0)
            assert np.all(np.diff(bpx) <= 0) and np.all(np.diff(apx) >= 0)
            for s, n in ((0, nb), (1, na)):
                px, ts = sn["px"][s][:n], sn["ts"][s][:n]
                same = px[1:] == px[:-1]
                assert np.all(ts[1:][same] > ts[:-1][same])   # FIFO within a price
            if nb and na:
                assert bpx[0] < apx[0]                        # book never left crossed
        cnt = dict(zip(oracle.COUNTER_NAMES, o.counters()[0].tolist()))
        n2, px, qty, oid, ts = o.book(0)
        resting = int(qty[0, :n2[0]].sum() + qty[1, :n2[1]].sum())
        assert cnt["add_vol"] + cnt["mkt_vol"] == (2 * cnt["fill_vol"] + resting + cnt["cancel_vol"]
                                                   + cnt["drop_vol"] + cnt["evict_vol"]
                                                   + cnt["mkt_discard_vol"])
        ag = o.agents()[0]
        assert ag[:, 1].sum() + cnt["bg_cash"] == 0
        assert ag[:, 0].sum() + cnt["bg_inv"] == 0
        # each agent's resting quantity in the observation matches the book
        obs, _, _ = o.observe()
        for a in range(2):
            own = sum(int(qty[s, j]) for s in range(2) for j in range(n2[s])
                      if oid[s, j] < 0 and _owner(int(oid[s, j])) == a)
            assert obs[0, a, -1] == own


def test_arrival_stamps_unique_and_increasing():
    T = 6
    seeds = mbogen.env_seeds(5, 3)
    st = mbogen.generate(_tiny_model(), seeds, T)
    o = oracle.Oracle(3, cap=6, top_levels=2, episode_len=T, action_mode=1)
    o.reset(seeds)
    o.load_messages(st.msgs, st.offsets)
    for _ in range(T):
        o.step()
    misc = o.env_misc()
    for e in range(3):
        n2, px, qty, oid, ts = o.book(e)
        live = np.concatenate([ts[0, :n2[0]], ts[1, :n2[1]]])
        assert len(set(live.tolist())) == len(live)
        assert np.all(live < misc[e, 0])


# ---------------------------------------------------------------- episodes

def _episode_inputs(g, levels_per_side=4):
    msgs, off = single_env_stream(g["data_steps"])
    n = len(g["starts"])
    starts = np.zeros(n, oracle.START_DTYPE)
    levels = np.zeros((n, 2, levels_per_side, 2), np.int32)
    for j, s in enumerate(g["starts"]):
        starts[j] = (s["data_step"], s["last_px"], len(s["bids"]), len(s["asks"]))
        for side, key in enumerate(("bids", "asks")):
            for i, lv in enumerate(s[key]):
                levels[j, side, i] = lv
    return msgs, off[0], starts, levels


def _labelled_book(o, env=0):
    out = []
    for side in _book_rows(o, env):
        rows = []
        for px, q, oid, ts in side:
            init = oid >= oracle.INIT_ID
            rows.append([px, q, "init" if init else "bg", oid - oracle.INIT_ID if init else oid, ts])
        out.append(rows)
    return out


def test_hand_worked_episodes_over_shared_stream():
    g = _gold("episodes.json")
    c = g["config"]
    msgs, step_off, starts, levels = _episode_inputs(g)
    o = oracle.Oracle(1, n_agents=2, cap=c["cap"], top_levels=c["top_levels"], episode_len=c["episode_len"],
                      exec_target=c["exec_target"], exec_dir=c["exec_dir"], mm_lot=c["mm_lot"],
                      start_px=c["start_px"], action_mode=0, trace=1)
    o.set_episodes(msgs, step_off, starts, levels)
    o.reset(np.array([c["seed"]], np.uint64))
    r = g["reset"]
    assert o.episode_starts().tolist() == [r["episode_start"]]
    assert _labelled_book(o) == [r["bids"], r["asks"]]
    obs, _, _ = o.observe()
    np.testing.assert_array_equal(obs[0, 0], np.array(r["obs"], np.float32))
    for s in g["steps"]:
        assert o.step(np.array([s["actions"]], np.int32)) == 0
        assert o.episode_starts().tolist() == [s["episode_start"]]
        assert _labelled_book(o) == [s["bids"], s["asks"]]
        fills = [[int(f["maker_id"]) - oracle.INIT_ID if f["maker_id"] >= oracle.INIT_ID else int(f["maker_id"]),
                  int(f["taker_id"]), int(f["px"]), int(f["qty"])] for f in o.fills(0)]
        assert fills == s["fills"]
        obs, rew, done = o.observe()
        np.testing.assert_array_equal(obs[0, 0], np.array(s["obs"], np.float32))
        np.testing.assert_array_equal(obs[0, 1], np.array(s["obs"], np.float32))
        assert rew[0].tolist() == s["rewards"]
        assert int(done[0]) == s["done"]
    cnt = dict(zip(oracle.COUNTER_NAMES, o.counters()[0].tolist()))
    for k, v in g["final_counters"].items():
        assert cnt[k] == v, k


def test_episode_start_draws_match_restatement():
    """The start of episode k is snapshot Lemire(first SplitMix64 output keyed
    by (seed, k), n_starts): checked against the brute env's own SplitMix64."""
    import brute_lob
    n_data, T = 40, 3
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=5), mbogen.env_seeds(5, 1), n_data)
    starts, levels = mbogen.start_books(9, st.mids[0], np.arange(0, n_data - T + 1, 2), 3)
    seeds = mbogen.env_seeds(44, 16)
    o = oracle.Oracle(16, n_agents=0, cap=8, episode_len=T)
    o.set_episodes(st.msgs, st.offsets[0], starts, levels)
    o.reset(seeds)
    for k in range(5):
        want = [int(starts[brute_lob.bounded(brute_lob.keyed_draws(int(s), k, brute_lob.TAG_EPISODE, 1)[0],
                                             len(starts))]["data_step"]) for s in seeds]
        assert o.episode_starts().tolist() == want
        for _ in range(T):
            o.step()


def test_episodes_counters_accumulate_and_books_restart():
    """Across an episode boundary the book is exactly the drawn snapshot and
    counters keep counting; with one snapshot every episode replays the same data."""
    n_data, T = 12, 4
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=30), mbogen.env_seeds(6, 1), n_data)
    starts, levels = mbogen.start_books(2, st.mids[0], [3], 6, min_levels=2)
    o = oracle.Oracle(2, n_agents=2, cap=16, episode_len=T, action_mode=1, exec_target=20)
    o.set_episodes(st.msgs, st.offsets[0], starts, levels)
    o.reset(mbogen.env_seeds(7, 2))
    first = _book_rows(o)
    msgs_per_episode = int(st.offsets[0, 3 + T] - st.offsets[0, 3])
    for ep in range(3):
        for _ in range(T):
            o.step()
        assert _book_rows(o) == first
        assert o.counters()[0][oracle.COUNTER_NAMES.index("msgs")] >= (ep + 1) * msgs_per_episode
        assert o.agents()[0].tolist() == [[0, 0, 0, 0], [0, 0, 0, 0]]


def test_drawn_task_side_at_reset():
    """exec_dir 0 (Table 2: task side uniformly sampled): each env's side is the
    top bit of a keyed SplitMix64 draw (set -> sell), seen as the sign of the
    remaining-target observation; both sides occur about equally often."""
    import brute_lob
    n, L = 400, 3
    seeds = mbogen.env_seeds(11, n)
    o = oracle.Oracle(n, n_agents=2, cap=8, top_levels=L, episode_len=5, exec_target=50, exec_dir=0)
    o.reset(seeds)
    rem = o.observe()[0][:, 0, 4 * L + 3]
    want = np.array([-50.0 if brute_lob.keyed_draws(int(s), 0, brute_lob.TAG_TASKDIR, 1)[0] >> 63 else 50.0
                     for s in seeds], np.float32)
    np.testing.assert_array_equal(rem, want)
    assert 150 < int((want < 0).sum()) < 250

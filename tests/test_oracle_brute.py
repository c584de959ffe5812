"""Oracle vs. a brute-force sorted-list book on tiny random inputs.

Capacities of 1-8 per side and a narrow price band make every branch of the
matcher fire (evictions, drops, sweeps to empty, partial cancels to zero,
misses), and both agents act every step.
"""
import numpy as np
import pytest

import brute_lob
import oracle
from paper_2511_02136_gb300 import mbogen


def _compare(o, b, env, step_fills):
    n2, px, qty, oid, ts = o.book(env)
    got = [[(int(px[s, j]), int(qty[s, j]), int(oid[s, j]), int(ts[s, j])) for j in range(n2[s])]
           for s in range(2)]
    assert got == b.book_arrays()
    if step_fills is not None:
        assert [tuple(int(v) for v in f) for f in step_fills] == [tuple(f) for f in b.fills]
    cnt = dict(zip(oracle.COUNTER_NAMES, o.counters()[env].tolist()))
    for k, v in b.c.items():
        assert cnt[k] == v, k
    assert cnt["bg_cash"] == b.bg_cash and cnt["bg_inv"] == b.bg_inv


@pytest.mark.parametrize("seed", range(12))
def test_oracle_matches_brute(seed):
    _run_against_brute(seed, {})


@pytest.mark.parametrize("seed", range(6))
def test_oracle_matches_brute_drawn_task_side(seed):
    """Table 2's uniformly sampled task side (exec_dir 0): per env at reset,
    signed remaining-target observation, both action modes."""
    _run_against_brute(1200 + seed, {"exec_dir": 0})


@pytest.mark.parametrize("seed", range(8))
def test_oracle_matches_brute_reward_variants(seed):
    """Eqs. 3-4 and the Table 2 penalties, against exact fractions in the brute env."""
    rng = np.random.default_rng(500 + seed)
    rw = dict(reward_mode=int(rng.integers(0, 3)), spooner_lambda_pct=int(rng.integers(0, 101)),
              inv_penalty=int(rng.integers(0, 3)), exec_penalty_milli=int(rng.choice([0, 10, 50, 100, 2500])),
              mm_space=int(rng.integers(0, 3)), pv_ref=int(rng.integers(0, 2)))
    _run_against_brute(100 + seed, rw)


def _run_against_brute(seed, rw):
    rng = np.random.default_rng(seed)
    cap = int(rng.integers(1, 9))
    T = 10
    n_env = 3
    model = mbogen.MessageModel(price_p=float(rng.uniform(0.4, 0.8)), size_p=0.3,
                                msgs_per_step=int(rng.integers(5, 30)),
                                mix_market=float(rng.uniform(0.05, 0.3)))
    seeds = mbogen.env_seeds(1000 + seed, n_env)
    st = mbogen.generate(model, seeds, T)
    host = seed % 2 == 0
    kw = dict(top_levels=3, episode_len=T, mm_lot=int(rng.integers(1, 4)),
              exec_target=int(rng.integers(5, 60)), exec_dir=int(rng.choice([-1, 1])),
              start_px=10_000)
    kw.update(rw)
    o = oracle.Oracle(n_env, n_agents=2, cap=cap, action_mode=0 if host else 1, trace=1, **kw)
    o.reset(seeds)
    o.load_messages(st.msgs, st.offsets)
    brutes = [brute_lob.BruteEnv(cap, n_agents=2, seed=int(seeds[e]), action_mode=0 if host else 1, **kw)
              for e in range(n_env)]
    for t in range(T):
        acts = rng.integers(0, 12, size=(n_env, 2)).astype(np.int32) if host else None
        o.step(acts)
        obs, rew, done = o.observe()
        for e in range(n_env):
            b = brutes[e]
            msgs = st.msgs[st.offsets[e, t]:st.offsets[e, t + 1]]
            b.step(msgs, None if acts is None else acts[e].tolist())
            fl = o.fills(e)
            _compare(o, b, e, [(f["maker_id"], f["taker_id"], f["px"], f["qty"], f["msg_idx"], f["taker_side"])
                               for f in fl])
            np.testing.assert_array_equal(obs[e], np.array(b.obs, np.float32))
            assert rew[e].tolist() == b.rew
            assert int(done[e]) == b.done
            assert o.actions()[e].tolist() == b.acts


def test_oracle_matches_brute_replay_only():
    """No agents: the plain replay configuration."""
    st = mbogen.generate(mbogen.MessageModel(price_p=0.6, size_p=0.2, msgs_per_step=200),
                         mbogen.env_seeds(77, 1), 3)
    for cap in (1, 4, 100):
        o = oracle.Oracle(1, n_agents=0, cap=cap, episode_len=3, trace=1)
        o.reset(st.seeds)
        o.load_messages(st.msgs, st.offsets)
        b = brute_lob.BruteEnv(cap, n_agents=0, episode_len=3)
        for t in range(3):
            o.step()
            b.step(st.msgs[st.offsets[0, t]:st.offsets[0, t + 1]])
            fl = o.fills(0)
            _compare(o, b, 0, [(f["maker_id"], f["taker_id"], f["px"], f["qty"], f["msg_idx"], f["taker_side"])
                               for f in fl])


@pytest.mark.parametrize("seed", range(8))
def test_oracle_matches_brute_episodes(seed):
    """Episode mode over one shared stream: overlapping starts, snapshots with
    empty sides, several episodes per env, both action modes."""
    rng = np.random.default_rng(900 + seed)
    cap = int(rng.integers(2, 9))
    T = int(rng.integers(2, 5))
    n_data = 30
    n_env = 3
    model = mbogen.MessageModel(price_p=float(rng.uniform(0.4, 0.8)), size_p=0.3,
                                msgs_per_step=int(rng.integers(3, 20)), mix_market=0.15)
    st = mbogen.generate(model, mbogen.env_seeds(2000 + seed, 1), n_data)
    start_steps = rng.integers(0, n_data - T + 1, size=int(rng.integers(1, 6)))
    starts, levels = mbogen.start_books(seed, st.mids[0], start_steps, cap, min_levels=0)
    host = seed % 2 == 0
    kw = dict(top_levels=3, episode_len=T, mm_lot=int(rng.integers(1, 4)),
              exec_target=int(rng.integers(5, 40)), exec_dir=int(rng.choice([-1, 1])), start_px=10_000,
              reward_mode=int(rng.integers(0, 3)), spooner_lambda_pct=30, inv_penalty=int(rng.integers(0, 2)),
              exec_penalty_milli=int(rng.choice([0, 100])), mm_space=seed % 3)
    if seed % 2:
        kw["exec_dir"] = 0      # the task side drawn per episode
    seeds = mbogen.env_seeds(3000 + seed, n_env)
    o = oracle.Oracle(n_env, n_agents=2, cap=cap, action_mode=0 if host else 1, trace=1, **kw)
    o.set_episodes(st.msgs, st.offsets[0], starts, levels)
    o.reset(seeds)
    brutes = []
    for e in range(n_env):
        b = brute_lob.BruteEnv(cap, n_agents=2, seed=int(seeds[e]), action_mode=0 if host else 1, **kw)
        b.set_episodes(st.msgs, st.offsets[0], starts, levels)
        b.begin_episode(0)
        b.reset_obs()
        brutes.append(b)
    obs, _, _ = o.observe()
    for e in range(n_env):
        np.testing.assert_array_equal(obs[e], np.array(brutes[e].obs, np.float32))
    for t in range(4 * T + 1):
        acts = rng.integers(0, 12, size=(n_env, 2)).astype(np.int32) if host else None
        o.step(acts)
        obs, rew, done = o.observe()
        for e in range(n_env):
            b = brutes[e]
            b.step_episode(None if acts is None else acts[e].tolist())
            fl = o.fills(e)
            _compare(o, b, e, [(f["maker_id"], f["taker_id"], f["px"], f["qty"], f["msg_idx"], f["taker_side"])
                               for f in fl])
            np.testing.assert_array_equal(obs[e], np.array(b.obs, np.float32))
            assert rew[e].tolist() == b.rew
            assert int(done[e]) == b.done
            assert o.episode_starts()[e] == b.ep_start


@pytest.mark.parametrize("seed", range(9))
def test_oracle_matches_brute_agents_per_type(seed):
    """P = 2..10 agents per type (Table 1 runs 5 and 10): per-agent actions,
    carry-over, shuffle over up to 3P new orders, fills, tasks, obs, rewards."""
    rng = np.random.default_rng(700 + seed)
    P = [2, 3, 5, 10][seed % 4]
    A = 2 * P
    cap = int(rng.integers(2, 12))
    T = 8
    n_env = 2
    model = mbogen.MessageModel(price_p=0.6, size_p=0.3, msgs_per_step=int(rng.integers(3, 25)), mix_market=0.2)
    seeds = mbogen.env_seeds(4000 + seed, n_env)
    st = mbogen.generate(model, seeds, T)
    host = seed % 2 == 0
    space = seed % 3
    n_mm = (12, 8, 3)[space]
    kw = dict(top_levels=3, episode_len=T, mm_lot=int(rng.integers(1, 4)), exec_target=int(rng.integers(5, 40)),
              exec_dir=int(rng.choice([-1, 1])), start_px=10_000, mm_space=space,
              reward_mode=seed % 3, spooner_lambda_pct=60, inv_penalty=seed % 2, exec_penalty_milli=100)
    if seed % 3 == 1:
        kw["exec_dir"] = 0      # the task side drawn per env, shared by its execution agents
    o = oracle.Oracle(n_env, n_agents=A, cap=cap, action_mode=0 if host else 1, trace=1, **kw)
    o.reset(seeds)
    o.load_messages(st.msgs, st.offsets)
    brutes = [brute_lob.BruteEnv(cap, n_agents=A, seed=int(seeds[e]), action_mode=0 if host else 1, **kw)
              for e in range(n_env)]
    for t in range(T):
        acts = None
        if host:
            acts = np.concatenate([rng.integers(0, 12, size=(n_env, P)), rng.integers(0, n_mm, size=(n_env, P))],
                                  axis=1).astype(np.int32)
        o.step(acts)
        obs, rew, done = o.observe()
        for e in range(n_env):
            b = brutes[e]
            msgs = st.msgs[st.offsets[e, t]:st.offsets[e, t + 1]]
            b.step(msgs, None if acts is None else acts[e].tolist())
            fl = o.fills(e)
            _compare(o, b, e, [(f["maker_id"], f["taker_id"], f["px"], f["qty"], f["msg_idx"], f["taker_side"])
                               for f in fl])
            np.testing.assert_array_equal(obs[e], np.array(b.obs, np.float32))
            assert rew[e].tolist() == b.rew
            assert int(done[e]) == b.done
            assert o.actions()[e].tolist() == b.acts
        ag = o.agents()
        for e in range(n_env):
            assert ag[e, :, 3].tolist() == brutes[e].exec_done

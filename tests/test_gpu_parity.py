"""GPU (liblob.so, sm_103a) vs. the CPU oracle, element by element, through the C ABI."""
import os

import numpy as np
import pytest

from harness import Pair
from paper_2511_02136_gb300 import lob, mbogen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    lob.build()
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"


def test_plain_replay_one_env_trace_every_message():
    """1 env, 10,000 messages from seed 0, capacity 100, no agents: book after
    every message and every fill identical to the oracle."""
    T, M = 100, 100
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=M), mbogen.env_seeds(0, 1), T)
    pr = Pair(1, st, n_agents=0, cap=100, fill_cap=4 * M, snap_cap=M)
    for _ in range(T):
        pr.step()
        pr.check_fills()
        pr.check_snapshots()
    pr.check_outputs()
    pr.check_state()
    pr.close()


@pytest.mark.parametrize("wpb,persistent", [(4, 0), (1, 0), (8, 0), (2, 1), (4, 1)])
def test_two_agents_random_policy_ragged(wpb, persistent):
    """37 envs (ragged against every warps-per-block), 45 messages per step
    (one full 32-message tile plus a ragged tail), 25 steps."""
    n, T = 37, 25
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=45), mbogen.env_seeds(11, n), T)
    pr = Pair(n, st, cap=100, exec_target=60, fill_cap=256, warps_per_block=wpb, persistent=persistent)
    for _ in range(T):
        pr.step()
        pr.check_outputs()
        pr.check_fills()
    pr.check_state()
    assert pr.env.sync() == 0
    pr.close()


def test_host_actions_and_buy_task():
    n, T = 29, 30
    rng = np.random.default_rng(5)
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=70), mbogen.env_seeds(12, n), T)
    pr = Pair(n, st, cap=100, exec_target=200, exec_dir=1, mm_lot=3, top_levels=20,
              action_mode=lob.LOB_ACT_HOST, fill_cap=512)
    for _ in range(T):
        pr.step(rng.integers(0, 12, size=(n, 2)).astype(np.int32))
        pr.check_outputs()
        pr.check_fills()
    pr.check_state()
    pr.close()


@pytest.mark.parametrize("seed", range(4))
def test_tiny_capacities_every_branch(seed):
    """Capacities 1..8 and a narrow price band: evictions, drops, sweeps to an
    empty side, partial cancels to zero and misses all fire."""
    n, T = 40, 20
    rng = np.random.default_rng(seed)
    caps = rng.integers(1, 9, size=n).astype(np.int32)
    model = mbogen.MessageModel(price_p=0.6, size_p=0.3, msgs_per_step=int(rng.integers(20, 70)),
                                mix_market=0.2)
    st = mbogen.generate(model, mbogen.env_seeds(100 + seed, n), T)
    pr = Pair(n, st, caps=caps, cap=8, exec_target=30, top_levels=3,
              action_mode=lob.LOB_ACT_HOST if seed % 2 else lob.LOB_ACT_RANDOM, fill_cap=512)
    for _ in range(T):
        pr.step(rng.integers(0, 12, size=(n, 2)).astype(np.int32) if seed % 2 else None)
        pr.check_outputs()
        pr.check_fills()
        pr.check_state()
    pr.close()


@pytest.mark.parametrize("L", [1, 64])
def test_pool_boundary_capacities_filled(L):
    """Capacities at and beside every pool size (32 K slots per side for
    K = 1 .. 32, up to the 1,024 maximum), an add-heavy mix over a wide price
    band that fills every side to capacity (no free slot left, evictions and
    drops), and the fewest / most observation levels."""
    caps = np.array([32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 511, 512, 513, 1023, 1024], np.int32)
    n, T = len(caps), 10
    model = mbogen.MessageModel(mix_add=0.88, mix_partial=0.03, mix_delete=0.03, mix_market=0.06,
                                price_p=0.05, msgs_per_step=600)
    st = mbogen.generate(model, mbogen.env_seeds(300 + L, n), T)
    pr = Pair(n, st, caps=caps, cap=1024, top_levels=L, exec_target=200, fill_cap=2048)
    for _ in range(T):
        pr.step()
        pr.check_outputs()
        pr.check_fills()
    pr.check_state()
    full = [e for e in range(n) if max(pr.orc.book(e)[0]) == caps[e]]
    assert len(full) == n, f"sides at capacity only for envs {full}"
    cnt = pr.orc.counters()
    assert (cnt[:, 12] > 0).all() and (cnt[:, 10] > 0).all()   # evictions and drops everywhere
    assert pr.env.sync() == 0
    pr.close()


def test_extended_kernel_default_budget_many_envs():
    """Enough envs (1,600 per class at capacities 50 and 100) that the host
    launches the extended kernel in its default register budget rather than
    the one-wave wide budget; reward variants on, every env checked."""
    n, T = 3200, 3
    caps = np.where(np.arange(n) % 2 == 0, 50, 100).astype(np.int32)
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=50), mbogen.env_seeds(160, n), T)
    pr = Pair(n, st, caps=caps, cap=100, exec_target=40, n_threads=os.cpu_count() or 1,
              rewards=dict(reward_mode=lob.LOB_REWARD_SPOONER, spooner_lambda_pct=30, inv_penalty=1,
                           exec_penalty_milli=100))
    for _ in range(T):
        pr.step()
        pr.check_outputs()
    pr.check_state()
    assert pr.env.sync() == 0
    pr.close()


def test_uneven_caps_and_poisson_counts():
    """Capacities from 20 to 1,000 (every capacity class) and
    M_t ~ Poisson(lambda_env), including empty steps."""
    n, T = 96, 15
    caps = mbogen.env_caps(3, n, choices=(20, 50, 100, 200, 256, 500, 1000))
    st = mbogen.generate(mbogen.MessageModel(poisson=True, lam_lo=0.5, lam_hi=300.0), mbogen.env_seeds(13, n), T)
    assert (st.counts == 0).any()
    pr = Pair(n, st, caps=caps, cap=1000, exec_target=100, fill_cap=1024)
    for _ in range(T):
        pr.step()
        pr.check_outputs()
        pr.check_fills()
    pr.check_state()
    pr.close()


def test_rollout_matches_stepwise_oracle():
    """Several steps in one persistent launch with the book kept on chip."""
    import torch
    n, T = 50, 12
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=60), mbogen.env_seeds(21, n), T)
    for mode in (lob.LOB_ACT_RANDOM, lob.LOB_ACT_HOST):
        pr = Pair(n, st, cap=100, exec_target=40, action_mode=mode)
        rng = np.random.default_rng(1)
        acts = rng.integers(0, 12, size=(T, n, 2)).astype(np.int32)
        D = pr.env.D
        obs = torch.zeros((T, n, 2, D), dtype=torch.float32, device="cuda")
        rew = torch.zeros((T, n, 2), dtype=torch.int64, device="cuda")
        done = torch.zeros((T, n), dtype=torch.uint8, device="cuda")
        a_d = torch.from_numpy(acts).cuda() if mode == lob.LOB_ACT_HOST else None
        # first 5 steps as one rollout, then the remaining 7 as another
        lob.lob_rollout(pr.env.h, 5, a_d[:5].contiguous() if a_d is not None else None, obs[:5], rew[:5], done[:5])
        lob.lob_rollout(pr.env.h, 7, a_d[5:].contiguous() if a_d is not None else None, obs[5:], rew[5:], done[5:])
        for t in range(T):
            pr.orc.step(acts[t] if mode == lob.LOB_ACT_HOST else None)
            o_obs, o_rew, o_done = pr.orc.observe()
            np.testing.assert_allclose(obs[t].cpu().numpy(), o_obs, rtol=1e-6, atol=0)
            np.testing.assert_array_equal(rew[t].cpu().numpy(), o_rew)
            np.testing.assert_array_equal(done[t].cpu().numpy(), o_done)
        pr.check_state()
        pr.check_outputs()
        pr.close()


def test_step_host_buffers():
    n, T = 33, 6
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=50), mbogen.env_seeds(31, n), T)
    pr = Pair(n, st, cap=100, exec_target=30, action_mode=lob.LOB_ACT_HOST)
    rng = np.random.default_rng(2)
    D = pr.env.D
    for t in range(T):
        acts = rng.integers(0, 12, size=(n, 2)).astype(np.int32)
        lo = st.offsets[:, t]
        hi = st.offsets[:, t + 1]
        chunk = np.concatenate([st.msgs[lo[e]:hi[e]] for e in range(n)])
        off = np.zeros(n + 1, np.int64)
        off[1:] = np.cumsum(hi - lo)
        obs = np.zeros((n, 2, D), np.float32)
        rew = np.zeros((n, 2), np.int64)
        done = np.zeros(n, np.uint8)
        lob.lob_step_host(pr.env.h, chunk, off, acts, obs, rew, done)
        pr.orc.step(acts)
        o_obs, o_rew, o_done = pr.orc.observe()
        np.testing.assert_allclose(obs, o_obs, rtol=1e-6, atol=0)
        np.testing.assert_array_equal(rew, o_rew)
        np.testing.assert_array_equal(done, o_done)
    pr.check_state()
    pr.close()


@pytest.mark.parametrize("pinned", [True, False])
def test_step_host_async_pipelined(pinned):
    """The pipelined host step: all steps enqueued back to back, outputs of
    every step kept in their own host buffers; after one final synchronise
    every step matches the oracle.  Pinned buffers take the zero-copy path
    (the kernel reads and writes host memory), pageable ones the staged
    copies."""
    import torch
    n, T = 41, 9
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=70), mbogen.env_seeds(33, n), T)
    pr = Pair(n, st, cap=100, exec_target=30, action_mode=lob.LOB_ACT_HOST)
    rng = np.random.default_rng(4)
    D = pr.env.D
    pin = (lambda x: x.pin_memory()) if pinned else (lambda x: x)
    acts = [pin(torch.from_numpy(rng.integers(0, 12, size=(n, 2)).astype(np.int32))) for _ in range(T)]
    ins, outs = [], []
    for t in range(T):
        lo, hi = st.offsets[:, t], st.offsets[:, t + 1]
        chunk = pin(torch.from_numpy(np.concatenate([st.msgs[lo[e]:hi[e]] for e in range(n)]).view(np.uint8)))
        off = np.zeros(n + 1, np.int64)
        off[1:] = np.cumsum(hi - lo)
        ins.append((chunk, off))
        outs.append((pin(torch.zeros((n, 2, D), dtype=torch.float32)), pin(torch.zeros((n, 2), dtype=torch.int64)),
                     pin(torch.zeros(n, dtype=torch.uint8))))
    stream = torch.cuda.Stream()
    for t in range(T):
        lob.lob_step_host_async(pr.env.h, ins[t][0], ins[t][1], acts[t], *outs[t], stream=stream)
    stream.synchronize()
    for t in range(T):
        pr.orc.step(acts[t].numpy())
        o_obs, o_rew, o_done = pr.orc.observe()
        np.testing.assert_allclose(outs[t][0].numpy(), o_obs, rtol=1e-6, atol=0)
        np.testing.assert_array_equal(outs[t][1].numpy(), o_rew)
        np.testing.assert_array_equal(outs[t][2].numpy(), o_done)
    pr.check_state()
    assert pr.env.sync() == 0
    pr.close()


def test_full_size_1024_envs_1000_steps():
    """The benchmark workload in the benchmark's launch configuration: 1,024
    envs x capacity 100 x 100 messages x 1,000 steps, random policy.  Every
    step: observations, rewards, actions and done flags of every env against
    the oracle; books, counters and agents at the end."""
    n, T = 1024, 1000
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=100), mbogen.env_seeds(1, n), T)
    pr = Pair(n, st, cap=100, exec_target=500, n_threads=os.cpu_count() or 1)
    for t in range(T):
        pr.env.step()
        pr.orc.step()
        pr.check_outputs()
    pr.check_state()
    assert pr.env.sync() == 0
    pr.close()


def test_error_status_paths():
    import torch
    n = 4
    bad = mbogen.generate(mbogen.MessageModel(msgs_per_step=10), mbogen.env_seeds(41, n), 2)
    msgs = bad.msgs.copy()
    msgs["type"][3] = 9                   # unknown type
    msgs["qty"][5] = 0 if msgs["type"][5] != 3 else msgs["qty"][5]
    bad.msgs = msgs
    pr = Pair(n, bad, cap=50, action_mode=lob.LOB_ACT_HOST)
    assert lob.lob_sync(pr.env.h) == 0
    pr.step(np.zeros((n, 2), np.int32))
    assert lob.lob_sync(pr.env.h) == lob.LOB_EBADMSG
    assert lob.lob_sync(pr.env.h) == 0                      # cleared after reporting
    pr.check_state()                                        # skipped messages counted like the oracle
    acts = torch.full((n, 2), 12, dtype=torch.int32, device="cuda")
    lob.lob_step(pr.env.h, acts)
    assert lob.lob_sync(pr.env.h) == lob.LOB_EINVAL
    with pytest.raises(lob.LobError) as ei:                 # window of 2 steps exhausted
        lob.lob_step(pr.env.h, acts)
    assert ei.value.code == lob.LOB_ESTATE
    pr.close()


def test_create_rejects_bad_configs():
    cfg = lob.lob_config(4, 2, 100, 10, 10, 1, 10, -1, 1, 0, 10000, 0)
    h = lob.lob_create(cfg)
    with pytest.raises(lob.LobError) as ei:                 # step before reset
        lob.lob_step(h)
    assert ei.value.code == lob.LOB_ESTATE
    lob.lob_destroy(h)
    for field, val, code in (("n_envs", 0, lob.LOB_EINVAL), ("n_agents", 1, lob.LOB_EINVAL),
                             ("cap_per_side", lob.LOB_MAX_CAP + 1, lob.LOB_ECAPACITY),
                             ("top_levels", 65, lob.LOB_EINVAL), ("exec_dir", 2, lob.LOB_EINVAL),
                             ("action_mode", 7, lob.LOB_EINVAL), ("reward_mode", 3, lob.LOB_EINVAL),
                             ("spooner_lambda_pct", 101, lob.LOB_EINVAL), ("inv_penalty", -1, lob.LOB_EINVAL),
                             ("exec_penalty_milli", -5, lob.LOB_EINVAL), ("mm_space", 3, lob.LOB_EINVAL),
                             ("pv_ref", 2, lob.LOB_EINVAL)):
        c = lob.lob_config(4, 2, 100, 10, 10, 1, 10, -1, 1, 0, 10000, 0)
        setattr(c, field, val)
        with pytest.raises(lob.LobError) as ei:
            lob.lob_create(c)
        assert ei.value.code == code, field


REWARD_CASES = [
    dict(reward_mode=lob.LOB_REWARD_BUYSELL),
    dict(reward_mode=lob.LOB_REWARD_SPOONER, spooner_lambda_pct=50),
    dict(reward_mode=lob.LOB_REWARD_SPOONER, spooner_lambda_pct=33, inv_penalty=50, exec_penalty_milli=100),
    dict(reward_mode=lob.LOB_REWARD_PV, inv_penalty=2, exec_penalty_milli=2500),
    dict(reward_mode=lob.LOB_REWARD_PV, pv_ref=lob.LOB_PV_MID, exec_penalty_milli=100),
]


@pytest.mark.parametrize("rw", REWARD_CASES, ids=lambda r: "-".join(f"{k}{v}" for k, v in r.items()))
def test_reward_variants_random_policy(rw):
    """Eqs. 3-4 and the Table 2 penalties: every reward of every step, whole
    episodes (the penalty lands on the last step), envs in every capacity class."""
    n, T = 96, 24
    caps = np.array([[5, 40, 100, 300, 700, 1000][e % 6] for e in range(n)], np.int32)
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=60), mbogen.env_seeds(31, n), T)
    pr = Pair(n, st, caps=caps, cap=int(caps.max()), exec_target=150, rewards=rw)
    for _ in range(T):
        pr.step()
        pr.check_outputs()
    pr.check_state()
    pr.close()


def test_reward_variants_host_actions_buy_task():
    n, T = 33, 16
    rng = np.random.default_rng(8)
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=50), mbogen.env_seeds(32, n), T)
    pr = Pair(n, st, cap=100, exec_target=300, exec_dir=1, mm_lot=4, action_mode=lob.LOB_ACT_HOST,
              rewards=dict(reward_mode=lob.LOB_REWARD_SPOONER, spooner_lambda_pct=71, inv_penalty=1,
                           exec_penalty_milli=10))
    for _ in range(T):
        pr.step(rng.integers(0, 12, size=(n, 2)).astype(np.int32))
        pr.check_outputs()
    pr.close()


@pytest.mark.parametrize("space,n_mm", [(lob.LOB_MM_FIXED_QUANT, 8), (lob.LOB_MM_DIRECTIONAL, 3)])
def test_mm_action_spaces(space, n_mm):
    """Fixed Quantity and directional market-maker heads (Sec. 4.1.1): random
    policy and host actions, every step's outputs and the final books."""
    n, T = 40, 15
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=60), mbogen.env_seeds(41 + space, n), T)
    pr = Pair(n, st, cap=100, exec_target=60, fill_cap=256, mm_space=space)
    for _ in range(T):
        pr.step()
        pr.check_outputs()
        pr.check_fills()
    pr.check_state()
    pr.close()
    rng = np.random.default_rng(space)
    pr = Pair(n, st, cap=100, exec_target=60, mm_space=space, action_mode=lob.LOB_ACT_HOST)
    for _ in range(T - 1):
        acts = np.stack([rng.integers(0, 12, n), rng.integers(0, n_mm, n)], axis=1).astype(np.int32)
        pr.step(acts)
        pr.check_outputs()
    pr.check_state()
    assert pr.env.sync() == 0
    # an action outside the space is reported
    import torch
    bad = np.zeros((n, 2), np.int32)
    bad[3, 1] = n_mm
    pr.env.step(torch.from_numpy(bad).cuda())
    assert pr.env.sync() == lob.LOB_EINVAL
    pr.close()


def _gold(name):
    import json
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        return json.load(f)


def test_reward_variants_hand_worked_on_gpu():
    """The hand-worked Sec. 5 / Table 2 fixture, through the kernel directly."""
    import torch
    from conftest import single_env_stream
    for sc in _gold("reward_variants.json")["scenarios"]:
        c = sc["config"]
        msgs, off = single_env_stream([s["msgs"] for s in sc["steps"]])
        for ex in sc["expected"]:
            rw = {k: v for k, v in ex.items() if k != "rewards"}
            env = lob.LobEnv(1, cap=c["cap"], top_levels=c["top_levels"], episode_len=c["episode_len"],
                             mm_lot=c["mm_lot"], exec_target=c["exec_target"], exec_dir=c["exec_dir"],
                             action_mode=lob.LOB_ACT_HOST, start_px=c["start_px"], **rw)
            md = torch.from_numpy(msgs.view(np.uint8).copy()).cuda() if len(msgs) else \
                torch.zeros(32, dtype=torch.uint8, device="cuda")
            env.load_messages(md, torch.from_numpy(off.copy()).cuda())
            env.reset(torch.tensor([7], dtype=torch.int64, device="cuda"))
            got = []
            for s in sc["steps"]:
                env.step(torch.tensor([s["actions"]], dtype=torch.int32, device="cuda"))
                got.append(env.observe()[1][0].cpu().tolist())
            assert got == ex["rewards"], (sc["name"], rw)
            assert env.sync() == 0
            env.close()


def test_stress_mix_cap1000_top20():
    """Heavy-tailed mix at capacity 1,000 per side: 30 % aggressive orders,
    Pareto(1.5) sizes capped at 10,000, delete bursts, top-20 levels."""
    n, T = 48, 6
    st = mbogen.generate(mbogen.STRESS_MODEL, mbogen.env_seeds(51, n), T)
    pr = Pair(n, st, cap=1000, top_levels=20, exec_target=2000, fill_cap=4096)
    for _ in range(T):
        pr.step()
        pr.check_outputs()
        pr.check_fills()
    pr.check_state()
    pr.close()


def _sampled_pair_check(n_all, sample, model, T, cap=None, caps=None, top_levels=10, exec_target=500,
                        rollout=False, graph=False):
    """All n_all envs on the GPU; the oracle runs the sampled envs only (env
    streams depend on their own seed only) and must agree on them exactly:
    observations, rewards and done flags of every sampled env at every step,
    then books, counters and agents."""
    import oracle
    import torch
    from harness import to_dev
    seeds = mbogen.env_seeds(77, n_all)
    st = mbogen.generate(model, seeds, T)
    caps_all = caps
    env = lob.LobEnv(n_all, cap=cap or 100, top_levels=top_levels, episode_len=T, exec_target=exec_target,
                     action_mode=lob.LOB_ACT_RANDOM, caps=caps_all)
    lob.lob_set_launch(env.h, 4, 1)
    md, od = to_dev(st.msgs), to_dev(st.offsets)
    del st
    env.load_messages(md, od)
    env.reset(to_dev(seeds))
    D = env.D
    sidx = torch.from_numpy(np.asarray(sample, np.int64)).cuda()
    if rollout:
        obs = torch.zeros((T, n_all, 2, D), dtype=torch.float32, device="cuda")
        rew = torch.zeros((T, n_all, 2), dtype=torch.int64, device="cuda")
        done = torch.zeros((T, n_all), dtype=torch.uint8, device="cuda")
        if graph:
            s_ = torch.cuda.Stream()
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s_):
                lob.lob_rollout(env.h, T, None, obs, rew, done, stream=s_)
            g.replay()
        else:
            lob.lob_rollout(env.h, T, None, obs, rew, done)
        torch.cuda.synchronize()
        g_obs = obs.index_select(1, sidx).cpu().numpy()
        g_rew = rew.index_select(1, sidx).cpu().numpy()
        g_done = done.index_select(1, sidx).cpu().numpy()
        del obs, rew, done
    else:
        g_obs = np.zeros((T, len(sample), 2, D), np.float32)
        g_rew = np.zeros((T, len(sample), 2), np.int64)
        g_done = np.zeros((T, len(sample)), np.uint8)
        for t in range(T):
            env.step()
            o_, r_, d_ = env.observe()
            g_obs[t] = o_.index_select(0, sidx).cpu().numpy()
            g_rew[t] = r_.index_select(0, sidx).cpu().numpy()
            g_done[t] = d_.index_select(0, sidx).cpu().numpy()
    assert env.sync() == 0
    g_cnt = env.counters().cpu().numpy()
    g_books = env.books()
    g_agents = env.agents().cpu().numpy()
    env.close()
    del md, od
    o = oracle.Oracle(len(sample), cap=cap or 100, top_levels=top_levels, episode_len=T, exec_target=exec_target,
                      action_mode=1, n_threads=os.cpu_count() or 1,
                      caps=None if caps is None else np.asarray(caps)[sample])
    sub = mbogen.generate(model, seeds[sample], T)
    o.reset(sub.seeds)
    o.load_messages(sub.msgs, sub.offsets)
    for t in range(T):
        o.step()
        o_obs, o_rew, o_done = o.observe()
        np.testing.assert_array_equal(g_rew[t], o_rew, err_msg=f"rewards at step {t}")
        np.testing.assert_allclose(g_obs[t], o_obs, rtol=1e-6, atol=0, err_msg=f"observations at step {t}")
        np.testing.assert_array_equal(g_done[t], o_done, err_msg=f"done at step {t}")
    np.testing.assert_array_equal(g_cnt[sample], o.counters())
    np.testing.assert_array_equal(g_agents[sample], o.agents())
    for i, e in enumerate(sample):
        n2, px, qty, oid, ts = o.book(i)
        b = g_books[e]
        assert b["n"].tolist() == n2.tolist()
        for sd in range(2):
            k = n2[sd]
            np.testing.assert_array_equal(b["px"][sd][:k], px[sd][:k])
            np.testing.assert_array_equal(b["qty"][sd][:k], qty[sd][:k])
            np.testing.assert_array_equal(b["id"][sd][:k], oid[sd][:k])
            np.testing.assert_array_equal(b["ts"][sd][:k], ts[sd][:k])


def test_uneven_batch_8192_envs_one_graph_launch():
    """The uneven batch at its stated length: 8,192 envs, capacities uniform in
    {50, 100, 200, 500}, M_t ~ Poisson with lambda log-uniform in [10, 500],
    all 500 steps in one persistent launch under a captured CUDA graph; every
    64th env checked against the oracle at every step."""
    n = 8192
    caps = mbogen.env_caps(5, n)
    _sampled_pair_check(n, np.arange(0, n, 64), mbogen.MessageModel(poisson=True), 500, cap=500, caps=caps,
                        rollout=True, graph=True)


def test_uneven_batch_one_kernel_over_all_classes():
    """The uneven batch's classes (capacities 50, 100, 200, 500 and a few of 20)
    in one persistent launch whose warps steal smaller classes' envs, for two
    block splits; every 16th of 2,048 envs checked at every step."""
    import oracle
    import torch
    from harness import to_dev
    n, T = 2048, 30
    caps = mbogen.env_caps(9, n, choices=(20, 50, 100, 200, 500))
    seeds = mbogen.env_seeds(78, n)
    st = mbogen.generate(mbogen.MessageModel(poisson=True), seeds, T)
    sample = np.arange(0, n, 16)
    sub = mbogen.generate(mbogen.MessageModel(poisson=True), seeds[sample], T)
    for split in ((1, 1, 1, 1, 1, 0), (0, 0, 0, 0, 6, 0)):   # one warp per class; all warps of the largest
        env = lob.LobEnv(n, cap=500, episode_len=T, exec_target=300, action_mode=lob.LOB_ACT_RANDOM, caps=caps)
        lob.lob_set_multi_split(env.h, np.array(split, np.int32))
        env.load_messages(to_dev(st.msgs), to_dev(st.offsets))
        env.reset(to_dev(seeds))
        D = env.D
        obs = torch.zeros((T, n, 2, D), dtype=torch.float32, device="cuda")
        rew = torch.zeros((T, n, 2), dtype=torch.int64, device="cuda")
        lob.lob_rollout(env.h, T, None, obs, rew, None)
        assert env.sync() == 0
        sidx = torch.from_numpy(sample).cuda()
        g_obs = obs.index_select(1, sidx).cpu().numpy()
        g_rew = rew.index_select(1, sidx).cpu().numpy()
        g_cnt = env.counters().cpu().numpy()[sample]
        env.close()
        o = oracle.Oracle(len(sample), cap=500, episode_len=T, exec_target=300, action_mode=1,
                          n_threads=os.cpu_count() or 1, caps=caps[sample])
        o.reset(sub.seeds)
        o.load_messages(sub.msgs, sub.offsets)
        for t in range(T):
            o.step()
            o_obs, o_rew, _ = o.observe()
            np.testing.assert_array_equal(g_rew[t], o_rew, err_msg=f"split {split} step {t}")
            np.testing.assert_allclose(g_obs[t], o_obs, rtol=1e-6, atol=0)
        np.testing.assert_array_equal(g_cnt, o.counters())


def test_stress_65536_envs_cap1000():
    """65,536 envs x capacity 1,000 x 1,000 messages of the heavy-tailed mix,
    top-20 levels (a window of 4 steps, random policy); every 256th env
    checked at every step."""
    n = 65536
    _sampled_pair_check(n, np.arange(0, n, 256), mbogen.STRESS_MODEL, 4, cap=1000, top_levels=20,
                        exec_target=2000)


def test_stress_full_length_with_bf16_policy_every_256th_env():
    """The stress configuration at its stated length: 65,536 envs x capacity
    1,000 x 1,000 messages x 256 steps (16.8 G messages, generated on the
    device 8 steps at a time into a double-buffered ring), top-20
    observations, actions from the BF16 policy.  Every 256th env: the GPU's
    actions replayed into the oracle give identical observations, rewards and
    done flags at every step, and identical books and counters at the end."""
    import oracle
    import torch
    n, T, C = 65536, 256, 8
    sample = np.arange(0, n, 256)
    sidx = torch.from_numpy(sample).cuda()
    seeds = mbogen.env_seeds(4, n)
    gen = mbogen.GpuStreams(mbogen.STRESS_MODEL, seeds)
    M = mbogen.STRESS_MODEL.msgs_per_step
    ring = [torch.empty(n * C * M * 32, dtype=torch.uint8, device="cuda") for _ in range(2)]
    off = torch.from_numpy(gen.offsets(C)).cuda()
    env = lob.LobEnv(n, cap=1000, top_levels=20, episode_len=T, exec_target=2000, action_mode=lob.LOB_ACT_HOST)
    params = lob.init_policy_params(7, 2, env.D)
    pol = lob.lob_policy_create(2, env.D, params)
    lob.lob_set_launch(env.h, 4, 1)
    env.reset(torch.from_numpy(seeds.view(np.int64).copy()).cuda())
    D = env.D
    obs = torch.zeros((C, n, 2, D), dtype=torch.float32, device="cuda")
    rew = torch.zeros((C, n, 2), dtype=torch.int64, device="cuda")
    done = torch.zeros((C, n), dtype=torch.uint8, device="cuda")
    acts = torch.zeros((C, n, 2), dtype=torch.int32, device="cuda")
    g_obs, g_rew, g_done, g_acts = [], [], [], []
    for k in range(T // C):
        gen.chunk(C, ring[k % 2])
        env.load_messages(ring[k % 2], off)
        lob.lob_rollout_policy(env.h, pol, C, lob.LOB_PREC_BF16, obs, rew, done, acts)
        g_obs.append(obs.index_select(1, sidx).cpu().numpy())
        g_rew.append(rew.index_select(1, sidx).cpu().numpy())
        g_done.append(done.index_select(1, sidx).cpu().numpy())
        g_acts.append(acts.index_select(1, sidx).cpu().numpy())
    assert gen.ok()
    assert env.sync() == 0 and lob.lob_policy_sync(pol) == 0
    g_cnt = env.counters().cpu().numpy()[sample]
    g_books = env.books()
    lob.lob_policy_destroy(pol)
    env.close()
    gen.close()
    del ring, obs, rew, done, acts
    g_obs, g_rew = np.concatenate(g_obs), np.concatenate(g_rew)
    g_done, g_acts = np.concatenate(g_done), np.concatenate(g_acts)
    sub = mbogen.generate(mbogen.STRESS_MODEL, seeds[sample], T)
    o = oracle.Oracle(len(sample), cap=1000, top_levels=20, episode_len=T, exec_target=2000,
                      action_mode=lob.LOB_ACT_HOST, n_threads=os.cpu_count() or 1)
    o.reset(sub.seeds)
    o.load_messages(sub.msgs, sub.offsets)
    for t in range(T):
        o.step(g_acts[t])
        o_obs, o_rew, o_done = o.observe()
        np.testing.assert_array_equal(g_rew[t], o_rew, err_msg=f"rewards at step {t}")
        np.testing.assert_allclose(g_obs[t], o_obs, rtol=1e-6, atol=0, err_msg=f"observations at step {t}")
        np.testing.assert_array_equal(g_done[t], o_done)
    np.testing.assert_array_equal(g_cnt, o.counters())
    for i, e in enumerate(sample):
        n2, px, qty, oid, ts = o.book(i)
        b = g_books[e]
        assert b["n"].tolist() == n2.tolist()
        for sd in range(2):
            kk = n2[sd]
            np.testing.assert_array_equal(b["px"][sd][:kk], px[sd][:kk])
            np.testing.assert_array_equal(b["id"][sd][:kk], oid[sd][:kk])
            np.testing.assert_array_equal(b["ts"][sd][:kk], ts[sd][:kk])


def test_checkpoint_resume_bit_identical():
    """Save after 5 steps, run 6 more; restore (same handle, and a fresh handle
    from a host copy) and run the 6 steps again: identical outputs and state."""
    import torch
    from harness import to_dev
    n, T = 61, 11
    caps = mbogen.env_caps(8, n, choices=(50, 100, 200))
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=80), mbogen.env_seeds(81, n), T)
    md, od, sd = to_dev(st.msgs), to_dev(st.offsets), to_dev(st.seeds)

    def make():
        env = lob.LobEnv(n, cap=200, caps=caps, episode_len=T, exec_target=60, action_mode=lob.LOB_ACT_RANDOM)
        env.load_messages(md, od)
        return env

    def run(env, k):
        outs = []
        for _ in range(k):
            env.step()
            o, r, d = env.observe()
            outs.append((o.clone(), r.clone(), d.clone()))
        return outs

    env = make()
    env.reset(sd)
    run(env, 5)
    ck = torch.zeros(lob.lob_checkpoint_bytes(env.h), dtype=torch.uint8, device="cuda")
    lob.lob_save(env.h, ck)
    host = torch.zeros(ck.numel(), dtype=torch.uint8).pin_memory()
    lob.lob_save(env.h, host)
    first = run(env, 6)
    final_books = env.books()
    final_cnt = env.counters().cpu().numpy()
    lob.lob_load(env.h, ck)
    again = run(env, 6)
    env2 = make()
    lob.lob_load(env2.h, host)
    third = run(env2, 6)
    for a, b, c in zip(first, again, third):
        for x, y, z in zip(a, b, c):
            assert torch.equal(x, y) and torch.equal(x, z)
    for got in (env.books(), env2.books()):
        for b0, b1 in zip(final_books, got):
            assert b0.tobytes() == b1.tobytes()
    np.testing.assert_array_equal(final_cnt, env2.counters().cpu().numpy())
    # a checkpoint of another shape is refused
    other = lob.LobEnv(n + 1, cap=100, episode_len=T, action_mode=lob.LOB_ACT_RANDOM)
    with pytest.raises(lob.LobError) as ei:
        lob.lob_load(other.h, host)
    assert ei.value.code == lob.LOB_EINVAL
    for e in (env, env2, other):
        e.close()


def _with_malformed(st):
    msgs = st.msgs.copy()
    msgs["type"][5] = 9
    msgs["side"][17] = 0
    msgs["qty"][23] = 0 if msgs["type"][23] != 3 else msgs["qty"][23]
    st.msgs = msgs
    return st


def test_compact_messages_parity():
    """The GPU reads 16-byte compact records, the oracle the 32-byte originals
    (malformed ones included): every step's outputs, fills and the final state."""
    n, T = 37, 12
    st = _with_malformed(mbogen.generate(mbogen.MessageModel(msgs_per_step=75), mbogen.env_seeds(91, n), T))
    pr = Pair(n, st, cap=100, exec_target=60, fill_cap=512, compact=True)
    for _ in range(T):
        pr.step()
        pr.check_outputs()
        pr.check_fills()
    pr.check_state()
    assert pr.env.sync() == lob.LOB_EBADMSG
    pr.close()


def test_compact_messages_rollout_agents_and_episodes():
    import torch
    n, T = 30, 10
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=90), mbogen.env_seeds(92, n), T)
    pr = Pair(n, st, n_agents=6, cap=200, exec_target=40, compact=True)
    obs = torch.zeros((T, n, 6, pr.env.D), dtype=torch.float32, device="cuda")
    rew = torch.zeros((T, n, 6), dtype=torch.int64, device="cuda")
    done = torch.zeros((T, n), dtype=torch.uint8, device="cuda")
    lob.lob_rollout(pr.env.h, T, None, obs, rew, done)
    for t in range(T):
        pr.orc.step()
        o_obs, o_rew, o_done = pr.orc.observe()
        np.testing.assert_allclose(obs[t].cpu().numpy(), o_obs, rtol=1e-6, atol=0)
        np.testing.assert_array_equal(rew[t].cpu().numpy(), o_rew)
    pr.check_state()
    pr.check_outputs()
    pr.close()
    ds = mbogen.generate(mbogen.MessageModel(msgs_per_step=60), mbogen.env_seeds(93, 1), 30)
    steps = np.random.default_rng(93).integers(0, 30 - 4 + 1, size=5)
    starts, levels = mbogen.start_books(93, ds.mids[0], steps, 10)
    pr = Pair(n, ds, cap=100, episode_len=4, exec_target=30, episodes=(starts, levels),
              seeds=mbogen.env_seeds(94, n), compact=True)
    for _ in range(9):
        pr.step()
        pr.check_outputs()
    pr.check_state()
    pr.close()


def test_pack_kernel_matches_packer():
    import torch
    from harness import to_dev
    st = _with_malformed(mbogen.generate(mbogen.MessageModel(msgs_per_step=64), mbogen.env_seeds(95, 8), 6))
    n = len(st.msgs)
    src = to_dev(st.msgs)
    dst = torch.zeros(n * 16, dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    lob.lob_pack_messages16(src, n, dst, status)
    assert dst.cpu().numpy().tobytes() == mbogen.pack16(st.msgs).tobytes()
    assert int(status.item()) == 0
    big = st.msgs[:4].copy()
    big["oid"][2] = 1 << 60
    src = to_dev(big)
    dst = torch.zeros(4 * 16, dtype=torch.uint8, device="cuda")
    lob.lob_pack_messages16(src, 4, dst, status)
    assert int(status.item()) == lob.LOB_EINVAL


def test_misaligned_message_buffer_rejected():
    import torch
    from harness import to_dev
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=10), mbogen.env_seeds(96, 2), 3)
    env = lob.LobEnv(2, cap=50, episode_len=3)
    raw = torch.zeros(len(st.msgs) * 32 + 16, dtype=torch.uint8, device="cuda")
    off = to_dev(st.offsets)
    with pytest.raises(lob.LobError) as ei:
        env.load_messages(raw[8:], off)
    assert ei.value.code == lob.LOB_EINVAL
    env.close()


@pytest.mark.parametrize("price_p,cap", [(0.02, 100), (0.05, 200), (0.1, 100), (0.05, 8)])
def test_wide_price_spans_leave_the_ladder(price_p, cap):
    """Add prices spread over hundreds of ticks: many sides come to span more
    than the step kernel's 128-tick price ladder, so envs switch to the
    sorted-index form in the middle of a step (and later steps start in it
    when the loaded book is already that wide), while others stay on the
    ladder.  Every step must still match the oracle."""
    n, T = 33, 12
    model = mbogen.MessageModel(price_p=price_p, msgs_per_step=80)
    st = mbogen.generate(model, mbogen.env_seeds(300 + int(price_p * 100) + cap, n), T)
    pr = Pair(n, st, cap=cap, exec_target=100, fill_cap=512)
    for _ in range(T):
        pr.step()
        pr.check_outputs()
        pr.check_fills()
    pr.check_state()
    assert pr.env.sync() == 0
    pr.close()


@pytest.mark.parametrize("side", [1, -1])
def test_ladder_window_edge_by_hand(side):
    """One env, no agents: orders at 127 ticks from the best still fit the
    ladder; one at 128 ticks converts the env to the sorted form in the middle
    of the step; a sweep, cancels and rests follow in both forms.  The book and
    fills after every step equal the oracle's."""
    from conftest import single_env_stream
    import types
    s = side
    far, edge = 10_000 - s * 127, 10_000 - s * 128
    steps = [
        # type, side, px, qty, oid
        [(1, s, 10_000, 5, 1), (1, s, far, 5, 2), (1, s, 10_000 - s * 60, 7, 3), (1, s, far, 2, 4)],
        [(1, s, edge, 3, 5), (1, s, 10_000 - s * 5, 4, 6), (2, s, far, 1, 2), (3, s, 10_000, 0, 1)],
        [(4, -s, 0, 20, 7), (1, s, 10_000 - s * 3, 9, 8), (1, -s, 10_000 + s * 50, 6, 9)],
        [(1, -s, edge, 30, 10), (1, s, 10_000, 2, 11)],
    ]
    msgs, off = single_env_stream(steps)
    st = types.SimpleNamespace(msgs=msgs, offsets=off, seeds=np.array([5], np.uint64))
    pr = Pair(1, st, n_agents=0, cap=100, fill_cap=64)
    for _ in range(len(steps)):
        pr.step()
        pr.check_outputs()
        pr.check_fills()
        pr.check_state()
    assert pr.env.sync() == 0
    pr.close()

"""Several agents per type on the GPU (Sec. 3, Table 1: 1, 5 and 10 agents
of each type) vs. the CPU oracle, through the C ABI."""
import json
import os

import numpy as np
import pytest

from harness import Pair, to_dev
from paper_2511_02136_gb300 import lob, mbogen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    lob.build()
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"


@pytest.mark.parametrize("P", [2, 5, 10])
def test_agents_per_type_random_policy(P):
    """Every step: outputs, per-agent actions and the fill log; at the end
    books, counters and per-agent state."""
    n, T = 37, 14
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=45), mbogen.env_seeds(50 + P, n), T)
    pr = Pair(n, st, n_agents=2 * P, cap=100, exec_target=40, fill_cap=512)
    for _ in range(T):
        pr.step()
        pr.check_outputs()
        pr.check_fills()
    pr.check_state()
    assert pr.env.sync() == 0
    pr.close()


@pytest.mark.parametrize("cap", [8, 40, 100, 250, 600, 1000])
def test_agents_per_type_each_capacity_class(cap):
    n, T = 24, 8
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=60), mbogen.env_seeds(60 + cap, n), T)
    pr = Pair(n, st, n_agents=10, cap=cap, exec_target=30)
    for _ in range(T):
        pr.step()
        pr.check_outputs()
    pr.check_state()
    pr.close()


def test_agents_per_type_host_actions_variants():
    """Host actions over each type's space, Fixed Quantity market makers,
    Spooner reward with penalties, a buy task."""
    n, T, P = 29, 10, 3
    rng = np.random.default_rng(9)
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=50), mbogen.env_seeds(71, n), T)
    pr = Pair(n, st, n_agents=2 * P, cap=100, exec_target=50, exec_dir=1, mm_lot=2,
              action_mode=lob.LOB_ACT_HOST, mm_space=lob.LOB_MM_FIXED_QUANT,
              rewards=dict(reward_mode=lob.LOB_REWARD_SPOONER, spooner_lambda_pct=25, inv_penalty=2,
                           exec_penalty_milli=300, pv_ref=lob.LOB_PV_MID))
    for _ in range(T):
        acts = np.concatenate([rng.integers(0, 12, (n, P)), rng.integers(0, 8, (n, P))], axis=1).astype(np.int32)
        pr.step(acts)
        pr.check_outputs()
    pr.check_state()
    assert pr.env.sync() == 0
    pr.close()


def test_agents_per_type_rollout_with_episodes():
    """Five agents per type in episode mode: one rollout launch of 3T + 1
    steps resets the agents on chip at every episode end."""
    import torch
    n, T, P = 30, 4, 5
    A = 2 * P
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=70), mbogen.env_seeds(81, 1), 40)
    steps = np.random.default_rng(81).integers(0, 40 - T + 1, size=6)
    starts, levels = mbogen.start_books(81, st.mids[0], steps, 12)
    K = 3 * T + 1
    pr = Pair(n, st, n_agents=A, cap=100, episode_len=T, exec_target=30, episodes=(starts, levels),
              seeds=mbogen.env_seeds(82, n))
    D = pr.env.D
    obs = torch.zeros((K, n, A, D), dtype=torch.float32, device="cuda")
    rew = torch.zeros((K, n, A), dtype=torch.int64, device="cuda")
    done = torch.zeros((K, n), dtype=torch.uint8, device="cuda")
    lob.lob_rollout(pr.env.h, K, None, obs, rew, done)
    for t in range(K):
        pr.orc.step()
        o_obs, o_rew, o_done = pr.orc.observe()
        np.testing.assert_allclose(obs[t].cpu().numpy(), o_obs, rtol=1e-6, atol=0)
        np.testing.assert_array_equal(rew[t].cpu().numpy(), o_rew)
        np.testing.assert_array_equal(done[t].cpu().numpy(), o_done)
    pr.check_state()
    pr.check_outputs()
    pr.close()


def test_agents_per_type_hand_worked_on_gpu():
    import torch
    from conftest import single_env_stream
    with open(os.path.join(os.path.dirname(__file__), "golden", "multi_agent.json")) as f:
        g = json.load(f)
    c = g["config"]
    A = 2 * c["agents_per_type"]
    msgs, off = single_env_stream([s["msgs"] for s in g["steps"]])
    env = lob.LobEnv(1, n_agents=A, cap=c["cap"], top_levels=c["top_levels"], episode_len=c["episode_len"],
                     mm_lot=c["mm_lot"], exec_target=c["exec_target"], exec_dir=c["exec_dir"],
                     action_mode=lob.LOB_ACT_HOST, start_px=c["start_px"])
    env.load_messages(to_dev(msgs), to_dev(off))
    env.reset(torch.tensor([5], dtype=torch.int64, device="cuda"))

    def owner(oid):
        return A if oid >= 0 else (-oid - 1) % A

    for s in g["steps"]:
        env.step(torch.tensor([s["actions"]], dtype=torch.int32, device="cuda"))
        obs, rew, done = env.observe()
        b = env.books()[0]
        for sd, key in enumerate(("bids", "asks")):
            got = [[int(b["px"][sd][i]), int(b["qty"][sd][i]), owner(int(b["id"][sd][i]))]
                   for i in range(int(b["n"][sd]))]
            assert got == s[key]
        np.testing.assert_array_equal(obs[0].cpu().numpy(), np.array(s["obs"], np.float32))
        assert rew[0].cpu().tolist() == s["rewards"]
        assert int(done[0]) == s["done"]
    assert env.agents()[0].cpu().tolist() == g["final_agents"]
    assert env.sync() == 0
    env.close()


def test_agents_per_type_checkpoint_resume():
    import torch
    n, T, A = 25, 12, 8
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=60), mbogen.env_seeds(91, n), T)
    md, od, sd = to_dev(st.msgs), to_dev(st.offsets), to_dev(st.seeds)

    def make():
        env = lob.LobEnv(n, n_agents=A, cap=100, episode_len=T, exec_target=40)
        env.load_messages(md, od)
        return env

    def run(env, k):
        out = []
        for _ in range(k):
            env.step()
            o, r, d = env.observe()
            out.append((o.clone(), r.clone(), d.clone(), env.agents().clone()))
        return out

    env = make()
    env.reset(sd)
    run(env, 4)
    host = torch.zeros(lob.lob_checkpoint_bytes(env.h), dtype=torch.uint8).pin_memory()
    lob.lob_save(env.h, host)
    first = run(env, 6)
    env2 = make()
    lob.lob_load(env2.h, host)
    second = run(env2, 6)
    for a, b in zip(first, second):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    env.close()
    env2.close()


def test_agents_per_type_config_limits():
    import torch
    for A in (3, 2 * lob.LOB_MAX_PER_TYPE + 2):
        with pytest.raises(lob.LobError) as ei:
            lob.LobEnv(2, n_agents=A)
        assert ei.value.code == lob.LOB_EINVAL
    env = lob.LobEnv(4, n_agents=6, action_mode=lob.LOB_ACT_HOST, episode_len=3)
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=5), mbogen.env_seeds(1, 4), 3)
    env.load_messages(to_dev(st.msgs), to_dev(st.offsets))
    env.reset(to_dev(st.seeds))
    bad = torch.zeros((4, 6), dtype=torch.int32, device="cuda")
    bad[1, 4] = 12                                       # market maker action outside 0..11
    env.step(bad)
    assert env.sync() == lob.LOB_EINVAL
    env.close()


def test_most_agents_smallest_books():
    """The largest agent count (16 per type, up to 48 agent orders a step) on
    the smallest capacity class: the agents' chunk is the longest and the
    per-warp buffers the smallest."""
    n, T = 12, 10
    P = lob.LOB_MAX_PER_TYPE
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=40), mbogen.env_seeds(170, n), T)
    pr = Pair(n, st, n_agents=2 * P, cap=20, exec_target=50, fill_cap=512)
    for _ in range(T):
        pr.step()
        pr.check_outputs()
        pr.check_fills()
    pr.check_state()
    assert pr.env.sync() == 0
    pr.close()

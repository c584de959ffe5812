"""Episode mode on the GPU (one shared message stream, snapshot starts,
auto-reset inside the step kernel) vs. the CPU oracle, through the C ABI."""
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


def _dataset(seed, n_data, T, n_starts, ls, msgs_per_step=80, min_levels=0):
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=msgs_per_step), mbogen.env_seeds(seed, 1), n_data)
    rng = np.random.default_rng(seed)
    steps = rng.integers(0, n_data - T + 1, size=n_starts)
    starts, levels = mbogen.start_books(seed, st.mids[0], steps, ls, min_levels=min_levels)
    return st, starts, levels


@pytest.mark.parametrize("cap", [8, 40, 100, 250, 600, 1000])
def test_episodes_random_policy_each_capacity_class(cap):
    """Envs cross three episode boundaries; the snapshots overlap in the data
    and some have empty sides.  Every step's outputs and the final books match."""
    n, T = 45, 5
    st, starts, levels = _dataset(100 + cap, 60, T, 9, min(cap, 24))
    pr = Pair(n, st, cap=cap, episode_len=T, exec_target=70, episodes=(starts, levels),
              seeds=mbogen.env_seeds(7 + cap, n))
    for _ in range(3 * T + 2):
        pr.step()
        pr.check_outputs()
    pr.check_state()
    assert pr.env.sync() == 0
    pr.close()


def test_episodes_host_actions_and_reward_variants():
    n, T = 33, 4
    rng = np.random.default_rng(3)
    st, starts, levels = _dataset(61, 40, T, 5, 10, msgs_per_step=50)
    pr = Pair(n, st, cap=100, episode_len=T, exec_target=30, exec_dir=1, mm_lot=2, action_mode=lob.LOB_ACT_HOST,
              episodes=(starts, levels), seeds=mbogen.env_seeds(62, n),
              rewards=dict(reward_mode=lob.LOB_REWARD_SPOONER, spooner_lambda_pct=40, inv_penalty=1,
                           exec_penalty_milli=250))
    for _ in range(3 * T):
        pr.step(rng.integers(0, 12, size=(n, 2)).astype(np.int32))
        pr.check_outputs()
    pr.check_state()
    pr.close()


def test_episodes_rollout_resets_inside_one_launch():
    """One persistent launch of 3T + 1 steps: the env resets on chip at every
    episode end; per-step outputs and final state match the stepwise oracle."""
    import torch
    n, T = 50, 4
    st, starts, levels = _dataset(71, 30, T, 6, 16)
    K = 3 * T + 1
    for persistent in (0, 1):
        pr = Pair(n, st, cap=100, episode_len=T, exec_target=40, episodes=(starts, levels),
                  seeds=mbogen.env_seeds(72, n), persistent=persistent)
        D = pr.env.D
        obs = torch.zeros((K, n, 2, D), dtype=torch.float32, device="cuda")
        rew = torch.zeros((K, n, 2), dtype=torch.int64, device="cuda")
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


def test_episodes_hand_worked_on_gpu():
    """The hand-worked two-episode fixture, through the kernel."""
    import torch
    from conftest import single_env_stream
    with open(os.path.join(os.path.dirname(__file__), "golden", "episodes.json")) as f:
        g = json.load(f)
    c = g["config"]
    msgs, off = single_env_stream(g["data_steps"])
    starts = np.zeros(len(g["starts"]), lob.START_DTYPE)
    levels = np.zeros((len(g["starts"]), 2, 4, 2), np.int32)
    for j, s in enumerate(g["starts"]):
        starts[j] = (s["data_step"], s["last_px"], len(s["bids"]), len(s["asks"]))
        for sd, key in enumerate(("bids", "asks")):
            for i, lv in enumerate(s[key]):
                levels[j, sd, i] = lv
    env = lob.LobEnv(1, cap=c["cap"], top_levels=c["top_levels"], episode_len=c["episode_len"],
                     mm_lot=c["mm_lot"], exec_target=c["exec_target"], exec_dir=c["exec_dir"],
                     action_mode=lob.LOB_ACT_HOST, start_px=c["start_px"])
    md, od = to_dev(msgs), to_dev(off[0])
    env.set_episodes(md, od, starts, levels)
    env.reset(torch.tensor([c["seed"]], dtype=torch.int64, device="cuda"))

    def labelled():
        b = env.books()[0]
        out = []
        for sd in range(2):
            rows = []
            for i in range(int(b["n"][sd])):
                oid = int(b["id"][sd][i])
                init = oid >= lob.LOB_INIT_ID
                rows.append([int(b["px"][sd][i]), int(b["qty"][sd][i]), "init" if init else "bg",
                             oid - lob.LOB_INIT_ID if init else oid, int(b["ts"][sd][i])])
            out.append(rows)
        return out

    r = g["reset"]
    assert env.episode_starts().cpu().tolist() == [r["episode_start"]]
    assert labelled() == [r["bids"], r["asks"]]
    np.testing.assert_array_equal(env.observe()[0][0, 0].cpu().numpy(), np.array(r["obs"], np.float32))
    for s in g["steps"]:
        env.step(torch.tensor([s["actions"]], dtype=torch.int32, device="cuda"))
        obs, rew, done = env.observe()
        assert env.episode_starts().cpu().tolist() == [s["episode_start"]]
        assert labelled() == [s["bids"], s["asks"]]
        for a in range(2):
            np.testing.assert_array_equal(obs[0, a].cpu().numpy(), np.array(s["obs"], np.float32))
        assert rew[0].cpu().tolist() == s["rewards"]
        assert int(done[0]) == s["done"]
    assert env.sync() == 0
    env.close()


def test_episode_tables_rejected_and_call_order():
    import torch
    st, starts, levels = _dataset(5, 20, 4, 3, 6, min_levels=2)
    md, od = to_dev(st.msgs), to_dev(st.offsets[0])

    def attempt(starts_, levels_, env=None, code=lob.LOB_EINVAL):
        e = env or lob.LobEnv(2, cap=6, episode_len=4)
        with pytest.raises(lob.LobError) as ei:
            e.set_episodes(md, od, starts_, levels_)
        assert ei.value.code == code
        if env is None:
            e.close()

    bad = starts.copy(); bad[0]["data_step"] = 17            # 17 + 4 > 20 data steps
    attempt(bad, levels)
    bad = starts.copy(); bad[1]["n_bid"] = 7                  # more levels than given
    attempt(bad, levels)
    lv = levels.copy(); lv[0, 0, 1, 0] = lv[0, 0, 0, 0]       # bid prices not strictly falling
    attempt(starts, lv)
    lv = levels.copy(); lv[2, 1, 0, 1] = 0                    # zero quantity
    attempt(starts, lv)
    lv = levels.copy(); lv[0, 0, 0, 0] = lv[0, 1, 0, 0]       # crossed snapshot
    attempt(starts, lv)
    small = lob.LobEnv(2, cap=1, episode_len=4)                # two bid levels > capacity 1
    attempt(starts, levels, env=small)
    small.close()
    per_env = lob.LobEnv(2, cap=6, caps=np.array([6, 6], np.int32), episode_len=4)
    attempt(starts, levels, env=per_env)                       # per-env capacities
    per_env.close()
    env = lob.LobEnv(2, cap=6, episode_len=4)
    env.set_episodes(md, od, starts, levels)
    with pytest.raises(lob.LobError) as ei:                    # set_episodes needs a reset
        env.step()
    assert ei.value.code == lob.LOB_ESTATE
    env.reset(to_dev(mbogen.env_seeds(1, 2)))
    for _ in range(9):                                         # past T: episodes continue
        env.step()
    assert env.sync() == 0
    env.close()


def test_episodes_checkpoint_resume():
    """A checkpoint taken mid-episode resumes bit-identically across later
    episode boundaries in a fresh handle given the same episode table."""
    import torch
    n, T = 40, 5
    st, starts, levels = _dataset(91, 40, T, 7, 20)
    md, od = to_dev(st.msgs), to_dev(st.offsets[0])
    sd = to_dev(mbogen.env_seeds(92, n))

    def make():
        env = lob.LobEnv(n, cap=100, episode_len=T, exec_target=50)
        env.set_episodes(md, od, starts, levels)
        return env

    def run(env, k):
        outs = []
        for _ in range(k):
            env.step()
            o, r, d = env.observe()
            outs.append((o.clone(), r.clone(), d.clone(), env.episode_starts().clone()))
        return outs

    env = make()
    env.reset(sd)
    run(env, 7)
    host = torch.zeros(lob.lob_checkpoint_bytes(env.h), dtype=torch.uint8).pin_memory()
    lob.lob_save(env.h, host)
    first = run(env, 11)
    env2 = make()
    lob.lob_load(env2.h, host)
    second = run(env2, 11)
    for a, b in zip(first, second):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    plain = lob.LobEnv(n, cap=100, episode_len=T, exec_target=50)   # not in episode mode
    with pytest.raises(lob.LobError) as ei:
        lob.lob_load(plain.h, host)
    assert ei.value.code == lob.LOB_EINVAL
    for e in (env, env2, plain):
        e.close()

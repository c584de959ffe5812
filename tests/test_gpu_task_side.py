"""The execution task's side drawn per env and episode (Table 2: the task
direction is sampled uniformly) on the GPU vs. the CPU oracle, through the
C ABI.  With exec_dir = 0 the remaining-target observation is signed
(+ buy, - sell), so every obs comparison also checks the drawn side."""
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


def _signs(obs, L, P):
    """Signs of the execution agents' remaining-target entries."""
    return np.sign(obs[:, :P, 4 * L + 3])


def test_drawn_side_random_policy_both_sides_occur():
    n, T, L = 64, 10, 10
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=60), mbogen.env_seeds(140, n), T)
    pr = Pair(n, st, cap=100, top_levels=L, exec_target=80, exec_dir=0, fill_cap=256)
    obs, _ = pr.check_outputs()
    s = _signs(obs, L, 1)
    assert (s > 0).any() and (s < 0).any(), "both task sides among 64 envs"
    for _ in range(T):
        pr.step()
        pr.check_outputs()
        pr.check_fills()
    pr.check_state()
    assert pr.env.sync() == 0
    pr.close()


@pytest.mark.parametrize("cap", [8, 40, 250, 1000])
def test_drawn_side_host_actions_each_capacity_class(cap):
    n, T = 29, 8
    rng = np.random.default_rng(cap)
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=50), mbogen.env_seeds(141 + cap, n), T)
    pr = Pair(n, st, cap=cap, exec_target=40, exec_dir=0, mm_lot=2, action_mode=lob.LOB_ACT_HOST,
              rewards=dict(reward_mode=lob.LOB_REWARD_BUYSELL, exec_penalty_milli=500))
    for _ in range(T):
        pr.step(rng.integers(0, 12, size=(n, 2)).astype(np.int32))
        pr.check_outputs()
    pr.check_state()
    pr.close()


def test_drawn_side_redrawn_each_episode():
    """Episode mode: the side is drawn again at every auto-reset, inside the
    step kernel; one rollout launch crosses three episode boundaries."""
    import torch
    n, T, L = 40, 4, 10
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=70), mbogen.env_seeds(142, 1), 40)
    steps = np.random.default_rng(142).integers(0, 40 - T + 1, size=6)
    starts, levels = mbogen.start_books(142, st.mids[0], steps, 12)
    K = 3 * T + 1
    pr = Pair(n, st, cap=100, top_levels=L, episode_len=T, exec_target=30, exec_dir=0,
              episodes=(starts, levels), seeds=mbogen.env_seeds(143, n))
    D = pr.env.D
    obs = torch.zeros((K, n, 2, D), dtype=torch.float32, device="cuda")
    rew = torch.zeros((K, n, 2), dtype=torch.int64, device="cuda")
    done = torch.zeros((K, n), dtype=torch.uint8, device="cuda")
    lob.lob_rollout(pr.env.h, K, None, obs, rew, done)
    changed = 0
    first = _signs(obs[0].cpu().numpy(), L, 1)
    for t in range(K):
        pr.orc.step()
        o_obs, o_rew, o_done = pr.orc.observe()
        np.testing.assert_allclose(obs[t].cpu().numpy(), o_obs, rtol=1e-6, atol=0)
        np.testing.assert_array_equal(rew[t].cpu().numpy(), o_rew)
        np.testing.assert_array_equal(done[t].cpu().numpy(), o_done)
        if o_done.any():
            changed += int((_signs(o_obs, L, 1)[o_done.astype(bool)] != first[o_done.astype(bool)]).sum())
    assert changed > 0, "some env changes side at an episode boundary"
    pr.check_state()
    pr.check_outputs()
    pr.close()


def test_drawn_side_agents_per_type():
    """Five agents of each type: all execution agents of an env share the
    episode's side."""
    n, T, P, L = 31, 9, 5, 10
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=60), mbogen.env_seeds(144, n), T)
    pr = Pair(n, st, n_agents=2 * P, cap=100, top_levels=L, exec_target=30, exec_dir=0, fill_cap=512)
    obs, _ = pr.check_outputs()
    s = _signs(obs, L, P)
    assert np.all(s == s[:, :1])
    for _ in range(T):
        pr.step()
        pr.check_outputs()
        pr.check_fills()
    pr.check_state()
    pr.close()


def test_drawn_side_checkpoint_resume():
    """The drawn side lives in the env state: a restored checkpoint carries it."""
    import torch
    n, T = 37, 9
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=60), mbogen.env_seeds(145, n), T)
    pr = Pair(n, st, cap=100, exec_target=50, exec_dir=0)
    for _ in range(4):
        pr.step()
    ck = torch.zeros(lob.lob_checkpoint_bytes(pr.env.h), dtype=torch.uint8, device="cuda")
    lob.lob_save(pr.env.h, ck)
    outs = []
    for _ in range(4):
        pr.env.step()
        outs.append(tuple(x.clone() for x in pr.env.observe()))
    lob.lob_load(pr.env.h, ck)
    for t in range(4):
        pr.step()
        o = pr.env.observe()
        assert all(torch.equal(x, y) for x, y in zip(o, outs[t]))
        pr.check_outputs()
    pr.check_state()
    pr.close()

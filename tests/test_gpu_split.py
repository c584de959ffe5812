"""The plain step with one warp per book side (lob_set_threads_per_env 64)
against the CPU oracle, every step, element by element: observations,
rewards, done flags and actions after every step; books (arrival stamps
included), counters, agents and env scalars at the end.  The two warps hand
over only the remainders of adds that may cross and merge stamps and totals
at every chunk and step, so these tests cover the hand-over (crossing
streams), the merge (agents on both sides, fills of both warps in one step)
and the classes the mode takes (K = 2, 4, 8), plus launches it leaves to one
warp per env."""
import numpy as np
import pytest

from harness import Pair
from paper_2511_02136_gb300 import lob, mbogen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    lob.build()


def _run(pr, T, actions=None):
    for t in range(T):
        pr.step(None if actions is None else actions[t])
        pr.check_outputs()
    pr.check_state()
    assert pr.env.sync() == 0
    pr.close()


@pytest.mark.parametrize("cap", [50, 100, 200])
def test_split_random_policy_each_class(cap):
    n, T = 203, 40
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=100), mbogen.env_seeds(300 + cap, n), T)
    _run(Pair(n, st, cap=cap, exec_target=500, threads_per_env=64), T)


def test_split_host_actions_buy_task_small_capacity():
    n, T = 97, 30
    rng = np.random.default_rng(301)
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=120), mbogen.env_seeds(301, n), T)
    pr = Pair(n, st, cap=40, exec_target=300, exec_dir=1, mm_lot=3, action_mode=lob.LOB_ACT_HOST,
              threads_per_env=64)
    _run(pr, T, rng.integers(0, 12, size=(T, n, 2)).astype(np.int32))


def test_split_no_agents_long_window():
    n, T = 64, 120
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=80), mbogen.env_seeds(302, n), T)
    _run(Pair(n, st, n_agents=0, cap=100, threads_per_env=64), T)


def test_split_stress_mix_many_crossings():
    """The heavy-tailed mix (30 % market orders, large sizes, delete bursts):
    most adds fail the no-cross bound and wait for the other warp's take."""
    n, T = 48, 12
    model = mbogen.MessageModel(mix_add=0.35, mix_partial=0.15, mix_delete=0.20, mix_market=0.30, size_model=1,
                                pareto_alpha=1.5, size_cap=10_000, p_burst=0.05, msgs_per_step=300)
    st = mbogen.generate(model, mbogen.env_seeds(303, n), T)
    _run(Pair(n, st, cap=200, top_levels=20, exec_target=2000, threads_per_env=64), T)


def test_split_rollout_matches_one_warp_per_env_bit_for_bit():
    """One lob_rollout of 60 steps, per-step outputs: 64 threads per env give
    the same bytes as 32, and the oracle's."""
    import torch
    n, T = 150, 60
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=100), mbogen.env_seeds(304, n), T)
    outs = []
    for tpe in (32, 64):
        pr = Pair(n, st, cap=100, exec_target=500, threads_per_env=tpe)
        D = pr.env.D
        obs = torch.zeros((T, n, 2, D), dtype=torch.float32, device="cuda")
        rew = torch.zeros((T, n, 2), dtype=torch.int64, device="cuda")
        done = torch.zeros((T, n), dtype=torch.uint8, device="cuda")
        lob.lob_rollout(pr.env.h, T, None, obs, rew, done)
        assert pr.env.sync() == 0
        outs.append((obs.cpu().numpy(), rew.cpu().numpy(), done.cpu().numpy(), pr.env.counters().cpu().numpy(),
                     pr.env.books()))
        if tpe == 64:
            for t in range(T):
                pr.orc.step()
                o_obs, o_rew, o_done = pr.orc.observe()
                np.testing.assert_allclose(outs[-1][0][t], o_obs, rtol=1e-6, atol=0)
                np.testing.assert_array_equal(outs[-1][1][t], o_rew)
                np.testing.assert_array_equal(outs[-1][2][t], o_done)
            pr.check_state()
        pr.close()
    a, b = outs
    for x, y in zip(a[:4], b[:4]):
        np.testing.assert_array_equal(x, y)
    for e in range(n):
        for k in ("n", "px", "qty", "id", "ts"):
            np.testing.assert_array_equal(a[4][e][k], b[4][e][k])


def test_split_uneven_capacities_mixed_with_one_warp_classes():
    """Capacities across classes: K = 2, 4, 8 run two warps per env, K = 16
    and 32 stay on one warp; one step launch covers both."""
    n, T = 120, 20
    caps = np.array([30, 50, 100, 150, 200, 256, 300, 500, 1000] * 14, np.int32)[:n]
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=150), mbogen.env_seeds(305, n), T)
    _run(Pair(n, st, caps=caps, cap=int(caps.max()), exec_target=500, threads_per_env=64), T)


def test_threads_per_env_validated():
    n, T = 8, 2
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=10), mbogen.env_seeds(306, n), T)
    pr = Pair(n, st, cap=100)
    for bad in (0, 16, 48, 96):
        with pytest.raises(lob.LobError):
            lob.lob_set_threads_per_env(pr.env.h, bad)
    lob.lob_set_threads_per_env(pr.env.h, 64)
    lob.lob_set_threads_per_env(pr.env.h, 32)
    pr.close()

"""Message tiles of 16 and 64 records (lob_set_tile_records) against the CPU
oracle, every step, element by element: observations, rewards and done
flags after every step; books (arrival stamps included), counters, agents
and env scalars at the end.  A step's messages are staged tile by tile, so
these cases put the chunk boundaries and the ragged last tile in other
places than the default 32: fixed counts that are not multiples of the tile,
Poisson counts (including empty steps and steps of several tiles), every
capacity class, host actions, no agents.  The plain step has its own
instances for 16 and 64; launches of the extended, traced and several-agent
kernels stage 32 whatever the setting, which the last cases check."""
import numpy as np
import pytest

from harness import Pair
from paper_2511_02136_gb300 import lob, mbogen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    lob.build()


def _run(pr, T, actions=None, fills=False):
    for t in range(T):
        pr.step(None if actions is None else actions[t])
        pr.check_outputs()
        if fills:
            pr.check_fills()
    pr.check_state()
    assert pr.env.sync() == 0
    pr.close()


@pytest.mark.parametrize("tile", [16, 64])
@pytest.mark.parametrize("cap", [20, 60, 100, 200, 500, 1000])
def test_tile_each_class_random_policy(tile, cap):
    n, T = (97, 20) if cap <= 200 else (40, 12)
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=100), mbogen.env_seeds(400 + cap, n), T)
    _run(Pair(n, st, cap=cap, exec_target=500, tile_records=tile), T)


@pytest.mark.parametrize("tile", [16, 64])
def test_tile_poisson_counts_with_empty_and_long_steps(tile):
    n, T = 128, 25
    model = mbogen.MessageModel(poisson=True, lam_lo=1.0, lam_hi=300.0)
    st = mbogen.generate(model, mbogen.env_seeds(410 + tile, n), T)
    counts = np.diff(st.offsets, axis=1)
    assert (counts == 0).any() and (counts > 2 * tile).any()
    _run(Pair(n, st, cap=100, exec_target=300, tile_records=tile), T)


@pytest.mark.parametrize("tile", [16, 64])
def test_tile_host_actions_buy_task(tile):
    n, T = 97, 20
    rng = np.random.default_rng(420 + tile)
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=130), mbogen.env_seeds(420 + tile, n), T)
    pr = Pair(n, st, cap=40, exec_target=300, exec_dir=1, mm_lot=3, action_mode=lob.LOB_ACT_HOST,
              tile_records=tile)
    _run(pr, T, rng.integers(0, 12, size=(T, n, 2)).astype(np.int32))


@pytest.mark.parametrize("tile", [16, 64])
def test_tile_no_agents_stress_mix(tile):
    n, T = 48, 10
    model = mbogen.MessageModel(mix_add=0.35, mix_partial=0.15, mix_delete=0.20, mix_market=0.30, size_model=1,
                                pareto_alpha=1.5, size_cap=10_000, p_burst=0.05, msgs_per_step=300)
    st = mbogen.generate(model, mbogen.env_seeds(430 + tile, n), T)
    _run(Pair(n, st, n_agents=0, cap=200, tile_records=tile), T)


def test_tile_setting_with_launches_that_stage_32():
    """Compact records, host-memory messages, several agents per type,
    episode mode and the fill log run the kernels that stage 32 records: with
    64 set they stay exact."""
    import torch
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=150), mbogen.env_seeds(440, 40), 12)
    _run(Pair(40, st, cap=100, exec_target=400, compact=True, tile_records=64), 12)
    _run(Pair(40, st, n_agents=6, cap=100, exec_target=40, tile_records=64), 12)
    _run(Pair(40, st, cap=100, exec_target=300, fill_cap=2048, tile_records=64), 12, fills=True)
    # host-memory messages
    n, T = 33, 5
    st2 = mbogen.generate(mbogen.MessageModel(msgs_per_step=90), mbogen.env_seeds(441, n), T)
    pr = Pair(n, st2, cap=100, exec_target=30, action_mode=lob.LOB_ACT_HOST, tile_records=64)
    rng = np.random.default_rng(441)
    D = pr.env.D
    for t in range(T):
        acts = rng.integers(0, 12, size=(n, 2)).astype(np.int32)
        lo, hi = st2.offsets[:, t], st2.offsets[:, t + 1]
        chunk = np.concatenate([st2.msgs[lo[e]:hi[e]] for e in range(n)])
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
    # episode mode: one rollout launch over three episodes
    n, T = 40, 5
    st3 = mbogen.generate(mbogen.MessageModel(msgs_per_step=110), mbogen.env_seeds(442, 1), 40)
    steps = np.random.default_rng(442).integers(0, 40 - T + 1, size=6)
    starts, levels = mbogen.start_books(442, st3.mids[0], steps, 12)
    K = 3 * T + 1
    pr = Pair(n, st3, cap=100, episode_len=T, exec_target=30, episodes=(starts, levels),
              seeds=mbogen.env_seeds(443, n), tile_records=64)
    obs = torch.zeros((K, n, 2, pr.env.D), dtype=torch.float32, device="cuda")
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
    pr.close()


def test_tile_sizes_give_the_same_rollout_bytes():
    """One lob_rollout of 50 steps over mixed capacities: 16, 32 and 64
    records per tile give identical outputs, books and counters."""
    import torch
    n, T = 120, 50
    caps = np.array([[50, 100, 200, 500][i % 4] for i in range(n)], np.int32)
    st = mbogen.generate(mbogen.MessageModel(poisson=True, lam_lo=5.0, lam_hi=200.0), mbogen.env_seeds(460, n), T)
    from harness import to_dev
    outs = []
    for tile in (16, 32, 64):
        env = lob.LobEnv(n, caps=caps, exec_target=300, action_mode=lob.LOB_ACT_RANDOM)
        if tile != 32:
            lob.lob_set_tile_records(env.h, tile)
        env.load_messages(to_dev(st.msgs), to_dev(st.offsets))
        env.reset(to_dev(st.seeds))
        D = env.D
        obs = torch.zeros((T, n, 2, D), dtype=torch.float32, device="cuda")
        rew = torch.zeros((T, n, 2), dtype=torch.int64, device="cuda")
        done = torch.zeros((T, n), dtype=torch.uint8, device="cuda")
        lob.lob_rollout(env.h, T, None, obs, rew, done)
        assert env.sync() == 0
        outs.append((obs.cpu().numpy(), rew.cpu().numpy(), done.cpu().numpy(), env.counters().cpu().numpy()))
        env.close()
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            np.testing.assert_array_equal(a, b)


def test_tile_records_refused_values():
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=10), mbogen.env_seeds(470, 4), 2)
    pr = Pair(4, st, cap=100)
    for bad in (0, 8, 31, 48, 128, -32):
        with pytest.raises(lob.LobError):
            lob.lob_set_tile_records(pr.env.h, bad)
    pr.close()

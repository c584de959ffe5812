"""The allocation-free step, lob_step_noalloc, checked against lob_step.

Some callers of this library cannot call cudaMalloc: a host program that
reserves all device memory up front through its own allocator or a fixed
budget, or a loop that must not take cudaMalloc's device-wide
synchronisation.  lob_step_noalloc serves them: the caller passes every
input and output buffer, and the scratch of the persistent step kernel (its
work-queue counter and env tables) lives in a static device array of the
library.  Here the buffers are caller-owned torch tensors, the call goes
through the C ABI, and two consecutive steps must equal the handle-based
lob_step on the same inputs (integers exactly, observations within 1e-6).
This file is collected last and depends on no other test.
"""
import numpy as np
import pytest

from paper_2511_02136_gb300 import lob, mbogen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [lob.LOB_ACT_RANDOM, lob.LOB_ACT_HOST])
def test_noalloc_step_matches_lob_step_on_two_calls(mode):
    import torch
    lob.build()
    n, T, cap = 300, 4, 100
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=70), mbogen.env_seeds(99, n), T)
    msgs_d = torch.from_numpy(st.msgs.view(np.uint8).copy()).cuda()
    off_d = torch.from_numpy(st.offsets).cuda()
    seeds_d = torch.from_numpy(st.seeds.view(np.int64).copy()).cuda()
    acts = torch.from_numpy(np.random.default_rng(3).integers(0, 12, size=(T, n, 2)).astype(np.int32)).cuda()

    env = lob.LobEnv(n, cap=cap, top_levels=10, episode_len=T, exec_target=50, action_mode=mode)
    env.load_messages(msgs_d, off_d)
    env.reset(seeds_d)

    cfg = lob.lob_config(n, 2, cap, 10, T, 1, 50, -1, mode, 0, 10_000, 0)
    D = lob.lob_obs_dim(cfg)
    books = torch.zeros(n * lob.noalloc_book_block_bytes(cap), dtype=torch.uint8, device="cuda")
    state = torch.zeros(n * 128, dtype=torch.uint8, device="cuda")
    counters = torch.zeros((n, lob.LOB_NCOUNTERS), dtype=torch.int64, device="cuda")
    obs = torch.zeros((n, 2, D), dtype=torch.float32, device="cuda")
    rew = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
    done = torch.zeros(n, dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")

    for t in range(2):
        a_t = acts[t].contiguous()
        env.step(a_t if mode == lob.LOB_ACT_HOST else None)
        h_obs, h_rew, h_done = env.observe()
        args = lob.lob_noalloc_args(
            cfg=lob.ctypes.pointer(cfg), d_books=books.data_ptr(), d_env_state=state.data_ptr(),
            d_counters=counters.data_ptr(), d_env_seeds=seeds_d.data_ptr(), d_msgs=msgs_d.data_ptr(),
            d_offsets=off_d.data_ptr(), stride=off_d.shape[1], k=t, t=t,
            d_actions=a_t.data_ptr() if mode == lob.LOB_ACT_HOST else None, d_obs=obs.data_ptr(),
            d_rewards=rew.data_ptr(), d_done=done.data_ptr(), d_status=status.data_ptr())
        lob.lob_step_noalloc(args)
        torch.cuda.synchronize()
        np.testing.assert_allclose(obs.cpu().numpy(), h_obs.cpu().numpy(), rtol=1e-6, atol=0)
        np.testing.assert_array_equal(rew.cpu().numpy(), h_rew.cpu().numpy())
        np.testing.assert_array_equal(done.cpu().numpy(), h_done.cpu().numpy())
        np.testing.assert_array_equal(counters.cpu().numpy(), env.counters().cpu().numpy())
    assert int(status.item()) == 0
    assert env.sync() == 0
    env.close()


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch
    lob.build()
    cfg = lob.lob_config(lob.LOB_NOALLOC_MAX_ENVS + 1, 2, 100, 10, 4, 1, 50, -1, 1, 0, 10_000, 0)
    dummy = torch.zeros(64, dtype=torch.int64, device="cuda")
    p = dummy.data_ptr()
    args = lob.lob_noalloc_args(cfg=lob.ctypes.pointer(cfg), d_books=p, d_env_state=p, d_counters=p,
                                d_env_seeds=p, d_msgs=p, d_offsets=p, stride=5, k=0, t=0, d_actions=None,
                                d_obs=None, d_rewards=None, d_done=None, d_status=p)
    with pytest.raises(lob.LobError) as ei:
        lob.lob_step_noalloc(args)
    assert ei.value.code == lob.LOB_ECAPACITY
    cfg.n_envs = 8
    cfg.cap_per_side = lob.LOB_MAX_CAP + 1
    with pytest.raises(lob.LobError) as ei:
        lob.lob_step_noalloc(args)
    assert ei.value.code == lob.LOB_ECAPACITY


def test_noalloc_rejects_extended_options():
    """The allocation-free step runs the plain kernel only: every extended
    option (reward variants, penalties, other market-maker spaces, the mid as
    value reference, a drawn task side) is refused, not ignored."""
    import torch
    lob.build()
    dummy = torch.zeros(64, dtype=torch.int64, device="cuda")
    p = dummy.data_ptr()
    for field, val in (("reward_mode", lob.LOB_REWARD_SPOONER), ("inv_penalty", 1), ("exec_penalty_milli", 10),
                       ("mm_space", lob.LOB_MM_DIRECTIONAL), ("pv_ref", lob.LOB_PV_MID), ("exec_dir", 0),
                       ("n_agents", 4)):
        cfg = lob.lob_config(8, 2, 100, 10, 4, 1, 50, -1, 1, 0, 10_000, 0)
        setattr(cfg, field, val)
        args = lob.lob_noalloc_args(cfg=lob.ctypes.pointer(cfg), d_books=p, d_env_state=p, d_counters=p,
                                    d_env_seeds=p, d_msgs=p, d_offsets=p, stride=5, k=0, t=0, d_actions=None,
                                    d_obs=None, d_rewards=None, d_done=None, d_status=p)
        with pytest.raises(lob.LobError) as ei:
            lob.lob_step_noalloc(args)
        assert ei.value.code == lob.LOB_EINVAL, field

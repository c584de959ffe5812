"""The allocation-free step, lob_step_noalloc, checked against lob_step and the oracle.

Some callers of this library cannot call cudaMalloc: a host program that
reserves all device memory up front through its own allocator or a fixed
budget, or a loop that must not take cudaMalloc's device-wide
synchronisation.  lob_step_noalloc serves them: the caller passes every
input and output buffer, and the scratch of the persistent step kernel (its
work-queue counter and env tables) lives in a static device array of the
library.  Here the buffers are caller-owned torch tensors filled with a byte
pattern (not zeros) before the first call, the calls go through the C ABI,
and every step of two whole episodes on the same buffers must equal both
the handle-based lob_step and the CPU oracle on the same inputs: integers
(books, counters, rewards, done) exactly, observations within 1e-6.
This file is collected last and depends on no other test.
"""
import numpy as np
import pytest

import oracle
from paper_2511_02136_gb300 import lob, mbogen

pytestmark = pytest.mark.gpu

PATTERN = 0xA5   # what the caller's buffers hold before the first call


def _book_from_block(block, n_bid, n_ask, S):
    """Decode one env's book block (int32 px[2][S], int32 qty[2][S], int64 id[2][S],
    int64 ts[2][S], each side in priority order) into the live orders per side."""
    b = np.frombuffer(block.tobytes(), dtype=np.uint8)
    px = b[:8 * S].view(np.int32).reshape(2, S)
    qty = b[8 * S:16 * S].view(np.int32).reshape(2, S)
    oid = b[16 * S:32 * S].view(np.int64).reshape(2, S)
    ts = b[32 * S:48 * S].view(np.int64).reshape(2, S)
    n = (n_bid, n_ask)
    return [(px[s, :n[s]], qty[s, :n[s]], oid[s, :n[s]], ts[s, :n[s]]) for s in range(2)]


@pytest.mark.parametrize("mode,cap,exec_dir,n", [
    (lob.LOB_ACT_RANDOM, 100, -1, 300),
    (lob.LOB_ACT_HOST, 50, 1, 200),
    (lob.LOB_ACT_RANDOM, 1000, 1, 48),
])
def test_noalloc_two_episodes_match_lob_step_and_oracle(mode, cap, exec_dir, n):
    import torch
    lob.build()
    T, M = 6, 70
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=M), mbogen.env_seeds(99 + cap, n), T)
    msgs_d = torch.from_numpy(st.msgs.view(np.uint8).copy()).cuda()
    off_d = torch.from_numpy(st.offsets).cuda()
    seeds_d = torch.from_numpy(st.seeds.view(np.int64).copy()).cuda()
    rng = np.random.default_rng(3)
    acts = rng.integers(0, 12, size=(2, T, n, 2)).astype(np.int32)

    env = lob.LobEnv(n, cap=cap, top_levels=10, episode_len=T, exec_target=50, exec_dir=exec_dir, action_mode=mode)
    orc = oracle.Oracle(n, cap=cap, top_levels=10, episode_len=T, exec_target=50, exec_dir=exec_dir,
                        action_mode=mode)

    cfg = lob.lob_config(n, 2, cap, 10, T, 1, 50, exec_dir, mode, 0, 10_000, 0)
    D = lob.lob_obs_dim(cfg)
    block = lob.noalloc_book_block_bytes(cap)
    S = block // 48   # slots per side: 48 * S is already a multiple of 256

    def patterned(shape, dtype):
        t = torch.empty(shape, dtype=dtype, device="cuda")
        t.view(torch.uint8).fill_(PATTERN)
        return t

    books = patterned(n * block, torch.uint8)
    state = patterned(n * 128, torch.uint8)
    counters = patterned((n, lob.LOB_NCOUNTERS), torch.int64)
    obs = patterned((n, 2, D), torch.float32)
    rew = patterned((n, 2), torch.int64)
    done = patterned(n, torch.uint8)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")

    for ep in range(2):   # the second episode starts from t = 0 on the first one's buffers
        env.load_messages(msgs_d, off_d)
        env.reset(seeds_d)
        orc.load_messages(st.msgs, st.offsets)
        orc.reset(st.seeds)
        for t in range(T):
            a_h = acts[ep, t] if mode == lob.LOB_ACT_HOST else None
            a_d = torch.from_numpy(acts[ep, t].copy()).cuda() if mode == lob.LOB_ACT_HOST else None
            env.step(a_d)
            orc.step(a_h)
            h_obs, h_rew, h_done = env.observe()
            args = lob.lob_noalloc_args(
                cfg=lob.ctypes.pointer(cfg), d_books=books.data_ptr(), d_env_state=state.data_ptr(),
                d_counters=counters.data_ptr(), d_env_seeds=seeds_d.data_ptr(), d_msgs=msgs_d.data_ptr(),
                d_offsets=off_d.data_ptr(), stride=off_d.shape[1], k=t, t=t,
                d_actions=a_d.data_ptr() if a_d is not None else None, d_obs=obs.data_ptr(),
                d_rewards=rew.data_ptr(), d_done=done.data_ptr(), d_status=status.data_ptr())
            lob.lob_step_noalloc(args)
            torch.cuda.synchronize()
            g_obs, g_rew, g_done = obs.cpu().numpy(), rew.cpu().numpy(), done.cpu().numpy()
            g_cnt = counters.cpu().numpy()
            # against the handle-based step
            np.testing.assert_allclose(g_obs, h_obs.cpu().numpy(), rtol=1e-6, atol=0)
            np.testing.assert_array_equal(g_rew, h_rew.cpu().numpy())
            np.testing.assert_array_equal(g_done, h_done.cpu().numpy())
            np.testing.assert_array_equal(g_cnt, env.counters().cpu().numpy())
            # against the oracle
            o_obs, o_rew, o_done = orc.observe()
            np.testing.assert_allclose(g_obs, o_obs, rtol=1e-6, atol=0)
            np.testing.assert_array_equal(g_rew, o_rew)
            np.testing.assert_array_equal(g_done, o_done)
            np.testing.assert_array_equal(g_cnt, orc.counters())
        assert int(done.sum().item()) == n   # the episode's last step is flagged
        # books after the episode, decoded from the caller's blocks
        raw = books.cpu().numpy().reshape(n, block)
        st_raw = state.cpu().numpy().reshape(n, 128)
        for e in range(0, n, max(1, n // 24)):
            nb, na = np.frombuffer(st_raw[e, 76:84].tobytes(), dtype=np.int32)
            got = _book_from_block(raw[e], int(nb), int(na), S)
            n2, px, qty, oid, ts = orc.book(e)
            assert [int(nb), int(na)] == n2.tolist(), f"env {e}: counts"
            for s in range(2):
                k = n2[s]
                np.testing.assert_array_equal(got[s][0], px[s][:k])
                np.testing.assert_array_equal(got[s][1], qty[s][:k])
                np.testing.assert_array_equal(got[s][2], oid[s][:k])
                np.testing.assert_array_equal(got[s][3], ts[s][:k])
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

"""Fused actor-critic forward on the GPU (BF16 tcgen05 and FP32) vs the FP64 oracle,
and the policy-in-the-loop rollout replayed into the CPU env oracle."""
import numpy as np
import pytest

from harness import Pair
from oracle import mlp
from paper_2511_02136_gb300 import lob, mbogen

pytestmark = pytest.mark.gpu

LOGIT_TOL_BF16 = 2e-2     # max |logit error| against FP64
AGREE_BF16 = 0.995        # greedy-action agreement against FP64
LOGIT_TOL_FP32 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    lob.build()


def _env_obs(n, T, seed, cap=100):
    """Observations of a real rollout (random policy) from the CPU oracle."""
    import oracle
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=100), mbogen.env_seeds(seed, n), T)
    o = oracle.Oracle(n, cap=cap, episode_len=T, exec_target=500, action_mode=1, n_threads=8)
    o.reset(st.seeds)
    o.load_messages(st.msgs, st.offsets)
    for _ in range(T):
        o.step()
    return o.observe()[0]


@pytest.mark.parametrize("prec,tol", [(lob.LOB_PREC_BF16, LOGIT_TOL_BF16), (lob.LOB_PREC_FP32, LOGIT_TOL_FP32)])
def test_forward_vs_fp64(prec, tol):
    import torch
    n = 4096 + 37                                    # full tiles plus a ragged tail
    obs = _env_obs(n, 20, 7)
    params = lob.init_policy_params(11, 2, 45)
    pol = lob.lob_policy_create(2, 45, params)
    obs_d = torch.from_numpy(obs).cuda()
    lg = torch.zeros((n, 2, 12), dtype=torch.float32, device="cuda")
    vl = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    ac = torch.zeros((n, 2), dtype=torch.int32, device="cuda")
    lob.lob_policy_forward(pol, obs_d, n, prec, lg, vl, ac)
    assert lob.lob_policy_sync(pol) == 0
    o_lg, o_vl, o_ac = mlp.forward(obs, params.astype(np.float64))
    err = np.abs(lg.cpu().numpy() - o_lg).max()
    verr = np.abs(vl.cpu().numpy() - o_vl).max()
    agree = np.mean(ac.cpu().numpy() == o_ac)
    print(f"precision {prec}: max logit err {err:.3e}, value err {verr:.3e}, greedy agreement {agree:.5f}")
    assert err <= tol and verr <= tol
    assert agree >= (AGREE_BF16 if prec == lob.LOB_PREC_BF16 else 0.999)
    # the action is the argmax of the returned logits (ties to the lowest index)
    assert np.array_equal(ac.cpu().numpy(), np.argmax(lg.cpu().numpy(), axis=2))
    lob.lob_policy_destroy(pol)


def _policy_rollout(n, T, cap, prec, graph=False, seed=3, A=2, exec_dir=-1):
    import torch
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=100), mbogen.env_seeds(seed, n), T)
    pr = Pair(n, st, n_agents=A, cap=cap, exec_target=512, action_mode=lob.LOB_ACT_HOST, n_threads=16,
              exec_dir=exec_dir)
    params = lob.init_policy_params(5, A, pr.env.D)
    pol = lob.lob_policy_create(A, pr.env.D, params)
    D = pr.env.D
    obs = torch.zeros((T, n, A, D), dtype=torch.float32, device="cuda")
    rew = torch.zeros((T, n, A), dtype=torch.int64, device="cuda")
    done = torch.zeros((T, n), dtype=torch.uint8, device="cuda")
    acts = torch.zeros((T, n, A), dtype=torch.int32, device="cuda")
    if graph:
        s = torch.cuda.Stream()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            lob.lob_rollout_policy(pr.env.h, pol, T, prec, obs, rew, done, acts, stream=s)
        g.replay()
        torch.cuda.synchronize()
    else:
        lob.lob_rollout_policy(pr.env.h, pol, T, prec, obs, rew, done, acts)
    assert pr.env.sync() == 0 and lob.lob_policy_sync(pol) == 0
    g_acts = acts.cpu().numpy()
    agree = []
    prev_obs = pr.orc.observe()[0]
    for t in range(T):
        _, _, o_ac = mlp.forward(prev_obs, params.astype(np.float64))
        agree.append(np.mean(o_ac == g_acts[t]))
        pr.orc.step(g_acts[t])                       # replay the GPU's actions
        o_obs, o_rew, o_done = pr.orc.observe()
        np.testing.assert_array_equal(obs[t].cpu().numpy(), o_obs)
        np.testing.assert_array_equal(rew[t].cpu().numpy(), o_rew)
        np.testing.assert_array_equal(done[t].cpu().numpy(), o_done)
        prev_obs = o_obs
    pr.check_state()
    lob.lob_policy_destroy(pol)
    pr.close()
    return float(np.mean(agree))


@pytest.mark.parametrize("prec", [lob.LOB_PREC_BF16, lob.LOB_PREC_FP32, lob.LOB_PREC_BF16_FUSED])
def test_policy_rollout_replayed_into_oracle(prec):
    agree = _policy_rollout(300, 12, 100, prec)
    print(f"greedy agreement with FP64 along the rollout: {agree:.5f}")
    assert agree >= (AGREE_BF16 if prec != lob.LOB_PREC_FP32 else 0.999)


def test_policy_rollout_ten_agents_per_type():
    """20 agents (10 per type, Table 1), each with its own network, BF16 in the loop."""
    agree = _policy_rollout(150, 8, 100, lob.LOB_PREC_BF16, A=20, seed=7)
    assert agree >= AGREE_BF16


def test_policy_rollout_under_cuda_graph():
    agree = _policy_rollout(200, 8, 100, lob.LOB_PREC_BF16, graph=True)
    assert agree >= AGREE_BF16


def test_policy_rollout_4096_envs_cap200_128_steps():
    """The policy-in-the-loop configuration: 4,096 envs x capacity 200 x 100
    msgs x 128 steps with the batched BF16 policy between step launches,
    replayed into the oracle."""
    agree = _policy_rollout(4096, 128, 200, lob.LOB_PREC_BF16)
    print(f"greedy agreement with FP64 along the 4096-env rollout: {agree:.5f}")
    assert agree >= AGREE_BF16


def test_fused_rollout_4096_envs_cap200_128_steps_one_launch():
    """The same configuration with the forward inside the step kernel: one
    launch for the whole rollout, replayed into the oracle step by step."""
    agree = _policy_rollout(4096, 128, 200, lob.LOB_PREC_BF16_FUSED)
    print(f"fused: greedy agreement with FP64 along the 4096-env rollout: {agree:.5f}")
    assert agree >= AGREE_BF16


def test_fused_rollout_buy_task_ragged_ctas():
    """A buy task and an env count that leaves the last CTA partly empty."""
    agree = _policy_rollout(157, 20, 100, lob.LOB_PREC_BF16_FUSED, seed=9, exec_dir=1)
    assert agree >= AGREE_BF16


def test_fused_rollout_matches_two_launch_bf16():
    """The fused forward and the batched BF16 forward take the same hidden-layer
    products; their greedy actions agree except on near-ties."""
    import torch
    n, T = 512, 16
    runs = []
    for prec in (lob.LOB_PREC_BF16, lob.LOB_PREC_BF16_FUSED):
        st = mbogen.generate(mbogen.MessageModel(msgs_per_step=100), mbogen.env_seeds(21, n), T)
        pr = Pair(n, st, cap=100, exec_target=512, action_mode=lob.LOB_ACT_HOST, n_threads=16)
        params = lob.init_policy_params(5, 2, pr.env.D)
        pol = lob.lob_policy_create(2, pr.env.D, params)
        acts = torch.zeros((T, n, 2), dtype=torch.int32, device="cuda")
        lob.lob_rollout_policy(pr.env.h, pol, T, prec, None, None, None, acts)
        assert pr.env.sync() == 0 and lob.lob_policy_sync(pol) == 0
        runs.append(acts[0].cpu().numpy())          # the first step: the same observation
        lob.lob_policy_destroy(pol)
        pr.close()
    agree = np.mean(runs[0] == runs[1])
    print(f"first-step action agreement fused vs two-launch: {agree:.5f}")
    assert agree >= 0.99


def test_fused_rollout_refuses_other_configurations():
    """Capacity classes without a fused kernel are refused, not run another way."""
    n, T = 64, 4
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=50), mbogen.env_seeds(22, n), T)
    pr = Pair(n, st, cap=1000, exec_target=100, action_mode=lob.LOB_ACT_HOST)
    pol = lob.lob_policy_create(2, pr.env.D, lob.init_policy_params(5, 2, pr.env.D))
    with pytest.raises(lob.LobError):
        lob.lob_rollout_policy(pr.env.h, pol, T, lob.LOB_PREC_BF16_FUSED, None, None, None, None)
    lob.lob_policy_destroy(pol)
    pr.close()
    # a drawn task side runs on the extended step, which has no fused form
    pr = Pair(n, st, cap=100, exec_target=100, exec_dir=0, action_mode=lob.LOB_ACT_HOST)
    pol = lob.lob_policy_create(2, pr.env.D, lob.init_policy_params(5, 2, pr.env.D))
    with pytest.raises(lob.LobError):
        lob.lob_rollout_policy(pr.env.h, pol, T, lob.LOB_PREC_BF16_FUSED, None, None, None, None)
    lob.lob_policy_destroy(pol)
    pr.close()


def test_fused_rollout_without_step_outputs_keeps_the_handle_state():
    """With no per-step output buffers the fused rollout writes each step's
    outputs into the handle's own buffers; the last step's observation,
    rewards and done flags, the books and the counters equal those of the
    same rollout with every output kept."""
    import torch
    n, T = 97, 10
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=100), mbogen.env_seeds(41, n), T)
    res = []
    for keep in (True, False):
        pr = Pair(n, st, cap=100, exec_target=300, action_mode=lob.LOB_ACT_HOST)
        pol = lob.lob_policy_create(2, pr.env.D, lob.init_policy_params(5, 2, pr.env.D))
        D = pr.env.D
        if keep:
            outs = (torch.zeros((T, n, 2, D), dtype=torch.float32, device="cuda"),
                    torch.zeros((T, n, 2), dtype=torch.int64, device="cuda"),
                    torch.zeros((T, n), dtype=torch.uint8, device="cuda"),
                    torch.zeros((T, n, 2), dtype=torch.int32, device="cuda"))
        else:
            outs = (None, None, None, None)
        lob.lob_rollout_policy(pr.env.h, pol, T, lob.LOB_PREC_BF16_FUSED, *outs)
        assert pr.env.sync() == 0 and lob.lob_policy_sync(pol) == 0
        obs, rew, done = pr.env.observe()
        res.append((obs.cpu().numpy(), rew.cpu().numpy(), done.cpu().numpy(), pr.env.counters().cpu().numpy(),
                    pr.env.books(), None if outs[0] is None else outs[0][T - 1].cpu().numpy()))
        lob.lob_policy_destroy(pol)
        pr.close()
    a, b = res
    for x, y in zip(a[:4], b[:4]):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(a[0], a[5])          # the handle's observation is the last step's
    for e in range(n):
        for k in ("n", "px", "qty", "id", "ts"):
            np.testing.assert_array_equal(a[4][e][k], b[4][e][k])

"""The IPPO update on the GPU (lob_ppo_update) against the FP64 oracle.

Both sides get the same seeded synthetic rollout: observations with the
magnitudes of the 10-level benchmark observations, uniform actions, rewards,
episode ends, behaviour log-probabilities and values near the FP64 network's
own, and each agent's minibatch order.  The GPU computes the forward and
backward passes with BF16 operands (FP32 accumulation), so its gradients are
compared at BF16 precision: relative L2 error <= 3e-2 and cosine >= 0.999 per
agent on the first minibatch (identical weights on both sides).  After the
epoch (4 Adam steps, each moving a weight by at most about lr) the weight
changes must agree: relative L2 error of the change <= 0.15, and no weight
more than 2 * 4 * lr away from the FP64 result.  The repacked BF16 weights of
the rollout's forward are checked by running it against the FP64 forward of
the updated FP32 weights."""
import numpy as np
import pytest

from oracle import mlp, ppo
from paper_2511_02136_gb300 import lob

pytestmark = pytest.mark.gpu


def _synthetic_batch(seed, T, n, A, L, params):
    rng = np.random.default_rng(seed)
    D = 4 * L + 5
    obs = np.zeros((T, n, A, D))
    lv = 4 * L
    obs[..., 0:lv:2] = rng.integers(-30, 30, size=(T, n, A, lv // 2))        # level price - anchor
    obs[..., 1:lv:2] = rng.integers(0, 400, size=(T, n, A, lv // 2))         # level size
    obs[..., lv] = rng.integers(-60, 60, size=(T, n, A))                    # inventory
    obs[..., lv + 1] = rng.integers(-200000, 200000, size=(T, n, A))        # cash
    obs[..., lv + 2] = rng.uniform(0, 1, size=(T, n, A))                    # time left
    obs[..., lv + 3] = rng.integers(0, 500, size=(T, n, A))                 # remaining target
    obs[..., lv + 4] = rng.integers(0, 10, size=(T, n, A))                  # own resting
    obs = obs.astype(np.float32)
    actions = rng.integers(0, 12, size=(T, n, A)).astype(np.int32)
    logits, values = np.zeros((T, n, A, 12)), np.zeros((T + 1, n, A))
    for t in range(T):
        lg, v, _ = mlp.forward(obs[t].astype(np.float64), params.astype(np.float64))
        logits[t], values[t] = lg, v
    values[T] = values[T - 1]
    lp = ppo.log_softmax(logits)
    logp_old = np.take_along_axis(lp, actions[..., None].astype(np.int64), -1)[..., 0]
    logp_old = (logp_old + rng.normal(0, 0.05, size=logp_old.shape)).astype(np.float32)
    values = (values + rng.normal(0, 0.2, size=values.shape)).astype(np.float32)
    rewards = rng.integers(-800, 800, size=(T, n, A)).astype(np.int64)
    done = np.zeros((T, n), np.uint8)
    done[T - 1] = 1
    done[T // 2, ::3] = 1
    perm = np.stack([rng.permutation(T * n) for _ in range(A)]).astype(np.int32)
    return dict(obs=obs, actions=actions, logp_old=logp_old, values=values, rewards=rewards, dones=done), perm


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("T,n", [(16, 64), (8, 100)])   # 1,024 samples (8 full tiles per minibatch); a ragged 800
def test_ppo_epoch_matches_fp64_oracle(T, n):
    import torch
    lob.build()
    A, L, nmb = 2, 10, 4
    D = 4 * L + 5
    params = lob.init_policy_params(11, A, D)
    # biases away from zero so that every term of the update is exercised
    rng = np.random.default_rng(12)
    P = params.shape[1]
    for a in range(A):
        params[a, H_D(D):H_D(D) + 128] = rng.normal(0, 0.1, 128)
    batch, perm = _synthetic_batch(13 + T, T, n, A, L, params)
    hp64 = ppo.PPOHyper()
    hp = lob.ppo_hparams(n_minibatches=nmb)
    pol = lob.lob_policy_create(A, D, params)
    grad_out = torch.zeros((nmb, A, P), dtype=torch.float32, device="cuda")
    lob.lob_ppo_update(pol, T, n, _dev(batch["obs"]), _dev(batch["actions"]), _dev(batch["logp_old"]),
                       _dev(batch["values"]), _dev(batch["rewards"]), _dev(batch["dones"]), _dev(perm), hp,
                       grad_out=grad_out)
    new = torch.zeros((A, P), dtype=torch.float32, device="cuda")
    lob.lob_policy_get_params(pol, new)
    torch.cuda.synchronize()
    assert lob.lob_policy_sync(pol) == 0
    g_gpu = grad_out.cpu().numpy().astype(np.float64)
    new_gpu = new.cpu().numpy().astype(np.float64)
    # the oracle: the same epoch in FP64, and its first minibatch's gradient
    p64 = params.astype(np.float64)
    new64, _, info = ppo.ppo_epoch(p64, D, batch, perm, nmb, hp64)
    mb = T * n // nmb
    for a in range(A):
        r = hp64.reward_scale * batch["rewards"][:, :, a].astype(np.float64)
        adv, ret = ppo.gae(r, batch["values"][:, :, a], np.broadcast_to(batch["dones"], (T, n)), hp64.gamma,
                           hp64.gae_lambda)
        idx = perm[a][:mb]
        o = batch["obs"][:, :, a, :].reshape(T * n, D)
        _, g64 = ppo.loss_and_grads(p64[a], D, o[idx], batch["actions"][:, :, a].reshape(-1)[idx],
                                    batch["logp_old"][:, :, a].reshape(-1)[idx], adv.reshape(-1)[idx],
                                    ret.reshape(-1)[idx], hp64)
        g = g_gpu[0, a]
        rel = np.linalg.norm(g - g64) / np.linalg.norm(g64)
        cos = float(g @ g64 / (np.linalg.norm(g) * np.linalg.norm(g64)))
        assert rel <= 3e-2 and cos >= 0.999, (a, rel, cos)
        d_gpu, d64 = new_gpu[a] - p64[a], new64[a] - p64[a]
        rel_d = np.linalg.norm(d_gpu - d64) / np.linalg.norm(d64)
        assert rel_d <= 0.15, (a, rel_d)
        assert np.max(np.abs(d_gpu - d64)) <= 2 * nmb * hp64.lr, (a, np.max(np.abs(d_gpu - d64)))
    # the rollout forward now runs the updated weights
    ob = _dev(batch["obs"][0])
    logits = torch.zeros((n, A, 12), dtype=torch.float32, device="cuda")
    lob.lob_policy_forward(pol, ob, n, lob.LOB_PREC_BF16, logits)
    lg64, _, _ = mlp.forward(batch["obs"][0].astype(np.float64), new_gpu)
    assert np.max(np.abs(logits.cpu().numpy() - lg64)) <= 2e-2
    lob.lob_policy_destroy(pol)


def H_D(D):
    """Offset of b1 in a parameter block."""
    return 128 * D


def test_ppo_update_rejects_bad_arguments():
    import torch
    lob.build()
    D = 45
    pol = lob.lob_policy_create(2, D, lob.init_policy_params(1, 2, D))
    x = torch.zeros(64, dtype=torch.float32, device="cuda")
    with pytest.raises(lob.LobError) as ei:   # 3 * 5 samples in 4 minibatches
        lob.lob_ppo_update(pol, 3, 5, x, x, x, x, x, x, x, lob.ppo_hparams(n_minibatches=4))
    assert ei.value.code == lob.LOB_EINVAL
    lob.lob_policy_destroy(pol)
    pol = lob.lob_policy_create(2, 85, lob.init_policy_params(1, 2, 85))   # 20 levels: beyond the update's tiles
    with pytest.raises(lob.LobError) as ei:
        lob.lob_ppo_update(pol, 4, 4, x, x, x, x, x, x, x, lob.ppo_hparams(n_minibatches=4))
    assert ei.value.code == lob.LOB_ECAPACITY
    lob.lob_policy_destroy(pol)


def test_ppo_epoch_on_the_fused_policy_rollout():
    """One IPPO epoch on a real policy-in-the-loop rollout of the 4,096-env,
    capacity-200, 128-step configuration (the fused BF16 rollout), against
    the FP64 oracle's epoch on the same data, at the BF16 tolerances above.
    The behaviour log-probabilities and values come from the batched BF16
    forward on the observations each action was taken on (the reset
    observation, then each step's output)."""
    import torch
    from paper_2511_02136_gb300 import mbogen
    lob.build()
    n, T, A, nmb = 4096, 128, 2, 4
    seeds = mbogen.env_seeds(31, n)
    st = mbogen.generate(mbogen.MessageModel(msgs_per_step=100), seeds, T)
    env = lob.LobEnv(n, cap=200, episode_len=T, exec_target=512, action_mode=lob.LOB_ACT_HOST)
    env.load_messages(_dev(st.msgs.view(np.uint8)), _dev(st.offsets))
    env.reset(_dev(seeds.view(np.int64)))
    D = env.D
    params = lob.init_policy_params(5, A, D)
    pol = lob.lob_policy_create(A, D, params)
    obs0, _, _ = env.observe()
    obs = torch.zeros((T, n, A, D), dtype=torch.float32, device="cuda")
    rew = torch.zeros((T, n, A), dtype=torch.int64, device="cuda")
    done = torch.zeros((T, n), dtype=torch.uint8, device="cuda")
    acts = torch.zeros((T, n, A), dtype=torch.int32, device="cuda")
    lob.lob_rollout_policy(env.h, pol, T, lob.LOB_PREC_BF16_FUSED, obs, rew, done, acts)
    assert env.sync() == 0 and lob.lob_policy_sync(pol) == 0
    # the observation each action was taken on, and the behaviour policy's outputs on it
    before = torch.cat([obs0.clone()[None], obs[:T - 1]], 0)
    logits = torch.zeros((T + 1, n, A, 12), dtype=torch.float32, device="cuda")
    values = torch.zeros((T + 1, n, A), dtype=torch.float32, device="cuda")
    for t in range(T + 1):
        src = before[t] if t < T else obs[T - 1]
        lob.lob_policy_forward(pol, src.contiguous(), n, lob.LOB_PREC_BF16, logits[t], values[t])
    assert lob.lob_policy_sync(pol) == 0
    logp_old = torch.log_softmax(logits[:T].double(), -1).gather(-1, acts.long()[..., None])[..., 0].float()
    perm = np.stack([np.random.default_rng(32 + a).permutation(T * n) for a in range(A)]).astype(np.int32)
    P = params.shape[1]
    grad_out = torch.zeros((nmb, A, P), dtype=torch.float32, device="cuda")
    hp = lob.ppo_hparams(n_minibatches=nmb)
    lob.lob_ppo_update(pol, T, n, before.contiguous(), acts, logp_old.contiguous(), values, rew, done, _dev(perm), hp,
                       grad_out=grad_out)
    new = torch.zeros((A, P), dtype=torch.float32, device="cuda")
    lob.lob_policy_get_params(pol, new)
    torch.cuda.synchronize()
    assert lob.lob_policy_sync(pol) == 0
    batch = dict(obs=before.cpu().numpy(), actions=acts.cpu().numpy(), logp_old=logp_old.cpu().numpy(),
                 values=values.cpu().numpy(), rewards=rew.cpu().numpy(), dones=done.cpu().numpy())
    assert batch["dones"][T - 1].all() and not batch["dones"][:T - 1].any()
    hp64 = ppo.PPOHyper()
    p64 = params.astype(np.float64)
    new64, _, _ = ppo.ppo_epoch(p64, D, batch, perm, nmb, hp64)
    g_gpu = grad_out.cpu().numpy().astype(np.float64)
    new_gpu = new.cpu().numpy().astype(np.float64)
    mb = T * n // nmb
    for a in range(A):
        r = hp64.reward_scale * batch["rewards"][:, :, a].astype(np.float64)
        adv, ret = ppo.gae(r, batch["values"][:, :, a], np.broadcast_to(batch["dones"], (T, n)), hp64.gamma,
                           hp64.gae_lambda)
        idx = perm[a][:mb]
        o = batch["obs"][:, :, a, :].reshape(T * n, D)
        _, g64 = ppo.loss_and_grads(p64[a], D, o[idx], batch["actions"][:, :, a].reshape(-1)[idx],
                                    batch["logp_old"][:, :, a].reshape(-1)[idx], adv.reshape(-1)[idx],
                                    ret.reshape(-1)[idx], hp64)
        g = g_gpu[0, a]
        rel = np.linalg.norm(g - g64) / np.linalg.norm(g64)
        cos = float(g @ g64 / (np.linalg.norm(g) * np.linalg.norm(g64)))
        print(f"agent {a}: gradient rel err {rel:.3e}, cosine {cos:.6f}")
        assert rel <= 3e-2 and cos >= 0.999, (a, rel, cos)
        d_gpu, d64 = new_gpu[a] - p64[a], new64[a] - p64[a]
        rel_d = np.linalg.norm(d_gpu - d64) / np.linalg.norm(d64)
        print(f"agent {a}: weight change rel err {rel_d:.3e}")
        assert rel_d <= 0.15, (a, rel_d)
        assert np.max(np.abs(d_gpu - d64)) <= 2 * nmb * hp64.lr, (a, np.max(np.abs(d_gpu - d64)))
    lob.lob_policy_destroy(pol)
    env.close()

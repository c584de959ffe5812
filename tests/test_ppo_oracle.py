"""Pins of the FP64 IPPO-update oracle (oracle/ppo.py): GAE by hand and in
its lambda = 1 closed form, the loss gradient against central finite
differences of the loss itself, a hand-computed two-sample gradient, Adam's
first step in closed form, the clipped branch and the global-norm clip."""
import numpy as np
import pytest

from oracle import mlp, ppo

H, NOUT = mlp.H, mlp.NOUT


def _zero_block(D):
    return np.zeros(H * D + H + H * H + H + NOUT * H + NOUT)


def _views(block, D):
    o, out = 0, {}
    for name, shape in (("W1", (H, D)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (NOUT, H)),
                        ("b3", (NOUT,))):
        size = int(np.prod(shape))
        out[name] = block[o:o + size].reshape(shape)
        o += size
    return out


def test_gae_three_steps_by_hand():
    """gamma = lambda = 0.5, rewards 1, 2, 3, values 0.5, 1, 1.5 and bootstrap
    2, the episode ending at the last step:
      t=2: delta = 3 - 1.5 = 1.5 (no bootstrap), A = 1.5
      t=1: delta = 2 + 0.5 * 1.5 - 1 = 1.75, A = 1.75 + 0.25 * 1.5 = 2.125
      t=0: delta = 1 + 0.5 * 1 - 0.5 = 1, A = 1 + 0.25 * 2.125 = 1.53125."""
    adv, ret = ppo.gae([1.0, 2.0, 3.0], [0.5, 1.0, 1.5, 2.0], [0, 0, 1], 0.5, 0.5)
    assert adv.tolist() == [1.53125, 2.125, 1.5]
    assert ret.tolist() == [2.03125, 3.125, 3.0]


def test_gae_lambda_one_is_discounted_return():
    rng = np.random.default_rng(0)
    T, g = 7, 0.9
    r, v = rng.normal(size=T), rng.normal(size=T + 1)
    adv, _ = ppo.gae(r, v, np.zeros(T), g, 1.0)
    for t in range(T):
        want = sum(g ** k * r[t + k] for k in range(T - t)) + g ** (T - t) * v[T] - v[t]
        assert adv[t] == pytest.approx(want, rel=1e-12, abs=1e-12)


def _random_case(seed, B=6, D=13):
    rng = np.random.default_rng(seed)
    blk = rng.normal(size=len(_zero_block(D))) * 0.3
    obs = rng.normal(size=(B, D)) * 5.0
    acts = rng.integers(0, 12, size=B)
    lpo = np.log(rng.uniform(0.02, 0.3, size=B))
    adv = rng.normal(size=B)
    ret = rng.normal(size=B)
    return blk, obs, acts, lpo, adv, ret


@pytest.mark.parametrize("seed", range(3))
def test_gradient_matches_central_differences(seed):
    """Every parameter group's gradient against (L(w + h) - L(w - h)) / 2h."""
    D = 13   # L = 2 levels: 4 * 2 + 5 features
    hp = ppo.PPOHyper(clip_eps=0.2, ent_coef=0.05, vf_coef=0.7)
    blk, obs, acts, lpo, adv, ret = _random_case(seed, D=D)
    _, g = ppo.loss_and_grads(blk, D, obs, acts, lpo, adv, ret, hp)
    rng = np.random.default_rng(100 + seed)
    sizes = [H * D, H, H * H, H, NOUT * H, NOUT]
    starts = np.cumsum([0] + sizes[:-1])
    idx = np.concatenate([s + rng.choice(n, size=min(n, 12), replace=False) for s, n in zip(starts, sizes)])
    h = 1e-5   # the cash feature's 1e-6 input scale makes some gradients ~1e-7: roundoff sets the floor
    for i in idx:
        wp, wm = blk.copy(), blk.copy()
        wp[i] += h
        wm[i] -= h
        fd = (ppo.loss_only(wp, D, obs, acts, lpo, adv, ret, hp) - ppo.loss_only(wm, D, obs, acts, lpo, adv, ret, hp)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=2e-5, abs=2e-10), int(i)


def test_two_sample_gradient_by_hand():
    """Zero network except b2[5] = atanh(1/2) (so h2[5] = 1/2) and W3[12][5] = 2
    (value path only): logits are 0, p = 1/12, V = 1 for both samples.  With
    rho = 1 (logp_old = -log 12), advantages (1, -1) -> normalised (1, -1),
    returns (3, 0), c_v = 1/2, B = 2:
      dz_b = -A'_b (e_{a_b} - 1/12) / 2 (the entropy term is 0 at the uniform p)
      dV_b = c_v (V - R_b) / 2 = (-1/2, 1/4)
      db3[a_0 = 0] = (-(11/12) + (1/12) * (-1)) / 2 ... = -1/2, db3[3] = +1/2
      db3[12] = -1/4, dW3[12][5] = (1/2)(-1/4) = -1/8,
      db2[5] = sum_b dV_b * W3[12][5] * (1 - 1/4) = -1/4 * 2 * 3/4 = -3/8."""
    D = 13
    blk = _zero_block(D)
    v = _views(blk, D)
    v["b2"][5] = np.arctanh(0.5)
    v["W3"][12, 5] = 2.0
    hp = ppo.PPOHyper(vf_coef=0.5, ent_coef=0.01)
    obs = np.zeros((2, D))
    acts = np.array([0, 3])
    lpo = np.full(2, -np.log(12.0))
    loss, g = ppo.loss_and_grads(blk, D, obs, acts, lpo, np.array([1.0, -1.0]), np.array([3.0, 0.0]), hp)
    gv = _views(g, D)
    s = 1.0 / (1.0 + 1e-8)   # the normalisation's 1e-8
    assert gv["b3"][0] == pytest.approx(-0.5 * s, rel=1e-12)
    assert gv["b3"][3] == pytest.approx(0.5 * s, rel=1e-12)
    for k in (1, 2, 4, 5, 6, 7, 8, 9, 10, 11):
        assert gv["b3"][k] == pytest.approx(0.0, abs=1e-15)
    assert gv["b3"][12] == pytest.approx(-0.25, rel=1e-12)
    assert gv["W3"][12, 5] == pytest.approx(-0.125, rel=1e-12)
    assert gv["W3"][0, 5] == pytest.approx(0.5 * -0.5 * s, rel=1e-12)
    assert gv["b2"][5] == pytest.approx(-0.375, rel=1e-12)
    assert np.all(gv["W1"] == 0) and np.all(gv["b1"] == 0) and np.all(gv["W2"] == 0)
    # loss: policy term -mean(A') = 0, value 0.5 * 0.5 * ((1-3)^2 + 1^2) / 2, entropy log 12
    assert loss == pytest.approx(0.5 * 0.5 * 5 / 2 - 0.01 * np.log(12.0), rel=1e-12)


def test_clipped_branch_carries_no_policy_gradient():
    """rho = e for both samples (logp_old one nat below the uniform log 1/12);
    advantages (2, 1) normalise to (1, -1).  Sample 0 (A' = 1): the clipped
    term 1.2 is below rho A' = e, so min picks the constant and that sample
    sends no policy gradient.  Sample 1 (A' = -1): rho A' = -e is below
    -1.2, so min picks the unclipped term: dz = -A' rho (e_a - 1/12) / 2 =
    e (e_2 - 1/12) / 2.  Hence db3[k] = -e/24 for every k != 2 (including
    sample 0's action 1) and db3[2] = 11 e / 24."""
    D = 13
    blk = _zero_block(D)
    hp = ppo.PPOHyper(clip_eps=0.2, ent_coef=0.0, vf_coef=0.0)
    obs = np.zeros((2, D))
    acts = np.array([1, 2])
    lpo = np.full(2, -np.log(12.0) - 1.0)
    _, g = ppo.loss_and_grads(blk, D, obs, acts, lpo, np.array([2.0, 1.0]), np.zeros(2), hp)
    gv = _views(g, D)
    s = 0.5 / (0.5 + 1e-8)   # std 1/2 plus the normalisation's 1e-8
    for k in range(12):
        want = 11 * np.e / 24 if k == 2 else -np.e / 24
        assert gv["b3"][k] == pytest.approx(want * s, rel=1e-12), k
    assert gv["b3"][12] == 0.0


def test_adam_first_step_closed_form():
    hp = ppo.PPOHyper(lr=1e-3, adam_eps=1e-5)
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4e-6, 0.0])
    w1, m, v = ppo.adam(w, g, np.zeros(3), np.zeros(3), 1, hp)
    np.testing.assert_allclose(w1, w - 1e-3 * g / (np.abs(g) + 1e-5), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)


def test_global_norm_clip():
    g = np.array([3.0, 4.0])
    c, n = ppo.clip_global_norm(g, 0.5)
    assert n == 5.0
    np.testing.assert_allclose(c, [0.3, 0.4], rtol=1e-15)
    c2, _ = ppo.clip_global_norm(np.array([0.1, 0.2]), 0.5)
    assert c2.tolist() == [0.1, 0.2]

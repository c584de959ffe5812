"""Pins of the FP64 actor-critic oracle (oracle/mlp.py) and of the reset observation."""
import numpy as np

import oracle
from oracle import mlp

H = mlp.H


def _zero_block(D):
    return np.zeros(H * D + H + H * H + H + mlp.NOUT * H + mlp.NOUT)


def _views(block, D):
    o = 0
    out = {}
    for name, size in (("W1", H * D), ("b1", H), ("W2", H * H), ("b2", H), ("W3", mlp.NOUT * H), ("b3", mlp.NOUT)):
        out[name] = block[o:o + size]
        o += size
    return out


def test_input_scale_layout():
    s = mlp.input_scale(10)
    assert len(s) == 45
    assert np.all(s[0:40:2] == 0.1) and np.all(s[1:40:2] == 1e-3)
    assert s[40:].tolist() == [1e-2, 1e-6, 1.0, 1e-2, 1e-2]


def test_hand_built_network():
    """A network that routes feature 0 through one unit per layer:
    y[3] = 2 * tanh(0.5 * tanh(3 * 0.1 * obs0) + 0.25) - 1, y[12] = b3[12]."""
    D = 45
    blk = _zero_block(D)
    v = _views(blk, D)
    v["W1"].reshape(H, D)[7, 0] = 3.0
    v["W2"].reshape(H, H)[2, 7] = 0.5
    v["b2"][2] = 0.25
    v["W3"].reshape(mlp.NOUT, H)[3, 2] = 2.0
    v["b3"][3] = -1.0
    v["b3"][12] = 0.125
    obs = np.zeros((2, 1, D))
    obs[0, 0, 0] = 4.0
    obs[1, 0, 0] = -7.0
    logits, values, actions = mlp.forward(obs, blk[None, :])
    for r, x in enumerate((4.0, -7.0)):
        want = 2 * np.tanh(0.5 * np.tanh(3 * 0.1 * x) + 0.25) - 1
        assert abs(logits[r, 0, 3] - want) < 1e-15
        assert np.all(np.delete(logits[r, 0], 3) == 0.0)
        assert values[r, 0] == 0.125
    # logit 3 is positive for obs0 = 4 and negative for obs0 = -7
    assert actions[0, 0] == 3 and actions[1, 0] == 0


def test_odd_symmetry_without_biases():
    rng = np.random.default_rng(0)
    D = 45
    blk = rng.standard_normal(len(_zero_block(D)))
    v = _views(blk, D)
    for b in ("b1", "b2", "b3"):
        v[b][:] = 0.0
    obs = rng.standard_normal((16, 1, D)) * 50
    l1, v1, _ = mlp.forward(obs, blk[None, :])
    l2, v2, _ = mlp.forward(-obs, blk[None, :])
    np.testing.assert_allclose(l1, -l2, rtol=0, atol=1e-12)
    np.testing.assert_allclose(v1, -v2, rtol=0, atol=1e-12)


def test_argmax_ties_go_to_lowest_index():
    D = 45
    blk = _zero_block(D)
    v = _views(blk, D)
    v["b3"][[2, 5, 9]] = 1.0
    _, _, a = mlp.forward(np.zeros((1, 1, D)), blk[None, :])
    assert a[0, 0] == 2


def test_agents_use_their_own_weights():
    D = 45
    b0, b1 = _zero_block(D), _zero_block(D)
    _views(b0, D)["b3"][4] = 1.0
    _views(b1, D)["b3"][8] = 1.0
    _, _, a = mlp.forward(np.zeros((3, 2, D)), np.stack([b0, b1]))
    assert a[:, 0].tolist() == [4, 4, 4] and a[:, 1].tolist() == [8, 8, 8]


def test_reset_observation():
    o = oracle.Oracle(3, cap=10, top_levels=10, episode_len=50, exec_target=123)
    o.reset(np.arange(3, dtype=np.uint64))
    obs, rew, done = o.observe()
    want = np.zeros((2, 45), np.float32)
    want[:, 42] = 1.0
    want[0, 43] = 123.0
    for e in range(3):
        np.testing.assert_array_equal(obs[e], want)

"""FP64 oracle of the IPPO update -- TEST INFRASTRUCTURE ONLY.

JaxMARL-HFT trains its agents with independent PPO (Sec. 4.2): every agent
keeps its own actor-critic network and is updated from its own rollout data
only; the paper gives no further algorithmic detail, so the update here is
the textbook one, written out from its published definitions:

* generalised advantage estimation (Schulman et al. 2016, "High-dimensional
  continuous control using generalized advantage estimation", Eqs. 11-16):
      delta_t = r_t + gamma (1 - d_t) V_{t+1} - V_t
      A_t     = delta_t + gamma lambda (1 - d_t) A_{t+1},   A_T = 0
      R_t     = A_t + V_t                                  (value target)
  where d_t = 1 when step t ended the episode and V_T is the value of the
  observation after the last step;
* the clipped surrogate objective with a value and an entropy term
  (Schulman et al. 2017, "Proximal policy optimization algorithms", Eqs. 7
  and 9), minimised as the minibatch mean of
      l = -min(rho A', clip(rho, 1 - eps, 1 + eps) A')
          + c_v * 0.5 (V - R)^2 - c_e * S
  with rho = exp(log pi(a|s) - log pi_old(a|s)), S the policy's entropy and
  A' the advantage normalised over the minibatch ((A - mean) / (std + 1e-8),
  population std);
* the gradient of that loss through the network of oracle/mlp.py
  (x = obs * s, h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2),
  y = W3 h2 + b3, logits y[:12], value y[12]), by the chain rule written
  out per layer;
* clipping of the whole gradient (all six tensors) to a global L2 norm;
* Adam (Kingma & Ba 2015, Algorithm 1) with bias correction.

Rewards enter scaled: r = reward_scale * (int64 reward).  The derivative of
min(u, c) where both are equal is taken from u (the unclipped term), and the
derivative of clip at its bounds is 0.

Pins (tests/test_ppo_oracle.py): GAE against a hand-computed 3-step example
and against the plain discounted sum when lambda = 1; the loss gradient
against central finite differences of the loss itself; a hand-computed
two-sample gradient of a network with one active path; Adam's first step
against its closed form; the clipped-ratio branch selection.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import mlp

H = mlp.H
NOUT = mlp.NOUT
NA = 12


@dataclass
class PPOHyper:
    gamma: float = 0.99
    gae_lambda: float = 0.95
    clip_eps: float = 0.2
    vf_coef: float = 0.5
    ent_coef: float = 0.01
    lr: float = 2.5e-4
    beta1: float = 0.9
    beta2: float = 0.999
    adam_eps: float = 1e-5
    max_grad_norm: float = 0.5
    reward_scale: float = 1e-2


def gae(rewards, values, dones, gamma, lam):
    """rewards, dones [T, ...]; values [T + 1, ...] (the last row bootstraps).
    Returns (advantages, value targets), both [T, ...]."""
    r = np.asarray(rewards, np.float64)
    v = np.asarray(values, np.float64)
    d = np.asarray(dones, np.float64)
    T = r.shape[0]
    adv = np.zeros_like(r)
    nxt = np.zeros_like(r[0])
    for t in range(T - 1, -1, -1):
        live = 1.0 - d[t]
        delta = r[t] + gamma * live * v[t + 1] - v[t]
        nxt = delta + gamma * lam * live * nxt
        adv[t] = nxt
    return adv, adv + v[:T]


def log_softmax(z):
    m = z.max(axis=-1, keepdims=True)
    e = np.exp(z - m)
    return z - m - np.log(e.sum(axis=-1, keepdims=True))


def loss_and_grads(block, D, obs, actions, logp_old, adv, ret, hp: PPOHyper):
    """One agent, one minibatch.  obs [B, D] (unscaled), actions [B],
    logp_old [B], adv [B] (not yet normalised), ret [B].  Returns (loss,
    grads) with grads a flat block laid out like the parameters."""
    W1, b1, W2, b2, W3, b3 = mlp.unpack(block, D)
    L = (D - 5) // 4
    x = np.asarray(obs, np.float64) * mlp.input_scale(L)
    B = x.shape[0]
    a = np.asarray(actions, np.int64)
    # forward
    h1 = np.tanh(x @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    y = h2 @ W3.T + b3
    z, V = y[:, :NA], y[:, NA]
    lp = log_softmax(z)
    p = np.exp(lp)
    logp = lp[np.arange(B), a]
    ent = -(p * lp).sum(axis=1)
    A = np.asarray(adv, np.float64)
    An = (A - A.mean()) / (A.std() + 1e-8)
    rho = np.exp(logp - np.asarray(logp_old, np.float64))
    rc = np.clip(rho, 1.0 - hp.clip_eps, 1.0 + hp.clip_eps)
    un, cl = rho * An, rc * An
    R = np.asarray(ret, np.float64)
    per = -np.minimum(un, cl) + hp.vf_coef * 0.5 * (V - R) ** 2 - hp.ent_coef * ent
    loss = per.mean()
    # d loss / d y, per sample (the mean divides by B)
    g_rho = np.where(un <= cl, -An, 0.0)                     # through the chosen branch
    onehot = np.zeros_like(z)
    onehot[np.arange(B), a] = 1.0
    dz = (g_rho * rho)[:, None] * (onehot - p)               # d rho / d z = rho (e_a - p)
    dz += hp.ent_coef * p * (lp + ent[:, None])              # - c_e dS/dz, dS/dz = -p (log p + S)
    dV = hp.vf_coef * (V - R)
    dy = np.concatenate([dz, dV[:, None]], axis=1) / B
    # backward
    dW3 = dy.T @ h2
    db3 = dy.sum(axis=0)
    du2 = (dy @ W3) * (1.0 - h2 * h2)
    dW2 = du2.T @ h1
    db2 = du2.sum(axis=0)
    du1 = (du2 @ W2) * (1.0 - h1 * h1)
    dW1 = du1.T @ x
    db1 = du1.sum(axis=0)
    grads = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return loss, grads


def loss_only(block, D, obs, actions, logp_old, adv, ret, hp: PPOHyper):
    return loss_and_grads(block, D, obs, actions, logp_old, adv, ret, hp)[0]


def clip_global_norm(g, max_norm):
    n = np.sqrt(np.sum(np.asarray(g, np.float64) ** 2))
    return g * min(1.0, max_norm / n) if n > 0 else g, n


def adam(block, g, m, v, t, hp: PPOHyper):
    """Adam step t (1-based): returns (block', m', v')."""
    m = hp.beta1 * m + (1.0 - hp.beta1) * g
    v = hp.beta2 * v + (1.0 - hp.beta2) * g * g
    mh = m / (1.0 - hp.beta1 ** t)
    vh = v / (1.0 - hp.beta2 ** t)
    return block - hp.lr * mh / (np.sqrt(vh) + hp.adam_eps), m, v


def ppo_epoch(params, D, batch, perm, n_minibatches, hp: PPOHyper, adam_state=None):
    """One PPO epoch for every agent (separate networks, separate data).

    params float[A, P]; batch: dict with obs [T, n, A, D], actions [T, n, A],
    logp_old [T, n, A], values [T + 1, n, A], rewards [T, n, A] (int64),
    dones [T, n]; perm int[A, T * n]: each agent's sample order (sample
    index t * n + e), cut into n_minibatches equal consecutive parts.
    Returns (params', adam_state', per-minibatch info)."""
    params = np.array(params, np.float64)
    A = params.shape[0]
    obs = np.asarray(batch["obs"], np.float64)
    T, n = obs.shape[0], obs.shape[1]
    if adam_state is None:
        adam_state = (np.zeros_like(params), np.zeros_like(params), 0)
    m, v, step = adam_state
    m, v = m.copy(), v.copy()
    info = []
    for a in range(A):
        r = hp.reward_scale * np.asarray(batch["rewards"], np.float64)[:, :, a]
        d = np.broadcast_to(np.asarray(batch["dones"], np.float64), (T, n))
        adv, ret = gae(r, np.asarray(batch["values"], np.float64)[:, :, a], d, hp.gamma, hp.gae_lambda)
        o = obs[:, :, a, :].reshape(T * n, D)
        act = np.asarray(batch["actions"])[:, :, a].reshape(T * n)
        lpo = np.asarray(batch["logp_old"], np.float64)[:, :, a].reshape(T * n)
        adv, ret = adv.reshape(T * n), ret.reshape(T * n)
        mb = (T * n) // n_minibatches
        s = step
        for k in range(n_minibatches):
            idx = np.asarray(perm[a][k * mb:(k + 1) * mb])
            loss, g = loss_and_grads(params[a], D, o[idx], act[idx], lpo[idx], adv[idx], ret[idx], hp)
            g, gn = clip_global_norm(g, hp.max_grad_norm)
            s += 1
            params[a], m[a], v[a] = adam(params[a], g, m[a], v[a], s, hp)
            info.append({"agent": a, "minibatch": k, "loss": loss, "grad_norm": gn})
    return params, (m, v, step + n_minibatches), info

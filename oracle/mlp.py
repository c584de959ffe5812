"""FP64 oracle of the per-agent actor-critic forward -- TEST INFRASTRUCTURE ONLY.

The IPPO networks of JaxMARL-HFT Sec. 4.2 keep separate weights per agent.
Here each agent's network is the plain definition, evaluated in float64:

    x  = obs * s                    (fixed per-feature input scale)
    h1 = tanh(W1 x + b1)            W1: 128 x D
    h2 = tanh(W2 h1 + b2)           W2: 128 x 128
    y  = W3 h2 + b3                 W3: 13 x 128; y[:12] logits, y[12] value
    action = argmax(y[:12])         ties to the lowest index

Parameters per agent are one flat block: W1, b1, W2, b2, W3, b3 (row-major,
W[out][in]).  The input scale is: level prices 1/10, level sizes 1/1000,
inventory 1/100, cash 1e-6, time left 1, remaining target 1/100, own resting
quantity 1/100.
"""
import numpy as np

H = 128
NOUT = 13


def input_scale(L):
    s = np.empty(4 * L + 5, np.float64)
    s[0:4 * L:2] = 0.1
    s[1:4 * L:2] = 1e-3
    s[4 * L:] = [1e-2, 1e-6, 1.0, 1e-2, 1e-2]
    return s


def unpack(block, D):
    b = np.asarray(block, np.float64)
    o = 0
    W1 = b[o:o + H * D].reshape(H, D); o += H * D
    b1 = b[o:o + H]; o += H
    W2 = b[o:o + H * H].reshape(H, H); o += H * H
    b2 = b[o:o + H]; o += H
    W3 = b[o:o + NOUT * H].reshape(NOUT, H); o += NOUT * H
    b3 = b[o:o + NOUT]; o += NOUT
    assert o == len(b)
    return W1, b1, W2, b2, W3, b3


def forward(obs, params):
    """obs float[n, A, D]; params float[A, P] -> (logits [n, A, 12], values [n, A], actions [n, A])."""
    obs = np.asarray(obs, np.float64)
    n, A, D = obs.shape
    L = (D - 5) // 4
    s = input_scale(L)
    logits = np.zeros((n, A, 12))
    values = np.zeros((n, A))
    for a in range(A):
        W1, b1, W2, b2, W3, b3 = unpack(params[a], D)
        x = obs[:, a, :] * s
        h1 = np.tanh(x @ W1.T + b1)
        h2 = np.tanh(h1 @ W2.T + b2)
        y = h2 @ W3.T + b3
        logits[:, a] = y[:, :12]
        values[:, a] = y[:, 12]
    return logits, values, np.argmax(logits, axis=2).astype(np.int32)

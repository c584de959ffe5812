import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def make_msgs(rows, ts0=0):
    """Message array from (type, side, px, qty, oid) rows."""
    from paper_2511_02136_gb300.mbogen import MSG_DTYPE
    out = np.zeros(len(rows), dtype=MSG_DTYPE)
    for i, (t, s, p, q, o) in enumerate(rows):
        out[i] = (ts0 + i, o, p, q, t, s, 0)
    return out


def single_env_stream(steps_rows):
    """One env, one list of message rows per step -> (msgs, offsets[1, T+1])."""
    from paper_2511_02136_gb300.mbogen import MSG_DTYPE
    chunks = [make_msgs(r) for r in steps_rows]
    msgs = np.concatenate(chunks) if chunks else np.zeros(0, MSG_DTYPE)
    off = np.zeros((1, len(steps_rows) + 1), np.int64)
    off[0, 1:] = np.cumsum([len(r) for r in steps_rows])
    return msgs, off

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU oracle runs")


def rng(seed=0):
    import numpy as np
    return np.random.default_rng(seed)


def random_rotation(r):
    import numpy as np
    q, _ = np.linalg.qr(r.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


@pytest.fixture
def gen():
    return rng(1234)


def oracle_trajectory(sc):
    """The CPU oracle's states (z, zd) at every step of the scene's trajectory, and its Scene.

    Runs the oracle over the whole trajectory.  The states are kept in tests/_oracle_cache (not part of the
    repository), keyed by a hash of the scene and of the oracle's sources, so that a second test run with
    the same scene and oracle reuses them."""
    import hashlib
    import numpy as np
    from oracle import ipc as orc
    h = hashlib.sha256()
    for name in ("ipc_oracle.cpp", "ipc.py"):
        with open(os.path.join(ROOT, "oracle", name), "rb") as f:
            h.update(f.read())

    def feed(v):
        if isinstance(v, dict):
            for k in sorted(v):
                h.update(k.encode())
                feed(v[k])
        elif isinstance(v, (list, tuple)):
            for u in v:
                feed(u)
        elif isinstance(v, np.ndarray):
            h.update(str(v.dtype).encode() + str(v.shape).encode())
            h.update(np.ascontiguousarray(v).tobytes())
        else:
            h.update(repr(v).encode())

    feed(sc)
    cache_dir = os.path.join(ROOT, "tests", "_oracle_cache")
    path = os.path.join(cache_dir, f"{sc['name']}_{h.hexdigest()[:20]}.npz")
    S = orc.Scene(sc)
    if os.path.exists(path):
        d = np.load(path)
        return S, list(zip(d["z"], d["zd"]))
    o = orc.Oracle(sc)
    states = [(o.z.copy(), o.zd.copy())]
    for _ in range(sc["kin_T"].shape[0] - 1):
        o.step()
        states.append((o.z.copy(), o.zd.copy()))
    os.makedirs(cache_dir, exist_ok=True)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, z=np.stack([s[0] for s in states]), zd=np.stack([s[1] for s in states]))
    os.replace(tmp, path)
    return S, states

"""Checkpoint file of the proposer's trainer (host code only): the state
comes back exactly, and a corrupted byte, a truncated file, a foreign
file or another network shape is refused before anything reaches the
network."""
import numpy as np
import pytest

from paper_1109_3186_gb300 import checkpoint


class _FakeNet:
    """Stands in for PropNet: the same shape attributes and state calls."""

    def __init__(self, n_dm=8, hidden=4, k1=3, k2=3, seed=0):
        self.n_dm, self.hidden, self.k1, self.k2 = n_dm, hidden, k1, k2
        n = hidden * n_dm * k1 + hidden + hidden * hidden * k2 + hidden + n_dm * hidden + n_dm
        r = np.random.default_rng(seed)
        self.state = {"params": r.standard_normal(n).astype(np.float32),
                      "m": r.standard_normal(n).astype(np.float32),
                      "v": r.random(n).astype(np.float32), "step": 37}

    def get_state(self):
        return {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in self.state.items()}

    def set_state(self, state):
        self.state = {k: state[k] for k in ("params", "m", "v", "step")}


def test_round_trip_is_exact(tmp_path):
    a, b = _FakeNet(seed=1), _FakeNet(seed=2)
    path = str(tmp_path / "ck.bin")
    checkpoint.save(a, path)
    assert checkpoint.load(b, path) == 37
    for k in ("params", "m", "v"):
        assert np.array_equal(a.state[k], b.state[k])


@pytest.mark.parametrize("damage", ["flip", "truncate", "magic", "shape"])
def test_damaged_or_foreign_checkpoints_are_refused(tmp_path, damage):
    a = _FakeNet(seed=1)
    data = bytearray(checkpoint.encode((a.n_dm, a.hidden, a.k1, a.k2), a.get_state()))
    target = _FakeNet(seed=3)
    if damage == "flip":
        data[60] ^= 0x01
    elif damage == "truncate":
        data = data[:-10]
    elif damage == "magic":
        data[0:4] = b"XXXX"
    else:
        target = _FakeNet(n_dm=9, seed=3)
    path = tmp_path / "ck.bin"
    path.write_bytes(bytes(data))
    before = target.get_state()
    with pytest.raises(ValueError):
        checkpoint.load(target, str(path))
    for k in ("params", "m", "v"):
        assert np.array_equal(before[k], target.state[k])

"""Checkpoint and resume of the proposal network's trainer.

One flat little-endian file:
  magic  b"CHPN", format version (u32),
  network shape: n_dm, hidden, k1, k2 (4 x u32),
  n_params (u64), Adam step (u64),
  parameters, Adam first moments, Adam second moments (3 x n_params float32),
  CRC-32 of every preceding byte (u32).
The Adam step also counts the batches the trainer has drawn, so resuming
with it continues the same batch sequence (Proposer.train's start_step).
Loading checks the magic, the version, the shape and the CRC and raises
ValueError on any mismatch; nothing of a bad file reaches the network.
"""
import struct
import zlib

import numpy as np

MAGIC = b"CHPN"
VERSION = 1
_HEAD = struct.Struct("<4sI4IQQ")


def encode(shape, state) -> bytes:
    """Bytes of a checkpoint: shape (n_dm, hidden, k1, k2), state as returned
    by PropNet.get_state()."""
    arrs = [np.ascontiguousarray(state[k], dtype="<f4") for k in ("params", "m", "v")]
    n = arrs[0].size
    if any(a.size != n for a in arrs):
        raise ValueError("parameter and moment arrays differ in size")
    body = _HEAD.pack(MAGIC, VERSION, *[int(s) for s in shape], n, int(state["step"]))
    body += b"".join(a.tobytes() for a in arrs)
    return body + struct.pack("<I", zlib.crc32(body) & 0xFFFFFFFF)


def decode(data: bytes, shape=None) -> dict:
    """State of a checkpoint's bytes; shape (if given) must match the file's."""
    if len(data) < _HEAD.size + 4:
        raise ValueError("checkpoint too short")
    body, (crc,) = data[:-4], struct.unpack("<I", data[-4:])
    if zlib.crc32(body) & 0xFFFFFFFF != crc:
        raise ValueError("checkpoint CRC mismatch")
    magic, version, n_dm, hidden, k1, k2, n, step = _HEAD.unpack(body[:_HEAD.size])
    if magic != MAGIC or version != VERSION:
        raise ValueError("not a version-%d proposal-network checkpoint" % VERSION)
    if shape is not None and tuple(int(s) for s in shape) != (n_dm, hidden, k1, k2):
        raise ValueError("checkpoint network shape %s differs from %s"
                         % ((n_dm, hidden, k1, k2), tuple(shape)))
    if len(body) != _HEAD.size + 3 * 4 * n:
        raise ValueError("checkpoint length does not match its parameter count")
    arrs = np.frombuffer(body, dtype="<f4", offset=_HEAD.size).reshape(3, n)
    return {"params": arrs[0].astype(np.float32), "m": arrs[1].astype(np.float32),
            "v": arrs[2].astype(np.float32), "step": int(step),
            "shape": (n_dm, hidden, k1, k2)}


def save(net, path: str) -> None:
    """Write the trainer state of a PropNet to path (atomically: a temporary
    file renamed over it)."""
    import os
    data = encode((net.n_dm, net.hidden, net.k1, net.k2), net.get_state())
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        f.write(data)
    os.replace(tmp, path)


def load(net, path: str) -> int:
    """Restore a PropNet's trainer state from path; returns the Adam step."""
    with open(path, "rb") as f:
        state = decode(f.read(), (net.n_dm, net.hidden, net.k1, net.k2))
    net.set_state(state)
    return state["step"]

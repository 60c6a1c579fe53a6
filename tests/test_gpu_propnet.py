"""GPU parity of the learned proposer's hand-written kernels against the FP64
numpy oracle (oracle/propnet.py, itself pinned by central differences):
forward logits, loss and every parameter gradient, three Adam steps, the
per-DM z-score and the window-maximum proposal mask."""
import numpy as np
import pytest

import paper_1109_3186_gb300 as chirp
from oracle import propnet as pn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = [(20, 24, 9, 5, 3, 150), (7, 16, 3, 1, 2, 67), (64, 32, 9, 5, 4, 256)]


def _setup(C, H, K1, K2, B, T, seed):
    rng = np.random.default_rng(seed)
    theta = pn.init(C, H, K1, K2, seed) + 0.01 * rng.standard_normal(pn.n_params(C, H, K1, K2))
    theta = theta.astype(np.float32).astype(np.float64)
    x = rng.standard_normal((B, C, T)).astype(np.float32)
    y = (rng.random((B, C, T)) < 0.05).astype(np.float32)
    net = chirp.PropNet(C, H, K1, K2, B, T)
    assert net.n_params == theta.size
    net.set_params(theta)
    return net, theta, x, y


@pytest.mark.parametrize("C,H,K1,K2,B,T", SHAPES)
def test_forward_matches_oracle(C, H, K1, K2, B, T):
    net, theta, x, _ = _setup(C, H, K1, K2, B, T, 1)
    z = torch.empty((B, C, T), dtype=torch.float32, device="cuda")
    net.forward(torch.from_numpy(x).cuda(), z)
    zo, _ = pn.forward(theta, x.astype(np.float64), C, H, K1, K2)
    assert np.abs(z.cpu().numpy() - zo).max() <= 1e-5 * np.abs(zo).max()


@pytest.mark.parametrize("C,H,K1,K2,B,T", SHAPES)
def test_gradients_match_oracle(C, H, K1, K2, B, T):
    net, theta, x, y = _setup(C, H, K1, K2, B, T, 2)
    loss = net.backward(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), 8.0)
    lo, go = pn.loss_and_grad(theta, x.astype(np.float64), y.astype(np.float64), 8.0, C, H, K1, K2)
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    g = net.grads()
    for a, b_ in zip(pn.unflatten(g, C, H, K1, K2), pn.unflatten(go, C, H, K1, K2)):
        assert np.abs(a - b_).max() <= 1e-4 * np.abs(b_).max() + 1e-9


def test_adam_steps_match_oracle():
    C, H, K1, K2, B, T = 12, 16, 5, 3, 2, 90
    net, theta, x, y = _setup(C, H, K1, K2, B, T, 3)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    th, m, v = theta.copy(), np.zeros_like(theta), np.zeros_like(theta)
    for step in range(1, 4):
        loss_g = net.train_step(xd, yd, 5.0, 1e-3)
        lo, g = pn.loss_and_grad(th, x.astype(np.float64), y.astype(np.float64), 5.0, C, H, K1, K2)
        assert abs(loss_g - lo) <= 1e-5 * abs(lo)
        th, m, v = pn.adam(th, g, m, v, step, 1e-3)
    assert np.abs(net.params() - th).max() <= 1e-5


def test_normalize_and_windows():
    rng = np.random.default_rng(4)
    D = np.abs(rng.standard_normal((5, 300))).astype(np.float32) + 1.0
    D[:, :13] = 0
    D[2, 250:] = 0
    net = chirp.PropNet(5, 4, 3, 3, 1, 300)
    Dd = torch.from_numpy(D).cuda()
    xd = torch.empty_like(Dd)
    net.normalize(Dd, xd)
    x = xd.cpu().numpy()
    for d in range(5):
        v = D[d][D[d] != 0].astype(np.float64)
        ref = np.where(D[d] != 0, (D[d] - v.mean()) / v.std(ddof=1), 0.0)
        assert np.abs(x[d] - ref).max() < 1e-5
    z = rng.standard_normal((5, 300)).astype(np.float32)
    mask = torch.empty((5, 7), dtype=torch.int32, device="cuda")
    net.propose(torch.from_numpy(z).cuda(), 45, 1.5, mask)
    ref = np.array([[z[d, w * 45:(w + 1) * 45].max() > 1.5 for w in range(7)] for d in range(5)])
    assert np.array_equal(mask.cpu().numpy().astype(bool), ref)


def test_checkpoint_resume_continues_bit_for_bit(tmp_path):
    """Six Adam steps in one go equal three steps, a checkpoint written to a
    file, a fresh network restored from it and three more steps -- the
    parameters and both Adam moments bit for bit; restoring the parameters
    alone (Adam state lost) gives a different trainer."""
    from paper_1109_3186_gb300 import checkpoint
    C, H, K1, K2, B, T = 12, 16, 5, 3, 2, 90
    rng = np.random.default_rng(11)
    theta = pn.init(C, H, K1, K2, 4).astype(np.float32)
    batches = [(torch.from_numpy(rng.standard_normal((B, C, T)).astype(np.float32)).cuda(),
                torch.from_numpy((rng.random((B, C, T)) < 0.05).astype(np.float32)).cuda())
               for _ in range(6)]

    def fresh():
        net = chirp.PropNet(C, H, K1, K2, B, T)
        net.set_params(theta)
        return net

    whole = fresh()
    for xb, yb in batches:
        whole.train_step(xb, yb, 5.0, 1e-3)
    first = fresh()
    for xb, yb in batches[:3]:
        first.train_step(xb, yb, 5.0, 1e-3)
    path = str(tmp_path / "trainer.ck")
    checkpoint.save(first, path)
    resumed = chirp.PropNet(C, H, K1, K2, B, T)
    assert checkpoint.load(resumed, path) == 3
    for xb, yb in batches[3:]:
        resumed.train_step(xb, yb, 5.0, 1e-3)
    a, b = whole.get_state(), resumed.get_state()
    assert a["step"] == b["step"] == 6
    for k in ("params", "m", "v"):
        assert np.array_equal(a[k], b[k]), k
    params_only = fresh()
    params_only.set_params(first.params())
    for xb, yb in batches[3:]:
        params_only.train_step(xb, yb, 5.0, 1e-3)
    assert not np.array_equal(params_only.params(), a["params"])

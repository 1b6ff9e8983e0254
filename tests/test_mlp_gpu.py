"""GPU: the surrogate MLP kernels (BF16 operands, FP32 accumulation) against
the FP64 oracle that rounds the same operands to BF16 (oracle/mlp.py)."""
import numpy as np
import pytest

from oracle import mlp as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2506_03127_gb300 import build  # noqa: E402

build.build()
from paper_2506_03127_gb300.surrogate import MLP  # noqa: E402


def _setup(d_in, w, d_out, B, seed):
    rng = np.random.default_rng(seed)
    p = O.init_params(rng, d_in, w, d_out, out_gain=1.0).astype(np.float32)
    p[: p.size] += (0.05 * rng.normal(size=p.size)).astype(np.float32)
    x = rng.normal(size=(B, d_in)).astype(np.float32)
    t = rng.normal(size=(B, d_out)).astype(np.float32)
    net = MLP(d_in, w, d_out, max_batch=max(B, 64))
    net.set_params(p)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    return net, p.astype(np.float64), x.astype(np.float64), t.astype(np.float64), xd, td


@pytest.mark.parametrize("d_in,w,d_out,B", [(258, 256, 8, 100), (7, 5, 3, 13), (64, 96, 8, 33)])
def test_forward_matches_oracle(d_in, w, d_out, B):
    net, p, x, t, xd, td = _setup(d_in, w, d_out, B, 1)
    y = net.forward(xd).cpu().numpy().astype(np.float64)
    yo, _ = O.forward(p, x, d_in, w, d_out, bf16=True)
    assert np.abs(y - yo).max() <= 2e-3 * max(1.0, np.abs(yo).max())
    net.close()


@pytest.mark.parametrize("d_in,w,d_out,B", [(258, 256, 8, 77), (7, 5, 3, 13), (64, 96, 8, 200)])
def test_gradients_match_oracle(d_in, w, d_out, B):
    net, p, x, t, xd, td = _setup(d_in, w, d_out, B, 2)
    loss, g = net.gradients(xd, td)
    lo, go = O.loss_and_grads(p, x, t, d_in, w, d_out, bf16=True)
    assert abs(loss - lo) <= 1e-3 * lo
    g = g.astype(np.float64)
    # per parameter block: W1 b1 W2 b2 W3 b3; BF16 rounding of the back-
    # propagated terms bounds the agreement at ~2^-8 relative
    sizes = [d_in * w, w, w * w, w, w * d_out, d_out]
    o = 0
    for n in sizes:
        a, b = g[o:o + n], go[o:o + n]
        assert np.linalg.norm(a - b) <= 1.5e-2 * np.linalg.norm(b) + 1e-9, (n, np.linalg.norm(a - b) / np.linalg.norm(b))
        o += n
    net.close()


def test_adam_step_matches_oracle_update():
    d_in, w, d_out, B = 40, 32, 8, 50
    net, p, x, t, xd, td = _setup(d_in, w, d_out, B, 3)
    loss, g = net.gradients(xd, td)
    net.train_step(xd, td, 1e-3)
    q = net.params().astype(np.float64)
    qo, _, _ = O.adam_step(p.astype(np.float32).astype(np.float64), g.astype(np.float64), np.zeros(p.size),
                           np.zeros(p.size), 1, 1e-3)
    np.testing.assert_allclose(q, qo, rtol=0, atol=2e-6)
    net.close()


def test_training_fits_a_smooth_map():
    rng = np.random.default_rng(4)
    d_in, w, d_out, B = 16, 64, 8, 512
    x = rng.normal(size=(B, d_in)).astype(np.float32)
    A = rng.normal(size=(d_in, d_out)) / 4
    t = np.tanh(x @ A).astype(np.float32)
    net = MLP(d_in, w, d_out, B)
    net.init(0, out_gain=0.5)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    l0 = net.train_step(xd, td, 3e-3, want_loss=True)
    for _ in range(400):
        net.train_step(xd, td, 3e-3)
    l1 = net.train_step(xd, td, 3e-3, want_loss=True)
    assert l1 < 0.02 * l0
    net.close()

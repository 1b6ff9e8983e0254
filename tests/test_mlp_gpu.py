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


def _grad_magnitudes(p, x, t, d_in, w, d_out):
    """Per parameter, the sum of the magnitudes of the terms the oracle adds
    for its gradient, (|A|^T |B|)_ij over the same BF16-rounded operands
    (for a bias: the sum of |dh| over the batch)."""
    W1, b1, W2, b2, W3, b3 = O.unpack(p, d_in, w, d_out)
    r = O.bf16_round
    y, (h1, h2) = O.forward(p, x, d_in, w, d_out, bf16=True)
    B = x.shape[0]
    dy = 2.0 * (y - t) / (B * d_out)
    dh2 = (r(dy) @ r(W3).T) * (1.0 - h2 * h2)
    dh1 = (r(dh2) @ r(W2).T) * (1.0 - h1 * h1)
    a = np.abs
    return O.pack([a(r(x)).T @ a(r(dh1)), a(dh1).sum(axis=0), a(r(h1)).T @ a(r(dh2)), a(dh2).sum(axis=0),
                   a(r(h2)).T @ a(r(dy)), a(dy).sum(axis=0)])


@pytest.mark.parametrize("d_in,w,d_out,B", [(258, 256, 8, 77), (7, 5, 3, 13), (64, 96, 8, 200)])
def test_gradients_match_oracle(d_in, w, d_out, B):
    """Element by element: both sides multiply the same BF16 operands; the
    kernels accumulate in FP32, and a back-propagated operand (dy, dh2, dh1)
    that the kernels form in FP32 may round to the neighbouring BF16 value,
    one unit (2^-8 relative) from the oracle's.  Every gradient element is
    therefore within 2^-8 of the sum of its terms' magnitudes (all terms
    flipped, the worst case) plus FP32 accumulation; a wrong row or column
    would miss by the size of the terms."""
    net, p, x, t, xd, td = _setup(d_in, w, d_out, B, 2)
    loss, g = net.gradients(xd, td)
    lo, go = O.loss_and_grads(p, x, t, d_in, w, d_out, bf16=True)
    assert abs(loss - lo) <= 1e-3 * lo
    g = g.astype(np.float64)
    mag = _grad_magnitudes(p, x, t, d_in, w, d_out)
    bound = (2.0 ** -8 + B * 2.0 ** -23) * mag + 1e-12
    worst = np.max(np.abs(g - go) / bound)
    assert worst <= 1.0, worst
    # a systematic error (a wrong rounding of every operand, a scaled block)
    # would move the typical element by a good part of 2^-8; rounding flips
    # and accumulation leave the median far below that
    rel = np.abs(g - go) / (mag + 1e-30)
    print(f"gradients: worst {worst:.3f} of the bound; median {np.median(rel):.2e} of the terms' magnitude")
    assert np.median(rel) <= 2.0 ** -12
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

"""The MLP surrogate of the grain optics on the GPU: its labels, forward pass and
gradients against the FP64 CPU reference (oracle/mlp_oracle.py), and training.
Needs a GB300 (``-m gpu``).

Tolerances: labels are FP32 arithmetic on the same tables (1e-5 of the output
scale); the forward pass runs BF16 activations with FP32 accumulation (2e-2 of the
output scale against FP64 with the same BF16-rounded weights); gradients 5e-2
relative in norm per layer (BF16 backward).
"""
import numpy as np
import pytest

from oracle import mlp_oracle as MO
from paper_2512_01283_gb300 import build as B
from paper_2512_01283_gb300 import mcrt as M
from paper_2512_01283_gb300 import workloads as W

pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(77)


@pytest.fixture(scope="module")
def sur():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for -m gpu tests")
    B.build()
    model = W.rayleigh_sphere(n=4)
    model["optics"] = W.table_optics()
    m = M.Model(model)
    s = M.Surrogate(m, seed=3)
    yield s, model["optics"]
    s.close()
    m.close()


def inputs(k):
    a = RNG.normal(size=(k, 3))
    b = RNG.normal(size=(k, 3))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b /= np.linalg.norm(b, axis=1, keepdims=True)
    s = RNG.uniform(-1, 1, size=(k, 1))
    return np.concatenate([a, b, s], axis=1).astype(np.float32)


def bf16(x):
    x = np.asarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_labels_match_oracle(sur):
    s, opt = sur
    u = inputs(300)
    g = s.labels(u)
    for ui, gi in zip(u.astype(np.float64), g):
        ref = MO.label(ui, opt["mueller"], opt["kext"])
        assert np.allclose(gi, ref, atol=2e-5 * (1 + np.abs(ref)))


def test_forward_matches_reference(sur):
    s, _ = sur
    layers = s.get_params()
    ref_params = [(bf16(W_), b_.astype(np.float64)) for W_, b_ in layers]
    u = inputs(512)
    x = bf16(MO.pad_inputs(u))
    # reference with BF16 rounding of the activations between layers, as on the GPU
    h = x
    for i, (W_, b_) in enumerate(ref_params):
        z = h @ W_.T + b_
        h = bf16(MO.silu(z)) if i < len(ref_params) - 1 else z
    y = s.eval(u)
    scale = np.abs(h[:, :20]).max()
    assert np.abs(y - h[:, :20]).max() < 2e-2 * scale


def test_gradients_match_reference(sur):
    """GPU backward (BF16 operands, FP32 accumulation) against the FP64 reference
    backward with the same BF16-rounded weights and inputs."""
    s, opt = sur
    layers = s.get_params()
    u = inputs(1024)
    t = RNG.normal(scale=0.3, size=(1024, 20)).astype(np.float32)
    w = RNG.uniform(0.5, 2.0, size=20).astype(np.float32)
    loss, grads = s.grad(u, t, w)
    ref_params = [(bf16(W_), b_.astype(np.float64)) for W_, b_ in layers]
    rloss, rgrads = MO.loss_and_grads(ref_params, bf16(MO.pad_inputs(u)), t.astype(np.float64), w.astype(np.float64))
    assert abs(loss - rloss) < 2e-2 * rloss
    for li, ((gW, gb), (rW, rb)) in enumerate(zip(grads, rgrads)):
        if li == 0:
            gW, rW = gW[:, :MO.N_IN], rW[:, :MO.N_IN]
        if li == len(grads) - 1:
            gW, rW, gb, rb = gW[:20], rW[:20], gb[:20], rb[:20]
        assert np.linalg.norm(gW - rW) < 5e-2 * np.linalg.norm(rW), li
        assert np.linalg.norm(gb - rb) < 5e-2 * np.linalg.norm(rb), li


def test_training_reduces_the_error(sur):
    s, opt = sur
    u = inputs(2000)
    lab = s.labels(u)
    before = np.sqrt(np.mean((s.eval(u) - lab) ** 2))
    hist = s.train(n_steps=300, batch=4096, lr=3e-3)
    assert np.all(np.isfinite(hist))
    assert hist[-20:].mean() < 0.2 * hist[:20].mean()
    after = np.sqrt(np.mean((s.eval(u) - lab) ** 2))
    assert after < 0.3 * before

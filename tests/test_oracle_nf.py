"""Pins of the surrogate oracle (oracle/nf.py): the hand-written backward pass
against central finite differences and against torch autograd, the bf16
rounding against torch's bfloat16 cast, and Adam against torch.optim.Adam."""
import numpy as np
import pytest
import torch

from oracle import nf


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    uvr = np.column_stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(0, 1, n)])
    return uvr, rng.uniform(0.05, 0.95, n)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = rng.normal(scale=3.0, size=10000).astype(np.float32)
    x[:4] = [0.0, -0.0, 1e-40, 65504.0]
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(nf.bf16(x), ref)


def test_features_are_the_fourier_basis():
    uvr = np.array([[0.25, -0.5, 0.75]])
    f = nf.features(uvr, round_bf16=False)[0]
    for a in range(3):
        for m in range(16):
            ang = np.pi * 2.0 ** (8 * m / 15) * uvr[0, a]
            assert f[32 * a + m] == pytest.approx(np.sin(ang), abs=1e-12)
            assert f[32 * a + 16 + m] == pytest.approx(np.cos(ang), abs=1e-12)


def test_gradient_matches_finite_differences():
    p = nf.init_params(1).astype(np.float64)
    p[nf.N_PARAMS - 1] = 0.3
    uvr, tgt = _batch(16, 2)
    _, g = nf.loss_and_grad(p, uvr, tgt, round_bf16=False)
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(nf.N_PARAMS, 40, replace=False), [nf.N_PARAMS - 1]])
    for i in idx:
        h = 1e-6 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (nf.loss_and_grad(pp, uvr, tgt, False)[0] - nf.loss_and_grad(pm, uvr, tgt, False)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-11)


def test_gradient_matches_torch_autograd():
    p = nf.init_params(4).astype(np.float64)
    uvr, tgt = _batch(32, 5)
    loss, g = nf.loss_and_grad(p, uvr, tgt, round_bf16=False)
    P = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in nf.unpack(p).items()}
    h = torch.tensor(nf.features(uvr, round_bf16=False))
    for l in (1, 2, 3, 4):
        h = torch.relu(h @ P[f"W{l}"].T + P[f"b{l}"])
    T = torch.sigmoid(h @ P["w5"] + P["b5"][0])
    L = torch.mean((T - torch.tensor(tgt)) ** 2)
    L.backward()
    ref = np.concatenate([P[name].grad.numpy().ravel() for name, _ in nf.SHAPES])
    assert float(L) == pytest.approx(loss, rel=1e-12)
    np.testing.assert_allclose(g, ref, rtol=1e-9, atol=1e-15)


def test_adam_matches_torch():
    rng = np.random.default_rng(6)
    p0 = rng.normal(size=50)
    grads = [rng.normal(size=50) for _ in range(5)]
    t = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.Adam([t], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for s, gr in enumerate(grads, 1):
        opt.zero_grad()
        t.grad = torch.tensor(gr)
        opt.step()
        p, m, v = nf.adam_step(p, gr, m, v, s)
    np.testing.assert_allclose(p, t.detach().numpy(), rtol=1e-12, atol=1e-14)

"""FP64 oracle of the learned transmittance surrogate (the per-light neural
transmittance field that stands in for the static-scene atlas lookup).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Architecture (fixed):
  input (u, v, rho): octahedral coordinates of the direction (Eq. 6) and the
  fractional shell coordinate rho = (k + w) / (K - 1) in [0, 1];
  features: for each input x and m = 0..15, sin(pi p) and cos(pi p) of the
  phase p = f_m x, f_m = 2^(8m/15) (1 .. 256); feature index 32*axis + m for
  the sine, 32*axis + 16 + m for the cosine (96 features).  Because each
  feature is then rounded to bfloat16 (a quantisation decision), the phase
  is the float32 product of float32(f_m) and the float32 input, as the GPU
  forms it; sin and cos are FP64;
  four hidden layers of width 64 with ReLU, one linear output, sigmoid.
Numerics of the "BF16 MLP with FP32 accumulation": features, weights and
hidden activations are rounded to bfloat16 (round to nearest even) before
each product; sums and biases are exact here (FP64); the backward pass treats
each rounding as the identity (straight-through).

Parameter vector (float32, 18753 values): W1 (64x96, [out][in]), b1 (64),
W2, b2, W3, b3 (64x64, 64 each), W4 (64x64), b4 (64), w5 (64), b5 (1).
"""
from __future__ import annotations

import numpy as np

N_FREQ = 16
N_FEAT = 96
HID = 64
FREQ = 2.0 ** (8.0 * np.arange(N_FREQ) / 15.0)
FREQ32 = FREQ.astype(np.float32)
SHAPES = [("W1", (HID, N_FEAT)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (HID, HID)), ("b3", (HID,)), ("W4", (HID, HID)), ("b4", (HID,)),
          ("w5", (HID,)), ("b5", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    nan = np.isnan(f)
    out = rounded.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def unpack(params) -> dict:
    p = np.asarray(params, dtype=np.float64).ravel()
    assert p.size == N_PARAMS
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def features(uvr, round_bf16: bool = True) -> np.ndarray:
    """(n,3) -> (n,96) Fourier features.  With round_bf16 the phase is the
    float32 product (see the module docstring); without, everything is FP64."""
    if round_bf16:
        x32 = np.asarray(uvr, dtype=np.float32).reshape(-1, 3)
        p = (x32[:, :, None] * FREQ32[None, None, :]).astype(np.float64)   # float32 products
        p = p - 2.0 * np.rint(0.5 * p)                                      # exact reduction
        ph = np.pi * p
    else:
        uvr = np.asarray(uvr, dtype=np.float64).reshape(-1, 3)
        ph = np.pi * uvr[:, :, None] * FREQ[None, None, :]              # (n,3,16)
    f = np.concatenate([np.sin(ph), np.cos(ph)], axis=2).reshape(-1, N_FEAT)
    return bf16(f) if round_bf16 else f


def forward(params, uvr, round_bf16: bool = True):
    """T_hat (n,) and the cache the backward pass needs."""
    P = unpack(params)
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    h = features(uvr, round_bf16)
    cache = {"h": [h], "z": []}
    for l in (1, 2, 3, 4):
        z = h @ r(P[f"W{l}"]).T + P[f"b{l}"]
        h = r(np.maximum(z, 0.0))
        cache["z"].append(z)
        cache["h"].append(h)
    y = h @ r(P["w5"]) + P["b5"][0]
    T = 1.0 / (1.0 + np.exp(-y))
    cache["T"] = T
    return T, cache


def loss_and_grad(params, uvr, target, round_bf16: bool = True):
    """Mean squared error over the batch and its gradient (packed like params)."""
    P = unpack(params)
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    T, c = forward(params, uvr, round_bf16)
    target = np.asarray(target, dtype=np.float64).ravel()
    B = T.size
    loss = float(np.mean((T - target) ** 2))
    dy = 2.0 * (T - target) * T * (1.0 - T) / B
    g = {"w5": c["h"][4].T @ dy, "b5": np.array([dy.sum()])}
    dh = np.outer(dy, r(P["w5"]))
    for l in (4, 3, 2, 1):
        dz = dh * (c["z"][l - 1] > 0)
        g[f"W{l}"] = dz.T @ c["h"][l - 1]
        g[f"b{l}"] = dz.sum(0)
        dh = dz @ r(P[f"W{l}"])
    return loss, pack(g)


def adam_step(params, grad, m, v, step: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (params, m, v)."""
    params = np.asarray(params, dtype=np.float64)
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights, zero biases (float32)."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in SHAPES:
        if name.startswith("b"):
            d[name] = np.zeros(shape)
        else:
            fan_in = shape[-1] if len(shape) == 2 else HID
            lim = np.sqrt(6.0 / fan_in)
            d[name] = rng.uniform(-lim, lim, shape)
    return pack(d).astype(np.float32)

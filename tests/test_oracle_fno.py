"""Pins of the FP64 surrogate reference (oracle/fno_ref.py).

- Its gradient equals central finite differences of its loss along random
  directions (the autodiff is checked, not trusted).
- A spectral layer with identity mixing (A_k = I, B_k = 0) reproduces a
  signal made of modes below K and removes modes at or above K: the inverse
  basis scaling (1/n at k = 0, 2/n above) and the truncation.
- With A_k = 0, B_k = I (the weight i) it maps cos(2 pi k x / n) to
  sin(2 pi k x / n): the orientation of the complex mixing that the
  library's real 2 x 2 blocks [[A, -B], [B, A]] implement.
"""
import math

import numpy as np
import pytest
import torch

from oracle import fno_ref


def _rand(dims, seed, scale=0.3):
    nx, ny, C, K, L = dims
    r = np.random.default_rng(seed)
    n = sum(int(np.prod(s)) for _, s in fno_ref.layout(C, K, L))
    p = r.standard_normal(n) * scale / np.sqrt(C)
    P = nx * ny
    now = r.standard_normal((6, P))
    nxt = now + 0.1 * r.standard_normal((6, P))
    norm = (r.uniform(-0.5, 0.5, 6), r.uniform(0.5, 2.0, 6), r.uniform(0.5, 2.0, 6))
    return p, now, nxt, norm


@pytest.mark.parametrize("cons", [0.0, 30.0])
def test_gradient_matches_finite_differences(cons):
    dims = (16, 12, 4, 3, 2)
    p, now, nxt, norm = _rand(dims, 1)
    loss, g = fno_ref.loss_and_grad(p, now, nxt, dims, norm, cons)
    r = np.random.default_rng(2)
    for _ in range(4):
        d = r.standard_normal(p.size)
        eps = 1e-6
        lp, _ = fno_ref.loss_and_grad(p + eps * d, now, nxt, dims, norm, cons)
        lm, _ = fno_ref.loss_and_grad(p - eps * d, now, nxt, dims, norm, cons)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-6 * max(1.0, abs(fd)), (fd, g @ d)


@pytest.mark.parametrize("axis", [-1, -2])
def test_identity_mixing_reproduces_band_limited_signals(axis):
    C, K, nx, ny = 3, 4, 20, 16
    r = np.random.default_rng(3)
    n = nx if axis == -1 else ny
    coord = np.arange(n)
    low = np.zeros((C, ny, nx))
    high = np.zeros((C, ny, nx))
    for c in range(C):
        for k in range(K):
            a, b = r.standard_normal(2)
            wave = a * np.cos(2 * np.pi * k * coord / n) + b * np.sin(2 * np.pi * k * coord / n)
            low[c] += wave[None, :] if axis == -1 else wave[:, None]
        k = K + 1 + c
        wave = np.cos(2 * np.pi * k * coord / n)
        high[c] = wave[None, :] if axis == -1 else wave[:, None]
    A = torch.eye(C, dtype=torch.float64).repeat(K, 1, 1)
    B = torch.zeros_like(A)
    out_low = fno_ref.spectral(torch.from_numpy(low), A, B, axis, K).numpy()
    out_high = fno_ref.spectral(torch.from_numpy(high), A, B, axis, K).numpy()
    assert np.allclose(out_low, low, atol=1e-12)
    assert np.abs(out_high).max() < 1e-12


def test_imaginary_unit_weight_turns_cosine_into_sine():
    C, K, nx, ny = 2, 4, 24, 8
    x = np.arange(nx)
    h = np.zeros((C, ny, nx))
    k = 3
    h[:] = np.cos(2 * np.pi * k * x / nx)[None, None, :]
    A = torch.zeros((K, C, C), dtype=torch.float64)
    B = torch.eye(C, dtype=torch.float64).repeat(K, 1, 1)
    out = fno_ref.spectral(torch.from_numpy(h), A, B, -1, K).numpy()
    assert np.allclose(out, np.sin(2 * np.pi * k * x / nx)[None, None, :].repeat(ny, 1).repeat(C, 0), atol=1e-12)


def test_zero_model_loss_is_the_target_moments():
    # all parameters zero: y = 0, so the loss is mean(t^2) over the six state
    # channels plus cons * mean(t_0)^2, and the gradient of the output bias
    # b_out[c] is -2 mean(t_c) / 6 (+ the conservation term's -2 cons mean(t_0) on c = 0)
    dims = (8, 8, 4, 2, 1)
    _, now, nxt, norm = _rand(dims, 4)
    n = sum(int(np.prod(s)) for _, s in fno_ref.layout(4, 2, 1))
    _, t = fno_ref.pack(now, nxt, 8, 8, *norm)
    t = t.numpy()
    cons = 7.0
    loss, g = fno_ref.loss_and_grad(np.zeros(n), now, nxt, dims, norm, cons)
    assert np.isclose(loss, (t[:6] ** 2).mean() + cons * t[0].mean() ** 2, rtol=1e-12)
    gb = g[-16:]
    expect = -2.0 * t[:6].mean(axis=(1, 2)) / 6.0
    expect[0] -= 2.0 * cons * t[0].mean()
    assert np.allclose(gb[:6], expect, rtol=1e-10, atol=1e-14)
    assert np.all(gb[6:] == 0.0)


def test_parameter_count_of_the_workload_model():
    # C = 64, K = 32, L = 4: about 2.1 M parameters (the surrogate workload)
    n = sum(int(np.prod(s)) for _, s in fno_ref.layout(64, 32, 4))
    assert n == 2115920
    assert abs(fno_ref.gelu(torch.tensor(0.0)).item()) == 0.0
    assert math.isclose(fno_ref.gelu(torch.tensor(10.0)).item(), 10.0, rel_tol=1e-12)

"""FP64 CPU reference of the learned surrogate (factorised Fourier neural
operator), for tests only.

TEST INFRASTRUCTURE (see oracle/__init__.py): only tests/ may use it.  Written
independently of the library's kernels: the spectral layers use the FFT
(torch.fft.rfft / irfft along one axis, truncated to K modes) where the
library uses BF16 matrix products with truncated real-DFT bases, and the
gradient comes from automatic differentiation in float64, pinned to central
finite differences by tests/test_oracle_fno.py.

Model (the definition the library documents in include/lbm.h), channels C, K
modes per axis, L layers, state channels padded to 16:
  h_0 = W_in x + b_in
  h_l = GELU(W_l h_{l-1} + b_l + S^x_l(h_{l-1}) + S^y_l(h_{l-1}))
  y   = W_out h_L + b_out
S^x(h)[c] along x: F_k = rfft(h)[k] (k < K); with the mode's complex weight
W_k = A_k + i B_k the layer returns irfft of G_k = conj(W_k) F_k (zero above
K).  In real terms this is the coefficient pair (c_k, s_k) = (Re F_k, -Im F_k)
mixed by [[A, -B], [B, A]] and summed back as (1/n)(c_0) + (2/n) sum_k
(c_k cos + s_k sin), the library's form.  GELU is the tanh approximation.
Loss: mean over the 6 state channels and all nodes of (y - t)^2, plus
cons * (mean over the nodes of y_0 - t_0)^2 (channel 0 is alpha_g).
Pinned by tests/test_oracle_fno.py: its gradient against central finite
differences of its loss (with and without the conservation term), identity
mixing reproducing band-limited signals and removing modes >= K, the weight i
turning cos into sin, and the all-zero model's loss and output-bias gradient
in closed form.  The surrogate is not the paper's method: these pins fix the
model the library defines, not a result of the paper.
"""
import math

import numpy as np
import torch

CIN = COUT = 16
CV = 6


def layout(C, K, L):
    """(name, shape) of every parameter block in the library's order."""
    out = [("W_in", (C, CIN)), ("b_in", (C,))]
    for l in range(L):
        out += [("W%d" % l, (C, C)), ("b%d" % l, (C,)), ("Ax%d" % l, (K, C, C)), ("Bx%d" % l, (K, C, C)),
                ("Ay%d" % l, (K, C, C)), ("By%d" % l, (K, C, C))]
    out += [("W_out", (COUT, C)), ("b_out", (COUT,))]
    return out


def unflatten(flat, C, K, L):
    d, at = {}, 0
    for name, shape in layout(C, K, L):
        n = int(np.prod(shape))
        d[name] = flat[at:at + n].reshape(shape)
        at += n
    assert at == flat.numel() if isinstance(flat, torch.Tensor) else at == flat.size
    return d


def gelu(z):
    return 0.5 * z * (1.0 + torch.tanh(math.sqrt(2.0 / math.pi) * (z + 0.044715 * z ** 3)))


def spectral(h, A, B, axis, K):
    """h: (C, ny, nx); axis -1 (x) or -2 (y)."""
    n = h.shape[axis]
    F = torch.fft.rfft(h, dim=axis)
    F = F.narrow(axis, 0, K)                       # (C, ..., K, ...)
    W = torch.complex(A, B)                        # (K, C_out, C_in)
    Wc = torch.conj(W)
    if axis == -1:
        G = torch.einsum("koi,iyk->oyk", Wc, F)
    else:
        G = torch.einsum("koi,ikx->okx", Wc, F)
    pad = n // 2 + 1 - K
    shape = list(G.shape)
    shape[axis] = pad
    G = torch.cat([G, torch.zeros(shape, dtype=G.dtype)], dim=axis)
    return torch.fft.irfft(G, n=n, dim=axis)


def forward(params, x, C, K, L):
    """params: float64 tensor (flat); x: (16, ny, nx) float64.  Returns y (16, ny, nx)."""
    p = unflatten(params, C, K, L)
    h = torch.einsum("oi,iyx->oyx", p["W_in"], x) + p["b_in"][:, None, None]
    for l in range(L):
        z = torch.einsum("oi,iyx->oyx", p["W%d" % l], h) + p["b%d" % l][:, None, None]
        z = z + spectral(h, p["Ax%d" % l], p["Bx%d" % l], -1, K) + spectral(h, p["Ay%d" % l], p["By%d" % l], -2, K)
        h = gelu(z)
    return torch.einsum("oi,iyx->oyx", p["W_out"], h) + p["b_out"][:, None, None]


def pack(now, nxt, nx, ny, mean, std_in, std_out):
    """Input x (16, ny, nx) and target t from FP64 states (6, nx*ny)."""
    x = np.zeros((CIN, ny, nx))
    t = np.zeros((COUT, ny, nx))
    for c in range(CV):
        x[c] = ((now[c] - mean[c]) / std_in[c]).reshape(ny, nx)
        if nxt is not None:
            t[c] = ((nxt[c] - now[c]) / std_out[c]).reshape(ny, nx)
    return torch.from_numpy(x), torch.from_numpy(t)


def loss_and_grad(params, now, nxt, dims, norm, cons=0.0):
    """FP64 loss and gradient (numpy, the library's parameter order)."""
    nx, ny, C, K, L = dims
    x, t = pack(now, nxt, nx, ny, *norm)
    p = torch.tensor(np.asarray(params, np.float64), requires_grad=True)
    y = forward(p, x, C, K, L)
    loss = ((y[:CV] - t[:CV]) ** 2).mean() + cons * (y[0] - t[0]).mean() ** 2
    loss.backward()
    return float(loss.detach()), p.grad.numpy().copy()


def advance(params, now, dims, norm):
    """next = now + std_out * y (numpy (6, nx*ny))."""
    nx, ny, C, K, L = dims
    mean, std_in, std_out = norm
    x, _ = pack(now, None, nx, ny, mean, std_in, std_out)
    with torch.no_grad():
        y = forward(torch.tensor(np.asarray(params, np.float64)), x, C, K, L).numpy()
    return np.stack([now[c] + std_out[c] * y[c].reshape(-1) for c in range(CV)])

"""FP64 CPU oracle of the learned-closure CNN: forward pass, MSE loss and its
gradient with respect to every parameter.

TEST INFRASTRUCTURE ONLY (tests, smoke and the CPU legs of bench.py).  Plain
PyTorch CPU ops in float64; the gradient comes from the chain rule written out
with conv2d / conv_transpose2d primitives, not from the CUDA code.

Network (the closure of a 2x-coarsened lattice Boltzmann run):
  x [4, ny, nx] -> conv3x3 (4 -> 32) + b1 -> ReLU -> conv3x3 (32 -> 32) + b2 -> ReLU
    -> conv3x3 (32 -> 4) + b3 -> y [4, ny, nx]
Every 3x3 convolution is a cross-correlation out[o, y, x] = sum_{c, dy, dx}
w[o, c, dy + 1, dx + 1] in[c, y + dy, x + dx], with x periodic and zero padding
beyond the walls in y.  Loss: mean over all 4 * ny * nx outputs of (y - t)^2.
Parameters are one flat vector in the order w1, b1, w2, b2, w3, b3 with w of
shape [out, in, 3, 3].
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

SHAPES = [(32, 4, 3, 3), (32,), (32, 32, 3, 3), (32,), (4, 32, 3, 3), (4,)]
N_PARAMS = int(sum(np.prod(s) for s in SHAPES))


def unpack(params: np.ndarray) -> list[torch.Tensor]:
    out, k = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(torch.tensor(np.asarray(params[k:k + n], dtype=np.float64).reshape(s)))
        k += n
    return out


def pad(a: torch.Tensor) -> torch.Tensor:
    """[C, ny, nx] -> [C, ny + 2, nx + 2]: periodic in x, zeros in y."""
    a = torch.cat([a[:, :, -1:], a, a[:, :, :1]], dim=2)
    z = torch.zeros_like(a[:, :1, :])
    return torch.cat([z, a, z], dim=1)


def conv(a: torch.Tensor, w: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    return F.conv2d(pad(a)[None], w)[0] + b[:, None, None]


def forward(params: np.ndarray, x: np.ndarray) -> dict:
    w1, b1, w2, b2, w3, b3 = unpack(params)
    x = torch.tensor(np.asarray(x, dtype=np.float64))
    z1 = conv(x, w1, b1)
    a1 = torch.relu(z1)
    z2 = conv(a1, w2, b2)
    a2 = torch.relu(z2)
    y = conv(a2, w3, b3)
    return dict(x=x, z1=z1, a1=a1, z2=z2, a2=a2, y=y)


def round_bf16(a: torch.Tensor) -> torch.Tensor:
    """Round to FP32 and then to BFloat16 (8 significant bits), both to nearest
    even, returned in float64: the storage format of 16-bit activations."""
    b = a.to(torch.float32).numpy().view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return torch.tensor(b.astype(np.uint32).view(np.float32).astype(np.float64))


def forward_bf16_activations(params: np.ndarray, x: np.ndarray) -> dict:
    """The network as evaluated with BF16 activations: the input and both hidden
    layers (after ReLU) are rounded to BF16 before the next convolution, all
    arithmetic in float64."""
    w1, b1, w2, b2, w3, b3 = unpack(params)
    x = round_bf16(torch.tensor(np.asarray(x, dtype=np.float64)))
    a1 = round_bf16(torch.relu(conv(x, w1, b1)))
    a2 = round_bf16(torch.relu(conv(a1, w2, b2)))
    return dict(x=x, a1=a1, a2=a2, y=conv(a2, w3, b3))


def loss(params: np.ndarray, x: np.ndarray, t: np.ndarray) -> float:
    y = forward(params, x)["y"]
    return float(torch.mean((y - torch.tensor(np.asarray(t, dtype=np.float64))) ** 2))


def conv_backward(a: torch.Tensor, w: torch.Tensor, g: torch.Tensor):
    """Gradients of out = conv(a, w, b) given dL/dout = g: (dL/da, dL/dw, dL/db)."""
    ap = pad(a)
    dw = F.conv2d(ap[:, None], g[:, None])          # [C_in, C_out, 3, 3] -> transpose below
    dw = dw.permute(1, 0, 2, 3).contiguous()
    db = g.sum(dim=(1, 2))
    dap = F.conv_transpose2d(g[None], w)[0]          # gradient w.r.t. the padded input
    ny, nx = a.shape[1], a.shape[2]
    da = dap[:, 1:ny + 1, 1:nx + 1].clone()
    da[:, :, 0] += dap[:, 1:ny + 1, nx + 1]          # periodic images in x fold back
    da[:, :, nx - 1] += dap[:, 1:ny + 1, 0]
    return da, dw, db


def loss_and_grad(params: np.ndarray, x: np.ndarray, t: np.ndarray) -> tuple[float, np.ndarray]:
    w1, b1, w2, b2, w3, b3 = unpack(params)
    c = forward(params, x)
    t = torch.tensor(np.asarray(t, dtype=np.float64))
    diff = c["y"] - t
    L = float(torch.mean(diff ** 2))
    gy = 2.0 * diff / diff.numel()
    ga2, gw3, gb3 = conv_backward(c["a2"], w3, gy)
    gz2 = ga2 * (c["z2"] > 0)
    ga1, gw2, gb2 = conv_backward(c["a1"], w2, gz2)
    gz1 = ga1 * (c["z1"] > 0)
    _, gw1, gb1 = conv_backward(c["x"], w1, gz1)
    grad = np.concatenate([g.numpy().ravel() for g in (gw1, gb1, gw2, gb2, gw3, gb3)])
    return L, grad


def init_params(seed: int) -> np.ndarray:
    """He-scaled normal weights and zero biases (float64)."""
    rng = np.random.default_rng(seed)
    out = []
    for s in SHAPES:
        if len(s) == 4:
            out.append(rng.normal(0.0, np.sqrt(2.0 / (s[1] * 9)), size=s).ravel())
        else:
            out.append(np.zeros(s))
    return np.concatenate(out)

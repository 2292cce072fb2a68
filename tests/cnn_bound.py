"""Worst-case error bound of the CNN evaluated with BF16 activations and FP32
accumulation (the tensor-core inference path) against the exact FP64 network
with the same BF16 weights.  A catch-all (it sums |w| |a| over 288 terms per
layer, so it is ~100 times the typical error); the tight comparison is with
the oracle's forward_bf16_activations.

Rounding to BF16 (nearest; 8 significant bits) moves a value v by at most u |v|,
u = 2^-8; an FP32 sum of K products errs by at most K 2^-24 times the sum of their
magnitudes.
Both propagate through a convolution as through the convolution with |w|, and
through ReLU without growth (it is 1-Lipschitz).  With e the bound on a layer's
input error and a its exact value:
    e_z = |w| * e + g_K |w| * (|a| + e)          (input error + accumulation)
    e_next = e_z + u (|relu z| + e_z)             (the stored activation is rounded)
and the output error is bounded by the last e_z (plus the FP32 bias addition).
"""
from __future__ import annotations

import numpy as np
import torch

from oracle import cnn_oracle as N

U_BF16 = 2.0 ** -8
EPS_F32 = 2.0 ** -24


def _absconv(a: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
    return N.conv(a, w.abs(), torch.zeros(w.shape[0], dtype=w.dtype))


def bf16_activation_bound(params: np.ndarray, x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(exact y, elementwise bound on |y_bf16-activations - y|) for FP64 params
    that already hold the BF16-rounded weights."""
    f = N.forward(params, x)
    w1, _, w2, _, w3, _ = N.unpack(params)
    ex = U_BF16 * f["x"].abs()
    ez1 = _absconv(ex, w1) + 36 * EPS_F32 * _absconv(f["x"].abs() + ex, w1)
    e1 = ez1 + U_BF16 * (f["a1"].abs() + ez1)
    ez2 = _absconv(e1, w2) + 288 * EPS_F32 * _absconv(f["a1"].abs() + e1, w2)
    e2 = ez2 + U_BF16 * (f["a2"].abs() + ez2)
    ey = _absconv(e2, w3) + 288 * EPS_F32 * _absconv(f["a2"].abs() + e2, w3)
    y = f["y"]
    ey = ey + 2 * EPS_F32 * (y.abs() + ey)
    return y.numpy(), ey.numpy()

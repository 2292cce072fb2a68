"""Seeded synthetic inputs shared by the oracle and the CUDA tests.

Holds no arithmetic of the method: parameter sets (the workloads' shapes and
physical constants) and seeded random arrays only.
"""
from __future__ import annotations

import numpy as np

# Plain method, small: 128 x 256, tau 1, G 1.4, masses 1.0 / 0.9, g 1e-5,
# interface at ny/2 with an 8-mode sinusoid-sum perturbation of amplitude 2.
C0 = dict(nx=128, ny=256, tau_A=1.0, tau_B=1.0, G=1.4, mass_A=1.0, mass_B=0.9, g=1e-5,
          n_modes=8, amp=2.0, width=1.5, minority=0.08, crop_rows=10)
# Same physics at 1024 x 2048 (the measured workload); miscible variant with G = 0.
C1 = dict(C0, nx=1024, ny=2048)
C1_MISCIBLE = dict(C1, G=0.0, minority=0.0)
# Full-size grid 10000 x 5000.
C2 = dict(C0, nx=10000, ny=5000)


def params(base: dict, **kw) -> dict:
    d = dict(base)
    d.update(kw)
    return d


def random_populations(seed: int, nx: int, ny: int, lo: float = 0.01, hi: float = 0.25) -> np.ndarray:
    """Positive uniform random populations, shape (2, 9, ny, nx), float64."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(2, 9, ny, nx))


def as_float32(a: np.ndarray) -> np.ndarray:
    """Round to float32 and back (the values an FP32 store can hold exactly)."""
    return a.astype(np.float32).astype(np.float64)

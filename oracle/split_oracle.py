"""Domain decomposition of the FP64 oracle along x (an extension: the paper runs one
grid per GPU).

TEST INFRASTRUCTURE ONLY: used by tests/, never by the product path.  It checks the
split-grid protocol against the whole-grid oracle: a grid cut into sub-grids of
consecutive columns advances each sub-grid with the whole-grid step of
lbm_oracle on the sub-grid widened by two columns on each side, which hold the
neighbours' edge columns ("ghost" columns, exchanged before every step).  One step
at a site needs the densities of its neighbours (the Shan-Chen force) and the
post-collision populations of its neighbours (streaming), so two columns of
post-streaming populations on each side make the sub-grid's own columns exact; the
widened array's own periodic wrap only touches the ghost columns, which are dropped.
"""
from __future__ import annotations

import numpy as np

from oracle import lbm_oracle as O

GHOST = 2


def split_columns(nx: int, parts: int) -> list[tuple[int, int]]:
    """Column ranges [x0, x1) of `parts` sub-grids of nearly equal width."""
    edges = [round(k * nx / parts) for k in range(parts + 1)]
    return [(edges[k], edges[k + 1]) for k in range(parts)]


def widen(own: np.ndarray, left: np.ndarray, right: np.ndarray) -> np.ndarray:
    """The sub-grid's populations with the left neighbour's last two columns before
    and the right neighbour's first two after."""
    return np.concatenate([left, own, right], axis=-1)


def step_widened(wide: np.ndarray, p: O.Params) -> np.ndarray:
    """One whole-grid oracle step on the widened sub-grid; returns the sub-grid's own
    columns."""
    pw = p.with_(nx=wide.shape[-1])
    return O.stream(O.collide(wide, pw))[..., GHOST:-GHOST]


def step_split(parts: list[np.ndarray], p: O.Params, nsteps: int = 1) -> list[np.ndarray]:
    """Advance sub-grids (in order along x, periodic) by exchanging ghost columns and
    stepping each widened sub-grid, nsteps times."""
    n = len(parts)
    for _ in range(nsteps):
        edges = [(q[..., :GHOST], q[..., -GHOST:]) for q in parts]
        parts = [step_widened(widen(parts[k], edges[k - 1][1], edges[(k + 1) % n][0]), p) for k in range(n)]
    return parts

"""Lattice stencils D3Q7 / D3Q15 / D3Q19 / D3Q27 (App. B, Fig. stencils).

The paper gives the velocity *classes* and the weights of each class
(App. B, weight equations for w_{q,D3Q7} ... w_{q,D3Q27}); it fixes no
ordering inside a class.  Ordering used here: rest; the six face neighbours
(+x, -x, +y, -y, +z, -z); the twelve edge neighbours; the eight corners.
Weights are exact rationals (``fractions.Fraction``) taken from App. B,
including w_0 = 0 for D3Q7 (taken literally: c_s^2 = 1/3 for every stencil).
"""
from __future__ import annotations

from dataclasses import dataclass
from fractions import Fraction
from typing import Tuple

import numpy as np

_REST = [(0, 0, 0)]
_FACES = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
_EDGES = [(1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
          (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
          (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
_CORNERS = [(1, 1, 1), (-1, -1, -1), (1, 1, -1), (-1, -1, 1),
            (1, -1, 1), (-1, 1, -1), (-1, 1, 1), (1, -1, -1)]

# App. B: weight per velocity class (rest, faces, edges, corners).
_CLASS_WEIGHTS = {
    7: (Fraction(0, 6), Fraction(1, 6), None, None),
    15: (Fraction(16, 72), Fraction(8, 72), None, Fraction(1, 72)),
    19: (Fraction(12, 36), Fraction(2, 36), Fraction(1, 36), None),
    27: (Fraction(64, 216), Fraction(16, 216), Fraction(4, 216), Fraction(1, 216)),
}


@dataclass(frozen=True)
class Stencil:
    Q: int
    c: np.ndarray            # (Q, 3) int
    w_exact: Tuple[Fraction, ...]
    w: np.ndarray            # (Q,) float64
    opp: np.ndarray          # (Q,) index of -c_i


def stencil(Q: int) -> Stencil:
    if Q not in _CLASS_WEIGHTS:
        raise ValueError(f"unsupported stencil D3Q{Q}")
    wr, wf, we, wc = _CLASS_WEIGHTS[Q]
    vel, wts = [], []
    for cls, wt in ((_REST, wr), (_FACES, wf), (_EDGES, we), (_CORNERS, wc)):
        if wt is None:
            continue
        vel += cls
        wts += [wt] * len(cls)
    c = np.array(vel, dtype=np.int64)
    opp = np.array([vel.index((-a, -b, -d)) for (a, b, d) in vel], dtype=np.int64)
    return Stencil(Q, c, tuple(wts), np.array([float(x) for x in wts]), opp)

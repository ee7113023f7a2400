"""Far-field steps on either side of the translation: aggregation (Eq. 4) and
disaggregation (Eq. 6).

Oracle / test infrastructure only (see package docstring).

    A_v(k_p) = sum_{n in B_v} P^+(k_p, b_n) I_n                          (Eq. 4)
    y_m      = sum_p w_p P^-(k_p, b_m) . B_{v'}(k_p),   P^- = conj(P^+)    (Eq. 6)

with theta / phi components for the patterns and the spectra (Sec. II.A: only
those two components of the far-field patterns are kept) and w_p the
quadrature weights of the directions.  Arrays, nb basis functions per box:
patterns P[p][c][i][z][y][x] (c = 0 theta, 1 phi), coefficients
I[r][i][z][y][x], spectra A, B [p][c][r][z][y][x] (the translation's field
layout), results y[r][i][z][y][x].
"""
from __future__ import annotations

import numpy as np


def aggregate(P: np.ndarray, I: np.ndarray) -> np.ndarray:
    """Eq. 4 for every box, direction, polarisation and right-hand side."""
    return np.einsum("pcizyx,rizyx->pcrzyx", P, I)


def disaggregate(P: np.ndarray, w: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Eq. 6: the quadrature over directions of conj(P^+) . B, per basis function."""
    return np.einsum("p,pcizyx,pcrzyx->rizyx", np.asarray(w), np.conj(P), B)

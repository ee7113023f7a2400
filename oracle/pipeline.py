"""Whole-stage drivers: operators of a box grid, compression, translation.

Oracle / test infrastructure only (see package docstring).

Readings (the paper does not fix these):
  * FFT extents: n_i = the smallest power of two >= 2 K_i - 1.  This equals the
    paper's n_i = 2 K_i (Sec. II.B) whenever K_i is a power of two, which is the
    case in every workload the paper and the benchmark suite use; for other K_i
    it is the shortest power-of-two circulant embedding without wrap-around.
  * 3D format: each direction's T~_p (n1 x n2 x n3) is compressed on its own,
    with its own ranks.  4D format: T_4D[:, :, :, p] = T~_p (directions last,
    Sec. II.B) is compressed as one tensor.
  * The compressed translation restores T~_p (Sec. II.C, one direction at a
    time) and then applies Eq. 5 exactly as the plain translation does.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import decomp as D
from .directions import direction_grid
from .operator import fft_operator
from .translate import translate_field_fft


def embed_extent(K: int) -> int:
    n = 1
    while n < 2 * K - 1:
        n *= 2
    return max(n, 2)


@dataclass
class Plan:
    K: tuple              # (Kx, Ky, Kz) boxes
    a: float = 0.5        # box edge (wavelengths when k0 = 2 pi)
    k0: float = 2 * np.pi
    L: int = 5
    nphi_rule: str = "benchmark"
    near_rule: str = "chebyshev"
    prefactor: str = "unit"
    kappa: float = 4.0
    eps_r: complex = 1.0  # relative permittivity of the medium (Sec. III.A.5)

    @property
    def n(self):
        return tuple(embed_extent(k) for k in self.K)

    def directions(self):
        return direction_grid(self.L, self.nphi_rule)[0]

    @property
    def n_dir(self):
        return len(self.directions())


def operators(plan: Plan, dirs=None) -> list:
    """T~_p for the listed directions (default all): list of (n1, n2, n3) arrays."""
    kh = plan.directions()
    idx = range(len(kh)) if dirs is None else dirs
    return [fft_operator(kh[p], plan.K, plan.n, plan.a, plan.k0, plan.L,
                         plan.near_rule, plan.prefactor, plan.kappa, plan.eps_r) for p in idx]


def stack4d(Thats) -> np.ndarray:
    return np.stack(list(Thats), axis=3)


class Compressed:
    """A compressed operator store: `restore(p)` gives T~_p (Sec. II.C)."""

    def __init__(self, fmt: str, decomp: str, parts, shape):
        self.fmt, self.decomp, self.parts, self.shape = fmt, decomp, parts, shape

    # ---- restoration, one direction at a time -----------------------------
    def restore(self, p: int) -> np.ndarray:
        f, d, P = self.fmt, self.decomp, self.parts
        if d == "none":
            return P[p]
        if f == "3d" and d == "tucker":
            tk = P[p]
            return D.tucker3d_restore_steps(tk.core, *tk.factors)
        if f == "3d" and d == "tt":
            tt = P[p]
            return D.tt3d_restore_steps(tt.U1, tt.cores[0], tt.Ud)
        if f == "4d" and d == "tucker":
            tk = P
            core = D.tucker4d_core_for(tk.core, tk.factors[3], p)
            return D.tucker3d_restore_steps(core, *tk.factors[:3])
        if f == "4d" and d == "tt":
            tt = P
            return D.tt4d_restore_for(tt.U1, tt.cores[0], tt.cores[1], tt.Ud, p)
        if f == "4d" and d == "htucker":
            core = D.htucker_core_for(P, p)
            return D.tucker3d_restore_steps(core, *P.U[:3])
        raise ValueError((f, d))

    # ---- storage accounting (elements of the stored arrays) ---------------
    def elements(self) -> int:
        f, d, P = self.fmt, self.decomp, self.parts
        if d == "none":
            return sum(x.size for x in P)
        if f == "3d" and d == "tucker":
            return sum(t.core.size + sum(u.size for u in t.factors) for t in P)
        if f == "3d" and d == "tt":
            return sum(t.U1.size + t.cores[0].size + t.Ud.size for t in P)
        if d == "tucker":
            return P.core.size + sum(u.size for u in P.factors)
        if d == "tt":
            return P.U1.size + sum(c.size for c in P.cores) + P.Ud.size
        if d == "htucker":
            return sum(u.size for u in P.U) + P.C12.size + P.C34.size + P.B.size
        raise ValueError((f, d))

    def saving(self) -> float:
        """Memory saving 1 - compressed / original (Sec. III)."""
        return 1.0 - self.elements() / float(np.prod(self.shape))


def compress(Thats, fmt: str, decomp: str, tol: float, rule: str = "tail") -> Compressed:
    """Compress the FFT'ed operators in the 3D or 4D format (Sec. II.B)."""
    Thats = list(Thats)
    shape = Thats[0].shape + (len(Thats),)
    if decomp == "none":
        return Compressed("none", "none", Thats, shape)
    if fmt == "3d":
        if decomp == "tucker":
            return Compressed(fmt, decomp, [D.tucker_hosvd(T, tol, rule) for T in Thats], shape)
        if decomp == "tt":
            return Compressed(fmt, decomp, [D.tt_svd(T, tol, rule) for T in Thats], shape)
        raise ValueError(f"decomposition {decomp!r} has no 3D format")
    if fmt == "4d":
        T4 = stack4d(Thats)
        if decomp == "tucker":
            return Compressed(fmt, decomp, D.tucker_hosvd(T4, tol, rule), shape)
        if decomp == "tt":
            return Compressed(fmt, decomp, D.tt_svd(T4, tol, rule), shape)
        if decomp == "htucker":
            return Compressed(fmt, decomp, D.htucker_svd(T4, tol, rule), shape)
    raise ValueError((fmt, decomp))


def translate_with(restore, S_in: np.ndarray, dirs=None) -> np.ndarray:
    """Eq. 5 for every field; `restore(p)` supplies T~_p (restored one by one)."""
    n_dir = S_in.shape[0]
    idx = range(n_dir) if dirs is None else dirs
    out = np.zeros(S_in.shape, dtype=np.complex128)
    for p in idx:
        Th = restore(p)
        for pol in range(S_in.shape[1]):
            for r in range(S_in.shape[2]):
                out[p, pol, r] = translate_field_fft(Th, S_in[p, pol, r])
    return out


def translate_occupied(restore, S_in: np.ndarray, occupied: np.ndarray, dirs=None) -> np.ndarray:
    """Eq. 5 on a grid whose empty boxes hold no basis function (Sec. II.A):
    the aggregated field of an empty box is zero (A_v = 0) and no translated
    field is needed there.  `occupied` is a (Kz, Ky, Kx) boolean array; inputs
    at empty boxes are taken as zero and outputs there are zero."""
    m = np.asarray(occupied, dtype=bool)
    out = translate_with(restore, np.where(m, S_in, 0), dirs)
    return np.where(m, out, 0)


def relative_l2(x, ref) -> float:
    ref = np.asarray(ref)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(np.asarray(x) - ref) / (den if den > 0 else 1.0))

"""Tensor decompositions of the FFT'ed operators and their restorations (Sec. II.B-C).

Oracle / test infrastructure only (see package docstring).

Conventions
  * a mode product Y = X x_i M with M of shape (J, n_i) replaces mode i of X:
    Y[.., j, ..] = sum_k X[.., k, ..] M[j, k]                      (Eq. 10)
  * the mode-i unfolding puts mode i on the rows and the remaining modes, in
    their natural order (C order), on the columns;
  * truncation (reading of Alg. 1 step 7, Alg. 3 step 7 and Alg. 2 step 7):
    for a per-step tolerance delta (an absolute Frobenius-norm budget) keep the
    smallest rank r >= 1 whose discarded singular values satisfy
    sqrt(sum_{j > r} sigma_j^2) <= delta.  Tucker uses delta = gamma ||T|| / sqrt(d),
    TT uses gamma ||T|| / sqrt(d - 1), H-Tucker uses gamma ||T|| / sqrt(6) at
    each of its six non-root nodes.  Each rule bounds the total restoration
    error by gamma ||T||.  A "paper_sv" rule (cut where sigma_j / sigma_1 first
    drops below the per-step tolerance) is available for replication studies.

The SVD itself is numpy.linalg.svd (a library primitive).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


# --------------------------------------------------------------------------
# basic multilinear algebra
# --------------------------------------------------------------------------

def unfold(T: np.ndarray, mode: int) -> np.ndarray:
    """Mode-`mode` unfolding: shape (n_mode, prod of the other extents)."""
    return np.moveaxis(T, mode, 0).reshape(T.shape[mode], -1)


def mode_product(X: np.ndarray, M: np.ndarray, mode: int) -> np.ndarray:
    """X x_mode M (Eq. 10): contract mode `mode` of X with the columns of M."""
    Y = np.tensordot(M, X, axes=([1], [mode]))      # new axis first
    return np.moveaxis(Y, 0, mode)


def truncation_rank(s: np.ndarray, delta: float, rule: str = "tail") -> int:
    """Rank kept for singular values `s` (descending) at per-step budget `delta`."""
    s = np.asarray(s, dtype=np.float64)
    if s.size == 0:
        return 0
    if rule == "tail":
        # tail[r] = sqrt(sum_{j >= r} s_j^2): error when r values are kept
        tail = np.sqrt(np.cumsum((s * s)[::-1])[::-1])
        tail = np.append(tail, 0.0)
        ok = np.nonzero(tail <= delta)[0]
        r = int(ok[0]) if ok.size else s.size
        return max(r, 1)
    if rule == "paper_sv":
        # delta is relative here: first index whose normalised value is below it
        small = np.nonzero(s / s[0] < delta)[0]
        r = int(small[0]) if small.size else s.size
        return max(r, 1)
    raise ValueError(f"unknown truncation rule {rule!r}")


def _step_budget(normT: float, gamma: float, parts: float, rule: str) -> float:
    if rule == "tail":
        return gamma * normT / np.sqrt(parts)
    return gamma / np.sqrt(parts)


def truncated_left_basis(A: np.ndarray, delta: float, rule: str = "tail"):
    """Leading left singular vectors of A at budget delta; returns (U_r, s, r)."""
    U, s, _ = np.linalg.svd(A, full_matrices=False)
    r = truncation_rank(s, delta, rule)
    return U[:, :r], s, r


# --------------------------------------------------------------------------
# Tucker (HOSVD, Alg. 1) and its restorations (Fig. 3(a), 3(b))
# --------------------------------------------------------------------------

@dataclass
class Tucker:
    core: np.ndarray                 # r1 x ... x rd
    factors: list                    # U^i, n_i x r_i
    sigmas: list = field(default_factory=list)   # full singular values per mode

    @property
    def ranks(self):
        return tuple(self.core.shape)


def tucker_hosvd(T: np.ndarray, gamma: float, rule: str = "tail") -> Tucker:
    """Tucker-SVD (Alg. 1): factors from the SVDs of the unfoldings of T itself,
    core C = T x_1 U^1* ... x_d U^d* (U* = conjugate transpose)."""
    d = T.ndim
    normT = float(np.linalg.norm(T))
    delta = _step_budget(normT, gamma, d, rule)
    C = np.array(T, dtype=np.complex128, copy=True)
    factors, sig = [], []
    for i in range(d):
        U, s, _ = truncated_left_basis(unfold(T, i), delta, rule)
        factors.append(U)
        sig.append(s)
        C = mode_product(C, U.conj().T, i)
    return Tucker(C, factors, sig)


def tucker_restore(tk: Tucker) -> np.ndarray:
    """C x_1 U^1 x_2 U^2 ... x_d U^d (Eqs. 8, 9)."""
    X = tk.core
    for i, U in enumerate(tk.factors):
        X = mode_product(X, U, i)
    return X


def tucker3d_restore_steps(core: np.ndarray, U1, U2, U3) -> np.ndarray:
    """Tucker-3D restoration as the matrix steps of Fig. 3(a).

    Step 1: the core, as an r1 x (r2 r3) matrix, is multiplied by U^1.
    Step 2: the result, reshaped with mode 2 on the rows, is multiplied by U^2.
    Step 3: reshaped with mode 3 on the rows, multiplied by U^3.
    Finally the matrix is put back into n1 x n2 x n3 order.
    """
    r1, r2, r3 = core.shape
    n1, n2, n3 = U1.shape[0], U2.shape[0], U3.shape[0]
    X = U1 @ core.reshape(r1, r2 * r3)                               # n1 x (r2 r3)
    X = X.reshape(n1, r2, r3).transpose(1, 0, 2).reshape(r2, n1 * r3)
    X = U2 @ X                                                        # n2 x (n1 r3)
    X = X.reshape(n2, n1, r3).transpose(2, 1, 0).reshape(r3, n1 * n2)
    X = U3 @ X                                                        # n3 x (n1 n2)
    return X.reshape(n3, n1, n2).transpose(1, 2, 0)


def tucker4d_core_for(core4: np.ndarray, U4: np.ndarray, p: int) -> np.ndarray:
    """Fig. 3(b): the 4D core as an (r1 r2 r3) x r4 matrix times row p of U^4."""
    r1, r2, r3, r4 = core4.shape
    return (core4.reshape(r1 * r2 * r3, r4) @ U4[p, :]).reshape(r1, r2, r3)


# --------------------------------------------------------------------------
# TT (TT-SVD, Alg. 3) and its restorations (Fig. 4)
# --------------------------------------------------------------------------

@dataclass
class TensorTrain:
    U1: np.ndarray          # n1 x r1
    cores: list             # C^i, r_i x n_{i+1} x r_{i+1}, i = 1 .. d-2
    Ud: np.ndarray          # n_d x r_{d-1}  (called U^3_TT in Eqs. 13, 14)
    sigmas: list = field(default_factory=list)

    @property
    def ranks(self):
        return (self.U1.shape[1],) + tuple(c.shape[2] for c in self.cores)


def tt_svd(T: np.ndarray, gamma: float, rule: str = "tail") -> TensorTrain:
    """TT-SVD (Alg. 3): sequential SVDs of reshaped remainders.

    C starts as T reshaped to n1 x (n2 ... nd).  At step i it is reshaped to
    (r_{i-1} n_i) x (n_{i+1} ... n_d), its left singular vectors (truncated)
    become core i (r_{i-1} x n_i x r_i) and C <- Sigma V* carries on.  The last
    remainder (r_{d-1} x n_d) is stored transposed as the n_d x r_{d-1} factor
    so that Eqs. 13/14 rebuild T with a mode-d product.
    """
    d = T.ndim
    n = T.shape
    normT = float(np.linalg.norm(T))
    delta = _step_budget(normT, gamma, d - 1, rule)
    C = np.asarray(T, dtype=np.complex128).reshape(n[0], -1)
    r_prev = 1
    raw_cores, sig = [], []
    for i in range(d - 1):
        C = C.reshape(r_prev * n[i], -1)
        U, s, Vh = np.linalg.svd(C, full_matrices=False)
        r = truncation_rank(s, delta, rule)
        raw_cores.append(U[:, :r].reshape(r_prev, n[i], r))
        sig.append(s)
        C = s[:r, None] * Vh[:r, :]
        r_prev = r
    U1 = raw_cores[0].reshape(n[0], -1)
    return TensorTrain(U1, raw_cores[1:], np.ascontiguousarray(C.T), sig)


def tt_restore(tt: TensorTrain) -> np.ndarray:
    """Contract the train U1 - C^1 - ... - U_d^T back into the full tensor."""
    X = tt.U1                                        # n1 x r1
    shape = [tt.U1.shape[0]]
    for c in tt.cores:
        r, m, r2 = c.shape
        X = X @ c.reshape(r, m * r2)                 # (prod) x (m r2)
        shape.append(m)
        X = X.reshape(-1, r2)
    X = X @ tt.Ud.T                                  # (prod) x n_d
    shape.append(tt.Ud.shape[0])
    return X.reshape(shape)


def tt3d_restore_steps(U1, C1, U3) -> np.ndarray:
    """Fig. 4(a): T1 = U^1 mat(C^1) (n1 x n2 r2), reshape to (n1 n2) x r2, times U^3^T."""
    r1, n2, r2 = C1.shape
    n1, n3 = U1.shape[0], U3.shape[0]
    T1 = (U1 @ C1.reshape(r1, n2 * r2)).reshape(n1 * n2, r2)
    return (T1 @ U3.T).reshape(n1, n2, n3)


def tt4d_slice_for(C2: np.ndarray, U3: np.ndarray, p: int) -> np.ndarray:
    """Fig. 4(b) steps 1-2: column p of mat(C^2) U^3^T, reshaped r2 x n3."""
    r2, n3, r3 = C2.shape
    T2 = C2.reshape(r2 * n3, r3) @ U3.T             # (r2 n3) x n4
    return T2[:, p].reshape(r2, n3)


def tt4d_restore_for(U1, C1, C2, U3, p: int) -> np.ndarray:
    """Fig. 4(b): T_p = T1 . S_p with T1 from Fig. 4(a) step 1."""
    r1, n2, r2 = C1.shape
    n1 = U1.shape[0]
    n3 = C2.shape[1]
    T1 = (U1 @ C1.reshape(r1, n2 * r2)).reshape(n1 * n2, r2)
    return (T1 @ tt4d_slice_for(C2, U3, p)).reshape(n1, n2, n3)


# --------------------------------------------------------------------------
# H-Tucker (Alg. 2, balanced tree {1,2},{3,4}) and its restoration (Fig. 3(c))
# --------------------------------------------------------------------------

@dataclass
class HTucker:
    U: list                 # leaf bases U^i, n_i x r_i
    C12: np.ndarray         # r1 x r2 x r12
    C34: np.ndarray         # r3 x r4 x r34
    B: np.ndarray           # r12 x r34 transfer matrix
    sigmas: list = field(default_factory=list)

    @property
    def ranks(self):
        return tuple(u.shape[1] for u in self.U) + (self.C12.shape[2], self.C34.shape[2])


def htucker_svd(T4: np.ndarray, gamma: float, rule: str = "tail") -> HTucker:
    """H-Tucker-SVD (Alg. 2) for a 4D tensor.

    Leaves: left singular bases of the four unfoldings of T (Alg. 1 step).
    W = T x_1 U^1* x_2 U^2* x_3 U^3* x_4 U^4* (the projected core).
    Node {1,2}: left singular vectors of W12 = W as (r1 r2) x (r3 r4).
    Node {3,4}: left singular vectors of W34 = W12^T.
    Root transfer matrix B = C12* W12 conj(C34), so that W ~ C12 B C34^T.
    All six non-root truncations use the budget gamma ||T|| / sqrt(6).
    """
    assert T4.ndim == 4
    normT = float(np.linalg.norm(T4))
    delta = _step_budget(normT, gamma, 6, rule)
    U, sig = [], []
    W = np.asarray(T4, dtype=np.complex128)
    for i in range(4):
        Ui, s, _ = truncated_left_basis(unfold(T4, i), delta, rule)
        U.append(Ui)
        sig.append(s)
    for i in range(4):
        W = mode_product(W, U[i].conj().T, i)
    r1, r2, r3, r4 = W.shape
    W12 = W.reshape(r1 * r2, r3 * r4)
    C12, s12, r12 = truncated_left_basis(W12, delta, rule)
    C34, s34, r34 = truncated_left_basis(W12.T, delta, rule)
    sig += [s12, s34]
    B = C12.conj().T @ W12 @ C34.conj()
    return HTucker(U, C12.reshape(r1, r2, r12), C34.reshape(r3, r4, r34), B, sig)


def htucker_core_for(ht: HTucker, p: int) -> np.ndarray:
    """Fig. 3(c): the 3D core of direction p.

    M = C34 contracted with row p of U^4 over its r4 index (r3 x r34);
    M B^T (r3 x r12); contracted with C12 over r12 gives the r1 x r2 x r3 core.
    """
    r3, r4, r34 = ht.C34.shape
    M = np.einsum("klt,l->kt", ht.C34, ht.U[3][p, :])
    MB = M @ ht.B.T                                   # r3 x r12
    return np.einsum("ijs,ks->ijk", ht.C12, MB)


def htucker_restore(ht: HTucker) -> np.ndarray:
    W = np.einsum("ijs,st,klt->ijkl", ht.C12, ht.B, ht.C34)
    for i in range(4):
        W = mode_product(W, ht.U[i], i)
    return W

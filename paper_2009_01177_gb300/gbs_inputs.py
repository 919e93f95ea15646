"""Seeded synthetic lossy-GBS inputs (covariance matrices and click patterns).

This module only builds inputs.  It holds none of the Torontonian's
arithmetic and is the one piece of code that both the CUDA path's callers and
the CPU oracle's callers share.

Conventions (paper Sec. 3.1, Eq. 1):
  * xxpp ordering: for M modes, index j is x_j and M + j is p_j.
  * hbar = 1: the vacuum covariance is sigma = I/2.  The matrix of Eq. 1 is
    Sigma = sigma + I/2 (vacuum -> Sigma = I), and the sampling matrix is
    O = I - Sigma^-1 (the paper's A), symmetrised.
  * A click pattern S selects row/col j and M + j of O for each clicked mode
    j (selection rule under Eq. 1), giving the 2k x 2k matrix O_S in xxpp
    order: x_{s1..sk} then p_{s1..sk}.

State recipe: a Haar-random M x M unitary U (QR of a complex Ginibre matrix
with the phases of R's diagonal removed), single-mode squeezing r_i drawn
uniformly from [r_lo, r_hi], the squeezed vacuum
sigma0 = diag(e^{-2r}, e^{2r}) / 2, the interferometer
S_U = [[Re U, -Im U], [Im U, Re U]], and uniform transmission eta:
sigma = eta S_U sigma0 S_U^T + (1 - eta)/2 I.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class GBSState:
    M: int
    r: np.ndarray          # (M,) squeezing parameters
    eta: float             # uniform transmission
    U: np.ndarray          # (M, M) complex unitary
    Sigma: np.ndarray      # (2M, 2M) xxpp, Sigma = sigma + I/2
    O: np.ndarray          # (2M, 2M) xxpp, O = I - Sigma^-1


def haar_unitary(M: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random unitary (QR of a complex Ginibre matrix, phase-fixed)."""
    z = (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


def lossy_gbs_state(M: int, r_lo: float, r_hi: float, eta: float, seed: int,
                    U: np.ndarray | None = None, r: np.ndarray | None = None) -> GBSState:
    """Lossy squeezed-light GBS state; see the module docstring for the recipe."""
    rng = np.random.default_rng(seed)
    if U is None:
        U = haar_unitary(M, rng)
    if r is None:
        r = rng.uniform(r_lo, r_hi, size=M)
    r = np.asarray(r, dtype=np.float64)
    sigma0 = 0.5 * np.diag(np.concatenate([np.exp(-2.0 * r), np.exp(2.0 * r)]))
    SU = np.block([[U.real, -U.imag], [U.imag, U.real]])
    sigma = eta * SU @ sigma0 @ SU.T + 0.5 * (1.0 - eta) * np.eye(2 * M)
    sigma = 0.5 * (sigma + sigma.T)
    Sigma = sigma + 0.5 * np.eye(2 * M)
    O = np.eye(2 * M) - np.linalg.inv(Sigma)
    O = 0.5 * (O + O.T)
    return GBSState(M=M, r=r, eta=float(eta), U=U, Sigma=Sigma, O=O)


def random_pattern(M: int, k: int, seed: int) -> np.ndarray:
    """Sorted indices of k distinct clicked modes out of M."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(M, size=k, replace=False))


def select(O: np.ndarray, modes) -> np.ndarray:
    """O_S of Eq. 1: rows/cols j and M + j for each clicked mode j (xxpp)."""
    M = O.shape[0] // 2
    modes = np.asarray(modes, dtype=np.int64)
    idx = np.concatenate([modes, M + modes])
    return np.ascontiguousarray(O[np.ix_(idx, idx)])


def thermal_O(k: int, a: float) -> np.ndarray:
    """O = a I_{2k}: the 'diagonal' matrix of the paper's bound analysis."""
    return a * np.eye(2 * k)


def block_diag_modes(O1: np.ndarray, O2: np.ndarray) -> np.ndarray:
    """Mode-wise direct sum of two xxpp matrices (k1 + k2 modes, xxpp)."""
    k1, k2 = O1.shape[0] // 2, O2.shape[0] // 2
    k = k1 + k2
    O = np.zeros((2 * k, 2 * k))
    i1 = np.concatenate([np.arange(k1), k + np.arange(k1)])
    i2 = np.concatenate([k1 + np.arange(k2), k + k1 + np.arange(k2)])
    O[np.ix_(i1, i1)] = O1
    O[np.ix_(i2, i2)] = O2
    return O


# The workloads, by what they are.  Each returns (state, pattern, O_S).
def workload_m16_k10(seed: int = 1):
    """M = 16, r ~ U[0.5, 1.0], eta = 0.5; a random 10-click pattern."""
    st = lossy_gbs_state(16, 0.5, 1.0, 0.5, seed)
    pat = random_pattern(16, 10, seed + 1000)
    return st, pat, select(st.O, pat)


def workload_m100(k: int, seed: int = 2, r_lo: float = 0.6, r_hi: float = 1.2, eta: float = 0.3,
                  pattern_seed: int | None = None):
    """M = 100 lossy state (default r ~ U[0.6, 1.2], eta = 0.3); a random k-click pattern."""
    st = lossy_gbs_state(100, r_lo, r_hi, eta, seed)
    pat = random_pattern(100, k, seed + 1000 if pattern_seed is None else pattern_seed)
    return st, pat, select(st.O, pat)


def nested_patterns(pattern: np.ndarray, ks) -> list:
    """Leading sub-patterns of one click pattern (same state, fewer clicks)."""
    return [np.asarray(pattern[:k]) for k in ks]


def batch_patterns(M: int, n: int, k_lo: int, k_hi: int, seed: int) -> list:
    """n click patterns with click counts spread over [k_lo, k_hi].

    Click counts are drawn from a binomial-shaped law centred in the range
    (the shape a sampler of a moderately bright state produces), clipped to
    [k_lo, k_hi]; modes are uniform without replacement.
    """
    rng = np.random.default_rng(seed)
    mid = 0.5 * (k_lo + k_hi)
    span = k_hi - k_lo
    ks = np.clip(np.rint(rng.normal(mid, span / 4.0, size=n)), k_lo, k_hi).astype(int)
    return [np.sort(rng.choice(M, size=int(k), replace=False)) for k in ks]

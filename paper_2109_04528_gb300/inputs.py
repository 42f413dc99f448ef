"""Seeded synthetic inputs for Torontonian evaluation.

This module builds the sampling matrix O = I - Sigma^{-1} (Eq. A of the paper,
Sec. 1) from the complex Husimi covariance Sigma of squeezed vacua sent through
a lossy interferometer.  It holds no Torontonian arithmetic: no subset sums,
no determinants of submatrices, no factor updates.  Both the CUDA path and the
CPU oracle consume what it returns, so it is the one module they share.

Conventions
-----------
* Block layout (default): rows/cols ordered (a_1..a_n, a_1^dag..a_n^dag), so
  mode j owns rows {j, j+n}.
* Pairs layout: rows/cols ordered (a_1, a_1^dag, a_2, a_2^dag, ...), the order
  the paper uses for its recursion (Sec. 2); mode j owns rows {2j, 2j+1}.
* Squeezing phase: input mode j has <a_j a_j> = +sinh(r_j) cosh(r_j) and
  <a_j^dag a_j> = sinh(r_j)^2.  With b = T a (T = diag(sqrt(eta)) U) the output
  moments are N = conj(T) diag(sinh^2 r) T^T (N_ik = <b_i^dag b_k>) and
  M = T diag(sinh r cosh r) T^T (M_ik = <b_i b_k>); loss adds vacuum, which
  leaves normally ordered moments unchanged.  Then
  Sigma = [[N^T + I, M], [conj(M), N + I]].
* Haar unitaries: QR of a complex Gaussian matrix with the phases of R's
  diagonal moved into Q (Mezzadri, "How to generate random matrices from the
  classical compact groups", Notices AMS 54 (2007)).

Random numbers come from numpy's PCG64 generator, whose streams are the same
on every platform.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BLOCK = 0
PAIRS = 1


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def haar_unitary(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random n x n unitary (Mezzadri's phase-fixed QR)."""
    if n == 0:
        return np.zeros((0, 0), dtype=np.complex128)
    g = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    q, r = np.linalg.qr(g)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


def husimi_covariance(r: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Sigma for squeezed vacua with squeezing r sent through transfer matrix T."""
    r = np.asarray(r, dtype=np.float64)
    n = T.shape[0]
    sh = np.sinh(r)
    ch = np.cosh(r)
    N = T.conj() @ np.diag(sh * sh) @ T.T
    M = T @ np.diag(sh * ch) @ T.T
    I = np.eye(n)
    S = np.zeros((2 * n, 2 * n), dtype=np.complex128)
    S[:n, :n] = N.T + I
    S[:n, n:] = M
    S[n:, :n] = M.conj()
    S[n:, n:] = N + I
    return S


def sampling_matrix(sigma: np.ndarray) -> np.ndarray:
    """O = I - Sigma^{-1} (Eq. A) in complex128, projected exactly onto the form
    every Gaussian state's O has in block layout,
        O = [[P, Q], [conj(Q), conj(P)]],  P Hermitian, Q symmetric,
    which also makes O exactly Hermitian.  The projection moves O by about the
    rounding of the inverse; it removes that rounding's asymmetry so that the
    structure (and with it the real (x, p) form) holds exactly."""
    m = sigma.shape[0]
    n = m // 2
    O = np.eye(m) - np.linalg.inv(sigma)
    W = O[:n, :n] + O[n:, n:].conj()  # ~ 2 P
    S = O[:n, n:] + O[n:, :n].conj()  # ~ 2 Q
    P = 0.25 * (W + W.conj().T)       # exactly Hermitian (sums commute, 0.25 is exact)
    Q = 0.25 * (S + S.T)              # exactly symmetric
    out = np.empty_like(O)
    out[:n, :n] = P
    out[:n, n:] = Q
    out[n:, :n] = Q.conj()
    out[n:, n:] = P.conj()
    return out


@dataclass
class Instance:
    """One synthetic input: O in block layout plus how it was made."""
    O: np.ndarray
    n: int
    kind: str
    seed: int
    r: np.ndarray = field(default_factory=lambda: np.zeros(0))
    eta: np.ndarray = field(default_factory=lambda: np.zeros(0))
    sigma: np.ndarray | None = None

    def params(self) -> dict:
        return {"kind": self.kind, "n": self.n, "seed": self.seed}


def lossy_squeezed(n: int, seed: int, r_range=(0.3, 0.8), eta=0.5) -> Instance:
    """n squeezed vacua, r_j ~ U[r_range], through a Haar unitary, then loss.

    ``eta`` is either a scalar (uniform transmission) or a (lo, hi) range from
    which one transmission per output mode is drawn: T = diag(sqrt(eta_j)) U.
    """
    rng = rng_for(seed)
    r = rng.uniform(r_range[0], r_range[1], size=n)
    U = haar_unitary(n, rng)
    if np.ndim(eta) == 0:
        etas = np.full(n, float(eta))
    else:
        etas = rng.uniform(eta[0], eta[1], size=n)
    T = np.sqrt(etas)[:, None] * U
    sigma = husimi_covariance(r, T)
    return Instance(sampling_matrix(sigma), n, "lossy_squeezed", seed, r, etas, sigma)


def product_state(n: int, seed: int, r_range=(0.3, 0.8), eta_range=(0.3, 0.7)) -> Instance:
    """Independent lossy single-mode squeezed vacua (U = I): block-diagonal over modes."""
    rng = rng_for(seed)
    r = rng.uniform(r_range[0], r_range[1], size=n)
    etas = rng.uniform(eta_range[0], eta_range[1], size=n)
    T = np.diag(np.sqrt(etas)).astype(np.complex128)
    sigma = husimi_covariance(r, T)
    return Instance(sampling_matrix(sigma), n, "product_state", seed, r, etas, sigma)


def two_mode_squeezed_vacuum(r: float) -> Instance:
    """TMSV: squeezers (r, -r) on a 50:50 beam splitter; N = sinh^2 r I, M = sinh r cosh r X."""
    sh, ch = np.sinh(r), np.cosh(r)
    N = np.eye(2) * sh * sh
    M = np.array([[0.0, 1.0], [1.0, 0.0]]) * sh * ch
    I = np.eye(2)
    S = np.zeros((4, 4), dtype=np.complex128)
    S[:2, :2] = N.T + I
    S[:2, 2:] = M
    S[2:, :2] = M.conj()
    S[2:, 2:] = N + I
    return Instance(sampling_matrix(S), 2, "tmsv", 0, np.array([r, r]), np.ones(2), S)


def vacuum(n: int) -> Instance:
    return Instance(np.zeros((2 * n, 2 * n), dtype=np.complex128), n, "vacuum", 0)


def random_hermitian_contraction(n: int, seed: int, scale: float = 0.9) -> Instance:
    """A Hermitian O with I - O positive definite and no (a, a^dag) block structure.

    O = I - W W^H / ||.|| style: eigenvalues of O drawn in (-scale, scale), so
    I - O has eigenvalues in (1 - scale, 1 + scale).  Used to exercise the
    general complex path on inputs that are not physical covariances.
    """
    rng = rng_for(seed)
    m = 2 * n
    Q = haar_unitary(m, rng)
    ev = rng.uniform(-scale, scale, size=m)
    O = (Q * ev[None, :]) @ Q.conj().T
    O = 0.5 * (O + O.conj().T)
    return Instance(O, n, "random_hermitian", seed)


def mode_indices(n: int, modes, layout: int = BLOCK) -> np.ndarray:
    """Row indices of the given modes (ascending mode order, a before a^dag)."""
    modes = list(modes)
    if layout == BLOCK:
        return np.array([j for j in modes] + [j + n for j in modes], dtype=np.int64)
    return np.array([2 * j + c for j in modes for c in (0, 1)], dtype=np.int64)


def submatrix(O: np.ndarray, modes, layout: int = BLOCK) -> np.ndarray:
    """O_S: keep each selected mode together with its conjugate (block layout in and out)."""
    n = O.shape[0] // 2
    idx = mode_indices(n, sorted(modes), layout)
    return O[np.ix_(idx, idx)].copy()


def to_pairs(O: np.ndarray) -> np.ndarray:
    """Block layout -> pairs layout (same matrix, rows and columns permuted together)."""
    n = O.shape[0] // 2
    perm = np.array([j + c * n for j in range(n) for c in (0, 1)], dtype=np.int64)
    return O[np.ix_(perm, perm)].copy()


def permute_modes(O: np.ndarray, perm) -> np.ndarray:
    """Relabel modes (block layout): new mode k is old mode perm[k]."""
    n = O.shape[0] // 2
    perm = np.asarray(perm, dtype=np.int64)
    idx = np.concatenate([perm, perm + n])
    return O[np.ix_(idx, idx)].copy()


def local_phase(O: np.ndarray, theta) -> np.ndarray:
    """O -> D O D^H with D = diag(e^{i theta_j} on a_j, e^{-i theta_j} on a_j^dag)."""
    theta = np.asarray(theta, dtype=np.float64)
    d = np.concatenate([np.exp(1j * theta), np.exp(-1j * theta)])
    return (d[:, None] * O) * d.conj()[None, :]


# --- workload recipes (sizes and distributions of the benchmark configurations) ---

SEED_BASE = 2109045280


def config_single(n: int, seed: int | None = None, eta=(0.3, 0.7)) -> Instance:
    """Lossy squeezed state, r ~ U[0.3, 0.8], per-mode eta ~ U[0.3, 0.7]."""
    return lossy_squeezed(n, SEED_BASE + 1000 + n if seed is None else seed, (0.3, 0.8), eta)


def config_n8(seed: int | None = None) -> Instance:
    """n = 8, r ~ U[0.3, 0.8], uniform eta = 0.5 (the 256-subset worked case)."""
    return lossy_squeezed(8, SEED_BASE if seed is None else seed, (0.3, 0.8), 0.5)


def click_pattern_batch(n_total: int, count: int, kmin: int, kmax: int, seed: int,
                        r_range=(0.5, 1.2), eta=0.4):
    """`count` submatrices O_S of one n_total-mode lossy squeezed state.

    Each S is a seeded k-subset of the modes with k ~ U{kmin..kmax}.
    Returns (parent Instance, list of mode lists, list of O_S).
    """
    parent = lossy_squeezed(n_total, seed, r_range, eta)
    rng = rng_for(seed + 7)
    pats, mats = [], []
    for _ in range(count):
        k = int(rng.integers(kmin, kmax + 1))
        S = np.sort(rng.choice(n_total, size=k, replace=False))
        pats.append(S.tolist())
        mats.append(submatrix(parent.O, S))
    return parent, pats, mats

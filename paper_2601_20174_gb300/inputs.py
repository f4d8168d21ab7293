"""Seeded synthetic inputs for the two-level PCG path (host side, numpy).

This module is the single source of random and structured inputs for both the
CUDA path and the FP64 oracle.  It holds no solver arithmetic: it produces the
cell diffusion coefficients of the PDE families, right-hand sides and the random
test vectors S^(0) that the method draws (Sec. 3 "Near-Nullspace Vectors";
Algorithm 1 input), and nothing else.  It imports neither the oracle nor the
CUDA binding.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the
i-th draw of stream s under seed q is the SplitMix64 output number i+1 of a
generator whose state starts at base(q, s).  Uniforms take the top 53 bits;
normals use the Box-Muller transform on consecutive uniform pairs.

Grid conventions (shared with the operator definitions):
  * 2D: N x N interior nodes of the unit square, h = 1/(N+1), node (i, j) at
    ((i+1)h, (j+1)h), flattened as j*N + i (x fastest).  Homogeneous Dirichlet
    boundary nodes are eliminated.  Cells are the (N+1) x (N+1) squares of side
    h; cell (ci, cj) has centre ((ci+1/2)h, (cj+1/2)h), array index [cj, ci].
  * 3D: N^3 interior nodes, flattened (l*N + j)*N + i; (N+1)^3 cells indexed
    [cl, cj, ci].
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = 0xD1B54A32D192ED03
_MASK64 = (1 << 64) - 1

# Named streams so that independent inputs of one instance never share draws.
STREAM_KAPPA = 1
STREAM_RHS = 2
STREAM_S0 = 3
STREAM_THETA = 4
STREAM_SIZES = 5
STREAM_NOISE = 6
STREAM_DIRECTION = 7
STREAM_SKETCH = 11  # Gaussian sketch of the randomised SVD (same number as the library's)


def _fin(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser (xor-shift-multiply), on uint64 arrays."""
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_base(seed: int, stream: int) -> int:
    """Starting state of stream `stream` under `seed` (a 64-bit integer)."""
    v = (int(seed) ^ ((int(stream) * _STREAM_MUL) & _MASK64)) & _MASK64
    with np.errstate(over="ignore"):
        return int(_fin(np.array([v], dtype=np.uint64) + _GOLDEN)[0])


def splitmix64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of one stream, as uint64."""
    base = np.uint64(stream_base(seed, stream))
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _fin(base + idx * _GOLDEN)


def uniform(seed: int, stream: int, count: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """`count` uniforms in [lo, hi) from the top 53 bits of each draw."""
    u = (splitmix64(seed, stream, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """`count` standard normals by Box-Muller on uniform pairs (2j, 2j+1)."""
    pairs = (count + 1) // 2
    u = (splitmix64(seed, stream, 2 * pairs) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    u1, u2 = u[0::2], u[1::2]
    rad = np.sqrt(-2.0 * np.log1p(-u1))
    out = np.empty(2 * pairs)
    out[0::2] = rad * np.cos(2.0 * math.pi * u2)
    out[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return out[:count]


# ----------------------------------------------------------------------------
# Coefficient fields (the PDE families of the benchmark configurations)
# ----------------------------------------------------------------------------

def grf_log_kappa_2d(N: int, seed: int, length: float = 0.1, sigma: float = 1.0) -> np.ndarray:
    """Gaussian random field on the (N+1)^2 cell centres, squared-exponential
    covariance C(x, y) = sigma^2 exp(-|x-y|^2 / (2 length^2)).

    The covariance is separable, C = C1 (x) C1, so G = L1 Z L1^T with L1 the
    symmetric square root of the 1D covariance C1 (eigenvalues clamped at 0)
    and Z i.i.d. N(0, 1).  Returns log kappa as an (N+1, N+1) array [cj, ci].
    """
    m = N + 1
    h = 1.0 / m
    c = (np.arange(m) + 0.5) * h
    d2 = (c[:, None] - c[None, :]) ** 2
    c1 = sigma * np.exp(-d2 / (2.0 * length * length))  # sigma^2 split over the two factors
    w, v = np.linalg.eigh(c1)
    w = np.clip(w, 0.0, None)
    l1 = (v * np.sqrt(w)) @ v.T
    z = normal(seed, STREAM_KAPPA, m * m).reshape(m, m)
    return l1 @ z @ l1.T


def iid_log_kappa(shape: tuple[int, ...], seed: int, sigma: float = 1.0) -> np.ndarray:
    """log kappa i.i.d. N(0, sigma^2) per cell."""
    return sigma * normal(seed, STREAM_KAPPA, int(np.prod(shape))).reshape(shape)


def rotated_aniso_tensor(theta: float, eps: float) -> np.ndarray:
    """Constant diffusion tensor K = R(theta) diag(1, eps) R(theta)^T as
    [a_xx, a_yy, a_xy] (Appendix, anisotropic family, with the per-instance
    angle and ratio of the 9-point configuration)."""
    c, s = math.cos(theta), math.sin(theta)
    axx = c * c + eps * s * s
    ayy = s * s + eps * c * c
    axy = (1.0 - eps) * c * s
    return np.array([axx, ayy, axy], dtype=np.float64)


def rhs_uniform(n: int, m: int, seed: int) -> np.ndarray:
    """Right-hand sides f ~ U[-1, 1], column-major n x m (m columns)."""
    return uniform(seed, STREAM_RHS, n * m, -1.0, 1.0).reshape(m, n).T.copy()


def sketch_normal(K: int, l: int, seed: int) -> np.ndarray:
    """Gaussian sketch Omega ~ N(0, 1), K x l (column j = draws j*K ..)."""
    return normal(seed, STREAM_SKETCH, K * l).reshape(l, K).T.copy()


def samples_normal(n: int, K: int, seed: int) -> np.ndarray:
    """Random test vectors S^(0) ~ N(0, 1), n x K (column j = draws j*n..)."""
    return normal(seed, STREAM_S0, n * K).reshape(K, n).T.copy()


# ----------------------------------------------------------------------------
# Problem descriptions
# ----------------------------------------------------------------------------

LAYOUT_CELL_KAPPA = 0     # coeffs = cell-centred kappa, (N+1)^dim values
LAYOUT_CONST_TENSOR = 1   # coeffs = constant tensor: 2D [axx, ayy, axy]


@dataclasses.dataclass
class Problem:
    """One SPD stencil system plus its setup parameters.

    coeffs is either cell kappa (layout 0; shape (N+1,)*dim, C order, x last)
    or a constant tensor (layout 1).  f is n x m column-major, S0 is n x K.
    """
    name: str
    dim: int
    N: int
    points: int
    layout: int
    coeffs: np.ndarray
    k: int
    K: int
    s1: int = 20
    omega: float = 2.0 / 3.0
    nu: int = 2
    tol: float = 1e-8
    m: int = 1
    seed: int = 0
    f: np.ndarray | None = None
    S0: np.ndarray | None = None

    @property
    def n(self) -> int:
        return self.N ** self.dim

    @property
    def grid(self) -> tuple[int, int, int]:
        return (self.N, self.N, self.N if self.dim == 3 else 1)


def _finish(p: Problem, with_samples: bool = True) -> Problem:
    p.f = rhs_uniform(p.n, p.m, p.seed)
    if with_samples:
        p.S0 = samples_normal(p.n, p.K, p.seed)
    return p


def poisson_2d(N: int = 32, k: int = 16, K: int = 64, seed: int = 0, tol: float = 1e-10,
               with_samples: bool = True) -> Problem:
    """Constant-coefficient Poisson, 5-point, N x N interior grid (kappa = 1)."""
    p = Problem("poisson2d", 2, N, 5, LAYOUT_CELL_KAPPA, np.ones((N + 1, N + 1)), k, K,
                tol=tol, seed=seed)
    return _finish(p, with_samples)


def grf_diffusion_2d(N: int = 512, k: int = 64, K: int = 128, seed: int = 0, tol: float = 1e-8,
                     with_samples: bool = True) -> Problem:
    """Variable-coefficient diffusion, 5-point, log kappa a squared-exponential
    Gaussian random field (length 0.1, sigma 1)."""
    kap = np.exp(grf_log_kappa_2d(N, seed))
    p = Problem("grf_diffusion2d", 2, N, 5, LAYOUT_CELL_KAPPA, kap, k, K, tol=tol, seed=seed)
    return _finish(p, with_samples)


def iid_diffusion_2d(N: int, k: int, K: int | None = None, seed: int = 0, tol: float = 1e-8,
                     with_samples: bool = True) -> Problem:
    """Variable-coefficient diffusion, 5-point, log kappa i.i.d. N(0,1) per cell."""
    kap = np.exp(iid_log_kappa((N + 1, N + 1), seed))
    p = Problem("iid_diffusion2d", 2, N, 5, LAYOUT_CELL_KAPPA, kap, k, K or 2 * k, tol=tol, seed=seed)
    return _finish(p, with_samples)


def aniso_9pt_2d(N: int = 1024, k: int = 128, K: int = 256, m: int = 32, seed: int = 0,
                 eps: float = 1e-3, tol: float = 1e-8, with_samples: bool = True) -> Problem:
    """Rotated anisotropic diffusion, 9-point, theta ~ U[0, pi) per instance."""
    theta = float(uniform(seed, STREAM_THETA, 1, 0.0, math.pi)[0])
    p = Problem("aniso9pt2d", 2, N, 9, LAYOUT_CONST_TENSOR, rotated_aniso_tensor(theta, eps),
                k, K, tol=tol, m=m, seed=seed)
    return _finish(p, with_samples)


def iid_diffusion_3d(N: int = 64, k: int = 64, K: int = 128, seed: int = 0, tol: float = 1e-8,
                     with_samples: bool = True) -> Problem:
    """3D variable-coefficient diffusion, 7-point, log kappa i.i.d. N(0,1) per cell."""
    kap = np.exp(iid_log_kappa((N + 1, N + 1, N + 1), seed))
    p = Problem("iid_diffusion3d", 3, N, 7, LAYOUT_CELL_KAPPA, kap, k, K, tol=tol, seed=seed)
    return _finish(p, with_samples)


BATCH_SIDES = (64, 128, 192, 256, 384, 512)
BATCH_RANKS = (16, 32, 64)


def batch_instances(count: int = 256, seed: int = 0, sides=BATCH_SIDES, ranks=BATCH_RANKS,
                    tol: float = 1e-8, with_samples: bool = True) -> list[Problem]:
    """Uneven batch: side ~ U(sides), rank ~ U(ranks), K = 2k, log kappa i.i.d.
    N(0, 1) per cell; instance i uses seed (seed, i) folded into one integer."""
    draws = splitmix64(seed, STREAM_SIZES, 2 * count)
    out = []
    for i in range(count):
        N = sides[int(draws[2 * i] % np.uint64(len(sides)))]
        k = ranks[int(draws[2 * i + 1] % np.uint64(len(ranks)))]
        out.append(iid_diffusion_2d(N, k, 2 * k, seed=(seed << 20) + i + 1, tol=tol,
                                    with_samples=with_samples))
    return out

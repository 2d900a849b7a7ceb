"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the eigensolver: it only draws random
numbers and evaluates the problem's potential on the grid.  Everything that
the orthogonality-preserving scheme computes lives either in ``oracle/``
(FP64 CPU reference) or in the CUDA library; both take these arrays as input.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: output k of stream ``key`` is ``mix64(key + (k + 1) * GAMMA)``.
Gaussians use the Box-Muller transform (one normal from each pair of
uniforms: ``sqrt(-2 ln u1) * cos(2 pi u2)``).

Grid ordering (shared by every consumer): point (ix, iy, iz) of an
``nx x ny x nz`` interior grid has linear index ``ix + nx * (iy + ny * iz)``;
its coordinate along axis d is ``lo[d] + (i_d + 1) * h_d`` with
``h_d = (hi[d] - lo[d]) / (n_d + 1)`` (homogeneous Dirichlet boundary on the
box, §5 of the paper discretises on a bounded box with zero boundary values).
Orbital blocks are row-major ``n x p`` (the p orbital values of one grid point
are contiguous).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = np.uint64(0xD1B54A32D192ED03)

# Stream tags: independent counter streams derived from one seed.
STREAM_U0 = 1
STREAM_WELLS = 2
STREAM_BATCH = 3
STREAM_LEARN = 4
STREAM_INIT = 5


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        return np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(stream) * _STREAM_MUL)


def splitmix64(key: np.uint64, start: int, count: int) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the counter stream ``key`` (uint64)."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(key + k * GAMMA)


def uniform01(key: np.uint64, start: int, count: int) -> np.ndarray:
    """Doubles in the open interval (0, 1): ((z >> 11) + 0.5) * 2**-53."""
    z = splitmix64(key, start, count)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def gaussian(key: np.uint64, start: int, count: int) -> np.ndarray:
    """Standard normals; normal k uses uniforms 2(start+k) and 2(start+k)+1."""
    u = uniform01(key, 2 * start, 2 * count)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def gaussian_block(seed: int, n: int, p: int) -> np.ndarray:
    """Raw (not yet orthonormal) initial block U0: n x p, row-major, FP64."""
    return gaussian(stream_key(seed, STREAM_U0), 0, n * p).reshape(n, p)


def gaussian_at(key: np.uint64, idx: np.ndarray) -> np.ndarray:
    """Normals number idx (any indices) of the stream `key` (as gaussian())."""
    k = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z1 = _mix64(key + (np.uint64(2) * k + np.uint64(1)) * GAMMA)
        z2 = _mix64(key + (np.uint64(2) * k + np.uint64(2)) * GAMMA)
    u1 = ((z1 >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)
    u2 = ((z2 >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def gaussian_columns(seed: int, n: int, p: int, cols) -> np.ndarray:
    """Columns `cols` of gaussian_block(seed, n, p) without drawing the whole block."""
    cols = np.asarray(cols, dtype=np.int64)
    idx = np.arange(n, dtype=np.int64)[:, None] * p + cols[None, :]
    return gaussian_at(stream_key(seed, STREAM_U0), idx)


# ----------------------------------------------------------------------------
# Problems
# ----------------------------------------------------------------------------
@dataclass
class Well:
    center: tuple
    depth: float
    width: float


@dataclass
class Problem:
    """A discretised eigenproblem H = -1/2 Delta_h + V on an interior grid."""

    shape: tuple                      # (nx, ny) or (nx, ny, nz)
    lo: tuple
    hi: tuple
    V: np.ndarray                     # n values, FP64, grid ordering above
    p: int
    name: str = ""
    wells: list = field(default_factory=list)

    @property
    def dim(self) -> int:
        return len(self.shape)

    @property
    def n(self) -> int:
        return int(np.prod(self.shape))

    @property
    def h(self) -> tuple:
        return tuple((b - a) / (m + 1) for a, b, m in zip(self.lo, self.hi, self.shape))


def grid_coords(shape, lo, hi):
    """Per-axis coordinate vectors of the interior points."""
    return [lo[d] + (np.arange(shape[d]) + 1.0) * ((hi[d] - lo[d]) / (shape[d] + 1))
            for d in range(len(shape))]


def _mesh(shape, lo, hi):
    xs = grid_coords(shape, lo, hi)
    # index ix + nx*(iy + ny*iz): x fastest => meshgrid with 'ij' on reversed axes
    grids = np.meshgrid(*xs[::-1], indexing="ij")[::-1]
    return [g.reshape(-1) for g in grids]


def draw_wells(seed: int, count: int, lo, hi, depth=(1.0, 5.0), width=(0.5, 1.5),
               start: int = 0):
    """Gaussian wells; per well the draw order is centre coords, depth, width."""
    dim = len(lo)
    per = dim + 2
    u = uniform01(stream_key(seed, STREAM_WELLS), start, per * count).reshape(count, per)
    wells = []
    for r in u:
        c = tuple(lo[d] + (hi[d] - lo[d]) * r[d] for d in range(dim))
        wells.append(Well(c, depth[0] + (depth[1] - depth[0]) * r[dim],
                          width[0] + (width[1] - width[0]) * r[dim + 1]))
    return wells


def potential(shape, lo, hi, harmonic: float, wells) -> np.ndarray:
    """V(x) = harmonic * |x|^2 - sum_k d_k exp(-|x - c_k|^2 / (2 w_k^2))."""
    X = _mesh(shape, lo, hi)
    V = np.zeros(X[0].shape)
    if harmonic:
        V += harmonic * sum(x * x for x in X)
    for w in wells:
        r2 = sum((x - c) ** 2 for x, c in zip(X, w.center))
        V -= w.depth * np.exp(-r2 / (2.0 * w.width ** 2))
    return V


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------
def laplace_2d(N: int = 32, p: int = 8) -> Problem:
    """-1/2 Delta on the unit square, N x N interior points, V = 0."""
    shape = (N, N)
    return Problem(shape, (0.0, 0.0), (1.0, 1.0), np.zeros(N * N), p, f"laplace2d_{N}x{N}_p{p}")


def harmonic_2d(N: int = 199, p: int = 15, L: float = 5.5) -> Problem:
    """2D harmonic oscillator -1/2 Delta + 1/2 |x|^2 on (-L, L)^2 (test problem I of §5.1)."""
    shape = (N, N)
    lo, hi = (-L, -L), (L, L)
    return Problem(shape, lo, hi, potential(shape, lo, hi, 0.5, []), p, f"ho2d_{N}x{N}_p{p}")


def wells_3d(N: int, p: int, n_wells: int, seed: int, harmonic: float = 0.5,
             box: float = 8.0, depth=(1.0, 5.0), width=(0.5, 1.5)) -> Problem:
    """3D harmonic trap plus seeded Gaussian wells on [-box, box]^3."""
    shape = (N, N, N)
    lo, hi = (-box,) * 3, (box,) * 3
    wells = draw_wells(seed, n_wells, lo, hi, depth, width)
    V = potential(shape, lo, hi, harmonic, wells)
    return Problem(shape, lo, hi, V, p, f"wells3d_{N}^3_p{p}_w{n_wells}_s{seed}", wells)


def config_2d_laplace() -> Problem:
    """2D 5-point -1/2 Delta, Dirichlet unit square, 32 x 32 interior, V = 0, p = 8."""
    return laplace_2d(32, 8)


def config_3d_wells(seed: int = 0, N: int = 64, p: int = 128) -> Problem:
    """3D 7-point H on 64^3, box [-8, 8]^3, V = 1/2|x|^2 + 8 wells, p = 128."""
    return wells_3d(N, p, 8, seed)


def batch_problems(seed: int, count: int = 64, nmin: int = 24, nmax: int = 48,
                   pmin: int = 16, pmax: int = 96, wmin: int = 2, wmax: int = 12):
    """Uneven batch: per problem N ~ U{nmin..nmax}, p ~ U{pmin..pmax}, wells ~ U{wmin..wmax}."""
    u = uniform01(stream_key(seed, STREAM_BATCH), 0, 3 * count).reshape(count, 3)
    out = []
    for i, r in enumerate(u):
        N = nmin + int(r[0] * (nmax - nmin + 1))
        p = pmin + int(r[1] * (pmax - pmin + 1))
        k = wmin + int(r[2] * (wmax - wmin + 1))
        out.append(wells_3d(N, p, k, seed * 1000 + i))
    return out


def warm_start_problem(seed: int, N: int = 48, p: int = 64, box: float = 8.0,
                       wells=(4, 16), depth=(1.0, 6.0), width=(0.5, 1.5),
                       harmonic: float = 0.0) -> Problem:
    """Learned-warm-start workload: V = sum of U{4..16} Gaussian wells on [-box, box]^3,
    depths U[1, 6], centres uniform in the box (plus harmonic * |x|^2, zero by
    default); N^3 grid, p orbitals."""
    u = uniform01(stream_key(seed, STREAM_LEARN), 0, 1)[0]
    k = wells[0] + int(u * (wells[1] - wells[0] + 1))
    shape = (N, N, N)
    lo, hi = (-box,) * 3, (box,) * 3
    w = draw_wells(seed, k, lo, hi, depth, width)
    return Problem(shape, lo, hi, potential(shape, lo, hi, harmonic, w), p,
                   f"warmstart_{N}^3_p{p}_w{k}_s{seed}", w)


def uniform_init(seed: int, fans) -> np.ndarray:
    """Initial parameters of a layered network as one flat FP32-ready vector.

    ``fans`` lists, per layer in order, (fan_in, n_weights, n_bias).  Weights are
    uniform on (-a, a) with a = sqrt(6 / fan_in) (variance 2 / fan_in, He et al.,
    ICCV 2015); biases are zero.
    """
    total = sum(nw + nb for _, nw, nb in fans)
    u = uniform01(stream_key(seed, STREAM_INIT), 0, total)
    out = np.zeros(total)
    off = 0
    for fan_in, nw, nb in fans:
        a = math.sqrt(6.0 / fan_in)
        out[off:off + nw] = a * (2.0 * u[off:off + nw] - 1.0)
        off += nw + nb
    return out

"""Seeded input generators.

Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), evaluated in counter form: the
k-th draw of stream `seed` is mix(seed + (k+1)*GOLDEN) mod 2^64.  Doubles take
the top 53 bits: u = (z >> 11) * 2^-53 in [0, 1).

Grids follow one convention everywhere in this repository: a level with n
interior points per side is stored as an (n+2) x (n+2) row-major array indexed
[j, i] (i = x, fastest), interior i, j in 1..n, and a ghost ring at 0 and n+1
that carries the Dirichlet value zero.

Stencils are stored as five planes [O, W, S, SW, NW] of shape (n+2, n+2): the
matrix entries a(p, p) and a(p, p-x), a(p, p-y), a(p, p-x-y), a(p, p-x+y).  The
other four couplings follow from the symmetry of A: E(p) = W(p+x),
N(p) = S(p+y), NE(p) = SW(p+x+y), SE(p) = NW(p+x-y).  Couplings that would
reach a ghost point are not entries of A (Dirichlet rows drop them) and are
stored as zero, as is the whole ghost ring of every plane.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

PLANES = ("O", "W", "S", "SW", "NW")


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of the SplitMix64 stream `seed` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    """count doubles in [0, 1) from stream `seed`."""
    z = splitmix64(seed, count)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, count: int) -> np.ndarray:
    """count doubles in [-1, 1) from stream `seed`."""
    return 2.0 * uniform01(seed, count) - 1.0


def normal(seed: int, count: int) -> np.ndarray:
    """count standard normals (Box-Muller on pairs of uniforms of stream `seed`)."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]                 # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return z[:count]


def is_level_size(n: int) -> bool:
    """n = 2^m - 1 with m >= 2 (3, 7, 15, ...)."""
    return n >= 3 and ((n + 1) & n) == 0


def grid_zeros(n: int) -> np.ndarray:
    return np.zeros((n + 2, n + 2), dtype=np.float64)


def rhs_uniform(n: int, seed: int, ny: int | None = None) -> np.ndarray:
    """Right-hand side: interior i.i.d. uniform[-1, 1), ghost ring zero; an
    (n+2)^2 grid, or (ny+2) x (n+2) when ny is given."""
    ny = n if ny is None else ny
    f = np.zeros((ny + 2, n + 2), dtype=np.float64)
    f[1:ny + 1, 1:n + 1] = uniform_pm1(seed, n * ny).reshape(ny, n)
    return f


def zero_ghost_couplings(planes: np.ndarray) -> np.ndarray:
    """Zero the ghost ring of all planes and the couplings of interior points to
    ghost points (in place; returns planes).  Planes are (ny+2, nx+2)."""
    O, W, S, SW, NW = planes
    ny, nx = planes.shape[1] - 2, planes.shape[2] - 2
    for a in planes:
        a[0, :] = 0.0
        a[ny + 1, :] = 0.0
        a[:, 0] = 0.0
        a[:, nx + 1] = 0.0
    W[:, 1] = 0.0          # (1, j) -> (0, j)
    S[1, :] = 0.0          # (i, 1) -> (i, 0)
    SW[:, 1] = 0.0
    SW[1, :] = 0.0
    NW[:, 1] = 0.0
    NW[ny, :] = 0.0        # (i, ny) -> (i-1, ny+1)
    return planes


def poisson5(n: int) -> np.ndarray:
    """5-point finite-difference Laplacian (unscaled): O = 4, W = S = -1."""
    planes = np.zeros((5, n + 2, n + 2), dtype=np.float64)
    planes[0, 1:n + 1, 1:n + 1] = 4.0
    planes[1, 1:n + 1, 1:n + 1] = -1.0
    planes[2, 1:n + 1, 1:n + 1] = -1.0
    return zero_ghost_couplings(planes)


def poisson5_rect(nx: int, ny: int) -> np.ndarray:
    """5-point Laplacian (4, -1) on an nx x ny interior grid: planes (5, ny+2, nx+2)."""
    planes = np.zeros((5, ny + 2, nx + 2), dtype=np.float64)
    planes[0, 1:ny + 1, 1:nx + 1] = 4.0
    planes[1, 1:ny + 1, 1:nx + 1] = -1.0
    planes[2, 1:ny + 1, 1:nx + 1] = -1.0
    return zero_ghost_couplings(planes)


def anisotropic5(n: int, eps: float) -> np.ndarray:
    """5-point finite differences of -(u_xx + eps u_yy) (unscaled): O = 2 (1 + eps),
    W = -1, S = -eps, ghost couplings zero; planes SW, NW are zero."""
    planes = np.zeros((5, n + 2, n + 2))
    planes[0, 1:-1, 1:-1] = 2.0 * (1.0 + eps)
    planes[1, 1:-1, 1:-1] = -1.0
    planes[2, 1:-1, 1:-1] = -eps
    return zero_ghost_couplings(planes)


def transposed_stencil(planes: np.ndarray) -> np.ndarray:
    """The planes of the same operator with x and y exchanged (point (i, j)
    becomes (j, i)), for square planes: W and S swap and SW stays (each
    transposed); the new NW coupling at (i, j) is the old SE coupling at
    (j, i), which the old planes store as NW at (j + 1, i - 1)."""
    O, W, S, SW, NW = planes
    n = O.shape[0] - 2
    nw = np.zeros_like(NW)
    nw[0:n + 1, 1:n + 2] = NW[0:n + 1, 1:n + 2].T
    return np.stack([O.T, S.T, W.T, SW.T, nw])


def fe9_from_cells(k: np.ndarray) -> np.ndarray:
    """9-point bilinear (Q1) finite-element stiffness stencil of -div(k grad u)
    on a uniform grid, with k constant on each cell.

    k has shape (ny+1, nx+1) (square: (n+1, n+1)), k[cj, ci] on the cell whose
    lower-left node is (ci, cj); the planes are (5, ny+2, nx+2).  The Q1 element matrix of a square cell, scaled by k, has 2k/3 on
    its diagonal, -k/6 between nodes sharing a cell edge and -k/3 between
    opposite corners.  Summing the cells around each node gives
      O(i,j)  = (2/3) (k[j-1,i-1] + k[j-1,i] + k[j,i-1] + k[j,i])
      W(i,j)  = -(k[j-1,i-1] + k[j,i-1]) / 6
      S(i,j)  = -(k[j-1,i-1] + k[j-1,i]) / 6
      SW(i,j) = -k[j-1,i-1] / 3
      NW(i,j) = -k[j,i-1] / 3
    """
    return zero_ghost_couplings(_fe9_assemble(k))


def _fe9_assemble(k: np.ndarray) -> np.ndarray:
    """The node sums of fe9_from_cells over every interior node, ghost
    couplings kept."""
    ny, nx = k.shape[0] - 1, k.shape[1] - 1
    planes = np.zeros((5, ny + 2, nx + 2), dtype=np.float64)
    kll = k[0:ny, 0:nx]              # cell (i-1, j-1) for interior node (i, j)
    klr = k[0:ny, 1:nx + 1]          # cell (i,   j-1)
    kul = k[1:ny + 1, 0:nx]          # cell (i-1, j)
    kur = k[1:ny + 1, 1:nx + 1]      # cell (i,   j)
    I = (slice(1, ny + 1), slice(1, nx + 1))
    planes[0][I] = (2.0 / 3.0) * (kll + klr + kul + kur)
    planes[1][I] = -(kll + kul) / 6.0
    planes[2][I] = -(kll + klr) / 6.0
    planes[3][I] = -kll / 3.0
    planes[4][I] = -kul / 3.0
    return planes


def fe9_periodic(k: np.ndarray, px: bool, py: bool) -> np.ndarray:
    """9-point Q1 stencil of -div(k grad u) (the sums of fe9_from_cells) on a
    grid whose periodic axes wrap around.  k[cj, ci] is the cell whose
    lower-left node is (ci, cj); along a periodic axis of N nodes there are N
    cells, cell 0 lying between node N and node 1, along a Dirichlet axis of
    N nodes there are N + 1.  Planes (5, ny+2, nx+2): the ghost lines zero,
    couplings toward a Dirichlet ghost zero, couplings across a periodic side
    kept (W at i = 1 couples node 1 to node N through cell 0)."""
    ke = np.asarray(k, dtype=np.float64)
    if px:
        ke = np.concatenate([ke, ke[:, :1]], axis=1)
    if py:
        ke = np.concatenate([ke, ke[:1, :]], axis=0)
    planes = _fe9_assemble(ke)
    O, W, S, SW, NW = planes
    ny, nx = planes.shape[1] - 2, planes.shape[2] - 2
    for a in planes:
        a[0, :] = 0.0
        a[ny + 1, :] = 0.0
        a[:, 0] = 0.0
        a[:, nx + 1] = 0.0
    if not px:
        W[:, 1] = 0.0
        SW[:, 1] = 0.0
        NW[:, 1] = 0.0
    if not py:
        S[1, :] = 0.0
        SW[1, :] = 0.0
        NW[ny, :] = 0.0
    return planes


def binary_blocks(n: int, block: int, lo: float, hi: float, seed: int, p: float = 0.5) -> np.ndarray:
    """Cell field on (n+1)^2 cells, constant on block x block tiles, each tile
    `hi` with probability p (uniform draw < p) else `lo`."""
    cells = n + 1
    nb = (cells + block - 1) // block
    u = uniform01(seed, nb * nb).reshape(nb, nb)
    tile = np.where(u < p, hi, lo)
    return np.repeat(np.repeat(tile, block, axis=0), block, axis=1)[:cells, :cells].copy()


def gaussian_field(cells: int, std: float, corr_len: float, seed: int) -> np.ndarray:
    """Periodic Gaussian random field on cells x cells with covariance close to
    std^2 exp(-r^2 / (2 corr_len^2)): white noise smoothed by a Gaussian filter
    of width corr_len/sqrt(2), then shifted and scaled to sample mean 0 and
    sample standard deviation std."""
    from scipy.ndimage import gaussian_filter
    w = normal(seed, cells * cells).reshape(cells, cells)
    g = gaussian_filter(w, sigma=corr_len / np.sqrt(2.0), mode="wrap", truncate=4.0)
    g = g - g.mean()
    return g * (std / g.std())


def lognormal_cells(n: int, std: float, corr_len: float, seed: int) -> np.ndarray:
    """k = exp(g) on (n+1)^2 cells, g a Gaussian random field (see gaussian_field)."""
    return np.exp(gaussian_field(n + 1, std, corr_len, seed))


def layered_cells(n: int, values_by_column: np.ndarray) -> np.ndarray:
    """k depending on the cell column ci only (k[cj, ci] = values_by_column[ci])."""
    v = np.asarray(values_by_column, dtype=np.float64)
    assert v.shape == (n + 1,)
    return np.tile(v, (n + 1, 1))


# ----------------------------------------------------------------------------
# The named workloads.  Each returns (kind, planes, rhs) with float64 arrays.
# ----------------------------------------------------------------------------

def poisson_problem(n: int = 127, seed: int = 1):
    """2D Poisson, 5-point stencil, Dirichlet zero boundary, RHS uniform[-1,1)."""
    return 5, poisson5(n), rhs_uniform(n, seed)


def binary_contrast_problem(n: int = 2047, block: int = 16, lo: float = 1.0, hi: float = 1e4,
                            seed_k: int = 2, seed_f: int = 3, p: float = 0.5):
    """-div(k grad u) with k in {lo, hi} on block x block tiles (Bernoulli p),
    9-point Q1 stencil, RHS uniform[-1,1)."""
    k = binary_blocks(n, block, lo, hi, seed_k, p)
    return 9, fe9_from_cells(k), rhs_uniform(n, seed_f)


def lognormal_problem(n: int = 8191, std: float = 2.0, corr_len: float = 32.0,
                      seed_k: int = 4, seed_f: int = 7):
    """-div(k grad u) with k = exp(g), g a Gaussian field; 9-point Q1 stencil."""
    k = lognormal_cells(n, std, corr_len, seed_k)
    return 9, fe9_from_cells(k), rhs_uniform(n, seed_f)


def batched_sizes(count: int = 256, seed: int = 5, choices=(63, 127, 255, 511, 1023), first: int = 0):
    """Interior sides of problems first .. first+count-1, drawn uniformly from
    `choices` (one draw per problem from stream `seed`)."""
    u = uniform01(seed, first + count)[first:]
    idx = np.minimum((u * len(choices)).astype(np.int64), len(choices) - 1)
    return [int(choices[i]) for i in idx]


def batched_problems(count: int = 256, seed: int = 5, std: float = 1.0, corr_len: float = 32.0,
                     choices=(63, 127, 255, 511, 1023), first: int = 0):
    """Independent 9-point log-normal problems of uneven sizes; problem b
    (b counted from 0 over the whole sequence, this call returning
    first .. first+count-1) uses coefficient seed 10000 + 2b and RHS seed
    10001 + 2b."""
    out = []
    for j, n in enumerate(batched_sizes(count, seed, choices, first)):
        b = first + j
        k = lognormal_cells(n, std, corr_len, 10000 + 2 * b)
        out.append((9, fe9_from_cells(k), rhs_uniform(n, 10001 + 2 * b)))
    return out


def general_size_problem(nx: int, ny: int, kind: int = 9, std: float = 1.0, corr_len: float = 8.0,
                         seed_k: int = 30, seed_f: int = 31):
    """(kind, planes, f) on an nx x ny interior grid of any size: 9-point Q1 with
    k = exp(g) (g the Gaussian field of the square of side max(nx, ny) + 1 cells,
    cropped), or the 5-point Laplacian; RHS uniform[-1, 1)."""
    if kind == 5:
        planes = poisson5_rect(nx, ny)
    else:
        g = gaussian_field(max(nx, ny) + 1, std, corr_len, seed_k)
        planes = fe9_from_cells(np.exp(g)[:ny + 1, :nx + 1].copy())
    return kind, planes, rhs_uniform(nx, seed_f, ny)


def neumann_problem(nx: int, ny: int, sides: str = "EN", std: float = 1.0, corr_len: float = 8.0,
                    seed_k: int = 40, seed_f: int = 41):
    """9-point Q1 problem of -div(k grad u) = f with natural (Neumann) boundary
    conditions on the listed sides (E, W, N, S) and u = 0 on the others.  The
    nodes of a Neumann side are unknowns (the outermost interior row or column
    of the nx x ny grid) and the cells beyond them have k = 0, so their
    stencils sum over the cells inside the domain only, the element-by-element
    assembly of the natural condition.  k = exp(g) inside, RHS uniform[-1, 1)."""
    g = gaussian_field(max(nx, ny) + 1, std, corr_len, seed_k)
    k = np.exp(g)[:ny + 1, :nx + 1].copy()
    if "E" in sides:
        k[:, nx] = 0.0       # cells east of the column i = nx
    if "W" in sides:
        k[:, 0] = 0.0        # cells west of the column i = 1
    if "N" in sides:
        k[ny, :] = 0.0
    if "S" in sides:
        k[0, :] = 0.0
    return 9, fe9_from_cells(k), rhs_uniform(nx, seed_f, ny)


def periodic_shape(n: int, axes: str) -> tuple[int, int]:
    """(nx, ny) of a grid with side n = 2^m - 1 whose `axes` ("x", "y" or
    "xy") are periodic: a periodic axis has n + 1 = 2^m nodes."""
    return (n + 1 if "x" in axes else n), (n + 1 if "y" in axes else n)


def periodic_problem(n: int = 4095, axes: str = "x", std: float = 2.0, corr_len: float = 32.0,
                     seed_k: int = 50, seed_f: int = 51, shift: float = 0.0):
    """-div(k grad u) (+ shift u) on a grid periodic along `axes` (sizes from
    periodic_shape), zero Dirichlet on the other sides: k = exp(g) on the
    (n+1)^2 cells, g the periodic Gaussian field of gaussian_field (so k
    itself wraps smoothly across a periodic side), 9-point Q1 stencil, `shift`
    added to every diagonal (needed when both axes are periodic, where the
    diffusion operator annihilates constants); RHS uniform[-1, 1).
    Returns (kind, planes, rhs, px, py)."""
    nx, ny = periodic_shape(n, axes)
    px, py = "x" in axes, "y" in axes
    k = np.exp(gaussian_field(n + 1, std, corr_len, seed_k))
    planes = fe9_periodic(k, px, py)
    planes[0, 1:ny + 1, 1:nx + 1] += shift
    return 9, planes, rhs_uniform(nx, seed_f, ny), px, py


def high_contrast_problem(n: int = 4095, block: int = 8, lo: float = 1.0, hi: float = 1e6,
                          seed: int = 6):
    """Binary blocks k in {1, 1e6} on 8 x 8 cell tiles (the learned-interpolation
    family); RHS seed = seed + 100000."""
    return binary_contrast_problem(n, block, lo, hi, seed_k=seed, seed_f=seed + 100000)


def training_crops(count: int, first_seed: int = 1000, n: int = 255, m: int = 31, block: int = 8,
                   lo: float = 1.0, hi: float = 1e6, vectors: int = 4, crops_per_problem: int = 1):
    """Training inputs of the learned interpolation: for each of `count`
    problems of the family (n x n interior, k in {lo, hi} on block x block
    cell tiles, Bernoulli 0.5, cell field seed first_seed + s), crops of
    (m+1) x (m+1) cells at offsets that are multiples of the tile size (so the
    tile edges fall on the crop's coarse grid lines as they do in the full
    problem), each assembled as its own m x m Dirichlet problem, with `vectors`
    uniform[-1,1) error vectors.  Offsets: draws of stream 7_000_000 + s;
    vectors: seeds 8_000_000 + (s * crops_per_problem + c) * vectors + k.
    Returns a list of (planes (5, m+2, m+2), vectors (vectors, m+2, m+2))."""
    out = []
    slots = (n + 1 - (m + 1)) // block + 1
    for s in range(first_seed, first_seed + count):
        cells = binary_blocks(n, block, lo, hi, s)
        off = (splitmix64(7_000_000 + s, 2 * crops_per_problem) % np.uint64(slots)).astype(np.int64) * block
        for c in range(crops_per_problem):
            j0, i0 = int(off[2 * c]), int(off[2 * c + 1])
            planes = fe9_from_cells(cells[j0:j0 + m + 1, i0:i0 + m + 1].copy())
            base = 8_000_000 + (s * crops_per_problem + c) * vectors
            vecs = np.stack([rhs_uniform(m, base + k) for k in range(vectors)])
            out.append((planes, vecs))
    return out

"""Seeded synthetic inputs for the heat-conduction topology-optimisation solve.

This module only *generates problem data*: density fields, the Dirichlet node
mask and the element source.  It holds none of the solver's arithmetic (no
operator, no preconditioner, no sensitivity), so both the CPU oracle and the
CUDA path can draw the same inputs from it.

The problems mirror the paper's model problem (Sec. 2.1, Fig. "design domain"):
the unit cube, a square Dirichlet patch centred on one face, all other faces
adiabatic, and a density x in [0, 1] per element.  The paper optimises
tree-like high-conductivity layouts (Sec. 4.1, Figs. of optimised designs);
the "channels" generator below produces seeded binary trees of square tubes
with that structure, which is what makes high contrast hard for a solver.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), keyed by (seed, index), so every
field is reproducible element by element on any machine.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, index) -> np.ndarray:
    """SplitMix64 output for stream ``seed`` at positions ``index`` (uint64).

    The state for position i is seed * 2**32 + i + 1 times the golden gamma,
    followed by the standard SplitMix64 finaliser.
    """
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (np.uint64(seed) * np.uint64(1 << 32) + idx + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1): (splitmix64 >> 11) * 2**-53."""
    z = splitmix64(seed, np.arange(n, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ----------------------------------------------------------------------------
# Grid helpers (layout convention shared by every caller of the C ABI)
#   elements e = ex + Nx*(ey + Ny*ez), nodes n = i + (Nx+1)*(j + (Ny+1)*k)
# Arrays returned here are flat and x-fastest.
# ----------------------------------------------------------------------------

def dirichlet_patch_mask(grid, half_width: float = 0.1, face: str = "z0",
                         centre=(0.5, 0.5)) -> np.ndarray:
    """uint8 node mask, 1 on the square patch |x-cx|<=w, |y-cy|<=w of z = 0.

    The cube is [0,1]^3 with h = 1/N per axis.  Membership uses a closed
    interval with a 1e-12*h tolerance, so grid points exactly on the patch edge
    are inside.
    """
    Nx, Ny, Nz = grid
    nx, ny, nz = Nx + 1, Ny + 1, Nz + 1
    mask = np.zeros((nz, ny, nx), dtype=np.uint8)
    xs = np.arange(nx) / Nx
    ys = np.arange(ny) / Ny
    tol = 1e-12 / max(Nx, Ny)
    inx = np.abs(xs - centre[0]) <= half_width + tol
    iny = np.abs(ys - centre[1]) <= half_width + tol
    if face != "z0":
        raise ValueError("only the z = 0 face is used by the model problem")
    mask[0][np.ix_(iny, inx)] = 1
    return mask.reshape(-1)


def full_face_mask(grid, face: str = "z0") -> np.ndarray:
    """uint8 node mask covering an entire face (z0, z1, or 'all')."""
    Nx, Ny, Nz = grid
    mask = np.zeros((Nz + 1, Ny + 1, Nx + 1), dtype=np.uint8)
    if face in ("z0", "z01", "all"):
        mask[0] = 1
    if face in ("z1", "z01", "all"):
        mask[-1] = 1
    if face == "all":
        mask[:, 0, :] = 1
        mask[:, -1, :] = 1
        mask[:, :, 0] = 1
        mask[:, :, -1] = 1
    return mask.reshape(-1)


def uniform_source(grid, q: float = 1.0) -> np.ndarray:
    Nx, Ny, Nz = grid
    return np.full(Nx * Ny * Nz, q, dtype=np.float64)


def smoothed_threshold_density(N: int, seed: int, volfrac: float,
                               sigma: float = 2.0) -> np.ndarray:
    """Binary density: seeded U[0,1) noise, Gaussian-smoothed (sigma elements,
    truncated at 4 sigma, reflecting boundary), then x = 1 on the
    round(volfrac*M) largest smoothed values (ties to the lower index)."""
    from scipy.ndimage import gaussian_filter

    M = N ** 3
    noise = uniform01(seed, M).reshape(N, N, N)
    sm = gaussian_filter(noise, sigma=sigma, mode="reflect", truncate=4.0)
    flat = sm.reshape(-1)
    k = int(np.floor(volfrac * M + 0.5))
    order = np.argsort(-flat, kind="stable")
    x = np.zeros(M, dtype=np.float64)
    x[order[:k]] = 1.0
    return x


def smooth_random_density(N: int, seed: int, lo: float = 0.05,
                          hi: float = 1.0, sigma: float = 1.5) -> np.ndarray:
    """Continuous density in [lo, hi]: smoothed seeded noise rescaled.

    Every block sees a different coefficient field, so local eigenvalues are
    generically simple; used where parity must compare bases element by
    element.
    """
    from scipy.ndimage import gaussian_filter

    M = N ** 3
    noise = uniform01(seed, M).reshape(N, N, N)
    sm = gaussian_filter(noise, sigma=sigma, mode="reflect", truncate=4.0)
    sm = (sm - sm.min()) / max(sm.max() - sm.min(), 1e-300)
    return (lo + (hi - lo) * sm).reshape(-1)


def channel_tree_density(N: int, seed: int, volfrac: float,
                         trunk_height: float = 0.6, dtype=np.float64) -> np.ndarray:
    """Binary tree of axis-aligned square tubes rooted at the heat sink.

    The trunk runs along z from the patch centre (x = y = 1/2) up to
    z = trunk_height with width w = max(2, N // 64) elements.  Each further
    tube starts at a seeded element of an existing tube, runs along an axis
    different from its parent's, in a seeded direction, with length
    U[0.1, 0.5] (domain units), clipped to the domain.  Tubes are added until
    the volume reaches round(volfrac * M); the last tube is trimmed in raster
    order to hit that count exactly.  ``dtype`` is the returned array's type
    (the values are 0 and 1 in any type).
    """
    M = N ** 3
    target = int(np.floor(volfrac * M + 0.5))
    w = max(2, N // 64)
    x = np.zeros((N, N, N), dtype=np.uint8)  # [z, y, x]
    counter = [0]

    def rnd():
        v = uniform01_at(seed, counter[0])
        counter[0] += 1
        return v

    c0 = N // 2 - w // 2
    tubes = []  # (axis, lo corner (x,y,z), hi corner exclusive)
    trunk = (2, (c0, c0, 0), (c0 + w, c0 + w, max(1, int(round(trunk_height * N)))))
    tubes.append(trunk)

    def raster(t):
        _, lo, hi = t
        return lo, hi

    def paint(t, budget):
        lo, hi = raster(t)
        region = x[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        free = np.flatnonzero(region.reshape(-1) == 0)
        take = free[:budget]
        flat = region.reshape(-1)
        flat[take] = 1
        region[...] = flat.reshape(region.shape)
        return len(take)

    vol = paint(trunk, target)
    guard = 0
    while vol < target and guard < 100000:
        guard += 1
        parent = tubes[int(rnd() * len(tubes)) % len(tubes)]
        pax, plo, phi = parent
        # seeded start element on the parent tube
        sx = plo[0] + int(rnd() * (phi[0] - plo[0]))
        sy = plo[1] + int(rnd() * (phi[1] - plo[1]))
        sz = plo[2] + int(rnd() * (phi[2] - plo[2]))
        axes = [a for a in range(3) if a != pax]
        ax = axes[int(rnd() * 2) % 2]
        sign = 1 if rnd() < 0.5 else -1
        length = max(1, int(round((0.1 + 0.4 * rnd()) * N)))
        start = [sx, sy, sz]
        lo = [min(max(s - w // 2, 0), N - w) for s in start]
        hi = [l + w for l in lo]
        if sign > 0:
            lo[ax] = start[ax]
            hi[ax] = min(N, start[ax] + length)
        else:
            hi[ax] = start[ax] + 1
            lo[ax] = max(0, start[ax] + 1 - length)
        t = (ax, tuple(lo), tuple(hi))
        tubes.append(t)
        vol += paint(t, target - vol)
    return x.reshape(-1).astype(dtype)


def uniform01_at(seed: int, i: int) -> float:
    z = splitmix64(seed, np.array([i], dtype=np.uint64))[0]
    return float(z >> np.uint64(11)) * (1.0 / 9007199254740992.0)


def fisher_yates_sample(seed: int, n: int, k: int) -> np.ndarray:
    """k distinct indices from range(n) by a seeded partial Fisher-Yates shuffle
    (stream ``seed``; step i uses draw i)."""
    perm = {}
    out = np.empty(k, dtype=np.int64)
    for i in range(k):
        j = i + int(uniform01_at(seed, i) * (n - i))
        vi = perm.get(i, i)
        vj = perm.get(j, j)
        perm[i], perm[j] = vj, vi
        out[i] = vj
    return out


# ----------------------------------------------------------------------------
# Named workloads (sizes, contrasts, densities of the solver's benchmark set)
# ----------------------------------------------------------------------------

def problem(name: str) -> dict:
    """Inputs for a named workload: grid, h, mask, source, x, p, kmin, kmax.

    * ``cube32``: 32^3, Gaussian-smoothed threshold density (sigma 2, V=0.3,
      seed 1), p=3, kmin=1e-3, kmax=1.
    * ``chan128``: 128^3, channel tree (V=0.2, seed 2), kmin=1e-6.
    * ``chan128_1e3|1e6|1e9``: the chan128 design at contrast 1e3 / 1e6 / 1e9.
    * ``chan256_1e3|1e6|1e9``: 256^3, channel tree (V=0.2, seed 3).
    * ``smoothNN``: NN^3 continuous density in [0.05, 1] (seed 7), kmin=1e-3.
    * ``chanNN``: NN^3 channel tree (V=0.2, seed 3), kmin=1e-6.
    * ``chanNNvFF``: NN^3 channel tree at volume fraction FF/100 (seed 5),
      kmin=1e-6; the design as float32 and no source array (``source`` is
      None: q = 1 everywhere, for callers that fill it on the device).  The
      large configuration is ``chan1024v10``.
    All use q = 1 and T = 0 on the centred 0.2 x 0.2 patch of z = 0.
    """
    if name == "cube32":
        N, x, kmin = 32, smoothed_threshold_density(32, 1, 0.3), 1e-3
    elif name == "chan128":
        N, x, kmin = 128, channel_tree_density(128, 2, 0.2), 1e-6
    elif name.startswith("chan256_"):
        N = 256
        kmin = float(name.split("_")[1])
        kmin = 1.0 / kmin
        x = channel_tree_density(256, 3, 0.2)
    elif name.startswith("chan128_"):
        N = 128
        kmin = 1.0 / float(name.split("_")[1])
        x = channel_tree_density(128, 2, 0.2)
    elif name.startswith("smooth"):
        N = int(name[len("smooth"):])
        x, kmin = smooth_random_density(N, 7), 1e-3
    elif name.startswith("chan") and "v" in name:
        N, vf = name[len("chan"):].split("v")
        N = int(N)
        grid = (N, N, N)
        x = channel_tree_density(N, 5, int(vf) / 100.0, dtype=np.float32)
        return dict(name=name, grid=grid, h=(1.0 / N,) * 3, mask=dirichlet_patch_mask(grid), source=None,
                    x=x, p=3.0, kmin=1e-6, kmax=1.0)
    elif name.startswith("chan"):
        N = int(name[len("chan"):])
        x, kmin = channel_tree_density(N, 3, 0.2), 1e-6
    elif name.startswith("thresh"):
        N = int(name[len("thresh"):])
        x, kmin = smoothed_threshold_density(N, 1, 0.3), 1e-3
    else:
        raise KeyError(name)
    grid = (N, N, N)
    return dict(name=name, grid=grid, h=(1.0 / N,) * 3,
                mask=dirichlet_patch_mask(grid), source=uniform_source(grid),
                x=x, p=3.0, kmin=kmin, kmax=1.0)

"""Seeded synthetic inputs for the block-hydro packet task.

This module holds the initial conditions and the mesh geometry of the
workloads, and pure index reshuffles between a global cell array and the
block layout. It holds none of the scheme's arithmetic (no reconstruction,
flux, update or time step), so the CUDA path and the CPU oracle can both take
their inputs from here.

Initial states are conserved variables U = (rho, m_x, m_y[, m_z], E) with
E = p / (gamma - 1) + rho |u|^2 / 2 (ideal gamma-law gas; the paper's Sedov
section names this EOS).

Block layout: ``U[block, var, k, j, i]`` (i fastest), block id
``bx + nbx * (by + nby * bz)``; 2D meshes have ``nb[2] = bs[2] = 1``.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

GAMMA = 1.4
CFL = 0.8


@dataclass(frozen=True)
class MeshSpec:
    """Uniform grid of equal blocks covering the box [lo, hi]."""
    ndim: int
    nb: tuple            # blocks per axis
    bs: tuple            # interior cells per block per axis
    periodic: tuple = (0, 0, 0)
    gamma: float = GAMMA
    cfl: float = CFL
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)

    def __post_init__(self):
        if self.ndim not in (2, 3):
            raise ValueError("ndim must be 2 or 3")
        if self.ndim == 2 and (self.nb[2] != 1 or self.bs[2] != 1):
            raise ValueError("2D meshes have nb[2] = bs[2] = 1")

    @property
    def nvar(self) -> int:
        return self.ndim + 2

    @property
    def nblocks(self) -> int:
        return int(self.nb[0] * self.nb[1] * self.nb[2])

    @property
    def ncells(self) -> tuple:
        return tuple(int(self.nb[d] * self.bs[d]) for d in range(3))

    @property
    def zones(self) -> int:
        return int(np.prod(self.ncells))

    def block_shape(self) -> tuple:
        return (self.nblocks, self.nvar, self.bs[2], self.bs[1], self.bs[0])

    def dx(self, d: int) -> float:
        return (self.hi[d] - self.lo[d]) / self.ncells[d]

    def centers(self):
        """Cell-centre coordinates (x, y, z) as 3D arrays indexed [k, j, i]."""
        ax = []
        for d in range(3):
            n = self.ncells[d]
            ax.append(self.lo[d] + (np.arange(n) + 0.5) * ((self.hi[d] - self.lo[d]) / n))
        z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        return x, y, z

    def oracle_kwargs(self) -> dict:
        return dict(ndim=self.ndim, nb=tuple(self.nb), bs=tuple(self.bs),
                    periodic=tuple(self.periodic), gamma=self.gamma, cfl=self.cfl,
                    lo=tuple(self.lo), hi=tuple(self.hi))


# ------------------------------------------------------------------ layout

def to_blocks(spec: MeshSpec, Ug: np.ndarray) -> np.ndarray:
    """Global array [var, k, j, i] -> block array [block, var, k, j, i]."""
    nv = spec.nvar
    (nbx, nby, nbz), (bx, by, bz) = spec.nb, spec.bs
    a = Ug.reshape(nv, nbz, bz, nby, by, nbx, bx)
    a = a.transpose(1, 3, 5, 0, 2, 4, 6)          # nbz, nby, nbx, v, bz, by, bx
    return np.ascontiguousarray(a.reshape(spec.nblocks, nv, bz, by, bx))


def from_blocks(spec: MeshSpec, Ub: np.ndarray) -> np.ndarray:
    """Block array [block, var, k, j, i] -> global array [var, k, j, i]."""
    nv = spec.nvar
    (nbx, nby, nbz), (bx, by, bz) = spec.nb, spec.bs
    a = Ub.reshape(nbz, nby, nbx, nv, bz, by, bx)
    a = a.transpose(3, 0, 4, 1, 5, 2, 6)          # v, nbz, bz, nby, by, nbx, bx
    return np.ascontiguousarray(a.reshape(nv, nbz * bz, nby * by, nbx * bx))


def cons_from_prim_global(spec: MeshSpec, rho, vel, p) -> np.ndarray:
    """Assemble a global conserved array from primitive fields (initial data)."""
    rho = np.asarray(rho, dtype=np.float64)
    shape = rho.shape
    U = np.zeros((spec.nvar,) + shape)
    U[0] = rho
    ke = np.zeros(shape)
    for d in range(spec.ndim):
        vd = np.broadcast_to(np.asarray(vel[d], dtype=np.float64), shape)
        U[1 + d] = rho * vd
        ke = ke + vd * vd
    U[spec.nvar - 1] = np.broadcast_to(p, shape) / (spec.gamma - 1.0) + 0.5 * rho * ke
    return U


# ------------------------------------------------------------------ problems

def sod_spec(N: int = 64, b: int = 8, ny_cells: int | None = None) -> MeshSpec:
    """2D Sod tube mesh: N x N cells (or N x ny_cells) as blocks of b x b,
    outflow; cells are square (the y extent is ny_cells / N)."""
    ny = N if ny_cells is None else ny_cells
    return MeshSpec(ndim=2, nb=(N // b, ny // b, 1), bs=(b, b, 1), hi=(1.0, ny / N, 1.0))


def sod_state(spec: MeshSpec, split: float = 0.5, axis: int = 0,
              left=(1.0, 1.0), right=(0.125, 0.1)) -> np.ndarray:
    """Sod shock tube: (rho, p) = left for cell centres below `split` along
    `axis`, right otherwise; at rest. Returns the block array."""
    x, y, z = spec.centers()
    xc = (x, y, z)[axis]
    if spec.ndim == 2:
        xc = xc[0]
    lmask = xc < split
    rho = np.where(lmask, left[0], right[0])
    p = np.where(lmask, left[1], right[1])
    vel = [np.zeros_like(rho)] * spec.ndim
    return to_blocks(spec, _globalize(spec, cons_from_prim_global(spec, rho, vel, p)))


def _globalize(spec: MeshSpec, U: np.ndarray) -> np.ndarray:
    """2D problems are built as [var, j, i]; give them the unit k axis."""
    if spec.ndim == 2 and U.ndim == 3:
        return U[:, None, :, :]
    return U


def sedov_spec(N: int = 128, b: int = 16, periodic: bool = False) -> MeshSpec:
    per = (1, 1, 1) if periodic else (0, 0, 0)
    return MeshSpec(ndim=3, nb=(N // b,) * 3, bs=(b,) * 3, periodic=per)


def sedov_deposit_mask(spec: MeshSpec, radius_cells: float = 3.5, center=(0.5, 0.5, 0.5)):
    """Cells whose centre lies within radius_cells * dx of the centre (<=)."""
    x, y, z = spec.centers()
    dx = spec.dx(0)
    r2 = ((x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2) / (dx * dx)
    return r2 <= radius_cells ** 2 * (1.0 + 1e-12)


def sedov_state(spec: MeshSpec, rho0: float = 1.0, p0: float = 1e-5, energy: float = 1.0,
                radius_cells: float = 3.5, center=(0.5, 0.5, 0.5)) -> np.ndarray:
    """Sedov blast: uniform rho0, p0, at rest; total energy `energy` added in
    equal parts to the cells within `radius_cells` cells of `center`."""
    mask = sedov_deposit_mask(spec, radius_cells, center)
    ndep = int(mask.sum())
    dV = spec.dx(0) * spec.dx(1) * spec.dx(2)
    shape = mask.shape
    rho = np.full(shape, rho0)
    vel = [np.zeros(shape)] * 3
    U = cons_from_prim_global(spec, rho, vel, np.full(shape, p0))
    U[4] = U[4] + np.where(mask, energy / (ndep * dV), 0.0)
    return to_blocks(spec, U)


def uniform_state(spec: MeshSpec, rho: float, vel, p: float) -> np.ndarray:
    shape = (spec.ncells[2], spec.ncells[1], spec.ncells[0])
    U = cons_from_prim_global(spec, np.full(shape, rho), [np.full(shape, v) for v in vel[:spec.ndim]],
                              np.full(shape, p))
    return to_blocks(spec, U)


def advected_wave_state(spec: MeshSpec, amp: float = 0.2, u: float = 1.0, p: float = 1.0,
                        t: float = 0.0) -> np.ndarray:
    """rho = 1 + amp sin(2 pi (x - u t)), uniform velocity u along x and
    pressure p: an exact solution of the Euler equations on a periodic box."""
    x, y, z = spec.centers()
    rho = 1.0 + amp * np.sin(2.0 * np.pi * (x - u * t))
    shape = rho.shape
    vel = [np.full(shape, u)] + [np.zeros(shape)] * (spec.ndim - 1)
    if spec.ndim == 2:
        rho = rho[0]
        vel = [v[0] for v in vel]
    return to_blocks(spec, _globalize(spec, cons_from_prim_global(spec, rho, vel, np.full(rho.shape, p))))


def random_smooth_state(spec: MeshSpec, seed: int, amp: float = 0.3) -> np.ndarray:
    """Positive density and pressure with low-order random Fourier modes plus
    random velocities; periodic in the unit box."""
    rng = np.random.default_rng(seed)
    x, y, z = spec.centers()
    if spec.ndim == 2:
        x, y = x[0], y[0]
        z = np.zeros_like(x)

    def field(base):
        f = np.full(x.shape, base)
        for _ in range(3):
            kx, ky, kz = rng.integers(1, 3, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            kz = kz if spec.ndim == 3 else 0
            f = f + amp * base * rng.uniform(-1, 1) * np.sin(2 * np.pi * (kx * x + ky * y + kz * z) + ph) / 3
        return f

    rho = field(1.0)
    p = field(1.0)
    vel = [field(0.0) + rng.uniform(-0.5, 0.5) for _ in range(spec.ndim)]
    return to_blocks(spec, _globalize(spec, cons_from_prim_global(spec, rho, vel, p)))


def random_blocky_state(spec: MeshSpec, seed: int) -> np.ndarray:
    """Piecewise-constant random states on a coarse lattice (strong jumps in
    every direction, ratios up to 100 in pressure): exercises limiter and
    upwind branches."""
    rng = np.random.default_rng(seed)
    n = spec.ncells
    shape = (n[2], n[1], n[0]) if spec.ndim == 3 else (n[1], n[0])
    coarse = tuple(max(1, s // 3) for s in shape)
    def pick(lo, hi, log=False):
        c = rng.uniform(np.log(lo), np.log(hi), size=coarse) if log else rng.uniform(lo, hi, size=coarse)
        c = np.exp(c) if log else c
        for ax, s in enumerate(shape):
            c = np.repeat(c, -(-s // c.shape[ax]), axis=ax)
        return c[tuple(slice(0, s) for s in shape)]
    rho = pick(0.1, 10.0, log=True)
    p = pick(0.01, 1.0, log=True)
    vel = [pick(-1.0, 1.0) for _ in range(spec.ndim)]
    return to_blocks(spec, _globalize(spec, cons_from_prim_global(spec, rho, vel, p)))


def mirror(spec: MeshSpec, Ub: np.ndarray, axis: int) -> np.ndarray:
    """Reflect a block state across the mid-plane of `axis` (0 = x), flipping
    the sign of the momentum component along that axis."""
    Ug = from_blocks(spec, Ub)
    ax = 3 - axis                                   # [var, k, j, i]
    Ug = np.flip(Ug, axis=ax).copy()
    Ug[1 + axis] = -Ug[1 + axis]
    return to_blocks(spec, Ug)


def swap_axes(spec: MeshSpec, Ub: np.ndarray, a: int, b: int) -> np.ndarray:
    """Exchange coordinate axes a and b (and the matching momenta); the mesh
    must have equal cell counts and block sizes on both axes."""
    Ug = from_blocks(spec, Ub)
    Ug = np.swapaxes(Ug, 3 - a, 3 - b).copy()
    Ug[[1 + a, 1 + b]] = Ug[[1 + b, 1 + a]]
    return to_blocks(spec, Ug)


# ------------------------------------------------------------------ benchmark-size problems

def sedov128_packets(packet_blocks: int = 64):
    """3D Sedov, 128^3 cells as 512 blocks of 16^3, packets of 64 blocks in
    block-id order, 10 steps."""
    spec = sedov_spec(128, 16)
    ids = np.arange(spec.nblocks, dtype=np.int32)
    packets = [ids[i:i + packet_blocks] for i in range(0, spec.nblocks, packet_blocks)]
    return spec, packets


def sedov256_uneven_packets(seed: int = 0):
    """3D Sedov, 256^3 cells as 4096 blocks of 16^3; packet sizes drawn
    seed-uniform in [1, 256] until they cover every block (the last one is
    truncated); blocks assigned in id order."""
    spec = sedov_spec(256, 16)
    rng = np.random.default_rng(seed)
    sizes = []
    tot = 0
    while tot < spec.nblocks:
        s = int(rng.integers(1, 257))
        s = min(s, spec.nblocks - tot)
        sizes.append(s)
        tot += s
    ids = np.arange(spec.nblocks, dtype=np.int32)
    packets, o = [], 0
    for s in sizes:
        packets.append(ids[o:o + s])
        o += s
    return spec, packets


# ------------------------------------------------------------------ serving requests

def most_cubic(K: int) -> tuple:
    """Factor K = nbx * nby * nbz with nbx >= nby >= nbz, as close to a cube as
    possible (smallest nbx - nbz, then smallest nbx)."""
    best = None
    for nz in range(1, K + 1):
        if nz * nz * nz > K:
            break
        if K % nz:
            continue
        r = K // nz
        for ny in range(nz, r + 1):
            if ny * ny > r:
                break
            if r % ny:
                continue
            nx = r // ny
            key = (nx - nz, nx)
            if best is None or key < best[0]:
                best = (key, (nx, ny, nz))
    return best[1]


def region_mask(spec: MeshSpec, kind: int, region) -> np.ndarray:
    """Inside-cell mask [k, j, i] of a two-region initial state, with the
    integer rule of the device recipe: cell g (global index) is inside when
    sum_d (2 g_d + 1 - region[d])^2 <= region[3] (kind 1, sphere, half-cell
    units), or when g[region[0]] < region[1] (kind 2, half-space)."""
    n = spec.ncells
    gk, gj, gi = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    g = (gi, gj, gk)
    if kind == 1:
        d2 = np.zeros(gi.shape, dtype=np.int64)
        for d in range(spec.ndim):
            t = 2 * g[d].astype(np.int64) + 1 - int(region[d])
            d2 += t * t
        return d2 <= int(region[3])
    return g[int(region[0])] < int(region[1])


def sphere_count(spec: MeshSpec, region) -> int:
    """Number of cells inside a sphere region (same rule as region_mask, kind
    1), counted over the window of cells the sphere can reach."""
    r = int(np.floor(np.sqrt(region[3]))) + 1
    ax = []
    for d in range(spec.ndim):
        lo = max(0, (int(region[d]) - 1 - r) // 2 - 1)
        hi = min(spec.ncells[d], (int(region[d]) - 1 + r) // 2 + 2)
        ax.append(np.arange(lo, hi, dtype=np.int64))
    g = np.meshgrid(*ax, indexing="ij")
    d2 = sum((2 * g[d] + 1 - int(region[d])) ** 2 for d in range(spec.ndim))
    return int((d2 <= int(region[3])).sum())


def region_state(spec: MeshSpec, kind: int, region, u_in, u_out) -> np.ndarray:
    """Block array of a two-region initial state (same values as the device recipe)."""
    mask = region_mask(spec, kind, region)
    Ug = np.empty((spec.nvar,) + mask.shape)
    for v in range(spec.nvar):
        Ug[v] = np.where(mask, u_in[v], u_out[v])
    return to_blocks(spec, Ug)


def _cons(gamma, rho, p, ndim):
    u = [rho] + [0.0] * ndim + [p / (gamma - 1.0)]
    return (u + [0.0] * 5)[:5]


def serving_request(rng: np.random.Generator, max_blocks: int = 512, sizes=(8, 16, 32), nsteps: int = 1) -> dict:
    """One serving request: an independent 3D problem of K ~ U[1, max_blocks]
    blocks of b^3 cells (b ~ U{sizes}) laid out as the most cubic nbx >= nby >=
    nbz, cubic cells, outflow; Sedov-like (random centre and energy) or
    Sod-like (random axis and states) initial state as a two-region recipe."""
    K = int(rng.integers(1, max_blocks + 1))
    b = int(rng.choice(sizes))
    nb = most_cubic(K)
    ncell = [nb[d] * b for d in range(3)]
    L = max(ncell)
    spec = MeshSpec(ndim=3, nb=nb, bs=(b, b, b), hi=tuple(c / L for c in ncell))
    g = spec.gamma
    if rng.integers(0, 2) == 0:       # Sedov-like
        kind = 1
        c2 = [int(rng.integers(2, 2 * n - 1)) for n in ncell]
        r2 = 49                         # radius 3.5 cells
        region = (c2[0], c2[1], c2[2], r2)
        ndep = sphere_count(spec, region)
        energy = float(rng.uniform(0.5, 2.0))
        dV = spec.dx(0) ** 3
        p0 = 1e-5
        u_out = _cons(g, 1.0, p0, 3)
        u_in = list(u_out)
        u_in[4] = u_out[4] + energy / (ndep * dV)
    else:                               # Sod-like
        kind = 2
        axis = int(rng.integers(0, 3))
        region = (axis, ncell[axis] // 2, 0, 0)
        u_in = _cons(g, float(rng.uniform(0.5, 2.0)), float(rng.uniform(0.5, 2.0)), 3)
        u_out = _cons(g, float(rng.uniform(0.05, 0.5)), float(rng.uniform(0.05, 0.5)), 3)
    return dict(spec=spec, kind=kind, region=tuple(int(x) for x in region), u_in=tuple(u_in),
                u_out=tuple(u_out), nsteps=nsteps)


def serving_stream(n: int, rate: float, seed_arrivals: int = 1, seed_requests: int = 2, **kw):
    """n requests with exponential inter-arrival times of mean 1/rate (seconds)
    and request parameters from serving_request. For one seed the request
    sequence is the same at every rate and the arrival times scale as 1/rate."""
    ra = np.random.default_rng(seed_arrivals)
    rr = np.random.default_rng(seed_requests)
    t = np.cumsum(ra.exponential(1.0, size=n)) / rate
    return [(float(t[i]), serving_request(rr, **kw)) for i in range(n)]


def ramp_state(spec: MeshSpec, var: str, delta: float = 0.1, u: float = 10.0, base: float = 1.0) -> np.ndarray:
    """Uniform flow u along x with a linear ramp along x in one primitive:
    var = "p": rho = base, p = delta (i + 1); var = "rho": p = base,
    rho = delta (i + 1) (i the global x index); v = w = 0. Initial data of the
    first-order fallback cases (a large time step drives the low end of the
    ramp's Hancock face states negative)."""
    x, y, z = spec.centers()
    if spec.ndim == 2:
        x = x[0]
    ramp = np.broadcast_to(delta * (np.arange(spec.ncells[0]) + 1.0), x.shape)
    flat = np.full(x.shape, base)
    rho, p = (flat, ramp) if var == "p" else (ramp, flat)
    vel = [np.full(x.shape, u)] + [np.zeros(x.shape)] * (spec.ndim - 1)
    return to_blocks(spec, _globalize(spec, cons_from_prim_global(spec, rho, vel, p)))


# ------------------------------------------------------------------ two-level meshes

def fine_spec(spec: MeshSpec) -> MeshSpec:
    """The fine level of a two-level mesh as a uniform mesh: twice the blocks
    per active axis, the same block size, half the cell width."""
    nb = tuple(2 * spec.nb[d] if d < spec.ndim else spec.nb[d] for d in range(3))
    return replace(spec, nb=nb)


def refined_blocks(spec: MeshSpec, kind: str = "sphere", frac: float = 0.3) -> np.ndarray:
    """Coarse block ids to refine: blocks whose centres lie within radius frac
    of the domain centre ("sphere"), or in the upper half along x ("half")."""
    ids = []
    for b in range(spec.nblocks):
        bc = (b % spec.nb[0], (b // spec.nb[0]) % spec.nb[1], b // (spec.nb[0] * spec.nb[1]))
        c = [(bc[d] + 0.5) / spec.nb[d] if d < spec.ndim else 0.5 for d in range(3)]
        if kind == "sphere":
            inside = sum((c[d] - 0.5) ** 2 for d in range(spec.ndim)) <= frac ** 2
        else:
            inside = c[0] > 0.5
        if inside:
            ids.append(b)
    return np.array(ids, dtype=np.int32)


def amr_split(spec: MeshSpec, refined, Ub_fine: np.ndarray):
    """Initial data of a two-level mesh from a state on the uniform fine mesh
    (block array of fine_spec(spec)): the coarse state is the mean of each
    2^ndim group of fine cells, the fine state holds the children of the
    refined blocks [refined index * 2^ndim + octant][var][k][j][i] (octant bits
    x | y << 1 | z << 2)."""
    fs = fine_spec(spec)
    G = from_blocks(fs, Ub_fine)                  # var, z, y, x
    nv = spec.nvar
    if spec.ndim == 3:
        Gc = G.reshape(nv, G.shape[1] // 2, 2, G.shape[2] // 2, 2, G.shape[3] // 2, 2).mean(axis=(2, 4, 6))
    else:
        Gc = G.reshape(nv, 1, G.shape[2] // 2, 2, G.shape[3] // 2, 2).mean(axis=(3, 5))
    U0 = to_blocks(spec, Gc)
    nch = 1 << spec.ndim
    U1 = np.empty((len(refined) * nch,) + spec.block_shape()[1:])
    for r, b in enumerate(refined):
        bc = (b % spec.nb[0], (b // spec.nb[0]) % spec.nb[1], b // (spec.nb[0] * spec.nb[1]))
        for o in range(nch):
            fc = [2 * bc[d] + ((o >> d) & 1) if d < spec.ndim else 0 for d in range(3)]
            fb = fc[0] + fs.nb[0] * (fc[1] + fs.nb[1] * fc[2])
            U1[r * nch + o] = Ub_fine[fb]
    return U0, U1

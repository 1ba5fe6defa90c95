"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module draws the random scattering media, the source vector ``g``, the
frequency lists and the output-plane positions.  It holds none of the
method's arithmetic: no operator, no averaging of the permittivity onto the
staggered grid, no damping profile and no time integration.  Everything it
returns is an *input* of the problem ``y' = -A y + sin(Omega t) g``
(Sect. 2.1, eqs. (mxw), (src), (ode)).

Workload structure mirrors the paper's test problem (Sect. 4.1): randomly
placed, non-overlapping round inclusions with permittivity contrast 1 : 2.25,
an absorbing layer at the two ends of the propagation axis, perfectly
conducting walls, and a sine source on one line (2D) or plane (3D).  The
paper's own 750-cylinder geometry is not published; these seeded media
stand in for it.

Random numbers come from PCG32 (O'Neill 2014, "PCG: a family of simple fast
space-efficient statistically good algorithms for random number
generation"), implemented here from its published definition.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

_M64 = (1 << 64) - 1
_PCG_MULT = 6364136223846793005


class PCG32:
    """PCG-XSH-RR 64/32 generator (published definition)."""

    def __init__(self, seed: int, seq: int = 54):
        self.state = 0
        self.inc = ((seq << 1) | 1) & _M64
        self._step()
        self.state = (self.state + (seed & _M64)) & _M64
        self._step()

    def _step(self) -> None:
        self.state = (self.state * _PCG_MULT + self.inc) & _M64

    def next_u32(self) -> int:
        old = self.state
        self._step()
        xorshifted = (((old >> 18) ^ old) >> 27) & 0xFFFFFFFF
        rot = old >> 59
        return ((xorshifted >> rot) | (xorshifted << ((-rot) & 31))) & 0xFFFFFFFF

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """Uniform double in [lo, hi) from 53 random bits."""
        a = self.next_u32() >> 5
        b = self.next_u32() >> 6
        u = (a * 67108864.0 + b) / 9007199254740992.0
        return lo + (hi - lo) * u

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive), by rejection."""
        span = hi - lo + 1
        limit = (1 << 32) - ((1 << 32) % span)
        while True:
            r = self.next_u32()
            if r < limit:
                return lo + (r % span)

    def normal_array(self, size: int) -> np.ndarray:
        """Standard normal samples by the Box-Muller transform."""
        out = np.empty(size)
        for i in range(0, size, 2):
            u1 = max(self.uniform(), 1e-300)
            u2 = self.uniform()
            r = math.sqrt(-2.0 * math.log(u1))
            out[i] = r * math.cos(2.0 * math.pi * u2)
            if i + 1 < size:
                out[i + 1] = r * math.sin(2.0 * math.pi * u2)
        return out


#: Vacuum angular frequency of a 16-cell wavelength (c = 1, cell size 1).
OMEGA0 = 2.0 * math.pi / 16.0

PEC = 1
PERIODIC = 0


@dataclass
class Grid:
    """Geometry of one Yee grid.

    ``n`` = cells per axis (x, y[, z]).  ``bc[a]`` is PEC or PERIODIC for axis
    a.  The absorbing layer lies inside the grid at both ends of
    ``layer_axis`` and is ``layer_cells`` thick; ``sigma_max`` is its peak
    conductivity (linear ramp).  ``pml = 1`` (2D, layer along x) selects the
    paper's perfectly matched layer instead: a fourth field P on the Ez
    nodes and a quadratic conductivity profile.
    """

    dim: int
    n: Tuple[int, ...]
    bc: Tuple[int, ...]
    layer_axis: int
    layer_cells: int
    sigma_max: float
    pml: int = 0

    @property
    def ncell(self) -> int:
        return int(np.prod(self.n))

    @property
    def ncomp(self) -> int:
        return (3 + self.pml) if self.dim == 2 else 6

    @property
    def nunk(self) -> int:
        return self.ncomp * self.ncell

    @property
    def shape(self) -> Tuple[int, ...]:
        """numpy shape of one component array: slowest axis first."""
        return tuple(reversed(self.n))


@dataclass
class Scenario:
    grid: Grid
    eps_cell: np.ndarray          # per-cell relative permittivity, shape grid.shape
    g: np.ndarray                 # source vector, length grid.nunk
    omegas: np.ndarray            # angular frequencies, alpha(t) = sin(Omega t)
    T: float                      # final time
    krylov_dim: int
    plane: Tuple[int, int]        # (axis, index) of the output plane
    name: str = ""
    inclusions: List[Tuple] = field(default_factory=list)
    overlap_allowed_after: Optional[int] = None


def _place_disks_2d(rng: PCG32, n: int, region, count, rmin, rmax, gap,
                    max_reject=2000):
    (xlo, xhi), (ylo, yhi) = region
    disks = []
    rejects = 0
    overlap_from = None
    while len(disks) < count:
        r = rng.uniform(rmin, rmax)
        cx = rng.uniform(xlo + r, xhi - r)
        cy = rng.uniform(ylo + r, yhi - r)
        ok = True
        if rejects < max_reject:
            for (ox, oy, orr) in disks:
                if math.hypot(cx - ox, cy - oy) < r + orr + gap:
                    ok = False
                    break
        elif overlap_from is None:
            overlap_from = len(disks)
        if ok:
            disks.append((cx, cy, r))
            rejects = 0
        else:
            rejects += 1
    return disks, overlap_from


def _raster_disks(n, disks, eps_in, eps_bg):
    ny, nx = n, n
    eps = np.full((ny, nx), eps_bg)
    xc = np.arange(nx) + 0.5
    yc = np.arange(ny) + 0.5
    X, Y = np.meshgrid(xc, yc)
    for (cx, cy, r) in disks:
        eps[(X - cx) ** 2 + (Y - cy) ** 2 < r * r] = eps_in
    return eps


def _place_spheres_3d(rng: PCG32, n, zlo, zhi, fill, rmin, rmax, eps_choices,
                      eps_bg, gap, max_reject=2000):
    """Random sequential addition of spheres, periodic in x and y.

    Stops once the rasterised fill fraction of the slab zlo <= z < zhi reaches
    ``fill``.  After ``max_reject`` consecutive rejections overlap is allowed.
    """
    eps = np.full((n, n, n), eps_bg)
    centres = np.zeros((0, 3))
    radii = np.zeros(0)
    spheres = []
    slab_cells = n * n * (zhi - zlo)
    filled = 0
    rejects = 0
    overlap_from = None
    c = np.arange(n) + 0.5
    batch = 1
    while filled < fill * slab_cells:
        # candidates are drawn in batches; the first one that overlaps no
        # placed sphere is accepted and the rest of the batch is discarded
        cand = []
        for _ in range(batch):
            r = rng.uniform(rmin, rmax)
            cx = rng.uniform(0.0, n)
            cy = rng.uniform(0.0, n)
            cz = rng.uniform(zlo + r, zhi - r)
            e_in = eps_choices[rng.randint(0, len(eps_choices) - 1)] if len(eps_choices) > 1 else eps_choices[0]
            cand.append((r, cx, cy, cz, e_in))
        cb = np.array([q[:4] for q in cand])
        if rejects < max_reject and len(radii):
            d = centres[None, :, :] - cb[:, None, 1:4]
            d[:, :, 0] -= n * np.round(d[:, :, 0] / n)
            d[:, :, 1] -= n * np.round(d[:, :, 1] / n)
            dist = np.sqrt((d * d).sum(2))
            ok = np.all(dist >= radii[None, :] + cb[:, 0:1] + gap, axis=1)
        else:
            if rejects >= max_reject and overlap_from is None:
                overlap_from = len(spheres)
            ok = np.ones(batch, bool)
        if not ok.any():
            rejects += batch
            batch = min(2 * batch, 64)      # near jamming: test more candidates at once
            continue
        r, cx, cy, cz, e_in = cand[int(np.argmax(ok))]
        batch = max(1, batch // 2)
        rejects = 0
        centres = np.vstack([centres, [cx, cy, cz]])
        radii = np.append(radii, r)
        spheres.append((cx, cy, cz, r, e_in))
        # raster: cell centre inside the sphere (minimum image in x and y)
        k0 = max(int(math.floor(cz - r)), 0)
        k1 = min(int(math.ceil(cz + r)), n)
        dz = c[k0:k1] - cz
        # bounding box in x and y, indices wrapped periodically
        ix = np.arange(int(math.floor(cx - r)), int(math.ceil(cx + r)) + 1) % n
        iy = np.arange(int(math.floor(cy - r)), int(math.ceil(cy + r)) + 1) % n
        ix, iy = np.unique(ix), np.unique(iy)
        dx = c[ix] - cx
        dx -= n * np.round(dx / n)
        dy = c[iy] - cy
        dy -= n * np.round(dy / n)
        inside = (dz[:, None, None] ** 2 + dy[None, :, None] ** 2
                  + dx[None, None, :] ** 2) < r * r
        sub = eps[k0:k1][:, iy][:, :, ix]
        newly = inside & (sub == eps_bg)
        filled += int(newly.sum())
        sub[inside] = e_in
        eps[k0:k1, iy[:, None], ix[None, :]] = sub
    return eps, spheres, overlap_from


def source_2d(grid: Grid, ix: int) -> np.ndarray:
    """Line source on the Ez nodes at x = ix.

    Mirrors the paper's source (Sect. 4.1): value 1 on the inner 8/10 of the
    line and a linear taper to 0 over the outer 1/10 next to each conducting
    wall.  Vector layout [Hx, Hy, Ez], each component (ny, nx) x-fastest.
    """
    nx, ny = grid.n
    g = np.zeros(grid.nunk)
    ez = g[2 * grid.ncell:3 * grid.ncell].reshape(ny, nx)
    edge = ny / 10.0
    for j in range(ny):
        y = float(j)
        if y < edge:
            val = y / edge
        elif y > ny - edge:
            val = (ny - y) / edge
        else:
            val = 1.0
        ez[j, ix] = val
    return g


def source_3d(grid: Grid, kz: int) -> np.ndarray:
    """Ex-polarised plane source: value 1 on every Ex node of plane z = kz.

    Vector layout [Hx, Hy, Hz, Ex, Ey, Ez], each component (nz, ny, nx).
    """
    nx, ny, nz = grid.n
    g = np.zeros(grid.nunk)
    ex = g[3 * grid.ncell:4 * grid.ncell].reshape(nz, ny, nx)
    ex[kz, :, :] = 1.0
    return g


def config_2d(n=64, seed=1708, ndisks=40, T=200.0, m=30, omegas=None) -> Scenario:
    """2D (Hx, Hy, Ez) waveguide: 40 random eps=2.25 disks of radius 2-4
    cells in eps=1, PEC on all outer walls, a 6-cell linear absorbing layer
    (sigma_max = 1) at both x ends, a tapered line source."""
    L = 6 if n >= 32 else max(2, n // 8)
    grid = Grid(2, (n, n), (PEC, PEC), 0, L, 1.0)
    rng = PCG32(seed)
    xs = L + 1
    xo = n - L - 2
    region = ((xs + 2.0, xo - 2.0), (1.0, n - 1.0))
    rmin, rmax = (2.0, 4.0) if n >= 32 else (1.0, 2.0)
    disks, ov = _place_disks_2d(rng, n, region, ndisks, rmin, rmax, 1.0)
    eps = _raster_disks(n, disks, 2.25, 1.0)
    g = source_2d(grid, xs)
    om = np.array([OMEGA0]) if omegas is None else np.asarray(omegas, float)
    return Scenario(grid, eps, g, om, T, m, (0, xo), f"2d_n{n}", disks, ov)


def config_2d_pml(n=64, seed=1708, ndisks=40, T=200.0, m=30, omegas=None, sigma_max=3.0) -> Scenario:
    """The medium and source of ``config_2d`` with the paper's perfectly
    matched layer (auxiliary field P, quadratic conductivity rising to
    sigma_max over the 6-cell layer at both x ends) instead of the lossy
    layer."""
    sc = config_2d(n=n, seed=seed, ndisks=ndisks, T=T, m=m, omegas=omegas)
    g0 = sc.grid
    grid = Grid(2, g0.n, g0.bc, g0.layer_axis, g0.layer_cells, sigma_max, pml=1)
    g = np.zeros(grid.nunk)
    g[:g0.nunk] = sc.g
    return Scenario(grid, sc.eps_cell, g, sc.omegas, T, m, sc.plane, f"2d_pml_n{n}", sc.inclusions,
                    sc.overlap_allowed_after)


def config_3d(n=64, seed=1709, fill=0.3, T=400.0, m=64, omegas=None,
              rmin=2.0, rmax=5.0, eps_choices=(2.25,), layer=8) -> Scenario:
    """3D Yee grid: random spheres (radius rmin-rmax cells) of eps from
    ``eps_choices`` in eps=1 at volume fraction ``fill`` of the scattering
    slab, periodic in x and y, a linear absorbing layer (sigma_max = 1) at
    both z ends backed by PEC, an Ex plane source."""
    L = layer if n >= 32 else max(2, n // 8)
    grid = Grid(3, (n, n, n), (PERIODIC, PERIODIC, PEC), 2, L, 1.0)
    rng = PCG32(seed)
    ks = L + 1
    ko = n - L - 2
    zlo, zhi = ks + 2, ko - 1
    if n < 32:
        rmin, rmax = min(rmin, 1.0), min(rmax, 2.0)
    eps, spheres, ov = _place_spheres_3d(rng, n, zlo, zhi, fill, rmin, rmax,
                                         list(eps_choices), 1.0, 0.0)
    g = source_3d(grid, ks)
    om = np.array([OMEGA0]) if omegas is None else np.asarray(omegas, float)
    return Scenario(grid, eps, g, om, T, m, (2, ko), f"3d_n{n}", spheres, ov)


def freq_list(count: int, lo: float = 0.8, hi: float = 1.2) -> np.ndarray:
    """``count`` angular frequencies spread uniformly over [lo, hi] * OMEGA0."""
    if count == 1:
        return np.array([OMEGA0])
    return OMEGA0 * np.linspace(lo, hi, count)


def random_vector(n: int, seed: int) -> np.ndarray:
    """Seeded standard-normal vector (numpy's PCG64 stream, for test inputs)."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(n)


def masked_random_vector(grid: Grid, seed: int) -> np.ndarray:
    """Random field vector with zeros on the conducting-wall nodes.

    A node is on a wall when its component has an integer coordinate along a
    PEC axis and its index along that axis is 0 (the wall plane; index n
    wraps onto it).  This is geometry of the input, not of the operator.
    """
    v = random_vector(grid.nunk, seed)
    return v * wall_keep_mask(grid)


def component_offsets(dim: int):
    """Staggered offsets (in cells) of each stored component along x, y[, z].

    2D (Hx, Hy, Ez): E at grid vertices, H at edge centres (Sect. 2.1).
    3D (Hx, Hy, Hz, Ex, Ey, Ez): the textbook Yee cell.
    """
    if dim == 2:
        return [(0.0, 0.5), (0.5, 0.0), (0.0, 0.0)]
    return [(0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0),
            (0.5, 0.0, 0.0), (0.0, 0.5, 0.0), (0.0, 0.0, 0.5)]


def wall_keep_mask(grid: Grid) -> np.ndarray:
    """1 for unknowns of the system, 0 for nodes on a conducting wall."""
    keep = np.ones((grid.ncomp,) + grid.shape)
    offs = list(component_offsets(grid.dim))
    if grid.dim == 2 and grid.pml:
        offs.append(offs[2])          # P lives on the Ez nodes
    for c in range(grid.ncomp):
        for a in range(grid.dim):
            if grid.bc[a] == PEC and offs[c][a] == 0.0:
                sl = [slice(None)] * grid.dim
                sl[grid.dim - 1 - a] = 0
                keep[c][tuple(sl)] = 0.0
    return keep.reshape(-1)


def uneven_batch(count=48, seed=1711, nmin=32, nmax=96, step=1):
    """Instances for the uneven batch: cubic sizes drawn uniformly from
    {nmin, nmin + step, ..., nmax}, inclusion permittivity from {2.25, 4},
    fill from U[0.2, 0.4], four frequencies each in [0.9, 1.1] * OMEGA0."""
    rng = PCG32(seed)
    out = []
    for b in range(count):
        n = nmin + step * rng.randint(0, (nmax - nmin) // step)
        e = 2.25 if rng.randint(0, 1) == 0 else 4.0
        f = rng.uniform(0.2, 0.4)
        out.append((n, e, f, seed * 1000 + b))
    return out


def config_uneven(count=48, seed=1711, nmin=32, nmax=96, T=400.0, m=64, nfreq=4, step=1):
    """The uneven batch: ``count`` 3D instances with cubic sizes drawn from
    {nmin, nmin + step, ..., nmax}, inclusion permittivity from {2.25, 4},
    fill U[0.2, 0.4], each with ``nfreq`` frequencies in [0.9, 1.1] * OMEGA0."""
    out = []
    for (n, e, f, s) in uneven_batch(count, seed, nmin, nmax, step):
        sc = config_3d(n=n, seed=s, fill=f, T=T, m=m, eps_choices=(e,))
        sc.omegas = OMEGA0 * np.linspace(0.9, 1.1, nfreq)
        sc.name = f"uneven_n{n}_e{e}_f{f:.2f}"
        out.append(sc)
    return out

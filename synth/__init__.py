"""Seeded synthetic inputs for the WRI augmented-system workloads.

This module is shared by the CPU oracle's tests and by the GPU path's tests and
benchmark.  It holds no arithmetic of the method itself (no operator, no solve,
no gradient): only grids, velocity models, acquisition geometry, source weights,
random vectors and synthetic receiver traces, all drawn from numpy's PCG64
generator with a stated seed.

Conventions (shared with every consumer):
  * computational grid = physical grid + ``npml`` padding cells on each of the
    six faces; arrays are C-ordered ``[nz][ny][nx]`` so the linear node index is
    ``(k*ny + j)*nx + i`` with ``x`` fastest;
  * velocities in m/s, squared slowness ``m = 1/v**2`` in s^2/m^2;
  * source and receiver positions are grid nodes, given as physical-grid
    coordinates and converted to computational linear indices here.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "GridSpec", "Group", "rng", "grid", "pad_pml", "to_m",
    "velocity_homogeneous", "velocity_gaussian_anomaly", "velocity_layered",
    "velocity_salt", "node_index", "surface_sources", "borehole_receivers",
    "source_weights", "random_complex", "synthetic_traces",
    "workload_c1", "workload_c2", "workload_c3", "workload_c4", "workload_c5",
    "workload_camembert_shape", "workload_small",
]


def rng(seed: int) -> np.random.Generator:
    """PCG64 generator; every input of the project is drawn from one of these."""
    return np.random.Generator(np.random.PCG64(seed))


@dataclass(frozen=True)
class GridSpec:
    """Physical grid ``nphys`` (x, y, z) with ``npml`` padding cells per face."""

    nphys: tuple
    npml: int
    h: float

    @property
    def nx(self) -> int:
        return self.nphys[0] + 2 * self.npml

    @property
    def ny(self) -> int:
        return self.nphys[1] + 2 * self.npml

    @property
    def nz(self) -> int:
        return self.nphys[2] + 2 * self.npml

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self) -> tuple:
        """Array shape ``(nz, ny, nx)``."""
        return (self.nz, self.ny, self.nx)


def grid(nphys, npml: int, h: float) -> GridSpec:
    if isinstance(nphys, int):
        nphys = (nphys, nphys, nphys)
    return GridSpec(tuple(int(v) for v in nphys), int(npml), float(h))


def pad_pml(v_phys: np.ndarray, npml: int) -> np.ndarray:
    """Extend a physical-grid array ``[z][y][x]`` into the padding by edge copy."""
    return np.pad(v_phys, npml, mode="edge")


def to_m(v: np.ndarray) -> np.ndarray:
    """Squared slowness from velocity (float64)."""
    return 1.0 / np.asarray(v, dtype=np.float64) ** 2


def _phys_coords(g: GridSpec):
    nxp, nyp, nzp = g.nphys
    z, y, x = np.meshgrid(np.arange(nzp), np.arange(nyp), np.arange(nxp), indexing="ij")
    return x, y, z


def velocity_homogeneous(g: GridSpec, v: float) -> np.ndarray:
    return np.full(g.shape, float(v))


def velocity_gaussian_anomaly(g: GridSpec, v0: float, amp: float = 0.10, sigma_cells: float = 3.0,
                              seed: int = 0, lo: float = 8.0, hi: float = 16.0) -> np.ndarray:
    """Homogeneous ``v0`` plus ``amp*v0`` Gaussian bump; centre uniform in [lo, hi]^3 cells."""
    r = rng(seed)
    c = r.uniform(lo, hi, size=3)
    x, y, z = _phys_coords(g)
    d2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
    v = v0 * (1.0 + amp * np.exp(-0.5 * d2 / sigma_cells ** 2))
    return pad_pml(v, g.npml)


def velocity_layered(g: GridSpec, vs=(1500.0, 2000.0, 2500.0, 3000.0), seed: int = 1,
                     anomaly_amp: float = 0.10, anomaly_sigma: float = 4.0) -> np.ndarray:
    """Flat layers with seeded interface depths plus one seeded Gaussian anomaly."""
    r = rng(seed)
    nxp, nyp, nzp = g.nphys
    nl = len(vs)
    # interfaces drawn in ordered depth bands so every layer has some thickness
    edges = np.linspace(0, nzp, nl + 1)
    cuts = [int(r.uniform(edges[i] + 0.25 * (edges[i + 1] - edges[i]),
                          edges[i + 1] - 0.25 * (edges[i + 1] - edges[i]))) for i in range(nl - 1)]
    x, y, z = _phys_coords(g)
    v = np.full((nzp, nyp, nxp), float(vs[0]))
    for i, c in enumerate(cuts):
        v[z >= c] = vs[i + 1]
    cen = r.uniform(0.3, 0.7, size=3) * np.array([nxp, nyp, nzp])
    d2 = (x - cen[0]) ** 2 + (y - cen[1]) ** 2 + (z - cen[2]) ** 2
    v = v * (1.0 + anomaly_amp * np.exp(-0.5 * d2 / anomaly_sigma ** 2))
    return pad_pml(v, g.npml)


def velocity_salt(g: GridSpec, seed: int = 5, v_top: float = 1800.0, v_bot: float = 3500.0,
                  v_salt: float = 4500.0) -> np.ndarray:
    """Linear-in-depth background with a salt-like body: union of 3 seeded ellipsoids."""
    r = rng(seed)
    nxp, nyp, nzp = g.nphys
    x, y, z = _phys_coords(g)
    v = v_top + (v_bot - v_top) * z / max(nzp - 1, 1)
    body = np.zeros(v.shape, dtype=bool)
    for _ in range(3):
        c = r.uniform(0.3, 0.7, size=3) * np.array([nxp, nyp, nzp])
        ax = r.uniform(0.08, 0.2, size=3) * np.array([nxp, nyp, nzp])
        body |= ((x - c[0]) / ax[0]) ** 2 + ((y - c[1]) / ax[1]) ** 2 + ((z - c[2]) / ax[2]) ** 2 <= 1.0
    v = np.where(body, v_salt, v)
    return pad_pml(v, g.npml)


def node_index(g: GridSpec, ix: int, iy: int, iz: int) -> int:
    """Computational linear index of physical node (ix, iy, iz)."""
    p = g.npml
    return int(((iz + p) * g.ny + (iy + p)) * g.nx + (ix + p))


def surface_sources(g: GridSpec, xs, ys, z: int) -> np.ndarray:
    return np.array([node_index(g, x, y, z) for y in ys for x in xs], dtype=np.int64)


def borehole_receivers(g: GridSpec, x: int, y: int, zs) -> np.ndarray:
    return np.array([node_index(g, x, y, z) for z in zs], dtype=np.int32)


def source_weights(nsys: int, seed: int) -> np.ndarray:
    """Complex weights: amplitude U(5, 15), phase U(-pi, pi)."""
    r = rng(seed)
    a = r.uniform(5.0, 15.0, nsys)
    ph = r.uniform(-np.pi, np.pi, nsys)
    return a * np.exp(1j * ph)


def random_complex(shape, seed: int) -> np.ndarray:
    """Standard complex Gaussian (complex128)."""
    r = rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


def synthetic_traces(g: GridSpec, src: np.ndarray, rec_off: np.ndarray, rec_idx: np.ndarray,
                     freq: float, v_ref: float, alpha: np.ndarray, seed: int,
                     noise: float = 0.02) -> np.ndarray:
    """Receiver traces for grids too large for a direct forward solve.

    Geometric spreading and travel-time phase of a homogeneous ``v_ref`` medium,
    scaled by the per-system weight, plus 2 % seeded complex noise.  These are
    inputs only: nothing checks a solve against them.
    """
    r = rng(seed)
    out = np.zeros(int(rec_off[-1]), dtype=np.complex128)
    k = 2 * np.pi * freq / v_ref
    for s in range(len(src)):
        sz, rem = divmod(int(src[s]), g.ny * g.nx)
        sy, sx = divmod(rem, g.nx)
        idx = rec_idx[rec_off[s]:rec_off[s + 1]].astype(np.int64)
        rz, rem = np.divmod(idx, g.ny * g.nx)
        ry, rx = np.divmod(rem, g.nx)
        dist = g.h * np.sqrt((rx - sx) ** 2 + (ry - sy) ** 2 + (rz - sz) ** 2) + 0.5 * g.h
        tr = -alpha[s] * g.h ** 3 * np.exp(1j * k * dist) / (4 * np.pi * dist)
        n = len(idx)
        tr = tr * (1 + noise * (r.standard_normal(n) + 1j * r.standard_normal(n)))
        out[rec_off[s]:rec_off[s + 1]] = tr
    return out


@dataclass
class Group:
    """One frequency group: a grid, a model and ``nsys`` (source, frequency) systems."""

    spec: GridSpec
    freq: float
    v: np.ndarray                 # computational-grid velocity [nz][ny][nx]
    src: np.ndarray               # int64 [nsys] linear node index
    rec_off: np.ndarray           # int32 [nsys+1]
    rec_idx: np.ndarray           # int32 [nnz]
    lam: float
    v_max: float
    pml_R: float = 1e-3
    alpha: np.ndarray = field(default=None)   # known / true weights, complex128 [nsys]
    d: np.ndarray = field(default=None)       # complex128 [nnz] or None (computed by a forward solve)

    @property
    def omega(self) -> float:
        return 2 * np.pi * self.freq

    @property
    def nsys(self) -> int:
        return len(self.src)

    @property
    def m(self) -> np.ndarray:
        return to_m(self.v)


def _shared_receivers(nsys: int, rec: np.ndarray):
    off = np.arange(nsys + 1, dtype=np.int32) * len(rec)
    return off, np.tile(rec.astype(np.int32), nsys)


def default_lambda(h: float) -> float:
    """Data weight used by the synthetic workloads: 1/h^2, the scale of the
    stencil's off-diagonal entries, so data and PDE rows are balanced."""
    return 1.0 / h ** 2


def workload_small(nphys=8, npml=4, h=10.0, freq=15.0, nsys=2, seed=11, v=2000.0,
                   lam=None, nrec=6) -> Group:
    """Small seeded case for oracle checks and kernel parity (several tiles at nphys>=16)."""
    g = grid(nphys, npml, h)
    r = rng(seed)
    vel = velocity_gaussian_anomaly(g, v, seed=seed, lo=0.3 * min(g.nphys), hi=0.7 * min(g.nphys),
                                    sigma_cells=max(1.0, min(g.nphys) / 6))
    nxp, nyp, nzp = g.nphys
    src = np.array([node_index(g, int(r.integers(1, nxp - 1)), int(r.integers(1, nyp - 1)), 1)
                    for _ in range(nsys)], dtype=np.int64)
    zs = np.unique(r.integers(0, nzp, size=nrec))
    rx, ry = int(r.integers(0, nxp)), int(r.integers(0, nyp))
    rec = borehole_receivers(g, rx, ry, zs)
    # keep receivers off the source nodes
    off, idx = [0], []
    for s in range(nsys):
        keep = rec[rec != src[s]]
        idx.extend(keep.tolist())
        off.append(len(idx))
    return Group(g, freq, vel, src, np.array(off, np.int32), np.array(idx, np.int32),
                 lam if lam is not None else default_lambda(h), float(vel.max()),
                 alpha=source_weights(nsys, seed + 1))


def workload_c1() -> Group:
    """24^3 physical + 6 PML, h=10, v=2000, 5 Hz, source (12,12,2), 20 receivers at
    x=y=18, z=2..21, lambda=10, true model +10 % Gaussian anomaly (seed 0)."""
    g = grid(24, 6, 10.0)
    src = np.array([node_index(g, 12, 12, 2)], dtype=np.int64)
    rec = borehole_receivers(g, 18, 18, range(2, 22))
    off, idx = _shared_receivers(1, rec)
    v0 = velocity_homogeneous(g, 2000.0)
    grp = Group(g, 5.0, v0, src, off, idx, 10.0, 2000.0 * 1.1, alpha=np.array([-10.0 + 0j]))
    return grp


def workload_c1_true_velocity() -> np.ndarray:
    return velocity_gaussian_anomaly(grid(24, 6, 10.0), 2000.0, amp=0.10, sigma_cells=3.0, seed=0)


def workload_c2() -> list:
    """64^3 + 10 PML, h=10, layered model, 16 surface sources (4x4), 48 receivers
    at x=y=32, z=8..55, three groups 3/5/7 Hz, seeded unknown source weights."""
    g = grid(64, 10, 10.0)
    v = velocity_layered(g, seed=1)
    src = surface_sources(g, (8, 24, 40, 56), (8, 24, 40, 56), 2)
    rec = borehole_receivers(g, 32, 32, range(8, 56))
    off, idx = _shared_receivers(len(src), rec)
    out = []
    for j, f in enumerate((3.0, 5.0, 7.0)):
        al = source_weights(len(src), 100 + j)
        grp = Group(g, f, v, src, off, idx, default_lambda(g.h), float(v.max()), alpha=al)
        grp.d = synthetic_traces(g, src, off, idx, f, 2000.0, al, seed=200 + j)
        out.append(grp)
    return out


def workload_c3() -> Group:
    """96^3 + 10 PML, h=10, 32 surface sources (4x8), 48 receivers, 6 Hz."""
    g = grid(96, 10, 10.0)
    v = velocity_layered(g, seed=3)
    src = surface_sources(g, (12, 36, 60, 84), tuple(6 + 12 * i for i in range(8)), 2)
    rec = borehole_receivers(g, 48, 48, range(12, 84, 1)[:48])
    off, idx = _shared_receivers(len(src), rec)
    al = source_weights(len(src), 300)
    grp = Group(g, 6.0, v, src, off, idx, default_lambda(g.h), float(v.max()), alpha=al)
    grp.d = synthetic_traces(g, src, off, idx, 6.0, 2000.0, al, seed=301)
    return grp


def workload_c4(nsrc: int = 128, freqs=((3.0, 64), (5.0, 96), (8.0, 128)), nrec: int = 96,
                shard: int = 0) -> list:
    """Frequency-dependent grids over a 2560 m cube: 3 Hz 64^3 (h=40), 5 Hz 96^3
    (h=26.67), 8 Hz 128^3 (h=20), each + 10 PML; 128 surface sources (8x16 grid),
    96 borehole receivers, layered + anomaly model (seed 4).  ``shard`` > 0 draws the
    weights and traces of another shot record over the same geometry (seeds offset by
    1000 * shard), the share of one rank in a job of several such records."""
    out = []
    extent = 2560.0
    for j, (f, n) in enumerate(freqs):
        h = extent / n
        g = grid(n, 10, h)
        v = velocity_layered(g, seed=4)
        xs = tuple(int(round((i + 0.5) * n / 8)) for i in range(8))
        ys = tuple(int(round((i + 0.5) * n / 16)) for i in range(16))
        src = surface_sources(g, xs, ys, 2)[:nsrc]
        zs = np.unique(np.linspace(2, n - 3, nrec).round().astype(int))
        rec = borehole_receivers(g, n // 2 + 1, n // 2 + 1, zs)
        off, idx = _shared_receivers(len(src), rec)
        al = source_weights(len(src), 400 + j + 1000 * shard)
        grp = Group(g, f, v, src, off, idx, default_lambda(h), float(v.max()), alpha=al)
        grp.d = synthetic_traces(g, src, off, idx, f, 2000.0, al, seed=410 + j + 1000 * shard)
        out.append(grp)
    return out


def workload_c5(nsrc: int = 64) -> Group:
    """256x256x160 + 10 PML, h=8, salt body in a 1800-3500 m/s gradient, 64 sources,
    96 borehole receivers, 10 Hz."""
    g = grid((256, 256, 160), 10, 8.0)
    v = velocity_salt(g, seed=5)
    src = surface_sources(g, tuple(16 + 32 * i for i in range(8)), tuple(16 + 32 * i for i in range(8)), 2)[:nsrc]
    rec = borehole_receivers(g, 128, 128, np.linspace(2, 157, 96).round().astype(int))
    off, idx = _shared_receivers(len(src), rec)
    al = source_weights(len(src), 500)
    grp = Group(g, 10.0, v, src, off, idx, default_lambda(g.h), float(v.max()), alpha=al)
    grp.d = synthetic_traces(g, src, off, idx, 10.0, 2500.0, al, seed=501)
    return grp


def workload_camembert_shape(nphys: int = 61) -> Group:
    """Shape of the Camembert timing case: 3 km cube, h=50 (61^3) + 10 PML, 9 sources
    at z=0.35 km, 45x45 receivers at z=2.3 km, 5 Hz; velocities are our choice.  ``nphys`` = 60
    gives the nearest cube with an x extent (80) that is a multiple of 4."""
    g = grid(nphys, 10, 50.0)
    v = velocity_gaussian_anomaly(g, 2500.0, amp=0.1, sigma_cells=8.0, seed=7, lo=25, hi=35)
    src = surface_sources(g, (10, 30, 50), (10, 30, 50), 7)
    rx = np.linspace(8, 52, 45).round().astype(int)
    rec = np.array([node_index(g, x, y, 46) for y in rx for x in rx], dtype=np.int32)
    off, idx = _shared_receivers(len(src), rec)
    al = np.full(len(src), -10.0 + 0j)
    grp = Group(g, 5.0, v, src, off, idx, default_lambda(g.h), float(v.max()), alpha=al)
    grp.d = synthetic_traces(g, src, off, idx, 5.0, 2500.0, al, seed=71)
    return grp

"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle, the tests and the bench.

This module only draws random numbers and lays out points; it holds none of the
method's arithmetic (no wrapping, no minimum image, no binning, no histograms).

Box convention: upper-triangular box matrix with tilt factors (HOOMD style, the
code base the paper's cell list was adapted from, Section "General Utilities"):

    a1 = (Lx, 0, 0),  a2 = (xy*Ly, Ly, 0),  a3 = (xz*Lz, yz*Lz, Lz)

and the box is centred on the origin (listing "LAMMPS RDF" shifts data by L/2 to
reach that frame). A point with fractional coordinates s in [0,1)^3 sits at
M @ (s - 1/2).

Workloads (the paper benchmarks random points with about 12 neighbours inside
r = 1, Fig. 3 and Fig. 6; the sizes below scale that recipe):
  c1  cubic L=16, N=4096 uniform; ball r=4; RDF 100 bins [0,4]
  c2  triclinic (xy=0.1, xz=0.05) FCC 50^3 cells, a=1.5874, sigma=0.05; r=1.3; q4,q6; RDF 200 bins [0,5]
  c3  cubic rho=0.85, N=4,194,304 uniform; ball r=2.5 + RDF 500 bins [0,5]; kNN k=12
  c4  cubic L=64a, N=2^20: half perturbed FCC slab, half uniform liquid slab at density 1
  c5  256 frames, N log-uniform in [1e3, 2e5], cubic/triclinic, uniform/FCC
  p6  2D (Lz = 0) square box, 10 frames x 20,000 uniform points at 12 neighbours per
      unit disc, orientation angles uniform in [-pi, pi): the PMFT-vs-RDF system of Fig. 6

A 2D box has Lz = 0 (and xz = yz = 0); its points have z = 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
BCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
SC_BASIS = np.array([[0.0, 0.0, 0.0]])


@dataclass
class Box:
    Lx: float
    Ly: float
    Lz: float
    xy: float = 0.0
    xz: float = 0.0
    yz: float = 0.0

    @staticmethod
    def cube(L: float) -> "Box":
        return Box(L, L, L)

    @staticmethod
    def square(L: float, xy: float = 0.0) -> "Box":
        return Box(L, L, 0.0, xy)

    @property
    def is2D(self) -> bool:
        return self.Lz == 0.0

    @property
    def area(self) -> float:
        return self.Lx * self.Ly

    def matrix(self) -> np.ndarray:
        return np.array([[self.Lx, self.xy * self.Ly, self.xz * self.Lz],
                         [0.0, self.Ly, self.yz * self.Lz],
                         [0.0, 0.0, self.Lz]], dtype=np.float64)

    def params(self) -> np.ndarray:
        """(Lx, Ly, Lz, xy, xz, yz) as float64, the layout every entry point takes."""
        return np.array([self.Lx, self.Ly, self.Lz, self.xy, self.xz, self.yz], dtype=np.float64)

    @property
    def volume(self) -> float:
        return self.Lx * self.Ly * self.Lz


@dataclass
class Workload:
    name: str
    box: Box
    points: np.ndarray            # (N,3) float32, C-contiguous
    params: dict = field(default_factory=dict)


def _to_f32(x: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(x.astype(np.float32))


def frac_to_cart(box: Box, s: np.ndarray) -> np.ndarray:
    """Map fractional coordinates (rows) to Cartesian positions, box centred on 0."""
    return (s - 0.5) @ box.matrix().T


def uniform_points(rng: np.random.Generator, box: Box, n: int) -> np.ndarray:
    return _to_f32(frac_to_cart(box, rng.random((n, 3))))


def lattice_sites(n_cells, basis=FCC_BASIS) -> np.ndarray:
    """Fractional coordinates of an n_x*n_y*n_z supercell of a cubic lattice with `basis`."""
    nx, ny, nz = (n_cells, n_cells, n_cells) if np.isscalar(n_cells) else n_cells
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1).reshape(-1, 3)
    s = (g[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    return s / np.array([nx, ny, nz], dtype=np.float64)


def lattice_points(rng: np.random.Generator | None, box: Box, n_cells, sigma: float = 0.0,
                   basis=FCC_BASIS) -> np.ndarray:
    """Perturbed lattice in `box`: sites placed in fractional space then mapped with the box
    matrix (so a triclinic box holds a sheared, periodic-consistent crystal)."""
    x = frac_to_cart(box, lattice_sites(n_cells, basis))
    if sigma > 0.0:
        x = x + rng.normal(0.0, sigma, size=x.shape)
    return _to_f32(x)


def fcc_lattice_constant(density: float) -> float:
    return (4.0 / density) ** (1.0 / 3.0)


# ---------------------------------------------------------------------------------------
# The five workloads


def c1(seed: int = 1) -> Workload:
    rng = np.random.default_rng(seed)
    box = Box.cube(16.0)
    return Workload("c1_cubic16_uniform4096", box, uniform_points(rng, box, 4096),
                    dict(r_max=4.0, rdf_bins=100, rdf_r_max=4.0, rdf_r_min=0.0))


def c2(seed: int = 2, n_cells: int = 50) -> Workload:
    rng = np.random.default_rng(seed)
    a = 1.5874
    L = a * n_cells
    box = Box(L, L, L, xy=0.1, xz=0.05, yz=0.0)
    return Workload(f"c2_triclinic_fcc{4 * n_cells ** 3}", box,
                    lattice_points(rng, box, n_cells, sigma=0.05),
                    dict(r_max=1.3, ls=(4, 6), rdf_bins=200, rdf_r_max=5.0, rdf_r_min=0.0))


def c3(seed: int = 3, n: int = 4_194_304, density: float = 0.85) -> Workload:
    rng = np.random.default_rng(seed)
    L = (n / density) ** (1.0 / 3.0)
    box = Box.cube(L)
    return Workload(f"c3_cubic_uniform{n}", box, uniform_points(rng, box, n),
                    dict(r_max=2.5, rdf_bins=500, rdf_r_max=5.0, rdf_r_min=0.0, k=12))


def c4(seed: int = 4, n_cells: int = 64) -> Workload:
    """Half perturbed FCC (z < 0), half uniform liquid (z >= 0), density 1, N = 8*n_cells^3."""
    rng = np.random.default_rng(seed)
    a = fcc_lattice_constant(1.0)
    L = n_cells * a
    box = Box.cube(L)
    half = n_cells // 2
    s = lattice_sites((n_cells, n_cells, half))
    s[:, 2] *= 0.5                                  # crystal fills fractional z in [0, 1/2)
    xtal = frac_to_cart(box, s) + rng.normal(0.0, 0.05, size=s.shape)
    n_liq = s.shape[0]
    u = rng.random((n_liq, 3))
    u[:, 2] = 0.5 + 0.5 * u[:, 2]                   # liquid fills fractional z in [1/2, 1)
    liq = frac_to_cart(box, u)
    return Workload(f"c4_fcc_liquid{2 * n_liq}", box, _to_f32(np.concatenate([xtal, liq])),
                    dict(r_max=1.3, l=6))


@dataclass
class Frame:
    box: Box
    points: np.ndarray
    kind: str


def c5(seed: int = 5, n_frames: int = 256, n_lo: int = 1000, n_hi: int = 200_000,
       density: float = 1.0) -> list[Frame]:
    """Frames of uneven size: N log-uniform in [n_lo, n_hi]; box cubic or triclinic (tilts
    uniform in [-0.2, 0.2]); positions uniform or perturbed FCC (sigma 0.05) at `density`."""
    rng = np.random.default_rng(seed)
    frames = []
    for _ in range(n_frames):
        n_target = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        triclinic = rng.random() < 0.5
        crystal = rng.random() < 0.5
        tilts = rng.uniform(-0.2, 0.2, size=3) if triclinic else np.zeros(3)
        if crystal:
            nc = max(2, int(round((n_target / 4.0) ** (1.0 / 3.0))))
            L = nc * fcc_lattice_constant(density)
            box = Box(L, L, L, *tilts)
            pts = lattice_points(rng, box, nc, sigma=0.05)
        else:
            L = (n_target / density) ** (1.0 / 3.0)
            box = Box(L, L, L, *tilts)
            pts = uniform_points(rng, box, n_target)
        frames.append(Frame(box, pts, ("fcc" if crystal else "uniform") + ("_tri" if triclinic else "_cub")))
    return frames


C5_PARAMS = dict(r_max=1.5, rdf_bins=200, rdf_r_max=3.0, rdf_r_min=0.0, l=6)


@dataclass
class OrientedFrame:
    box: Box
    points: np.ndarray   # (N, 3) float32, z = 0
    theta: np.ndarray    # (N,) float32 orientation angles about z


def p6(seed: int = 6, n: int = 20_000, n_frames: int = 10, neighbors: float = 12.0, r: float = 1.0,
       xy: float = 0.0) -> list[OrientedFrame]:
    """2D frames of uniform points with `neighbors` expected points inside radius r of a
    point (density neighbors / (pi r^2)) and uniform orientation angles."""
    rng = np.random.default_rng(seed)
    L = math.sqrt(n * math.pi * r * r / neighbors)
    box = Box.square(L, xy)
    out = []
    for _ in range(n_frames):
        pts = uniform_points(rng, box, n)
        theta = rng.uniform(-math.pi, math.pi, size=n).astype(np.float32)
        out.append(OrientedFrame(box, pts, theta))
    return out


P6_PARAMS = dict(x_max=1.0, y_max=1.0, bins_x=100, bins_y=100, rdf_bins=100, rdf_r_max=math.sqrt(2.0))


def blobs(seed: int = 7, n_blobs: int = 2000, per_blob: int = 1000, sigma: float = 0.5,
          density: float = 0.1) -> Workload:
    """Clustered points: Gaussian blobs (standard deviation sigma) at uniform centres in
    a cubic box sized for the given overall density; a workload of very uneven cell
    occupancy for comparing the tree query with the cell list."""
    rng = np.random.default_rng(seed)
    n = n_blobs * per_blob
    box = Box.cube((n / density) ** (1.0 / 3.0))
    centres = frac_to_cart(box, rng.random((n_blobs, 3)))
    x = np.repeat(centres, per_blob, axis=0) + rng.normal(0.0, sigma, size=(n, 3))
    return Workload(f"blobs{n_blobs}x{per_blob}", box, _to_f32(x), dict(r_max=1.0))


def small_random(seed: int, n: int, box: Box) -> np.ndarray:
    return uniform_points(np.random.default_rng(seed), box, n)


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])

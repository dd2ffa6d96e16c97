"""Seeded synthetic workloads shared by the CUDA path's tests/bench and the CPU oracle.

This module holds problem *descriptions* and random draws only: grid sizes, material
constants, load parameters, seeds, random tensor-train cores and arrival times.  It contains
none of the method's arithmetic (no assembly, no tensor-train algebra, no solver), so both
the oracle and the CUDA path may import it without sharing any computation.

The paper's only workload is a 2D cantilever under self-weight (Section 6); the problems
below are synthetic problems of the same kind (rectangular/box domains, isotropic linear
elasticity, clamped faces, body force and traction loads), expressed in the paper's QTT
layout (Section 4, Section 5.2): a component core followed by ``levels`` level cores.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict
from typing import List, Optional, Sequence

import numpy as np

# Faces are numbered -x, +x, -y, +y, -z, +z.
FACE_XLO, FACE_XHI, FACE_YLO, FACE_YHI, FACE_ZLO, FACE_ZHI = range(6)

GRAVITY = 9.81  # m/s^2, standard gravity (the paper writes f = (0, -rho g) without a value)


@dataclass
class Grid:
    """Tensor grid with 2**levels equidistant nodes per axis, boundary nodes included.

    ``clamped[f]`` is True when face ``f`` carries a homogeneous Dirichlet condition on all
    displacement components; other faces are traction (Neumann) faces.
    """
    dim: int
    levels: int
    lo: Sequence[float] = (0.0, 0.0, 0.0)
    hi: Sequence[float] = (1.0, 1.0, 1.0)
    clamped: Sequence[bool] = (True, False, False, False, False, False)
    plane_stress: bool = False
    # parallelogram / parallelepiped domain {lo + sum_d xi_d edges[d] : xi in [0,1]^dim} when set
    # (edges[d] is the image of reference axis d); `hi` is then unused
    edges: Optional[Sequence[Sequence[float]]] = None
    # 2D general quadrilateral when set: corners (P0, P1, P2, P3) at reference (0,0), (1,0), (0,1),
    # (1,1), the bilinear map of the unit square; `lo`, `hi` and `edges` are then unused
    quad: Optional[Sequence[Sequence[float]]] = None

    @property
    def n(self) -> int:
        return 1 << self.levels

    @property
    def dofs(self) -> int:
        return self.dim * (self.n ** self.dim)


@dataclass
class Material:
    """Isotropic material; ``E[0]`` left of ``split_x`` (element centroid), ``E[1]`` right."""
    E: Sequence[float] = (1.0, 1.0)
    nu: float = 0.3
    split_x: float = math.inf


@dataclass
class Load:
    """Body force and traction description.

    kind:
      "gravity"      f = rho*g along -y (2D) / -z (3D)
      "traction"     uniform traction vector ``traction`` on face ``face``
      "fourier"      f_c(x) = scale * sum_m a[c,m] sin(pi k_m . x + phi_m)
      "manufactured" body force and free-face tractions of the manufactured field
                     u* = (sin(pi x) sin(pi y), x(1-x) y(1-y)) (2D, unit square)
      "nodal"        a body force given by its nodal values f0 (Section 5.3): ``nodal`` is the
                     library's train of them, ``values`` the same values densely (natural order,
                     component-major) for the oracle
    """
    kind: str
    rho: float = 0.0
    g: float = GRAVITY
    face: int = FACE_XHI
    traction: Sequence[float] = (0.0, 0.0, 0.0)
    amp: Optional[np.ndarray] = None     # (dim, n_modes)
    wave: Optional[np.ndarray] = None    # (n_modes, dim) integer wave numbers
    phase: Optional[np.ndarray] = None   # (n_modes,)
    scale: float = 1.0
    nodal: Optional[object] = None       # "nodal": the library's TT of f0
    values: Optional[np.ndarray] = None  # "nodal": f0 densely, natural order, component-major


@dataclass
class SolveOpts:
    tol: float = 1e-10
    rank_cap: int = 16
    kickrank: int = 4
    max_sweeps: int = 40
    precision: str = "fp64"   # "fp64", "mixed" (outer TT-residual refinement), "mixed-local" or "mixed-tf32"
    refine_tol: float = 1e-6
    max_refine: int = 20
    seed: int = 0
    precond: bool = True      # block-Jacobi preconditioned local solves
    tensor_cores: bool = False  # binary32 contractions on the tcgen05 tensor cores
    local_rtol: float = -1.0    # local solves to this fraction of their starting residual (<0: default)
    fused_cg: bool = True       # local CG as one persistent kernel (False: a launch per step)
    timeout_us: int = 0         # wall-clock limit of the solve (0: none)


@dataclass
class Problem:
    name: str
    grid: Grid
    material: Material
    loads: List[Load]
    opts: SolveOpts


# ---------------------------------------------------------------------------------------
# random draws
# ---------------------------------------------------------------------------------------

def rng(seed: int) -> np.random.Generator:
    """Counter-based generator (Philox 4x64) keyed by ``seed``."""
    return np.random.Generator(np.random.Philox(key=seed))


def fourier_modes(seed: int, dim: int, n_modes: int = 8):
    """Amplitudes a[c,m] ~ N(0,1), wave numbers k_m in {1..4}^dim, phases phi_m ~ U[0, 2pi)."""
    r = rng(seed)
    amp = r.standard_normal((dim, n_modes))
    wave = r.integers(1, 5, size=(n_modes, dim))
    phase = r.uniform(0.0, 2.0 * math.pi, size=n_modes)
    return amp, wave, phase


def random_tt(seed: int, modes: Sequence[int], ranks: Sequence[int]) -> List[np.ndarray]:
    """Gaussian tensor-train cores ``[r_{k-1}, n_k, r_k]`` (ranks has len(modes)+1 entries)."""
    r = rng(seed)
    return [r.standard_normal((ranks[k], modes[k], ranks[k + 1])) for k in range(len(modes))]


def random_mpo(seed: int, modes: Sequence[int], ranks: Sequence[int]) -> List[np.ndarray]:
    """Gaussian operator cores ``[a_{k-1}, n_k, n_k, a_k]``."""
    r = rng(seed)
    return [r.standard_normal((ranks[k], modes[k], modes[k], ranks[k + 1]))
            for k in range(len(modes))]


def random_matrix(seed: int, m: int, n: int) -> np.ndarray:
    return rng(seed).standard_normal((m, n))


def qtt_modes(dim: int, levels: int) -> List[int]:
    """Mode sizes of the QTT layout: the component core, then one 2**dim core per level."""
    return [dim] + [1 << dim] * levels


def max_ranks(modes: Sequence[int], cap: int) -> List[int]:
    """Largest attainable ranks min(prod of left modes, prod of right modes, cap)."""
    d = len(modes)
    out = [1]
    for k in range(1, d):
        left = 1
        for m in modes[:k]:
            left = min(left * m, 1 << 40)
        right = 1
        for m in modes[k:]:
            right = min(right * m, 1 << 40)
        out.append(int(min(left, right, cap)))
    out.append(1)
    return out


def poisson_arrivals(seed: int, n: int, rate: float) -> np.ndarray:
    """Arrival times (s) of a Poisson process with ``rate`` arrivals per second."""
    gaps = rng(seed).exponential(1.0 / rate, size=n)
    return np.cumsum(gaps)


# ---------------------------------------------------------------------------------------
# the five problem shapes
# ---------------------------------------------------------------------------------------

def manufactured_2d(levels: int = 5, rank_cap: int = 16, tol: float = 1e-10) -> Problem:
    """2D plane strain, unit square, E=1, nu=0.3, left edge clamped, manufactured load."""
    return Problem(
        name=f"2d-manufactured-L{levels}",
        grid=Grid(dim=2, levels=levels, clamped=(True, False, False, False, False, False)),
        material=Material(E=(1.0, 1.0), nu=0.3),
        loads=[Load(kind="manufactured")],
        opts=SolveOpts(tol=tol, rank_cap=rank_cap),
    )


def steel_plate_2d(levels: int = 10, rank_cap: int = 64, tol: float = 1e-9,
                   precision: str = "fp64") -> Problem:
    """2D plane strain steel plate: clamped left edge, gravity (rho=7850) plus a uniform
    downward traction of 1 MN/m^2 on the right edge."""
    return Problem(
        name=f"2d-steel-L{levels}",
        grid=Grid(dim=2, levels=levels, clamped=(True, False, False, False, False, False)),
        material=Material(E=(210e9, 210e9), nu=0.3),
        loads=[Load(kind="gravity", rho=7850.0),
               Load(kind="traction", face=FACE_XHI, traction=(0.0, -1e6, 0.0))],
        opts=SolveOpts(tol=tol, rank_cap=rank_cap, precision=precision),
    )


def cantilever_3d(levels: int = 7, rank_cap: int = 96, tol: float = 1e-8, seed: int = 0,
                  precision: str = "fp64", two_material: bool = False) -> Problem:
    """3D cantilever on the unit cube, clamped x=0 face, gravity plus an 8-mode Fourier force."""
    amp, wave, phase = fourier_modes(seed, 3, 8)
    rho = 2700.0
    mat = Material(E=(210e9, 70e9), nu=0.33, split_x=0.5) if two_material else \
        Material(E=(70e9, 70e9), nu=0.33)
    return Problem(
        name=f"3d-cantilever-L{levels}" + ("-2mat" if two_material else ""),
        grid=Grid(dim=3, levels=levels, clamped=(True, False, False, False, False, False)),
        material=mat,
        loads=[Load(kind="gravity", rho=rho),
               Load(kind="fourier", amp=amp, wave=wave, phase=phase, scale=rho * GRAVITY)],
        opts=SolveOpts(tol=tol, rank_cap=rank_cap, precision=precision, seed=seed),
    )


def cantilever_paper_2d(levels: int = 8, rank_cap: int = 64, tol: float = 1e-10,
                        precision: str = "fp64") -> Problem:
    """The results section's workload: an aluminium cantilever 20 m long and 1 m high, plane
    stress, E = 68 GPa, nu = 0.33, density 2700 kg/m^3 under its own weight, clamped at x = 0."""
    return Problem(
        name=f"2d-cantilever-paper-L{levels}",
        grid=Grid(dim=2, levels=levels, lo=(0.0, 0.0, 0.0), hi=(20.0, 1.0, 0.0),
                  clamped=(True, False, False, False, False, False), plane_stress=True),
        material=Material(E=(68e9, 68e9), nu=0.33),
        loads=[Load(kind="gravity", rho=2700.0)],
        opts=SolveOpts(tol=tol, rank_cap=rank_cap, precision=precision),
    )


QUAD_PLATE = ((0.0, 0.0), (1.0, 0.1), (0.2, 0.9), (1.3, 1.4))


def quad_plate_2d(levels: int = 10, rank_cap: int = 64, tol: float = 1e-9, precision: str = "mixed-local") -> Problem:
    """Steel on a convex, non-parallelogram quadrilateral (corners QUAD_PLATE at unit-square
    (0,0), (1,0), (0,1), (1,1)), plane strain, clamped on the xi = 0 side, self-weight plus a
    1 MN/m^2 downward traction on the xi = 1 side; element Jacobians frozen at the centres."""
    return Problem(
        name=f"2d-quad-plate-L{levels}",
        grid=Grid(dim=2, levels=levels, quad=QUAD_PLATE, clamped=(True, False, False, False, False, False)),
        material=Material(E=(210e9, 210e9), nu=0.3),
        loads=[Load(kind="gravity", rho=7850.0), Load(kind="traction", face=FACE_XHI, traction=(0.0, -1e6, 0.0))],
        opts=SolveOpts(tol=tol, rank_cap=rank_cap, precision=precision),
    )


def served_requests(seed: int = 0, n: int = 512, rate: float = 200.0):
    """Mixed request stream: per request, dimension, levels, material, load and rank cap."""
    arrivals = poisson_arrivals(seed, n, rate)
    reqs = []
    for i in range(n):
        r = rng(1000 + i)
        dim = int(r.integers(2, 4))
        levels = int(r.integers(6, 11)) if dim == 2 else int(r.integers(5, 10))
        E = float(math.exp(r.uniform(math.log(1e9), math.log(3e11))))
        nu = float(r.uniform(0.2, 0.45))
        kind = ["gravity", "traction", "fourier"][int(r.integers(0, 3))]
        cap = [16, 32, 64, 96][int(r.integers(0, 4))]
        if kind == "gravity":
            load = Load(kind="gravity", rho=float(r.uniform(1000.0, 9000.0)))
        elif kind == "traction":
            t = [0.0, 0.0, 0.0]
            t[dim - 1] = -float(r.uniform(1e5, 1e7))
            load = Load(kind="traction", face=FACE_XHI, traction=tuple(t))
        else:
            amp, wave, phase = fourier_modes(1000 + i, dim, 8)
            load = Load(kind="fourier", amp=amp, wave=wave, phase=phase, scale=2700.0 * GRAVITY)
        reqs.append(Problem(
            name=f"req{i}",
            grid=Grid(dim=dim, levels=levels,
                      clamped=(True, False, False, False, False, False)),
            material=Material(E=(E, E), nu=nu),
            loads=[load],
            opts=SolveOpts(tol=1e-6, rank_cap=cap, precision="mixed-local", seed=1000 + i),
        ))
    return arrivals, reqs

"""The C-ABI library loads, exports every symbol include/tnfem.h declares, and its host-side
builders (exact QTT construction, no GPU) reproduce the oracle's operator and load."""
import math
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import fem, mpo, tt
from paper_2501_12151_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_2501_12151_gb300 import tnfem
    return tnfem


def test_library_exports_every_declared_symbol():
    T = _lib()
    with open(os.path.join(ROOT, "include", "tnfem.h")) as fh:
        src = fh.read()
    declared = sorted(set(re.findall(r"\b(tnfem_[a-z0-9_]+)\s*\(", src)))
    assert len(declared) >= 30
    missing = [s for s in declared if not hasattr(T.lib, s)]
    assert not missing, missing
    # and through the dynamic symbol table, for C callers
    out = subprocess.run(["nm", "-D", "--defined-only", T._LIB_PATH], capture_output=True, text=True).stdout
    for s in declared:
        assert re.search(r"\bT\s+" + s + r"\b", out), s


@pytest.mark.parametrize("dim,levels,clamped,split", [
    (2, 2, (True, False, False, False, False, False), math.inf),
    (2, 4, (True, False, False, True, False, False), 0.5),
    (2, 3, (True, True, False, False, False, False), math.inf),
    (3, 2, (True, False, False, False, False, False), 0.5),
])
def test_host_stiffness_matches_oracle(dim, levels, clamped, split):
    T = _lib()
    g = W.Grid(dim=dim, levels=levels, lo=(0.0, 0.5, -1.0), hi=(2.0, 1.5, 0.0), clamped=clamped)
    m = W.Material(E=(210.0, 70.0), nu=0.33, split_x=split)
    cores, s = T.host_stiffness(g, m)
    A, _ = fem.assemble(g, m)
    Aq = tt.matrix_to_qtt_order(fem.apply_bc(g, A), dim, levels)
    assert s == pytest.approx(fem.bc_shift(g, A), rel=1e-13)
    assert np.abs(tt.mpo_full(cores) - Aq).max() <= 1e-12 * np.abs(Aq).max()


def test_host_stiffness_plane_stress():
    T = _lib()
    g = W.Grid(dim=2, levels=3, lo=(0.0, 0.0, 0.0), hi=(20.0, 1.0, 0.0), plane_stress=True)
    m = W.Material(E=(68e9, 68e9), nu=0.33)
    cores, _ = T.host_stiffness(g, m)
    A, _ = fem.assemble(g, m)
    Aq = tt.matrix_to_qtt_order(fem.apply_bc(g, A), 2, 3)
    assert np.abs(tt.mpo_full(cores) - Aq).max() <= 1e-12 * np.abs(Aq).max()


def test_host_mass_matches_oracle():
    T = _lib()
    g = W.Grid(dim=3, levels=2, lo=(0.0, 0.0, 0.0), hi=(1.0, 2.0, 3.0))
    _, M = fem.assemble(g, W.Material())
    np.testing.assert_allclose(tt.mpo_full(T.host_mass(g)), tt.matrix_to_qtt_order(M, 3, 2), atol=1e-14)


@pytest.mark.parametrize("problem", ["manufactured", "steel", "cube", "traction_all_faces"])
def test_host_load_matches_oracle(problem):
    T = _lib()
    if problem == "manufactured":
        pr = W.manufactured_2d(levels=4)
    elif problem == "steel":
        pr = W.steel_plate_2d(levels=4)
    elif problem == "cube":
        pr = W.cantilever_3d(levels=2)
    else:
        g = W.Grid(dim=3, levels=2, clamped=(False, False, True, False, False, False))
        loads = [W.Load(kind="traction", face=f, traction=(1.0 + f, -2.0, 0.5 * f)) for f in range(6)]
        pr = W.Problem("t", g, W.Material(E=(1.0, 1.0), nu=0.25), loads, W.SolveOpts())
    cores = T.host_load(pr.grid, pr.material, pr.loads)
    A, M = fem.assemble(pr.grid, pr.material)
    f = fem.load_vector(pr.grid, pr.material, pr.loads, M)
    f = f * np.tile(~fem.constrained_nodes(pr.grid), pr.grid.dim)
    fq = tt.to_qtt_order(f, pr.grid.dim, pr.grid.levels)
    np.testing.assert_allclose(tt.tt_full(cores), fq, rtol=0, atol=1e-13 * np.abs(fq).max())


def test_host_builders_reject_bad_input():
    T = _lib()
    g = W.Grid(dim=4, levels=3)
    with pytest.raises(T.TnfemError):
        T.host_stiffness(g, W.Material())
    g = W.Grid(dim=2, levels=3)
    with pytest.raises(T.TnfemError):
        T.host_stiffness(g, W.Material(E=(1.0, 1.0), nu=0.5))
    with pytest.raises(T.TnfemError):
        T.host_load(g, W.Material(), [W.Load(kind="traction", face=5)])


MAPPED = [(2, 3, ((1.5, 0.3), (0.6, 1.0)), (True, False, False, True, False, False)),
          (2, 4, ((2.0, -0.5), (0.4, 1.0)), (True, True, False, False, False, False)),
          (3, 2, ((1.2, 0.2, 0.1), (0.3, 0.9, 0.0), (0.1, 0.4, 0.8)), (True, False, False, False, False, True))]


@pytest.mark.parametrize("dim,levels,edges,clamped", MAPPED)
def test_host_builders_on_affine_domains_match_oracle(dim, levels, edges, clamped):
    """Parallelogram / parallelepiped domains (affine element maps, Section 5.1): the host-built
    operator (with its boundary-condition shift), mass operator and load equal the oracle's
    element-loop matrices and load vector on the mapped nodes (permuted to the QTT order)."""
    T = _lib()
    g = W.Grid(dim=dim, levels=levels, lo=(0.2, -0.1, 0.3), edges=edges, clamped=clamped)
    m = W.Material(E=(2.0, 2.0), nu=0.3)
    cores, s = T.host_stiffness(g, m)
    K, M = fem.assemble(g, m)
    Aq = tt.matrix_to_qtt_order(fem.apply_bc(g, K), dim, levels)
    assert np.abs(tt.mpo_full(cores) - Aq).max() <= 1e-12 * np.abs(Aq).max()
    assert s == pytest.approx(fem.bc_shift(g, K), rel=1e-12)
    Mq = tt.matrix_to_qtt_order(M, dim, levels)
    assert np.abs(tt.mpo_full(T.host_mass(g)) - Mq).max() <= 1e-12 * np.abs(Mq).max()
    loads = [W.Load(kind="gravity", rho=3.0)] + [
        W.Load(kind="traction", face=f, traction=(0.5, -1.0, 0.2)) for f in range(2 * dim) if not clamped[f]]
    fv = fem.load_vector(g, m, loads, M) * np.tile(~fem.constrained_nodes(g), dim)
    fq = tt.to_qtt_order(fv, dim, levels)
    assert np.abs(tt.tt_full(T.host_load(g, m, loads)) - fq).max() <= 1e-12 * np.abs(fq).max()


def test_affine_domain_rejects_what_it_does_not_build():
    """A two-material split inside a sheared domain and a Fourier load on it are refused."""
    T = _lib()
    g = W.Grid(dim=2, levels=3, edges=((1.0, 0.0), (0.5, 1.0)))
    with pytest.raises(T.TnfemError):
        T.host_stiffness(g, W.Material(E=(1.0, 2.0), split_x=0.7))
    amp, wave, phase = W.fourier_modes(0, 2, 2)
    with pytest.raises(T.TnfemError):
        T.host_load(g, W.Material(), [W.Load(kind="fourier", amp=amp, wave=wave, phase=phase)])
    # a split outside the domain is a homogeneous material
    T.host_stiffness(g, W.Material(E=(1.0, 2.0), split_x=5.0))


QUADS = [(2, ((0.0, 0.0), (1.0, 0.1), (0.2, 0.9), (1.3, 1.4)), (True, False, False, False), math.inf),
         (3, ((0.0, 0.0), (1.0, 0.1), (0.2, 0.9), (1.3, 1.4)), (True, False, False, True), 0.6),
         (4, ((0.3, -0.2), (2.0, 0.0), (0.5, 1.0), (1.6, 1.3)), (False, True, True, False), math.inf),
         (3, ((0.0, 0.0), (0.0, 1.0), (1.0, 0.0), (1.2, 0.9)), (False, False, True, True), math.inf)]


@pytest.mark.parametrize("levels,quad,clamped,split", QUADS)
def test_host_builders_on_general_quadrilaterals_match_oracle(levels, quad, clamped, split):
    """General convex quadrilaterals with each element's Jacobian frozen at its centre
    (Algorithm 1): the host-built operator with its boundary-condition shift, the mass operator and
    the load (gravity, a Fourier body force, tractions on the free sides) equal the oracle's
    frozen-Jacobian element loop, two materials included; the last case is clockwise (det J < 0)."""
    T = _lib()
    g = W.Grid(dim=2, levels=levels, quad=quad, clamped=clamped)
    m = W.Material(E=(2.0, 5.0), nu=0.3, split_x=split)
    cores, s = T.host_stiffness(g, m)
    K, M = fem.assemble(g, m, frozen_jacobian=True)
    Aq = tt.matrix_to_qtt_order(fem.apply_bc(g, K), 2, levels)
    assert np.abs(tt.mpo_full(cores) - Aq).max() <= 1e-12 * np.abs(Aq).max()
    assert s == pytest.approx(fem.bc_shift(g, K), rel=1e-12)
    Mq = tt.matrix_to_qtt_order(M, 2, levels)
    assert np.abs(tt.mpo_full(T.host_mass(g)) - Mq).max() <= 1e-12 * np.abs(Mq).max()
    amp, wave, phase = W.fourier_modes(1, 2, 2)
    loads = [W.Load(kind="gravity", rho=3.0), W.Load(kind="fourier", amp=amp, wave=wave, phase=phase)] + [
        W.Load(kind="traction", face=f, traction=(0.5, -1.0, 0.0)) for f in range(4) if not clamped[f]]
    fv = fem.load_vector(g, m, loads, M) * np.tile(~fem.constrained_nodes(g), 2)
    fq = tt.to_qtt_order(fv, 2, levels)
    assert np.abs(tt.tt_full(T.host_load(g, m, loads)) - fq).max() <= 1e-12 * np.abs(fq).max()


def test_general_quadrilateral_rejects_what_it_does_not_build():
    """A non-convex or degenerate quadrilateral, more than 2^12 nodes per axis, a 3D grid and the
    unit-square manufactured load are refused."""
    T = _lib()
    m = W.Material()
    for quad in (((0.0, 0.0), (1.0, 0.0), (0.0, 1.0), (0.2, 0.2)),      # re-entrant corner
                 ((0.0, 0.0), (1.0, 0.0), (2.0, 0.0), (3.0, 0.0))):     # collinear
        with pytest.raises(T.TnfemError):
            T.host_stiffness(W.Grid(dim=2, levels=3, quad=quad), m)
    good = ((0.0, 0.0), (1.0, 0.1), (0.2, 0.9), (1.3, 1.4))
    with pytest.raises(T.TnfemError):
        T.host_mass(W.Grid(dim=2, levels=13, quad=good))
    with pytest.raises(T.TnfemError):
        T.host_mass(W.Grid(dim=3, levels=2, quad=good))
    with pytest.raises(T.TnfemError):
        T.host_load(W.Grid(dim=2, levels=3, quad=good), m, [W.Load(kind="manufactured")])


def test_nodal_train_load_is_refused_by_the_host_builder():
    """A nodal-train load needs the device (mass operator times the train): the host-only builder
    refuses it with an error status rather than ignoring it."""
    import ctypes

    T = _lib()

    class FakeTT:                      # a non-null handle; the host builder must not touch it
        h = ctypes.c_void_p(1)

    g = W.Grid(dim=2, levels=3)
    with pytest.raises(T.TnfemError):
        T.host_load(g, W.Material(), [W.Load(kind="nodal", nodal=FakeTT())])


def test_serving_estimate_covers_the_quadrilateral_build():
    """The serving loop's memory estimate for a general quadrilateral covers the dense stencil
    coefficients its build holds on the device (36 doubles per node, several copies), and grows
    fourfold per level where those dominate."""
    T = _lib()
    e = {}
    for L in (8, 10, 11, 12):
        pr = W.quad_plate_2d(levels=L)
        e[L] = T.serve_estimate(pr.grid, pr.opts)
        assert e[L] >= 3 * 36 * 8 * 4 ** L
    assert e[12] == pytest.approx(4 * e[11], rel=0.05)
    box = W.steel_plate_2d(levels=10)
    assert e[10] > T.serve_estimate(box.grid, box.opts)

"""Structural pins of the oracle's right-hand side (Sec. 3.1 DGSEM): discrete
conservation, free-stream preservation, mirror / rotation symmetry, 2D <-> 3D
consistency, and the wall boundary conditions of Sec. 2.4 on states whose answer is
known in closed form."""
import math

import numpy as np
import pytest

from cases import (PAPER_PARAMS, cycle_xyz, droplet_state, mesh_spec, mirror, oracle_objects, quad_weights,
                   transpose_xy)


def thermo(orc, T=0.85, gK=1e-4):
    rv, rl = orc.maxwell(T)
    return rv, rl, orc.interface_width(T, 5.0, gK)


def integrals(o, mspec, Ut):
    xi, w = o_gl(o, mspec["N"])
    h = [(mspec["hi"][d] - mspec["lo"][d]) / mspec["n"][d] for d in range(mspec["dim"])]
    W = quad_weights(w, mspec["dim"], h)
    return np.einsum("ven,n->v", Ut, W)


def o_gl(o, N):
    import oracle
    return oracle.gauss_legendre(N + 1)


@pytest.mark.parametrize("dim,N,n,model", [(2, 3, [5, 3], 1), (2, 4, [3, 4], 2), (3, 2, [3, 2, 3], 1),
                                           (3, 3, [2, 2, 2], 2)])
def test_mass_conservation_two_phase(orc, dim, N, n, model):
    """Mass: no source, no viscous flux, single-valued numerical flux -> the quadrature
    of rho_t vanishes to round-off on a periodic box, for the full two-phase model."""
    ms = mesh_spec(dim, N, n)
    o = oracle_objects(orc, ms, dict(PAPER_PARAMS, model=model))
    x = o.node_coords()
    prim = droplet_state(x, thermo(orc), radius=0.3, perturb_seed=3)
    U = o.set_primitive(prim)
    Ut = o.rhs(U)
    I = integrals(o, ms, Ut)
    scale = np.abs(Ut[0]).max() * np.prod([1.0 / k for k in n])
    assert abs(I[0]) < 1e-13 * max(scale, 1.0)


@pytest.mark.parametrize("dim,N,n", [(2, 3, [4, 3]), (3, 2, [2, 3, 2])])
def test_full_conservation_without_sources(orc, dim, N, n):
    """With alpha = 0 and gamma_K = 0 every equation is in divergence form, so mass,
    momentum, energy and c are all conserved to round-off (single-phase state, T > 1)."""
    ms = mesh_spec(dim, N, n)
    o = oracle_objects(orc, ms, dict(PAPER_PARAMS, alpha=0.0, gammaK=0.0))
    x = o.node_coords()
    prim = droplet_state(x, (0.8, 1.2, 0.3), T0=1.3, radius=0.3, perturb_seed=5)
    U = o.set_primitive(prim)
    Ut = o.rhs(U)
    I = integrals(o, ms, Ut)
    scale = np.abs(Ut).max(axis=(1, 2))
    assert np.all(np.abs(I) < 1e-13 * np.maximum(scale, 1.0))


@pytest.mark.parametrize("dim,model", [(2, 1), (2, 2), (3, 1)])
def test_free_stream(orc, dim, model):
    """A uniform state with uniform velocity and c = rho is a steady solution."""
    ms = mesh_spec(dim, 3, [3] * dim)
    o = oracle_objects(orc, ms, dict(PAPER_PARAMS, model=model))
    x = o.node_coords()
    prim = np.zeros((dim + 3,) + x[0].shape)
    prim[0] = 1.7
    for k in range(dim):
        prim[1 + k] = 0.3 * (k + 1)
    prim[dim + 1] = 0.9
    prim[dim + 2] = 1.7
    Ut = o.rhs(o.set_primitive(prim))
    assert np.abs(Ut).max() < 1e-10


@pytest.mark.parametrize("axis", [0, 1])
def test_mirror_symmetry_2d(orc, axis):
    """Reflecting the state across a mid-plane reflects the right-hand side (the normal
    momentum changes sign)."""
    n = [4, 3]
    ms = mesh_spec(2, 3, n, hi=[1.0, 0.75])
    o = oracle_objects(orc, ms, PAPER_PARAMS)
    x = o.node_coords()
    prim = droplet_state(x, thermo(orc), center=[0.45, 0.4], radius=0.2, perturb_seed=11, lengths=[1.0, 0.75])
    U = o.set_primitive(prim)
    Ut = o.rhs(U)
    Um = mirror(U, 2, n, 4, axis, [1 + axis])
    Utm = o.rhs(Um)
    ref = mirror(Ut, 2, n, 4, axis, [1 + axis])
    for v in range(5):
        assert np.abs(Utm[v] - ref[v]).max() < 1e-10 * max(1.0, np.abs(ref[v]).max())


def test_transpose_symmetry_2d(orc):
    """Swapping x and y (and the momentum components) commutes with the right-hand side."""
    n = [4, 4]
    ms = mesh_spec(2, 3, n)
    o = oracle_objects(orc, ms, dict(PAPER_PARAMS, model=2))
    x = o.node_coords()
    prim = droplet_state(x, thermo(orc), center=[0.45, 0.55], radius=0.2, perturb_seed=12)
    U = o.set_primitive(prim)
    perm = [0, 2, 1, 3, 4]
    Ut = o.rhs(U)
    Utt = o.rhs(transpose_xy(U, n, 4, perm))
    ref = transpose_xy(Ut, n, 4, perm)
    assert np.abs(Utt - ref).max() < 1e-10 * np.abs(ref).max()


def test_axis_cycle_symmetry_3d(orc):
    n = [2, 2, 2]
    ms = mesh_spec(3, 2, n)
    o = oracle_objects(orc, ms, PAPER_PARAMS)
    x = o.node_coords()
    prim = droplet_state(x, thermo(orc), center=[0.45, 0.55, 0.5], radius=0.25, perturb_seed=13)
    U = o.set_primitive(prim)
    perm = [0, 2, 3, 1, 4, 5]  # new mx = old my, new my = old mz, new mz = old mx
    Ut = o.rhs(U)
    Utc = o.rhs(cycle_xyz(U, n, 3, perm))
    ref = cycle_xyz(Ut, n, 3, perm)
    assert np.abs(Utc - ref).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("model", [1, 2])
def test_2d_equals_extruded_3d(orc, model):
    """A z-independent state with u_z = 0 on a 3D mesh periodic in z gives the 2D
    right-hand side in every z-layer and zero z-momentum change."""
    N, n2 = 3, [3, 4]
    ms2 = mesh_spec(2, N, n2, hi=[1.0, 1.0])
    ms3 = mesh_spec(3, N, n2 + [2], hi=[1.0, 1.0, 0.5])
    p = dict(PAPER_PARAMS, model=model)
    o2, o3 = oracle_objects(orc, ms2, p), oracle_objects(orc, ms3, p)
    x2 = o2.node_coords()
    th = thermo(orc)
    prim2 = droplet_state(x2, th, center=[0.5, 0.45], radius=0.25, perturb_seed=21)
    P = N + 1
    # extrude: value at (ez, ey, ex, k, j, i) = 2D value at (ey, ex, j, i); u_z = 0
    g2p = prim2.reshape(5, n2[1], n2[0], P, P)
    g3p = np.broadcast_to(g2p[:, None, :, :, None, :, :], (5, 2, n2[1], n2[0], P, P, P))
    g3p = np.concatenate([g3p[:3], np.zeros_like(g3p[:1]), g3p[3:]])
    prim3 = np.ascontiguousarray(g3p).reshape(6, -1, P ** 3)
    Ut2 = o2.rhs(o2.set_primitive(prim2))
    Ut3 = o3.rhs(o3.set_primitive(prim3))
    g3 = Ut3.reshape(6, 2, n2[1], n2[0], P, P, P)
    g2 = Ut2.reshape(5, n2[1], n2[0], P, P)
    for v2, v3 in zip([0, 1, 2, 3, 4], [0, 1, 2, 4, 5]):
        scale = np.abs(g2[v2]).max()
        for ez in range(2):
            for k in range(P):
                assert np.abs(g3[v3, ez, :, :, k] - g2[v2]).max() < 1e-10 * scale
    assert np.abs(g3[3]).max() < 1e-10 * np.abs(g2[1]).max()


@pytest.mark.parametrize("theta,c_state", [(90.0, "mid"), (45.0, "liquid"), (135.0, "vapour")])
def test_wall_rest_state_is_steady(orc, theta, c_state):
    """Uniform fluid at rest at the wall temperature between two isothermal walls is
    steady when the wall energy derivative vanishes (theta = 90 deg, or c at a Maxwell
    density, Eq. (helmfreesurftot_derivative))."""
    T = 0.85
    rv, rl = orc.maxwell(T)
    rho = {"mid": 1.0, "liquid": rl, "vapour": rv}[c_state]
    ms = mesh_spec(2, 3, [3, 3], periodic=[1, 0], walls={2: (T, theta), 3: (T, theta)})
    o = oracle_objects(orc, ms, PAPER_PARAMS)
    x = o.node_coords()
    prim = np.zeros((5,) + x[0].shape)
    prim[0], prim[3], prim[4] = rho, T, rho
    Ut = o.rhs(o.set_primitive(prim))
    assert np.abs(Ut).max() < 1e-9


@pytest.mark.parametrize("theta", [30.0, 60.0, 120.0])
def test_wall_contact_angle_flux(orc, theta):
    """Uniform c = rho at rest between two walls: the only net change of total c is the
    order-parameter flux gamma_K beta (grad c . n) through the walls, with grad c . n
    given by the contact-angle condition Eq. (bc_contactangle_alpha):
    d/dt int c = sum_walls area * gamma_K beta * (-(1/gamma_K) dpsi_w/dc).
    Hydrophilic walls (theta < 90) draw c up, hydrophobic ones push it down.  Mass stays
    conserved (impermeable walls)."""
    T = 0.85
    rv, rl = orc.maxwell(T)
    sig = orc.sigma_vl(T, 5.0, 1e-4)
    rho = 1.1
    ms = mesh_spec(2, 3, [3, 4], hi=[0.6, 1.0], periodic=[1, 0], walls={2: (T, theta), 3: (T, theta)})
    o = oracle_objects(orc, ms, PAPER_PARAMS)
    x = o.node_coords()
    prim = np.zeros((5,) + x[0].shape)
    prim[0], prim[3], prim[4] = rho, T, rho
    Ut = o.rhs(o.set_primitive(prim))
    I = integrals(o, ms, Ut)
    dpsi = 6 * (rho - rl) * (rho - rv) / (rl - rv) ** 3 * sig * math.cos(math.radians(theta))
    gn = -dpsi / PAPER_PARAMS["gammaK"]
    expected = 2 * 0.6 * PAPER_PARAMS["gammaK"] * PAPER_PARAMS["beta"] * gn
    assert abs(I[4] - expected) < 1e-10 * abs(expected)
    assert (I[4] > 0) == (theta < 90)
    assert abs(I[0]) < 1e-12


def test_isothermal_wall_cools_hot_fluid(orc):
    """Fluid at rest hotter than the walls loses total energy through the heat flux
    kappa grad T . n of the isothermal walls; momentum normal to the walls is balanced."""
    ms = mesh_spec(2, 3, [2, 4], periodic=[1, 0], walls={2: (0.8, 90.0), 3: (0.8, 90.0)})
    o = oracle_objects(orc, ms, PAPER_PARAMS)
    x = o.node_coords()
    prim = np.zeros((5,) + x[0].shape)
    prim[0], prim[3], prim[4] = 1.7, 0.9, 1.7
    Ut = o.rhs(o.set_primitive(prim))
    I = integrals(o, ms, Ut)
    assert I[3] < 0
    assert abs(I[0]) < 1e-12

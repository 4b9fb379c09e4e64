"""Pins of the oracle's curved-element path (Sec. 3.1 on curvilinear hexahedra: metric
terms, strong-form BR1 with the chain rule, contravariant volume fluxes, numerical
fluxes along the face metric).  None of these compares the path with itself:

* an affine map of the box reproduces the straight-box discretisation (its weak-form
  lifting and diagonal metrics are pinned by the other oracle tests);
* a rotated box gives the rotated right-hand side (mass, energy, c unchanged, momentum
  rotated): this catches transposed metric terms and wrong normals, also at walls
  (no-slip, sliding with a rotated wall velocity, and Navier slip, whose tractions and
  tangential projections then run along oblique normals);
* a uniform state is preserved on curved elements (discrete metric identities and one
  face metric for both elements), also at rest against bent walls at 90 degrees;
* mass (and, without sources, momentum) is conserved on a periodic curved mesh;
* a manufactured solution converges at the design order on a curved mesh.
"""
import numpy as np
import pytest

import mms_gen
from cases import PAPER_PARAMS, mesh_spec, oracle_objects, rel_l2
from paper_2208_05310_gb300 import inputs

WALLS2 = {2: (0.85, 60.0), 3: (0.8, 120.0)}
WALLS3 = {4: (0.85, 60.0), 5: (0.8, 120.0)}
# Navier slip below (all of gamma_1..4), a sliding no-slip wall above
SLIP2 = {2: (0.9, 70.0, 0.02, 0.1, 0.3, 0.5), 3: (0.85, 110.0, (0.3, 0.0, 0.0))}
SLIP3 = {4: (0.85, 60.0, 0.03, 0.05, 0.2, 0.3), 5: (0.8, 100.0, (0.2, -0.1, 0.0))}


def _rotated_walls(walls, R):
    """The wall table of the rotated box: sliding velocities rotated with the box."""
    out = {}
    for f, spec in walls.items():
        if len(spec) == 3:
            u = np.zeros(R.shape[0])
            u[:] = spec[2][:R.shape[0]]
            out[f] = spec[:2] + (tuple(R @ u) + (0.0,) * (3 - R.shape[0]),)
        else:
            out[f] = spec
    return out
# beta = 1 keeps the relaxation bound 2/(alpha beta) from deciding max_dt
DT_PARAMS = dict(PAPER_PARAMS, beta=1.0)


def _rot2(th):
    return np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])


def _rot3(axis, th):
    a = np.asarray(axis, dtype=float)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K


BOX_CASES = {
    "2d_N3_walls": mesh_spec(2, 3, [4, 3], periodic=[1, 0], walls=WALLS2),
    "2d_N4_periodic": mesh_spec(2, 4, [3, 3]),
    "3d_N3_walls": mesh_spec(3, 3, [2, 3, 2], periodic=[1, 1, 0], walls=WALLS3),
    "2d_N3_slip_sliding": mesh_spec(2, 3, [4, 3], periodic=[1, 0], walls=SLIP2),
    "3d_N3_slip_sliding": mesh_spec(3, 3, [2, 3, 2], periodic=[1, 1, 0], walls=SLIP3),
}


@pytest.mark.parametrize("name", sorted(BOX_CASES))
def test_affine_map_equals_box(orc, name):
    ms = BOX_CASES[name]
    mc = dict(ms, geometry=dict(ngeo=1))
    ob, oc = oracle_objects(orc, ms, DT_PARAMS), oracle_objects(orc, mc, DT_PARAMS)
    assert np.abs(oc.node_coords() - ob.node_coords()).max() < 1e-15
    assert np.allclose(oc.node_weights(), ob.node_weights(), rtol=1e-14, atol=0)
    prim = inputs.random_admissible(ms["dim"], ob.nelem, ob.np, 7)
    Ub, Uc = ob.set_primitive(prim), oc.set_primitive(prim)
    assert np.all(rel_l2(Uc, Ub) < 1e-14)
    err = rel_l2(oc.rhs(Uc), ob.rhs(Ub))
    assert np.all(err < 1e-12), err
    assert abs(oc.max_dt(Uc) - ob.max_dt(Ub)) < 1e-13 * ob.max_dt(Ub)
    db, dc = ob.diagnostics(Ub), oc.diagnostics(Uc)
    for k in db:
        assert abs(dc[k] - db[k]) <= 1e-13 * max(1.0, abs(db[k])), k


ROT_CASES = {
    "2d_periodic": (mesh_spec(2, 4, [4, 3]), _rot2(0.4)),
    "2d_walls": (mesh_spec(2, 3, [4, 3], periodic=[1, 0], walls=WALLS2), _rot2(-1.1)),
    "3d_periodic": (mesh_spec(3, 3, [2, 2, 3]), _rot3([1.0, 2.0, 0.5], 0.7)),
    "3d_walls": (mesh_spec(3, 3, [3, 2, 2], periodic=[1, 1, 0], walls=WALLS3), _rot3([-0.3, 1.0, 0.8], 2.0)),
    "2d_slip_sliding": (mesh_spec(2, 3, [4, 3], periodic=[1, 0], walls=SLIP2), _rot2(0.9)),
    "3d_slip_sliding": (mesh_spec(3, 3, [3, 2, 2], periodic=[1, 1, 0], walls=SLIP3), _rot3([0.5, -1.0, 0.3], 1.3)),
}


@pytest.mark.parametrize("name", sorted(ROT_CASES))
def test_rotated_box_rotates_the_rhs(orc, name):
    ms, R = ROT_CASES[name]
    d = ms["dim"]
    mr = dict(ms, geometry=dict(ngeo=1, rotation=R), walls=_rotated_walls(ms["walls"], R))
    ob, orr = oracle_objects(orc, ms, DT_PARAMS), oracle_objects(orc, mr, DT_PARAMS)
    assert np.abs(orr.node_coords() - np.einsum("kj,jen->ken", R, ob.node_coords())).max() < 1e-14
    prim = inputs.random_admissible(d, ob.nelem, ob.np, 3)
    pr = prim.copy()
    pr[1:1 + d] = np.einsum("kj,jen->ken", R, prim[1:1 + d])
    Ub, Ur = ob.set_primitive(prim), orr.set_primitive(pr)
    Rb = ob.rhs(Ub)
    exp = Rb.copy()
    exp[1:1 + d] = np.einsum("kj,jen->ken", R, Rb[1:1 + d])
    err = rel_l2(orr.rhs(Ur), exp)
    assert np.all(err < 1e-12), err
    assert abs(orr.max_dt(Ur) - ob.max_dt(Ub)) < 1e-12 * ob.max_dt(Ub)


FREE_CASES = [(2, 4, 2, [4, 3]), (2, 3, 3, [3, 3]), (3, 4, 2, [2, 3, 2]), (3, 3, 1, [3, 2, 2])]


@pytest.mark.parametrize("dim,N,ngeo,n", FREE_CASES)
def test_free_stream_on_curved_elements(orc, dim, N, ngeo, n):
    ms = mesh_spec(dim, N, n, geometry=dict(ngeo=ngeo, amp=0.05))
    o = oracle_objects(orc, ms, PAPER_PARAMS)
    prim = np.zeros((dim + 3, o.nelem, o.np))
    prim[0] = 0.6
    prim[1:1 + dim] = np.array([0.3, -0.2, 0.1][:dim])[:, None, None]
    prim[dim + 1] = 0.95
    prim[dim + 2] = 0.6
    Ut = o.rhs(o.set_primitive(prim))
    # the flux differences are O(p |J a| / J) ~ 1e1 here
    assert np.abs(Ut).max() < 1e-10, np.abs(Ut).max(axis=(1, 2))


@pytest.mark.parametrize("slip", [False, True])
@pytest.mark.parametrize("dim,N,ngeo,n", [(2, 4, 2, [4, 3]), (3, 4, 2, [2, 2, 3])])
def test_rest_against_bent_walls(orc, dim, N, ngeo, n, slip):
    """Uniform fluid at rest at the wall temperature, contact angle 90 degrees: the walls
    (bent by the map) exert the pressure only, which the curved volume terms balance.
    Navier-slip walls (all gamma non-zero) exert no traction and no heat flux on it."""
    wk = (0.9, 90.0, 0.02, 0.1, 0.3, 0.5) if slip else (0.9, 90.0)
    walls = {2 * (dim - 1): wk, 2 * (dim - 1) + 1: wk}
    per = [1] * (dim - 1) + [0]
    ms = mesh_spec(dim, N, n, periodic=per, walls=walls, geometry=dict(ngeo=ngeo, amp=0.05))
    o = oracle_objects(orc, ms, PAPER_PARAMS)
    prim = np.zeros((dim + 3, o.nelem, o.np))
    prim[0] = 1.7
    prim[dim + 1] = 0.9
    prim[dim + 2] = 1.7
    Ut = o.rhs(o.set_primitive(prim))
    assert np.abs(Ut).max() < 1e-10, np.abs(Ut).max(axis=(1, 2))


@pytest.mark.parametrize("dim,N,ngeo,n", [(2, 4, 2, [4, 3]), (3, 4, 2, [2, 3, 2])])
def test_conservation_on_curved_elements(orc, dim, N, ngeo, n):
    ms = mesh_spec(dim, N, n, geometry=dict(ngeo=ngeo, amp=0.05))
    o = oracle_objects(orc, ms, PAPER_PARAMS)
    W = o.node_weights()
    prim = inputs.random_admissible(dim, o.nelem, o.np, 5)
    Ut = o.rhs(o.set_primitive(prim))
    assert abs((W * Ut[0]).sum()) < 1e-13 * (W * np.abs(Ut[0])).sum()
    # without the non-conservative sources (alpha = 0) momentum is conserved too
    o0 = oracle_objects(orc, ms, dict(PAPER_PARAMS, alpha=0.0))
    Ut = o0.rhs(o0.set_primitive(prim))
    for v in range(1 + dim):
        assert abs((W * Ut[v]).sum()) < 1e-12 * (W * np.abs(Ut[v])).sum(), v


MMS = dict(gammaK=0.01, mu=0.01, kappa=0.02, cv=5.0, alpha=10.0, beta=10.0)


def _mms_error(orc, lib, fo, prm, N, n, geometry, dt, tend):
    ms = mesh_spec(2, N, [n, n], geometry=geometry)
    o = oracle_objects(orc, ms, prm)
    x = o.node_coords()
    nsteps = int(round(tend / dt))
    U = o.run(mms_gen.exact_state(lib, x, 0.0), nsteps, dt, rk=4, forcing=fo)
    Ue = mms_gen.exact_state(lib, x, nsteps * dt)
    return np.sqrt(((U - Ue) ** 2).mean(axis=(1, 2)))


@pytest.mark.parametrize("model,N,dt", [(1, 3, 2e-4), (2, 4, 5e-5)])
def test_mms_convergence_on_curved_mesh(orc, model, N, dt):
    """The periodic map tiles the same periodic square, so the manufactured solution of
    the straight-box pins applies unchanged.  Curved elements converge at the design
    order (N+1, with a pre-asymptotic margin) and stay within a factor 10 of the
    straight box's error."""
    prm = dict(MMS, model=model)
    lib, _, fo = mms_gen.build(prm)
    geo = dict(ngeo=2, amp=0.04)
    e8 = _mms_error(orc, lib, fo, prm, N, 8, geo, dt, 0.02)
    e16 = _mms_error(orc, lib, fo, prm, N, 16, geo, dt, 0.02)
    eoc = np.log2(e8 / e16)
    assert np.all(eoc > N + 0.3), eoc
    box16 = _mms_error(orc, lib, fo, prm, N, 16, None, dt, 0.02)
    assert np.all(e16 < 10.0 * box16), e16 / box16


def test_curved_input_checks(orc):
    p = orc.make_params(**PAPER_PARAMS)

    def sizes(ms):
        m = orc.make_mesh(ms["dim"], ms["N"], ms["n"] + [1] * (3 - ms["dim"]), ms["lo"] + [0.0] * (3 - ms["dim"]),
                          ms["hi"] + [1.0] * (3 - ms["dim"]), ms["periodic"] + [1] * (3 - ms["dim"]), ms["walls"],
                          geometry=(ms["geometry"]["ngeo"],
                                    inputs.box_geometry(ms["dim"], ms["n"], ms["lo"], ms["hi"], ms["geometry"]["ngeo"],
                                                        rotation=ms["geometry"].get("rotation"))))
        import ctypes as C
        ne, np_, nv = C.c_long(), C.c_int(), C.c_int()
        return orc.lib().or_sizes(C.byref(m), C.byref(p), C.byref(ne), C.byref(np_), C.byref(nv))

    assert sizes(mesh_spec(3, 4, [2, 2, 2], geometry=dict(ngeo=2))) == 0
    assert sizes(mesh_spec(3, 3, [2, 2, 2], geometry=dict(ngeo=2))) != 0    # 2 ngeo > N in 3D
    assert sizes(mesh_spec(2, 3, [2, 2], geometry=dict(ngeo=4))) != 0       # ngeo > N in 2D
    # a reflection inverts the elements (J < 0)
    assert sizes(mesh_spec(2, 3, [2, 2], geometry=dict(ngeo=1, rotation=np.diag([1.0, -1.0])))) != 0
    # a wall velocity along the wall's box axis: refused on the box, projected on curved walls
    slide = {2: (0.85, 90.0), 3: (0.85, 90.0, (0.1, 0.2, 0.0))}
    assert sizes(mesh_spec(2, 3, [2, 2], periodic=[1, 0], walls=slide, geometry=dict(ngeo=1))) == 0
    # the HLLC flux (model 2) is taken along the face normal
    oracle_objects(orc, mesh_spec(2, 3, [2, 2], geometry=dict(ngeo=1)), dict(PAPER_PARAMS, model=2, flux="hllc"))


UNSTRUCTURED_CASES = {
    "2d_walls": (mesh_spec(2, 3, [4, 3], periodic=[1, 0], walls=WALLS2, geometry=dict(ngeo=2, amp=0.05)), 3),
    "3d_walls": (mesh_spec(3, 3, [2, 3, 2], periodic=[1, 1, 0], walls=WALLS3, geometry=dict(ngeo=1, amp=0.05)), 4),
    "3d_periodic": (mesh_spec(3, 4, [2, 2, 3], geometry=dict(ngeo=2, amp=0.04)), 5),
}


def _unstructured(orc, ms, seed, params):
    from cases import geometry_array
    d = ms["dim"]
    ngeo, xg = geometry_array(ms)
    xn, conn, ni = inputs.reoriented_mesh(d, ms["N"], ms["n"], ms["periodic"], ngeo, xg, seed)
    m = orc.make_mesh(d, ms["N"], ms["n"] + [1] * (3 - d), [0.0] * 3, [1.0] * 3, ms["periodic"] + [1] * (3 - d),
                      ms["walls"], geometry=(ngeo, xn), conn=conn)
    return orc.Oracle(m, orc.make_params(**params)), conn, ni


@pytest.mark.parametrize("name", sorted(UNSTRUCTURED_CASES))
def test_renumbered_reoriented_mesh(orc, name):
    """The same physical mesh with its elements renumbered and each element in a random
    orientation-preserving local frame, connected through the unstructured tables
    (neighbour, its face, face-point orientation): node coordinates, state, right-hand
    side, max_dt and diagnostics equal those of the structured mesh (permuted)."""
    ms, seed = UNSTRUCTURED_CASES[name]
    d = ms["dim"]
    o1 = oracle_objects(orc, ms, DT_PARAMS)
    o2, conn, ni = _unstructured(orc, ms, seed, DT_PARAMS)
    assert np.abs(o2.node_coords() - o1.node_coords().reshape(d, -1)[:, ni]).max() < 1e-14
    prim = inputs.random_admissible(d, o1.nelem, o1.np, 5)
    U1 = o1.set_primitive(prim)
    U2 = o2.set_primitive(prim.reshape(prim.shape[0], -1)[:, ni])
    perm = lambda A: A.reshape(A.shape[0], -1)[:, ni]
    assert np.all(rel_l2(U2, perm(U1)) < 1e-14)
    err = rel_l2(o2.rhs(U2), perm(o1.rhs(U1)))
    assert np.all(err < 1e-12), err
    assert abs(o2.max_dt(U2) / o1.max_dt(U1) - 1) < 1e-13
    d1, d2 = o1.diagnostics(U1), o2.diagnostics(U2)
    for k in d1:
        assert abs(d2[k] - d1[k]) <= 1e-13 * max(1.0, abs(d1[k])), k
    # the orientations matter: a wrong one on one interior face changes the result
    bad = conn.copy()
    e, f = next((e, f) for e in range(bad.shape[0]) for f in range(bad.shape[1]) if bad[e, f, 0] >= 0)
    bad[e, f, 2] ^= 2
    from cases import geometry_array
    ngeo, _ = geometry_array(ms)
    xn = inputs.reoriented_mesh(d, ms["N"], ms["n"], ms["periodic"], ngeo, geometry_array(ms)[1], seed)[0]
    m3 = orc.make_mesh(d, ms["N"], ms["n"] + [1] * (3 - d), [0.0] * 3, [1.0] * 3, ms["periodic"] + [1] * (3 - d),
                       ms["walls"], geometry=(ngeo, xn), conn=bad)
    o3 = orc.Oracle(m3, orc.make_params(**DT_PARAMS))
    assert np.any(rel_l2(o3.rhs(o3.set_primitive(prim.reshape(prim.shape[0], -1)[:, ni])), perm(o1.rhs(U1))) > 1e-6)


@pytest.mark.parametrize("dim,N,n,periodic,walls,ngeo", [(2, 3, [4, 3], [1, 0], WALLS2, 2),
                                                         (3, 3, [2, 3, 2], [1, 1, 0], WALLS3, 1),
                                                         (3, 4, [3, 2, 2], [1, 1, 1], {}, 2)])
def test_reoriented_frames_generator(orc, dim, N, n, periodic, walls, ngeo):
    """The vectorised generator of random element frames (used for the large bench mesh)
    gives the same physical mesh: per element, the integrals of the right-hand side of a
    smooth state equal the box frames' (the node order inside an element differs)."""
    from cases import droplet_state, geometry_array
    ms = mesh_spec(dim, N, n, periodic=periodic, walls=walls, geometry=dict(ngeo=ngeo, amp=0.05))
    xn, conn = inputs.reoriented_frames(dim, N, n, periodic, ngeo, geometry_array(ms)[1], seed=9)
    assert np.any(conn[:, :, 2] > 1)
    o1 = oracle_objects(orc, ms, PAPER_PARAMS)
    m2 = orc.make_mesh(dim, N, n + [1] * (3 - dim), [0.0] * 3, [1.0] * 3, periodic + [1] * (3 - dim), walls,
                       geometry=(ngeo, xn), conn=conn)
    o2 = orc.Oracle(m2, orc.make_params(**PAPER_PARAMS))
    r1 = o1.rhs(o1.set_primitive(droplet_state(o1.node_coords(), (0.3, 1.8, 0.15), radius=0.3)))
    r2 = o2.rhs(o2.set_primitive(droplet_state(o2.node_coords(), (0.3, 1.8, 0.15), radius=0.3)))
    i1, i2 = (o1.node_weights() * r1).sum(axis=2), (o2.node_weights() * r2).sum(axis=2)
    assert np.all(np.abs(i1 - i2).max(axis=1) < 1e-12 * np.abs(i1).max(axis=1))


HLLC = dict(DT_PARAMS, model=2, flux="hllc")


@pytest.mark.parametrize("name", ["2d_N3_walls", "3d_N3_walls"])
def test_hllc_affine_map_equals_box(orc, name):
    """HLLC along the face normal: on an affine map it reproduces the box's HLLC along
    the coordinate directions (interior faces and the wall HLLC against the ghost)."""
    ms = BOX_CASES[name]
    ob = oracle_objects(orc, ms, HLLC)
    oc = oracle_objects(orc, dict(ms, geometry=dict(ngeo=1)), HLLC)
    prim = inputs.random_admissible(ms["dim"], ob.nelem, ob.np, 7)
    err = rel_l2(oc.rhs(oc.set_primitive(prim)), ob.rhs(ob.set_primitive(prim)))
    assert np.all(err < 1e-12), err


@pytest.mark.parametrize("name", ["2d_walls", "3d_walls"])
def test_hllc_rotated_box_rotates_the_rhs(orc, name):
    ms, R = ROT_CASES[name]
    d = ms["dim"]
    ob = oracle_objects(orc, ms, HLLC)
    orr = oracle_objects(orc, dict(ms, geometry=dict(ngeo=1, rotation=R)), HLLC)
    prim = inputs.random_admissible(d, ob.nelem, ob.np, 3)
    pr = prim.copy()
    pr[1:1 + d] = np.einsum("kj,jen->ken", R, prim[1:1 + d])
    Rb = ob.rhs(ob.set_primitive(prim))
    exp = Rb.copy()
    exp[1:1 + d] = np.einsum("kj,jen->ken", R, Rb[1:1 + d])
    err = rel_l2(orr.rhs(orr.set_primitive(pr)), exp)
    assert np.all(err < 1e-12), err


def test_hllc_free_stream_and_conservation(orc):
    ms = mesh_spec(3, 4, [2, 3, 2], geometry=dict(ngeo=2, amp=0.05))
    o = oracle_objects(orc, ms, HLLC)
    prim = np.zeros((6, o.nelem, o.np))
    prim[0], prim[1], prim[2], prim[3], prim[4], prim[5] = 0.6, 0.3, -0.2, 0.1, 0.95, 0.6
    assert np.abs(o.rhs(o.set_primitive(prim))).max() < 1e-10
    W = o.node_weights()
    Ut = o.rhs(o.set_primitive(inputs.random_admissible(3, o.nelem, o.np, 5)))
    assert abs((W * Ut[0]).sum()) < 1e-13 * (W * np.abs(Ut[0])).sum()

"""Pins of the oracle's mortars (Sec. 3.1: non-conforming 2:1 faces).  A big face facing
2 (2D) or 4 (3D) half-size faces: the small sides see the big side's traces interpolated
to their points; the big side sees the L2 projection of the small sides' traces
(lifting) and of their numerical fluxes, turned to its orientation and surface element
(surface integral).  Meshes from inputs.refined_mesh: the upper half in x refined 2:1,
so mortars sit at mid-domain and at the periodic wrap; fine elements carry their parent's
exact geometry, so the hanging faces are watertight.

Pinned by: uniform flow preserved (and rest against bent walls), mass conserved to
round-off (momentum too without sources on periodic meshes), and a manufactured solution
converging at the design order on refined curved meshes."""
import numpy as np
import pytest

import mms_gen
from cases import PAPER_PARAMS
from paper_2208_05310_gb300 import inputs

WALLS = {2: {2: (0.9, 90.0), 3: (0.9, 90.0)}, 3: {4: (0.9, 90.0), 5: (0.9, 90.0)}}


def refined_oracle(orc, dim, N, n, periodic, walls, ngeo, amp, params):
    xg, conn, mort = inputs.refined_mesh(dim, N, n, periodic, walls, ngeo, amp=amp)
    ne = xg.shape[1]
    m = orc.make_mesh(dim, N, [ne, 1, 1], [0.0] * 3, [1.0] * 3, list(periodic) + [1] * (3 - dim), walls,
                      geometry=(ngeo, xg), conn=conn, mortar=mort)
    return orc.Oracle(m, orc.make_params(**params)), mort


CASES = [(2, 4, [4, 3], [1, 0], 2), (3, 3, [2, 2, 2], [1, 1, 1], 1), (3, 4, [2, 2, 2], [1, 1, 0], 2)]


@pytest.mark.parametrize("dim,N,n,periodic,ngeo", CASES)
def test_uniform_states_preserved(orc, dim, N, n, periodic, ngeo):
    walls = WALLS[dim] if not all(periodic) else {}
    o, mort = refined_oracle(orc, dim, N, n, periodic, walls, ngeo, 0.05, PAPER_PARAMS)
    assert len(mort) > 0
    prim = np.zeros((dim + 3, o.nelem, o.np))
    if walls:  # at rest at the wall temperature, contact angle 90 degrees
        prim[0], prim[dim + 1], prim[dim + 2] = 1.7, 0.9, 1.7
    else:  # uniform flow
        prim[0], prim[dim + 1], prim[dim + 2] = 0.6, 0.95, 0.6
        prim[1:1 + dim] = np.array([0.3, -0.2, 0.1][:dim])[:, None, None]
    Ut = o.rhs(o.set_primitive(prim))
    assert np.abs(Ut).max() < 1e-10, np.abs(Ut).max(axis=(1, 2))


@pytest.mark.parametrize("dim,N,n,periodic,ngeo", CASES)
def test_conservation_across_mortars(orc, dim, N, n, periodic, ngeo):
    walls = WALLS[dim] if not all(periodic) else {}
    o, _ = refined_oracle(orc, dim, N, n, periodic, walls, ngeo, 0.05, PAPER_PARAMS)
    W = o.node_weights()
    prim = inputs.random_admissible(dim, o.nelem, o.np, 5)
    Ut = o.rhs(o.set_primitive(prim))
    assert abs((W * Ut[0]).sum()) < 1e-13 * (W * np.abs(Ut[0])).sum()
    if not walls:
        o0, _ = refined_oracle(orc, dim, N, n, periodic, walls, ngeo, 0.05, dict(PAPER_PARAMS, alpha=0.0))
        Ut = o0.rhs(o0.set_primitive(prim))
        for v in range(1, 1 + dim):
            assert abs((W * Ut[v]).sum()) < 1e-12 * (W * np.abs(Ut[v])).sum(), v


MMS = dict(gammaK=0.01, mu=0.01, kappa=0.02, cv=5.0, alpha=10.0, beta=10.0)


@pytest.mark.parametrize("model,N,dt", [(1, 3, 1e-4), (2, 4, 3e-5)])
def test_mms_convergence_with_mortars(orc, model, N, dt):
    prm = dict(MMS, model=model)
    lib, _, fo = mms_gen.build(prm)
    errs = []
    for nn in (4, 8):
        o, _ = refined_oracle(orc, 2, N, [nn, nn], [1, 1], {}, 2, 0.04, prm)
        x = o.node_coords()
        nst = int(round(0.02 / dt))
        U = o.run(mms_gen.exact_state(lib, x, 0.0), nst, dt, rk=4, forcing=fo)
        errs.append(np.sqrt(((U - mms_gen.exact_state(lib, x, nst * dt)) ** 2).mean(axis=(1, 2))))
    eoc = np.log2(errs[0] / errs[1])
    assert np.all(eoc > N + 0.3), eoc


REORIENT = [(2, 3, [4, 3], [1, 0], 2, 5), (3, 3, [2, 2, 2], [1, 1, 0], 1, 6), (3, 4, [2, 2, 2], [1, 1, 1], 2, 7)]


@pytest.mark.parametrize("params", [dict(PAPER_PARAMS), dict(PAPER_PARAMS, model=2, flux="hllc")])
@pytest.mark.parametrize("dim,N,n,periodic,ngeo,seed", REORIENT)
def test_reoriented_refined_mesh(orc, dim, N, n, periodic, ngeo, seed, params):
    """The refined mesh with every element in a random local frame (inputs.reoriented_refined:
    mortar sub-faces renumbered and face-point orientations of all eight kinds) is the
    same discretisation as in the box frames: coordinates, right-hand side, max_dt and
    diagnostics to 1e-12 after the node permutation.  A wrong orientation bit on one
    mortar sub-face changes the result."""
    walls = WALLS[dim] if not all(periodic) else {}
    xg, conn, mort = inputs.refined_mesh(dim, N, n, periodic, walls, ngeo, amp=0.05)
    xn, cn, mn, ni = inputs.reoriented_refined(dim, N, ngeo, xg, conn, mort, seed)
    ne = xg.shape[1]

    def oracle(x, c, m):
        mesh = orc.make_mesh(dim, N, [ne, 1, 1], [0.0] * 3, [1.0] * 3, list(periodic) + [1] * (3 - dim), walls,
                             geometry=(ngeo, x), conn=c, mortar=m)
        return orc.Oracle(mesh, orc.make_params(**params))

    o1, o2 = oracle(xg, conn, mort), oracle(xn, cn, mn)
    perm = lambda A: A.reshape(A.shape[0], -1)[:, ni.ravel()].reshape(A.shape)
    assert np.abs(o2.node_coords() - perm(o1.node_coords())).max() < 1e-14
    prim = inputs.random_admissible(dim, ne, o1.np, 3)
    U1, U2 = o1.set_primitive(prim), o2.set_primitive(perm(prim))
    R1, R2 = o1.rhs(U1), o2.rhs(U2)
    err = np.sqrt(((R2 - perm(R1)) ** 2).sum(axis=(1, 2)) / (perm(R1) ** 2).sum(axis=(1, 2)))
    assert np.all(err < 1e-12), err
    assert abs(o2.max_dt(U2) / o1.max_dt(U1) - 1) < 1e-12
    d1, d2 = o1.diagnostics(U1), o2.diagnostics(U2)
    for k in d1:
        assert abs(d2[k] - d1[k]) <= 1e-12 * max(1.0, abs(d1[k])), k
    # a wrong orientation on one sub-face (both table entries, so that they stay consistent)
    bad_m, bad_c = mn.copy(), cn.copy()
    s, fs, o = (int(v) for v in bad_m[0, 0])
    o_bad = o ^ (2 if dim == 2 else 4)
    bad_m[0, 0, 2] = o_bad
    bad_c[s, fs, 2] = o_bad | (int(bad_c[s, fs, 2]) >> 3 << 3)
    Rb = oracle(xn, bad_c, bad_m).rhs(U2)
    assert np.abs(Rb - R2).max() > 1e-6 * np.abs(R2).max()


GRADED = [(2, 3, [8, 2], 2), (3, 3, [8, 2, 2], 1)]


@pytest.mark.parametrize("dim,N,n,ngeo", GRADED)
def test_graded_mesh_two_levels(orc, dim, N, n, ngeo):
    """Two levels of 2:1 refinement (coarse | 2:1 | 4:1 | 2:1 | coarse in x: mortars between
    levels 0 and 1 and between levels 1 and 2): a uniform flow is preserved on the periodic
    curved mesh, mass is conserved to round-off with walls, and the mesh in random local
    frames equals the box frames."""
    from cases import graded_levels
    per = [1] * dim
    xg, conn, mort = inputs.graded_mesh(dim, N, n, per, {}, ngeo, graded_levels(n[0]), amp=0.05)
    ne = xg.shape[1]
    # mortars: two level-0 | level-1 interfaces (one big face per coarse cell of the
    # cross-section) and two level-1 | level-2 interfaces (2^(dim-1) per coarse cell)
    cross = int(np.prod(n[1:]))
    assert len(mort) == 2 * cross + 2 * cross * 2 ** (dim - 1)

    def oracle(x, c, m, periodic, walls, params=PAPER_PARAMS):
        mesh = orc.make_mesh(dim, N, [ne, 1, 1], [0.0] * 3, [1.0] * 3, list(periodic) + [1] * (3 - dim), walls,
                             geometry=(ngeo, x), conn=c, mortar=m)
        return orc.Oracle(mesh, orc.make_params(**params))

    o = oracle(xg, conn, mort, per, {})
    prim = np.zeros((dim + 3, ne, o.np))
    prim[0], prim[dim + 1], prim[dim + 2] = 0.6, 0.95, 0.6
    prim[1:1 + dim] = np.array([0.3, -0.2, 0.1][:dim])[:, None, None]
    assert np.abs(o.rhs(o.set_primitive(prim))).max() < 1e-10
    # walls in the last direction
    pw = per[:-1] + [0]
    walls = WALLS[dim]
    xg2, conn2, mort2 = inputs.graded_mesh(dim, N, n, pw, walls, ngeo, graded_levels(n[0]), amp=0.05)
    ow = oracle(xg2, conn2, mort2, pw, walls)
    W = ow.node_weights()
    Ut = ow.rhs(ow.set_primitive(inputs.random_admissible(dim, ne, ow.np, 5)))
    assert abs((W * Ut[0]).sum()) < 1e-13 * (W * np.abs(Ut[0])).sum()
    # random local frames
    xn, cn, mn, ni = inputs.reoriented_refined(dim, N, ngeo, xg2, conn2, mort2, 13)
    orr = oracle(xn, cn, mn, pw, walls)
    perm = lambda A: A.reshape(A.shape[0], -1)[:, ni.ravel()].reshape(A.shape)
    prim2 = inputs.random_admissible(dim, ne, ow.np, 6)
    R1 = ow.rhs(ow.set_primitive(prim2))
    R2 = orr.rhs(orr.set_primitive(perm(prim2)))
    err = np.sqrt(((R2 - perm(R1)) ** 2).sum(axis=(1, 2)) / (perm(R1) ** 2).sum(axis=(1, 2)))
    assert np.all(err < 1e-12), err

"""Pins of the sliding isothermal no-slip wall (the moving wall of the sliding-droplet
case, Sec. 4: a no-slip wall moving with velocity u_wall in its own plane) in the oracle,
on states whose right-hand side is known in closed form:

- plane Couette flow: uniform density and temperature, u = U s/H along the wall (s the
  distance from the resting wall) between a resting and a sliding wall.  Stress and
  pressure are uniform, so the momentum does not change, and the energy grows at the
  viscous dissipation rate mu (U/H)^2 everywhere (the traction of the sliding wall does
  the work mu U^2/H per unit area);
- Galilean invariance: a uniform flow with the velocity of both walls is steady (the
  same flow between resting walls is not);
- mirror symmetry: the problem mirrored across a plane normal to the sliding direction
  gives the mirrored right-hand side;
- refusals: a wall velocity with a normal component on a box mesh."""
import numpy as np
import pytest

from cases import PAPER_PARAMS, mesh_spec, oracle_objects

T0 = 0.85
RHO = 1.75  # liquid, away from the spinodal at T0


def _state(o, dim, u_of_x):
    x = o.node_coords()
    prim = np.zeros((dim + 3,) + x[0].shape)
    prim[0] = RHO
    u = u_of_x(x)
    for k in range(dim):
        prim[1 + k] = u[k]
    prim[dim + 1] = T0
    prim[dim + 2] = RHO
    return o.set_primitive(prim)


# (dim, wall-normal direction, sliding direction, N, elements)
COUETTE = [(2, 1, 0, 3, [3, 4]), (2, 0, 1, 4, [3, 2]), (3, 2, 0, 3, [2, 2, 3]), (3, 2, 1, 3, [2, 2, 3]),
           (3, 0, 2, 2, [3, 2, 2])]


@pytest.mark.parametrize("model,flux", [(1, "rusanov"), (2, "rusanov"), (2, "hllc")])
@pytest.mark.parametrize("dim,nd,sd,N,n", COUETTE)
def test_couette_flow(orc, dim, nd, sd, N, n, model, flux):
    U, H = 0.2, 0.7
    hi = [1.0] * dim
    hi[nd] = H
    u_top = [0.0] * 3
    u_top[sd] = U
    periodic = [1] * dim
    periodic[nd] = 0
    walls = {2 * nd: (T0, 90.0), 2 * nd + 1: (T0, 90.0, tuple(u_top))}
    ms = mesh_spec(dim, N, n, hi=hi, periodic=periodic, walls=walls)
    prm = dict(PAPER_PARAMS, model=model, flux=flux)
    o = oracle_objects(orc, ms, prm)

    def shear(x):
        u = [np.zeros_like(x[0]) for _ in range(dim)]
        u[sd] = U * x[nd] / H
        return u

    Ut = o.rhs(_state(o, dim, shear))
    heat = prm["mu"] * (U / H) ** 2  # 8.2e-4
    # round-off of the state (|rho e| ~ 10) times the Rusanov speed (~13) and the lifting
    # factor ((N+1)^2 / h ~ 50) gives ~1e-12; a missing wall term is of the order of heat
    for v in range(dim + 3):
        want = heat if v == dim + 1 else 0.0
        err = np.abs(Ut[v] - want).max()
        assert err < 1e-10, (v, err)
    # the same state with both walls at rest: the sliding wall's value and work are needed
    walls0 = {2 * nd: (T0, 90.0), 2 * nd + 1: (T0, 90.0)}
    o0 = oracle_objects(orc, mesh_spec(dim, N, n, hi=hi, periodic=periodic, walls=walls0), prm)
    Ut0 = o0.rhs(_state(o0, dim, shear))
    assert np.abs(Ut0[1 + sd]).max() > 1e-3


@pytest.mark.parametrize("dim,nd,N,n", [(2, 1, 3, [3, 3]), (3, 2, 3, [2, 2, 2])])
def test_walls_moving_with_the_flow(orc, dim, nd, N, n):
    uw = [0.15, -0.1, 0.05][:dim]
    uw[nd] = 0.0
    periodic = [1] * dim
    periodic[nd] = 0
    walls = {2 * nd: (T0, 90.0, tuple(uw)), 2 * nd + 1: (T0, 90.0, tuple(uw))}
    o = oracle_objects(orc, mesh_spec(dim, N, n, periodic=periodic, walls=walls), PAPER_PARAMS)
    flow = lambda x: [np.full_like(x[0], uw[k]) for k in range(dim)]
    Ut = o.rhs(_state(o, dim, flow))
    assert np.abs(Ut).max() < 1e-10
    walls0 = {2 * nd: (T0, 90.0), 2 * nd + 1: (T0, 90.0)}
    o0 = oracle_objects(orc, mesh_spec(dim, N, n, periodic=periodic, walls=walls0), PAPER_PARAMS)
    assert np.abs(o0.rhs(_state(o0, dim, flow))[1]).max() > 1e-3


def test_mirror_symmetry(orc):
    """2D, walls at y = 0 (at rest) and y = 1 (sliding in +x); a two-phase state.  The
    problem mirrored across x = 1/2 (wall sliding in -x, state mirrored) gives the
    mirrored right-hand side with the x-momentum negated."""
    N, n = 3, [4, 3]

    def run(sign):
        walls = {2: (T0, 70.0), 3: (0.8, 100.0, (sign * 0.3, 0.0, 0.0))}
        o = oracle_objects(orc, mesh_spec(2, N, n, periodic=[1, 0], walls=walls), PAPER_PARAMS)
        x = o.node_coords()
        xs = x[0] if sign > 0 else 1.0 - x[0]
        prim = np.zeros((5,) + x[0].shape)
        r = np.hypot(xs - 0.4, x[1] - 0.2)
        prim[0] = 0.3197 + 0.5 * (1.8071 - 0.3197) * (1 - np.tanh((r - 0.25) / 0.08))
        prim[1] = sign * (0.1 * np.sin(2 * np.pi * xs) + 0.2 * x[1])
        prim[2] = 0.05 * np.sin(np.pi * x[1]) * np.cos(2 * np.pi * xs)
        prim[3] = T0 + 0.02 * x[1]
        prim[4] = prim[0] * (1 + 1e-3 * np.cos(2 * np.pi * xs))
        return o, o.rhs(o.set_primitive(prim))

    o, Ut = run(1.0)
    om, Utm = run(-1.0)
    # mirrored node of (e, i, j): element ix -> n0 - 1 - ix, node i -> N - i
    P = N + 1
    idx = np.arange(o.nelem * o.np).reshape(n[1], n[0], P, P)[:, ::-1, :, ::-1].reshape(o.nelem, o.np)
    M = Utm[:, idx // o.np, idx % o.np]
    sgn = np.array([1, -1, 1, 1, 1])[:, None, None]
    scale = np.abs(Ut).max(axis=(1, 2))[:, None, None]
    assert np.abs(sgn * M - Ut).max(axis=(1, 2)).max() < 1e-11 * scale.max()
    assert np.abs(Ut[1]).max() > 1e-3


def test_refusals(orc):
    # a normal component
    with pytest.raises(Exception):
        oracle_objects(orc, mesh_spec(2, 3, [2, 2], periodic=[1, 0], walls={2: (T0, 90.0), 3: (T0, 90.0, (0.1, 0.2, 0))}),
                       PAPER_PARAMS)

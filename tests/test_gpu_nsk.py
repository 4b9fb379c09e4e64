"""The original NSK model (model 0) on the GPU against the oracle's model 0.

The library keeps the relaxation layout (rho, rho u, rho e, c) and holds rho in the c
slot (the kernels give it the mass flux and no source, so it stays rho bitwise); the
oracle's NSK state is (rho, rho u, rho e).  Checks: set-up, right-hand side and states
after 1 and 10 steps to 1e-12 (FP64) and within the FP32-bulk bounds, the c slot equal
to rho, max_dt, and the refusal of meshes with walls."""
import numpy as np
import pytest

from cases import PAPER_PARAMS, dgk_context, droplet_state, mesh_spec, oracle_objects, rel_l2
from test_gpu_parity import TOL32_RHS, TOL64, _thermo_dgk, _thermo_oracle, tol32_step

pytestmark = pytest.mark.gpu

NSK = dict(PAPER_PARAMS, model=0)
CASES = {"2d_N3": mesh_spec(2, 3, [5, 3]), "2d_N5": mesh_spec(2, 5, [3, 3]), "3d_N3": mesh_spec(3, 3, [2, 3, 2]),
         "3d_N5": mesh_spec(3, 5, [2, 2, 2])}


def _pair(orc, ms, precision="fp64", exact=True, seed=13):
    from paper_2208_05310_gb300 import inputs
    o = oracle_objects(orc, ms, NSK)
    g = dgk_context(ms, NSK, precision=precision)
    if exact:
        prim = inputs.random_admissible(ms["dim"], o.nelem, o.np, seed)
        po = pg = prim
    else:
        kw = dict(radius=0.3, perturb_seed=seed)
        po = droplet_state(o.node_coords(), _thermo_oracle(orc), **kw)
        pg = droplet_state(g.node_coords(), _thermo_dgk(), **kw)
    Uo = o.set_primitive(po)
    g.set_primitive(pg)
    return o, g, Uo


def _split(U, dim):
    assert np.array_equal(U[dim + 2], U[0])  # the c slot holds rho
    return U[:dim + 2]


@pytest.mark.parametrize("name", sorted(CASES))
def test_nsk_rhs_and_steps_fp64(orc, name):
    ms = CASES[name]
    d = ms["dim"]
    o, g, Uo = _pair(orc, ms)
    assert np.all(rel_l2(_split(g.download_state(), d), Uo) < 1e-14)
    err = rel_l2(_split(g.rhs(), d), o.rhs(Uo))
    assert np.all(err < TOL64), err
    dt = 0.5 * o.max_dt(Uo)
    assert abs(g.max_dt() - o.max_dt(Uo)) < 1e-12 * o.max_dt(Uo)
    g.rk_step(dt)
    g.status()
    assert np.all(rel_l2(_split(g.download_state(), d), o.run(Uo, 1, dt, rk=4)) < TOL64)
    g.run(9, dt)
    g.status()
    err = rel_l2(_split(g.download_state(), d), o.run(Uo, 10, dt, rk=4))
    assert np.all(err < TOL64), err


@pytest.mark.parametrize("name", ["2d_N3", "3d_N5"])
def test_nsk_two_phase_fp32_bulk(orc, name):
    ms = CASES[name]
    d = ms["dim"]
    o, g, Uo = _pair(orc, ms, precision="fp32bulk", exact=False)
    assert np.all(rel_l2(_split(g.rhs(), d), o.rhs(Uo)) < TOL32_RHS)
    # the step rule has no capillary (dispersive) term: on these under-resolved two-phase
    # states the oracle itself needs 5% of it for 10 stable steps (measured: 10% diverges
    # in 3D)
    dt = 0.05 * o.max_dt(Uo)
    g.run(10, dt)
    g.status()
    ref = o.run(Uo, 10, dt, rk=4)
    err = rel_l2(_split(g.download_state(), d), ref)
    # FP32 rounding of the right-hand side (bound TOL32_RHS) accumulates in proportion to
    # how far the state moves; the under-resolved NSK interface moves it much more in 10
    # steps than the relaxation cases do, so the bound is the larger of the fixed
    # one-step-scale bound and TOL32_RHS x the relative change of the oracle's state
    change = rel_l2(ref, Uo)
    tol = np.maximum(np.delete(tol32_step(d), d + 2), TOL32_RHS * change)
    assert np.all(err < tol), (err, tol)


def test_nsk_refuses_walls():
    from paper_2208_05310_gb300 import dgk
    ms = mesh_spec(2, 3, [3, 3], periodic=[1, 0], walls={2: (0.85, 90.0), 3: (0.85, 90.0)})
    with pytest.raises(dgk.DgkError):
        dgk_context(ms, NSK)

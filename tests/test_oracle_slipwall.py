"""Pins of the generalized Navier-slip wall (Eq. bc_nsk_alpha, all of gamma_1..gamma_4;
Sec. 2.4) in the oracle, on states whose wall fluxes are known in closed form:

- free slip (gamma_1 = gamma_2 = gamma_3 = gamma_4 = 0, theta = 90 deg): a uniform flow
  along the wall is steady (a no-slip wall decelerates it);
- Navier friction: uniform tangential flow u0 between two walls loses momentum at
  gamma_2 u0 per unit wall area and energy at gamma_2 u0^2;
- heat transfer: fluid at rest at T between walls at T_w gains energy at
  -gamma_3 (1/T_w - 1/T) per unit wall area (Eq. bc_energy_alpha);
- contact-angle hysteresis: the order parameter flux through the wall is
  gamma_K beta (grad c . n) with grad c . n = gamma_1 div u / gamma_K at 90 deg
  (Eq. bc_contactangle_alpha), for a flow whose divergence at the wall is known;
- mass is conserved on a two-phase state, and rest at the wall temperature is steady."""
import numpy as np
import pytest

from cases import PAPER_PARAMS, droplet_state, mesh_spec, oracle_objects
from test_oracle_structure import integrals, thermo

L = 0.8  # wall length (periodic x extent)


def _box(walls, N=3, n=(4, 3)):
    return mesh_spec(2, N, list(n), hi=[L, 1.0], periodic=[1, 0], walls=walls)


def _uniform(o, rho, u, T):
    x = o.node_coords()
    prim = np.zeros((5,) + x[0].shape)
    prim[0], prim[1], prim[2], prim[3], prim[4] = rho, u[0], u[1], T, rho
    return o.set_primitive(prim)


def test_free_slip_uniform_flow_is_steady(orc):
    T = 0.9
    ms = _box({2: (T, 90.0, 0, 0, 0, 0), 3: (T, 90.0, 0, 0, 0, 0)})
    o = oracle_objects(orc, ms, PAPER_PARAMS)
    Ut = o.rhs(_uniform(o, 1.1, (0.3, 0.0), T))
    assert np.abs(Ut).max() < 1e-10
    # the same flow between no-slip walls is not steady
    ms1 = _box({2: (T, 90.0), 3: (T, 90.0)})
    o1 = oracle_objects(orc, ms1, PAPER_PARAMS)
    assert np.abs(o1.rhs(_uniform(o1, 1.1, (0.3, 0.0), T))[1]).max() > 1e-3


@pytest.mark.parametrize("g2", [0.05, 0.4])
def test_navier_friction(orc, g2):
    T, rho, u0 = 0.9, 1.1, 0.3
    ms = _box({2: (T, 90.0, 0, g2, 0, 0), 3: (T, 90.0, 0, g2, 0, 0)})
    o = oracle_objects(orc, ms, PAPER_PARAMS)
    I = integrals(o, ms, o.rhs(_uniform(o, rho, (u0, 0.0), T)))
    assert abs(I[0]) < 1e-12
    assert abs(I[1] - (-2 * L * g2 * u0)) < 1e-10 * 2 * L * g2 * u0
    assert abs(I[3] - (-2 * L * g2 * u0 ** 2)) < 1e-10 * 2 * L * g2 * u0 ** 2
    assert abs(I[4]) < 1e-12


@pytest.mark.parametrize("T,Tw", [(0.9, 0.8), (0.85, 0.95)])
def test_heat_transfer(orc, T, Tw):
    g3 = 0.2
    ms = _box({2: (Tw, 90.0, 0, 0, g3, 0), 3: (Tw, 90.0, 0, 0, g3, 0)})
    o = oracle_objects(orc, ms, PAPER_PARAMS)
    I = integrals(o, ms, o.rhs(_uniform(o, 1.1, (0.0, 0.0), T)))
    expect = -2 * L * g3 * (1.0 / Tw - 1.0 / T)
    assert abs(I[3] - expect) < 1e-10 * abs(expect)
    assert abs(I[0]) < 1e-12 and np.all(np.abs(I[1:3]) < 1e-10 * abs(expect))
    assert (I[3] < 0) == (T > Tw)


@pytest.mark.parametrize("g1", [0.01, 0.05])
def test_contact_angle_hysteresis_flux(orc, g1):
    """u_y = s y (1-y)^2 (cubic: exact at N = 3; zero normal velocity at both walls;
    div u = s at y = 0 and 0 at y = 1), uniform rho = c and T, 90 deg:
    d/dt int c = gamma_K beta * L * (gamma_1 s / gamma_K) = beta gamma_1 s L."""
    T, rho, s = 0.9, 1.1, 0.2
    ms = _box({2: (T, 90.0, g1, 0, 0, 0), 3: (T, 90.0, g1, 0, 0, 0)})
    o = oracle_objects(orc, ms, PAPER_PARAMS)
    x = o.node_coords()
    prim = np.zeros((5,) + x[0].shape)
    prim[0], prim[3], prim[4] = rho, T, rho
    prim[2] = s * x[1] * (1 - x[1]) ** 2
    I = integrals(o, ms, o.rhs(o.set_primitive(prim)))
    expect = PAPER_PARAMS["beta"] * g1 * s * L
    assert abs(I[4] - expect) < 1e-9 * abs(expect)
    assert abs(I[0]) < 1e-12


def test_mass_conservation_two_phase_slip_walls(orc):
    ms = mesh_spec(2, 4, [3, 4], periodic=[1, 0], walls={2: (0.85, 60.0, 0.02, 0.1, 0.3, 0.5),
                                                        3: (0.8, 120.0, 0.01, 0.2, 0.1, 1.0)})
    o = oracle_objects(orc, ms, PAPER_PARAMS)
    U = o.set_primitive(droplet_state(o.node_coords(), thermo(orc), radius=0.3, perturb_seed=3))
    Ut = o.rhs(U)
    I = integrals(o, ms, Ut)
    assert abs(I[0]) < 1e-13 * max(np.abs(Ut[0]).max() / 12, 1.0)


def test_rest_at_wall_temperature_is_steady(orc):
    T = 0.85
    ms = _box({2: (T, 90.0, 0.02, 0.1, 0.3, 0.5), 3: (T, 90.0, 0.02, 0.1, 0.3, 0.5)})
    o = oracle_objects(orc, ms, PAPER_PARAMS)
    assert np.abs(o.rhs(_uniform(o, 1.0, (0.0, 0.0), T))).max() < 1e-9

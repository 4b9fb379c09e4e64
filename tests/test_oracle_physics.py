"""Physics pins of the oracle: the relaxation model approaches the original NSK model as
the Korteweg parameter alpha grows (Sec. 4.1.1), a planar liquid-vapour interface stays
in place, the total energy is conserved and the mathematical entropy -int rho eta
decreases once the interface is resolved (Second Law, Sec. 2.2-2.3, 4.1.1), and models 1
and 2 discretise the same PDE (Eq. (modified_pressure): their right-hand sides differ
only by truncation error)."""
import numpy as np
import pytest

import mms_gen
from cases import droplet_state, mesh_spec, oracle_objects
from paper_2208_05310_gb300 import inputs


def test_relaxation_approaches_nsk(orc):
    """1D-like static bubble (T = 0.85, r = 0.1) on a resolved 32-element strip, beta =
    1000 fixed: the L2 distance of rho between relaxation model 1 and the original NSK
    model after a short time decreases monotonically for alpha = 10, 100, 1000."""
    T0 = 0.85
    rv, rl = orc.maxwell(T0)
    L = orc.interface_width(T0, 5.0, 1e-4)
    Lx, ne = 0.5, 32
    ms = mesh_spec(2, 4, [ne, 1], hi=[Lx, Lx / ne])
    alphas, beta = (10.0, 100.0, 1000.0), 1000.0
    dt = 1.5 / (max(alphas) * beta)
    nst = int(round(0.001 / dt))

    def run(model, alpha):
        prm = dict(model=model, gammaK=1e-4, mu=0.01, kappa=1 / 150.0, cv=5.0, alpha=alpha, beta=beta)
        o = oracle_objects(orc, ms, prm)
        x = o.node_coords()
        prim = droplet_state(x, (rv, rl, L), T0=T0, center=[Lx / 2, 0.0], radius=0.1, liquid_inside=False,
                             axes=(0,))
        if model == 0:
            prim = prim[:4]
        return o.run(o.set_primitive(prim), nst, dt, rk=4)

    ref = run(0, 0.0)
    assert np.isfinite(ref).all()
    dist = [np.sqrt(((run(1, a)[0] - ref[0]) ** 2).mean()) for a in alphas]
    assert dist[0] > dist[1] > dist[2], dist
    assert dist[0] / dist[2] > 5.0, dist


def _crossings(x, rho, mid):
    xs, ys, r = x[0].ravel(), x[1].ravel(), rho.ravel()
    sel = np.isclose(ys, ys.min())
    xs, r = xs[sel], r[sel]
    o = np.argsort(xs)
    xs, r = xs[o], r[o]
    out = []
    for i in range(len(xs) - 1):
        if (r[i] - mid) * (r[i + 1] - mid) < 0:
            out.append(xs[i] + (mid - r[i]) * (xs[i + 1] - xs[i]) / (r[i + 1] - r[i]))
    return np.array(out)


def _planar_run(orc, nx, ny, T0=0.85):
    """The periodic strip of width 0.5 on nx x ny elements of N = 3 (height 0.125 for the
    specified 16x4 mesh, one square element row otherwise)."""
    rv, rl = orc.maxwell(T0)
    L = orc.interface_width(T0, 5.0, 1e-4)
    ms = mesh_spec(2, 3, [nx, ny], hi=[0.5, 0.125 if ny == 4 else 0.5 / nx])
    o = oracle_objects(orc, ms, dict(model=1, gammaK=1e-4, mu=0.01, kappa=1 / 150.0, cv=5.0, alpha=100.0,
                                     beta=100.0))
    x = o.node_coords()
    U = o.set_primitive(inputs.planar_slab(x, rv, rl, L, 0.125, 0.375, T0))
    dt = o.max_dt(U, cfl=0.5, dfl=0.4)
    return o, x, U, dt, rv, rl, L


def test_planar_interface_16x4_lsrk3(orc):
    """The planar-interface workload as specified (periodic strip [0,0.5]x[0,0.125], N = 3
    on 16x4 elements, T = 0.85, LSRK3, 200 steps at the CFL-limited dt).

    The tanh start is not the relaxation model's equilibrium profile, so both crossings of
    the mid density move inward by the same amount while the profile adjusts: 2.7e-3 L_i
    here, and 3.0e-3 L_i on 32, 64 elements and at N = 5 -- a converged motion of the
    PDE, not of the discretisation.  Checked: the interface does not translate (the two
    crossings move symmetrically to 1e-9); the motion of the specified mesh agrees with
    the resolved one (32 elements across, the same physical time) to 1e-3 L_i; the
    spurious velocity stays small; mass is conserved to round-off."""
    o, x, U, dt, rv, rl, L = _planar_run(orc, 16, 4)
    d0 = o.diagnostics(U)
    x0 = _crossings(x, U[0], 0.5 * (rv + rl))
    U = o.run(U, 200, dt, rk=3)
    d1 = o.diagnostics(U)
    x1 = _crossings(x, U[0], 0.5 * (rv + rl))
    assert len(x0) == 2 and len(x1) == 2
    drift = x1 - x0
    assert abs(drift[0] + drift[1]) < 1e-9
    assert d1["max_u"] < 0.05
    assert abs(d1["mass"] - d0["mass"]) < 1e-14
    # the same physical time on the resolved mesh (32 elements across the strip)
    o2, x2, U2, dt2, _, _, _ = _planar_run(orc, 32, 1)
    n2 = int(round(200 * dt / dt2))
    c0 = _crossings(x2, U2[0], 0.5 * (rv + rl))
    U2 = o2.run(U2, n2, 200 * dt / n2, rk=3)
    drift2 = _crossings(x2, U2[0], 0.5 * (rv + rl)) - c0
    print(f"planar interface: crossing motion / L_i {drift / L} (16x4), {drift2 / L} (32 across)")
    assert np.abs(drift - drift2).max() < 1e-3 * L


def test_resolved_interface_energy_and_entropy(orc):
    """Resolved planar interface (32 elements of N = 3 across 0.5): total energy drifts by
    less than 1e-6 relative over t = 0.02 (LSRK4, CFL 0.9) and the mathematical entropy
    -int rho eta decreases at every sample."""
    T0 = 0.85
    rv, rl = orc.maxwell(T0)
    L = orc.interface_width(T0, 5.0, 1e-4)
    ms = mesh_spec(2, 3, [32, 1], hi=[0.5, 0.5 / 32])
    o = oracle_objects(orc, ms, dict(model=1, gammaK=1e-4, mu=0.01, kappa=1 / 150.0, cv=5.0, alpha=100.0,
                                     beta=100.0))
    x = o.node_coords()
    U = o.set_primitive(inputs.planar_slab(x, rv, rl, L, 0.125, 0.375, T0))
    dt = o.max_dt(U, cfl=0.9, dfl=0.4)
    nst = int(0.02 / dt) // 8
    d = [o.diagnostics(U)]
    for _ in range(8):
        U = o.run(U, nst, dt, rk=4)
        d.append(o.diagnostics(U))
    E = np.array([q["energy"] for q in d])
    S = np.array([q["neg_entropy"] for q in d])
    assert np.abs(E - E[0]).max() < 1e-6 * abs(E[0])
    assert np.all(np.diff(S) < 0), np.diff(S)


def test_models_1_and_2_same_pde(orc):
    """Models 1 and 2 are one PDE (Eq. (modified_pressure)); on a smooth single-phase
    state their discrete right-hand sides differ by truncation error only: the momentum
    difference falls at least like h^N and the energy difference shrinks under
    refinement; mass and c are identical."""
    prm = dict(gammaK=0.01, mu=0.01, kappa=0.02, cv=5.0, alpha=10.0, beta=10.0, model=1)
    lib, _, _ = mms_gen.build(prm)
    N = 3
    diffs = []
    for n in (8, 16):
        ms = mesh_spec(2, N, [n, n])
        o1 = oracle_objects(orc, ms, dict(prm, model=1))
        o2 = oracle_objects(orc, ms, dict(prm, model=2))
        U = mms_gen.exact_state(lib, o1.node_coords(), 0.0)
        diffs.append(np.sqrt(((o1.rhs(U) - o2.rhs(U)) ** 2).mean(axis=(1, 2))))
    d8, d16 = diffs
    assert d8[0] == 0.0 and d16[0] == 0.0 and d8[4] == 0.0 and d16[4] == 0.0
    assert np.all(np.log2(d8[1:3] / d16[1:3]) > N)
    assert d16[3] < d8[3] / 4

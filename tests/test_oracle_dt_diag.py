"""Pins of the oracle's time-step rule and integral diagnostics against values the
mathematics fixes, independent of the oracle's own code paths.

Time step (the reading of the CFL rule for the paper's CFL = 0.9, Sec. 4):
    dt = min( CFL / ((2N+1) max_nodes sum_d (|u_d| + s)/h_d),
              DFL / ((2N+1)^2 nu_max sum_d h_d^-2),
              2 / (alpha beta) ),
    s^2 = c_s^2 + alpha rho,  nu = max(4 mu/(3 rho), kappa/(rho R cv), gamma_K beta),
with the van der Waals sound speed c_s^2 = R T (1 + 1/cv)/(1 - b rho)^2 - 2 a rho
(Sec. 2.3).  On a uniform state every node gives the same sums, so the rule has a closed
form.  The cases make each branch decide in turn (and each of the three terms of nu),
with different spacings and velocities per direction, so that a wrong (2N+1) factor, a
missing sum over directions, a transposed h_d or a wrong sound speed changes the result
far beyond rounding.  On a rotated (affine, curved-path) box the convective sum takes
the velocity along the rotated axes.

Diagnostics (collocated Gauss quadrature, exact for polynomials of degree <= 2N+1 per
direction): on states whose fields are low-degree polynomials the integrals are known in
closed form -- mass, momentum, ||rho - c||_2, and -int rho eta of a uniform state -- and
max|u| is the largest nodal speed, fixed by the Gauss nodes (numpy's leggauss)."""
import numpy as np
import pytest

R_GAS, A_VDW, B_VDW = 8.0 / 3.0, 3.0, 1.0 / 3.0


def cs2_closed(rho, T, cv):
    return R_GAS * T * (1.0 + 1.0 / cv) / (1.0 - B_VDW * rho) ** 2 - 2.0 * A_VDW * rho


def uniform_prim(o, rho, u, T, c=None):
    d = o.dim
    prim = np.zeros(o.shape())
    prim[0] = rho
    for k in range(d):
        prim[1 + k] = u[k]
    prim[d + 1] = T
    if o.nv > d + 2:
        prim[d + 2] = rho if c is None else c
    return prim


def expected_dt(dim, N, h, rho, u, T, prm, cfl=0.9, dfl=0.4):
    k1 = 2 * N + 1
    s2 = cs2_closed(rho, T, prm["cv"]) + (prm["alpha"] * rho if prm["model"] != 0 else 0.0)
    if prm["model"] == 0:
        s2 = abs(cs2_closed(rho, T, prm["cv"]))
    s = np.sqrt(max(s2, 0.0))
    lam = sum((abs(u[k]) + s) / h[k] for k in range(dim))
    nu = max(4.0 * prm["mu"] / (3.0 * rho), prm["kappa"] / (rho * R_GAS * prm["cv"]))
    if prm["model"] != 0:
        nu = max(nu, prm["gammaK"] * prm["beta"])
    ih2 = sum(1.0 / hk ** 2 for hk in h[:dim])
    branches = {"conv": cfl / (k1 * lam), "visc": dfl / (k1 * k1 * nu * ih2)}
    if prm["model"] != 0 and prm["alpha"] * prm["beta"] > 0:
        branches["relax"] = 2.0 / (prm["alpha"] * prm["beta"])
    which = min(branches, key=branches.get)
    return branches[which], which


BASE = dict(model=1, gammaK=1e-4, mu=1e-4, kappa=1e-4, cv=5.0, alpha=10.0, beta=1.0)

# (name, parameter overrides, the branch that must decide)
DT_CASES = [
    ("convective", {}, "conv"),
    ("viscous mu", dict(mu=2.0), "visc"),
    ("viscous kappa", dict(kappa=40.0), "visc"),
    ("viscous gammaK beta", dict(gammaK=1e-2, beta=300.0), "visc"),
    ("relaxation", dict(alpha=100.0, beta=20000.0, gammaK=1e-9), "relax"),
    ("model 2", dict(model=2), "conv"),
    ("original NSK", dict(model=0), "conv"),
]


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("name,over,branch", DT_CASES, ids=[c[0] for c in DT_CASES])
def test_max_dt_closed_form(orc, dim, name, over, branch):
    prm = dict(BASE, **over)
    N = 3 if dim == 3 else 4
    n = [3, 5, 2][:dim]
    L = [0.7, 1.3, 0.4][:dim]
    h = [L[k] / n[k] for k in range(dim)]
    rho, T = 1.6, 0.9
    u = [0.31, -0.17, 0.05][:dim]
    m = orc.make_mesh(dim, N, n + [1] * (3 - dim), [0.0] * 3, L + [1.0] * (3 - dim), [1, 1, 1])
    o = orc.Oracle(m, orc.make_params(**prm))
    U = o.set_primitive(uniform_prim(o, rho, u, T))
    want, which = expected_dt(dim, N, h, rho, u, T, prm)
    assert which == branch, (which, branch)
    got = o.max_dt(U)
    assert abs(got / want - 1.0) < 1e-12, (got, want)


def test_max_dt_rotated_box_closed_form(orc):
    """Curved path on an affine map: a square of side L rotated by theta, n x n elements.
    The convective sum per node is sum_dir (|u . q_dir| + s)/h with q_dir the rotated axes."""
    from paper_2208_05310_gb300 import inputs
    dim, N, n, side, theta = 2, 4, 4, 1.0, 0.6
    rot = np.array([[np.cos(theta), -np.sin(theta)], [np.sin(theta), np.cos(theta)]])
    x = inputs.box_geometry(dim, [n, n], [0.0, 0.0], [side, side], 1, rotation=rot)
    m = orc.make_mesh(dim, N, [n, n, 1], [0.0] * 3, [1.0] * 3, [1, 1, 1], geometry=(1, x))
    prm = dict(BASE)
    o = orc.Oracle(m, orc.make_params(**prm))
    rho, T, u = 1.4, 0.92, np.array([0.4, -0.25])
    U = o.set_primitive(uniform_prim(o, rho, u, T))
    q = [np.array([np.cos(theta), np.sin(theta)]), np.array([-np.sin(theta), np.cos(theta)])]
    s = np.sqrt(cs2_closed(rho, T, prm["cv"]) + prm["alpha"] * rho)
    h = side / n
    lam = sum((abs(u @ qd) + s) / h for qd in q)
    want = 0.9 / ((2 * N + 1) * lam)
    got = o.max_dt(U)
    assert abs(got / want - 1.0) < 1e-12, (got, want)


def _gauss_nodes_global(N, n, L):
    xi, _ = np.polynomial.legendre.leggauss(N + 1)
    h = L / n
    return np.concatenate([(i + 0.5) * h + 0.5 * h * xi for i in range(n)])


@pytest.mark.parametrize("dim", [2, 3])
def test_diagnostics_closed_forms(orc, dim):
    N = 3
    n = [4, 3, 2][:dim]
    L = [1.0, 0.8, 0.6][:dim]
    m = orc.make_mesh(dim, N, n + [1] * (3 - dim), [0.0] * 3, L + [1.0] * (3 - dim), [1, 1, 1])
    o = orc.Oracle(m, orc.make_params(**dict(BASE, model=1)))
    x = o.node_coords()
    vol = float(np.prod(L))
    # rho = 1.2 + 0.1 x_0 x_1 (degree 1 per direction); c = rho - delta x_0 x_1;
    # u = U0 x / L (linear, different per direction); T uniform
    prod = x[0] * x[1]
    rho = 1.2 + 0.1 * prod
    delta, U0 = 0.05, 0.3
    prim = np.zeros(o.shape())
    prim[0] = rho
    for k in range(dim):
        prim[1 + k] = U0 * (k + 1) * x[k] / L[k]
    prim[dim + 1] = 0.9
    prim[dim + 2] = rho - delta * prod
    U = o.set_primitive(prim)
    dg = o.diagnostics(U)
    def mono(*pw):  # int over the box of prod_j x_j^pw_j
        pw = list(pw) + [0] * (dim - len(pw))
        return float(np.prod([L[j] ** (pw[j] + 1) / (pw[j] + 1) for j in range(dim)]))

    assert abs(dg["mass"] - (1.2 * vol + 0.1 * mono(1, 1))) < 1e-13
    # momentum_k = int rho u_k = U0 (k+1)/L_k int (1.2 + 0.1 x_0 x_1) x_k
    for k in range(dim):
        e_k = [1 if j == k else 0 for j in range(dim)]
        e_k01 = [e_k[j] + (1 if j < 2 else 0) for j in range(dim)]
        want = U0 * (k + 1) / L[k] * (1.2 * mono(*e_k) + 0.1 * mono(*e_k01))
        assert abs(dg["mom_" + "xyz"[k]] - want) < 1e-13, (k, dg["mom_" + "xyz"[k]], want)
    i_prod2 = mono(2, 2)
    assert abs(dg["rho_minus_c_l2"] - delta * np.sqrt(i_prod2)) < 1e-14
    # max|u| at the node nearest the far corner
    top = [_gauss_nodes_global(N, n[k], L[k]).max() for k in range(dim)]
    want_u = np.sqrt(sum((U0 * (k + 1) * top[k] / L[k]) ** 2 for k in range(dim)))
    assert abs(dg["max_u"] - want_u) < 1e-14


def test_entropy_diagnostic_uniform_state(orc):
    """-int rho eta of a uniform state = -V rho eta(rho, T), with the vdW entropy per
    volume rho eta = rho R (cv ln T - ln(b rho/(1 - b rho))) (from psi, Sec. 2.1; the
    oracle's or_entropy_vol is pinned against finite differences of psi)."""
    dim, N = 2, 4
    m = orc.make_mesh(dim, N, [3, 2, 1], [0.0] * 3, [0.9, 0.5, 1.0], [1, 1, 1])
    o = orc.Oracle(m, orc.make_params(**BASE))
    rho, T = 0.7, 0.95
    U = o.set_primitive(uniform_prim(o, rho, [0.1, 0.2], T))
    dg = o.diagnostics(U)
    reta = rho * R_GAS * (5.0 * np.log(T) - np.log(B_VDW * rho / (1.0 - B_VDW * rho)))
    assert abs(dg["neg_entropy"] - (-0.45 * reta)) < 1e-13

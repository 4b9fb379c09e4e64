"""Pins of the oracle's rate of entropy production (Sec. 2.3) against the scheme's own
entropy balance.

On a periodic box the entropy flux integrates to zero, so the total entropy changes at
d/dt int rho eta = int Pi.  The discrete counterpart: the derivative of the oracle's
quadrature of rho eta (the negative of its -int rho eta diagnostic, with T recovered as
the scheme recovers it) along the oracle's own right-hand side, taken by a central
difference [S(U + eps U_t) - S(U - eps U_t)] / (2 eps), must equal the quadrature of Pi
up to the scheme's truncation error on a smooth, resolved single-phase state with shear,
compression, a temperature gradient and c != rho (every term of Pi active).  Measured:
4e-5 relative on 4x4 (2D and 3D, N = 4), <= 3e-7 on 8x8 (2D).  Planted by hand, each of
these fails: the heat term with 1/T^3 (1.4e-3), no relaxation term (0.12), the printed
viscous form 4/3 mu |div u|^2 + mu |D_dev|^2 in place of tau : grad u (0.3).

At rest with uniform T and c = rho every term vanishes: int Pi = 0."""
import numpy as np
import pytest

from cases import mesh_spec, oracle_objects

PARAMS = dict(gammaK=1e-4, mu=0.01, kappa=1.0 / 150.0, cv=5.0, alpha=100.0, beta=100.0)


def smooth_state(o, x, dim, model):
    tp = 2.0 * np.pi
    X, Y = x[0], x[1]
    Z = x[2] if dim == 3 else 0.0 * X
    prim = np.zeros(o.shape())
    rho = 1.8 + 0.03 * np.sin(tp * X) * np.cos(tp * Y) + 0.01 * np.sin(tp * Z)
    prim[0] = rho
    prim[1] = 0.1 * np.sin(tp * Y) + 0.05 * np.sin(tp * X)
    prim[2] = 0.05 * np.sin(tp * X) + 0.03 * np.cos(tp * Y)
    if dim == 3:
        prim[3] = 0.04 * np.sin(tp * (X + Z))
    prim[dim + 1] = 0.95 + 0.03 * np.cos(tp * X + 1.0) * np.cos(tp * Y)
    if model != 0:
        prim[dim + 2] = rho + 3e-5 * np.sin(tp * (X + Y))
    return prim


@pytest.mark.parametrize("dim,n,tol", [(2, 8, 1e-5), (3, 4, 1e-4)])
@pytest.mark.parametrize("model", [1, 2, 0])
def test_entropy_production_matches_discrete_entropy_rate(orc, dim, n, tol, model):
    ms = mesh_spec(dim, 4, [n] * dim)
    o = oracle_objects(orc, ms, dict(PARAMS, model=model))
    U = o.set_primitive(smooth_state(o, o.node_coords(), dim, model))
    Ut = o.rhs(U)
    eps = 1e-5
    rate = -(o.diagnostics(U + eps * Ut)["neg_entropy"] - o.diagnostics(U - eps * Ut)["neg_entropy"]) / (2 * eps)
    pi = o.diagnostics(U)["entropy_production"]
    assert pi > 0
    assert abs(rate - pi) < tol * pi, (rate, pi, (rate - pi) / pi)


@pytest.mark.parametrize("model", [1, 2, 0])
def test_entropy_production_vanishes_at_rest(orc, model):
    dim = 2
    ms = mesh_spec(dim, 4, [3, 3])
    o = oracle_objects(orc, ms, dict(PARAMS, model=model))
    x = o.node_coords()
    prim = np.zeros(o.shape())
    prim[0] = 0.4 + 0.3 * np.sin(2 * np.pi * x[0])  # density varies, u = 0, T uniform
    prim[dim + 1] = 0.9
    if model != 0:
        prim[dim + 2] = prim[0]
    U = o.set_primitive(prim)
    d = o.diagnostics(U)
    # lifted grad u and grad T are round-off; chi = gamma_K lap c is not zero for a varying
    # c: rest with uniform T and a *uniform* density has no production at all
    prim[0] = 0.4
    if model != 0:
        prim[dim + 2] = 0.4
    d0 = o.diagnostics(o.set_primitive(prim))
    assert abs(d0["entropy_production"]) < 1e-20
    assert d["entropy_production"] >= -1e-20

"""Pins of the oracle's original NSK model (model 0: Eq. navierstokeskorteweg with the
Korteweg stress of Eq. cauchystressnsk and the energy flux of Eq. energyfluxnsk; Delta
rho by BR1 twice, Sec. 3.1; periodic boxes):

- every equation is in divergence form, so mass, momentum and total energy are
  conserved to round-off on a periodic two-phase state;
- order N+1 on a manufactured solution of the NSK PDE typed independently in SymPy;
- a uniform state in uniform motion is steady.
(The relaxation models approach it as alpha grows: test_oracle_physics.)"""
import numpy as np
import pytest

import mms_gen
from cases import PAPER_PARAMS, droplet_state, mesh_spec, oracle_objects
from test_oracle_mms import MMS
from test_oracle_structure import integrals, thermo

NSK = dict(PAPER_PARAMS, model=0)


@pytest.mark.parametrize("dim,N,n", [(2, 3, [5, 3]), (2, 4, [3, 4]), (3, 3, [2, 2, 2])])
def test_full_conservation_two_phase(orc, dim, N, n):
    ms = mesh_spec(dim, N, n)
    o = oracle_objects(orc, ms, NSK)
    U = o.set_primitive(droplet_state(o.node_coords(), thermo(orc), radius=0.3, perturb_seed=3))
    assert U.shape[0] == dim + 2
    Ut = o.rhs(U)
    I = integrals(o, ms, Ut)
    vol = np.prod([1.0 / k for k in n])
    scale = np.abs(Ut).max(axis=(1, 2)) * vol
    assert np.all(np.abs(I) < 1e-13 * np.maximum(scale, 1.0)), (I, scale)


def _mms_error(orc, lib, fo, prm, N, n, dt, nsteps):
    ms = mesh_spec(2, N, [n, n])
    o = oracle_objects(orc, ms, prm)
    x = o.node_coords()
    U = o.run(mms_gen.exact_state(lib, x, 0.0)[:4], nsteps, dt, forcing=fo)
    Ue = mms_gen.exact_state(lib, x, nsteps * dt)[:4]
    return np.sqrt(((U - Ue) ** 2).mean(axis=(1, 2)))


@pytest.mark.parametrize("N", [2, 3])
def test_spatial_convergence_nsk(orc, N):
    prm = dict(MMS, model=0)
    lib, _, fo = mms_gen.build(prm)
    e8 = _mms_error(orc, lib, fo, prm, N, 8, 2e-4, 100)
    e16 = _mms_error(orc, lib, fo, prm, N, 16, 2e-4, 100)
    eoc = np.log2(e8 / e16)
    assert np.all(eoc > N + 0.5), eoc


def test_free_stream_nsk(orc):
    ms = mesh_spec(2, 3, [3, 3])
    o = oracle_objects(orc, ms, NSK)
    x = o.node_coords()
    prim = np.zeros((5,) + x[0].shape)
    prim[0], prim[1], prim[2], prim[3], prim[4] = 1.7, 0.3, -0.2, 0.9, 1.7
    assert np.abs(o.rhs(o.set_primitive(prim))).max() < 1e-10

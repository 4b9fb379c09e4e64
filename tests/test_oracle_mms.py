"""Order-of-accuracy pins of the oracle (Sec. 3.1) with a manufactured solution of the
relaxed NSK system: the PDE is typed in SymPy from the paper, the forcing is compiled
and added to the oracle's right-hand side, and the error against the exact solution
converges at order N+1 in space; the low-storage RK schemes show their design order in
time (self-convergence)."""
import numpy as np
import pytest

import mms_gen
from cases import mesh_spec, oracle_objects

MMS = dict(gammaK=0.01, mu=0.01, kappa=0.02, cv=5.0, alpha=10.0, beta=10.0)


def _run_error(orc, lib, fo, prm, N, n, dt, nsteps, rk=4):
    ms = mesh_spec(2, N, [n, n])
    o = oracle_objects(orc, ms, prm)
    x = o.node_coords()
    U = o.run(mms_gen.exact_state(lib, x, 0.0), nsteps, dt, rk=rk, forcing=fo)
    Ue = mms_gen.exact_state(lib, x, nsteps * dt)
    return np.sqrt(((U - Ue) ** 2).mean(axis=(1, 2))), U


@pytest.mark.parametrize("model,N", [(1, 2), (1, 3), (2, 3)])
def test_spatial_convergence(orc, model, N):
    prm = dict(MMS, model=model)
    lib, _, fo = mms_gen.build(prm)
    e8, _ = _run_error(orc, lib, fo, prm, N, 8, 2e-4, 100)
    e16, _ = _run_error(orc, lib, fo, prm, N, 16, 2e-4, 100)
    eoc = np.log2(e8 / e16)
    assert np.all(eoc > N + 0.5), eoc


@pytest.mark.parametrize("rk,order", [(3, 3), (4, 4)])
def test_temporal_convergence(orc, rk, order):
    prm = dict(MMS, model=1)
    lib, _, fo = mms_gen.build(prm)
    tend = 0.032
    sols = {}
    for dt in (2e-3, 1e-3, 2.5e-4):
        _, U = _run_error(orc, lib, fo, prm, 3, 4, dt, int(round(tend / dt)), rk=rk)
        sols[dt] = U
    ref = sols[2.5e-4]
    e1 = np.abs(sols[2e-3] - ref).max()
    e2 = np.abs(sols[1e-3] - ref).max()
    # error(dt) ~ dt^p; the reference has (1/8)^p of the coarse error
    p = np.log2(e1 / e2)
    assert p > order - 0.3, p

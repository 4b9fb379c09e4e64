"""The CUDA path against the FP64 oracle on two of the paper-derived workloads at their
full sizes (not reduced meshes):

- static droplet (2D, N = 4, 64x64 elements of [0,1]^2, T = 0.8, r = 0.25, tanh interface
  with L_i(0.8), 1e-3 seeded density noise, u = 0, c = rho; relaxation model 1, LSRK4):
  10 steps, FP64 form, relative L2 per conserved variable at 1e-12;
- sessile droplet (3D, N = 5, 32x32x16 elements of [0,1]^2 x [0,0.5], periodic in x and
  y, no-slip isothermal walls at T = 0.85 with contact angles 60 deg (bottom) and 90 deg
  (top), hemispherical cap r = 0.3 on the bottom wall, T = 0.85): a number of LSRK4
  steps (100 by default; DGK_SESSILE_ORACLE_STEPS), the FP64 form at 1e-12 and the
  FP32-bulk form within its per-variable bounds, both against the oracle.

Both sides evaluate the same seeded input recipe at their own node coordinates with
their own saturation densities and interface widths; dt is the oracle's."""
import os

import numpy as np
import pytest

from cases import PAPER_PARAMS, dgk_context, mesh_spec, oracle_objects, rel_l2
from paper_2208_05310_gb300 import inputs

pytestmark = pytest.mark.gpu

FP32_BOUND = np.array([1e-5, 1e-4, 1e-4, 1e-4, 1e-5, 1e-5])  # rho, momentum x/y/z, rho e, c


def _droplet_2d(x, thermo):
    rv, rl, width = thermo
    noise = inputs.uniform_noise(x[0].shape, 2208)
    return inputs.droplet(x, [0.5, 0.5], 0.25, rv, rl, width, 0.8, noise=noise, noise_amp=1e-3)


def test_static_droplet_against_oracle(orc):
    from paper_2208_05310_gb300 import dgk
    ms = mesh_spec(2, 4, [64, 64])
    o = oracle_objects(orc, ms, PAPER_PARAMS)
    Uo = o.set_primitive(_droplet_2d(o.node_coords(), (*orc.maxwell(0.8), orc.interface_width(0.8))))
    dt = o.max_dt(Uo)
    g = dgk_context(ms, PAPER_PARAMS)
    g.set_primitive(_droplet_2d(g.node_coords(), (*dgk.maxwell(0.8), dgk.interface_width(0.8))))
    e0 = rel_l2(g.download_state(), Uo)
    g.run(10, dt)
    g.status()
    ref = o.run(Uo, 10, dt, rk=4)
    err = rel_l2(g.download_state(), ref)
    print(f"static droplet 64x64 N=4, 10 steps: initial state {np.array2string(e0, precision=1)}, "
          f"after 10 steps {np.array2string(err, precision=1)}")
    assert np.all(e0 < 1e-12) and np.all(err < 1e-12), (e0, err)
    g.close()


def _sessile(x, thermo):
    rv, rl, width = thermo
    return inputs.droplet(x, [0.5, 0.5, 0.0], 0.3, rv, rl, width, 0.85)


def test_sessile_droplet_against_oracle(orc):
    from paper_2208_05310_gb300 import dgk
    steps = int(os.environ.get("DGK_SESSILE_ORACLE_STEPS", "100"))
    ms = mesh_spec(3, 5, [32, 32, 16], hi=[1.0, 1.0, 0.5], periodic=[1, 1, 0],
                   walls={4: (0.85, 60.0), 5: (0.85, 90.0)})
    o = oracle_objects(orc, ms, PAPER_PARAMS)
    Uo = o.set_primitive(_sessile(o.node_coords(), (*orc.maxwell(0.85), orc.interface_width(0.85))))
    dt = o.max_dt(Uo)
    got = {}
    for prec in ("fp64", "fp32bulk"):
        g = dgk_context(ms, PAPER_PARAMS, precision=prec)
        g.set_primitive(_sessile(g.node_coords(), (*dgk.maxwell(0.85), dgk.interface_width(0.85))))
        g.run(steps, dt)
        g.status()
        got[prec] = g.download_state()
        g.close()
    ref = o.run(Uo, steps, dt, rk=4)
    e64 = rel_l2(got["fp64"], ref)
    e32 = rel_l2(got["fp32bulk"], ref)
    print(f"sessile droplet 32x32x16 N=5, {steps} steps against the oracle: FP64 {np.array2string(e64, precision=2)}, "
          f"FP32-bulk {np.array2string(e32, precision=2)}")
    assert np.all(e64 < 1e-12), e64
    assert np.all(e32 < FP32_BOUND), e32

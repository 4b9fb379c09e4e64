"""Parity at full size: the confined-bridge workload the bench times (3D, N = 5,
64x64x32 elements, 28.3 M nodes, same kernels and launch shapes), right-hand side
sampled element by element against the oracle.

The right-hand side of an element depends on the state of elements at most three
elements away (pass-1 lifting -> temperature -> pass-2 lifting -> face data of the
neighbours), and the initial energy on one more (the lifted grad c of set-up).  The
oracle therefore evaluates the same input recipe on a 9x9x9-element sub-box centred on
the sampled element (aligned with a wall when the element is within four elements of
it, with an artificial wall or periodic wrap at the far side), and the centre element's
right-hand side is exact.

The check is on what a time step does with the right-hand side: per conserved variable
over the sampled element's nodes, the difference of the increments dt*U_t (dt the
oracle's stable step for the sub-box) relative to the element's state, with the floors
of rel_l2.  FP64: 1e-12, the bar for conserved variables; FP32-bulk: the per-variable
bounds of one step of the FP32-bulk parity tests.  (At rest, U_t is round-off in the
quiescent liquid and vapour and in the z-momentum away from the walls.)

The right-hand side's own relative error per variable is asserted against the oracle's
response to the inputs' known discrepancies: every state value perturbed by one unit
round-off of the precision (2^-52; 2^-24 for FP32-bulk), and the node coordinates
perturbed by the largest difference between the two sides' own coordinates of these
elements (each side evaluates the recipe at its own nodes; on curved elements the two
evaluate the element maps differently).  Bound: max(1e-12, or 2e-4 (4e-4 curved) for
FP32-bulk, 20 x the larger response).  The response matters at the interface, where
U_t is led by the Rusanov jump term lambda (U+ - U-) (lambda ~ 13), the difference of two
interpolated traces, which magnifies their rounding (the oracle's own response there
is ~2e-12 in rho in FP64 and ~4e-4 in FP32), and in the bulk, where the volume and
surface terms of the pressure (~300 in size) cancel to a U_t of ~1e-2.  Both states are
checked: at rest, and with a smooth velocity field (periodic with the box, 0.03..0.05 in
magnitude) added.

The curved variant (the bench's `--mesh curved`: degree-2 maps, walls bent) gives the
oracle's sub-box the full mesh's element maps of its elements; the sub-box's own seams
(its periodic wrap, its artificial far wall) are four elements from the sampled one, as
on the box.  Its FP32-bulk bounds are twice the box's, as in the curved parity tests."""
import numpy as np
import pytest

from cases import rel_l2

pytestmark = pytest.mark.gpu

# interface (bridge radius 0.5 about x = y = 1) at mid-height and at both walls, liquid
# core, vapour, vapour next to the bottom wall
SAMPLES = [(47, 32, 16), (16, 32, 0), (32, 47, 31), (31, 32, 8), (5, 5, 16), (48, 48, 1)]


def _sub_box(orc, wl, ix, iy, iz, W=9, geo=None):
    m = wl["mesh"]
    h = [(m["hi"][d] - m["lo"][d]) / m["n"][d] for d in range(3)]
    nz = m["n"][2]
    x0, y0 = ix - W // 2, iy - W // 2
    if iz <= W // 2:
        z0, periodic_z, walls = 0, 0, {4: m["walls"][4], 5: (0.85, 90.0)}
    elif iz >= nz - 1 - W // 2:
        z0, periodic_z, walls = nz - W, 0, {4: (0.85, 90.0), 5: m["walls"][5]}
    else:
        z0, periodic_z, walls = iz - W // 2, 1, {}
    lo = [m["lo"][0] + x0 * h[0], m["lo"][1] + y0 * h[1], m["lo"][2] + z0 * h[2]]
    hi = [lo[0] + W * h[0], lo[1] + W * h[1], lo[2] + W * h[2]]
    sub_geo = None
    if geo is not None:
        nx, ny = m["n"][0], m["n"][1]
        ez, ey, ex = np.meshgrid(np.arange(z0, z0 + W), np.arange(y0, y0 + W), np.arange(x0, x0 + W), indexing="ij")
        full = (ex + nx * (ey + ny * ez)).ravel()  # sub-box elements, x fastest
        sub_geo = (geo[0], np.ascontiguousarray(geo[1][:, full, :]))
    mesh = orc.make_mesh(3, m["N"], [W, W, W], lo, hi, [1, 1, periodic_z], walls, geometry=sub_geo)
    local = (ix - x0) + W * ((iy - y0) + W * (iz - z0))
    nx, ny = m["n"][0], m["n"][1]
    ez, ey, ex = np.meshgrid(np.arange(z0, z0 + W), np.arange(y0, y0 + W), np.arange(x0, x0 + W), indexing="ij")
    full = (ex % nx + nx * ((ey % ny) + ny * ez)).ravel()  # the sub-box's elements in the full mesh
    return orc.Oracle(mesh, orc.make_params(**wl["params"])), local, full


def moving_state(bench, wl, x, rv, rl, width):
    """The bench's initial state with a smooth velocity field added (periodic in x and y
    with the box's period 2): U_t is then led by the transport terms rather than by the
    interface jump terms."""
    prim = bench.primitive_state(wl, x, rv, rl, width)
    prim[1] += 0.05 * np.cos(np.pi * x[1])
    prim[2] += 0.04 * np.cos(np.pi * x[0] + 0.3)
    prim[3] += 0.03 * np.cos(np.pi * (x[0] + x[1])) * np.sin(np.pi * x[2])
    return prim


@pytest.mark.parametrize("state", ["rest", "moving"])
@pytest.mark.parametrize("mesh", ["box", "curved"])
@pytest.mark.parametrize("precision", ["fp64", "fp32bulk"])
def test_fullsize_sampled_rhs(orc, precision, mesh, state):
    import bench
    from paper_2208_05310_gb300 import dgk
    wl = bench.workload_c5()
    m = wl["mesh"]
    geo = bench.geometry_of(m, bench.CURVED_GEOMETRY) if mesh == "curved" else None
    recipe = bench.primitive_state if state == "rest" else (lambda w, x, a, b, c: moving_state(bench, w, x, a, b, c))
    g = dgk.Context()
    g.set_params(rk=wl["rk"], precision=precision, **wl["params"])
    if geo is not None:
        g.mesh_curved(3, m["N"], m["n"], m["periodic"], m["walls"], *geo)
    else:
        g.mesh_box(3, m["N"], m["n"], m["lo"], m["hi"], m["periodic"], m["walls"])
    rv, rl = dgk.maxwell(wl["T0"])
    width = dgk.interface_width(wl["T0"], wl["params"]["cv"], wl["params"]["gammaK"])
    xg = g.node_coords()
    g.set_primitive(recipe(wl, xg, rv, rl, width))
    Ut = g.rhs()
    g.close()
    orv, orl = orc.maxwell(wl["T0"])
    owidth = orc.interface_width(wl["T0"], wl["params"]["cv"], wl["params"]["gammaK"])
    nx, ny = m["n"][0], m["n"][1]
    for (ix, iy, iz) in SAMPLES:
        o, local, full = _sub_box(orc, wl, ix, iy, iz, geo=geo)
        xo = o.node_coords()
        Uo = o.set_primitive(recipe(wl, xo, orv, orl, owidth))
        ref = o.rhs(Uo)[:, local, :]
        dt = o.max_dt(Uo)
        e = ix + nx * (iy + ny * iz)
        got = Ut[:, e, :]
        snorm = np.sqrt((Uo[:, local, :] ** 2).sum(axis=1))
        den = np.maximum(snorm, 1e-3 * snorm.max())
        err = dt * np.sqrt(((got - ref) ** 2).sum(axis=1)) / den
        rhs_err = rel_l2(got[:, None, :], ref[:, None, :])
        print(f"{precision} {mesh} {state} sample {(ix, iy, iz)}: increment error / state "
              f"{np.array2string(err, precision=1)}, rhs relative {np.array2string(rhs_err, precision=1)}")
        tol = np.full(6, 1e-12) if precision == "fp64" else np.array([1e-7, 3e-5, 3e-5, 3e-5, 2e-7, 5e-7])
        if mesh == "curved" and precision != "fp64":
            tol = 2.0 * tol
        assert np.all(err < tol), ((ix, iy, iz), err, tol)
        # the right-hand side's own relative error per variable, against the oracle's own
        # response to the inputs' known discrepancies: every state value perturbed by one
        # unit round-off of the precision (2^-52, or 2^-24 for FP32-bulk), and the node
        # coordinates perturbed by the largest difference between the two sides' own
        # coordinates of these elements (each side evaluates the recipe at its own nodes);
        # bound max(the right-hand-side tolerance, 20 x the larger response)
        rng = np.random.default_rng(ix + 64 * iy + 4096 * iz)
        u_r = 2.0 ** -52 if precision == "fp64" else 2.0 ** -24
        sens_u = rel_l2(o.rhs(Uo * (1.0 + u_r * rng.uniform(-1.0, 1.0, Uo.shape)))[:, local, :][:, None, :],
                        ref[:, None, :])
        dx = np.abs(xg[:, full, :] - xo).max()
        Ux = o.set_primitive(recipe(wl, xo + dx * rng.uniform(-1.0, 1.0, xo.shape), orv, orl, owidth))
        sens_x = rel_l2(o.rhs(Ux)[:, local, :][:, None, :], ref[:, None, :])
        rtol = 1e-12 if precision == "fp64" else (2e-4 if mesh == "box" else 4e-4)
        bound = np.maximum(rtol, 20.0 * np.maximum(sens_u, sens_x))
        print(f"    oracle response: state ulp {np.array2string(sens_u, precision=1)}, "
              f"coordinates (max difference {dx:.1e}) {np.array2string(sens_x, precision=1)}")
        assert np.all(rhs_err < bound), ((ix, iy, iz), rhs_err, bound)

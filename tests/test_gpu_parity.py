"""GPU parity: libdgk (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Each side evaluates the input recipe at its own node coordinates, with its own
saturation densities and interface width, and converts it to its own conserved state.

Bar: FP64 form within 1e-12 relative L2 per conserved variable (right-hand side and
states after 1, 10 and 200 steps); FP32-bulk form within the per-variable tolerances
stated below."""
import numpy as np
import pytest

from cases import PAPER_PARAMS, dgk_context, droplet_state, mesh_spec, oracle_objects, rel_l2

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _thermo_oracle(orc, T=0.85, gK=1e-4):
    rv, rl = orc.maxwell(T)
    return rv, rl, orc.interface_width(T, 5.0, gK)


def _thermo_dgk(T=0.85, gK=1e-4):
    from paper_2208_05310_gb300 import dgk
    rv, rl = dgk.maxwell(T)
    return rv, rl, dgk.interface_width(T, 5.0, gK)


def _lengths(ms):
    return [ms["hi"][d] - ms["lo"][d] for d in range(ms["dim"])]


def _state_pair(orc, ms, ps, precision="fp64", rk=4, radius=0.3, center=None, seed=7):
    o = oracle_objects(orc, ms, ps)
    g = dgk_context(ms, ps, precision=precision, rk=rk)
    kw = dict(radius=radius, center=center, perturb_seed=seed, lengths=_lengths(ms))
    prim_o = droplet_state(o.node_coords(), _thermo_oracle(orc), **kw)
    prim_g = droplet_state(g.node_coords(), _thermo_dgk(), **kw)
    Uo = o.set_primitive(prim_o)
    g.set_primitive(prim_g)
    return o, g, Uo


CASES = {
    "2d_N2_periodic": (mesh_spec(2, 2, [5, 3]), dict(PAPER_PARAMS)),
    "2d_N3_periodic": (mesh_spec(2, 3, [5, 3]), dict(PAPER_PARAMS)),
    "2d_N4_periodic_m2": (mesh_spec(2, 4, [3, 4]), dict(PAPER_PARAMS, model=2)),
    "2d_N5_periodic": (mesh_spec(2, 5, [3, 3]), dict(PAPER_PARAMS)),
    "2d_N3_walls": (mesh_spec(2, 3, [4, 3], periodic=[1, 0], walls={2: (0.85, 60.0), 3: (0.8, 120.0)}),
                    dict(PAPER_PARAMS)),
    "2d_N4_walls_m2": (mesh_spec(2, 4, [3, 3], periodic=[1, 0], walls={2: (0.9, 30.0), 3: (0.85, 150.0)}),
                       dict(PAPER_PARAMS, model=2)),
    "3d_N2_periodic": (mesh_spec(3, 2, [2, 3, 2]), dict(PAPER_PARAMS)),
    "3d_N3_walls": (mesh_spec(3, 3, [2, 2, 3], periodic=[1, 1, 0], walls={4: (0.85, 60.0), 5: (0.85, 90.0)}),
                    dict(PAPER_PARAMS)),
    "3d_N4_periodic_m2": (mesh_spec(3, 4, [2, 1, 3]), dict(PAPER_PARAMS, model=2)),
    "3d_N5_walls": (mesh_spec(3, 5, [2, 2, 2], periodic=[1, 1, 0], walls={4: (0.95, 90.0), 5: (0.8, 90.0)}),
                    dict(PAPER_PARAMS)),
    "2d_N4_walls_m2_hllc": (mesh_spec(2, 4, [3, 3], periodic=[1, 0], walls={2: (0.9, 30.0), 3: (0.85, 150.0)}),
                            dict(PAPER_PARAMS, model=2, flux="hllc")),
    "3d_N3_walls_m2_hllc": (mesh_spec(3, 3, [2, 2, 3], periodic=[1, 1, 0], walls={4: (0.85, 60.0), 5: (0.85, 90.0)}),
                            dict(PAPER_PARAMS, model=2, flux="hllc")),
    "2d_N4_slip": (mesh_spec(2, 4, [3, 3], periodic=[1, 0], walls={2: (0.9, 30.0, 0.02, 0.1, 0.3, 0.5),
                                                                   3: (0.85, 150.0, 0.01, 0.2, 0.1, 1.0)}),
                   dict(PAPER_PARAMS)),
    "3d_N3_slip_m2": (mesh_spec(3, 3, [2, 2, 3], periodic=[1, 1, 0], walls={4: (0.85, 60.0, 0.03, 0.05, 0.2, 0.3),
                                                                            5: (0.8, 90.0, 0.0, 0.5, 1.0, 0.0)}),
                      dict(PAPER_PARAMS, model=2)),
    # sliding no-slip walls (the moving wall of the sliding-droplet case, Sec. 4)
    "2d_N4_sliding": (mesh_spec(2, 4, [3, 3], periodic=[1, 0], walls={2: (0.85, 60.0), 3: (0.8, 120.0, (0.3, 0.0, 0.0))}),
                      dict(PAPER_PARAMS)),
    "3d_N3_sliding_m2_hllc": (mesh_spec(3, 3, [2, 2, 3], periodic=[1, 1, 0],
                                        walls={4: (0.85, 60.0, (0.0, 0.1, 0.0)), 5: (0.85, 90.0, (0.2, -0.1, 0.0))}),
                              dict(PAPER_PARAMS, model=2, flux="hllc")),
    "2d_single_element": (mesh_spec(2, 3, [1, 1]), dict(PAPER_PARAMS)),
    "3d_single_element_walls": (mesh_spec(3, 3, [1, 1, 1], periodic=[1, 1, 0],
                                          walls={4: (0.85, 45.0), 5: (0.85, 135.0)}), dict(PAPER_PARAMS)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_set_primitive_parity(orc, name):
    ms, ps = CASES[name]
    o, g, Uo = _state_pair(orc, ms, ps)
    assert np.all(rel_l2(g.download_state(), Uo) < TOL64)


def _exact_input_pair(orc, ms, ps, precision="fp64", rk=4, seed=11):
    """Both sides receive the identical coordinate-free primitive array."""
    from paper_2208_05310_gb300 import inputs
    o = oracle_objects(orc, ms, ps)
    g = dgk_context(ms, ps, precision=precision, rk=rk)
    prim = inputs.random_admissible(ms["dim"], o.nelem, o.np, seed)
    Uo = o.set_primitive(prim)
    g.set_primitive(prim)
    return o, g, Uo


@pytest.mark.parametrize("name", sorted(CASES))
def test_rhs_parity_fp64_exact_inputs(orc, name):
    """Identical inputs: the right-hand side agrees to 1e-12 per variable."""
    ms, ps = CASES[name]
    o, g, Uo = _exact_input_pair(orc, ms, ps)
    assert np.all(rel_l2(g.download_state(), Uo) < 1e-14)
    err = rel_l2(g.rhs(), o.rhs(Uo))
    assert np.all(err < TOL64), err


def _coordinate_sensitivity(orc, ms, ps, make_prim):
    """The oracle's own right-hand-side response to perturbing the node coordinates by
    one ulp before evaluating the input recipe: the scale of the input difference the
    two sides see (each evaluates the steep tanh profile at its own coordinates)."""
    o = oracle_objects(orc, ms, ps)
    x = o.node_coords()
    xi = np.random.default_rng(5).uniform(-1, 1, x.shape)
    r1 = o.rhs(o.set_primitive(make_prim(x)))
    r2 = o.rhs(o.set_primitive(make_prim(x * (1 + 2.0 ** -52 * xi))))
    return rel_l2(r2, r1)


@pytest.mark.parametrize("name", sorted(CASES))
def test_rhs_parity_fp64_profile(orc, name):
    """Droplet profile evaluated by each side at its own node coordinates: the right-hand
    side agrees within max(1e-12, 20 x the oracle's sensitivity to a one-ulp coordinate
    perturbation), per variable."""
    ms, ps = CASES[name]
    o, g, Uo = _state_pair(orc, ms, ps)
    err = rel_l2(g.rhs(), o.rhs(Uo))
    kw = dict(radius=0.3, perturb_seed=7, lengths=_lengths(ms))
    th = _thermo_oracle(orc)
    sens = _coordinate_sensitivity(orc, ms, ps, lambda x: droplet_state(x, th, **kw))
    tol = np.maximum(TOL64, 20 * sens)
    assert np.all(err < tol), (err, tol)


@pytest.mark.parametrize("name", sorted(CASES))
def test_one_step_parity_fp64_exact_inputs(orc, name):
    ms, ps = CASES[name]
    o, g, Uo = _exact_input_pair(orc, ms, ps)
    dt = 0.5 * o.max_dt(Uo)
    g.rk_step(dt)
    g.status()
    err = rel_l2(g.download_state(), o.run(Uo, 1, dt, rk=4))
    assert np.all(err < TOL64), err


@pytest.mark.parametrize("name", sorted(CASES))
def test_one_step_parity_fp64(orc, name):
    ms, ps = CASES[name]
    o, g, Uo = _state_pair(orc, ms, ps)
    dt = o.max_dt(Uo)
    g.rk_step(dt)
    g.status()
    err = rel_l2(g.download_state(), o.run(Uo, 1, dt, rk=4))
    assert np.all(err < TOL64), err


@pytest.mark.parametrize("name,rk", [("2d_N3_walls", 3), ("3d_N3_walls", 4), ("2d_N4_periodic_m2", 4), ("2d_N4_sliding", 4)])
def test_ten_steps_parity_fp64(orc, name, rk):
    ms, ps = CASES[name]
    o, g, Uo = _state_pair(orc, ms, ps, rk=rk)
    dt = o.max_dt(Uo, cfl=0.5 if rk == 3 else 0.9)
    g.run(10, dt)
    g.status()
    err = rel_l2(g.download_state(), o.run(Uo, 10, dt, rk=rk))
    assert np.all(err < TOL64), err


def test_planar_interface_200_steps_lsrk3(orc):
    """Planar-interface workload: periodic strip [0,0.5]x[0,0.125], N = 3 on 16x4
    elements, T = 0.85, LSRK3, 200 steps at the oracle's CFL-limited dt."""
    from paper_2208_05310_gb300 import inputs
    ms = mesh_spec(2, 3, [16, 4], hi=[0.5, 0.125])
    o = oracle_objects(orc, ms, PAPER_PARAMS)
    g = dgk_context(ms, PAPER_PARAMS, rk=3)
    rv, rl, L = _thermo_oracle(orc)
    Uo = o.set_primitive(inputs.planar_slab(o.node_coords(), rv, rl, L, 0.125, 0.375, 0.85))
    rv, rl, L = _thermo_dgk()
    g.set_primitive(inputs.planar_slab(g.node_coords(), rv, rl, L, 0.125, 0.375, 0.85))
    dt = o.max_dt(Uo, cfl=0.5)
    g.run(200, dt)
    g.status()
    err = rel_l2(g.download_state(), o.run(Uo, 200, dt, rk=3))
    assert np.all(err < TOL64), err


@pytest.mark.parametrize("name", ["2d_N3_walls", "3d_N5_walls", "2d_N4_periodic_m2"])
def test_max_dt_and_diagnostics_parity(orc, name):
    ms, ps = CASES[name]
    o, g, Uo = _state_pair(orc, ms, ps)
    assert abs(g.max_dt() / o.max_dt(Uo) - 1) < 1e-12
    dg, do = g.diagnostics(), o.diagnostics(Uo)
    for k in dg:
        scale = max(abs(do[k]), 1e-12)
        assert abs(dg[k] - do[k]) <= 1e-12 * scale + 1e-15, (k, dg[k], do[k])


# FP32-bulk form: bulk lifting, volume and surface arithmetic in FP32; energy balance
# of the temperature recovery and the RK accumulation in FP64.  Tolerances per conserved
# variable (relative L2 with the floors of rel_l2).  The right-hand side carries the
# FP32 rounding unit 6e-8 amplified by two differentiations (about (2N^2/h)^2 ulp on
# these meshes); the state after 10 steps carries dt times that, accumulated in FP64.
# Momentum is normalised by its own (small) norm, hence its larger bound.
TOL32_RHS = 2e-4


def tol32_step(dim):
    return np.array([1e-7] + [3e-5] * dim + [2e-7, 5e-7])


@pytest.mark.parametrize("name", ["2d_N3_walls", "3d_N3_walls", "3d_N5_walls", "2d_N4_periodic_m2", "2d_N4_walls_m2_hllc",
                                  "3d_N3_walls_m2_hllc", "2d_N4_slip", "3d_N3_slip_m2", "2d_N4_sliding",
                                  "3d_N3_sliding_m2_hllc"])
def test_fp32_bulk_against_oracle(orc, name):
    ms, ps = CASES[name]
    o, g, Uo = _state_pair(orc, ms, ps, precision="fp32bulk")
    e_rhs = rel_l2(g.rhs(), o.rhs(Uo))
    assert np.all(e_rhs < TOL32_RHS), e_rhs
    dt = o.max_dt(Uo)
    g.run(10, dt)
    g.status()
    e_st = rel_l2(g.download_state(), o.run(Uo, 10, dt, rk=4))
    assert np.all(e_st < tol32_step(ms["dim"])), e_st


def test_device_status_flags_bad_state(orc):
    """A non-finite or out-of-domain state is reported through the status word (no
    trap); a later valid state runs cleanly."""
    from paper_2208_05310_gb300 import dgk
    ms, ps = CASES["2d_N3_periodic"]
    o, g, Uo = _state_pair(orc, ms, ps)
    bad = Uo.copy()
    bad[0, 3, 5] = np.nan
    g.upload_state(bad)
    g.run(1, 1e-5)
    assert g.status_code() == -3
    bad = Uo.copy()
    bad[0, 2, 1] = 3.5  # rho > 1/b
    g.upload_state(bad)
    g.rk_step(1e-6)
    assert g.status_code() in (-3, -4)
    g.upload_state(Uo)
    g.run(2, 1e-5)
    g.status()
    with pytest.raises(dgk.DgkError):
        g.upload_state(Uo[:, :-1])


def test_integer_conversions_match_hardware():
    """The FP32-bulk kernels convert double <-> float with integer arithmetic; the results
    are bit-identical to the GPU's round-to-nearest conversions (random magnitudes over
    the float range, exact halfway cases, signed zeros, infinities, NaN)."""
    from paper_2208_05310_gb300 import dgk
    rng = np.random.default_rng(3)
    x = np.concatenate([
        rng.standard_normal(200000) * 10.0 ** rng.uniform(-30, 30, 200000),
        rng.uniform(-4, 4, 100000),
        # halfway cases: a float plus exactly half an ulp (ties to even), and neighbours
        (np.float32(rng.uniform(0.5, 2, 20000)).astype(np.float64) * (1 + 2.0 ** -24)),
        (np.float32(rng.uniform(0.5, 2, 20000)).astype(np.float64) * (1 + 2.0 ** -24 + 2.0 ** -40)),
        np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 3.4028234663852886e38, 3.4028235e38 * 1.0000001,
                  1.1754943508222875e-38, 1.0, -1.0, 2.0 ** 127, 2.0 ** -126]),
    ])
    assert dgk.check_conversions(x) == 0


def test_sliding_wall_refusals():
    from paper_2208_05310_gb300 import dgk
    with pytest.raises(dgk.DgkError):  # a normal component
        dgk_context(mesh_spec(2, 3, [2, 2], periodic=[1, 0], walls={2: (0.85, 90.0), 3: (0.85, 90.0, (0.1, 0.2, 0.0))}),
                    PAPER_PARAMS)


def test_box_mesh_and_call_refusals():
    """Input checks of the C ABI (no kernel runs for a refused call): polynomial degree and
    dimension ranges, walls on every non-periodic face, wall parameters, wall
    temperatures with saturation states, the element-count and plane-size limits (refused
    before any allocation), call order, array sizes and step sizes."""
    from paper_2208_05310_gb300 import dgk, inputs

    def ctx():
        g = dgk.Context()
        g.set_params(**PAPER_PARAMS)
        return g

    g = ctx()
    with pytest.raises(dgk.DgkError):  # call order: no mesh yet
        g.rhs(np.zeros(10))
    for N in (1, 6):
        with pytest.raises(dgk.DgkError):
            ctx().mesh_box(2, N, [2, 2, 1], [0, 0, 0], [1, 1, 1], [1, 1, 1])
    with pytest.raises(dgk.DgkError):
        ctx().mesh_box(4, 3, [2, 2, 2], [0, 0, 0], [1, 1, 1], [1, 1, 1])
    with pytest.raises(dgk.DgkError):  # a non-periodic direction without walls
        ctx().mesh_box(2, 3, [2, 2, 1], [0, 0, 0], [1, 1, 1], [1, 0, 1])
    with pytest.raises(dgk.DgkError):  # a negative Navier-slip parameter
        ctx().mesh_box(2, 3, [2, 2, 1], [0, 0, 0], [1, 1, 1], [1, 0, 1],
                       {2: (0.85, 90.0, 0.0, -0.1, 0.0, 0.0), 3: (0.85, 90.0)})
    with pytest.raises(dgk.DgkError):  # no saturation states above the critical temperature
        ctx().mesh_box(2, 3, [2, 2, 1], [0, 0, 0], [1, 1, 1], [1, 0, 1], {2: (1.2, 90.0), 3: (0.85, 90.0)})
    with pytest.raises(dgk.DgkError):  # 2^33 elements
        ctx().mesh_box(3, 3, [2 ** 16, 2 ** 16, 2], [0, 0, 0], [1, 1, 1], [1, 1, 1])
    # fewer than 2^32 elements, but a node plane of 2^25 * 216 > 2^32 values: the kernels
    # index inside a plane with 32 bits
    with pytest.raises(dgk.DgkError, match="2\\^32 - 1 nodes"):
        ctx().mesh_box(3, 5, [1024, 1024, 32], [0, 0, 0], [1, 1, 1], [1, 1, 1])
    with pytest.raises(dgk.DgkError):  # an empty extent
        ctx().mesh_box(2, 3, [2, 2, 1], [0, 0, 0], [1, 0, 1], [1, 1, 1])
    g = ctx()
    g.mesh_box(2, 3, [2, 2, 1], [0, 0, 0], [1, 1, 1], [1, 1, 1])
    with pytest.raises(dgk.DgkError):  # a state of the wrong size
        g.upload_state(np.zeros(g.nv * g.nelem * g.np - 1))
    g.set_primitive(inputs.random_admissible(2, g.nelem, g.np, 1))
    for dt in (0.0, -1.0, float("nan")):
        with pytest.raises(dgk.DgkError):
            g.run(1, dt)
    with pytest.raises(dgk.DgkError):
        g.run(-1, 1e-4)

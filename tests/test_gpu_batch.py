"""Batched ensembles: many independent 2D droplet / bubble problems of different degree,
mesh size, temperature and contact angle advanced by one persistent launch per RK stage
(FP32-bulk form).

Checks: against the FP64 oracle within the FP32-bulk step tolerances; against the same
problems run one by one through single contexts; independence of the work
decomposition (bit-exact across tile lengths and grid sizes within a form, FP32
rounding between the persistent and the grouped kernels); the autotuner leaves the
states untouched; and at the full ensemble size (256 problems, 16x16 to 96x96 elements)
sampled problems match single-context runs and mass is conserved."""
import numpy as np
import pytest

from cases import PAPER_PARAMS, oracle_objects, rel_l2

pytestmark = pytest.mark.gpu


# batch kernels against single-problem kernels (and the two batch forms): the same
# arithmetic in separate kernels, whose compiled floating-point contraction may differ;
# FP32 rounding of U_t seen through dt in the FP64 state (momentum normalised by its own
# small norm)
SAME_FORM_TOL = np.array([1e-9, 1e-6, 1e-6, 1e-9, 1e-9])


def tol32_step():
    return np.array([1e-7, 3e-5, 3e-5, 2e-7, 5e-7])  # rho, rho u, rho v, E, c (after 10 steps)


def _thermo_dgk(T):
    from paper_2208_05310_gb300 import dgk
    rv, rl = dgk.maxwell(T)
    return rv, rl, dgk.interface_width(T, 5.0, PAPER_PARAMS["gammaK"])


def _thermo_oracle(orc, T):
    rv, rl = orc.maxwell(T)
    return rv, rl, orc.interface_width(T, 5.0, PAPER_PARAMS["gammaK"])


def ensemble(nprob, seed, n_range):
    from paper_2208_05310_gb300 import inputs
    specs = inputs.ensemble_specs(nprob, seed, n_range=n_range)
    return specs, [inputs.ensemble_mesh(s) for s in specs]


def _prim(x, spec, thermo):
    from paper_2208_05310_gb300 import inputs
    return inputs.ensemble_primitive(x, spec, *thermo)


def _batch(meshes, specs, dt_frac=0.5):
    from paper_2208_05310_gb300 import dgk
    b = dgk.Batch(meshes, **PAPER_PARAMS)
    prims, dts = [], []
    for q, s in zip(b.problems, specs):
        prim = _prim(q.node_coords(), s, _thermo_dgk(s["T"]))
        q.set_primitive(prim)
        prims.append(prim)
        dts.append(dt_frac * q.max_dt())
    b.set_dt(dts)
    return b, prims, dts


def _single(ms, prim, dt, nsteps):
    from cases import dgk_context
    g = dgk_context(ms, dict(PAPER_PARAMS), precision="fp32bulk")
    g.set_primitive(prim)
    g.run(nsteps, dt)
    g.status()
    U = g.download_state()
    g.close()
    return U


def test_batch_against_oracle(orc):
    specs, meshes = ensemble(3, 5, (3, 5))
    for k, N in enumerate((3, 4, 5)):
        specs[k]["N"] = N
        meshes[k]["N"] = N
    from paper_2208_05310_gb300 import dgk
    b = dgk.Batch(meshes, **PAPER_PARAMS)
    ref, dts = [], []
    for q, s, ms in zip(b.problems, specs, meshes):
        o = oracle_objects(orc, ms, dict(PAPER_PARAMS))
        Uo = o.set_primitive(_prim(o.node_coords(), s, _thermo_oracle(orc, s["T"])))
        q.set_primitive(_prim(q.node_coords(), s, _thermo_dgk(s["T"])))
        dt = 0.5 * o.max_dt(Uo)
        dts.append(dt)
        ref.append(o.run(Uo, 10, dt, rk=4))
    b.set_dt(dts)
    b.run(10)
    assert all(rc == 0 for rc in b.status())
    for q, Uo in zip(b.problems, ref):
        err = rel_l2(q.download_state(), Uo)
        assert np.all(err < tol32_step()), (q.N, err)
    b.close()


def test_batch_matches_single_contexts():
    specs, meshes = ensemble(8, 11, (4, 12))
    b, prims, dts = _batch(meshes, specs)
    b.run(5)
    assert all(rc == 0 for rc in b.status())
    for q, ms, prim, dt in zip(b.problems, meshes, prims, dts):
        ref = _single(ms, prim, dt, 5)
        err = rel_l2(q.download_state(), ref)
        assert np.all(err < SAME_FORM_TOL), (ms["N"], ms["n"], err)
    b.close()


def test_batch_decomposition_independence_and_autotune():
    specs, meshes = ensemble(12, 17, (6, 24))
    b, prims, dts = _batch(meshes, specs)
    U0 = [q.download_state() for q in b.problems]
    out = {}
    for cfg in [("persistent", 1, 1, 1, 1), ("persistent", 1, 4, 2, 1), ("persistent", 2, 2, 4, 3),
                ("grouped", 1, 1, 1, 1), ("grouped", 1, 3, 1, 2)]:
        for q, prim in zip(b.problems, prims):
            q.set_primitive(prim)
        try:
            b.set_config(*cfg)
        except Exception:
            if cfg[1] == 1:
                raise
            continue  # two blocks per SM above the occupancy limit
        b.run(3)
        b.status()
        out.setdefault(cfg[0], []).append([q.download_state() for q in b.problems])
    # within a form (one kernel): bit-exact for every decomposition
    for form, runs in out.items():
        for other in runs[1:]:
            for a, c in zip(runs[0], other):
                assert np.array_equal(a, c), form
    # across the forms (separate kernels, whose compiled floating-point contraction may
    # differ): to the FP32 rounding of U_t, seen through dt in the FP64 state
    for a, c in zip(out["persistent"][0], out["grouped"][0]):
        assert np.all(rel_l2(c, a) < SAME_FORM_TOL)
    for q, prim in zip(b.problems, prims):
        q.set_primitive(prim)
    tuned = b.autotune()
    assert tuned["form"] in ("persistent", "grouped") and tuned["blocks_per_sm"] >= 1
    assert min(tuned["k3"], tuned["k4"], tuned["k5"]) >= 1
    for q, u in zip(b.problems, U0):  # the autotuner restores the states
        assert np.array_equal(q.download_state(), u)
    b.run(3)
    b.status()
    for a, q in zip(out[tuned["form"]][0], b.problems):
        assert np.array_equal(a, q.download_state())
    b.close()


def test_batch_full_ensemble_sampled():
    """256 problems, 16x16 to 96x96 elements, N in {3, 4, 5}: autotuned, 20 steps;
    sampled problems against single contexts, every problem's mass conserved."""
    specs, meshes = ensemble(256, 2024, (16, 96))
    b, prims, dts = _batch(meshes, specs)
    b.autotune()
    m0 = [q.diagnostics()["mass"] for q in b.problems]
    b.run(20)
    assert all(rc == 0 for rc in b.status())
    m1 = [q.diagnostics()["mass"] for q in b.problems]
    # the FP32-bulk U_t is formed in float: an element's volume and surface mass terms
    # cancel only to float rounding (~6e-8 of the largest term), so each step moves the
    # mass by ~dt * 6e-8 * sum |flux terms|, a few 1e-13 per step here (measured 3.5e-12
    # after 20 steps); the FP64 form holds it to ~1e-16 per step
    drift = np.max(np.abs(np.array(m1) / np.array(m0) - 1.0))
    print(f"ensemble mass drift over 20 steps: {drift:.2e}")
    assert drift < 1e-11
    sizes = [ms["n"][0] * ms["N"] for ms in meshes]
    for k in sorted({0, 255, int(np.argmax(sizes)), int(np.argmin(sizes))}):
        ref = _single(meshes[k], prims[k], dts[k], 20)
        err = rel_l2(b.problems[k].download_state(), ref)
        assert np.all(err < SAME_FORM_TOL), (k, meshes[k]["N"], meshes[k]["n"], err)
    b.close()


def test_batch_refuses_hllc():
    from paper_2208_05310_gb300 import dgk
    _, meshes = ensemble(2, 3, (4, 6))
    with pytest.raises(dgk.DgkError):
        dgk.Batch(meshes, **dict(PAPER_PARAMS, model=2, flux="hllc"))


def test_batch_barrier_timeout_is_reported_and_recoverable():
    """The persistent form's grid barrier gives up after its spin limit: with a limit of
    one clock cycle the early blocks' waits run out, the kernel returns (no hang) and
    dgk_batch_status reports DGK_ERR_TIMEOUT.  With the default limit restored and the
    states set again, the next run succeeds and equals a clean run bit for bit."""
    from paper_2208_05310_gb300 import dgk
    specs, meshes = ensemble(6, 23, (6, 16))
    b, prims, dts = _batch(meshes, specs)
    b.set_config("persistent", 1, 1, 1, 1)
    b.run(2)
    b.status()
    clean = [q.download_state() for q in b.problems]
    for q, prim in zip(b.problems, prims):
        q.set_primitive(prim)
    b.set_barrier_limit(1)
    b.run(1)
    assert b.status_code() == -9  # DGK_ERR_TIMEOUT
    assert b.status_code() == 0   # reported once, then cleared
    b.set_barrier_limit(4_000_000_000)  # the default
    for q, prim in zip(b.problems, prims):
        q.set_primitive(prim)
    b.run(2)
    assert all(rc == 0 for rc in b.status())
    for q, u in zip(b.problems, clean):
        assert np.array_equal(q.download_state(), u)
    with pytest.raises(dgk.DgkError):
        b.set_barrier_limit(0)
    b.close()

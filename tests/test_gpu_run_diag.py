"""Diagnostics sampled inside dgk_run, and checkpoint / resume.

- dgk_run(nsteps, dt, diag_every, diag_out) takes the integral diagnostics on the device
  after every diag_every-th step (a captured graph, no host round trip per sample): the
  trajectory is bitwise the one of a run without samples, and every sample equals, bit
  for bit, dgk_diagnostics() called after the same number of steps of a second context.
  The sampled energy, entropy and entropy-production curves are those of the paper's
  conservation and Second-Law plots (Sec. 4).
- Checkpoint / resume: 2n steps equal n steps, a download of the state, an upload (which
  resets the RK register, correct at a step boundary: the first stage has A = 0) and n
  more steps, bit for bit, in both precision forms.
- The entropy-production diagnostic of the FP32-bulk form against the oracle (the FP64
  form's is in the diagnostics parity tests at 1e-12)."""
import numpy as np
import pytest

from cases import PAPER_PARAMS, dgk_context, droplet_state, mesh_spec, oracle_objects

pytestmark = pytest.mark.gpu

MS = mesh_spec(2, 4, [6, 5], periodic=[1, 0], walls={2: (0.85, 60.0), 3: (0.8, 120.0)})
MS3 = mesh_spec(3, 3, [3, 3, 2], periodic=[1, 1, 0], walls={4: (0.85, 60.0), 5: (0.85, 90.0)})
KW = dict(radius=0.3, perturb_seed=11, lengths=[1.0, 1.0])


def _ctx(ms, precision):
    from paper_2208_05310_gb300 import dgk
    g = dgk_context(ms, PAPER_PARAMS, precision=precision)
    rv, rl = dgk.maxwell(0.85)
    kw = dict(KW, lengths=[1.0] * ms["dim"])
    g.set_primitive(droplet_state(g.node_coords(), (rv, rl, dgk.interface_width(0.85)), **kw))
    return g


@pytest.mark.parametrize("precision", ["fp64", "fp32bulk"])
@pytest.mark.parametrize("ms", [MS, MS3], ids=["2d", "3d"])
def test_in_run_diagnostics(precision, ms):
    from paper_2208_05310_gb300 import dgk
    a, b = _ctx(ms, precision), _ctx(ms, precision)
    dt = 0.5 * a.max_dt()
    nsteps, every = 12, 3
    samples = a.run(nsteps, dt, diag_every=every)
    a.status()
    ref = []
    for _ in range(nsteps // every):
        b.run(every, dt)
        b.status()
        d = b.diagnostics()
        ref.append([d[k] for k in dgk.DIAG_NAMES])
    ref = np.array(ref)
    assert samples.shape == ref.shape
    assert np.array_equal(samples, ref), (samples - ref)
    assert np.array_equal(a.download_state(), b.download_state())
    assert np.all(samples[:, dgk.DIAG_NAMES.index("entropy_production")] > 0)
    # a device buffer for the samples
    import torch
    out = torch.zeros((nsteps // every, dgk.NDIAG), dtype=torch.float64, device="cuda")
    c = _ctx(ms, precision)
    c.run(nsteps, dt, diag_every=every, diag_out=out)
    c.status()
    assert np.array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32bulk"])
@pytest.mark.parametrize("ms", [MS, MS3], ids=["2d", "3d"])
def test_checkpoint_resume_bitwise(precision, ms):
    a, b = _ctx(ms, precision), _ctx(ms, precision)
    dt = 0.5 * a.max_dt()
    n = 7
    a.run(2 * n, dt)
    a.status()
    b.run(n, dt)
    b.status()
    saved = b.download_state()
    b.close()
    c = dgk_context(ms, PAPER_PARAMS, precision=precision)
    c.upload_state(saved)
    c.run(n, dt)
    c.status()
    assert np.array_equal(a.download_state(), c.download_state())


def test_entropy_production_fp32bulk_against_oracle(orc):
    """The FP32-bulk form computes Pi per node in float from float gradients; the sum is
    FP64.  Bound: 1e-4 relative (the float rounding of products of lifted gradients)."""
    from paper_2208_05310_gb300 import dgk
    o = oracle_objects(orc, MS, PAPER_PARAMS)
    rv, rl = orc.maxwell(0.85)
    Uo = o.set_primitive(droplet_state(o.node_coords(), (rv, rl, orc.interface_width(0.85)), **KW))
    g = _ctx(MS, "fp32bulk")
    do, dg = o.diagnostics(Uo), g.diagnostics()
    assert abs(dg["entropy_production"] / do["entropy_production"] - 1.0) < 1e-4, (dg, do)

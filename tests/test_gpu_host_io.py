"""dgk_run_host: independent states through host memory with the copies of the
neighbouring items overlapped with the steps.  Each result must be bitwise the result of
the plain sequence upload / run / download of the same input."""
import numpy as np
import pytest

from cases import PAPER_PARAMS, dgk_context, mesh_spec
from paper_2208_05310_gb300 import inputs

pytestmark = pytest.mark.gpu

MS = mesh_spec(3, 3, [3, 2, 4], periodic=[1, 1, 0], walls={4: (0.85, 60.0), 5: (0.8, 120.0)})


def _inputs(g, n):
    out = []
    for seed in range(n):
        g.set_primitive(inputs.random_admissible(3, g.nelem, g.np, 100 + seed))
        out.append(g.download_state())
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32bulk"])
def test_run_host_equals_sequential(precision):
    import torch
    g = dgk_context(MS, PAPER_PARAMS, precision=precision)
    ins = _inputs(g, 7)  # every one of the three item buffers takes two or three items
    dt = 0.5 * g.max_dt()
    ref = []
    for u in ins:
        g.upload_state(u)
        g.run(3, dt)
        g.status()
        ref.append(g.download_state())
    # numpy in/out
    outs = [np.zeros_like(u) for u in ins]
    g.run_host(ins, outs, 3, dt)
    g.status()
    for o, r in zip(outs, ref):
        assert np.array_equal(o, r)
    assert np.array_equal(g.download_state(), ref[-1])
    # page-locked tensors, one input and one output buffer shared by all items
    pin_in = [torch.from_numpy(u).pin_memory() for u in ins]
    pin_out = torch.empty(g.shape(), dtype=torch.float64).pin_memory()
    g.run_host(pin_in, [pin_out] * len(ins), 3, dt)
    g.status()
    assert np.array_equal(pin_out.numpy(), ref[-1])
    same = torch.from_numpy(ins[1]).pin_memory()
    outs2 = [torch.empty(g.shape(), dtype=torch.float64).pin_memory() for _ in range(3)]
    g.run_host([same] * 3, outs2, 3, dt)
    for o in outs2:
        assert np.array_equal(o.numpy(), ref[1])


def test_run_host_edge_cases_and_refusals():
    from paper_2208_05310_gb300 import dgk
    g = dgk_context(MS, PAPER_PARAMS)
    u = _inputs(g, 1)[0]
    dt = 0.5 * g.max_dt()
    g.run_host([], [], 3, dt)  # nothing to do
    assert np.array_equal(g.download_state(), u)
    out = np.zeros_like(u)
    g.run_host([u], [out], 0, dt)  # zero steps: in -> out unchanged
    assert np.array_equal(out, u)
    with pytest.raises(dgk.DgkError):
        g.run_host([u], [np.zeros(u.size - 1)], 1, dt)
    with pytest.raises(dgk.DgkError):
        g.run_host([u], [out], -1, dt)
    with pytest.raises(dgk.DgkError):
        g.run_host([u], [out], 1, 0.0)
    with pytest.raises(dgk.DgkError):
        g.run_host([u], [out, out], 1, dt)


def test_run_host_with_kernel_timing_and_after_a_parameter_change():
    """With per-kernel timing on, dgk_run_host launches the stage kernels one by one
    instead of replaying its step graphs; after new parameters it captures new graphs.
    Both give the sequential results bit for bit."""
    from paper_2208_05310_gb300 import dgk
    g = dgk_context(MS, PAPER_PARAMS, precision="fp32bulk")
    ins = _inputs(g, 4)
    dt = 0.5 * g.max_dt()

    def sequential():
        ref = []
        for u in ins:
            g.upload_state(u)
            g.run(2, dt)
            g.status()
            ref.append(g.download_state())
        return ref

    ref = sequential()
    g.set_timing(True)
    outs = [np.zeros_like(u) for u in ins]
    g.run_host(ins, outs, 2, dt)
    g.status()
    assert all(np.array_equal(o, r) for o, r in zip(outs, ref))
    assert g.kernel_time(1)[1] > 0  # the k_lift2vol launches were timed
    g.set_timing(False)
    g.run_host(ins, outs, 2, dt)  # graphs of the three buffers
    assert all(np.array_equal(o, r) for o, r in zip(outs, ref))
    g.set_params(rk=4, precision="fp32bulk", **dict(PAPER_PARAMS, beta=50.0))  # drops the graphs
    ref2 = sequential()
    g.run_host(ins, outs, 2, dt)
    g.status()
    assert all(np.array_equal(o, r) for o, r in zip(outs, ref2))
    assert not all(np.array_equal(a, b) for a, b in zip(ref, ref2))

"""dgk_rhs_static: the right-hand side for callers that cannot call cudaMalloc.

Callers whose device memory is entirely held by another allocator's pool, or that
must never let an allocation synchronise the device, cannot create a libdgk context
(it allocates its buffers).  dgk_rhs_static takes their own state and output buffers
and keeps every intermediate in a fixed-size array compiled into the library.  This
test calls it through the C ABI and checks:
  - its output equals dgk_rhs (the context entry point) bit for bit on the same state:
    the same kernels run on the same inputs; two calls in a row with different states,
    both precision forms;
  - repeated calls allocate nothing: the device's free memory and torch's allocated
    bytes are unchanged across the second and later calls;
  - the status word it returns flags a non-finite input state, and is clear again on
    the next call with a valid state (each call clears it);
  - a short output tensor and an oversized mesh are refused.
The file name makes pytest collect it last."""
import pytest

from cases import PAPER_PARAMS, dgk_context, mesh_spec

pytestmark = pytest.mark.gpu

CASES = [
    (mesh_spec(3, 3, [3, 2, 4], periodic=[1, 1, 0], walls={4: (0.85, 60.0), 5: (0.8, 120.0)}), dict(PAPER_PARAMS)),
    (mesh_spec(2, 4, [5, 3]), dict(PAPER_PARAMS, model=2)),
    # a Navier-slip wall and a sliding no-slip wall
    (mesh_spec(3, 3, [3, 2, 4], periodic=[1, 1, 0],
               walls={4: (0.85, 60.0, 0.03, 0.05, 0.2, 0.3), 5: (0.8, 120.0, (0.2, -0.1, 0.0))}), dict(PAPER_PARAMS)),
]


def _reference(ms, ps, precision, seed):
    """State on the device and dgk_rhs of it, through a context."""
    import torch

    from paper_2208_05310_gb300 import inputs
    g = dgk_context(ms, ps, precision=precision)
    prim = inputs.random_admissible(ms["dim"], g.nelem, g.np, seed)
    g.set_primitive(prim)
    U = torch.empty(g.shape(), dtype=torch.float64, device="cuda")
    ref = torch.empty_like(U)
    g.download_state(U)
    g.rhs(ref)
    torch.cuda.synchronize()
    return g, U, ref


def _static_args(ms, ps, precision):
    from paper_2208_05310_gb300 import dgk
    dim = ms["dim"]
    mesh = dgk.make_box_mesh(dim, ms["N"], ms["n"] + [1] * (3 - dim), ms["lo"] + [0.0] * (3 - dim),
                             ms["hi"] + [1.0] * (3 - dim), ms["periodic"] + [1] * (3 - dim), ms["walls"])
    return dgk.make_params(precision=precision, **ps), mesh


@pytest.mark.parametrize("precision", ["fp64", "fp32bulk"])
@pytest.mark.parametrize("case", [0, 1, 2])
def test_static_rhs_matches_context_rhs(case, precision):
    import torch

    from paper_2208_05310_gb300 import dgk
    ms, ps = CASES[case]
    params, mesh = _static_args(ms, ps, precision)
    for seed in (21, 22):  # two calls in a row, different states
        ctx, U, ref = _reference(ms, ps, precision, seed)
        out = torch.full_like(U, float("nan"))
        st = dgk.rhs_static(params, mesh, U, out, status=True)
        torch.cuda.synchronize()
        assert st == 0
        assert torch.equal(out, ref), (seed, (out - ref).abs().max().item())
        ctx.close()


def test_static_rhs_allocates_nothing():
    """Free device memory and torch's allocated bytes stay the same over repeated calls
    (the first call may load the library's device code and look up the scratch address)."""
    import torch

    from paper_2208_05310_gb300 import dgk
    ms, ps = CASES[0]
    params, mesh = _static_args(ms, ps, "fp64")
    ctx, U, ref = _reference(ms, ps, "fp64", 31)
    ctx.close()
    out = torch.empty_like(U)
    dgk.rhs_static(params, mesh, U, out)
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(3):
        dgk.rhs_static(params, mesh, U, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.equal(out, ref)


def test_static_rhs_reports_device_status():
    """A NaN in the input state is flagged in the returned status word (non-finite bit);
    the next call on a valid state finds the word cleared."""
    import torch

    from paper_2208_05310_gb300 import dgk
    ms, ps = CASES[1]
    params, mesh = _static_args(ms, ps, "fp64")
    ctx, U, ref = _reference(ms, ps, "fp64", 41)
    ctx.close()
    bad = U.clone()
    bad[0, 3, 5] = float("nan")
    out = torch.empty_like(U)
    st = dgk.rhs_static(params, mesh, bad, out, status=True)
    assert st & dgk.STATUS_NONFINITE
    st = dgk.rhs_static(params, mesh, U, out, status=True)
    torch.cuda.synchronize()
    assert st == 0
    assert torch.equal(out, ref)


def test_static_rhs_refuses_short_tensor_and_oversized_mesh():
    import torch

    from paper_2208_05310_gb300 import dgk
    ms, ps = CASES[1]
    params, mesh = _static_args(ms, ps, "fp64")
    n = 5 * 15 * 25  # nvar * nelem * np of the 2D N = 4, 5x3-element mesh
    U = torch.zeros(n - 5, dtype=torch.float64, device="cuda")
    with pytest.raises(dgk.DgkError, match="nvar"):
        dgk.rhs_static(params, mesh, U, torch.zeros(n, dtype=torch.float64, device="cuda"))
    ms = mesh_spec(3, 5, [16, 16, 16])
    params, mesh = _static_args(ms, dict(PAPER_PARAMS), "fp64")
    U = torch.zeros(6 * 4096 * 216, dtype=torch.float64, device="cuda")
    with pytest.raises(dgk.DgkError, match="static scratch"):
        dgk.rhs_static(params, mesh, U, torch.zeros_like(U))

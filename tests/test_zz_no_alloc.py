"""dgk_rhs_static: the right-hand side for callers that cannot call cudaMalloc.

Callers whose device memory is entirely held by another allocator's pool, or that
must never let an allocation synchronise the device, cannot create a libdgk context
(it allocates its buffers).  dgk_rhs_static takes their own state and output buffers
and keeps every intermediate in a fixed-size array compiled into the library.  This
test calls it through the C ABI and checks its output against dgk_rhs (the context
entry point) on the same state, for two calls in a row with different states, in both
precision forms, and checks that an oversized mesh is refused.  The file name makes
pytest collect it last."""
import numpy as np
import pytest

from cases import PAPER_PARAMS, dgk_context, mesh_spec, rel_l2

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32bulk": 2e-4}  # the FP64 and FP32-bulk right-hand-side tolerances

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
        dgk.rhs_static(params, mesh, U, out)
        torch.cuda.synchronize()
        err = rel_l2(out.cpu().numpy(), ref.cpu().numpy())
        assert np.all(err < TOL[precision]), (seed, err)
        ctx.close()


def test_static_rhs_refuses_oversized_mesh():
    import torch

    from paper_2208_05310_gb300 import dgk
    ms = mesh_spec(3, 5, [16, 16, 16])
    params, mesh = _static_args(ms, dict(PAPER_PARAMS), "fp64")
    U = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(dgk.DgkError, match="static scratch"):
        dgk.rhs_static(params, mesh, U, torch.zeros_like(U))

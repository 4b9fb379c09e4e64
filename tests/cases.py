"""Shared test helpers: mesh / parameter specifications as plain data, node permutations
for the symmetry tests, and the workload recipes used by the parity tests.  None of the
method's arithmetic lives here: thermodynamic numbers (saturation densities, interface
width) are always obtained from the side under test."""
import numpy as np

from paper_2208_05310_gb300 import inputs

PAPER_PARAMS = dict(model=1, gammaK=1e-4, mu=0.01, kappa=1.0 / 150.0, cv=5.0, alpha=100.0, beta=100.0)


def mesh_spec(dim, N, n, lo=None, hi=None, periodic=None, walls=None, geometry=None):
    """geometry: None (straight box) or dict(ngeo=, amp=, rotation=) for curved elements
    (inputs.box_geometry)."""
    lo = lo or [0.0] * dim
    hi = hi or [1.0] * dim
    periodic = periodic if periodic is not None else [1] * dim
    return dict(dim=dim, N=N, n=list(n), lo=list(lo), hi=list(hi), periodic=list(periodic), walls=dict(walls or {}),
                geometry=geometry)


def geometry_array(mspec):
    """(ngeo, xgeo) of a curved mesh specification, or None."""
    g = mspec.get("geometry")
    if g is None:
        return None
    x = inputs.box_geometry(mspec["dim"], mspec["n"], mspec["lo"], mspec["hi"], g["ngeo"], amp=g.get("amp", 0.0),
                            rotation=g.get("rotation"))
    return g["ngeo"], x


def graded_levels(nx):
    """Refinement levels of the coarse columns in x of a graded mesh: two levels in the
    middle quarter, one in the bands beside it, none elsewhere (2:1 balanced, also across
    the periodic wrap); nx a multiple of 8."""
    def level(c):
        x = (8 * c[0]) // nx
        return 2 if x in (3, 4) else (1 if x in (2, 5) else 0)
    return level


def refined_arrays(mspec):
    """(ngeo, xgeo, conn, mortar) of a specification whose geometry asks for "refine": the
    upper half in x refined 2:1 with mortars (inputs.refined_mesh), or with "graded": two
    levels of 2:1 refinement in the middle of x (inputs.graded_mesh, graded_levels); with
    "reorient": seed, every element in a random local frame (inputs.reoriented_refined);
    else None."""
    g = mspec.get("geometry")
    if g is None or not (g.get("refine") or g.get("graded")):
        return None
    if g.get("graded"):
        xg, conn, mort = inputs.graded_mesh(mspec["dim"], mspec["N"], mspec["n"], mspec["periodic"], mspec["walls"],
                                            g["ngeo"], graded_levels(mspec["n"][0]), amp=g.get("amp", 0.0),
                                            lo=mspec["lo"], hi=mspec["hi"])
    else:
        xg, conn, mort = inputs.refined_mesh(mspec["dim"], mspec["N"], mspec["n"], mspec["periodic"],
                                             mspec["walls"], g["ngeo"], amp=g.get("amp", 0.0), lo=mspec["lo"],
                                             hi=mspec["hi"])
    if g.get("reorient") is not None:  # every element in a random local frame
        xg, conn, mort, _ = inputs.reoriented_refined(mspec["dim"], mspec["N"], g["ngeo"], xg, conn, mort,
                                                      g["reorient"])
    return g["ngeo"], xg, conn, mort


def unstructured_arrays(mspec):
    """(ngeo, xgeo, conn, node_index) of a specification whose geometry asks for
    "reorient": seed (the same mesh renumbered, elements in random local frames, with
    unstructured connectivity; inputs.reoriented_mesh), or None."""
    g = mspec.get("geometry")
    if g is None or g.get("reorient") is None:
        return None
    ngeo, x = geometry_array(mspec)
    xn, conn, ni = inputs.reoriented_mesh(mspec["dim"], mspec["N"], mspec["n"], mspec["periodic"], ngeo, x,
                                          g["reorient"])
    return ngeo, xn, conn, ni


def oracle_objects(orc, mspec, pspec):
    d = mspec["dim"]
    rf = refined_arrays(mspec)
    if rf is not None:
        m = orc.make_mesh(d, mspec["N"], [rf[1].shape[1], 1, 1], [0.0] * 3, [1.0] * 3, mspec["periodic"] + [1] * (3 - d),
                          mspec["walls"], geometry=(rf[0], rf[1]), conn=rf[2], mortar=rf[3])
        return orc.Oracle(m, orc.make_params(**pspec))
    un = unstructured_arrays(mspec)
    geo, conn = (geometry_array(mspec), None) if un is None else ((un[0], un[1]), un[2])
    m = orc.make_mesh(mspec["dim"], mspec["N"], mspec["n"] + [1] * (3 - mspec["dim"]),
                      mspec["lo"] + [0.0] * (3 - mspec["dim"]), mspec["hi"] + [1.0] * (3 - mspec["dim"]),
                      mspec["periodic"] + [1] * (3 - mspec["dim"]), mspec["walls"], geometry=geo, conn=conn)
    p = orc.make_params(**pspec)
    return orc.Oracle(m, p)


def quad_weights(w1d, dim, h):
    """Per-node quadrature weight times the element Jacobian prod(h/2)."""
    P = len(w1d)
    W = np.ones(P ** dim)
    idx = np.arange(P ** dim)
    for d in range(dim):
        W = W * w1d[(idx // P ** d) % P]
    return W * np.prod([0.5 * hh for hh in h])


# ---------------- node / element permutations ----------------

def _grid(arr, dim, n, P):
    """view [v][e][node] as [v][ez][ey][ex][k][j][i] (3D) or [v][ey][ex][j][i] (2D)"""
    v = arr.shape[0]
    if dim == 2:
        return arr.reshape(v, n[1], n[0], P, P)
    return arr.reshape(v, n[2], n[1], n[0], P, P, P)


def mirror(arr, dim, n, P, axis, flip_vars):
    """Reflect a nodal field across the mid-plane normal to `axis` (0 = x); the
    components listed in flip_vars change sign."""
    g = _grid(arr, dim, n, P).copy()
    e_ax = dim - axis  # element axis index in the grid view (after v)
    n_ax = 2 * dim - axis
    g = np.flip(g, axis=e_ax)
    g = np.flip(g, axis=n_ax)
    for v in flip_vars:
        g[v] = -g[v]
    return np.ascontiguousarray(g.reshape(arr.shape))


def transpose_xy(arr, n, P, var_perm):
    """2D: swap x and y (requires nx == ny).  var_perm maps new variable -> old variable."""
    g = _grid(arr, 2, n, P)
    g = np.transpose(g, (0, 2, 1, 4, 3))
    g = g[list(var_perm)]
    return np.ascontiguousarray(g.reshape(arr.shape))


def cycle_xyz(arr, n, P, var_perm):
    """3D: new (x, y, z) = old (y, z, x) (requires nx == ny == nz)."""
    g = _grid(arr, 3, n, P)
    # grid axes: v, ez, ey, ex, k, j, i ; new x = old y etc.
    # new[ez', ey', ex'] with ex' = old ey, ey' = old ez, ez' = old ex
    g = np.transpose(g, (0, 3, 1, 2, 6, 4, 5))
    g = g[list(var_perm)]
    return np.ascontiguousarray(g.reshape(arr.shape))


# ---------------- workloads ----------------

def droplet_state(x, thermo, T0=0.85, center=None, radius=0.25, perturb_seed=None, lengths=None,
                  noise_seed=None, noise_amp=0.0, liquid_inside=True, axes=None):
    """thermo = (rho_v, rho_l, L_i) from the side under test."""
    rv, rl, L = thermo
    dim = x.shape[0]
    center = center if center is not None else [0.5] * dim
    noise = inputs.uniform_noise(x[0].shape, noise_seed) if noise_seed is not None else None
    prim = inputs.droplet(x, center, radius, rv, rl, L, T0, liquid_inside=liquid_inside, noise=noise,
                          noise_amp=noise_amp, axes=axes)
    if perturb_seed is not None:
        prim = inputs.perturbed(prim, x, perturb_seed, lengths=lengths)
    return prim


def dgk_context(mspec, pspec, precision="fp64", rk=4):
    """Library context for the same specification (GPU only)."""
    from paper_2208_05310_gb300 import dgk
    ctx = dgk.Context()
    ctx.set_params(rk=rk, precision=precision, **pspec)
    dim = mspec["dim"]
    rf = refined_arrays(mspec)
    if rf is not None:
        ctx.mesh_unstructured(dim, mspec["N"], [rf[1].shape[1], 1, 1], mspec["periodic"] + [1] * (3 - dim),
                              mspec["walls"], rf[0], rf[1], rf[2], rf[3])
        return ctx
    un = unstructured_arrays(mspec)
    if un is not None:
        ctx.mesh_unstructured(dim, mspec["N"], mspec["n"] + [1] * (3 - dim), mspec["periodic"] + [1] * (3 - dim),
                              mspec["walls"], un[0], un[1], un[2])
        return ctx
    geo = geometry_array(mspec)
    if geo is not None:
        ctx.mesh_curved(dim, mspec["N"], mspec["n"] + [1] * (3 - dim), mspec["periodic"] + [1] * (3 - dim),
                        mspec["walls"], geo[0], geo[1])
        return ctx
    ctx.mesh_box(dim, mspec["N"], mspec["n"] + [1] * (3 - dim), mspec["lo"] + [0.0] * (3 - dim),
                 mspec["hi"] + [1.0] * (3 - dim), mspec["periodic"] + [1] * (3 - dim), mspec["walls"])
    return ctx


def rel_l2(a, b, floor_frac=1e-3):
    """Per-variable relative L2 distance ||a - b|| / max(||b||, floor_frac * max_v ||b_v||)."""
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.sqrt((b.reshape(b.shape[0], -1) ** 2).sum(axis=1))
    den = np.maximum(nb, floor_frac * nb.max())
    return np.sqrt(((a - b).reshape(b.shape[0], -1) ** 2).sum(axis=1)) / den

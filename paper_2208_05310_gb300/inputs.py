"""Seeded synthetic inputs: initial primitive fields for the droplet / interface workloads.

This module holds none of the method's arithmetic.  It evaluates the tanh phase
profiles of Sec. 4 of the paper at node coordinates supplied by the caller, with the
vapour/liquid densities, interface width and temperature passed in as plain numbers,
and draws seeded random numbers.  Both the CUDA library and the CPU oracle are fed
from here; each converts the primitive fields to its own conserved state.

Primitive layout: prim[v][e][n] with v = (rho, u_1..u_dim, T, c).
"""
from __future__ import annotations

import numpy as np


def uniform_noise(shape, seed):
    """Seeded uniform(-1, 1) numbers (numpy PCG64)."""
    return np.random.Generator(np.random.PCG64(seed)).uniform(-1.0, 1.0, size=shape)


def _assemble(rho, vel, T, c):
    dim = len(vel)
    prim = np.empty((dim + 3,) + rho.shape)
    prim[0] = rho
    for k in range(dim):
        prim[1 + k] = vel[k]
    prim[dim + 1] = T
    prim[dim + 2] = c
    return prim


def profile(dist, rho_in, rho_out, width, radius):
    """rho = (rho_in+rho_out)/2 + (rho_out-rho_in)/2 tanh(4 (dist - radius)/width):
    rho_in inside dist < radius, rho_out outside (the tanh profiles of Sec. 4)."""
    return 0.5 * (rho_in + rho_out) + 0.5 * (rho_out - rho_in) * np.tanh(4.0 * (dist - radius) / width)


def planar_slab(x, rho_v, rho_l, width, x1, x2, T0):
    """Liquid slab x1 < x < x2 in vapour: two planar interfaces normal to x, zero velocity."""
    xx = x[0]
    mid, half = 0.5 * (x1 + x2), 0.5 * (x2 - x1)
    rho = profile(np.abs(xx - mid), rho_l, rho_v, width, half)
    vel = [np.zeros_like(rho) for _ in range(x.shape[0])]
    return _assemble(rho, vel, np.full_like(rho, T0), rho.copy())


def droplet(x, center, radius, rho_v, rho_l, width, T0, liquid_inside=True, noise=None, noise_amp=0.0,
            axes=None):
    """Spherical (3D) / circular (2D) droplet or bubble; optional seeded density noise
    (noise: array of the node shape, uniform(-1,1)); c = rho after the noise.
    axes: the directions the distance is measured in (default: all), e.g. (0, 1) for a
    cylinder along z."""
    dim = x.shape[0]
    axes = tuple(range(dim)) if axes is None else tuple(axes)
    dist = np.sqrt(sum((x[k] - center[k]) ** 2 for k in axes))
    rin, rout = (rho_l, rho_v) if liquid_inside else (rho_v, rho_l)
    rho = profile(dist, rin, rout, width, radius)
    if noise is not None and noise_amp:
        rho = rho + noise_amp * noise
    vel = [np.zeros_like(rho) for _ in range(dim)]
    return _assemble(rho, vel, np.full_like(rho, T0), rho.copy())


def perturbed(prim, x, seed, u_amp=0.05, T_amp=0.01, c_amp=0.01, lengths=None):
    """Adds smooth velocity and temperature fields and a c != rho perturbation so that every
    term of the right-hand side is exercised (parity tests).  Smooth parts are periodic on
    the box given by lengths (default 1 per direction); c gets a small seeded per-node
    component."""
    dim = x.shape[0]
    lengths = lengths or [1.0] * dim
    rng = np.random.Generator(np.random.PCG64(seed))
    ph = rng.uniform(0, 2 * np.pi, size=(dim, dim))
    out = prim.copy()
    for k in range(dim):
        f = np.ones_like(x[0])
        for j in range(dim):
            f = f * np.sin(2 * np.pi * x[j] / lengths[j] + ph[k, j])
        out[1 + k] = out[1 + k] + u_amp * f
    g = np.ones_like(x[0])
    for j in range(dim):
        g = g * np.cos(2 * np.pi * x[j] / lengths[j] + ph[0, j])
    out[dim + 1] = out[dim + 1] + T_amp * g
    out[dim + 2] = out[dim + 2] * (1.0 + c_amp * rng.uniform(-1.0, 1.0, size=x[0].shape))
    return out


def ensemble_specs(nprob, seed, n_range=(16, 96), N_choices=(3, 4, 5), T_range=(0.75, 0.9),
                   theta_range=(30.0, 150.0), r_range=(0.15, 0.35)):
    """Seeded draws for a batched ensemble of independent 2D droplet / bubble problems."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for i in range(nprob):
        specs.append(dict(
            n=int(rng.integers(n_range[0], n_range[1] + 1)),
            N=int(rng.choice(N_choices)),
            T=float(rng.uniform(*T_range)),
            theta=float(rng.uniform(*theta_range)),
            radius=float(rng.uniform(*r_range)),
            droplet=bool(rng.integers(0, 2)),
            seed=int(rng.integers(0, 2**31 - 1)),
        ))
    return specs


def ensemble_mesh(spec):
    """Mesh of one ensemble problem: [0,1]^2 on n x n elements of degree N, periodic in x,
    isothermal no-slip walls at y = 0 and y = 1 at the problem's temperature and contact
    angle (mesh dictionary with keys dim, N, n, lo, hi, periodic, walls)."""
    w = (spec["T"], spec["theta"])
    return dict(dim=2, N=spec["N"], n=[spec["n"], spec["n"]], lo=[0.0, 0.0], hi=[1.0, 1.0], periodic=[1, 0],
                walls={2: w, 3: w})


def ensemble_primitive(x, spec, rho_v, rho_l, width, noise_amp=1e-3):
    """Initial state of one ensemble problem: a droplet (or a bubble) of the drawn radius
    centred on the bottom wall, tanh interface between the saturation densities, seeded
    density noise, at rest at the problem's temperature."""
    noise = uniform_noise(x[0].shape, spec["seed"])
    return droplet(x, [0.5, 0.0], spec["radius"], rho_v, rho_l, width, spec["T"], liquid_inside=spec["droplet"],
                   noise=noise, noise_amp=noise_amp)


def random_admissible(dim, nelem, np_, seed, rho_range=(0.3, 1.9), T_range=(0.8, 0.95), u_amp=0.05, c_amp=0.01):
    """Coordinate-free seeded state for exact-input tests: per-element density levels
    plus per-node variation, small velocities, temperatures in T_range and c = rho
    perturbed by c_amp.  Both implementations receive the identical array."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = rng.uniform(*rho_range, size=(nelem, 1))
    rho = np.clip(base + 0.1 * rng.uniform(-1, 1, size=(nelem, np_)), rho_range[0], rho_range[1])
    prim = np.empty((dim + 3, nelem, np_))
    prim[0] = rho
    for k in range(dim):
        prim[1 + k] = u_amp * rng.uniform(-1, 1, size=(nelem, np_))
    prim[dim + 1] = rng.uniform(*T_range, size=(nelem, np_))
    prim[dim + 2] = rho * (1.0 + c_amp * rng.uniform(-1, 1, size=(nelem, np_)))
    return prim


def box_geometry(dim, n, lo, hi, ngeo, amp=0.0, rotation=None):
    """Element maps of a box mesh for the curved-element interface: xgeo[k][e][g], the
    coordinate k of element e = ix + nx (iy + ny iz) at its equispaced points
    g = a + (ngeo+1)(b + (ngeo+1)c), t_a = -1 + 2a/ngeo.

    The straight box point x is moved to
        x_k + amp L_k sin(2 pi (x_j - lo_j) / L_j),   j = k+1 cyclic,
    a map that is periodic in every direction (the faces of a periodic direction stay
    translates of one another) and bends the faces of the others; then multiplied by the
    orthogonal matrix `rotation` if given.  Points shared by neighbouring elements are
    computed from one integer index, so they coincide bit for bit.  The element maps are
    the degree-ngeo interpolants of this map (amp = 0, no rotation: the box itself)."""
    G = ngeo + 1
    n = [int(v) for v in n[:dim]]
    L = [float(hi[k]) - float(lo[k]) for k in range(dim)]
    ne = int(np.prod(n))
    a = np.arange(G)
    # global point index per direction, per element and local point
    idx = [None] * dim
    for k in range(dim):
        idx[k] = (np.arange(n[k])[:, None] * ngeo + a[None, :])  # [n_k][G]
    # element coordinates
    e = np.arange(ne)
    ec = [e % n[0], (e // n[0]) % n[1]] + ([e // (n[0] * n[1])] if dim == 3 else [])
    g = np.arange(G ** dim)
    gc = [g % G, (g // G) % G] + ([g // (G * G)] if dim == 3 else [])
    x = np.empty((dim, ne, G ** dim))
    for k in range(dim):
        gi = idx[k][ec[k][:, None], gc[k][None, :]]
        x[k] = float(lo[k]) + L[k] * (gi / float(n[k] * ngeo))
    y = x.copy()
    if amp:
        for k in range(dim):
            j = (k + 1) % dim
            y[k] = x[k] + amp * L[k] * np.sin(2.0 * np.pi * (x[j] - float(lo[j])) / L[j])
    if rotation is not None:
        R = np.asarray(rotation, dtype=np.float64)
        y = np.einsum("kj,jeg->keg", R, y)
    return y


def box_connectivity(dim, n, periodic):
    """The box's element connectivity in the unstructured format: conn[e][f] =
    (neighbour, its face, orientation 0), or (-1 - f, 0, 0) on the wall of box face f."""
    n = [int(v) for v in n[:dim]]
    ne = int(np.prod(n))
    conn = np.zeros((ne, 2 * dim, 3), dtype=np.int32)
    stride = [1, n[0], n[0] * (n[1] if dim > 1 else 1)]
    for e in range(ne):
        co = [e % n[0], (e // n[0]) % n[1]] + ([e // (n[0] * n[1])] if dim == 3 else [])
        for d in range(dim):
            for s in range(2):
                f = 2 * d + s
                c = co[d] + (1 if s else -1)
                if c < 0 or c >= n[d]:
                    if not periodic[d]:
                        conn[e, f] = (-1 - f, 0, 0)
                        continue
                    c %= n[d]
                conn[e, f] = (e + (c - co[d]) * stride[d], 2 * d + 1 - s, 0)
    return conn


def _frames(dim, ne, rng):
    """Random orientation-preserving changes of the reference frame, one per element:
    new axis a is old axis perm[a] with sign sgn[a] (xi_perm[a] = sgn[a] eta_a)."""
    import itertools
    frames = []
    for p in itertools.permutations(range(dim)):
        inv = sum(1 for i in range(dim) for j in range(i + 1, dim) if p[i] > p[j])
        for sg in itertools.product((1, -1), repeat=dim):
            if (-1) ** inv * int(np.prod(sg)) == 1:
                frames.append((p, sg))
    pick = rng.integers(0, len(frames), ne)
    return [frames[i] for i in pick]


def _old_index(dim, K, frame, idx):
    """Old tensor indices (along old axes) of the new tensor index vector idx."""
    p, sg = frame
    old = [0] * dim
    for a in range(dim):
        old[p[a]] = idx[a] if sg[a] > 0 else K - 1 - idx[a]
    return old


def reoriented_mesh(dim, N, n, periodic, ngeo, xgeo, seed):
    """The same physical mesh as the box mesh (n, periodic) with element maps xgeo, with
    the elements renumbered at random and each given a random orientation-preserving
    local frame.  Returns (xgeo', conn', node_index): node_index[e'][n'] is the flat
    index e * NP + n of the same node in the box numbering, so that a nodal array A of
    the box mesh is A[..., node_index] on the new one (the physical components of vectors
    are unchanged)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = [int(v) for v in n[:dim]]
    ne = int(np.prod(n))
    P, G = N + 1, ngeo + 1
    NP, NG = P ** dim, G ** dim
    order = rng.permutation(ne)          # new element k is old element order[k]
    new_of = np.empty(ne, dtype=np.int64)
    new_of[order] = np.arange(ne)
    frames = _frames(dim, ne, rng)       # frame of new element k
    box = box_connectivity(dim, n, periodic)

    def flat(idx, K):
        return sum(idx[a] * K ** a for a in range(dim))

    def unflat(v, K):
        return [(v // K ** a) % K for a in range(dim)]

    xnew = np.empty((dim, ne, NG))
    node_index = np.empty((ne, NP), dtype=np.int64)
    for k in range(ne):
        e, fr = order[k], frames[k]
        for g in range(NG):
            xnew[:, k, g] = xgeo[:, e, flat(_old_index(dim, G, fr, unflat(g, G)), G)]
        for q in range(NP):
            node_index[k, q] = e * NP + flat(_old_index(dim, P, fr, unflat(q, P)), P)

    def new_face(fr, d_old, s_old):
        p, sg = fr
        a = p.index(d_old)
        return 2 * a + (s_old if sg[a] > 0 else 1 - s_old)

    def face_old_tangential(fr, f, t):
        """old tensor indices of the new face point with tangential indices t (new axes
        other than the face's, increasing)"""
        a_n = f // 2
        idx, j = [0] * dim, 0
        for a in range(dim):
            if a == a_n:
                idx[a] = (P - 1) * (f % 2)
            else:
                idx[a] = t[j]
                j += 1
        return _old_index(dim, P, fr, idx)

    conn = np.zeros((ne, 2 * dim, 3), dtype=np.int32)
    nt = P ** (dim - 1)
    for k in range(ne):
        e, fr = order[k], frames[k]
        for f in range(2 * dim):
            # the old face this new face is
            a = f // 2
            d_old, sg = fr[0][a], fr[1][a]
            s_old = (f % 2) if sg > 0 else 1 - (f % 2)
            nb_old, fo_old, _ = box[e, 2 * d_old + s_old]
            if nb_old < 0:
                conn[k, f] = (nb_old, 0, 0)
                continue
            k2 = new_of[nb_old]
            fr2 = frames[k2]
            f2 = new_face(fr2, fo_old // 2, fo_old % 2)
            # where each face point of (k, f) lands on (k2, f2): the structured faces
            # match by the old tangential indices
            want = []
            for tp in range(nt):
                t = [tp % P, tp // P][:dim - 1]
                old = face_old_tangential(fr, f, t)
                old_t = [old[b] for b in range(dim) if b != d_old]
                # find the tangential indices on (k2, f2) with the same old tangential indices
                hit = None
                for tq in range(nt):
                    t2 = [tq % P, tq // P][:dim - 1]
                    old2 = face_old_tangential(fr2, f2, t2)
                    if [old2[b] for b in range(dim) if b != d_old] == old_t:
                        hit = tq
                        break
                want.append(hit)
            o_found = None
            for o in range(8 if dim == 3 else 3):
                if dim == 2 and o & 5:
                    continue
                ok = True
                for tp in range(nt):
                    aa, bb = tp % P, tp // P
                    u, v = (bb, aa) if o & 1 else (aa, bb)
                    if o & 2:
                        u = P - 1 - u
                    if o & 4:
                        v = P - 1 - v
                    if u + P * v != want[tp]:
                        ok = False
                        break
                if ok:
                    o_found = o
                    break
            assert o_found is not None
            conn[k, f] = (k2, f2, o_found)
    return xnew, conn, node_index


def reoriented_frames(dim, N, n, periodic, ngeo, xgeo, seed):
    """reoriented_mesh without the renumbering, vectorised for large meshes: every element
    keeps its index and gets a random orientation-preserving local frame; the face-point
    orientations follow from the two frames (a tangential axis of one element is the same
    box axis as one of the neighbour's, with the product of the two frame signs deciding
    the reversal).  Returns (xgeo', conn')."""
    import itertools
    rng = np.random.Generator(np.random.PCG64(seed))
    n = [int(v) for v in n[:dim]]
    ne = int(np.prod(n))
    P, G = N + 1, ngeo + 1
    frames = []
    for p in itertools.permutations(range(dim)):
        inv = sum(1 for i in range(dim) for j in range(i + 1, dim) if p[i] > p[j])
        for sg in itertools.product((1, -1), repeat=dim):
            if (-1) ** inv * int(np.prod(sg)) == 1:
                frames.append((p, sg))
    fid = rng.integers(0, len(frames), ne)
    perm = np.array([frames[i][0] for i in fid])    # [ne][dim]: new axis a is box axis perm[a]
    sgn = np.array([frames[i][1] for i in fid])     # sign of that correspondence
    # element maps in the new frames
    NG = G ** dim
    gidx = np.arange(NG)
    newidx = np.stack([(gidx // G ** a) % G for a in range(dim)])  # [dim][NG]
    xnew = np.empty_like(xgeo)
    for t, (p, sg) in enumerate(frames):
        sel = np.nonzero(fid == t)[0]
        if sel.size == 0:
            continue
        old = np.zeros(NG, dtype=np.int64)
        for a in range(dim):
            ia = newidx[a] if sg[a] > 0 else G - 1 - newidx[a]
            old += ia * G ** p[a]
        xnew[:, sel, :] = xgeo[:, sel][:, :, old]
    box = box_connectivity(dim, n, periodic)
    conn = np.zeros((ne, 2 * dim, 3), dtype=np.int32)
    e = np.arange(ne)
    for a in range(dim):
        for s in range(2):
            f = 2 * a + s
            d_old = perm[:, a]
            s_old = np.where(sgn[:, a] > 0, s, 1 - s)
            bx = box[e, 2 * d_old + s_old]                  # [ne][3] in the box frames
            wall = bx[:, 0] < 0
            nb = np.where(wall, 0, bx[:, 0])
            # the neighbour's new face: its new axis a2 with perm[nb][a2] == d_old
            a2 = np.argmax(perm[nb] == d_old[:, None], axis=1)
            so_old = bx[:, 1] % 2
            s2 = np.where(sgn[nb, a2] > 0, so_old, 1 - so_old)
            f2 = 2 * a2 + s2
            # tangential axes, increasing new-axis order
            tang = [b for b in range(dim) if b != a]
            o = np.zeros(ne, dtype=np.int32)
            if dim == 2:
                t0 = tang[0]
                t0n = np.where(a2 == 0, 1, 0)
                flip = sgn[e, t0] * sgn[nb, t0n] < 0
                o = np.where(flip, 2, 0)
            else:
                tn = np.array([[b for b in range(3) if b != x] for x in range(3)])[a2]  # [ne][2]
                t0, t1 = tang
                swap = perm[nb, tn[:, 0]] == perm[e, t1]
                # u' runs along the neighbour's first tangential axis: from u (no swap) or v
                src_u = np.where(swap, t1, t0)
                src_v = np.where(swap, t0, t1)
                flip_u = sgn[e, src_u] * sgn[nb, tn[:, 0]] < 0
                flip_v = sgn[e, src_v] * sgn[nb, tn[:, 1]] < 0
                o = swap.astype(np.int32) | (flip_u.astype(np.int32) << 1) | (flip_v.astype(np.int32) << 2)
            conn[:, f, 0] = np.where(wall, bx[:, 0], nb)
            conn[:, f, 1] = np.where(wall, 0, f2)
            conn[:, f, 2] = np.where(wall, 0, o)
    return xnew, conn


def _lagrange_equispaced_1d(g, x):
    """Lagrange basis of the equispaced points t_a = -1 + 2a/g at the points x: [len(x)][g+1]."""
    t = -1.0 + 2.0 * np.arange(g + 1) / g
    L = np.ones((len(x), g + 1))
    for a in range(g + 1):
        for k in range(g + 1):
            if k != a:
                L[:, a] *= (x - t[k]) / (t[a] - t[k])
    return L


def refined_mesh(dim, N, n, periodic, walls, ngeo, amp=0.0, lo=None, hi=None):
    """A 2:1 non-conforming mesh: the box mesh n (n[0] even) of [lo, hi] with the coarse
    elements of the upper half in x split into 2^dim elements each.  Element maps: the
    coarse elements sample the periodic map of box_geometry (degree ngeo); a fine element's
    map is its parent's polynomial restricted to the fine element (so the hanging faces
    are watertight).  Connectivity in the unstructured format with mortars (see the
    oracle's header): conn [ne][2 dim][3], mortar [nm][2^(dim-1)][3]; every element keeps
    the box frame.  walls: the faces (2 d + side) of the non-periodic directions.
    Returns (xgeo, conn, mortar)."""
    n = [int(v) for v in n[:dim]]
    assert n[0] % 2 == 0
    lo = lo or [0.0] * dim
    hi = hi or [1.0] * dim
    G = ngeo + 1
    NG = G ** dim
    xc = box_geometry(dim, n, lo, hi, ngeo, amp=amp)  # [dim][n_coarse][NG]
    half = n[0] // 2
    m = [2 * v for v in n]                             # fine lattice
    cstride = [1, n[0], n[0] * (n[1] if dim > 1 else 1)]
    # elements: coarse cells with ix < half, then fine cells with fx >= 2 half
    coarse_cells = [c for c in np.ndindex(*reversed(n))]
    coarse_cells = [tuple(reversed(c)) for c in coarse_cells if c[-1] < half]
    fine_cells = [tuple(reversed(c)) for c in np.ndindex(*reversed(m)) if c[-1] >= 2 * half]
    elem = {}
    for k, c in enumerate(coarse_cells):
        elem[("c",) + c] = k
    nc = len(coarse_cells)
    for k, c in enumerate(fine_cells):
        elem[("f",) + c] = nc + k
    ne = nc + len(fine_cells)

    def owner(fc):
        """element and level owning fine cell fc"""
        cc = tuple(v // 2 for v in fc)
        if cc[0] < half:
            return elem[("c",) + cc], 0, cc
        return elem[("f",) + tuple(fc)], 1, None

    # geometry
    xg = np.empty((dim, ne, NG))
    gidx = np.arange(NG)
    for k, c in enumerate(coarse_cells):
        ce = sum(c[d] * cstride[d] for d in range(dim))
        xg[:, k, :] = xc[:, ce, :]
    t = -1.0 + 2.0 * np.arange(G) / ngeo
    for s_off in np.ndindex(*([2] * dim)):
        Ls = [_lagrange_equispaced_1d(ngeo, 0.5 * (t + 2 * s_off[d] - 1)) for d in range(dim)]  # [G_new][G_old]
        W = np.ones((NG, NG))
        for d in range(dim):
            W *= Ls[d][(gidx // G ** d) % G][:, (gidx // G ** d) % G]
        for k, c in enumerate(fine_cells):
            if tuple(v % 2 for v in c) != s_off:
                continue
            parent = tuple(v // 2 for v in c)
            ce = sum(parent[d] * cstride[d] for d in range(dim))
            xg[:, nc + k, :] = xc[:, ce, :] @ W.T
    # connectivity
    conn = np.zeros((ne, 2 * dim, 3), dtype=np.int32)
    mortar = []
    for key, e in elem.items():
        level, cell = key[0], key[1:]
        for d in range(dim):
            tang = [b for b in range(dim) if b != d]
            for s in range(2):
                f = 2 * d + s
                if level == "c":
                    base = [2 * v for v in cell]
                    nd = base[d] + 2 if s else base[d] - 1
                else:
                    base = list(cell)
                    nd = base[d] + 1 if s else base[d] - 1
                if nd < 0 or nd >= m[d]:
                    if not periodic[d]:
                        conn[e, f] = (-1 - f, 0, 0)
                        continue
                    nd %= m[d]
                if level == "c":
                    cells = []
                    for offs in np.ndindex(*([2] * (dim - 1))):
                        fc = list(base)
                        fc[d] = nd
                        for j, b in enumerate(tang):
                            fc[b] = base[b] + offs[j]
                        cells.append((offs, owner(fc)))
                    if all(o[1] == 0 for _, o in cells):
                        conn[e, f] = (cells[0][1][0], 2 * d + 1 - s, 0)
                    else:
                        mid = len(mortar)
                        sub = [None] * (2 ** (dim - 1))
                        for offs, o in cells:
                            p = sum(offs[j] << j for j in range(dim - 1))
                            sub[p] = (o[0], 2 * d + 1 - s, 0)
                        mortar.append(sub)
                        conn[e, f] = (-100 - mid, 0, 0)
                else:
                    fc = list(base)
                    fc[d] = nd
                    nb, lev, cc = owner(fc)
                    if lev == 1:
                        conn[e, f] = (nb, 2 * d + 1 - s, 0)
                    else:
                        p = sum(((fc[b] - 2 * cc[b]) % 2) << j for j, b in enumerate(tang))
                        conn[e, f] = (nb, 2 * d + 1 - s, (p + 1) << 3)
    mort = np.array(mortar, dtype=np.int32).reshape(len(mortar), 2 ** (dim - 1), 3)
    return xg, conn, mort


def _orient_code(dim, P, src, dst):
    """The face-point orientation code o (the format of the connectivity tables: (u, v) =
    o & 1 ? (b, a) : (a, b); a' = o & 2 ? N - u : u; b' = o & 4 ? N - v : v) that maps
    every point src[i] = (a, b) to dst[i] = (a', b'); 2D points have b = 0."""
    N = P - 1
    for o in (range(8) if dim == 3 else (0, 2)):
        ok = True
        for (a, b), (a2, b2) in zip(src, dst):
            u, v = (b, a) if o & 1 else (a, b)
            u = N - u if o & 2 else u
            v = N - v if o & 4 else v
            if (u, v) != (a2, b2):
                ok = False
                break
        if ok:
            return o
    raise ValueError("no orientation code maps the face points")


def reoriented_refined(dim, N, ngeo, xgeo, conn, mortar, seed):
    """A mesh in the unstructured format whose elements all use the box frame (face-point
    orientations 0, e.g. refined_mesh's) with every element given a random
    orientation-preserving local frame, numbering kept: element maps, conforming faces,
    walls and mortars (sub-face order and face-point orientations in the new frames).
    Returns (xgeo', conn', mortar', node_index) with node_index[e][n'] = e * NP + n of the
    same node in the original frames."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ne = xgeo.shape[1]
    P, G = N + 1, ngeo + 1
    NP, NG, NFP = P ** dim, G ** dim, P ** (dim - 1)
    frames = _frames(dim, ne, rng)

    def flat(idx, K):
        return sum(idx[a] * K ** a for a in range(dim))

    def unflat(v, K):
        return [(v // K ** a) % K for a in range(dim)]

    xnew = np.empty_like(xgeo)
    node_index = np.empty((ne, NP), dtype=np.int64)
    for e in range(ne):
        fr = frames[e]
        for g in range(NG):
            xnew[:, e, g] = xgeo[:, e, flat(_old_index(dim, G, fr, unflat(g, G)), G)]
        for q in range(NP):
            node_index[e, q] = e * NP + flat(_old_index(dim, P, fr, unflat(q, P)), P)

    def new_face(e, f_old):
        p, sg = frames[e]
        a = p.index(f_old // 2)
        return 2 * a + ((f_old % 2) if sg[a] > 0 else 1 - (f_old % 2))

    def old_face_point(e, f_new, t):
        """old face index and old tangential indices (increasing old axes) of the point
        with new tangential indices t on new face f_new of element e"""
        a_n = f_new // 2
        idx, j = [0] * dim, 0
        for a in range(dim):
            if a == a_n:
                idx[a] = (P - 1) * (f_new % 2)
            else:
                idx[a] = t[j]
                j += 1
        old = _old_index(dim, P, frames[e], idx)
        d_old = frames[e][0][a_n]
        s_old = (f_new % 2) if frames[e][1][a_n] > 0 else 1 - (f_new % 2)
        return 2 * d_old + s_old, [old[b] for b in range(dim) if b != d_old]

    pts = [(a, b) for b in range(P if dim == 3 else 1) for a in range(P)]

    def new_point_of_old(e, f_old, t_old):
        """new tangential indices on e's new face of the point with old tangential t_old"""
        f_new = new_face(e, f_old)
        for t in pts:
            if old_face_point(e, f_new, list(t)[:dim - 1])[1] == list(t_old):
                return t
        raise AssertionError("face point not found")

    conn_new = np.zeros_like(conn)
    mort_new = np.array(mortar, copy=True) if mortar is not None and len(mortar) else None
    nsub = 2 ** (dim - 1)
    for e in range(ne):
        for f_old in range(2 * dim):
            nb, fo, oo = (int(v) for v in conn[e, f_old])
            f_new = new_face(e, f_old)
            if nb < 0 and nb > -100:  # wall
                conn_new[e, f_new] = (nb, 0, 0)
                continue
            if nb <= -100:  # the big side of a mortar: its sub-faces in the new frame
                m = -100 - nb
                conn_new[e, f_new] = (nb, 0, 0)
                for p_old in range(nsub):
                    s, fs, os_ = (int(v) for v in mortar[m][p_old])
                    assert os_ == 0
                    # the sub-face's new index: halves along the big face's new tangential axes
                    h_old = [(p_old >> j) & 1 for j in range(dim - 1)]
                    # a point of the sub-face in the big face's old tangential indices on the
                    # doubled lattice (half h, local index i -> 2 P h + i), mapped to the new frame
                    src, dst = [], []
                    p_new = None
                    for t in pts:
                        t_s = list(t)[:dim - 1]
                        # small face point (new frame) -> old tangential indices (box frame,
                        # the same order as the big face's old tangential axes)
                        _, t_old = old_face_point(s, new_face(s, fs), t_s)
                        big = [P * h_old[j] + t_old[j] for j in range(dim - 1)]
                        # the same lattice point in the big face's new frame (lattice of 2P)
                        bn = _big_new(dim, P, frames[e], f_old, big)
                        hn = [bn[j] // P for j in range(dim - 1)]
                        ln = [bn[j] % P for j in range(dim - 1)]
                        pn = sum(hn[j] << j for j in range(dim - 1))
                        assert p_new is None or p_new == pn
                        p_new = pn
                        src.append(tuple(t_s) + ((0,) if dim == 2 else ()))
                        dst.append(tuple(ln) + ((0,) if dim == 2 else ()))
                    o = _orient_code(dim, P, src, dst)
                    fs_new = new_face(s, fs)
                    mort_new[m][p_new] = (s, fs_new, o)
                    conn_new[s, fs_new] = (e, f_new, o | ((p_new + 1) << 3))
                continue
            if oo >> 3:  # the small side: written with its mortar above
                continue
            # conforming face: the neighbour's point for each of e's points
            fo_new = new_face(nb, fo)
            src, dst = [], []
            for t in pts:
                t_e = list(t)[:dim - 1]
                _, t_old = old_face_point(e, f_new, t_e)
                t_nb = new_point_of_old(nb, fo, t_old)
                src.append(tuple(t_e) + ((0,) if dim == 2 else ()))
                dst.append(tuple(list(t_nb)[:dim - 1]) + ((0,) if dim == 2 else ()))
            conn_new[e, f_new] = (nb, fo_new, _orient_code(dim, P, src, dst))
    return xnew, conn_new, mort_new, node_index


def _big_new(dim, P, frame, f_old, big_old):
    """Tangential indices, in the new frame, of a point on the doubled (2P) lattice of an
    element's face given in the old frame's tangential indices (increasing old axes)."""
    p, sg = frame
    d_old = f_old // 2
    t_old_axes = [b for b in range(dim) if b != d_old]
    a_n = p.index(d_old)
    t_new_axes = [a for a in range(dim) if a != a_n]
    out = []
    for a in t_new_axes:
        ob = p[a]
        v = big_old[t_old_axes.index(ob)]
        out.append(v if sg[a] > 0 else 2 * P - 1 - v)
    return out


def graded_mesh(dim, N, n, periodic, walls, ngeo, level_of, amp=0.0, lo=None, hi=None):
    """A 2:1-balanced non-conforming mesh with several refinement levels: the box mesh n of
    [lo, hi] whose coarse cell c (integer coordinates) is split into 2^(dim L) cells of
    level L = level_of(c) (neighbouring coarse cells may differ by one level at most).
    Element maps: each cell samples its coarse cell's periodic map (box_geometry, degree
    ngeo) restricted to the cell, so hanging faces are watertight.  Connectivity in the
    unstructured format with mortars, every element in the box frame; walls: the faces
    (2 d + side) of the non-periodic directions.  Returns (xgeo, conn, mortar)."""
    n = [int(v) for v in n[:dim]]
    lo = lo or [0.0] * dim
    hi = hi or [1.0] * dim
    G = ngeo + 1
    NG = G ** dim
    xc = box_geometry(dim, n, lo, hi, ngeo, amp=amp)
    cstride = [int(np.prod(n[:d])) for d in range(dim)]
    levels = {}
    for c in np.ndindex(*reversed(n)):
        c = tuple(reversed(c))
        levels[c] = int(level_of(c))
    # leaves: (level, integer coordinates on that level's lattice)
    leaves = []
    for c, L in levels.items():
        for sub in np.ndindex(*([2 ** L] * dim)):
            leaves.append((L, tuple(c[d] * 2 ** L + sub[d] for d in range(dim))))
    index = {leaf: k for k, leaf in enumerate(leaves)}
    ne = len(leaves)
    t = -1.0 + 2.0 * np.arange(G) / ngeo
    gidx = np.arange(NG)
    xg = np.empty((dim, ne, NG))
    for k, (L, q) in enumerate(leaves):
        c = tuple(v >> L for v in q)
        ce = sum(c[d] * cstride[d] for d in range(dim))
        W = np.ones((NG, NG))
        for d in range(dim):
            off = q[d] - (c[d] << L)
            Ld = _lagrange_equispaced_1d(ngeo, -1.0 + (2.0 * off + 1.0 + t) / 2 ** L)  # [G_new][G_old]
            W *= Ld[(gidx // G ** d) % G][:, (gidx // G ** d) % G]
        xg[:, k, :] = xc[:, ce, :] @ W.T

    def wrap(L, q, d):
        """q on level L moved into the domain along d (periodic), or None outside"""
        m = n[d] << L
        if 0 <= q[d] < m:
            return q
        if not periodic[d]:
            return None
        qq = list(q)
        qq[d] %= m
        return tuple(qq)

    conn = np.zeros((ne, 2 * dim, 3), dtype=np.int32)
    mortar = []
    for k, (L, q) in enumerate(leaves):
        for d in range(dim):
            tang = [b for b in range(dim) if b != d]
            for s in range(2):
                f = 2 * d + s
                qn = list(q)
                qn[d] += 1 if s else -1
                qn = wrap(L, tuple(qn), d)
                if qn is None:
                    conn[k, f] = (-1 - f, 0, 0)
                    continue
                if (L, qn) in index:  # same level
                    conn[k, f] = (index[(L, qn)], 2 * d + 1 - s, 0)
                elif L > 0 and (L - 1, tuple(v >> 1 for v in qn)) in index:  # coarser: small side
                    big = (L - 1, tuple(v >> 1 for v in qn))
                    p = sum(((q[b] & 1) << j) for j, b in enumerate(tang))
                    conn[k, f] = (index[big], 2 * d + 1 - s, (p + 1) << 3)
                else:  # finer: the big side of a mortar
                    sub = [None] * (2 ** (dim - 1))
                    for offs in np.ndindex(*([2] * (dim - 1))):
                        qf = [2 * v for v in qn]
                        qf[d] = 2 * qn[d] + (1 - s)
                        for j, b in enumerate(tang):
                            qf[b] += offs[j]
                        leaf = (L + 1, tuple(qf))
                        assert leaf in index, "the mesh is not 2:1 balanced"
                        sub[sum(offs[j] << j for j in range(dim - 1))] = (index[leaf], 2 * d + 1 - s, 0)
                    conn[k, f] = (-100 - len(mortar), 0, 0)
                    mortar.append(sub)
    mort = np.array(mortar, dtype=np.int32).reshape(len(mortar), 2 ** (dim - 1), 3)
    return xg, conn, mort

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

"""Manufactured solutions for the relaxed NSK system, written from the PDE of the paper
(Sec. 2.3, Eq. (navierstokeskorteweg_p) for model 1 and (..._palpha) for model 2) in
SymPy, independently of the oracle's C code.  The forcing Q = U_t + div F - S of a
chosen smooth periodic solution is turned into C with sympy.ccode and compiled into a
tiny shared library whose functions the oracle calls through a function pointer.
"""
import ctypes as C
import hashlib
import os
import subprocess
import tempfile

import sympy as sp

R, A, B = sp.Rational(8, 3), sp.Integer(3), sp.Rational(1, 3)


def _fields_2d(x, y, t):
    pi = sp.pi
    rho = 1.0 + 0.1 * sp.sin(2 * pi * x + t) * sp.cos(2 * pi * y)
    u = 0.1 * sp.sin(2 * pi * y - t) + 0.05
    v = 0.1 * sp.cos(2 * pi * x) * sp.sin(2 * pi * y + t)
    T = 1.2 + 0.05 * sp.cos(2 * pi * (x - y) + t)
    c = rho + 0.02 * sp.sin(2 * pi * x) * sp.sin(2 * pi * y - t)
    return rho, [u, v], T, c


def system_2d_nsk(prm):
    """The original NSK system (Eq. navierstokeskorteweg, Korteweg stress Eq.
    cauchystressnsk, energy flux Eq. energyfluxnsk): U = (rho, rho u, rho e) with
    rho e = rho eps + rho |u|^2/2 + gamma_K/2 |grad rho|^2, no source."""
    x, y, t = sp.symbols("x y t", real=True)
    X = [x, y]
    gK, mu, kap, cv = (sp.Float(prm[k]) for k in ("gammaK", "mu", "kappa", "cv"))
    rho, vel, T, _ = _fields_2d(x, y, t)
    grad = lambda f: [sp.diff(f, xi) for xi in X]  # noqa: E731
    gr = grad(rho)
    p = rho * R * T / (1 - B * rho) - A * rho ** 2
    gr2 = gr[0] ** 2 + gr[1] ** 2
    E = rho * (R * cv * T - A * rho) + sp.Rational(1, 2) * rho * (vel[0] ** 2 + vel[1] ** 2) + gK / 2 * gr2
    U = [rho, rho * vel[0], rho * vel[1], E]
    divu = sp.diff(vel[0], x) + sp.diff(vel[1], y)
    du = [[sp.diff(vel[k], X[i]) for k in range(2)] for i in range(2)]
    lap = sp.diff(rho, x, 2) + sp.diff(rho, y, 2)
    gT = grad(T)
    F = []
    for i in range(2):
        tau = [mu * (du[i][k] + du[k][i] - (sp.Rational(2, 3) * divu if k == i else 0))
               + gK * ((sp.Rational(1, 2) * gr2 + rho * lap if k == i else 0) - gr[k] * gr[i]) for k in range(2)]
        je = kap * gT[i] - gK * rho * gr[i] * divu
        Fc = [rho * vel[i]] + [rho * vel[k] * vel[i] + (p if k == i else 0) for k in range(2)] + [(E + p) * vel[i]]
        Fv = [0] + tau + [tau[0] * vel[0] + tau[1] * vel[1] + je]
        F.append([fc - fv for fc, fv in zip(Fc, Fv)])
    Q = [sp.diff(U[v], t) + sp.diff(F[0][v], x) + sp.diff(F[1][v], y) for v in range(4)]
    return (x, y, t), U + [rho], Q + [sp.Integer(0)]


def system_2d(prm):
    """Return (U, Q) expressions of the 2D manufactured solution for parameters prm."""
    if prm["model"] == 0:
        return system_2d_nsk(prm)
    x, y, t = sp.symbols("x y t", real=True)
    X = [x, y]
    gK, mu, kap, cv, al, be = (sp.Float(prm[k]) for k in ("gammaK", "mu", "kappa", "cv", "alpha", "beta"))
    model = prm["model"]
    rho, vel, T, c = _fields_2d(x, y, t)
    grad = lambda f: [sp.diff(f, xi) for xi in X]  # noqa: E731
    gc = grad(c)
    grho = grad(rho)
    p = rho * R * T / (1 - B * rho) - A * rho ** 2
    E = rho * (R * cv * T - A * rho) + sp.Rational(1, 2) * rho * (vel[0] ** 2 + vel[1] ** 2) \
        + al / 2 * (rho - c) ** 2 + gK / 2 * (gc[0] ** 2 + gc[1] ** 2)
    U = [rho, rho * vel[0], rho * vel[1], E, c]
    divu = sp.diff(vel[0], x) + sp.diff(vel[1], y)
    du = [[sp.diff(vel[k], X[i]) for k in range(2)] for i in range(2)]  # du[i][k] = d u_k / d x_i
    lapc = sp.diff(c, x, 2) + sp.diff(c, y, 2)
    phat = p + (al / 2 * rho ** 2 if model == 2 else 0)
    zeta = be * (gK * lapc + al * (rho - c))
    gT = grad(T)
    F = []  # F[i] = flux vector in direction i, F = F^C - F^V
    for i in range(2):
        tau = [mu * (du[i][k] + du[k][i] - (sp.Rational(2, 3) * divu if k == i else 0)) for k in range(2)]
        je = kap * gT[i] - gK * c * gc[i] * divu + gK * gc[i] * zeta
        Fc = [rho * vel[i]] + [rho * vel[k] * vel[i] + (phat if k == i else 0) for k in range(2)] \
            + [(E + phat) * vel[i], c * vel[i]]
        Fv = [0] + tau + [tau[0] * vel[0] + tau[1] * vel[1] + je, gK * be * gc[i]]
        F.append([fc - fv for fc, fv in zip(Fc, Fv)])
    korteweg = gK * (sp.Rational(1, 2) * (gc[0] ** 2 + gc[1] ** 2) * divu
                     - sum(gc[i] * gc[j] * du[i][j] for i in range(2) for j in range(2)))
    if model == 1:
        Sm = [al * rho * (gc[k] - grho[k]) for k in range(2)]
        SE = sum(Sm[k] * vel[k] for k in range(2)) + al / 2 * (c ** 2 - rho ** 2) * divu + korteweg
    else:
        Sm = [al * rho * gc[k] for k in range(2)]
        SE = sum(Sm[k] * vel[k] for k in range(2)) + al / 2 * c ** 2 * divu + korteweg
    S = [0, Sm[0], Sm[1], SE, al * be * (rho - c)]
    Q = [sp.diff(U[v], t) + sp.diff(F[0][v], x) + sp.diff(F[1][v], y) - S[v] for v in range(5)]
    return (x, y, t), U, Q


def _emit(name, syms, exprs):
    x, y, t = syms
    repl, red = sp.cse(exprs, optimizations="basic")
    lines = [f"void {name}(int dim, const double *X, double t, double *q, void *user) {{",
             "  const double x = X[0], y = X[1]; (void)dim; (void)user;"]
    for s, e in repl:
        lines.append(f"  const double {sp.ccode(s)} = {sp.ccode(e)};")
    for k, e in enumerate(red):
        lines.append(f"  q[{k}] = {sp.ccode(e)};")
    lines.append("}")
    return "\n".join(lines)


def build(prm):
    """Compile the exact solution and forcing for parameters prm; returns (lib, exact_fn, forcing_fn)."""
    key = hashlib.sha1(repr(sorted(prm.items())).encode()).hexdigest()[:12]
    d = os.path.join(tempfile.gettempdir(), f"dgk_mms_{os.getuid()}")
    os.makedirs(d, exist_ok=True)
    so = os.path.join(d, f"mms_{key}.so")
    if not os.path.exists(so):
        syms, U, Q = system_2d(prm)
        src = "#include <math.h>\n" + _emit("mms_exact", syms, U) + "\n" + _emit("mms_forcing", syms, Q) + "\n"
        cfile = os.path.join(d, f"mms_{key}_{os.getpid()}.c")
        with open(cfile, "w") as f:
            f.write(src)
        tmp = so + f".{os.getpid()}"
        subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-o", tmp, cfile, "-lm"], check=True)
        os.replace(tmp, so)
    lib = C.CDLL(so)
    return lib, C.cast(lib.mms_exact, C.c_void_p), C.cast(lib.mms_forcing, C.c_void_p)


def exact_state(lib, coords, t):
    """Evaluate the exact conserved state at node coordinates coords[d][e][n]."""
    import numpy as np
    f = lib.mms_exact
    f.argtypes = [C.c_int, C.POINTER(C.c_double), C.c_double, C.POINTER(C.c_double), C.c_void_p]
    ne, npn = coords.shape[1], coords.shape[2]
    U = np.zeros((5, ne, npn))
    X = (C.c_double * 3)()
    q = (C.c_double * 8)()
    for e in range(ne):
        for n in range(npn):
            X[0], X[1] = coords[0, e, n], coords[1, e, n]
            f(2, X, t, q, None)
            for v in range(5):
                U[v, e, n] = q[v]
    return U

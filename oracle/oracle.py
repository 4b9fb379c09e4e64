"""ctypes wrapper of the plain-C FP64 oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
import this module.  The product library never does.
"""
import ctypes as C
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)
import build as _build  # noqa: E402

_lib = None

OR_NDIAG = 9
DIAG_NAMES = ("mass", "mom_x", "mom_y", "mom_z", "energy", "neg_entropy", "rho_minus_c_l2", "max_u",
              "entropy_production")


class OrMesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("N", C.c_int), ("n", C.c_int * 3),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("periodic", C.c_int * 3),
                ("wall_kind", C.c_int * 6), ("wall_T", C.c_double * 6),
                ("wall_theta_deg", C.c_double * 6), ("wall_gamma", (C.c_double * 4) * 6),
                ("wall_u", (C.c_double * 3) * 6), ("ngeo", C.c_int), ("xgeo", C.POINTER(C.c_double)), ("conn", C.POINTER(C.c_int)),
                ("mortar", C.POINTER(C.c_int)), ("nmortar", C.c_int)]


class OrParams(C.Structure):
    _fields_ = [("model", C.c_int), ("gammaK", C.c_double), ("mu", C.c_double),
                ("kappa", C.c_double), ("cv", C.c_double), ("alpha", C.c_double),
                ("beta", C.c_double), ("flux", C.c_int)]


FORCING = C.CFUNCTYPE(None, C.c_int, C.POINTER(C.c_double), C.c_double, C.POINTER(C.c_double), C.c_void_p)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        for name in ("or_psi", "or_chem", "or_inner_energy", "or_entropy_vol", "or_cs2"):
            getattr(L, name).restype = C.c_double
            getattr(L, name).argtypes = [C.c_double, C.c_double, C.c_double]
        for name in ("or_pressure", "or_dpdrho_T"):
            getattr(L, name).restype = C.c_double
            getattr(L, name).argtypes = [C.c_double, C.c_double]
        L.or_spinodal.argtypes = [C.c_double, dp, dp]
        L.or_maxwell.argtypes = [C.c_double, dp, dp]
        L.or_sigma_vl.restype = C.c_double
        L.or_sigma_vl.argtypes = [C.c_double, C.c_double, C.c_double]
        L.or_interface_width.restype = C.c_double
        L.or_interface_width.argtypes = [C.c_double, C.c_double, C.c_double]
        L.or_rho_from_p.argtypes = [C.c_double, C.c_double, C.c_int, dp]
        L.or_wall_dpsi_dc.restype = C.c_double
        L.or_wall_dpsi_dc.argtypes = [C.c_double] * 5
        L.or_gauss_legendre.argtypes = [C.c_int, dp, dp]
        L.or_lagrange_at.argtypes = [C.c_int, dp, C.c_double, dp]
        L.or_lagrange_at.restype = None
        L.or_dmatrix.argtypes = [C.c_int, dp, dp]
        L.or_dmatrix.restype = None
        mp, pp = C.POINTER(OrMesh), C.POINTER(OrParams)
        L.or_sizes.argtypes = [mp, pp, C.POINTER(C.c_long), C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.or_node_coords.argtypes = [mp, dp]
        L.or_node_weights.argtypes = [mp, dp]
        L.or_set_primitive.argtypes = [mp, pp, dp, dp]
        L.or_temperature.argtypes = [mp, pp, dp, dp]
        L.or_rhs.argtypes = [mp, pp, dp, dp]
        L.or_rhs_forced.argtypes = [mp, pp, dp, dp, C.c_double, C.c_void_p, C.c_void_p]
        L.or_rk_coeffs.argtypes = [C.c_int, C.POINTER(C.c_int), dp, dp, dp]
        L.or_run.argtypes = [mp, pp, dp, C.c_int, C.c_double, C.c_int, C.c_double, C.c_void_p, C.c_void_p]
        L.or_max_dt.argtypes = [mp, pp, dp, C.c_double, C.c_double, dp]
        L.or_diagnostics.argtypes = [mp, pp, dp, dp]
        L.or_num_threads.restype = C.c_int
        L.or_set_num_threads.restype = None
        L.or_set_num_threads.argtypes = [C.c_int]
        L.or_conv_point.argtypes = [pp, C.c_int, C.c_int, dp, C.c_double, dp]
        L.or_hllc_point.argtypes = [pp, C.c_int, C.c_int, dp, C.c_double, dp, C.c_double, dp]
        L.or_rusanov_point.argtypes = [pp, C.c_int, C.c_int, dp, C.c_double, dp, C.c_double, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def make_mesh(dim, N, n, lo, hi, periodic, walls=None, geometry=None, conn=None, mortar=None):
    """walls: dict face -> (T_wall, theta_deg) for faces 0..5 (-x,+x,-y,+y,-z,+z): an
    isothermal no-slip wall; (T_wall, theta_deg, (u_1, u_2, u_3)): the same wall sliding
    with velocity u (tangential); or (T_wall, theta_deg, gamma_1, gamma_2, gamma_3,
    gamma_4): a generalized Navier-slip wall (Eq. bc_nsk_alpha).
    geometry: None (the straight box) or (ngeo, xgeo), xgeo[dim][nelem][(ngeo+1)^dim] the
    element maps at equispaced points (see dgk_oracle.h); the array is kept alive by the
    returned mesh.
    conn: None (the box's connectivity) or an int array [nelem][2 dim][3] (see
    dgk_oracle.h), with a geometry."""
    m = OrMesh()
    if conn is not None:
        cn = np.ascontiguousarray(conn, dtype=np.int32)
        m.conn = cn.ctypes.data_as(C.POINTER(C.c_int))
        m._conn_keep = cn
    if mortar is not None and len(mortar):
        mt = np.ascontiguousarray(mortar, dtype=np.int32)
        m.mortar = mt.ctypes.data_as(C.POINTER(C.c_int))
        m.nmortar = int(mt.shape[0])
        m._mortar_keep = mt
    if geometry is not None:
        ngeo, xgeo = geometry
        xgeo = np.ascontiguousarray(xgeo, dtype=np.float64)
        m.ngeo = int(ngeo)
        m.xgeo = _dp(xgeo)
        m._xgeo_keep = xgeo
    m.dim, m.N = dim, N
    for d in range(3):
        m.n[d] = int(n[d]) if d < dim else 1
        m.lo[d] = float(lo[d]) if d < dim else 0.0
        m.hi[d] = float(hi[d]) if d < dim else 1.0
        m.periodic[d] = int(periodic[d]) if d < dim else 1
    for f, spec in (walls or {}).items():
        moving = len(spec) == 3
        m.wall_kind[f] = 1 if len(spec) == 2 or moving else 2
        m.wall_T[f] = spec[0]
        m.wall_theta_deg[f] = spec[1]
        if moving:
            for k, uk in enumerate(spec[2]):
                m.wall_u[f][k] = uk
        else:
            for k, gk in enumerate(spec[2:6]):
                m.wall_gamma[f][k] = gk
    return m


FLUX = {"rusanov": 0, "hllc": 1}


def make_params(model=1, gammaK=1e-4, mu=0.01, kappa=1.0 / 150.0, cv=5.0, alpha=100.0, beta=100.0, flux="rusanov"):
    return OrParams(model, gammaK, mu, kappa, cv, alpha, beta, FLUX[flux])


def point_flux(kind, params, dim, direction, UL, TL, UR=None, TR=None):
    """kind: "conv" (F^C(UL) at TL), "hllc" or "rusanov" (numerical flux between UL, UR)."""
    import numpy as np
    nv = dim + 3 if params.model != 0 else dim + 2
    F = np.zeros(nv)
    ul = np.ascontiguousarray(UL, dtype=np.float64)
    dp = C.POINTER(C.c_double)
    if kind == "conv":
        rc = lib().or_conv_point(C.byref(params), dim, direction, ul.ctypes.data_as(dp), TL, F.ctypes.data_as(dp))
    else:
        ur = np.ascontiguousarray(UR, dtype=np.float64)
        fn = lib().or_hllc_point if kind == "hllc" else lib().or_rusanov_point
        rc = fn(C.byref(params), dim, direction, ul.ctypes.data_as(dp), TL, ur.ctypes.data_as(dp), TR,
                F.ctypes.data_as(dp))
    if rc:
        raise ValueError(f"or_{kind}_point failed ({rc})")
    return F


# ---------------- thermodynamics ----------------

def pressure(rho, T):
    return lib().or_pressure(rho, T)


def cs2(rho, T, cv):
    return lib().or_cs2(rho, T, cv)


def maxwell(T):
    a, b = C.c_double(), C.c_double()
    _check(lib().or_maxwell(T, C.byref(a), C.byref(b)), "maxwell")
    return a.value, b.value


def spinodal(T):
    a, b = C.c_double(), C.c_double()
    _check(lib().or_spinodal(T, C.byref(a), C.byref(b)), "spinodal")
    return a.value, b.value


def sigma_vl(T, cv=5.0, gammaK=1e-4):
    return lib().or_sigma_vl(T, cv, gammaK)


def interface_width(T, cv=5.0, gammaK=1e-4):
    return lib().or_interface_width(T, cv, gammaK)


def rho_from_p(T, p, liquid):
    r = C.c_double()
    _check(lib().or_rho_from_p(T, p, int(liquid), C.byref(r)), "rho_from_p")
    return r.value


def gauss_legendre(n):
    x, w = np.zeros(n), np.zeros(n)
    _check(lib().or_gauss_legendre(n, _dp(x), _dp(w)), "gauss_legendre")
    return x, w


def lagrange_at(N, xi, x):
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    out = np.zeros(N + 1)
    lib().or_lagrange_at(N, _dp(xi), float(x), _dp(out))
    return out


def dmatrix(N, xi):
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    D = np.zeros((N + 1) * (N + 1))
    lib().or_dmatrix(N, _dp(xi), _dp(D))
    return D.reshape(N + 1, N + 1)


def rk_coeffs(rk):
    ns = C.c_int()
    A, B, c = np.zeros(5), np.zeros(5), np.zeros(5)
    _check(lib().or_rk_coeffs(rk, C.byref(ns), _dp(A), _dp(B), _dp(c)), "rk_coeffs")
    n = ns.value
    return A[:n].copy(), B[:n].copy(), c[:n].copy()


# ---------------- discretisation ----------------

class Oracle:
    """One mesh + parameter set.  Arrays are numpy float64 in the SoA layout [v][e][n]."""

    def __init__(self, mesh, params):
        self.mesh, self.params = mesh, params
        ne, np_, nv = C.c_long(), C.c_int(), C.c_int()
        _check(lib().or_sizes(C.byref(mesh), C.byref(params), C.byref(ne), C.byref(np_), C.byref(nv)), "sizes")
        self.nelem, self.np, self.nv = ne.value, np_.value, nv.value
        self.dim = mesh.dim

    def shape(self):
        return (self.nv, self.nelem, self.np)

    def node_coords(self):
        x = np.zeros((self.dim, self.nelem, self.np))
        _check(lib().or_node_coords(C.byref(self.mesh), _dp(x)), "node_coords")
        return x

    def node_weights(self):
        W = np.zeros((self.nelem, self.np))
        _check(lib().or_node_weights(C.byref(self.mesh), _dp(W)), "node_weights")
        return W

    def set_primitive(self, prim):
        prim = np.ascontiguousarray(prim, dtype=np.float64)
        U = np.zeros(self.shape())
        _check(lib().or_set_primitive(C.byref(self.mesh), C.byref(self.params), _dp(prim), _dp(U)), "set_primitive")
        return U

    def temperature(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        T = np.zeros((self.nelem, self.np))
        _check(lib().or_temperature(C.byref(self.mesh), C.byref(self.params), _dp(U), _dp(T)), "temperature")
        return T

    def rhs(self, U, t=0.0, forcing=None, user=None):
        U = np.ascontiguousarray(U, dtype=np.float64)
        Ut = np.zeros(self.shape())
        if forcing is None:
            rc = lib().or_rhs(C.byref(self.mesh), C.byref(self.params), _dp(U), _dp(Ut))
        else:
            rc = lib().or_rhs_forced(C.byref(self.mesh), C.byref(self.params), _dp(U), _dp(Ut), t, forcing, user)
        _check(rc, "rhs")
        return Ut

    def run(self, U, nsteps, dt, rk=4, t0=0.0, forcing=None, user=None):
        U = np.array(U, dtype=np.float64, order="C", copy=True)
        _check(lib().or_run(C.byref(self.mesh), C.byref(self.params), _dp(U), int(nsteps), float(dt), int(rk),
                            float(t0), forcing, user), "run")
        return U

    def max_dt(self, U, cfl=0.9, dfl=0.4):
        U = np.ascontiguousarray(U, dtype=np.float64)
        dt = C.c_double()
        _check(lib().or_max_dt(C.byref(self.mesh), C.byref(self.params), _dp(U), cfl, dfl, C.byref(dt)), "max_dt")
        return dt.value

    def diagnostics(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        out = np.zeros(OR_NDIAG)
        _check(lib().or_diagnostics(C.byref(self.mesh), C.byref(self.params), _dp(U), _dp(out)), "diagnostics")
        return dict(zip(DIAG_NAMES, out))


def num_threads():
    return lib().or_num_threads()


def set_num_threads(n):
    lib().or_set_num_threads(int(n))

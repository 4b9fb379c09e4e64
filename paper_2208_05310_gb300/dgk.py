"""Python binding of libdgk (include/dgk.h): argument marshalling only.

Every step of the time step runs in the library's CUDA kernels.  There is no CPU
fallback: if libdgk.so is missing or no GPU is present, the calls raise.

Host arrays are numpy float64 arrays in the SoA layout [v][e][n]; device arrays are
torch CUDA float64 tensors of the same shape (on_device paths).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libdgk.so")

DGK_PREC = {"fp64": 0, "fp32bulk": 1}
DGK_FLUX = {"rusanov": 0, "hllc": 1}
NDIAG = 9
DIAG_NAMES = ("mass", "mom_x", "mom_y", "mom_z", "energy", "neg_entropy", "rho_minus_c_l2", "max_u",
              "entropy_production")

_lib = None


class DgkParams(C.Structure):
    _fields_ = [("model", C.c_int), ("rk", C.c_int), ("precision", C.c_int), ("gammaK", C.c_double),
                ("mu", C.c_double), ("kappa", C.c_double), ("cv", C.c_double), ("alpha", C.c_double),
                ("beta", C.c_double), ("flux", C.c_int)]


class DgkWall(C.Structure):
    _fields_ = [("kind", C.c_int), ("T_wall", C.c_double), ("theta_deg", C.c_double), ("gamma", C.c_double * 4),
                ("u_wall", C.c_double * 3)]


def _wall(spec):
    """(T_wall, theta_deg): isothermal no-slip wall; (T_wall, theta_deg, (u_1, u_2, u_3)):
    the same wall sliding with velocity u; (T_wall, theta_deg, gamma_1, gamma_2, gamma_3,
    gamma_4): generalized Navier-slip wall."""
    if len(spec) == 2:
        return DgkWall(1, spec[0], spec[1])
    if len(spec) == 3:
        u = list(spec[2]) + [0.0] * (3 - len(spec[2]))
        return DgkWall(1, spec[0], spec[1], (C.c_double * 4)(), (C.c_double * 3)(*u))
    return DgkWall(2, spec[0], spec[1], (C.c_double * 4)(*spec[2:6]))


class DgkBoxMesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("N", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("periodic", C.c_int * 3), ("wall", DgkWall * 6)]


class DgkError(RuntimeError):
    pass


EXPORTS = ("dgk_create", "dgk_destroy", "dgk_set_params", "dgk_mesh_box", "dgk_mesh_curved", "dgk_mesh_unstructured", "dgk_sizes", "dgk_node_coords",
           "dgk_set_primitive", "dgk_upload_state", "dgk_download_state", "dgk_rhs", "dgk_rk_step", "dgk_run",
           "dgk_run_host",
           "dgk_max_dt", "dgk_diagnostics", "dgk_status", "dgk_set_timing", "dgk_kernel_time", "dgk_maxwell",
           "dgk_sigma_vl", "dgk_interface_width", "dgk_status_string", "dgk_last_error", "dgk_check_conversions",
           "dgk_rhs_static", "dgk_node_temperature_pressure", "dgk_batch_create", "dgk_batch_destroy",
           "dgk_batch_problem", "dgk_batch_set_dt", "dgk_batch_run", "dgk_batch_autotune", "dgk_batch_status",
           "dgk_batch_set_config", "dgk_batch_set_barrier_limit", "dgk_fma_peak")


def lib():
    """Load libdgk.so (built by paper_2208_05310_gb300.build / __graft_entry__.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise DgkError(f"libdgk.so not found at {LIB_PATH}: run `python -m paper_2208_05310_gb300.build`")
    L = C.CDLL(LIB_PATH)
    vp, dp, i, d = C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_double
    sz = C.c_size_t
    sig = {
        "dgk_create": (i, [C.POINTER(vp), i, vp]),
        "dgk_destroy": (None, [vp]),
        "dgk_set_params": (i, [vp, C.POINTER(DgkParams)]),
        "dgk_mesh_box": (i, [vp, C.POINTER(DgkBoxMesh)]),
        "dgk_mesh_curved": (i, [vp, C.POINTER(DgkBoxMesh), i, dp]),
        "dgk_mesh_unstructured": (i, [vp, C.POINTER(DgkBoxMesh), i, dp, C.POINTER(C.c_int), C.POINTER(C.c_int), i]),
        "dgk_sizes": (i, [vp, C.POINTER(C.c_longlong), C.POINTER(i), C.POINTER(i)]),
        "dgk_node_coords": (i, [vp, vp, i]),
        "dgk_set_primitive": (i, [vp, vp, sz, i]),
        "dgk_upload_state": (i, [vp, vp, sz, i]),
        "dgk_download_state": (i, [vp, vp, sz, i]),
        "dgk_rhs": (i, [vp, vp, sz, i]),
        "dgk_rk_step": (i, [vp, d]),
        "dgk_run": (i, [vp, i, d, i, vp]),
        "dgk_run_host": (i, [vp, C.POINTER(vp), C.POINTER(vp), i, sz, i, d]),
        "dgk_max_dt": (i, [vp, d, d, dp]),
        "dgk_diagnostics": (i, [vp, dp]),
        "dgk_node_temperature_pressure": (i, [vp, vp, vp, sz, i]),
        "dgk_batch_create": (i, [C.POINTER(vp), i, vp, C.POINTER(DgkParams), i, C.POINTER(DgkBoxMesh)]),
        "dgk_batch_destroy": (None, [vp]),
        "dgk_batch_problem": (vp, [vp, i]),
        "dgk_batch_set_dt": (i, [vp, dp]),
        "dgk_batch_run": (i, [vp, i]),
        "dgk_batch_autotune": (i, [vp, C.POINTER(i)]),
        "dgk_batch_status": (i, [vp, C.POINTER(i)]),
        "dgk_batch_set_config": (i, [vp, C.POINTER(i)]),
        "dgk_batch_set_barrier_limit": (i, [vp, C.c_longlong]),
        "dgk_status": (i, [vp]),
        "dgk_set_timing": (i, [vp, i]),
        "dgk_kernel_time": (i, [vp, i, dp, C.POINTER(C.c_longlong)]),
        "dgk_maxwell": (i, [d, dp, dp]),
        "dgk_sigma_vl": (i, [d, d, d, dp]),
        "dgk_interface_width": (i, [d, d, d, dp]),
        "dgk_check_conversions": (i, [vp, sz, i, C.POINTER(C.c_ulonglong)]),
        "dgk_fma_peak": (i, [i, i, dp]),
        "dgk_rhs_static": (i, [C.POINTER(DgkParams), C.POINTER(DgkBoxMesh), vp, vp, sz, vp, C.POINTER(C.c_uint)]),
        "dgk_status_string": (C.c_char_p, [i]),
        "dgk_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc, what):
    if rc != 0:
        L = lib()
        raise DgkError(f"{what}: {L.dgk_status_string(rc).decode()} ({rc}): {L.dgk_last_error().decode()}")


def _ptr(a):
    """(pointer, count, on_device) of a numpy array or torch tensor of float64."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise DgkError("host arrays must be C-contiguous float64")
        return a.ctypes.data, a.size, 0
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise DgkError("tensors must be contiguous float64")
        return a.data_ptr(), a.numel(), 1 if a.is_cuda else 0
    raise DgkError(f"unsupported array type {type(a)}")


# ---------------- thermodynamics (host) ----------------

def maxwell(T):
    a, b = C.c_double(), C.c_double()
    _check(lib().dgk_maxwell(T, C.byref(a), C.byref(b)), "dgk_maxwell")
    return a.value, b.value


def sigma_vl(T, cv=5.0, gammaK=1e-4):
    s = C.c_double()
    _check(lib().dgk_sigma_vl(T, cv, gammaK, C.byref(s)), "dgk_sigma_vl")
    return s.value


def interface_width(T, cv=5.0, gammaK=1e-4):
    s = C.c_double()
    _check(lib().dgk_interface_width(T, cv, gammaK, C.byref(s)), "dgk_interface_width")
    return s.value


def check_conversions(x):
    """Number of doubles in x whose library conversions differ from the hardware's."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    bad = C.c_ulonglong()
    _check(lib().dgk_check_conversions(x.ctypes.data, x.size, 0, C.byref(bad)), "dgk_check_conversions")
    return bad.value


def fma_peak(device=0, precision="fp64"):
    """Measured FMA throughput of the device in flops/s (dgk_fma_peak)."""
    v = C.c_double()
    _check(lib().dgk_fma_peak(int(device), DGK_PREC[precision], C.byref(v)), "dgk_fma_peak")
    return v.value


def make_params(model=1, rk=4, precision="fp64", gammaK=1e-4, mu=0.01, kappa=1.0 / 150.0, cv=5.0, alpha=100.0,
                beta=100.0, flux="rusanov"):
    return DgkParams(model, rk, DGK_PREC[precision], gammaK, mu, kappa, cv, alpha, beta, DGK_FLUX[flux])


def make_box_mesh(dim, N, n, lo, hi, periodic, walls=None):
    """walls: {face: (T_wall, theta_deg)} (no-slip), {face: (T_wall, theta_deg, (u_1, u_2, u_3))}
    (no-slip, sliding with velocity u) or {face: (T_wall, theta_deg, g1, g2, g3, g4)} (Navier
    slip), faces 0..5 = -x,+x,-y,+y,-z,+z."""
    m = DgkBoxMesh()
    m.dim, m.N = dim, N
    for d in range(3):
        m.n[d] = int(n[d]) if d < dim else 1
        m.lo[d] = float(lo[d]) if d < dim else 0.0
        m.hi[d] = float(hi[d]) if d < dim else 1.0
        m.periodic[d] = int(periodic[d]) if d < dim else 1
    for f, spec in (walls or {}).items():
        m.wall[f] = _wall(spec)
    return m


def rhs_static(params, mesh, U, Ut, stream=None, status=False):
    """dgk_rhs_static: right-hand side of the device state U into the device array Ut
    without any device allocation (see include/dgk.h).  U, Ut: contiguous float64 CUDA
    tensors of nvar*nelem*np elements for the mesh passed in; stream: a
    torch.cuda.Stream or None (default stream).  Asynchronous, unless status is true:
    then the call waits for the kernels and returns the device status word (0, or
    DGK_STATUS_* bits)."""
    pu, nu, du = _ptr(U)
    po, no, do = _ptr(Ut)
    dim, P = mesh.dim, mesh.N + 1
    if dim not in (2, 3):
        raise DgkError("mesh.dim must be 2 or 3")
    count = (dim + 3) * int(np.prod([int(mesh.n[d]) for d in range(dim)], dtype=object)) * P ** dim
    if not (du and do) or nu != count or no != count:
        raise DgkError(f"U and Ut must be device tensors of nvar*nelem*np = {count} doubles for this mesh")
    h = C.c_void_p(stream.cuda_stream) if stream is not None else C.c_void_p()
    st = C.c_uint(0)
    _check(lib().dgk_rhs_static(C.byref(params), C.byref(mesh), pu, po, count, h, C.byref(st) if status else None),
           "dgk_rhs_static")
    return st.value if status else None


STATUS_NONFINITE = 1
STATUS_DOMAIN = 2


# ---------------- context ----------------

class Context:
    """One problem on one GPU.  stream: a torch.cuda.Stream to issue work on (default: a
    new non-default stream, so that runs can be captured in a CUDA graph)."""

    def __init__(self, device=0, stream=None):
        import torch
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        self._h = C.c_void_p()
        _check(lib().dgk_create(C.byref(self._h), device, C.c_void_p(self.stream.cuda_stream)), "dgk_create")
        self.dim = self.nelem = self.np = self.nv = None

    def close(self):
        if self._h:
            lib().dgk_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, model=1, rk=4, precision="fp64", gammaK=1e-4, mu=0.01, kappa=1.0 / 150.0, cv=5.0,
                   alpha=100.0, beta=100.0, flux="rusanov"):
        """flux: "rusanov" or "hllc" (model 2)."""
        p = make_params(model, rk, precision, gammaK, mu, kappa, cv, alpha, beta, flux)
        _check(lib().dgk_set_params(self._h, C.byref(p)), "dgk_set_params")

    def mesh_box(self, dim, N, n, lo, hi, periodic, walls=None):
        """walls: {face: (T_wall, theta_deg)} (no-slip), {face: (T_wall, theta_deg, (u_1, u_2, u_3))}
        (sliding no-slip) or {face: (T_wall, theta_deg, g1, g2, g3, g4)}
    (Navier slip), faces 0..5 = -x,+x,-y,+y,-z,+z."""
        m = make_box_mesh(dim, N, n, lo, hi, periodic, walls)
        _check(lib().dgk_mesh_box(self._h, C.byref(m)), "dgk_mesh_box")
        self._sizes(dim)

    def mesh_curved(self, dim, N, n, periodic, walls, ngeo, xgeo):
        """Curved elements with the box's connectivity (dgk_mesh_curved): xgeo is a float64
        array [dim][nelem][(ngeo+1)^dim] of the element maps at equispaced reference
        points; walls as for mesh_box (along the local normal; a wall velocity is projected
        on the local tangent plane)."""
        m = make_box_mesh(dim, N, n, [0.0] * 3, [1.0] * 3, periodic, walls)
        x = np.ascontiguousarray(xgeo, dtype=np.float64)
        _check(lib().dgk_mesh_curved(self._h, C.byref(m), int(ngeo), x.ctypes.data_as(C.POINTER(C.c_double))),
               "dgk_mesh_curved")
        self._sizes(dim)

    def mesh_unstructured(self, dim, N, n, periodic, walls, ngeo, xgeo, conn, mortar=None):
        """Curved elements with unstructured connectivity (dgk_mesh_unstructured): conn is
        an int array [nelem][2 dim][3], mortar an int array [nmortar][2^(dim-1)][3] or None;
        n gives the element count as a product and, with periodic, which entries of the
        wall table (walls) exist."""
        m = make_box_mesh(dim, N, n, [0.0] * 3, [1.0] * 3, periodic, walls)
        x = np.ascontiguousarray(xgeo, dtype=np.float64)
        cn = np.ascontiguousarray(conn, dtype=np.int32)
        mt = np.ascontiguousarray(mortar if mortar is not None else np.zeros((0, 1, 3)), dtype=np.int32)
        _check(lib().dgk_mesh_unstructured(self._h, C.byref(m), int(ngeo), x.ctypes.data_as(C.POINTER(C.c_double)),
                                           cn.ctypes.data_as(C.POINTER(C.c_int)),
                                           mt.ctypes.data_as(C.POINTER(C.c_int)), int(mt.shape[0])),
                   "dgk_mesh_unstructured")
        self._sizes(dim)

    def _sizes(self, dim):
        ne, npn, nv = C.c_longlong(), C.c_int(), C.c_int()
        _check(lib().dgk_sizes(self._h, C.byref(ne), C.byref(npn), C.byref(nv)), "dgk_sizes")
        self.dim, self.nelem, self.np, self.nv = dim, ne.value, npn.value, nv.value

    def shape(self):
        return (self.nv, self.nelem, self.np)

    def node_coords(self):
        x = np.zeros((self.dim, self.nelem, self.np))
        _check(lib().dgk_node_coords(self._h, x.ctypes.data, 0), "dgk_node_coords")
        return x

    def set_primitive(self, prim):
        ptr, n, dev = _ptr(prim)
        _check(lib().dgk_set_primitive(self._h, ptr, n, dev), "dgk_set_primitive")

    def upload_state(self, U):
        ptr, n, dev = _ptr(U)
        _check(lib().dgk_upload_state(self._h, ptr, n, dev), "dgk_upload_state")

    def download_state(self, out=None):
        out = np.zeros(self.shape()) if out is None else out
        ptr, n, dev = _ptr(out)
        _check(lib().dgk_download_state(self._h, ptr, n, dev), "dgk_download_state")
        return out

    def rhs(self, out=None):
        out = np.zeros(self.shape()) if out is None else out
        ptr, n, dev = _ptr(out)
        _check(lib().dgk_rhs(self._h, ptr, n, dev), "dgk_rhs")
        return out

    def rk_step(self, dt):
        _check(lib().dgk_rk_step(self._h, float(dt)), "dgk_rk_step")

    def run(self, nsteps, dt, diag_every=0, diag_out=None):
        """nsteps steps of dt (dgk_run).  With diag_every > 0: returns the diagnostics taken
        on the device after every diag_every-th step, a (nsteps // diag_every, NDIAG)
        array -- into diag_out if given (a float64 numpy array or CUDA tensor of that
        size), else into a new numpy array."""
        if not diag_every:
            _check(lib().dgk_run(self._h, int(nsteps), float(dt), 0, None), "dgk_run")
            return None
        nsamp = int(nsteps) // int(diag_every)
        out = np.zeros((nsamp, NDIAG)) if diag_out is None else diag_out
        ptr, n, _ = _ptr(out)
        if n != nsamp * NDIAG:
            raise DgkError(f"diag_out must hold {nsamp * NDIAG} doubles")
        _check(lib().dgk_run(self._h, int(nsteps), float(dt), int(diag_every), ptr), "dgk_run")
        return out

    def run_host(self, inputs, outputs, nsteps, dt):
        """Independent states through host memory, pipelined (dgk_run_host): each of
        inputs[i] is uploaded, advanced nsteps steps of dt and read into outputs[i].
        inputs, outputs: equal-length sequences of host float64 arrays (numpy, or CPU
        tensors; page-locked memory lets the copies overlap the steps)."""
        if len(inputs) != len(outputs):
            raise DgkError("inputs and outputs differ in length")
        n = len(inputs)
        pi, po = (C.c_void_p * max(n, 1))(), (C.c_void_p * max(n, 1))()
        count = int(np.prod(self.shape()))
        for k in range(n):
            for arr, tab in ((inputs[k], pi), (outputs[k], po)):
                ptr, m, dev = _ptr(arr)
                if dev or m != count:
                    raise DgkError("run_host takes host arrays of the state's size")
                tab[k] = ptr
        _check(lib().dgk_run_host(self._h, pi, po, n, count, int(nsteps), float(dt)), "dgk_run_host")

    def max_dt(self, cfl=0.9, dfl=0.4):
        dt = C.c_double()
        _check(lib().dgk_max_dt(self._h, cfl, dfl, C.byref(dt)), "dgk_max_dt")
        return dt.value

    def diagnostics(self):
        out = np.zeros(NDIAG)
        _check(lib().dgk_diagnostics(self._h, out.ctypes.data_as(C.POINTER(C.c_double))), "dgk_diagnostics")
        return dict(zip(DIAG_NAMES, out))

    def temperature_pressure(self):
        """Nodal temperature and pressure, numpy arrays of shape (nelem, np)."""
        T = np.zeros((self.nelem, self.np))
        p = np.zeros((self.nelem, self.np))
        _check(lib().dgk_node_temperature_pressure(self._h, T.ctypes.data, p.ctypes.data, T.size, 0),
               "dgk_node_temperature_pressure")
        return T, p

    def status(self):
        """Synchronise and raise if the device latched an error."""
        _check(lib().dgk_status(self._h), "dgk_status")

    def status_code(self):
        return lib().dgk_status(self._h)

    def set_timing(self, enable):
        _check(lib().dgk_set_timing(self._h, int(bool(enable))), "dgk_set_timing")

    def kernel_time(self, which):
        ms, cnt = C.c_double(), C.c_longlong()
        _check(lib().dgk_kernel_time(self._h, which, C.byref(ms), C.byref(cnt)), "dgk_kernel_time")
        return ms.value, cnt.value


class _BatchMember(Context):
    """A problem of a batch: the single-problem calls on a context owned by the batch."""

    def __init__(self, handle, stream, dim, N):
        self.device = None
        self.stream = stream
        self._h = C.c_void_p(handle)
        ne, npn, nv = C.c_longlong(), C.c_int(), C.c_int()
        _check(lib().dgk_sizes(self._h, C.byref(ne), C.byref(npn), C.byref(nv)), "dgk_sizes")
        self.dim, self.nelem, self.np, self.nv = dim, ne.value, npn.value, nv.value
        self.N = N

    def close(self):
        self._h = C.c_void_p()


class Batch:
    """An ensemble of independent 2D problems advanced by one persistent launch per RK
    stage (FP32-bulk form).  meshes: list of dicts with keys dim, N, n, lo, hi,
    periodic, walls (as for Context.mesh_box)."""

    def __init__(self, meshes, device=0, stream=None, **params):
        import torch
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        p = make_params(precision="fp32bulk", **params)
        arr = (DgkBoxMesh * len(meshes))()
        for k, m in enumerate(meshes):
            dim = m["dim"]
            arr[k] = make_box_mesh(dim, m["N"], list(m["n"]) + [1] * (3 - dim), list(m["lo"]) + [0.0] * (3 - dim),
                                   list(m["hi"]) + [1.0] * (3 - dim), list(m["periodic"]) + [1] * (3 - dim),
                                   m.get("walls"))
        self._h = C.c_void_p()
        _check(lib().dgk_batch_create(C.byref(self._h), device, C.c_void_p(self.stream.cuda_stream), C.byref(p),
                                      len(meshes), arr), "dgk_batch_create")
        self.problems = [_BatchMember(lib().dgk_batch_problem(self._h, k), self.stream, m["dim"], m["N"])
                         for k, m in enumerate(meshes)]

    def close(self):
        if self._h:
            for q in self.problems:
                q.close()
            lib().dgk_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_dt(self, dt):
        dt = np.ascontiguousarray(dt, dtype=np.float64)
        _check(lib().dgk_batch_set_dt(self._h, dt.ctypes.data_as(C.POINTER(C.c_double))), "dgk_batch_set_dt")

    def run(self, nsteps):
        _check(lib().dgk_batch_run(self._h, int(nsteps)), "dgk_batch_run")

    def autotune(self):
        """Time the persistent and grouped forms and the tile lengths; keep the fastest."""
        out = (C.c_int * 7)()
        _check(lib().dgk_batch_autotune(self._h, out), "dgk_batch_autotune")
        return dict(form=("persistent", "grouped", "persistent-wide")[out[0]], blocks_per_sm=out[1], k3=out[2], k4=out[3], k5=out[4],
                    persistent_ms=out[5] / 1e3, grouped_ms=out[6] / 1e3)

    def set_config(self, form, blocks_per_sm, k3, k4, k5):
        """form: "persistent", "grouped" or "persistent-wide" (the persistent kernel compiled
        for two blocks per SM: 128 registers)."""
        cfg = (C.c_int * 5)(("persistent", "grouped", "persistent-wide").index(form), blocks_per_sm, k3, k4, k5)
        _check(lib().dgk_batch_set_config(self._h, cfg), "dgk_batch_set_config")

    def set_barrier_limit(self, cycles):
        """Spin limit of the persistent form's grid barriers, in GPU clock cycles."""
        _check(lib().dgk_batch_set_barrier_limit(self._h, int(cycles)), "dgk_batch_set_barrier_limit")

    def status_code(self):
        """Synchronise; the first error code (0 if none), without raising."""
        per = (C.c_int * len(self.problems))()
        return lib().dgk_batch_status(self._h, per)

    def status(self):
        """Synchronise; raise on the first error (barrier timeout, then any problem's)."""
        per = (C.c_int * len(self.problems))()
        _check(lib().dgk_batch_status(self._h, per), "dgk_batch_status")
        return list(per)

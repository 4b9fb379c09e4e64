/*
 * dgk.h -- C ABI of libdgk: one explicit low-storage Runge-Kutta time step of the DGSEM
 * discretisation of the relaxed, non-isothermal Navier-Stokes-Korteweg equations
 * (Keim, Munz & Rohde, arXiv 2208.05310), on one GB300 (sm_103a).
 *
 * Method (paper references are sections / equations of the paper):
 *   unknowns U = (rho, rho u_1..rho u_d, rho e, c)        Sec. 2.3, Eq. (navierstokeskorteweg_p)
 *   van der Waals fluid, R = 8/3, a = 3, b = 1/3           Sec. 2.1, Eq. (helmholtzfreeenergyvol)
 *   total energy incl. alpha/2 (rho-c)^2 + gamma_K/2 |grad c|^2   Eq. (totalenergyalpha)
 *   relaxation model 1 (p in the flux, alpha rho grad(c - rho) as a source) or
 *   model 2 (modified pressure p + alpha/2 rho^2)          Eq. (navierstokeskorteweg_p), (..._palpha)
 *   DGSEM on Legendre-Gauss nodes; box meshes, curved elements, unstructured connectivity
 *   and 2:1 mortars; Rusanov or (model 2) HLLC flux; BR1 lifting of (rho, u, c), then of
 *   (T, grad c) for grad T and lap c; point-wise sources                Sec. 3.1, Sec. 4
 *   isothermal no-slip walls (at rest or sliding) with a static contact angle, Navier-slip walls
 *                                                          Sec. 2.4, Eq. (bc_nsk_alpha),
 *                                                          Eq. (helmfreesurftot_derivative)
 *   the original NSK model on periodic meshes              Eq. (navierstokeskorteweg)
 *   low-storage RK: 3-stage (Williamson) or 5-stage 4th order (Carpenter-Kennedy)  Sec. 3.1
 *
 * Conventions for every call:
 *   - Return value: DGK_OK (0) or a negative DGK_ERR_* code; no call aborts, throws or
 *     traps.  dgk_status_string() names a code; dgk_last_error() gives details.
 *   - Array layout: structure of arrays, FP64, X[v][e][n] with v the variable, e the
 *     element (e = ix + nx*(iy + ny*iz)) and n the node inside the element
 *     (n = i + P*(j + P*k), P = N+1, i along x).  Sizes from dgk_sizes().
 *   - on_device != 0: the pointer is device memory of the context's GPU; 0: host memory
 *     (pageable or pinned).  Caller-owned pointers are only read or written during the
 *     call (device pointers: in stream order on the context's stream).
 *   - The context owns all other device memory and releases it in dgk_destroy().
 *   - All device work is issued on the context's stream; calls that return data to the
 *     host synchronise that stream.  One context per host thread at a time.
 *   - Device-detected errors (non-finite state, density outside (0, 1/b), T <= 0) are
 *     latched in a device status word; dgk_status() synchronises and returns it, then
 *     clears it.
 */
#ifndef DGK_H
#define DGK_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DGK_OK 0
#define DGK_ERR_ARG (-1)         /* invalid argument (null pointer, size mismatch, bad enum) */
#define DGK_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define DGK_ERR_NONFINITE (-3)   /* device: non-finite value in the state */
#define DGK_ERR_DOMAIN (-4)      /* device: density outside (0, 1/b) or temperature <= 0 */
#define DGK_ERR_STATE (-5)       /* call order: no mesh / params / state yet */
#define DGK_ERR_UNSUPPORTED (-6) /* dimension / degree / model not compiled in */
#define DGK_ERR_NOMEM (-7)       /* device allocation failed */
#define DGK_ERR_THERMO (-8)      /* no saturation states at this temperature (T >= 1) */
#define DGK_ERR_TIMEOUT (-9)     /* device: a grid barrier of the batched kernel timed out */

#define DGK_PREC_FP64 0      /* every kernel in FP64 */
#define DGK_PREC_FP32BULK 1  /* lifting, volume and surface in FP32; the energy balance of
                                the nodal temperature recovery, the RK accumulation and the
                                diagnostics in FP64 */

#define DGK_FLUX_RUSANOV 0   /* Rusanov flux (the paper's flux for model 1) */
#define DGK_FLUX_HLLC 1      /* HLLC flux (the paper's flux for model 2) */

#define DGK_NDIAG 9 /* mass, momentum x/y/z, total energy, -int rho eta, ||rho-c||_2, max|u|,
                       int Pi (rate of entropy production) */

typedef struct dgk_ctx dgk_ctx;

/* Physical and numerical parameters.  Defaults of the paper (Sec. 4, table
   "fluidproperties"): gammaK 1e-4, mu 0.01, kappa 1/150, cv 5; alpha = beta = 100. */
typedef struct {
    int model;       /* 1: relaxation model 1 (Eq. navierstokeskorteweg_p); 2: model 2 (.._palpha);
                        0: the original NSK model (Eq. navierstokeskorteweg, Korteweg stress
                        Eq. cauchystressnsk, energy flux Eq. energyfluxnsk; periodic boxes only).
                        Model 0 keeps the state layout of the relaxation models: the c slot holds
                        rho (set by dgk_set_primitive, kept equal by the kernels) */
    int rk;          /* 3: three-stage LSRK3, 4: five-stage LSRK4 (the paper's default, Sec. 3.1) */
    int precision;   /* DGK_PREC_FP64 or DGK_PREC_FP32BULK */
    double gammaK;   /* capillarity coefficient gamma_K > 0 (Eq. non-dimensionals) */
    double mu;       /* viscosity, Stokes hypothesis (Sec. 2.2) */
    double kappa;    /* heat conductivity */
    double cv;       /* heat capacity ratio cv = c_v/R_gas */
    double alpha;    /* Korteweg relaxation parameter alpha > 0 (Sec. 2.3) */
    double beta;     /* order-parameter relaxation rate beta > 0 (Eq. orderparametersourcenskalpha) */
    int flux;        /* convective numerical flux: DGK_FLUX_RUSANOV, or DGK_FLUX_HLLC (model 2 only; the
                        paper's flux for model 2, Sec. 4; HLLC as in Toro 2009, Sec. 10.4, with the
                        model-2 pressure p + alpha/2 rho^2 and sound speed sqrt(cs^2 + alpha rho)) */
} dgk_params;

/* One face of the box.  kind 0: none (the direction must be periodic); kind 1:
   isothermal no-slip wall at temperature T_wall with static contact angle theta_deg
   (Eq. bc_nsk_alpha with gamma_1 = gamma_2 = gamma_4 = 0; the saturation densities and
   sigma_vl at T_wall are computed by the library, Eq. surftenscoef); kind 2: generalized
   Navier-slip wall, Eq. bc_nsk_alpha with the non-negative parameters gamma[0..3] =
   gamma_1 (contact-angle hysteresis), gamma_2 (slip friction), gamma_3 (heat transfer
   to the wall at T_wall) and gamma_4 (relaxation condition); the fluid slips along the
   wall (no normal velocity).
   u_wall: velocity of a kind-1 wall sliding in its own plane (the moving no-slip wall of
   the sliding-droplet case, Sec. 4): the lifting takes u* = u_wall at the wall and the
   wall's traction does the work (tau n) . u_wall in the energy flux.  Components beyond
   dim are ignored.  On box meshes the normal component must be zero; on curved meshes
   the velocity is projected on the tangent plane at each wall point.  Kind 2 takes
   none (the solid is at rest, Sec. 2.4).  DGK_ERR_ARG otherwise. */
typedef struct {
    int kind;
    double T_wall;
    double theta_deg;
    double gamma[4];    /* kind 2 only */
    double u_wall[3];   /* kind 1 only; zero: a wall at rest */
} dgk_wall;

/* Cartesian box mesh of hexahedral (dim 3) or quadrilateral (dim 2) elements. */
typedef struct {
    int dim;            /* 2 or 3 */
    int N;              /* polynomial degree, 2..5 */
    int n[3];           /* elements per direction (n[2] ignored for dim 2) */
    double lo[3], hi[3];
    int periodic[3];
    dgk_wall wall[6];   /* faces -x, +x, -y, +y, -z, +z */
} dgk_box_mesh;

/* ---------------- context ---------------- */

/* Create a context on CUDA device `device`.  cuda_stream: a cudaStream_t to issue all
   work on (e.g. PyTorch's current stream), or NULL for a stream owned by the context. */
int dgk_create(dgk_ctx **out, int device, void *cuda_stream);
/* Release all device memory and the owned stream.  Accepts NULL. */
void dgk_destroy(dgk_ctx *ctx);
/* Set the parameters (copied).  Must precede dgk_mesh_box; may be changed later for
   the same precision (a state present stays valid). */
int dgk_set_params(dgk_ctx *ctx, const dgk_params *p);
/* Build the box mesh: 1D operators on N+1 Legendre-Gauss nodes (Sec. 3.1), wall
   constants, and device buffers for the state, the RK register and the face traces. */
int dgk_mesh_box(dgk_ctx *ctx, const dgk_box_mesh *mesh);
/* Build a mesh of curved elements with the box's connectivity (Sec. 3.1: curvilinear
   elements described by their metric terms).  mesh gives dim, N, the element counts,
   periodic directions and walls (lo/hi are ignored); xgeo (host, caller-owned, read
   during the call) holds the element maps: coordinate k of element e
   (e = ix + nx (iy + ny iz)) at the equispaced reference points t_a = -1 + 2a/ngeo,
   xgeo[(k * nelem + e) * (ngeo+1)^dim + g], g = a + (ngeo+1)(b + (ngeo+1)c).  Each element
   is the tensor-product polynomial of degree ngeo through its points; neighbouring
   elements must share the points of their common face (periodic directions: up to the
   period's translation).  The library computes the metric terms J a^i (cofactors of
   dX/dxi) and 1/J at the nodes and face points; with ngeo <= N (2D) or 2 ngeo <= N (3D)
   they are polynomials the scheme differentiates exactly, so a uniform flow is
   preserved.  Liftings use the strong BR1 form with the chain rule, the volume integral
   the contravariant fluxes F . J a^i, the faces the numerical flux along the face metric
   (one per face point, shared by both elements; Rusanov, or for model 2 HLLC along the
   unit normal).  Walls of both kinds, along the local normal (Navier slip: the
   tangential projections and tractions of Eq. bc_nsk_alpha with the local normal; a
   sliding wall's velocity projected on the tangent plane).  Errors: DGK_ERR_ARG for an
   element map with J <= 0 at a node; otherwise as dgk_mesh_box.  Memory: the metric terms add
   (dim^2 + 1) values per node in the bulk type and in double, and dim values per face
   point. */
int dgk_mesh_curved(dgk_ctx *ctx, const dgk_box_mesh *mesh, int ngeo, const double *xgeo);
/* Curved elements with unstructured connectivity (Sec. 3.1: the method on general
   hexahedral meshes): as dgk_mesh_curved, with the element neighbours given by tables
   instead of the box's index arithmetic.  mesh gives dim, N, the element count
   (n[0] n[1] n[2]) and the wall table (wall[w] for the faces that name wall w; those
   walls' directions must be non-periodic, kind 1 or 2); lo/hi and the element layout are
   ignored.  conn (host, caller-owned, read during the call): for face f = 2 dir + side of
   element e (in the element's own reference frame), conn[(e * 2dim + f) * 3 + 0..2] =
   (neighbour element, the neighbour's face, orientation), or (-1 - w, 0, 0) on wall w.
   Orientation o maps the face point (a, b) of e's face (tangential indices in increasing
   direction order, a fastest) to the neighbour's (a', b'): (u, v) = o & 1 ? (b, a) : (a, b);
   a' = o & 2 ? N - u : u; b' = o & 4 ? N - v : v (2D: o = 0 or 2).  Every element may have
   its own orientation-preserving frame.  The tables must be symmetric (the neighbour's
   entry names e and f back) and match the element maps (the two elements' face metrics
   agree to 1e-6 relative); otherwise DGK_ERR_ARG.  Fewer than 2^31 elements.  Memory:
   3 ints per element face on the device.
   Mortars (Sec. 3.1: non-conforming faces, the mortar method): a big face facing
   2^(dim-1) half-size faces (2:1 in each tangential direction) has conn = (-100 - m, 0, 0)
   and mortar[(m * 2^(dim-1) + p) * 3 + 0..2] = (small element, its face, orientation) for
   sub-face p (bit 0: the upper half along the big face's first tangential axis, bit 1:
   along its second); the small face has conn = (big element, its face, o | (p + 1) << 3),
   o mapping its points onto the sub-face's points in the big face's frame.  nmortar
   mortars (mortar may be NULL when 0).  The small sides see the big side's traces
   interpolated to their points, the big side the L2 projection of the small sides'
   traces; each small side's numerical flux is evaluated from the big side's face state
   interpolated to its points, and the big side's flux is the L2 projection of the small
   sides' (conservative).  The big face's geometry must be the small faces' (a refinement
   of its element map).  Mortar faces cost three small kernels per stage. */
int dgk_mesh_unstructured(dgk_ctx *ctx, const dgk_box_mesh *mesh, int ngeo, const double *xgeo, const int *conn,
                          const int *mortar, int nmortar);
/* Problem sizes: elements, nodes per element (N+1)^dim, conserved variables dim+3. */
int dgk_sizes(const dgk_ctx *ctx, long long *nelem, int *nodes_per_elem, int *nvar);
/* Node coordinates x[d][e][n] (dim x nelem x np doubles). */
int dgk_node_coords(dgk_ctx *ctx, double *x, int on_device);

/* ---------------- state ---------------- */

/* Set the state from nodal primitive variables prim[v][e][n], v = (rho, u_1..u_dim, T, c):
   rho e = rho (R cv T - a rho) + rho|u|^2/2 + alpha/2 (rho-c)^2 + gamma_K/2 |grad c|^2
   (Eq. totalenergyalpha) with grad c the BR1-lifted gradient of c, so that the
   temperature the scheme recovers equals T.  Resets the RK register. */
int dgk_set_primitive(dgk_ctx *ctx, const double *prim, size_t count, int on_device);
/* Copy a conserved state in / out (count = nvar*nelem*np).  Upload resets the RK register. */
int dgk_upload_state(dgk_ctx *ctx, const double *U, size_t count, int on_device);
int dgk_download_state(dgk_ctx *ctx, double *U, size_t count, int on_device);

/* ---------------- the hot path ---------------- */

/* One evaluation of the semi-discrete right-hand side U_t = R(U) of the current state
   (all steps of Sec. 3.1: lifting, temperature, second lifting, volume integral with
   the derivative matrix per direction, Rusanov + viscous surface fluxes, Jacobian, point
   sources); Ut has count = nvar*nelem*np doubles.  The state is not changed. */
int dgk_rhs(dgk_ctx *ctx, double *Ut, size_t count, int on_device);
/* One low-storage RK step of size dt (all stages; per stage G = A_s G + dt R(U),
   U = U + B_s G, fused into the surface kernel).  Asynchronous. */
int dgk_rk_step(dgk_ctx *ctx, double dt);
/* nsteps RK steps of size dt, launched as a captured CUDA graph of one step.
   Asynchronous; check dgk_status() afterwards.
   Diagnostics inside the run: with diag_every > 0 and diag_out non-null, after every
   diag_every-th step the integral diagnostics of dgk_diagnostics() are taken on the device
   (a second captured graph: no host round trip per sample) and stored; at the end the
   nsteps / diag_every samples, DGK_NDIAG doubles each in step order, are copied to
   diag_out (device or host memory; host memory: the call then waits for the run).  The
   samples do not change the trajectory (bitwise the same states as without them), and
   each equals dgk_diagnostics() called after that step.  diag_every = 0 or diag_out
   NULL: no samples.  Device buffers for the samples are allocated on first use. */
int dgk_run(dgk_ctx *ctx, int nsteps, double dt, int diag_every, double *diag_out);
/* Independent problems through host memory, pipelined: for i = 0..nitems-1 the state
   becomes in[i] (as dgk_upload_state), advances nsteps RK steps of size dt (as dgk_run),
   and is read into out[i].  in[i] and out[i] are host pointers of count =
   nvar*nelem*np doubles each (page-locked memory lets the copies run asynchronously;
   the same pointer may appear in several entries, and an out[i] may alias an in[j] with
   j <= i only if the caller does not need in[j] afterwards: out[i] is written while
   item i+1 is copied in).  Item i steps in device buffer i mod 3 while item i+1 is
   copied into the next buffer and item i-1 out of the previous one, on two copy streams
   of the context; the three buffers of count doubles and a captured step graph per
   buffer are made on the first call and kept.  Blocks until out[nitems-1] is written;
   afterwards the context holds the last item's state.  Errors: DGK_ERR_ARG for null arrays or
   entries, a wrong count, nitems < 0, nsteps < 0 or dt <= 0; device-detected errors
   are latched as for dgk_run (check dgk_status()). */
int dgk_run_host(dgk_ctx *ctx, const double *const *in, double *const *out, int nitems, size_t count, int nsteps,
                 double dt);
/* Largest stable step for the current state: min of CFL/((2N+1) max sum_d (|u_d|+s)/h_d),
   DFL/((2N+1)^2 nu_max sum_d h_d^-2) and 2/(alpha beta); s^2 = c_s^2 + alpha rho. */
int dgk_max_dt(dgk_ctx *ctx, double cfl, double dfl, double *dt);
/* Integral diagnostics (Gauss quadrature, FP64 sums in a fixed order on the device):
   out[DGK_NDIAG] = mass, momentum x, y, z, total energy, -int rho eta, ||rho - c||_2,
   max|u|, and int Pi, the rate of entropy production (Sec. 2.3):
   Pi = tau : grad u / T + kappa |grad T|^2 / T^2 + beta (gamma_K lap c + alpha (rho - c))^2 / T
   (the last term for the relaxation models) with the scheme's lifted gradients (the
   bulk type computes Pi per node; the sums are FP64).  Synchronises. */
int dgk_diagnostics(dgk_ctx *ctx, double *out);
/* Nodal temperature (recovered from the total energy with the lifted grad c, as the
   scheme does) and pressure p(rho, T) (Eq. pressure), each nelem*np doubles [e][n];
   either pointer may be NULL.  Synchronises. */
int dgk_node_temperature_pressure(dgk_ctx *ctx, double *T, double *p, size_t count, int on_device);
/* Synchronise the stream and return (then clear) the latched device status. */
int dgk_status(dgk_ctx *ctx);
/* Event-timed duration (ms) of the last timed launch of each kernel class, for roofline
   accounting: which = 0 lift1, 1 lift2+volume, 2 surface+RK.  Enabled by dgk_set_timing. */
int dgk_set_timing(dgk_ctx *ctx, int enable);
int dgk_kernel_time(dgk_ctx *ctx, int which, double *ms_total, long long *launches);

/* Measured fused multiply-add throughput of device `device` (flops per second, 2 per
   FMA): precision DGK_PREC_FP64 for double, DGK_PREC_FP32BULK for float.  The roof of
   the arithmetic-bound kernels (the FP64 form's kernels are bound by the FP64 pipe): a
   grid of 8 blocks of 256 threads per SM, each thread running 8 independent FMA chains,
   best of five event-timed launches after a warm-up.  Allocates and frees a small
   output array; synchronises the device.  The paper has no counterpart (measurement). */
int dgk_fma_peak(int device, int precision, double *flops_per_s);

/* ---------------- thermodynamics (host) ---------------- */

/* Maxwell (saturation) densities at T in (0, 1) (Sec. 2.1). */
int dgk_maxwell(double T, double *rho_v, double *rho_l);
/* Equilibrium surface tension, Eq. (surftenscoef) with prefactor sqrt(2 gamma_K),
   15-point Gauss quadrature (Sec. 3.2). */
int dgk_sigma_vl(double T, double cv, double gammaK, double *sigma);
/* Initial interface width L_i = sqrt(2) gamma_K (rho_l - rho_v)^2 / sigma (Sec. 4). */
int dgk_interface_width(double T, double cv, double gammaK, double *width);

/* Self-check of the library's own binary64 <-> binary32 conversions (integer arithmetic,
   used by the FP32-bulk kernels to stay off the FP64 pipe) against the GPU's hardware
   conversions, bit for bit, on the n doubles at x.  *mismatches = number of inputs whose
   results differ (inputs rounding below the float normal range are skipped).  Allocates
   and synchronises the current device. */
int dgk_check_conversions(const double *x, size_t n, int on_device, unsigned long long *mismatches);

/* ---------------- batched ensembles ----------------
 *
 * Many independent 2D problems (degrees N = 3, 4, 5, any mesh sizes, walls and
 * temperatures; common physics parameters, FP32-bulk form) advanced together, one step
 * replayed as a captured CUDA graph.  Persistent form: every RK stage is ONE cooperative
 * launch that runs the three phases of the stage for all problems, separated by grid
 * barriers (bounded spin; a timeout is reported as DGK_ERR_TIMEOUT, never a hang).
 * Grouped form: every phase is one launch over all problems.  The autotuner picks.
 * Each problem has its own time step.  The problems are ordinary contexts owned by the
 * batch: use dgk_batch_problem() with the single-problem calls (set-up, download,
 * diagnostics, max_dt).
 */
typedef struct dgk_batch dgk_batch;
/* p: common parameters (precision must be DGK_PREC_FP32BULK, flux DGK_FLUX_RUSANOV);
   meshes[nprob]: 2D box
   meshes with N in 3..5.  cuda_stream as for dgk_create (shared by all problems). */
int dgk_batch_create(dgk_batch **out, int device, void *cuda_stream, const dgk_params *p, int nprob,
                     const dgk_box_mesh *meshes);
void dgk_batch_destroy(dgk_batch *b);
/* The context of problem i (owned by the batch; do not destroy). */
dgk_ctx *dgk_batch_problem(dgk_batch *b, int i);
/* Time step of every problem (dt[nprob]). */
int dgk_batch_set_dt(dgk_batch *b, const double *dt);
/* nsteps RK steps of every problem: stages x one persistent launch per step, replayed
   from a captured graph.  Asynchronous. */
int dgk_batch_run(dgk_batch *b, int nsteps);
/* Autotuner: times candidate forms and work decompositions -- the persistent form
   (one cooperative launch per stage, phases separated by grid barriers) for each count
   of resident blocks per SM, the grouped form (one launch per phase over the tiles of
   all problems, one element block per CTA), and, if the persistent form wins, element
   blocks per tile k_N for each degree N -- and keeps the fastest.  Every candidate runs three steps from the current states,
   which are restored afterwards; the status words are cleared after tuning (tuning
   refuses to start, returning the error, if a problem already reports one).
   out (nullable, 7 ints) = {form (0, 1 or 2 as for dgk_batch_set_config), blocks_per_sm,
   k_3, k_4, k_5, microseconds per step of the best persistent candidate (either
   allocation), microseconds per step of the grouped form}. */
int dgk_batch_autotune(dgk_batch *b, int *out);
/* Set the form and decomposition directly: cfg = {form (0 persistent, 1 grouped,
   2 persistent compiled for 2 blocks per SM: 128 registers instead of 80 with spills),
   blocks_per_sm (1..the occupancy limit of that persistent kernel), k_3, k_4, k_5 (>= 1;
   element blocks per tile of the persistent forms; the grouped form ignores them and
   blocks_per_sm)}.
   Results do not depend on it: every element's arithmetic is the same. */
int dgk_batch_set_config(dgk_batch *b, const int *cfg);
/* Synchronise; per_problem (nullable, nprob ints) receives each problem's status.
   Returns the first error: barrier timeout, then any problem's error.  After a barrier
   timeout the barrier's arrival counter is reset here; the problems' states are then
   partly advanced and must be set again before the next run. */
int dgk_batch_status(dgk_batch *b, int *per_problem);
/* Spin limit of the persistent form's grid barriers, in GPU clock cycles (cycles >= 1;
   default 4e9, about 2 s at 2 GHz).  A block that waits longer latches the barrier
   status and returns, and dgk_batch_status() reports DGK_ERR_TIMEOUT: the kernel never
   hangs on a missing block.  Synchronises the batch's stream; takes effect at the next
   dgk_batch_run (the limit is a kernel parameter; the step graph is captured again).  A limit of a
   few cycles makes the barrier waits run out, which exercises that error path. */
int dgk_batch_set_barrier_limit(dgk_batch *b, long long cycles);

/* ---------------- allocation-free right-hand side ----------------
 *
 * The paper has no counterpart to this entry point; it is a deployment variant of
 * dgk_rhs for callers that cannot call cudaMalloc: applications whose device memory is
 * entirely reserved by another allocator's pool (for example a framework's caching
 * allocator that owns the GPU), and loops that must never synchronise the device
 * (cudaMalloc and cudaFree may synchronise implicitly).
 *
 * dgk_rhs_static computes exactly what dgk_rhs computes, for the state U (device
 * pointer, SoA [nvar][nelem][np] FP64, read only) into Ut (device pointer, same layout),
 * each holding count = nvar*nelem*np doubles of the mesh passed in, on cuda_stream
 * (NULL: the default stream) of the current device, with the parameters and mesh passed
 * in.  It creates no context and calls no cudaMalloc, cudaFree or other allocating
 * routine: every intermediate array lives in one file-scope device array of
 * DGK_STATIC_SCRATCH_BYTES bytes inside libdgk, which every GPU that loads the library
 * holds until the process exits.  Asynchronous: synchronise cuda_stream before reading Ut.
 *   - Size limit: a mesh whose intermediates need more than DGK_STATIC_SCRATCH_BYTES is
 *     rejected with DGK_ERR_ARG and dgk_last_error() says so (e.g. 3D N = 5 in FP64 fits
 *     about 1490 elements, in the FP32-bulk form about 2900).  A count that does not
 *     match the mesh is rejected with DGK_ERR_ARG before any device work.
 *   - status (nullable): receives the call's device status word, DGK_STATUS_* bits (0: the
 *     kernels found every node finite and inside the EoS domain), copied in stream order
 *     after the kernels.  Host or device memory; with pageable host memory the copy, and
 *     so the call, waits for the kernels to finish.
 *   - The first call on a device looks up the scratch array's device address (once per
 *     device, with that device current); make that first call before any stream capture.
 *   - All calls share the array and it keeps the last call's contents; each call clears
 *     the only value that must start at zero (the status word).  Calls that overlap on
 *     the GPU (different streams or host threads) race on the array: serialise them.
 */
#define DGK_STATIC_SCRATCH_BYTES (64u << 20)
#define DGK_STATUS_NONFINITE 1u /* a non-finite density, temperature or energy at some node */
#define DGK_STATUS_DOMAIN 2u    /* a density outside (0, 1/b) or a temperature <= 0 at some node */
int dgk_rhs_static(const dgk_params *p, const dgk_box_mesh *mesh, const double *U, double *Ut, size_t count,
                   void *cuda_stream, unsigned *status);

const char *dgk_status_string(int status);
/* Text of the most recent error in this thread (empty if none). */
const char *dgk_last_error(void);

#ifdef __cplusplus
}
#endif
#endif

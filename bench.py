"""Throughput benchmark of the DGSEM relaxed-NSK time step on GB300.

Workload (default): non-isothermal confined liquid bridge between two parallel walls,
3D, N = 5 on 64x64x32 elements of [0,2]x[0,2]x[0,1] (28.3 M nodes), periodic in x and
y, bottom wall 0.95, top wall 0.8 (isothermal no-slip, contact angle 90 deg), T0 = 0.85,
relaxation model 1 with alpha = beta = 100, the paper's fluid properties, LSRK4 (5
stages).  Metric: DOF-stage updates per second (nodes x RK stages / time).

Arms:
  default             libdgk on the GPU (FP32-bulk form as the headline; FP64 form and
                      end-to-end host-buffer throughput reported beside it)
  --impl reference    the FP64 CPU oracle on the host cores, on a bounded sub-box of the
                      same workload (the paper publishes no timing to compare against)

Multi-GPU (torchrun): every rank runs its own replica (independent problems, no data
exchange); value = total DOF-stage updates of all ranks / max-over-ranks time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-stage updates/s (DGSEM RHS+RK), FP32/batched vs FP64 at stated err; % HBM roof"
UNIT = "DOF-stage/s"

# Algorithmic bytes per node and launch of each stage kernel: every array element the
# kernel consumes or produces, once (R = bulk type size; 3D: NV = 6, NL = 5, one face
# point per node for N = 5).  The lifting kernels read the state: in the FP64 form the
# double state, in the FP32-bulk form its float shadow (NV values and the energy
# balance), which the RK update writes beside the double state.
def kernel_bytes_per_node(dim, N, rsize, flux="rusanov", curved=False):
    """curved: the curved-element kernels read in addition the metric terms (dim^2 + 1
    values per node: J a^i and 1/J) and the face metrics (dim values per face point) in
    the lifting kernels, and 1/J in k_surf_rk (with HLLC also the face metrics, for the
    unit normal)."""
    nv, nl = dim + 3, dim + 2
    f = 2 * dim / (N + 1)  # face points per node (own faces)
    nfd = 2 * nv + (3 if flux == "hllc" else 1)  # face data values (HLLC: + pressure, sound speed)
    state = 8 * nv if rsize == 8 else rsize * (nv + 1)
    shadow_w = 0 if rsize == 8 else rsize * (nv + 1)
    lift1 = state + rsize * 1 * f + rsize * 2 * f                       # c traces in, T and dc/dn traces out
    lift2 = state + rsize * nl * f + rsize * 2 * f + rsize * nv + rsize * nfd * f
    surf = rsize * nfd * f + rsize * nv + 8 * nv * 4 + rsize * nl * f + shadow_w
    if curved:
        geo = rsize * (dim * dim + 1) + rsize * dim * f
        surf += rsize + (rsize * dim * f if flux == "hllc" else 0)
        return {"k_lift1c": lift1 + geo, "k_lift2volc": lift2 + geo, "k_surf_rk": surf}
    return {"k_lift1": lift1, "k_lift2vol": lift2, "k_surf_rk": surf}


# element maps of the curved variant of a workload (`--mesh curved`): degree 2, walls
# bent by 2% of the domain height
CURVED_GEOMETRY = dict(ngeo=2, amp=0.02)


def mesh_arrays(m, wl):
    """(ngeo, element maps, connectivity tables or None, mortar table or None) of a
    workload's curved, unstructured or refined variant, or None for the box."""
    if wl.get("refine"):
        from paper_2208_05310_gb300 import inputs
        g = wl["geometry"]
        xg, conn, mort = inputs.refined_mesh(m["dim"], m["N"], m["n"], m["periodic"], m["walls"], g["ngeo"],
                                             amp=g["amp"], lo=m["lo"], hi=m["hi"])
        return g["ngeo"], xg, conn, mort
    geo = geometry_of(m, wl.get("geometry"))
    if geo is None or wl.get("reorient") is None:
        return None if geo is None else (geo[0], geo[1], None, None)
    from paper_2208_05310_gb300 import inputs
    xn, conn = inputs.reoriented_frames(m["dim"], m["N"], m["n"], m["periodic"], geo[0], geo[1], wl["reorient"])
    return geo[0], xn, conn, None


def geometry_of(m, geo):
    """(ngeo, element maps) of a curved variant of mesh m (inputs.box_geometry), or None."""
    if not geo:
        return None
    from paper_2208_05310_gb300 import inputs
    return geo["ngeo"], inputs.box_geometry(m["dim"], m["n"], m["lo"], m["hi"], geo["ngeo"], amp=geo["amp"])


def workload_c5(scale=1):
    """Confined heated liquid bridge (3D, N = 5)."""
    n = [64 // scale, 64 // scale, 32]
    hi = [2.0 / scale, 2.0 / scale, 1.0]
    return dict(name="confined heated liquid bridge between walls (0.95 / 0.8 Tc), 3D N=5, "
                     f"{n[0]}x{n[1]}x{n[2]} elements, LSRK4",
                mesh=dict(dim=3, N=5, n=n, lo=[0.0, 0.0, 0.0], hi=hi, periodic=[1, 1, 0],
                          walls={4: (0.95, 90.0), 5: (0.8, 90.0)}),
                params=dict(model=1, gammaK=1e-4, mu=0.01, kappa=1.0 / 150.0, cv=5.0, alpha=100.0, beta=100.0),
                rk=4, T0=0.85, radius=0.5, center=[1.0, 1.0, 0.5], axes=(0, 1))


def workload_c2():
    return dict(name="static droplet, 2D N=4, 64x64 elements, LSRK4",
                mesh=dict(dim=2, N=4, n=[64, 64], lo=[0.0, 0.0], hi=[1.0, 1.0], periodic=[1, 1], walls={}),
                params=dict(model=1, gammaK=1e-4, mu=0.01, kappa=1.0 / 150.0, cv=5.0, alpha=100.0, beta=100.0),
                rk=4, T0=0.8, radius=0.25, center=[0.5, 0.5], axes=None, noise=1e-3)


def workload_c4(nprob=256):
    return dict(name=f"batched ensemble of {nprob} independent 2D droplets / bubbles on contact-angle walls, "
                     "16x16..96x96 elements, N in {3,4,5}, T in [0.75,0.9] Tc, theta in [30,150] deg, LSRK4",
                batch=dict(nprob=nprob, seed=2024, n_range=(16, 96)),
                params=dict(model=1, gammaK=1e-4, mu=0.01, kappa=1.0 / 150.0, cv=5.0, alpha=100.0, beta=100.0),
                rk=4)


WORKLOADS = {"c5": workload_c5, "c5s": lambda: workload_c5(scale=2), "c2": workload_c2, "c4": workload_c4,
             "c4s": lambda: workload_c4(32)}


def primitive_state(wl, x, rv, rl, width):
    from paper_2208_05310_gb300 import inputs
    noise = inputs.uniform_noise(x[0].shape, 2208) if wl.get("noise") else None
    return inputs.droplet(x, wl["center"], wl["radius"], rv, rl, width, wl["T0"], liquid_inside=True, noise=noise,
                          noise_amp=wl.get("noise", 0.0), axes=wl.get("axes"))


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


L2_BYTES = 129e6  # GB300 L2 (126 MiB)


def l2_note(state_bytes):
    """How the timed steps stand to the L2: the workloads the bench reports stream a state
    larger than L2 every stage (no flush needed); smaller ones say that they fit."""
    if state_bytes > L2_BYTES:
        return "inputs larger than L2: state %.2f GB" % (state_bytes / 1e9)
    return "inputs fit in L2 (state %.1f MB), L2 not flushed: a parity-size case, not a headline line" % (state_bytes / 1e6)


def kernel_sources_sha(curved=False, batch=False):
    """Hash of the sources of the stage kernels (with the curved-element kernels for a
    curved workload, the batched kernels for the ensemble): a committed ncu summary
    counts only while it matches."""
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2208_05310_gb300", "csrc")
    for fn in ("dgk_common.cuh", "dgk_kernels.cuh") + (("dgk_curved.cuh",) if curved else ()) + \
            (("dgk_batch.cu",) if batch else ()):
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    curved = any(k in workload for k in ("curved", "unstructured", "mortar"))
    if vals.get("kernel_source_sha1") != kernel_sources_sha(curved=curved):
        return None
    try:
        return float(vals["dram_bytes_per_launch_full"])
    except (KeyError, ValueError):
        return None


def batch_traffic(workload):
    """DRAM bytes of one RK stage of the grouped batched form (its three phase launches)
    from the committed ncu summary of that workload, while it matches the sources."""
    path = os.path.join(ROOT, "profiles", f"k_batch_phase_{workload}_fp32.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha1") != kernel_sources_sha(batch=True):
        return None
    try:
        return float(vals["dram_bytes_per_stage"])
    except (KeyError, ValueError):
        return None


def ncu_flops(kernel, workload):
    """Executed FP64 flops per node (2 per DFMA + DADD + DMUL, from the ncu counters of
    the committed summary) and the summary's DRAM bytes per launch, while the summary
    matches the current kernel sources; else (None, None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")
    if not os.path.exists(path):
        return None, None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha1") != kernel_sources_sha():
        return None, None
    try:
        return float(vals["fp64_flops_per_node"]), float(vals["dram_bytes_per_launch_full"])
    except (KeyError, ValueError):
        return None, None


def replica_max(v, dist=None, device="cuda"):
    """Max of a per-rank time over all ranks (replicas run independent problems; the
    slowest rank sets the whole job's time).  dist: torch.distributed or None."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank, world, ms_max):
    """Whole-job rate: the units all ranks processed over the max-over-ranks time."""
    return units_per_rank * world / (ms_max / 1e3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.out.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [s.strip() for s in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax = float(p[2])
                except ValueError:
                    continue
                for nm, val in zip(names, p[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def oracle_rate(wl, seconds_target=15.0, steps=None, sub=(6, 6, None), single_thread=False):
    """FP64 oracle DOF-stage/s on a sub-box of the workload with the same N and element
    size (periodic laterally, the workload's walls in z)."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import numpy as np
    import oracle as orc
    m = wl["mesh"]
    dim = m["dim"]
    h = [(m["hi"][d] - m["lo"][d]) / m["n"][d] for d in range(dim)]
    nsub = [sub[d] if sub[d] else m["n"][d] for d in range(dim)]
    hi = [m["lo"][d] + nsub[d] * h[d] for d in range(dim)]
    arrs = mesh_arrays(dict(m, n=nsub, hi=hi), wl)
    ncount = nsub if not (arrs and arrs[3] is not None) else [arrs[1].shape[1], 1, 1]
    mesh = orc.make_mesh(dim, m["N"], ncount + [1] * (3 - dim), m["lo"] + [0.0] * (3 - dim), hi + [1.0] * (3 - dim),
                         m["periodic"] + [1] * (3 - dim), m["walls"], geometry=arrs[:2] if arrs else None,
                         conn=arrs[2] if arrs else None, mortar=arrs[3] if arrs else None)
    o = orc.Oracle(mesh, orc.make_params(**wl["params"]))
    rv, rl = orc.maxwell(wl["T0"])
    width = orc.interface_width(wl["T0"], 5.0, wl["params"]["gammaK"])
    wl2 = dict(wl, center=[0.5 * hi[0], 0.5 * hi[1]] + wl["center"][2:], radius=min(wl["radius"], 0.3 * hi[0]))
    U = o.set_primitive(primitive_state(wl2, o.node_coords(), rv, rl, width))
    dt = o.max_dt(U)
    stages = 5 if wl["rk"] == 4 else 3
    dof = o.nelem * o.np
    t0 = time.perf_counter()
    U = o.run(U, 1, dt, rk=wl["rk"])
    t1 = time.perf_counter() - t0
    nsteps = steps if steps is not None else max(0, int(seconds_target / max(t1, 1e-3)) - 1)
    t0 = time.perf_counter()
    if nsteps:
        U = o.run(U, nsteps, dt, rk=wl["rk"])
    tt = time.perf_counter() - t0
    total_steps = nsteps if nsteps else 1
    total_t = tt if nsteps else t1
    assert np.isfinite(U).all()
    cores = orc.num_threads()
    single = None
    if single_thread:
        # the same sub-box on one thread, one RK step
        orc.set_num_threads(1)
        t0 = time.perf_counter()
        U = o.run(U, 1, dt, rk=wl["rk"])
        single = dof * stages / (time.perf_counter() - t0)
        orc.set_num_threads(cores)
    return dict(rate=dof * stages * total_steps / total_t, cores=cores, dof=dof, steps=total_steps,
                seconds=total_t, sub=f"a {nsub} sub-box", single=single)


def oracle_rate_batch(wl, steps, nsample=2):
    """FP64 oracle DOF-stage/s on the first `nsample` problems of the ensemble (full size),
    one after the other."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import numpy as np
    import oracle as orc
    from paper_2208_05310_gb300 import inputs
    b = wl["batch"]
    specs = inputs.ensemble_specs(b["nprob"], b["seed"], n_range=b["n_range"])[:nsample]
    stages = 5 if wl["rk"] == 4 else 3
    dof, total = 0, 0.0
    for sp in specs:
        m = inputs.ensemble_mesh(sp)
        o = orc.Oracle(orc.make_mesh(2, m["N"], m["n"] + [1], m["lo"] + [0.0], m["hi"] + [1.0], m["periodic"] + [1],
                                     m["walls"]), orc.make_params(**wl["params"]))
        rv, rl = orc.maxwell(sp["T"])
        U = o.set_primitive(inputs.ensemble_primitive(o.node_coords(), sp, rv, rl,
                                                      orc.interface_width(sp["T"], wl["params"]["cv"],
                                                                          wl["params"]["gammaK"])))
        dt = o.max_dt(U)
        t0 = time.perf_counter()
        U = o.run(U, steps, dt, rk=wl["rk"])
        total += time.perf_counter() - t0
        assert np.isfinite(U).all()
        dof += o.nelem * o.np
    return dict(rate=dof * stages * steps / total, cores=orc.num_threads(), dof=dof, steps=steps, seconds=total,
                sub=f"first {nsample} problems of the ensemble")


def run_reference(args, wl, rank, world):
    if rank != 0:
        return 0
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as orc
    orc.lib()
    # warm-up steps, then K timed steps; one step = one RK step on the sample
    rate = (lambda k: oracle_rate_batch(wl, k)) if "batch" in wl else (lambda k: oracle_rate(wl, steps=k))
    r_w = rate(max(args.warmup, 1))
    r = rate(max(args.steps, 1))
    sample = f"one RK step per bench step on {r['sub']} of the workload ({r['dof']} nodes)"
    line = dict(metric=METRIC, value=r["rate"], unit=UNIT, n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * r["seconds"] / r["steps"], higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=wl["name"], sample=sample, stages_per_step=5 if wl["rk"] == 4 else 3),
                cpu_baseline=dict(value=r["rate"], unit=UNIT, cores=r["cores"], kind="oracle", sample=sample,
                                  cpu_model=cpu_model()),
                e2e=dict(value=r["rate"], unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    del r_w
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, wl, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2208_05310_gb300 import dgk

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    m = wl["mesh"]
    stages = 5 if wl["rk"] == 4 else 3

    def make_ctx(precision):
        ctx = dgk.Context(device=local_rank)
        ctx.set_params(rk=wl["rk"], precision=precision, **wl["params"])
        dim = m["dim"]
        arrs = mesh_arrays(m, wl)
        if arrs and arrs[2] is not None:
            ncount = m["n"] if arrs[3] is None else [arrs[1].shape[1], 1, 1]
            ctx.mesh_unstructured(dim, m["N"], ncount + [1] * (3 - dim), m["periodic"] + [1] * (3 - dim), m["walls"],
                                  *arrs)
        elif arrs:
            ctx.mesh_curved(dim, m["N"], m["n"] + [1] * (3 - dim), m["periodic"] + [1] * (3 - dim), m["walls"],
                            arrs[0], arrs[1])
        else:
            ctx.mesh_box(dim, m["N"], m["n"] + [1] * (3 - dim), m["lo"] + [0.0] * (3 - dim),
                         m["hi"] + [1.0] * (3 - dim), m["periodic"] + [1] * (3 - dim), m["walls"])
        rv, rl = dgk.maxwell(wl["T0"])
        width = dgk.interface_width(wl["T0"], wl["params"]["cv"], wl["params"]["gammaK"])
        ctx.set_primitive(primitive_state(wl, ctx.node_coords(), rv, rl, width))
        return ctx

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v):
        return replica_max(v, dist)

    ctx = make_ctx(args.precision)
    dof = ctx.nelem * ctx.np
    # the original NSK model has no capillary term in the step rule: a fraction of it
    dt = ctx.max_dt(0.9, 0.4) * (0.05 if wl["params"].get("model") == 0 else 1.0)
    # warm-up (also captures the step graph)
    ctx.run(args.warmup, dt)
    ctx.status()

    # --- pass A: graph-launched steps, headline throughput
    s = ctx.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local_rank) as clk:
        e0.record(s)
        ctx.run(args.steps, dt)
        e1.record(s)
        s.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    ctx.status()
    ms_max = max_over_ranks(ms)
    value = replica_rate(dof * stages * args.steps, world, ms_max)

    # --- pass B: the same steps kernel by kernel with per-kernel CUDA events
    ctx.set_timing(True)
    barrier()
    ctx.run(args.steps, dt)
    ktimes = {}
    curved = bool(wl.get("geometry"))
    for k, name in enumerate(("k_lift1c", "k_lift2volc", "k_surf_rk") if curved else ("k_lift1", "k_lift2vol", "k_surf_rk")):
        tot, cnt = ctx.kernel_time(k)
        ktimes[name] = (tot, cnt)
    ctx.set_timing(False)
    ctx.status()
    rsize = 4 if args.precision == "fp32bulk" else 8
    kb = kernel_bytes_per_node(m["dim"], m["N"], rsize, wl["params"].get("flux", "rusanov"), curved=curved)
    total_k = sum(t for t, _ in ktimes.values())
    dom = max(ktimes, key=lambda k: ktimes[k][0])
    avg_ms = ktimes[dom][0] / max(ktimes[dom][1], 1)
    alg_bytes = kb[dom] * dof
    peak, peak_kind = measured_peak()
    achieved = alg_bytes / (avg_ms / 1e3) / 1e9
    kind = "" if not curved else ("mortar" if wl.get("refine") else
                                  "unstructured" if wl.get("reorient") is not None else "curved")
    traffic = ncu_traffic(dom, args.workload + kind + ("_fp32" if rsize == 4 else "_fp64"))
    roofline = dict(bound="hbm", achieved=achieved, peak=peak, unit="GB/s", frac=achieved / peak, traffic=traffic,
                    kernel=dom, peak_kind=peak_kind, alg_bytes_per_launch=alg_bytes,
                    avg_launch_ms=avg_ms,
                    share={k: ktimes[k][0] / total_k for k in ktimes},
                    step_bytes_alg=(8 * (m["dim"] + 3) * 4) * dof * stages,
                    step_frac_alg=(8 * (m["dim"] + 3) * 4) * dof * stages / (ms / args.steps / 1e3) / 1e9 / peak,
                    step_bytes_dataflow=sum(kb.values()) * dof * stages,
                    step_frac_dataflow=sum(kb.values()) * dof * stages / (ms / args.steps / 1e3) / 1e9 / peak)
    del ctx
    torch.cuda.synchronize()

    # --- FP64 form on the same GPU (fewer steps: FP64 is ALU-bound on this part)
    fp64 = None
    if args.precision != "fp64" and not args.no_fp64:
        c64 = make_ctx("fp64")
        k64 = max(1, args.steps // 4)
        c64.run(1, dt)
        c64.status()
        barrier()
        e0.record(c64.stream)
        c64.run(k64, dt)
        e1.record(c64.stream)
        c64.stream.synchronize()
        barrier()
        ms64 = max_over_ranks(e0.elapsed_time(e1))
        c64.status()
        fp64 = dict(value=dof * stages * k64 * world / (ms64 / 1e3), unit=UNIT, steps=k64, ms_per_step=ms64 / k64)
        # the FP64 form against its arithmetic roof: the dominant kernel's executed FP64 flops
        # per launch (ncu counters of the committed summary) over its CUDA-event launch
        # time, against the FP64 FMA throughput measured now on this GPU
        c64.set_timing(True)
        c64.run(1, dt)
        k64t = {}
        for k, name in enumerate(("k_lift1c", "k_lift2volc", "k_surf_rk") if curved else ("k_lift1", "k_lift2vol", "k_surf_rk")):
            k64t[name] = c64.kernel_time(k)
        c64.set_timing(False)
        c64.status()
        dom64 = max(k64t, key=lambda k: k64t[k][0])
        avg64 = k64t[dom64][0] / max(k64t[dom64][1], 1)
        fl_node, traffic64 = (None, None) if curved else ncu_flops(dom64, args.workload + "_fp64")
        peak64 = dgk.fma_peak(local_rank, "fp64") / 1e12
        ach64 = fl_node * dof / (avg64 / 1e3) / 1e12 if fl_node else None
        fp64["roofline"] = dict(bound="fp64_alu", kernel=dom64, achieved=ach64, peak=peak64, unit="TFLOP/s",
                                frac=(ach64 / peak64) if ach64 else None, peak_kind="measured (dgk_fma_peak, this run)",
                                flops_per_node=fl_node, avg_launch_ms=avg64, traffic=traffic64,
                                share={k: v[0] / sum(t for t, _ in k64t.values()) for k, v in k64t.items()})
        # the headline form against the FP64 form from the same initial state after the same
        # steps: relative L2 difference per conserved variable
        k_acc = max(args.accuracy_steps, 1 + k64)
        if k_acc > 1 + k64:
            c64.run(k_acc - 1 - k64, dt)
            c64.status()
        c32 = make_ctx(args.precision)
        c32.run(k_acc, dt)
        c32.status()
        u64 = torch.empty(c64.shape(), dtype=torch.float64, device=f"cuda:{c64.device}")
        u32 = torch.empty_like(u64)
        torch.cuda.synchronize()
        c64.download_state(u64)
        c32.download_state(u32)
        c64.stream.synchronize()
        c32.stream.synchronize()
        diff = torch.linalg.vector_norm((u32 - u64).reshape(u64.shape[0], -1), dim=1)
        ref = torch.linalg.vector_norm(u64.reshape(u64.shape[0], -1), dim=1)
        names = ["rho"] + [f"m_{'xyz'[k]}" for k in range(m["dim"])] + ["rho_e", "c"]
        # the parity norm: ||a - b|| / max(||b||, floor_v sqrt(nodes)) with the floors
        # rho_l (rho, rho e, c) and rho_l / 100 (momentum), rho_l the liquid saturation
        # density at the initial temperature (a state at rest has a near-zero momentum norm)
        rl = dgk.maxwell(wl["T0"])[1]
        fl = torch.tensor([rl] + [1e-2 * rl] * m["dim"] + [rl, rl], dtype=torch.float64, device=diff.device)
        den = torch.maximum(ref, fl * float(np.sqrt(u64[0].numel())))
        fp64["vs_headline"] = dict(steps=k_acc, rel_l2=dict(zip(names, (diff / den).tolist())),
                                   rel_l2_own_norm=dict(zip(names, (diff / ref).tolist())),
                                   note="relative L2 difference per conserved variable, headline form vs FP64 form; "
                                        "rel_l2 with the floors rho_l (rho, rho e, c) and rho_l/100 (momentum)")
        del c64, c32, u64, u32
        torch.cuda.synchronize()

    # --- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(args, make_ctx, dt, dof, stages, world, barrier, max_over_ranks)

    # --- the batched ensemble (256 independent 2D problems) on the same GPU
    batched = None
    if not args.no_batch:
        batched = batch_measure(WORKLOADS["c4"](), local_rank, max(3, args.steps // 2), 3, unbatched=True)
        if world > 1:  # one ensemble per rank: whole-job rate over the slowest rank
            bms = replica_max(batched["ms_per_step"] * batched["steps"], dist)
            stg = 5 if WORKLOADS["c4"]()["rk"] == 4 else 3
            batched = dict(batched, value=replica_rate(batched["nodes"] * stg * batched["steps"], world, bms),
                           ms_per_step=bms / batched["steps"], scope=f"{world} replicas")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = oracle_rate(wl, seconds_target=args.cpu_seconds, single_thread=True)
        cpu = dict(value=r["rate"], unit=UNIT, cores=r["cores"], kind="oracle",
                   sample=f"{r['steps']} RK steps on {r['sub']} of the workload ({r['dof']} nodes), "
                          f"{r['seconds']:.1f} s", single_thread_value=r["single"], cpu_model=cpu_model())

    if rank == 0:
        line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                    ms_per_step=ms_max / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                    dtype="f32/f64" if args.precision == "fp32bulk" else "f64", data="synthetic",
                    config=dict(workload=wl["name"], dof=dof, stages_per_step=stages, precision=args.precision,
                                l2=l2_note(dof * (m['dim'] + 3) * 8),
                                parallelism=f"replicas x{world}"),
                    e2e=e2e, gpu_launches=3 * stages * args.steps, roofline=roofline, cpu_baseline=cpu,
                    clocks=clk.summary(), fp64=fp64, batched=batched)
        print(json.dumps(line), flush=True)
    return 0


def batch_measure(wl, local_rank, steps, warmup, unbatched=True, e2e=False, name="c4"):
    """Batched ensemble: autotuned persistent launches per RK stage, timed over `steps`
    graph-replayed steps; beside it the same problems one context each (FP32-bulk and
    FP64, every context on its own stream so that small problems may overlap)."""
    import torch
    from paper_2208_05310_gb300 import dgk, inputs
    b = wl["batch"]
    stages = 5 if wl["rk"] == 4 else 3
    specs = inputs.ensemble_specs(b["nprob"], b["seed"], n_range=b["n_range"])
    meshes = [inputs.ensemble_mesh(sp) for sp in specs]
    thermo = {}

    def prim_of(q, sp):
        if sp["T"] not in thermo:
            rv, rl = dgk.maxwell(sp["T"])
            thermo[sp["T"]] = (rv, rl, dgk.interface_width(sp["T"], wl["params"]["cv"], wl["params"]["gammaK"]))
        return inputs.ensemble_primitive(q.node_coords(), sp, *thermo[sp["T"]])

    B = dgk.Batch(meshes, device=local_rank, rk=wl["rk"], **wl["params"])
    prims, dts = [], []
    for q, sp in zip(B.problems, specs):
        prims.append(prim_of(q, sp))
        q.set_primitive(prims[-1])
        dts.append(0.5 * q.max_dt(0.9, 0.4))
    B.set_dt(dts)
    dof_p = [q.nelem * q.np for q in B.problems]
    dof = sum(dof_p)
    t0 = time.perf_counter()
    cfg = B.autotune()
    t_tune = time.perf_counter() - t0
    B.run(warmup)
    B.status()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(B.stream)
    B.run(steps)
    e1.record(B.stream)
    B.stream.synchronize()
    ms = e0.elapsed_time(e1)
    B.status()
    alg = sum(d * sum(kernel_bytes_per_node(2, ms_["N"], 4).values()) for d, ms_ in zip(dof_p, meshes))
    peak, peak_kind = measured_peak()
    avg_launch_ms = ms / steps / stages
    achieved = alg / (avg_launch_ms / 1e3) / 1e9
    launches = stages * steps * (3 if cfg["form"] == "grouped" else 1)
    out = dict(value=dof * stages * steps / (ms / 1e3), unit=UNIT, ms_per_step=ms / steps, steps=steps,
               nodes=dof, problems=len(meshes), autotuned=cfg, autotune_s=t_tune, gpu_launches=launches,
               roofline=dict(bound="hbm",
                             kernel="k_batch_phase<0,1,2>" if cfg["form"] == "grouped" else "k_batch_stage",
                             achieved=achieved, peak=peak, unit="GB/s", frac=achieved / peak, peak_kind=peak_kind,
                             alg_bytes_per_launch=alg, avg_launch_ms=avg_launch_ms,
                             traffic=batch_traffic(name) if cfg["form"] == "grouped" else None,
                             note="per RK stage: one persistent launch, or the three grouped phase launches; "
                                  "time from the graph-replayed steps / stages"))
    if e2e:
        host_in = [torch.empty(q.shape(), dtype=torch.float64, pin_memory=True) for q in B.problems]
        host_out = [torch.empty(q.shape(), dtype=torch.float64, pin_memory=True) for q in B.problems]
        for q, h in zip(B.problems, host_in):
            q.download_state(h)
        k_e2e = max(1, min(steps, 5))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            for q, h in zip(B.problems, host_in):
                q.upload_state(h)
            B.run(1)
            for q, h in zip(B.problems, host_out):
                q.download_state(h)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        B.status()
        nbytes = sum(h.numel() * 8 for h in host_in)
        out["e2e"] = dict(value=dof * stages * k_e2e / t, unit=UNIT, h2d_bytes_per_step=nbytes,
                          d2h_bytes_per_step=nbytes, steps=k_e2e)
    B.close()
    del B
    torch.cuda.synchronize()
    if unbatched:
        for prec, k in (("fp32bulk", steps), ("fp64", max(1, steps // 4))):
            ctxs = []
            for ms_, prim in zip(meshes, prims):
                c = dgk.Context(device=local_rank)
                c.set_params(rk=wl["rk"], precision=prec, **wl["params"])
                c.mesh_box(2, ms_["N"], ms_["n"] + [1], ms_["lo"] + [0.0], ms_["hi"] + [1.0], ms_["periodic"] + [1],
                           ms_["walls"])
                c.set_primitive(prim)
                ctxs.append(c)
            for c, dt in zip(ctxs, dts):
                c.run(1, dt)  # warm-up, captures each context's step graph
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for c, dt in zip(ctxs, dts):
                c.run(k, dt)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            for c in ctxs:
                c.status()
                c.close()
            out["unbatched_" + prec] = dict(value=dof * stages * k / t, unit=UNIT, steps=k, ms_per_step=1e3 * t / k,
                                            launches_per_step=3 * stages * len(ctxs))
            torch.cuda.synchronize()
    return out


def run_batch(args, wl, rank, world, local_rank):
    """The batched-ensemble workload as the bench line (replicas under torchrun)."""
    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    if dist is not None:
        dist.barrier()
    with ClockSampler(local_rank) as clk:
        r = batch_measure(wl, local_rank, args.steps, args.warmup, unbatched=not args.no_fp64, e2e=not args.no_e2e,
                          name=args.workload)
    ms = replica_max(r["ms_per_step"] * args.steps, dist)
    stages = 5 if wl["rk"] == 4 else 3
    if rank == 0:
        e2e = r.pop("e2e", None)
        if e2e is not None:
            e2e = dict(e2e, value=e2e["value"] * world)
        line = dict(metric=METRIC, value=replica_rate(r["nodes"] * stages * args.steps, world, ms), unit=UNIT,
                    n_gpus=world, steps=args.steps, warmup=args.warmup, ms_per_step=ms / args.steps,
                    higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32/f64", data="synthetic",
                    config=dict(workload=wl["name"], dof=r["nodes"], problems=r["problems"], stages_per_step=stages,
                                precision="fp32bulk", autotuned=r["autotuned"],
                                l2=l2_note(r["nodes"] * 5 * 8),
                                parallelism=f"replicas x{world}"),
                    e2e=e2e, gpu_launches=r["gpu_launches"], roofline=r["roofline"], cpu_baseline=None,
                    clocks=clk.summary(), unbatched_fp32bulk=r.get("unbatched_fp32bulk"),
                    unbatched_fp64=r.get("unbatched_fp64"))
        print(json.dumps(line), flush=True)
    return 0


def end_to_end(args, make_ctx, dt, dof, stages, world, barrier, max_over_ranks):
    """K steps through the C ABI with pinned host buffers (dgk_run_host): each step
    uploads a state from host memory, runs one RK step and reads the result back; the
    host copies of the neighbouring steps overlap each step's kernels.  The plain
    sequence upload / run / download is timed beside it."""
    import torch
    ctx = make_ctx(args.precision)
    host_in = torch.empty(ctx.shape(), dtype=torch.float64, pin_memory=True)
    host_out = torch.empty(ctx.shape(), dtype=torch.float64, pin_memory=True)
    ctx.download_state(host_in)
    ctx.run_host([host_in], [host_out], 1, dt)
    ctx.status()
    k_e2e = max(2, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    ctx.run_host([host_in] * k_e2e, [host_out] * k_e2e, 1, dt)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(time.perf_counter() - t0)
    ctx.status()
    barrier()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        ctx.upload_state(host_in)
        ctx.run(1, dt)
        ctx.download_state(host_out)
    torch.cuda.synchronize()
    t_seq = max_over_ranks(time.perf_counter() - t0)
    ctx.status()
    nbytes = host_in.numel() * 8
    del ctx
    return dict(value=dof * stages * k_e2e * world / t_e2e, unit=UNIT, h2d_bytes_per_step=nbytes,
                d2h_bytes_per_step=nbytes, steps=k_e2e, api="dgk_run_host",
                sequential=dict(value=dof * stages * k_e2e * world / t_seq, api="dgk_upload_state, dgk_run, "
                                "dgk_download_state"))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c5", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32bulk", choices=["fp32bulk", "fp64"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--flux", default="rusanov", choices=["rusanov", "hllc"],
                    help="hllc runs the workload with relaxation model 2 and the HLLC flux")
    ap.add_argument("--model", type=int, default=None, choices=[0, 1, 2],
                    help="0: the original NSK model (the workload's walls become periodic)")
    ap.add_argument("--walls", default="noslip", choices=["noslip", "slip", "sliding", "slip-sliding"],
                    help="slip: generalized Navier-slip walls (gamma_1..4 = 1e-5, 0.1, 0.05, 1); sliding: the top "
                         "wall slides with u = (0.5, 0, 0), the wall velocity of the sliding-droplet case; "
                         "slip-sliding: the walls of that case (Navier slip below, the sliding no-slip wall above)")
    ap.add_argument("--mesh", default="box", choices=["box", "curved", "unstructured", "mortar"],
                    help="curved: the workload's box mapped to curved elements (degree-2 element maps of "
                         "x_k + 0.02 L_k sin(2 pi x_{k+1}/L_{k+1}); the walls are bent); unstructured: the same "
                         "curved mesh with every element in a random local frame, connected through tables; mortar: the "
                         "curved mesh at half the resolution with its upper half in x refined 2:1 (non-conforming faces)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--accuracy-steps", type=int, default=0,
                    help="steps after which the headline form is compared with the FP64 form (default: the FP64 "
                         "leg's own steps)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    wl = WORKLOADS[args.workload]()
    if (args.flux == "hllc" or args.model is not None or args.walls != "noslip") and "batch" in wl:
        print(json.dumps({"error": "the ensemble runs model 1, Rusanov, no-slip walls"}))
        return 2
    if args.flux == "hllc":
        wl["params"] = dict(wl["params"], model=2, flux="hllc")
        wl["name"] += ", model 2 + HLLC"
    if args.model is not None and args.flux != "hllc":
        wl["params"] = dict(wl["params"], model=args.model)
        if args.model == 0:
            wl["mesh"] = dict(wl["mesh"], periodic=[1] * wl["mesh"]["dim"], walls={})
            wl["name"] += ", original NSK model, periodic in every direction"
        else:
            wl["name"] += f", model {args.model}"
    if args.walls in ("slip", "slip-sliding") and wl["mesh"]["walls"]:
        # gamma_1 / gamma_K = 0.1: a hysteresis coupling of 200 (gamma_1 = 0.02) makes the
        # explicit step diverge on this mesh, in the oracle as well
        ws = wl["mesh"]["walls"]
        top = max(ws)
        wl["mesh"] = dict(wl["mesh"], walls={f: (Tw, th) + ((1e-5, 0.1, 0.05, 1.0) if args.walls == "slip" or f != top else ())
                                             for f, (Tw, th) in ws.items()})
        wl["name"] += ", Navier-slip walls" if args.walls == "slip" else ", Navier-slip bottom wall"
    if args.walls in ("sliding", "slip-sliding") and wl["mesh"]["walls"]:
        top = max(wl["mesh"]["walls"])
        wl["mesh"] = dict(wl["mesh"], walls=dict(wl["mesh"]["walls"]))
        wl["mesh"]["walls"][top] = tuple(wl["mesh"]["walls"][top][:2]) + ((0.5, 0.0, 0.0),)
        wl["name"] += ", top wall sliding with u = (0.5, 0, 0)"
    if args.mesh in ("curved", "unstructured", "mortar"):
        if "batch" in wl:
            print(json.dumps({"error": "curved elements: single problems"}))
            return 2
        wl["geometry"] = dict(CURVED_GEOMETRY)
        wl["name"] += ", curved elements (degree-2 maps, walls bent by 2% of the height)"
        if args.mesh == "unstructured":
            wl["reorient"] = 2208
            wl["name"] += ", unstructured connectivity (every element in a random local frame)"
        if args.mesh == "mortar":
            wl["refine"] = True
            wl["mesh"] = dict(wl["mesh"], n=[v // 2 for v in wl["mesh"]["n"]])
            wl["name"] += ", half resolution with the upper half in x refined 2:1 (mortars)"
    if args.impl == "reference":
        return run_reference(args, wl, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        if "batch" in wl:
            return run_batch(args, wl, rank, world, local_rank)
        return run_ours(args, wl, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())

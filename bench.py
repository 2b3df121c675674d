"""Benchmark of the coupled LBM-IBM time step on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                [--workload channel|shear|vessel|pipe]

Default workload: the largest configuration, a voxelised straight vessel
of 100 um diameter and 500 um length (lattice 1000 x 208 x 208 at dx = 0.5
um, 31.4 M fluid nodes, periodic ends, body-force driven) with 19,600 red
cells of 642 vertices (12.6 M vertices, ~45 % haematocrit), populations
stored as FP32 deviations; the same workload with FP16 and BF16 storage is
measured alongside.  `--workload channel` runs the 64 x 64 x 256 channel
with 440 red cells instead.  One step = the whole coupled step (membrane
forces, binning, spreading, collide + stream, velocity, interpolation +
move).  Prints one JSON line on rank 0.  Under torchrun every rank runs an
independent replica (the method is not sharded: replicas only) and rank 0
reports the whole-job rate.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2305_02752_gb300 import inputs as I  # noqa: E402

METRIC = 'coupled LBM-IBM MLUPS & RBC vertices/s; 16-bit/FP32 vs FP64 at fixed error'
UNIT = 'MLUPS'
FLUSH_BYTES = 256 << 20   # > 129 MB L2


def make_workload(name):
    if name == 'channel':
        cfg = I.channel()
        desc = 'channel 64x64x256 (walls y=0,63), 440 RBC x 642 vertices, FP32 deviations'
    elif name == 'shear':
        cfg = I.shear_cell()
        desc = 'shear box 32^3, 1 RBC x 642 vertices, FP64'
    elif name == 'vessel':
        cfg = I.channel(nx=128, ny=128, nz=512, ncell=4460, seed=20230502, steps=200, platelet_ratio=0.1,
                        name='vessel', pack_iter=60, exact_iter=0)
        desc = 'channel 128x128x512 (walls y=0,127), 4460 RBC + 446 platelets, 16-bit deviations'
    elif name == 'pipe':
        cfg = I.pipe()
        desc = 'pipe 1000x208x208 (radius 100, periodic in x), 19600 RBC x 642 vertices'
    else:
        raise SystemExit(f'unknown workload {name}')
    return cfg, desc


def default_precision(name):
    return {'channel': 'f32', 'shear': 'f64', 'vessel': 'bf16', 'pipe': 'f32'}[name]


def workload_config(cfg, desc, world):
    """The `config` object of the JSON line; both arms print the same one."""
    return {'workload': desc, 'lattice': [cfg.nx, cfg.ny, cfg.nz], 'fluid_nodes': cfg.n_fluid,
            'cells': len(cfg.centers), 'vertices': cfg.n_vertices,
            'parallelism': 'replicas' if world > 1 else 'single',
            'l2': f'flushed before every timed step ({FLUSH_BYTES >> 20} MiB write, then a {FLUSH_BYTES >> 20} MiB read)',
            'seed': cfg.seed, 'placement': cfg.note}


def bytes_per_node(precision):
    """Algorithmic DRAM bytes of the collide+stream kernel per fluid node:
    19 populations read + 19 written (38 S) plus the force density read."""
    S = {'f64': 8, 'f32': 4, 'f16': 2, 'bf16': 2}[precision]
    rs = 8 if precision == 'f64' else 4
    return 38 * S + 3 * rs


def hbm_peak():
    path = os.path.join(ROOT, 'MEASURED_PEAKS.json')
    try:
        with open(path) as f:
            return float(json.load(f)['hbm_gbs']), 'measured'
    except Exception:
        return 6800.0, 'fallback'


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while running."""

    FIELDS = ['index', 'clocks.sm', 'clocks.max.sm', 'power.draw', 'clocks_event_reasons.active',
              'clocks_event_reasons.hw_slowdown', 'clocks_event_reasons.hw_thermal_slowdown',
              'clocks_event_reasons.sw_thermal_slowdown', 'clocks_event_reasons.sw_power_cap']

    def __init__(self, device_index):
        fd, self.path = tempfile.mkstemp(prefix='clocks_', suffix='.csv')
        os.close(fd)
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.fh = open(self.path, 'w')
            self.proc = subprocess.Popen(['nvidia-smi', f'--query-gpu={",".join(self.FIELDS)}',
                                          '--format=csv,noheader,nounits', '-lms', '50', '-i', str(self.dev)],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(1.0)
        except Exception:
            self.proc = None
        self.t0 = None

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.proc is None:
            if os.path.exists(self.path):
                os.unlink(self.path)
            return self.summarise([])
        time.sleep(0.2)
        self.proc.terminate()
        self.proc.wait()
        self.fh.close()
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        return self.summarise(lines)

    @classmethod
    def summarise(cls, lines):
        """Median and largest SM clock and the throttle reasons seen active
        in `nvidia-smi --format=csv,noheader,nounits` lines of FIELDS
        (incomplete lines and non-numeric clocks are skipped)."""
        rows = []
        for line in lines:
            p = [x.strip() for x in line.split(',')]
            if len(p) == len(cls.FIELDS):
                rows.append(p)
        sm = [float(r[1]) for r in rows if r[1].replace('.', '').isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace('.', '').isdigit()]
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith('active')})
        return {'sm_mhz': statistics.median(sm) if sm else None, 'sm_max_mhz': max(mx) if mx else None,
                'reasons': reasons, 'samples': len(rows)}


class L2Flush:
    """Evicts the lattice from L2 between timed steps: writes a buffer
    larger than L2, then reads a second one so that the written lines are
    back in DRAM (clean) before the next timed step starts."""

    def __init__(self, torch):
        self.w = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device='cuda')
        self.r = torch.ones(FLUSH_BYTES // 4, dtype=torch.float32, device='cuda')
        self.sink = torch.empty(1, dtype=torch.float32, device='cuda')

    def __call__(self):
        self.w.zero_()
        self.sink.copy_(self.r.sum().reshape(1))


PHASE_STEPS = 50  # steps of the event-instrumented pass
PHASE_MARKS = 7   # event nodes per step graph with phase timing


def timed_steps(sim, torch, steps, flush, phase_every=5):
    """Run `steps` steps, each bracketed by CUDA events on the simulation's
    stream with an L2 flush before it; returns (total ms, per-phase ms
    averaged over the steps sampled every `phase_every` steps (0: none; the
    simulation must have phase timing on otherwise), kernels per step)."""
    st = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    phase_sum, nphase, kps = None, 0, 0
    for k in range(steps):
        flush()
        evs[k][0].record(st)
        sim.step(1)
        evs[k][1].record(st)
        if phase_every and (k % phase_every == phase_every - 1 or k == steps - 1):
            ph, kps = sim.phase_times()
            phase_sum = ph if phase_sum is None else {a: phase_sum[a] + ph[a] for a in ph}
            nphase += 1
    torch.cuda.synchronize()
    total = sum(a.elapsed_time(b) for a, b in evs)
    phases = {a: b / nphase for a, b in phase_sum.items()} if phase_sum else {}
    return total, phases, kps


def run_form(cfg, precision, warmup, steps, torch, flush, u_ref=None):
    from paper_2305_02752_gb300 import hemo
    sim = hemo.Simulation.from_config(cfg, precision)
    sim.step(warmup)
    sim.sync()
    total, _, _ = timed_steps(sim, torch, steps, flush, phase_every=0)
    out = sim.get_fields(hemo.HEMO_U)
    sim.set_phase_timing(True)
    sim.step(2)
    _, phases, kps = timed_steps(sim, torch, 20, flush, phase_every=1)
    sim.close()
    nf = cfg.n_fluid
    coll = phases.get('collide')
    peak, _ = hbm_peak()
    res = {'mlups': nf * steps / (total * 1e-3) / 1e6, 'ms_per_step': total / steps,
           'collide_ms': coll, 'phase_ms': phases,
           # the collision phase (both step parities) against the measured
           # copy bandwidth, at the form's algorithmic bytes per fluid node
           'collide_hbm_frac': nf * bytes_per_node(precision) / (coll * 1e-3) / 1e9 / peak if coll else None}
    u = out['u'].astype(np.float64)
    if u_ref is not None:
        res['u_rel_l2_vs_f64'] = float(np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref))
    return res, u


# (force_every, integrator, adaptive tolerance or None)
TIME_SCALES = [(1, 'euler', None), (2, 'euler', None), (4, 'euler', None), (4, 'ab2', None), (10, 'ab2', None),
               (10, 'ab2', 0.05), (10, 'ab2', 0.1)]


def time_scales(cfg, precision, warmup, steps, torch, flush):
    """Time-scale separation (membrane forces every N steps, held in
    between, or adaptively: when a vertex moved more than the tolerance since
    the last evaluation, at most N steps apart) and the vertex integrator:
    throughput of the same workload per setting, and the velocity and vertex
    drift after warmup + steps steps relative to forces every step with
    Euler."""
    from paper_2305_02752_gb300 import hemo
    out, ref = [], None
    for n, integ, tol in TIME_SCALES:
        sim = hemo.Simulation.from_config(cfg, precision)
        sim.set_time_scales(n, integ)
        if tol is not None:
            sim.set_force_tolerance(tol)
        sim.step(warmup)
        sim.sync()
        evals0 = sim.force_evaluations
        total, _, _ = timed_steps(sim, torch, steps, flush, phase_every=0)
        f = sim.get_fields(hemo.HEMO_U | hemo.HEMO_VERTS)
        evals = sim.force_evaluations - evals0
        sim.close()
        u, X = f['u'].astype(np.float64), f['X']
        r = {'force_every': n, 'integrator': integ, 'force_tolerance': tol,
             'mlups': cfg.n_fluid * steps / (total * 1e-3) / 1e6, 'ms_per_step': total / steps,
             'force_evaluations_timed': evals}
        if ref is None:
            ref = (u, X)
        else:
            r['u_rel_l2_vs_every_step'] = float(np.linalg.norm(u - ref[0]) / np.linalg.norm(ref[0]))
            r['X_max_abs_diff_vs_every_step'] = float(np.abs(X - ref[1]).max())
        out.append(r)
    return {'precision': precision, 'steps': warmup + steps, 'timed_steps': steps, 'results': out}


def model_variants(cfg, precision, warmup, steps, torch, flush):
    """Throughput of the same workload with the optional model terms on: the
    internal viscosity (ratio 5, cytosol against plasma) and the
    large-deformation membrane terms (theta_m = 0.5, k_local = 0.05)."""
    import dataclasses
    from paper_2305_02752_gb300 import hemo
    out = []
    nl = dataclasses.replace(cfg, meshes=[dataclasses.replace(mt, theta_m=0.5, k_local=0.05) for mt in cfg.meshes])
    for name, c, ratio in (('plain', cfg, 1.0), ('internal viscosity ratio 5', cfg, 5.0),
                           ('nonlinear bending and local area', nl, 1.0)):
        sim = hemo.Simulation.from_config(c, precision)
        sim.set_viscosity_ratio(ratio)
        sim.step(warmup)
        sim.sync()
        total, _, _ = timed_steps(sim, torch, steps, flush, phase_every=0)
        sim.close()
        out.append({'variant': name, 'mlups': cfg.n_fluid * steps / (total * 1e-3) / 1e6, 'ms_per_step': total / steps})
    return {'precision': precision, 'timed_steps': steps, 'results': out}


def lees_edwards_cost(torch, flush, steps=200, warmup=10):
    """The shear workload of the differentiation form (48^3, 4 red cells,
    FP32) with its moving walls, and the same cells in a wall-free box with
    the Lees-Edwards boundary (image velocity 0.02, the walls' velocity
    difference): fluid-node updates per second of each."""
    import dataclasses
    from paper_2305_02752_gb300 import hemo
    cfg = I.shear_cell(n=48, ncell=4, seed=20230503, steps=steps)
    le = dataclasses.replace(cfg, mask=None, periodic=(1, 1, 1), wall_velocity=np.zeros((2, 3)))
    out = []
    for name, c in (('moving walls', cfg), ('Lees-Edwards', le)):
        sim = hemo.Simulation.from_config(c, 'f32')
        if c is le:
            sim.set_lees_edwards(0.02)
        sim.step(warmup)
        sim.sync()
        total, _, _ = timed_steps(sim, torch, steps, flush, phase_every=0)
        sim.close()
        out.append({'boundary': name, 'mlups': c.n_fluid * steps / (total * 1e-3) / 1e6, 'ms_per_step': total / steps})
    return {'workload': 'shear 48^3, 4 RBC x 642 vertices, FP32', 'timed_steps': steps, 'results': out}


def adjoint_cost(torch, steps=200, every=100):
    """Differentiation form on the 48^3 shear box with 4 red cells: device
    time per recorded forward step and per step of the reverse sweep
    (hemo_backward: checkpoint recomputation + adjoint), FP64 and FP32."""
    from paper_2305_02752_gb300 import hemo
    cfg = I.shear_cell(n=48, ncell=4, seed=20230503, steps=steps)
    out = {'workload': 'shear 48^3, 4 RBC x 642 vertices', 'steps': steps, 'checkpoint_every': every}
    st = torch.cuda.current_stream()
    for prec in ('f64', 'f32'):
        sim = hemo.Simulation.from_config(cfg, prec)
        sim.step(2)
        sim.sync()
        sim.record(every)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(st)
        sim.step(steps)
        e1.record(st)
        L, dL = sim.deformation_loss()
        e1b = torch.cuda.Event(enable_timing=True)
        e1b.record(st)
        g = sim.backward(dL)
        e2.record(st)
        torch.cuda.synchronize()
        fwd = e0.elapsed_time(e1) / steps
        bwd = e1b.elapsed_time(e2) / steps
        sim.close()
        out[prec] = {'forward_ms_per_step': fwd, 'backward_ms_per_step': bwd, 'ratio': bwd / fwd,
                     'loss': L, 'grad': [float(x) for x in g]}
    return out


def cpu_baseline(cfg, budget_s=15.0, threads=1):
    """The CPU oracle as it stands, on `threads` threads (its loops over
    independent nodes, cells and vertices), on a bounded number of steps of
    the same workload: one untimed step, then as many as fit the budget;
    when one step alone takes more than half the budget, that first step is
    the sample."""
    import oracle as O
    used = O.set_threads(threads)
    s = O.from_config(cfg)
    t0 = time.perf_counter()
    s.step(1)
    t1 = time.perf_counter() - t0
    if t1 > 0.5 * budget_s:
        n, dt, how = 1, t1, 'the first full-lattice oracle step'
    else:
        n = int(max(1, min(20, budget_s / max(t1, 1e-3) - 1)))
        t0 = time.perf_counter()
        s.step(n)
        dt = time.perf_counter() - t0
        how = f'{n} full-lattice oracle steps (after 1 untimed)'
    s.close()
    O.set_threads(1)
    what = 'one thread' if used == 1 else f'{used} OpenMP threads'
    return {'value': cfg.n_fluid * n / dt / 1e6, 'unit': UNIT, 'cores': used, 'kind': 'oracle',
            'sample': f'{how} of the same workload, FP64, {what}',
            'vertices_per_s': cfg.n_vertices * n / dt}


def e2e_job(cfg, precision, torch):
    """The whole job through the public C ABI from pinned host buffers:
    create the lattice (wall mask), set the initial velocity, add the cells,
    run the configuration's steps reading the per-cell statistics back to
    host after every step, read the final velocity field and vertices back,
    destroy."""
    from paper_2305_02752_gb300 import hemo
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
    mask = pin(cfg.mask.astype(np.uint8)) if cfg.mask is not None else None
    u0 = pin(cfg.init_velocity) if cfg.init_velocity is not None else None
    meshes = [(pin(m.rest), pin(m.tri.astype(np.int32))) for m in cfg.meshes]
    centers = pin(cfg.centers)
    rots = pin(cfg.rotations)
    nc = len(cfg.centers)
    stats = pin(np.zeros((nc, 6)))
    u_out = pin(np.zeros((cfg.nz, cfg.ny, cfg.nx, 3), np.float64 if precision == 'f64' else np.float32))
    X_out = pin(np.zeros((cfg.n_vertices, 3)))
    steps = cfg.steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim = hemo.Simulation(cfg.nx, cfg.ny, cfg.nz, cfg.tau, precision, cfg.periodic, mask, cfg.wall_velocity,
                          cfg.body_force)
    if u0 is not None:
        sim.set_velocity(u0)
    types = np.asarray(cfg.cell_type)
    for t in range(len(cfg.meshes)):
        idx = np.where(types == t)[0]
        if len(idx):
            mt = cfg.meshes[t]
            mt2 = I.MeshType(mt.name, meshes[t][0], meshes[t][1], mt.k_link, mt.k_bend, mt.k_area, mt.k_volume,
                             mt.kbt, mt.persistence, mt.max_strain)
            sim.add_cells(mt2, centers[idx], rots[idx])
    for _ in range(steps):
        sim.step(1)
        sim.get_fields(hemo.HEMO_CELLSTATS, out={'cellstats': stats})
    sim.get_fields(hemo.HEMO_U | hemo.HEMO_VERTS, out={'u': u_out, 'X': X_out})
    sim.close()
    dt = time.perf_counter() - t0
    h2d = mask.nbytes if mask is not None else 0
    h2d += (u0.nbytes if u0 is not None else 0) + centers.nbytes + rots.nbytes
    h2d += sum(a.nbytes + b.nbytes for a, b in meshes)
    d2h = stats.nbytes * steps + u_out.nbytes + X_out.nbytes
    return {'value': cfg.n_fluid * steps / dt / 1e6, 'unit': UNIT, 'h2d_bytes_per_step': int(h2d // steps),
            'd2h_bytes_per_step': int(d2h // steps), 'steps': steps,
            'note': 'whole job from pinned host inputs: create, set velocity, add cells, steps each followed by a '
                    'per-cell statistics read-back, final field read-back, destroy'}


def traffic_from_profile(precision, workload):
    """DRAM bytes per collide launch from the committed ncu summary, if the
    kernel source has not changed since it was captured."""
    path = os.path.join(ROOT, 'profiles', f'collide_{precision}_{workload}.json')
    if not os.path.exists(path):
        return None
    try:
        with open(path) as f:
            prof = json.load(f)
        csrc = os.path.join(ROOT, 'paper_2305_02752_gb300', 'csrc')
        src = b''.join(open(os.path.join(csrc, f), 'rb').read() for f in ('k_lattice.cu', 'lattice_core.cuh'))
        if prof.get('source_sha256') != hashlib.sha256(src).hexdigest():
            return None
        return prof.get('dram_bytes_per_launch')
    except Exception:
        return None


def max_over_ranks(torch, dist, value, device):
    """The largest value over the ranks (a replicated job takes as long as
    its slowest rank); dist None: the value itself."""
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, secs):
    """Whole-job rate in millions of units per second: every rank processes
    its own replica, the job's time is the slowest rank's."""
    return world * units_per_rank / secs / 1e6


def reference_arm(args, rank, world):
    if rank != 0:
        return
    cfg, desc = make_workload(args.workload)
    import oracle as O
    cores = O.set_threads(os.cpu_count() or 1)
    s = O.from_config(cfg)
    t0 = time.perf_counter()
    s.step(1)
    t1 = time.perf_counter() - t0
    budget = 100.0
    w = min(args.warmup, max(0, int(budget * 0.2 / t1)))
    k = max(1, min(args.steps, int(budget / t1)))
    s.step(max(0, w - 1))
    t0 = time.perf_counter()
    s.step(k)
    dt = time.perf_counter() - t0
    s.close()
    value = cfg.n_fluid * k / dt / 1e6
    sample = (f'{k} of the requested {args.steps} timed steps (after {w} warm-up) of the full workload, '
              f'FP64 CPU oracle, {cores} OpenMP thread(s) over its independent loops')
    line = {'impl': 'reference', 'metric': METRIC, 'value': value, 'unit': UNIT, 'n_gpus': world,
            'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': dt / k * 1e3, 'higher_is_better': True,
            'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic',
            'config': workload_config(cfg, desc, world),
            'cpu_baseline': {'value': value, 'unit': UNIT, 'cores': cores, 'kind': 'oracle', 'sample': sample},
            'e2e': {'value': value, 'unit': UNIT, 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0},
            'vertices_per_s': cfg.n_vertices * k / dt}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=2000)
    ap.add_argument('--warmup', type=int, default=20)
    ap.add_argument('--impl', default='gb300', choices=['gb300', 'reference'])
    ap.add_argument('--workload', default='pipe', choices=['channel', 'shear', 'vessel', 'pipe'])
    ap.add_argument('--precision', default=None, choices=['f64', 'f32', 'f16', 'bf16'])
    ap.add_argument('--no-forms', action='store_true')
    ap.add_argument('--no-cpu', action='store_true')
    ap.add_argument('--no-e2e', action='store_true')
    ap.add_argument('--no-adjoint', action='store_true')
    ap.add_argument('--extras', action='store_true',
                    help='also measure the optional model terms on the 64x64x256 channel (time-scale '
                         'separation, internal viscosity, large-deformation terms, Lees-Edwards boundary)')
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    if args.impl == 'reference':
        return reference_arm(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl', device_id=torch.device('cuda', local))
    from paper_2305_02752_gb300 import hemo

    precision = args.precision or default_precision(args.workload)
    cfg, desc = make_workload(args.workload)
    flush = L2Flush(torch)
    sim = hemo.Simulation.from_config(cfg, precision)
    staged = sim.lattice_plan()[0] > 0  # 16-bit storage on long rows: the staged collision
    sim.step(args.warmup)
    sim.sync()
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # headline pass: the plain step graphs (event nodes inside the graph cost
    # a few microseconds each, so they stay out of this pass)
    total_ms, _, _ = timed_steps(sim, torch, args.steps, flush, phase_every=0)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop() if rank == 0 else None
    # kernel durations: a second timed pass whose step graphs carry an event
    # node at every phase boundary, read after every step (both parities)
    sim.set_phase_timing(True)
    sim.step(2)
    ptotal, phases, kps = timed_steps(sim, torch, PHASE_STEPS, flush, phase_every=1)
    sim.sync()
    sim.close()
    total_ms = max_over_ranks(torch, dist, total_ms, 'cuda')
    if rank != 0:
        dist.destroy_process_group()
        return

    nf, nv = cfg.n_fluid, cfg.n_vertices
    secs = total_ms * 1e-3
    value = job_rate(nf * args.steps, world, secs)
    peak, peak_kind = hbm_peak()
    bpn = bytes_per_node(precision)
    coll = phases.get('collide')
    achieved = nf * bpn / (coll * 1e-3) / 1e9 if coll else None
    line = {
        'metric': METRIC, 'value': value, 'unit': UNIT, 'n_gpus': world, 'steps': args.steps,
        'warmup': args.warmup, 'ms_per_step': total_ms / args.steps, 'higher_is_better': True,
        'scaling': 'weak', 'vs_baseline': None, 'dtype': precision, 'data': 'synthetic',
        'config': workload_config(cfg, desc, world),
        'vertices_per_s': world * nv * args.steps / secs,
        'phase_ms': phases,
        'phase_pass': {'steps': PHASE_STEPS, 'ms_per_step': ptotal / PHASE_STEPS,
                       'event_overhead_us_per_boundary': 1e3 * (ptotal / PHASE_STEPS - total_ms / args.steps) / PHASE_MARKS,
                       'note': 'phase and kernel times from event nodes in the step graph over a second timed pass; '
                               'each phase includes the overhead of one event boundary'},
        'roofline': {'bound': 'hbm', 'kernel': 'collide_tiles + collide_erows' if staged else 'collide_stream',
                     'achieved': achieved, 'peak': peak,
                     'unit': 'GB/s', 'frac': (achieved / peak) if achieved else None,
                     'traffic': traffic_from_profile(precision, args.workload),
                     'algorithmic_bytes_per_launch': nf * bpn, 'peak_kind': f'{peak_kind} HBM copy bandwidth'},
        'gpu_launches': kps * args.steps,
        'clocks': clk,
    }
    forms = None
    if not args.no_forms and args.workload != 'shear':
        # the same workload and seed with every storage form: throughput and
        # velocity error against the FP64 run after the same steps
        fsteps = min(args.steps, 200)
        res = {}
        r64, u64 = run_form(cfg, 'f64', args.warmup, fsteps, torch, flush)
        res['f64'] = r64
        for p in ('f32', 'f16', 'bf16'):
            res[p], _ = run_form(cfg, p, args.warmup, fsteps, torch, flush, u_ref=u64)
        forms = {'steps': args.warmup + fsteps, 'timed_steps': fsteps, 'results': res,
                 'summary': {p: {'mlups': res[p]['mlups'], 'vs_f32': res[p]['mlups'] / res['f32']['mlups'],
                                 'u_rel_l2_vs_f64': res[p].get('u_rel_l2_vs_f64'),
                                 'collide_hbm_frac': res[p]['collide_hbm_frac']} for p in ('f32', 'f16', 'bf16')}}
    if args.extras:
        ccfg, _ = make_workload('channel')
        line['extras_workload'] = 'channel 64x64x256, 440 RBC, FP32'
        line['time_scales'] = time_scales(ccfg, 'f32', args.warmup, min(args.steps, 200), torch, flush)
        line['model_variants'] = model_variants(ccfg, 'f32', args.warmup, min(args.steps, 200), torch, flush)
        line['lees_edwards'] = lees_edwards_cost(torch, flush, steps=min(args.steps, 200))
    if not args.no_adjoint:
        line['adjoint'] = adjoint_cost(torch)
    if not args.no_e2e:
        line['e2e'] = e2e_job(cfg, precision, torch)
    if not args.no_cpu:
        # all host cores (OpenMP over the oracle's independent loops); one
        # thread on the small channel only, where it fits the budget
        line['cpu_baseline'] = cpu_baseline(cfg, budget_s=20.0, threads=os.cpu_count() or 1)
        if cfg.n_nodes <= 4_000_000:
            line['cpu_baseline_one_core'] = cpu_baseline(cfg)
    if forms is not None:  # last, so that the end of the line carries the storage-form comparison
        line['forms'] = forms
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == '__main__':
    main()

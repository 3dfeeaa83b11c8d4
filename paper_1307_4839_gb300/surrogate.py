"""The learned surrogate around the solver: data, training and the checked
rollout (host orchestration of libswof's kernels).

Training data come from the solver's own trajectories.  Rainfall-runoff
hillslopes (rain, Manning friction, Green-Ampt infiltration, Sec. 3.5) are
stepped on the fine grid in fixed-dt mode, so a span of `span_steps` steps
is a fixed time and every step's dt is checked against Eq. (cfl).  Every
span the state is coarsened on the device by f x f block means
(swof_coarsen).  A coarse member is one sample of IN_CH channels:

    0 h, 1 hu, 2 hv, 3 V_inf         the state (the network's output too)
    4 rain rate averaged over the coming span [m/s]
    5 dz/dx, 6 dz/dy                 bed slopes of the coarse bed
    7 K_s                            coarse saturated conductivity [m/s]

The network (UNet) maps a sample to its state one span later; the rollout
(swof_surrogate_rollout) checks every prediction for positivity and mass
balance and falls back, member by member, to the plain solver on the
coarse grid.  All arithmetic of the path runs in libswof's kernels; this
module allocates device buffers, fills the constant channels, assembles
batches by indexing and loops.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import FP32, FRIC_MANNING, Solver, UNet, coarsen_static, rollout as _rollout

IN_CH, OUT_CH = 8, 4
CH_RAIN, CH_ZX, CH_ZY, CH_KS = 4, 5, 6, 7


def block_mean(a: np.ndarray, f: int) -> np.ndarray:
    ny, nx = a.shape
    return a.reshape(ny // f, f, nx // f, f).mean(axis=(1, 3))


def span_rain(rate: float, t_on: float, t_off: float, t0: float, span: float, n: int) -> float:
    """Rain rate averaged over the n steps of length span / n from t0: the
    solver adds rain in a step that starts in [t_on, t_off).  (Scenarios put
    t_off half a step off the step grid so the count is not a rounding tie.)"""
    c = sum(1 for j in range(n) if t_on <= t0 + j * (span / n) < t_off)
    return rate * c / n


def outflow_mask(bc) -> int:
    """Bits 1 W, 2 E, 4 S, 8 N of the outflow edges."""
    return sum(1 << k for k in range(4) if bc[k] == 1)


@dataclass
class Trajectory:
    work: object          # the fine scenario (swof_inputs.Workload)
    f: int                # coarsening factor
    dt: float             # fixed fine dt
    span_steps: int       # fine steps per span
    times: np.ndarray     # time of each snapshot
    z_c: np.ndarray       # coarse bed (block mean)
    ks_c: np.ndarray      # coarse K_s (block mean)

    @property
    def span(self) -> float:
        return self.dt * self.span_steps

    @property
    def dx(self) -> float:
        return self.work.dx * self.f

    @property
    def rain(self):
        w = self.work
        return (w.rain_rate, w.rain_t_on, w.rain_t_off)


class Dataset:
    """Coarse snapshots of fine trajectories: data [traj][snapshot][IN_CH]
    [Hc][Wc] (float32 CUDA); snapshot k is the state after k spans."""

    def __init__(self, data, trajs):
        self.data = data
        self.trajs = trajs
        self.n_traj, self.n_snap = data.shape[0], data.shape[1]
        self.flat = data.view(self.n_traj * self.n_snap, *data.shape[2:])

    def index(self, traj: int, k: int) -> int:
        return traj * self.n_snap + k

    def pairs(self, trajs=None) -> np.ndarray:
        """Flat indices of the inputs of all (snapshot, next snapshot) pairs."""
        trajs = range(self.n_traj) if trajs is None else trajs
        return np.array([self.index(i, k) for i in trajs for k in range(self.n_snap - 1)], dtype=np.int64)


def generate(works, f: int, dt: float, span_steps: int, n_spans: int, precision=FP32) -> Dataset:
    """Run every fine scenario for n_spans spans of span_steps fixed steps
    (Eq. (cfl) checked each step; a violation raises) and store the coarse
    snapshots.  The solvers run concurrently, one CUDA stream each."""
    import torch
    ny, nx = works[0].ny, works[0].nx
    if any(w.nx != nx or w.ny != ny for w in works) or nx % f or ny % f:
        raise ValueError("scenarios must share a grid divisible by f")
    Hc, Wc = ny // f, nx // f
    data = torch.zeros((len(works), n_spans + 1, IN_CH, Hc, Wc), dtype=torch.float32, device="cuda")
    trajs, solvers, streams = [], [], []
    span = dt * span_steps
    times = np.arange(n_spans + 1) * span
    for i, w in enumerate(works):
        # the static channels (bed slopes, K_s) on the device, every snapshot
        zd = torch.from_numpy(np.ascontiguousarray(w.z, dtype=np.float64)).to("cuda")
        ksd = (torch.from_numpy(np.ascontiguousarray(w.ks, dtype=np.float64)).to("cuda")
               if isinstance(w.ks, np.ndarray) else None)
        ks_const = 0.0 if isinstance(w.ks, np.ndarray) else float(w.ks)
        coarsen_static(zd, ksd, w.dx, w.dy, f, data[i, 0, CH_ZX], IN_CH * Hc * Wc, n_spans + 1, ks_const=ks_const)
        # the coarse bed and K_s the fallback solver runs on (host; its topography and map)
        z_c = block_mean(w.z, f)
        ks = w.ks if isinstance(w.ks, np.ndarray) else np.full((ny, nx), float(w.ks))
        ks_c = block_mean(ks, f)
        for k in range(n_spans + 1):
            data[i, k, CH_RAIN] = span_rain(w.rain_rate, w.rain_t_on, w.rain_t_off, times[k], span, span_steps)
        trajs.append(Trajectory(w, f, dt, span_steps, times, z_c, ks_c))
        st = torch.cuda.Stream()
        streams.append(st)
        solvers.append(Solver.from_workload(w, precision=precision, dt_fixed=dt, t_end=1e30,
                                            stream=st.cuda_stream))
    torch.cuda.synchronize()
    for s in solvers:
        s.use_graph(True)
    for k in range(n_spans + 1):
        for i, s in enumerate(solvers):
            if k:
                s.step(span_steps, sync=False)
            s.coarsen(f, data[i, k])
    for s in solvers:
        s.diagnostics()           # synchronises; raises on a latched error (e.g. SWOF_ECFL)
        s.close()
    torch.cuda.synchronize()
    return Dataset(data, trajs)


def fit_norm(ds: Dataset, pairs: np.ndarray, sample: int = 256, seed: int = 0):
    """Per-channel input mean / scale and output (increment) scale from a
    host sample of the training pairs.  h, hu and hv are scaled about 0 (by
    their RMS), so small depths and discharges keep their relative
    precision in the network's bf16 inputs."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(pairs, size=min(sample, len(pairs)), replace=False)
    x = ds.flat[idx].double().cpu().numpy()
    y = ds.flat[idx + 1][:, :OUT_CH].double().cpu().numpy()
    mean = x.mean(axis=(0, 2, 3))
    std = x.std(axis=(0, 2, 3))
    mean[:3] = 0.0
    std[:3] = np.sqrt((x[:, :3] ** 2).mean(axis=(0, 2, 3)))
    scale_in = np.where(std > 0, std, np.maximum(np.abs(mean), 1.0))
    inc = (y - x[:, :OUT_CH]).std(axis=(0, 2, 3))
    scale_out = np.where(inc > 0, inc, 1.0)
    return mean, scale_in, scale_out


def train(net: UNet, ds: Dataset, pairs: np.ndarray, steps: int, batch: int, lr: float = 2e-3,
          lr_min: float = 1e-5, weight_decay: float = 0.0, seed: int = 0, stream=None):
    """AdamW on random batches of (sample, next state) pairs with a cosine
    learning-rate decay; returns the per-step sums of squared errors."""
    import torch
    rng = np.random.default_rng(seed)
    losses = []
    order = rng.permutation(pairs)
    pos = 0
    for s in range(steps):
        if pos + batch > len(order):
            order, pos = rng.permutation(pairs), 0
        idx = torch.from_numpy(order[pos:pos + batch]).to("cuda")
        pos += batch
        x = ds.flat.index_select(0, idx)
        y = ds.flat.index_select(0, idx + 1)[:, :OUT_CH].contiguous()
        lr_s = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * s / max(steps - 1, 1)))
        losses.append(net.train_step(x, y, lr_s, weight_decay, stream))
    return np.array(losses)


def coarse_solver(traj: Trajectory, steps: int, precision=FP32, stream=None) -> Solver:
    """The plain solver on the coarse grid of a trajectory (its fallback and
    the method without the surrogate), fixed dt = span / steps."""
    w = traj.work
    Hc, Wc = traj.z_c.shape
    return Solver(Wc, Hc, traj.dx, traj.dx, traj.z_c, precision=precision, cfl=w.cfl, h_dry=w.h_dry,
                  dt_max=w.dt_max, t_end=1e30, bc=w.bc, friction=w.friction, manning_n=w.manning_n,
                  rain_rate=w.rain_rate, rain_t_on=w.rain_t_on, rain_t_off=w.rain_t_off,
                  infiltration=w.infiltration, ks_map=traj.ks_c, psi=w.psi, dtheta=w.dtheta,
                  dt_fixed=traj.span / steps, stream=stream)


class Rollout:
    """Members (trajectory, start snapshot) of a Dataset rolled forward by
    the network with the checked fallback; states [B][IN_CH][Hc][Wc].
    Each trajectory gets a pool of up to `pool` coarse solvers (own CUDA
    streams, CUDA graphs) that its failing members share round-robin, so
    fallbacks of different members run concurrently."""

    def __init__(self, ds: Dataset, net: UNet, members, fallback_steps: int | None = None,
                 fallback_precision=FP32, tol: float = 1e-3, pool: int = 8):
        import torch
        self.ds, self.net, self.tol = ds, net, tol
        self.members = [(int(a), int(b)) for a, b in members]
        tr = ds.trajs[self.members[0][0]]
        self.fallback_steps = fallback_steps or tr.span_steps
        idx = torch.tensor([ds.index(a, b) for a, b in self.members], device="cuda")
        self.states = ds.flat.index_select(0, idx).contiguous()
        self.t = np.array([ds.trajs[a].times[b] for a, b in self.members], dtype=np.float64)
        self.rain = np.array([ds.trajs[a].rain for a, _ in self.members], dtype=np.float64)
        self.fallback, self.fallback_of = [], np.zeros(len(self.members), dtype=np.int32)
        first, size, count = {}, {}, {}
        for b, (a, _) in enumerate(self.members):
            if a not in first:
                size[a] = min(pool, sum(1 for x, _ in self.members if x == a))
                first[a], count[a] = len(self.fallback), 0
                for _ in range(size[a]):
                    s = coarse_solver(ds.trajs[a], self.fallback_steps, fallback_precision)
                    s.use_graph(True)
                    self.fallback.append(s)
            self.fallback_of[b] = first[a] + count[a] % size[a]
            count[a] += 1
        self.calls = 0

    def run(self, calls: int, inject=None, stream=None):
        tr = self.ds.trajs[self.members[0][0]]
        acc, chk, self.t = _rollout(self.net, self.states, self.t, self.rain, self.fallback, self.fallback_of,
                                    calls=calls, span=tr.span, fallback_steps=self.fallback_steps, dx=tr.dx,
                                    dy=tr.dx, tol=self.tol, h_dry=tr.work.h_dry, rain_channel=CH_RAIN,
                                    outflow_mask=outflow_mask(tr.work.bc), inject=inject, stream=stream)
        self.calls += calls
        return acc, chk

    def judge(self):
        """The fine solver's coarsened states at the members' current times."""
        import torch
        idx = torch.tensor([self.ds.index(a, b + self.calls) for a, b in self.members], device="cuda")
        return self.ds.flat.index_select(0, idx)[:, :OUT_CH]

    def close(self):
        for s in self.fallback:
            s.close()


def rel_l1(pred, ref) -> np.ndarray:
    """Relative L1 error per state channel over all members:
    sum |pred - ref| / sum |ref| (host FP64)."""
    p = pred[:, :OUT_CH].double().cpu().numpy()
    r = ref[:, :OUT_CH].double().cpu().numpy()
    return np.abs(p - r).sum(axis=(0, 2, 3)) / np.maximum(np.abs(r).sum(axis=(0, 2, 3)), 1e-300)


def coarse_baseline(ds: Dataset, members, calls: int, steps: int | None = None, precision=FP32):
    """The method without the surrogate: the plain solver on the coarse grid
    from the same starting states for the same time; returns the final
    states [B][OUT_CH][Hc][Wc]."""
    import torch
    out = []
    cache = {}
    for a, b in members:
        tr = ds.trajs[a]
        n = steps or tr.span_steps
        if a not in cache:
            cache[a] = coarse_solver(tr, n, precision)
        s = cache[a]
        x = ds.data[a, b, :OUT_CH].clone()
        torch.cuda.synchronize()
        s.set_state_device(x[0], x[1], x[2])
        s.set_infiltrated_device(x[3])
        s.set_time(tr.times[b])
        s.step(calls * n)
        s.get_state_device(x[0], x[1], x[2])
        s.get_infiltrated_device(x[3])
        s.step(0)                 # synchronises the solver's stream
        out.append(x)
    for s in cache.values():
        s.close()
    return torch.stack(out)


def make_net(ds: Dataset, pairs: np.ndarray, base: int = 32, max_batch: int = 16, seed: int = 0) -> UNet:
    Hc, Wc = ds.data.shape[-2:]
    net = UNet(base=base, in_ch=IN_CH, out_ch=OUT_CH, H=Hc, W=Wc, max_batch=max_batch, seed=seed)
    mean, scale_in, scale_out = fit_norm(ds, pairs, seed=seed)
    net.set_norm(mean, scale_in, scale_out)
    return net


def hillslope_works(n: int, seeds, rain_mm_h, rain_s: float, dx: float = 1.0):
    """Fine rainfall-runoff scenarios: the hillslope of swof_inputs with its
    bed and K_s field drawn from each seed and the given rain rate."""
    from swof_inputs import hillslope
    return [hillslope(n=n, dx=dx, seed=2 * s + 100, ks_seed=2 * s + 101, rain_mm_h=r, rain_s=rain_s, t_end=1e30)
            for s, r in zip(seeds, rain_mm_h)]


__all__ = ["IN_CH", "OUT_CH", "CH_RAIN", "CH_ZX", "CH_ZY", "CH_KS", "Dataset", "Trajectory", "Rollout",
           "generate", "fit_norm", "train", "make_net", "coarse_solver", "coarse_baseline", "rel_l1",
           "hillslope_works", "block_mean", "span_rain", "outflow_mask", "FRIC_MANNING"]

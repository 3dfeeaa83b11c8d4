"""The learned surrogate's pipeline on the GPU: coarsening and budget
statistics against numpy, the rollout's checks on the solver's own
trajectories, training on those trajectories, what the trained network
gains over the plain solver, and the per-member fallback."""
import time

import numpy as np
import pytest

import paper_1307_4839_gb300 as sw
from swof_inputs import random_state

pytestmark = pytest.mark.gpu

F, DT, SPAN_STEPS, N_SPANS = 4, 0.1, 16, 150
TRAIN, HELD_OUT = list(range(6)), 6


@pytest.fixture(scope="module")
def ds():
    import torch
    assert torch.cuda.is_available()
    sw.build()
    from paper_1307_4839_gb300 import surrogate as S
    # rain heavy enough to pond within the 240 s (Green-Ampt capacity falls
    # below the rain rate once ~1-3 mm have infiltrated); t_off is half a
    # step off the step grid
    works = S.hillslope_works(256, seeds=range(7), rain_mm_h=[60, 80, 100, 120, 140, 160, 110], rain_s=200.05)
    return S.generate(works, F, DT, SPAN_STEPS, N_SPANS)


@pytest.fixture(scope="module")
def trained(ds):
    from paper_1307_4839_gb300 import surrogate as S
    pairs = ds.pairs(TRAIN)
    net = S.make_net(ds, pairs, base=16, max_batch=16, seed=1)
    t0 = time.perf_counter()
    losses = S.train(net, ds, pairs, steps=1500, batch=16, lr=2e-3, seed=1)
    print(f"training: {len(losses)} steps in {time.perf_counter() - t0:.1f} s, loss {losses[:20].mean():.4g} -> "
          f"{losses[-20:].mean():.4g}")
    return net, losses


def test_coarsen_is_block_mean():
    import torch
    sw.build()
    w = random_state(96, 64, seed=5)
    with sw.Solver.from_workload(w, precision=sw.FP64, infiltration=1, ks=1e-5, psi=0.1, dtheta=0.3,
                                 rain_rate=1e-4, rain_t_off=10.0) as s:
        s.step(3)
        out = torch.zeros((4, 16, 24), device="cuda")
        s.coarsen(4, out)
        torch.cuda.synchronize()
        h, qx, qy = s.state()
        v = s.infiltrated()
    from paper_1307_4839_gb300.surrogate import block_mean
    ref = np.stack([block_mean(a, 4) for a in (h, qx, qy, v)]).astype(np.float32)
    got = out.cpu().numpy()
    assert np.abs(v).max() > 0
    np.testing.assert_allclose(got, ref, rtol=2e-7, atol=1e-30)


def test_static_channels_on_the_device_match_numpy():
    """The surrogate's static inputs from swof_coarsen_static -- slopes of the
    block-mean bed (numpy.gradient's central and one-sided differences) and
    the block-mean K_s -- against numpy, written to every snapshot; a scalar
    K_s fills its channel."""
    import torch
    sw.build()
    from paper_1307_4839_gb300.surrogate import block_mean
    rng = np.random.default_rng(3)
    ny, nx, f, dx, dy = 48, 80, 4, 1.5, 2.0
    z = rng.standard_normal((ny, nx)).cumsum(axis=1) * 0.1
    ks = np.exp(rng.standard_normal((ny, nx))) * 1e-6
    out = torch.full((3, 5, 3, ny // f, nx // f), -1.0, device="cuda")     # [snapshot][slot][channel]
    stride = 5 * 3 * (ny // f) * (nx // f)
    sw.coarsen_static(torch.tensor(z, device="cuda"), torch.tensor(ks, device="cuda"), dx, dy, f,
                      out[0, 1, 0], stride, 1)
    torch.cuda.synchronize()
    zc = block_mean(z, f)
    zy, zx = np.gradient(zc, f * dy, f * dx)
    ref = np.stack([zx, zy, block_mean(ks, f)])
    got = out[0, 1].cpu().numpy().astype(np.float64)
    # FP64 sums in another order, then one rounding to float32
    assert np.all(np.abs(got - ref) <= 1e-7 * np.abs(ref) + 1e-20)
    others = out.cpu().numpy()
    others[0, 1] = -1.0
    assert np.all(others == -1.0)                   # nothing written outside its block
    # every snapshot (stride of one [slot][channel] block), scalar K_s
    out2 = torch.full((4, 8, ny // f, nx // f), -1.0, device="cuda")      # [snapshot][channel]
    sw.coarsen_static(torch.tensor(z, device="cuda"), None, dx, dy, f, out2[0, 5], 8 * (ny // f) * (nx // f), 4,
                      ks_const=2.5e-6)
    torch.cuda.synchronize()
    o2 = out2.cpu().numpy()
    for k in range(4):
        assert np.array_equal(o2[k, 5:8], o2[0, 5:8]) and np.all(o2[k, :5] == -1.0)
        assert np.all(o2[k, 7] == np.float32(2.5e-6))
    assert np.all(np.abs(o2[0, 5:7] - ref[:2]) <= 1e-7 * np.abs(ref[:2]) + 1e-20)


def test_batch_stats_against_numpy():
    import torch
    sw.build()
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, 4, 40, 24)).astype(np.float32)
    out = torch.zeros((5, 5), dtype=torch.float64, device="cuda")
    for mask in (0, 8, 15):
        sw.batch_stats(torch.tensor(x, device="cuda"), out, outmask=mask, dx=2.0, dy=3.0)
        got = out.cpu().numpy()
        xd = x.astype(np.float64)
        h, qx, qy, v = xd[:, 0], xd[:, 1], xd[:, 2], xd[:, 3]
        q = np.zeros(5)
        if mask & 8:
            q += qy[:, -1, :].sum(axis=1) * 2.0
        if mask & 4:
            q -= qy[:, 0, :].sum(axis=1) * 2.0
        if mask & 2:
            q += qx[:, :, -1].sum(axis=1) * 3.0
        if mask & 1:
            q -= qx[:, :, 0].sum(axis=1) * 3.0
        ref = np.stack([h.sum(axis=(1, 2)), np.minimum(h, 0).sum(axis=(1, 2)), q, v.sum(axis=(1, 2)),
                        h.min(axis=(1, 2))], axis=1)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-9)


def test_solver_trajectories_pass_the_checks(ds):
    """The positivity / mass check, restated on the host, accepts every
    pair of the solver's own coarsened evolution with margin: the check
    does not reject the method it stands in for.  (What remains is the FP32
    solver's rounding of V_inf, increments of ~1e-6 m added to ~1e-3 m
    each step, ~1e-4 of the span's rain while everything infiltrates.)"""
    from paper_1307_4839_gb300 import surrogate as S
    x = ds.data.double().cpu().numpy()
    worst = 0.0
    for i, tr in enumerate(ds.trajs):
        A = tr.dx * tr.dx
        area = A * x.shape[-1] * x.shape[-2]
        for k in range(ds.n_snap - 1):
            a, b = x[i, k], x[i, k + 1]
            R = S.span_rain(*tr.rain, tr.times[k], tr.span, tr.span_steps) * tr.span * area
            I = (b[3].sum() - a[3].sum()) * A
            Q = 0.5 * (a[2, -1].sum() + b[2, -1].sum()) * tr.dx * tr.span
            ref = max(a[0].sum() * A + R, area * tr.work.h_dry)
            worst = max(worst, abs(b[0].sum() * A - a[0].sum() * A - (R - I - Q)) / ref)
            assert b[0].min() >= 0
    print(f"largest mass-check error on solver pairs: {worst:.3g}")
    assert worst < 4e-4


def test_training_reduces_loss(trained):
    net, losses = trained
    assert np.all(np.isfinite(losses))
    assert losses[-50:].mean() < 0.2 * losses[:10].mean()


def test_training_is_reproducible(ds):
    """Two trainings from the same seed give the same losses and weights bit
    for bit: the weight and bias gradients and the loss are fixed-order
    reductions (no atomics), the batches come from a seeded generator."""
    from paper_1307_4839_gb300 import surrogate as S
    pairs = ds.pairs(TRAIN)
    runs = []
    for _ in range(2):
        net = S.make_net(ds, pairs, base=16, max_batch=16, seed=5)
        losses = S.train(net, ds, pairs, steps=60, batch=16, lr=2e-3, seed=5)
        runs.append((np.asarray(losses), net.params()))
        net.close()
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])


def test_surrogate_gain_over_plain_solver(ds, trained):
    """On a held-out scenario the trained network's 10-call rollout (160
    fine steps, 16 members) tracks the coarsened fine solver far better
    than persistence, and each member-span costs far less than the fine
    solver's 16 steps."""
    import torch
    from paper_1307_4839_gb300 import surrogate as S
    net, _ = trained
    members = [(HELD_OUT, k) for k in range(0, 128, 8)]
    calls = 10
    ro = S.Rollout(ds, net, members)
    start = ro.states[:, :S.OUT_CH].clone()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    acc, chk = ro.run(calls)
    torch.cuda.synchronize()
    t_sur = time.perf_counter() - t0
    judge = ro.judge()
    e_sur = S.rel_l1(ro.states, judge)
    e_per = S.rel_l1(start, judge)
    e_crs = S.rel_l1(S.coarse_baseline(ds, members, calls), judge)
    # the fine FP64 solver for one member-span, the cost the surrogate saves
    tr = ds.trajs[HELD_OUT]
    with sw.Solver.from_workload(tr.work, precision=sw.FP64, dt_fixed=DT, t_end=1e30) as fine:
        fine.step(SPAN_STEPS)
        t1 = time.perf_counter()
        fine.step(4 * SPAN_STEPS)
        t_fine = (time.perf_counter() - t1) / 4
    ro.close()
    per_span = t_sur / (calls * len(members))
    print(f"rel L1 (h, hu, hv, V_inf): surrogate {e_sur}, persistence {e_per}, coarse solver {e_crs}; "
          f"accepted {acc.mean():.3f}, worst check {chk.max():.3g}; s per member-span: surrogate "
          f"{per_span:.3g}, fine FP64 solver {t_fine:.3g}")
    assert e_sur[0] < 0.5 * e_per[0]
    assert e_sur[3] < 0.5 * e_per[3]
    assert acc.mean() > 0.5
    assert per_span < t_fine


def test_fallback_replaces_a_failing_member(ds, trained):
    """A prediction perturbed on request fails the mass check; that member
    (and only a failing member) takes exactly the plain coarse solver's
    state for the span, the others keep the network's."""
    import torch
    from paper_1307_4839_gb300 import surrogate as S
    net, _ = trained
    members = [(HELD_OUT, k) for k in (20, 40, 60, 80)]
    ro = S.Rollout(ds, net, members)
    acc, chk = ro.run(1, inject=(2, 0, 0.05))
    assert acc[0, 2] == 0 and chk[0, 2, 0] > 1e-3
    ref = S.coarse_baseline(ds, members, 1)
    for b in range(len(members)):
        if not acc[0, b]:
            assert torch.equal(ro.states[b, :S.OUT_CH], ref[b]), b
    # without a solver to fall back on the rollout reports SWOF_ESTATE
    ro2 = S.Rollout(ds, net, members[:1])
    with pytest.raises(sw.SwofError):
        S._rollout(net, ro2.states, ro2.t, ro2.rain, [], [-1], calls=1, span=DT * SPAN_STEPS,
                   fallback_steps=SPAN_STEPS, dx=4.0, dy=4.0, rain_channel=S.CH_RAIN, inject=(0, 0, 0.05))
    ro.close()
    ro2.close()

"""The adjoint at the adjoint workloads' full sizes, through the C ABI.

- The recomputation schedule inside checkpoint segments changes nothing in
  the gradient: any slot limit gives the same bits as the oracle's adjoint.
- Adjoint workload (nonlinear Landau 32^4, degree 1, FP64, dt 0.1, 100 steps,
  checkpoint every 10): dJ/d(alpha) and directional derivatives along seeded
  random directions against central finite differences with h = 1e-6 of the
  GPU forward, J the time-integrated electric energy.
- Large mixed-precision workload (128^4, degree 1, FP32 storage, dt 0.05,
  200 steps, checkpoint every 25): forward and adjoint fit in HBM with the
  slots that remain after the checkpoint pool; the FP32 electric-energy
  history is within 1e-5 of the FP64 one and the FP32 gradient dJ/d(alpha)
  within 1e-4 of the FP64 central difference.
- An allocation the device cannot hold (a checkpoint pool larger than all of
  HBM) fails with SLDG_ERR_OOM and leaves the context usable; nothing faults.
"""
import numpy as np
import pytest

from inputs import rng

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_02143_gb300 import build

    build.build()
    import paper_1803_02143_gb300 as P

    return P


def _J(s, kind, params, n, dt):
    s.set_initial(kind, params)
    W = s.step(n, history=True)
    return dt * float(np.sum(W)), np.asarray(W)


def test_gradient_independent_of_slot_limit(lib, orc):
    from inputs import LANDAU_HI, LANDAU_LO

    deg, nc, dt = 1, (8, 6, 10, 12), 0.1
    cfg = lib.Config(degree=deg, ncell=nc, lo=LANDAU_LO, hi=LANDAU_HI, dt=dt)
    og = orc.Grid(deg=deg, nc=nc, lo=LANDAU_LO, hi=LANDAU_HI, dt=dt)
    params = (0.5, 0.5, 0.5)
    n, ck = 13, 6
    grads, stats = [], []
    with lib.Sldg(cfg) as s:
        for limit in (0, 1, 2, 3, 5):
            s.set_slot_limit(limit)
            s.set_initial(0, params)
            s.record(n, ck)
            _, g = s.backward()
            torch.cuda.synchronize()
            grads.append(g.cpu().numpy().copy())
            stats.append(s.backward_stats())
    for g in grads[1:]:
        assert np.array_equal(g, grads[0])
    # 2 S + 1 = 13 slots: one pass per segment keeps every step's forward
    # intermediates (5 + 5 + 0 steps recomputed); S - 1 = 5 slots: the
    # segment's states are stored and each step's intermediates rebuilt; one
    # slot: every state from its checkpoint (1 + 2 + ... + 5 per segment)
    assert stats[0] == (10, 13)
    assert stats[4] == (10, 5)
    assert stats[1] == (30, 1)
    assert stats[2][1] == 2 and 10 < stats[2][0] < 30
    _, gr, _ = orc.backward(og, orc.init(og, 0, params), n, ck)
    rel = np.abs(grads[0] - gr.reshape(og.shape)).max() / np.abs(gr).max()
    assert rel < 1e-11, rel


@pytest.fixture(scope="module")
def adj_ws(lib):
    from paper_1803_02143_gb300 import configs

    return configs.workload("adjoint_landau_32")


def test_adjoint_workload_amplitude_fd(lib, adj_ws):
    w = adj_ws
    alpha, kap = w.params[0], w.params[1]
    h = 1e-6
    with lib.Sldg(w.cfg) as s:
        s.set_initial(w.kind, w.params)
        W = s.record(w.steps, w.ckpt)
        J, grad = s.backward()
        ga = s.initial_param_grad(w.kind, w.params, grad)
        Jp, _ = _J(s, w.kind, (alpha + h, kap, kap), w.steps, w.cfg.dt)
        Jm, _ = _J(s, w.kind, (alpha - h, kap, kap), w.steps, w.cfg.dt)
    fd = (Jp - Jm) / (2 * h)
    assert abs(J - w.cfg.dt * np.sum(W)) < 1e-12 * abs(J)
    assert abs(ga - fd) < 1e-6 * abs(fd), (ga, fd)


@pytest.mark.parametrize("seed", [0, 1])
def test_adjoint_workload_directional_fd(lib, adj_ws, seed):
    w = adj_ws
    h = 1e-6
    with lib.Sldg(w.cfg) as s:
        s.set_initial(w.kind, w.params)
        f0 = s.f.clone()
        s.record(w.steps, w.ckpt)
        _, grad = s.backward()
        # a seeded direction of the size of f0 (standard normal times f0)
        d = torch.from_numpy(rng(seed).standard_normal(tuple(f0.shape))).cuda() * f0
        exact = float(torch.sum(grad * d))
        Js = []
        for sign in (1.0, -1.0):
            s.set_f(f0 + sign * h * d)
            W = s.step(w.steps, history=True)
            Js.append(w.cfg.dt * float(np.sum(W)))
    fd = (Js[0] - Js[1]) / (2 * h)
    assert abs(exact - fd) < 1e-6 * abs(fd), (exact, fd)


def _mixed_fp64(lib, w64, n, dt, h):
    alpha, kap = w64.params[0], w64.params[1]
    with lib.Sldg(w64.cfg) as s:
        J64, W64 = _J(s, w64.kind, w64.params, n, dt)
        Jp, _ = _J(s, w64.kind, (alpha + h, kap, kap), n, dt)
        Jm, _ = _J(s, w64.kind, (alpha - h, kap, kap), n, dt)
    return J64, W64, (Jp - Jm) / (2 * h)


def _mixed_fp32(lib, w32, n, ck):
    with lib.Sldg(w32.cfg) as s:
        s.set_initial(w32.kind, w32.params)
        W32 = s.record(n, ck)
        J32, grad = s.backward()
        recomputed, slots = s.backward_stats()
        ga = s.initial_param_grad(w32.kind, w32.params, grad)
    return J32, W32, ga, recomputed, slots


def test_mixed_workload_forward_adjoint_fits_and_matches_fp64(lib):
    from paper_1803_02143_gb300 import configs

    w32 = configs.workload("mixed_landau_128")
    w64 = configs.workload("mixed_landau_128", "fp64")
    n, ck, dt = w32.steps, w32.ckpt, w32.cfg.dt
    torch.cuda.empty_cache()
    J64, W64, fd = _mixed_fp64(lib, w64, n, dt, 1e-6)
    torch.cuda.empty_cache()
    J32, W32, ga, recomputed, slots = _mixed_fp32(lib, w32, n, ck)
    torch.cuda.empty_cache()
    # the 8 checkpoints (137 GB) leave fewer slots than a 25-step segment
    # could use: the segments are bisected and recomputed more than once
    assert 1 <= slots < ck - 1
    assert recomputed > n - n // ck
    assert np.abs(W32 - W64).max() < 1e-5 * np.abs(W64).max()
    assert abs(J32 - J64) < 1e-5 * abs(J64)
    assert abs(ga - fd) < 1e-4 * abs(fd), (ga, fd)


def test_checkpoint_pool_beyond_hbm_is_oom_and_context_survives(lib, orc):
    from inputs import LANDAU_HI, LANDAU_LO

    # 64^2 x 128^2 nodal values of degree 1: 0.54 GB per copy of f
    cfg = lib.Config(degree=1, ncell=(32, 32, 64, 64), lo=LANDAU_LO, hi=LANDAU_HI, dt=0.1)
    fb = cfg.numel * 8
    total = torch.cuda.get_device_properties(0).total_memory
    nsteps = total // fb + 8  # one checkpoint per step: a pool larger than the device
    params = (0.5, 0.5, 0.5)
    s = lib.Sldg(cfg)
    s.set_initial(0, params)
    f0 = s.f.clone()
    with pytest.raises(lib.SldgError) as e:
        s.record(int(nsteps), 1)
    assert e.value.code == lib._native.SLDG_ERR_OOM
    torch.cuda.synchronize()  # no CUDA error is pending or sticky
    assert torch.equal(s.f, f0)  # nothing ran
    # the context still steps, records and differentiates like a fresh one
    s.step(2)
    with lib.Sldg(cfg) as t:
        t.set_initial(0, params)
        t.step(2)
        assert torch.equal(s.f, t.f)
    s.set_initial(0, params)
    W = s.record(3, 2)
    J, grad = s.backward()
    assert np.isfinite(W).all() and np.isfinite(J) and torch.isfinite(grad).all()
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_recordings_reuse_their_buffers(lib, prec):
    """A context keeps its checkpoint pool, W history and backward copies
    between recordings: recordings of other lengths in between (a smaller
    pool, then a larger one) leave J and the gradient of a recording
    bit-identical to those of a fresh context."""
    from inputs import LANDAU_HI, LANDAU_LO

    cfg = lib.Config(degree=2, ncell=(8, 6, 10, 12), lo=LANDAU_LO, hi=LANDAU_HI, dt=0.1,
                     precision=prec)
    params = (0.5, 0.5, 0.5)

    def run(s, n, ck):
        s.set_initial(0, params)
        W = s.record(n, ck)
        J, g = s.backward()
        torch.cuda.synchronize()
        return W.copy(), J, g.clone()

    with lib.Sldg(cfg) as fresh:
        W0, J0, g0 = run(fresh, 12, 4)
    with lib.Sldg(cfg) as s:
        run(s, 12, 4)
        run(s, 5, 2)    # the pool and the W history are larger than needed
        run(s, 30, 3)   # both grow
        W1, J1, g1 = run(s, 12, 4)
    assert np.array_equal(W0, W1) and J0 == J1
    assert torch.equal(g0, g1)

"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Grids are chosen so that tiles are ragged (line lengths and column counts
that are not multiples of the 32-wide tiles) and several tiles are spanned;
v-shifts cover several cells.  Tolerances: FP64 per operation 1e-13 and
per Strang step 1e-12 relative to max|f| (the per-step bound of the
specification); FP32 storage within the rounding of single precision.
"""
import numpy as np
import pytest

from inputs import LANDAU_HI, LANDAU_LO, TSI_HI, TSI_LO, random_f, random_field, smooth_field

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL64 = 1e-13     # one sweep / reduction, relative to max|.|
TOL64_STEP = 1e-12
TOL32 = 3e-6      # one FP32 sweep against the FP64 oracle on the same (rounded) input


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_02143_gb300 import build

    build.build()
    import paper_1803_02143_gb300 as P

    return P


def make(P, orc, deg, nc, lo=LANDAU_LO, hi=LANDAU_HI, dt=0.1, prec="fp64", vbc=0, kmax=-1,
         flags=0):
    cfg = P.Config(degree=deg, ncell=nc, lo=lo, hi=hi, dt=dt, precision=prec, vbc=vbc,
                   poisson_kmax=kmax, flags=flags)
    og = orc.Grid(deg=deg, nc=nc, lo=lo, hi=hi, dt=dt, vbc=vbc, kmax=kmax)
    return P.Sldg(cfg), og


def put(s, arr):
    s.f.copy_(torch.from_numpy(np.ascontiguousarray(arr).reshape(s.cfg.shape)).to(s.cfg.dtype))


def get(s):
    torch.cuda.synchronize()
    return s.f.double().cpu().numpy().reshape(s.cfg.shape)


def relerr(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300)


GRIDS = [
    (1, (5, 3, 7, 6)),     # every dimension ragged and short
    (2, (13, 11, 12, 9)),  # D = 39, 33, 36, 27: several tiles, ragged tails
    (3, (4, 6, 5, 7)),
    (0, (9, 8, 10, 7)),
    (3, (9, 8, 6, 5)),     # dG4: D = 36, 32, 24, 20, x1 lines past one lane tile
]
GRIDS32 = GRIDS[:3] + GRIDS[4:]


@pytest.mark.parametrize("deg,nc", GRIDS)
@pytest.mark.parametrize("dim", [0, 1, 2, 3])
@pytest.mark.parametrize("vbc", [0, 1])
@pytest.mark.parametrize("flags", [0, 1], ids=["doublefloat", "nativefp64"])
def test_sweep_fp64(lib, orc, deg, nc, dim, vbc, flags):
    s, og = make(lib, orc, deg, nc, vbc=vbc, dt=0.37, flags=flags)
    f = random_f(og.shape, seed=100 + dim)
    put(s, f)
    frac = 0.5 if dim < 2 else 1.0
    E = None
    if dim >= 2:
        # fields up to ~3 cells of shift, both signs
        E1 = random_field(og.xshape, seed=7, scale=2.5 * og.h(2) / og.dt)
        E2 = random_field(og.xshape, seed=8, scale=2.5 * og.h(3) / og.dt)
        s.set_field(torch.from_numpy(E1), torch.from_numpy(E2))
        E = E1 if dim == 2 else E2
    s.sweep(dim, frac)
    ref = orc.sweep(og, dim, f, Ed=E, frac=frac).reshape(og.shape)
    assert relerr(get(s), ref) < TOL64
    s.close()


@pytest.mark.parametrize("deg,nc", GRIDS32)
@pytest.mark.parametrize("dim", [0, 1, 2, 3])
def test_sweep_fp32(lib, orc, deg, nc, dim):
    s, og = make(lib, orc, deg, nc, dt=0.37, prec="fp32")
    f = random_f(og.shape, seed=200 + dim).astype(np.float32).astype(np.float64)
    put(s, f)
    frac = 0.5 if dim < 2 else 1.0
    E = None
    if dim >= 2:
        E1 = random_field(og.xshape, seed=9, scale=1.5 * og.h(2) / og.dt)
        E2 = random_field(og.xshape, seed=10, scale=1.5 * og.h(3) / og.dt)
        s.set_field(torch.from_numpy(E1), torch.from_numpy(E2))
        E = E1 if dim == 2 else E2
    s.sweep(dim, frac)
    ref = orc.sweep(og, dim, f, Ed=E, frac=frac).reshape(og.shape)
    assert relerr(get(s), ref) < TOL32
    s.close()


@pytest.mark.parametrize("deg,nc", GRIDS[:3])
@pytest.mark.parametrize("dim", [0, 1, 2, 3])
@pytest.mark.parametrize("vbc", [0, 1])
def test_sweep_adjoint_fp64(lib, orc, deg, nc, dim, vbc):
    s, og = make(lib, orc, deg, nc, vbc=vbc, dt=0.29)
    lam = random_f(og.shape, seed=300 + dim)
    gf = random_f(og.shape, seed=400 + dim)
    frac = 0.5 if dim < 2 else 1.0
    E = None
    if dim >= 2:
        E1 = random_field(og.xshape, seed=11, scale=2.0 * og.h(2) / og.dt)
        E2 = random_field(og.xshape, seed=12, scale=2.0 * og.h(3) / og.dt)
        s.set_field(torch.from_numpy(E1), torch.from_numpy(E2))
        E = E1 if dim == 2 else E2
    lt = torch.from_numpy(lam.reshape(og.shape)).cuda()
    if dim >= 2:
        gt = torch.from_numpy(gf.reshape(og.shape)).cuda()
        Eb = torch.full(og.xshape, 0.25, dtype=torch.float64, device="cuda")  # accumulates
        s.sweep_adjoint(dim, frac, lt, gt, Eb)
        ref, Ebr = orc.sweep_adj(og, dim, lam, Ed=E, frac=frac, gfwd=gf)
        torch.cuda.synchronize()
        assert relerr(Eb.cpu().numpy() - 0.25, Ebr) < 1e-12
    else:
        s.sweep_adjoint(dim, frac, lt)
        ref = orc.sweep_adj(og, dim, lam, Ed=E, frac=frac)
    torch.cuda.synchronize()
    assert relerr(lt.cpu().numpy(), ref.reshape(og.shape)) < TOL64
    s.close()


@pytest.mark.parametrize("deg,nc,lo,hi", [(1, (6, 5, 7, 8), LANDAU_LO, LANDAU_HI),
                                          (2, (13, 11, 9, 10), TSI_LO, TSI_HI),
                                          (3, (5, 7, 4, 4), LANDAU_LO, LANDAU_HI)])
@pytest.mark.parametrize("kmax", [-1, 3])
def test_fields(lib, orc, deg, nc, lo, hi, kmax):
    s, og = make(lib, orc, deg, nc, lo=lo, hi=hi, kmax=kmax)
    f = random_f(og.shape, seed=5, positive=True)
    put(s, f)
    s.compute_fields()
    rho, E1, E2 = s.fields()
    r0, F1, F2 = orc.fields(og, f)
    assert relerr(rho, r0) < TOL64
    assert relerr(E1, F1) < 1e-12 and relerr(E2, F2) < 1e-12
    s.close()


@pytest.mark.parametrize("kind,params", [(0, (0.5, 0.5, 0.5)), (0, (0.01, 0.5, 0.25)),
                                         (1, (1e-3, 0.2, 3.0)), (2, (1e-3, 0.2, 2.4))])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_initial_values(lib, orc, kind, params, prec):
    lo, hi = (LANDAU_LO, LANDAU_HI) if kind == 0 else (TSI_LO, TSI_HI)
    s, og = make(lib, orc, 2, (7, 6, 9, 8), lo=lo, hi=hi, prec=prec)
    s.set_initial(kind, params)
    ref = orc.init(og, kind, params).reshape(og.shape)
    assert relerr(get(s), ref) < (1e-14 if prec == "fp64" else 1e-7)
    s.close()


def test_diagnostics(lib, orc):
    s, og = make(lib, orc, 2, (7, 6, 9, 8))
    f = random_f(og.shape, seed=6)
    put(s, f)
    d = s.diagnostics()
    _, E1, E2 = orc.fields(og, f)
    ref = orc.diagnostics(og, f, E1, E2)
    for k in ("mass", "l1", "l2sq", "kinetic", "electric", "total"):
        assert abs(d[k] - ref[k]) <= 1e-13 * max(abs(ref[k]), 1e-300), k
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_nonfinite_detected(lib, orc, prec, bad):
    s, og = make(lib, orc, 1, (4, 4, 4, 4), prec=prec)
    f = random_f(og.shape, seed=7)
    f.reshape(-1)[123] = bad  # injected on the host before upload
    put(s, f)
    with pytest.raises(lib.SldgError) as e:
        s.diagnostics()
    assert e.value.code == lib._native.SLDG_ERR_NONFINITE
    # the sweeps carry the non-finite value on instead of hiding it
    s.set_initial(0, (0.1, 0.5, 0.5))
    put(s, f)
    s.sweep(0, 0.5)
    s.sweep(1, 0.5)
    assert not np.isfinite(get(s)).all()
    s.close()


def test_v_sweep_without_field_is_a_state_error(lib, orc):
    s, og = make(lib, orc, 1, (4, 4, 4, 4))
    s.set_initial(0, (0.1, 0.5, 0.5))
    with pytest.raises(lib.SldgError) as e:
        s.sweep(2, 1.0)
    assert e.value.code == lib._native.SLDG_ERR_STATE
    s.close()


@pytest.mark.parametrize("deg,nc,dt", [(1, (8, 6, 10, 12), 0.1), (2, (7, 9, 8, 6), 0.05),
                                       (3, (5, 4, 6, 5), 0.2)])
@pytest.mark.parametrize("nsteps", [1, 6])
@pytest.mark.parametrize("flags", [0, 1], ids=["doublefloat", "nativefp64"])
def test_strang_steps_fp64(lib, orc, deg, nc, dt, nsteps, flags):
    s, og = make(lib, orc, deg, nc, dt=dt, flags=flags)
    s.set_initial(0, (0.5, 0.5, 0.5))
    f0 = orc.init(og, 0, (0.5, 0.5, 0.5))
    W = s.step(nsteps, history=True)
    ref, Wr, _, _ = orc.step(og, f0, nsteps)
    # per step the bound is 1e-12; after several steps report growth within nsteps x bound
    assert relerr(get(s), ref.reshape(og.shape)) < TOL64_STEP * nsteps
    assert relerr(W, Wr) < 1e-11
    s.close()


def test_step_from_same_state_each_step(lib, orc):
    # the per-step bound from identical inputs f^m, for every m of a run
    s, og = make(lib, orc, 1, (16, 16, 16, 16), dt=0.1)
    s.set_initial(0, (0.01, 0.5, 0.5))
    f = orc.init(og, 0, (0.01, 0.5, 0.5))
    worst = 0.0
    for m in range(5):
        put(s, f)
        s.step(1)
        f, _, _, _ = orc.step(og, f, 1)
        worst = max(worst, relerr(get(s), f.reshape(og.shape)))
    assert worst < TOL64_STEP
    s.close()


def test_fp32_energy_history(lib, orc):
    # FP32 storage: electric-energy history within 1e-5 of the FP64 oracle
    s, og = make(lib, orc, 2, (8, 8, 12, 12), dt=0.1, prec="fp32")
    s.set_initial(0, (0.5, 0.5, 0.5))
    W = s.step(30, history=True)
    _, Wr, _, _ = orc.step(og, orc.init(og, 0, (0.5, 0.5, 0.5)), 30)
    err = np.abs(W - Wr).max() / np.abs(Wr).max()
    assert err < 1e-5, err
    s.close()


# Unfused (SLDG_FLAG_NO_XFUSION, and odd nc1 in FP64): every x drift and its
# adjoint as separate sweeps, the charge-density adjoint as its own kernel;
# fused: the transposed x pass adds the charge-density adjoint while it
# stages its planes.  FP64 keeps the adjoint in double-float pairs between
# the kernels of the backward; (0, (5, 7, 6, 6)) has an odd number of
# x-nodes per plane, where the v-sweep adjoints take the FP64 FMA kernel on
# IEEE doubles (converted there and back).  Degree 0: a v-sweep is piecewise
# linear in E with a kink at E = 0, where the symmetric Landau data puts the
# node of the middle cell of an odd cell count (to rounding, whose sign
# differs between implementations); a seeded perturbation of f0 keeps E off
# zero at every node, where the gradient is defined.  FP32: 7 steps of 6
# transposed sweeps and their recomputation, each within the one-sweep bound
# 3e-6 of the oracle.
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("deg,nc,fused", [(1, (6, 5, 8, 7), False), (1, (8, 6, 5, 4), False),
                                          (1, (8, 6, 5, 4), True), (2, (8, 8, 4, 3), True),
                                          (0, (5, 7, 6, 6), False), (0, (6, 7, 6, 6), False)])
def test_backward_matches_oracle(lib, orc, prec, deg, nc, fused):
    flags = 0 if fused else lib._native.SLDG_FLAG_NO_XFUSION
    s, og = make(lib, orc, deg, nc, dt=0.1, prec=prec, flags=flags)
    tol = {"W": 1e-12, "grad": 1e-11} if prec == "fp64" else {"W": 1e-5, "grad": 1e-4}
    params = (0.5, 0.5, 0.5)
    f0 = orc.init(og, 0, params)
    if deg == 0:
        f0 = f0 + 1e-3 * random_f(f0.shape, seed=77).reshape(f0.shape)
        if prec == "fp32":
            f0 = f0.astype(np.float32).astype(np.float64)
        s.set_f(torch.from_numpy(f0.reshape(s.cfg.shape)).to(s.cfg.dtype).contiguous())
    else:
        s.set_initial(0, params)
    n, ck = 7, 3
    W = s.record(n, ck)
    J, grad = s.backward()
    assert (s.x_pass_shape[0] > 0) == fused
    Jr, gr, Wr = orc.backward(og, f0, n, ck)
    assert relerr(W, Wr) < tol["W"]
    assert abs(J - Jr) < tol["W"] * abs(Jr)
    torch.cuda.synchronize()
    assert relerr(grad.double().cpu().numpy(), gr.reshape(og.shape)) < tol["grad"]
    # dJ/deps through the library's reduction
    dfde = orc.init(og, 0, (1.0, 0.5, 0.5)) - orc.init(og, 0, (0.0, 0.5, 0.5))
    ge = s.initial_param_grad(0, params, grad)
    assert abs(ge - np.sum(gr * dfde)) < tol["grad"] * abs(ge)
    s.close()


def test_autograd_function(lib, orc):
    from paper_1803_02143_gb300.autograd import time_integrated_energy

    s, og = make(lib, orc, 1, (6, 5, 8, 7), dt=0.1)
    f0 = torch.from_numpy(orc.init(og, 0, (0.5, 0.5, 0.5)).reshape(og.shape)).cuda()
    f0.requires_grad_(True)
    J = time_integrated_energy(f0, s, 5, 2)
    J.backward()
    Jr, gr, _ = orc.backward(og, f0.detach().cpu().numpy(), 5, 2)
    assert abs(J.item() - Jr) < 1e-12 * abs(Jr)
    assert relerr(f0.grad.cpu().numpy(), gr.reshape(og.shape)) < 1e-11
    s.close()


def test_launch_count_and_timing(lib, orc):
    s, og = make(lib, orc, 1, (8, 8, 8, 8))
    s.set_initial(0, (0.1, 0.5, 0.5))
    s.step(1)
    n0 = s.launch_count
    s.timing(True)
    s.step(2)
    t = s.timing_read()
    assert s.launch_count > n0
    for k in ("v1", "v2"):
        assert t[k][1] >= 2 and t[k][0] > 0
    # the x half drifts run as one fused pass each, or as two sweeps each
    if t["x12"][1]:
        assert t["x12"][1] >= 4 and t["x12"][0] > 0
    else:
        for k in ("x1", "x2"):
            assert t[k][1] >= 4 and t[k][0] > 0
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_host_batches_match_single_steps(lib, orc, prec):
    # three host states stepped with overlapped uploads give the bits of
    # one sldg_step each (the same kernels on the second buffer)
    s, og = make(lib, orc, 2, (7, 6, 8, 9), dt=0.1, prec=prec)
    host = torch.empty((3,) + s.cfg.shape, dtype=s.cfg.dtype, pin_memory=True)
    for b, eps in enumerate((0.5, 0.1, 0.3)):
        s.set_initial(0, (eps, 0.5, 0.5))
        s.get_f(host[b])
    torch.cuda.synchronize()
    W = s.step_host_batches(host)
    last = s.f.clone()
    for b in range(3):
        s.set_f(host[b].cuda())
        Wb = s.step(1, history=True)
        assert W[b] == Wb[0]
    assert torch.equal(s.f, last)
    # stride 0: the same state every time
    W0 = s.step_host_batches(host[1].contiguous(), 4)
    assert np.all(W0 == W[1])
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("deg,nc", [(2, (8, 8, 6, 5)), (1, (16, 12, 7, 6)), (2, (12, 16, 5, 4)),
                                    (0, (36, 10, 9, 8)), (3, (9, 8, 6, 5))])
def test_fused_x_pass_matches_separate_sweeps(lib, orc, deg, nc, prec):
    # one fused X1 X2 pass (thread-block clusters) gives the bits of the two
    # separate sweeps (the same arithmetic on the same values); both stay
    # within the precision's rounding of the oracle
    outs = []
    for flags in (0, lib._native.SLDG_FLAG_NO_XFUSION):
        s, og = make(lib, orc, deg, nc, dt=0.1, prec=prec, flags=flags)
        s.set_initial(0, (0.5, 0.5, 0.5))
        W = s.step(3, history=True)
        outs.append((get(s), W))
        s.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    ref, Wr, _, _ = orc.step(og, orc.init(og, 0, (0.5, 0.5, 0.5)), 3)
    assert relerr(outs[0][0], ref.reshape(og.shape)) < (1e-5 if prec == "fp32" else 3 * TOL64_STEP)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_step_graph_replay_matches_eager_steps(lib, orc, prec):
    # sldg_step(n >= 2) replays one recorded step (a CUDA graph); with
    # per-kernel timing on the same calls run eagerly: the same bits, W
    # history included, also when the context switches between history and
    # none.  Calls of one step each give the same bits in FP32; in FP64
    # (double-float sweeps, whose state stays in double-float pairs between
    # the steps of one call and is IEEE between calls) they agree to rounding.
    res = []
    for mode in ("graph", "eager", "single"):
        s, og = make(lib, orc, 2, (8, 6, 10, 12), dt=0.1, prec=prec)
        s.set_initial(0, (0.5, 0.5, 0.5))
        if mode == "single":
            W = np.concatenate([s.step(1, history=True) for _ in range(7)])
            s.step(1)
            s.step(1)
        else:
            s.timing(mode == "eager")
            W = np.concatenate([s.step(4, history=True), s.step(3, history=True)])
            s.step(2)
            s.timing(False)
        res.append((get(s), W))
        s.close()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    if prec == "fp32":
        assert np.array_equal(res[0][0], res[2][0]) and np.array_equal(res[0][1], res[2][1])
    else:
        # nine nonlinear steps; measured 3.5e-13 (rounding amplified by the
        # field's dependence on f), inside the 1e-12 per-step bound
        assert relerr(res[0][0], res[2][0]) < 1e-12 and relerr(res[0][1], res[2][1]) < 1e-12


# The fused X1 X2 pass in the launch shape of the full-size workloads: 64
# x1-cells of degree 2 (192-value lines) give whole warps per line pair in
# the X1 phase; 64 x2-cells split an FP64 x-plane over a cluster of 8 CTAs
# (FP32: 2).  (40, 64): a line length that is not a power of two, same
# cluster sizes.  Full Strang steps against the oracle's steps.
BENCH_X_GRIDS = [(2, (64, 64, 3, 2)), (2, (40, 64, 4, 3))]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("deg,nc", BENCH_X_GRIDS)
def test_bench_x_pass_shape_strang_steps(lib, orc, deg, nc, prec):
    params = (0.5, 0.5, 0.5)
    s, og = make(lib, orc, deg, nc, dt=0.05, prec=prec)
    s.set_initial(0, params)
    s.timing(True)  # eager launches, counted per kernel class
    W = s.step(2, history=True)
    t = s.timing_read()
    s.timing(False)
    assert t["x12"][1] == 4 and t["x1"][1] == 0 and t["x2"][1] == 0  # two fused passes per step
    assert s.x_pass_shape == ((8 if prec == "fp64" else 2), 32)
    ref, Wr, _, _ = orc.step(og, orc.init(og, 0, params), 2)
    tol = 2 * TOL64_STEP if prec == "fp64" else 1e-5
    assert relerr(get(s), ref.reshape(og.shape)) < tol
    assert relerr(W, Wr) < (1e-11 if prec == "fp64" else 1e-5)
    # one more step replayed as a CUDA graph (the path of sldg_step(n >= 2))
    W2 = s.step(2, history=True)
    ref2, Wr2, _, _ = orc.step(og, ref, 2)
    assert relerr(get(s), ref2.reshape(og.shape)) < 2 * tol
    assert relerr(W2, Wr2) < (1e-11 if prec == "fp64" else 1e-5)
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_drift_entry_point_is_the_step_drift(lib, orc, prec):
    # sldg_drift runs X1 X2 with the kernels of the step's drifts: the
    # oracle's two sweeps on random data, and the fused pass was used
    deg, nc = BENCH_X_GRIDS[1]
    s, og = make(lib, orc, deg, nc, dt=0.05, prec=prec)
    f = random_f(og.shape, seed=21)
    if prec == "fp32":
        f = f.astype(np.float32).astype(np.float64)
    put(s, f)
    s.timing(True)
    s.drift(0.5)
    t = s.timing_read()
    s.timing(False)
    assert t["x12"][1] == 1
    ref = orc.sweep(og, 1, orc.sweep(og, 0, f, frac=0.5), frac=0.5).reshape(og.shape)
    assert relerr(get(s), ref) < (2 * TOL64 if prec == "fp64" else 2 * TOL32)
    s.close()


def test_objective_and_weight_count(lib, orc):
    # J of a recording from the library (no arithmetic in Python), the
    # weight count checked against the recorded steps
    s, og = make(lib, orc, 1, (6, 5, 8, 7), dt=0.1)
    s.set_initial(0, (0.5, 0.5, 0.5))
    W = s.record(5, 2)
    c = np.linspace(0.1, 0.5, 5)
    J = s.objective(c)
    Jr, _, Wr = orc.backward(og, orc.init(og, 0, (0.5, 0.5, 0.5)), 5, 2, cW=c)
    assert abs(J - Jr) < 1e-12 * abs(Jr)
    assert abs(s.objective() - 0.1 * np.sum(W)) < 1e-13 * abs(s.objective())
    with pytest.raises(lib.SldgError) as e:
        s.objective(c[:4])
    assert e.value.code == lib._native.SLDG_ERR_ARG
    with pytest.raises(lib.SldgError) as e:
        s.backward(np.ones(7))
    assert e.value.code == lib._native.SLDG_ERR_ARG
    J2, _ = s.backward(c)
    assert J2 == J
    s.close()


def test_autograd_refuses_a_stale_recording(lib, orc):
    from paper_1803_02143_gb300.autograd import time_integrated_energy

    s, og = make(lib, orc, 1, (6, 5, 8, 7), dt=0.1)
    f0 = torch.from_numpy(orc.init(og, 0, (0.5, 0.5, 0.5)).reshape(og.shape)).cuda()
    a = f0.clone().requires_grad_(True)
    b = (1.01 * f0).requires_grad_(True)
    Ja = time_integrated_energy(a, s, 3, 2)
    Jb = time_integrated_energy(b, s, 4, 2)  # the solver now holds b's recording
    with pytest.raises(RuntimeError):
        Ja.backward()
    Jb.backward()
    _, gr, _ = orc.backward(og, b.detach().cpu().numpy(), 4, 2)
    assert relerr(b.grad.cpu().numpy(), gr.reshape(og.shape)) < 1e-11
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("deg,nc,dt", [(2, (40, 64, 3, 2), 1.0), (1, (16, 24, 4, 3), 2.0)])
def test_fused_drift_shifts_of_many_cells(lib, orc, deg, nc, dt, prec):
    # x-shifts of up to 15 cells: most X2 outputs read rows held by CTAs
    # several places away in the cluster (wrapping around the plane)
    s, og = make(lib, orc, deg, nc, dt=dt, prec=prec)
    f = random_f(og.shape, seed=23)
    if prec == "fp32":
        f = f.astype(np.float32).astype(np.float64)
    put(s, f)
    s.timing(True)
    s.drift(0.5)
    t = s.timing_read()
    s.timing(False)
    assert t["x12"][1] == 1 and s.x_pass_shape[0] >= (2 if prec == "fp64" else 1)
    ref = orc.sweep(og, 1, orc.sweep(og, 0, f, frac=0.5), frac=0.5).reshape(og.shape)
    assert relerr(get(s), ref) < (2 * TOL64 if prec == "fp64" else 2 * TOL32)
    s.close()

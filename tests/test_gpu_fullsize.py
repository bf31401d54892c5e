"""Parity at full size: the nonlinear Landau workload (64^4 cells, degree 2,
1.36e9 nodal values), the two-stream workload (64^2 x 128^2 cells, degree 2,
5.4e9 values), the large mixed-precision workload (128^4 cells, degree 1,
4.3e9 values, FP32 storage), the paper's dG4 Landau run (36^4 cells, degree
3, 4.3e8 values) and the cubic-spline comparison method at 128^4 points.

The oracle cannot step billions of values, so each stage of the Strang step
is run alone through the C ABI and sampled outputs are recomputed one by one
by the oracle:
  - the x drifts through sldg_drift, which launches the kernels a Strang
    step launches for them (the fused X1 X2 pass over each x-plane, in the
    cluster shape of the step, asserted): whole sampled x-planes against
    the oracle's X1 then X2 on the gathered plane;
  - single sweeps through sldg_sweep: the v-sweeps are the kernels of the
    step's kicks; the x-sweeps run the separate x1 and x2 kernels (used by
    the step only where the fused pass does not apply, e.g. degree 3 in
    FP64 or SLDG_FLAG_NO_XFUSION): whole sampled lines against the
    oracle's 1D advection of the gathered input line with its own shift;
  - rho at single x-nodes (the oracle's v-quadrature of the gathered
    v-plane) and the full Poisson map of the GPU's rho.
"""
import numpy as np
import pytest

from inputs import LANDAU_HI, LANDAU_LO, rng

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NLINES = 48


CASES = [("nonlinear_landau_64", "fp64"), ("nonlinear_landau_64", "fp32"),
         ("two_stream_64x128", "fp64"), ("two_stream_64x128", "fp32"),
         ("mixed_landau_128", "fp32"), ("landau_dg4_36", "fp64"), ("landau_dg4_36", "fp32"),
         ("spline_landau_128", "fp64"), ("spline_landau_128", "fp32")]


@pytest.fixture(scope="module")
def big():
    """One full-size context at a time, built on demand."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_02143_gb300 import build

    build.build()
    live = {}
    yield live
    for s, _ in live.values():
        s.close()


def _context(big, orc, name, prec):
    key = (name, prec)
    if key in big:
        return big[key]
    for s, _ in list(big.values()):
        s.close()
    big.clear()
    import paper_1803_02143_gb300 as P
    from paper_1803_02143_gb300 import configs

    torch.cuda.empty_cache()
    w = configs.workload(name, prec)
    s = P.Sldg(w.cfg)
    s.set_initial(w.kind, w.params)
    s.step(1)  # a developed state, not the separable initial value
    spl = 1 if w.cfg.flags & P._native.SLDG_FLAG_SPLINE else 0
    og = orc.Grid(deg=w.cfg.degree, nc=w.cfg.ncell, lo=w.cfg.lo, hi=w.cfg.hi, dt=w.cfg.dt,
                  vbc=w.cfg.vbc, spline=spl)
    big[key] = (s, og)
    return big[key]


def _lines(F, d, idx):
    """Gather the lines along direction d at the sampled other-indices."""
    if d == 0:
        return F[idx[:, 0], idx[:, 1], idx[:, 2], :]
    if d == 1:
        return F[idx[:, 0], idx[:, 1], :, idx[:, 2]]
    if d == 2:
        return F[idx[:, 0], :, idx[:, 1], idx[:, 2]]
    return F[:, idx[:, 0], idx[:, 1], idx[:, 2]].T


@pytest.mark.parametrize("name,prec", CASES)
@pytest.mark.parametrize("d", [0, 1, 2, 3])
def test_fullsize_sweep_sampled_lines(big, orc, name, prec, d):
    s, og = _context(big, orc, name, prec)
    F = s.f
    shp = og.shape
    other = [a for a in range(4) if a != 3 - d]  # numpy axes other than d's
    r = rng(1000 + d)
    idx = np.stack([r.integers(0, shp[a], NLINES) for a in other], axis=1)
    idx_t = torch.from_numpy(idx).cuda()
    if d >= 2:
        s.compute_fields()
        _, E1, E2 = s.fields()
    before = _lines(F, d, idx_t).double().cpu().numpy()
    frac = 0.5 if d < 2 else 1.0
    s.sweep(d, frac)
    torch.cuda.synchronize()
    after = _lines(F, d, idx_t).double().cpu().numpy()
    worst = 0.0
    for k in range(NLINES):
        # node coordinates / field at this line, from the oracle's grid
        if d == 0:
            a = og.nodes(2)[idx[k, 1]] * og.dt * frac        # axes (v2, v1, x2)
        elif d == 1:
            a = og.nodes(3)[idx[k, 0]] * og.dt * frac        # axes (v2, v1, x1)
        elif d == 2:
            a = E1[idx[k, 1], idx[k, 2]] * og.dt * frac      # axes (v2, x2, x1)
        else:
            a = E2[idx[k, 1], idx[k, 2]] * og.dt * frac      # axes (v1, x2, x1)
        if og.spline:
            ref = orc.spline_line(og.h(d), a, before[k])
        else:
            ref = orc.advect_line(og.deg, og.nc[d], og.h(d), a, d < 2, before[k])
        worst = max(worst, np.abs(after[k] - ref).max() / max(np.abs(ref).max(), 1e-300))
    assert worst < (1e-13 if prec == "fp64" else (5e-6 if og.spline else 2e-6)), worst


@pytest.mark.parametrize("name,prec", CASES)
def test_fullsize_rho_and_poisson(big, orc, name, prec):
    s, og = _context(big, orc, name, prec)
    s.compute_fields()
    rho, E1, E2 = s.fields()
    r = rng(77)
    F = s.f
    for _ in range(8):
        i1, i0 = int(r.integers(0, og.D(1))), int(r.integers(0, og.D(0)))
        col = F[:, :, i1, i0].double().cpu().numpy()
        ref = orc.rho_column(og, col)
        assert abs(rho[i1, i0] - ref) < 1e-13 * abs(ref)
    # the full Poisson map of the GPU's rho
    R1, R2 = orc.poisson(og, rho)
    scale = max(np.abs(R1).max(), np.abs(R2).max())
    assert np.abs(E1 - R1).max() < 1e-12 * scale and np.abs(E2 - R2).max() < 1e-12 * scale


DRIFT_CASES = [("nonlinear_landau_64", "fp64"), ("nonlinear_landau_64", "fp32"),
               ("two_stream_64x128", "fp64"), ("two_stream_64x128", "fp32")]
NPLANES = 6


@pytest.mark.parametrize("name,prec", DRIFT_CASES)
def test_fullsize_fused_drift_sampled_planes(big, orc, name, prec):
    s, og = _context(big, orc, name, prec)
    F = s.f
    r = rng(2024)
    i3 = r.integers(0, og.D(3), NPLANES)
    i2 = r.integers(0, og.D(2), NPLANES)
    it3, it2 = torch.from_numpy(i3).cuda(), torch.from_numpy(i2).cuda()
    before = F[it3, it2].double().cpu().numpy()  # (planes, D_x2, D_x1)
    s.timing(True)
    s.drift(0.5)
    t = s.timing_read()
    s.timing(False)
    assert t["x12"][1] == 1 and t["x1"][1] == 0 and t["x2"][1] == 0
    assert s.x_pass_shape == ((8 if prec == "fp64" else 2), 32)
    after = F[it3, it2].double().cpu().numpy()
    h0, h1 = og.h(0), og.h(1)
    worst = 0.0
    for k in range(NPLANES):
        a1 = og.nodes(2)[i2[k]] * og.dt * 0.5
        a2 = og.nodes(3)[i3[k]] * og.dt * 0.5
        P = before[k]
        X1 = np.stack([orc.advect_line(og.deg, og.nc[0], h0, a1, True, P[j]) for j in range(og.D(1))])
        X2 = np.stack([orc.advect_line(og.deg, og.nc[1], h1, a2, True, X1[:, i])
                       for i in range(og.D(0))], axis=1)
        worst = max(worst, np.abs(after[k] - X2).max() / max(np.abs(X2).max(), 1e-300))
    assert worst < (2e-13 if prec == "fp64" else 4e-6), worst

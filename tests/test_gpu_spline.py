"""The cubic-spline comparison method (Sec. 3, SLDG_FLAG_SPLINE) through the
C ABI, against the oracle's spline sweeps on degree-0 grids (periodic in
every direction): each sweep on ragged grids (lines not multiples of the
32-line tiles, shifts of several points of either sign), Strang steps, the
order-4 composition with merged drifts, and the refusals of the
configurations and entry points the method does not support.
"""
import numpy as np
import pytest

from inputs import LANDAU_HI, LANDAU_LO, random_f, random_field

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-13, "fp32": 5e-6}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_02143_gb300 import build

    build.build()
    import paper_1803_02143_gb300 as P

    return P


def _make(P, orc, nc, dt, prec, flags=0):
    N = P._native
    cfg = P.Config(degree=0, ncell=nc, lo=LANDAU_LO, hi=LANDAU_HI, dt=dt, precision=prec,
                   vbc=N.SLDG_VBC_PERIODIC, flags=N.SLDG_FLAG_SPLINE | flags)
    og = orc.Grid(deg=0, nc=nc, lo=LANDAU_LO, hi=LANDAU_HI, dt=dt, vbc=1, spline=1)
    return P.Sldg(cfg), og


def _get(s):
    torch.cuda.synchronize()
    return s.f.double().cpu().numpy().reshape(s.cfg.shape)


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(b).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
# (300, 4, 3, 310): FP64 lines too long for two staged tiles of 300 points
# (the single-buffer form); many tiles per CTA on the other grids
@pytest.mark.parametrize("nc", [(37, 5, 9, 40), (8, 33, 70, 3), (300, 4, 3, 310)])
@pytest.mark.parametrize("dim", [0, 1, 2, 3])
def test_spline_sweep_matches_oracle(lib, orc, prec, nc, dim):
    s, og = _make(lib, orc, nc, 0.37, prec)
    f = random_f(og.shape, seed=300 + dim)
    if prec == "fp32":
        f = f.astype(np.float32).astype(np.float64)
    s.f.copy_(torch.from_numpy(f.reshape(s.cfg.shape)).to(s.cfg.dtype))
    frac = 0.5 if dim < 2 else 1.0
    E = None
    if dim >= 2:
        E1 = random_field(og.xshape, seed=11, scale=3.5 * og.h(2) / og.dt)
        E2 = random_field(og.xshape, seed=12, scale=3.5 * og.h(3) / og.dt)
        s.set_field(torch.from_numpy(E1), torch.from_numpy(E2))
        E = E1 if dim == 2 else E2
    s.sweep(dim, frac)
    ref = orc.sweep(og, dim, f, Ed=E, frac=frac).reshape(og.shape)
    assert _rel(_get(s), ref) < TOL[prec]
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("order,merge", [(2, False), (4, True)])
def test_spline_steps_match_oracle(lib, orc, prec, order, merge):
    N = lib._native
    flags = (N.SLDG_FLAG_ORDER4 if order == 4 else 0) | (N.SLDG_FLAG_MERGE_DRIFTS if merge else 0)
    s, og = _make(lib, orc, (16, 12, 20, 18), 0.2, prec, flags)
    params = (0.5, 0.5, 0.5)
    s.set_initial(0, params)
    W = s.step(4, history=True)
    ref, Wr, _, _ = orc.step_split(og, orc.init(og, 0, params), 4, order=order, merge=merge)
    tol = 1e-12 * 4 * (3 if order == 4 else 1) if prec == "fp64" else 1e-5
    assert _rel(_get(s), ref.reshape(og.shape)) < tol
    assert _rel(W, Wr) < (1e-11 if prec == "fp64" else 1e-5)
    s.close()


def test_spline_refusals(lib, orc):
    N = lib._native
    P = lib
    for deg, vbc, nc in ((1, 1, (8, 6, 6, 6)), (0, 0, (8, 6, 6, 6)), (0, 1, (8, 2, 6, 6))):
        cfg = P.Config(degree=deg, ncell=nc, lo=LANDAU_LO, hi=LANDAU_HI, dt=0.1, vbc=vbc,
                       flags=N.SLDG_FLAG_SPLINE)
        with pytest.raises(N.SldgError) as ei:
            P.Sldg(cfg)
        assert ei.value.code == N.SLDG_ERR_BAD_CONFIG
    s, _ = _make(lib, orc, (8, 6, 6, 6), 0.1, "fp64")
    s.set_initial(0, (0.5, 0.5, 0.5))
    with pytest.raises(N.SldgError) as ei:
        s.record(2, 1)
    assert ei.value.code == N.SLDG_ERR_UNSUPPORTED
    lam = s.f.clone()
    with pytest.raises(N.SldgError) as ei:
        s.sweep_adjoint(0, 0.5, lam)
    assert ei.value.code == N.SLDG_ERR_UNSUPPORTED
    s.close()

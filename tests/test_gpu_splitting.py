"""The order-4 triple-jump splitting and merged drifts through the C ABI,
against the oracle's stage lists (Sec. 2 cites higher-order splittings).

- ORDER4: every step is S(w1 tau) S(w0 tau) S(w1 tau) of Strang steps; the
  GPU state and W history match the oracle's composition.
- MERGE_DRIFTS: consecutive drifts within one call run as one; one call of
  n steps matches the oracle's merged stage list of n steps (with n - 1
  replays of the recorded step body, or eagerly for n <= 2), and two calls
  match two merged oracle runs.
- The adjoint entry points refuse both modes.
"""
import numpy as np
import pytest

from inputs import LANDAU_HI, LANDAU_LO

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL64_STEP = 1e-12
TOL32_STEPS = 1e-5


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_02143_gb300 import build

    build.build()
    import paper_1803_02143_gb300 as P

    return P


def _make(P, orc, deg, nc, dt, prec, flags):
    cfg = P.Config(degree=deg, ncell=nc, lo=LANDAU_LO, hi=LANDAU_HI, dt=dt, precision=prec,
                   flags=flags)
    og = orc.Grid(deg=deg, nc=nc, lo=LANDAU_LO, hi=LANDAU_HI, dt=dt)
    return P.Sldg(cfg), og


def _get(s):
    torch.cuda.synchronize()
    return s.f.double().cpu().numpy().reshape(s.cfg.shape)


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(b).max()


def _flags(P, order, merge):
    N = P._native
    return (N.SLDG_FLAG_ORDER4 if order == 4 else 0) | (N.SLDG_FLAG_MERGE_DRIFTS if merge else 0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("order,merge", [(4, False), (4, True), (2, True)])
@pytest.mark.parametrize("deg,nc,nsteps", [(1, (8, 6, 10, 12), 1), (2, (7, 9, 8, 6), 2),
                                           (3, (6, 8, 5, 4), 4)])
def test_split_steps_match_oracle(lib, orc, prec, order, merge, deg, nc, nsteps):
    s, og = _make(lib, orc, deg, nc, 0.15, prec, _flags(lib, order, merge))
    params = (0.5, 0.5, 0.5)
    s.set_initial(0, params)
    W = s.step(nsteps, history=True)
    ref, Wr, _, _ = orc.step_split(og, orc.init(og, 0, params), nsteps, order=order, merge=merge)
    subs = 3 if order == 4 else 1
    tol = TOL64_STEP * subs * nsteps if prec == "fp64" else TOL32_STEPS
    assert _rel(_get(s), ref.reshape(og.shape)) < tol
    assert _rel(W, Wr) < (1e-11 if prec == "fp64" else TOL32_STEPS)
    s.close()


@pytest.mark.parametrize("order", [2, 4])
def test_merged_calls_are_separate_compositions(lib, orc, order):
    # two calls of 3 steps: each call merges its own drifts (graph replay of
    # the step body inside each call), the same as two oracle runs
    s, og = _make(lib, orc, 2, (8, 6, 10, 12), 0.1, "fp64", _flags(lib, order, True))
    params = (0.5, 0.5, 0.5)
    s.set_initial(0, params)
    W = np.concatenate([s.step(3, history=True), s.step(3, history=True)])
    f1, W1, _, _ = orc.step_split(og, orc.init(og, 0, params), 3, order=order, merge=True)
    f2, W2, _, _ = orc.step_split(og, f1, 3, order=order, merge=True)
    assert _rel(_get(s), f2.reshape(og.shape)) < TOL64_STEP * 6 * (3 if order == 4 else 1)
    assert _rel(W, np.concatenate([W1, W2])) < 1e-11
    # one call of 6 steps is a different (merged) composition
    f6, _, _, _ = orc.step_split(og, orc.init(og, 0, params), 6, order=order, merge=True)
    assert _rel(f6, f2) > 1e-9
    s.close()


def test_adjoint_refuses_split_modes(lib, orc):
    for flags in (lib._native.SLDG_FLAG_ORDER4, lib._native.SLDG_FLAG_MERGE_DRIFTS):
        s, _ = _make(lib, orc, 1, (6, 5, 6, 7), 0.1, "fp64", flags)
        s.set_initial(0, (0.5, 0.5, 0.5))
        with pytest.raises(lib._native.SldgError) as ei:
            s.record(2, 1)
        assert ei.value.code == lib._native.SLDG_ERR_UNSUPPORTED
        s.close()

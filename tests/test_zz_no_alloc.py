"""The allocation-free charge density against the context path.

sldg_rho_noalloc serves callers that cannot allocate device memory: it keeps
its partial sums in a fixed array inside the library instead of calling
cudaMalloc.  This file is collected last so that a failure here stops a
run only after every other test has run; it also passes alone in a fresh
process.  Two calls in a row check that the shared array carries nothing
from one call into the next.
"""
import numpy as np
import pytest

from inputs import LANDAU_HI, LANDAU_LO, TSI_HI, TSI_LO, random_f

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_02143_gb300 import build

    build.build()
    import paper_1803_02143_gb300 as P

    return P


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_rho_without_allocation_matches_context_rho(P, prec):
    from paper_1803_02143_gb300 import _native as N

    cases = [
        (2, (12, 10, 9, 11), LANDAU_LO, LANDAU_HI, 31),  # first call on the device
        (1, (7, 9, 14, 6), TSI_LO, TSI_HI, 32),          # second call, other grid and data
        # a large x-plane over few v-cells: the scratch limits the chunks to
        # 3 of 342 v-planes each (weights filled by a strided loop)
        (3, (100, 100, 8, 8), LANDAU_LO, LANDAU_HI, 33),
        # many v-planes: the chunk count is capped at 32
        (1, (4, 4, 64, 64), TSI_LO, TSI_HI, 34),
        # an x-plane just below the scratch size: a single chunk
        (1, (362, 362, 2, 2), LANDAU_LO, LANDAU_HI, 35),
    ]
    stream = torch.cuda.current_stream()
    for deg, nc, lo, hi, seed in cases:
        cfg = P.Config(degree=deg, ncell=nc, lo=lo, hi=hi, dt=0.1, precision=prec)
        f = torch.from_numpy(random_f(cfg.shape, seed=seed, positive=True)).to(cfg.dtype).cuda()
        with P.Sldg(cfg, f=f) as s:
            s.compute_fields()
            rho_ctx, _, _ = s.fields()
        rho = torch.full(cfg.xshape, np.nan, dtype=torch.float64, device="cuda")
        N.sldg_rho_noalloc(cfg.c(), f.data_ptr(), rho.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        got = rho.cpu().numpy()
        assert np.isfinite(got).all()
        err = np.abs(got - rho_ctx).max() / np.abs(rho_ctx).max()
        assert err < 1e-13, err


def test_rho_without_allocation_rejects_large_planes(P):
    from paper_1803_02143_gb300 import _native as N

    cfg = P.Config(degree=3, ncell=(200, 200, 2, 2), lo=LANDAU_LO, hi=LANDAU_HI, dt=0.1)
    with pytest.raises(N.SldgError) as e:
        # the size check comes before any device work: null-free dummy pointers
        N.sldg_rho_noalloc(cfg.c(), 256, 256, 0)
    assert e.value.code == N.SLDG_ERR_UNSUPPORTED

"""Device ray sets against the oracle's float64 restatement: at most one float32 ulp apart per
component (both evaluate in float64 and round once; the transcendental functions of the two
platforms may differ in the last float64 bit), and mostly identical."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_19652_gb300 as st
    return st.Context(0)


def ulp_diff(a, b):
    ai = a.view(np.int32).astype(np.int64)
    bi = b.view(np.int32).astype(np.int64)
    ai = np.where(ai < 0, -(ai & 0x7fffffff), ai)
    bi = np.where(bi < 0, -(bi & 0x7fffffff), bi)
    return np.abs(ai - bi)


@pytest.mark.parametrize("kind", ["zonal", "fibonacci"])
@pytest.mark.parametrize("n", [1, 2, 3, 7, 1000, 100_003, 1_000_000])
def test_ray_sets_match_oracle(ctx, kind, n):
    from oracle import rays
    g = ctx.ray_directions(n, kind).cpu().numpy()
    o = rays.zonal(n) if kind == "zonal" else rays.fibonacci(n)
    d = ulp_diff(g, o)
    assert d.max() <= 1, (kind, n, int(d.max()))
    assert (d == 0).mean() >= 0.99

"""Host side of the spatio-temporal box calls against the reference (CPU only; the
library loads without a GPU): Sec. VI-D's box traffic with and without clipping, Eq. 6
for the group's reaches, shared-memory feasibility and argument checks."""
import pytest

from oracle import partition as opart
from oracle import stbox as ost
from paper_1509_04394_gb300 import build as kbuild
from paper_1509_04394_gb300 import kfuse as K


@pytest.fixture(scope="module", autouse=True)
def lib():
    kbuild.build()


@pytest.mark.parametrize("W,H,T,x,t,n", [(1024, 1024, 1000, 32, 16, 2), (800, 600, 97, 64, 5, 4), (13, 9, 7, 8, 3, 1),
                                         (256, 256, 1000, 16, 64, 2)])
def test_traffic_equals_the_reference(W, H, T, x, t, n):
    model, clipped = K.kf_st_traffic(W, H, T, x, t, n)
    assert model == pytest.approx(ost.box_model_bytes(W, H, T, x, t, n), rel=1e-12)
    assert clipped == 4 * ost.box_exact_reads(W, H, T, x, t, n) + W * H * T


@pytest.mark.parametrize("beta", [4096.0, 16384.0, 65536.0, 1e6])
@pytest.mark.parametrize("n", ost.TAPS)
def test_eq6_equals_the_reference(beta, n):
    x, t = K.kf_st_box_eq6(beta, n)
    xr, tr = opart.eq6_box(beta, ost.DX, n)
    assert x == pytest.approx(xr, rel=1e-12) and t == pytest.approx(tr, rel=1e-12)


def test_smem_grows_with_the_box_and_the_ring():
    for n in ost.TAPS:
        b = [K.kf_st_smem_bytes(n, x) for x in (8, 16, 32, 48, 64, 96)]
        assert b == sorted(b) and b[-1] <= 227 * 1024
        # staging and temporal planes (4 bytes a pixel each), the ring of n frames (2 bytes
        # a pixel each) and the smoothed plane, each at least its raw size
        x = 64
        assert b[4] >= (x + 8) * (x + 4) * (8 + 2 * n) + (x + 2) * (x + 4) * 4
    assert K.kf_st_smem_bytes(4, 64) > K.kf_st_smem_bytes(2, 64) > K.kf_st_smem_bytes(1, 64)


@pytest.mark.parametrize("n,x", [(3, 16), (2, 12), (2, 4), (0, 8), (2, 128), (1, 24)])
def test_bad_arguments_are_rejected(n, x):
    with pytest.raises(K.KfuseError):
        K.kf_st_smem_bytes(n, x)


@pytest.mark.parametrize("n", [2, 4])
@pytest.mark.parametrize("beta", [4096, 16384, 65536])
def test_least_traffic_box_is_the_grid_point_nearest_eq6(n, beta):
    """On the benchmark's 1024 x 1024 x 1000 volume, among the box sides 8..96 with
    t = beta / x^2, the box of least clipped traffic is one of the grid points next to
    Eq. 6's x (the model's optimum; clipping at the volume's edges moves it little)."""
    sides = [x for x in (8, 16, 32, 48, 64, 96) if beta // (x * x) >= 1]
    clipped = {x: K.kf_st_traffic(1024, 1024, 1000, x, beta // (x * x), n)[1] for x in sides}
    best = min(clipped, key=clipped.get)
    x6, _ = K.kf_st_box_eq6(beta, n)
    below = max([x for x in sides if x <= x6], default=min(sides))
    above = min([x for x in sides if x >= x6], default=max(sides))
    assert best in (below, above)


@pytest.mark.parametrize("beta", [1, 100, 4096, 16384, 65536, 1e6])
@pytest.mark.parametrize("n", ost.TAPS)
def test_eq6_plan_is_the_nearest_supported_side(beta, n):
    x, t = K.kf_st_plan_eq6(beta, n)
    x6, _ = opart.eq6_box(beta, ost.DX, n)
    sides = (8, 16, 32, 48, 64, 96)
    ratio = lambda s: max(s / x6, x6 / s)  # noqa: E731
    assert x in sides and ratio(x) == min(ratio(s) for s in sides)
    assert t == max(1, round(beta / (x * x)))
    with pytest.raises(K.KfuseError):
        K.kf_st_plan_eq6(0.5, n)

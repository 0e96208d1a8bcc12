"""Host logic of sampled-multipole grids (no GPU): the sampling list and the
argument checks of gcamb_grid_create_lsampled."""
import numpy as np
import pytest

from paper_2509_25110_gb300 import build, gcamb


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


@pytest.mark.parametrize("lmin,lmax,boost", [(2, 2500, 1.0), (2, 2500, 3.0), (0, 6000, 0.5), (2, 40, 1.0), (7, 7, 1.0)])
def test_l_sampling_list(lmin, lmax, boost):
    lv = gcamb.l_sampling(lmin, lmax, boost)
    assert lv[0] == lmin and lv[-1] == lmax
    assert np.all(np.diff(lv) >= 1)
    steps = np.diff(lv)
    cap = max(1, int(np.ceil(50.0 / boost)))
    assert np.all(steps <= cap)
    assert np.all(lv[lv < min(20 * boost, lmax)] == np.arange(lmin, lmin + np.sum(lv < min(20 * boost, lmax))))


def test_l_sampling_boost_50_is_every_l():
    assert np.array_equal(gcamb.l_sampling(2, 3000, 50.0), np.arange(2, 3001))


def test_lsampled_grid_arguments():
    k = np.geomspace(1e-4, 0.3, 10)
    tau = np.linspace(200.0, 14000.0, 20)
    g = gcamb.grid_create_lsampled(k, tau, 14000.0, [2, 3, 10, 50, 400])
    assert g.nl == 5 and g.lmin == 2 and g.lmax == 400
    info = gcamb.grid_info(g)
    assert info["nl"] == 5 and info["lmin"] == 2 and info["lmax"] == 400
    for bad in ([3, 2], [2, 2], [-1, 4], [2, 20001]):
        with pytest.raises(gcamb.GcambError) as ei:
            gcamb.grid_create_lsampled(k, tau, 14000.0, bad)
        assert ei.value.code == gcamb.EINVAL

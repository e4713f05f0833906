"""Feature-specialised tile kernels: a run launches the narrowest specialised instantiation whose
feature set covers the run's features, and the generic instantiation otherwise (the parity tests
check each workload family against the oracle, so both kinds are exercised there)."""
import pytest

from paper_2307_14302_gb300 import dgswe as D
from paper_2307_14302_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# Feature bits (include/dgswe.h, dgswe_get_tile_features)
RIVER, OCEAN, PRESS, RAIN1, RAIN2, RAIN3 = 1, 2, 4, 8, 16, 32
MANNING, QUAD, NOFRIC, POW2, GENSSP, RAIN0 = 64, 128, 256, 512, 1024, 2048
ALL = 4095


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2307_14302_gb300 import build as B

    B.build()
    D.lib()


def _coastal_no_rain():
    w = W.coastal_c2(n_tri=4000, seed=9, steps=10)
    w.storm = None
    return w


CASES = {
    # workload, precision, expected run features, expected kernel features
    "coastal": (lambda: W.coastal_c2(n_tri=4000, seed=3, steps=10), D.MIXED,
                OCEAN | RAIN2 | MANNING | POW2, OCEAN | RAIN2 | MANNING | POW2),
    "coastal_no_rain": (_coastal_no_rain, D.MIXED, OCEAN | RAIN0 | MANNING | POW2, ALL),
    "hurricane": (lambda: W.hurricane_c5(n_tri=20_000), D.MIXED,
                  OCEAN | RAIN3 | MANNING | POW2, OCEAN | RAIN3 | MANNING | POW2),
    "basin": (lambda: W.basin_c1(), D.MIXED, RAIN1 | MANNING | POW2, RAIN1 | MANNING | POW2),
    "river": (lambda: W.river_basin(), D.MIXED, RIVER | RAIN0 | MANNING | POW2, ALL),
    "graded_p2": (lambda: W.graded_c3(n_tri=20_000, steps=10), D.MIXED,
                  OCEAN | RAIN2 | PRESS | MANNING | POW2 | GENSSP, OCEAN | RAIN2 | PRESS | MANNING | POW2 | GENSSP),
    "coastal_fp64": (lambda: W.coastal_c2(n_tri=4000, seed=3, steps=10), D.FP64,
                     OCEAN | RAIN2 | MANNING | POW2, ALL),
}


@pytest.mark.parametrize("case", list(CASES))
def test_tile_form_launches_the_narrowest_covering_instantiation(case):
    make, prec, want_run, want_kernel = CASES[case]
    dev = D.from_workload(make(), precision=prec, block=64, waves=1, split=2)
    run, kernel = dev.tile_features()
    assert run == want_run, (case, run)
    assert kernel == want_kernel, (case, kernel)
    assert run & ~kernel == 0  # the instantiation covers the run
    dev.step(2)
    dev.sync()
    dev.close()

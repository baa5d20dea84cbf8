"""The measured cluster-size autotuner of the mixed kernel: it picks a size
that fits, records every candidate's throughput in its JSON cache, and
reads the cache back instead of measuring again.  (Every cluster size's results are
checked against the oracle in the mixed-path tests.)"""
import json
import os

import pytest

from paper_2402_18471_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CACHE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_build",
                     "test_autotune_cache.json")


@pytest.fixture(scope="module")
def coag_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_18471_b300 import coag
    return coag


def test_autotune_cluster_measures_caches_and_reuses(coag_mod):
    if os.path.exists(CACHE):
        os.remove(CACHE)
    d = synth.make_disc(74, 64, 40, 1e-5, 1.0, 5.0, 100.0, 50.0, seed=5)
    P = coag_mod.autotune_cluster(d, cache_path=CACHE)
    assert P in (1, 2, 4, 8)
    entry = json.load(open(CACHE))[f"N40_cells{d.n_cells}_mixed"]
    assert entry["best"] == P and len(entry["rates"]) >= 2
    assert max(entry["rates"].values()) == entry["rates"][str(P)]
    # a second call reads the cache: with no candidates it could not measure
    assert coag_mod.autotune_cluster(d, candidates=(), cache_path=CACHE) == P
    os.remove(CACHE)


def test_autotune_launch_searches_cluster_pair_mode_and_rings(coag_mod):
    cache = CACHE.replace(".json", "_launch.json")
    if os.path.exists(cache):
        os.remove(cache)
    d = synth.make_disc(74, 64, 40, 1e-5, 1.0, 5.0, 100.0, 50.0, seed=5)
    best = coag_mod.autotune_launch(d, clusters=(1, 2, 4), cache_path=cache)
    assert best["mixed_cluster"] in (1, 2, 4) and best["mixed_pair"] in (1, 2)
    entry = json.load(open(cache))[f"N40_cells{d.n_cells}_mixed_launch"]
    rates = entry["rates"]
    assert any("pair2_" in k for k in rates) and any("pair1_" in k for k in rates)
    # ring depths were measured for the best layout (some fit at 40 bins)
    assert any(not k.endswith("sb0_ks0") for k in rates)
    key = "P{mixed_cluster}_pair{mixed_pair}_sb{mixed_tile_stages}_ks{mixed_k_stages}".format(**best)
    assert max(rates.values()) == rates[key]
    # the layout it returns is the one a context then runs
    g = coag_mod.Coag(d, "mixed", **best)
    assert g.mixed_cluster()[0] == best["mixed_cluster"] and g.mixed_pair() == (best["mixed_pair"] == 2)
    if best["mixed_tile_stages"]:
        assert g.mixed_rings()[:2] == (best["mixed_tile_stages"], best["mixed_k_stages"])
    g.close()
    assert coag_mod.autotune_launch(d, clusters=(), cache_path=cache) == best
    os.remove(cache)

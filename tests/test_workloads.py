"""Seeded input recipes: the mocks follow the paper's stated ranges (Sec. 4.1
for the integration-rule comparison of Sec. 4.5; Sec. 5 for the J0808-like
model) and every truth lies inside its prior box."""
import math

import numpy as np

import workloads as W


def test_rules_mocks_follow_the_paper_recipe():
    for k in range(40):
        s = W.rules_mock(k)
        t = dict(zip(s["param_names"], s["truth"]))
        assert s["n_params"] == 18 and len(s["truth"]) == 18
        assert (t["x_L"], t["y_L"], t["r_L"], t["q_L"], t["pa_L"]) == (0.0, 0.0, 1.3624, 0.75, 45.0)
        assert t["r_H"] == 2.0 and t["mag_H"] == 16.5 and 0.6 <= t["q_H"] <= 0.9
        assert 25 <= t["pa_H"] <= 65 and t["x_H"] == t["x_L"] and t["y_H"] == t["y_L"]
        assert 0.5 <= t["n_S"] <= 8 and 0.1 <= t["r_S"] <= 0.4 and 0.1 <= t["q_S"] <= 1
        assert 0 <= t["pa_S"] < 180 and t["mag_S"] == 23.0
        assert math.hypot(t["x_S"], t["y_S"]) <= 0.5 * 1.3624
        lo, hi = np.array(s["prior_lo"]), np.array(s["prior_hi"])
        assert np.all((np.array(s["truth"]) >= lo) & (np.array(s["truth"]) <= hi))
        assert (s["nx"], s["ny"], s["h"]) == (120, 120, 0.05)
    # different mocks differ, the same mock is reproducible
    assert W.rules_mock(3)["truth"] == W.rules_mock(3)["truth"]
    assert W.rules_mock(3)["truth"] != W.rules_mock(4)["truth"]


def test_j0808_like_has_35_free_parameters_and_the_paper_components():
    for ip in (False, True):
        s = W.j0808_like(image_prior=ip)
        assert s["n_params"] == 35 == len(s["truth"]) == len(s["param_names"])
        types = [c["type"] for c in s["components"]]
        assert types.count("sie") == 2 and types.count("sky") == 1 and types.count("sersic") == 5
        planes = [c["plane"] for c in s["components"] if c["type"] == "sersic"]
        assert planes.count("foreground") == 3
        assert planes.count("source_image" if ip else "source") >= 1
        used = sorted({p[1] for c in s["components"] for p in c["params"] if p[0] == "free"})
        assert used == list(range(35))
        lo, hi = np.array(s["prior_lo"]), np.array(s["prior_hi"])
        assert np.all((np.array(s["truth"]) >= lo) & (np.array(s["truth"]) <= hi))


def test_uneven_batch_follows_its_recipe():
    specs = W.c3_batch(256)
    assert len(specs) == 256
    sizes, orders, psfs, pms = set(), set(), set(), 0
    for s in specs:
        assert 48 <= s["nx"] <= 320 and 48 <= s["ny"] <= 320
        kind, order = s["rule"]
        assert kind == "gl" and 3 <= order <= 7
        n = s["psf"].shape[0]
        assert s["psf"].shape == (n, n) and n % 2 == 1 and 7 <= n <= 31
        types = [c["type"] for c in s["components"]]
        assert types[:2] == ["sie", "shear"] and types[-1] == "sersic"
        pms += "pointmass" in types
        assert s["n_params"] in (13, 16)
        lo, hi = np.array(s["prior_lo"]), np.array(s["prior_hi"])
        assert np.all((np.array(s["truth"]) >= lo) & (np.array(s["truth"]) <= hi))
        sizes.add((s["nx"], s["ny"])); orders.add(order); psfs.add(n)
    # the batch is uneven in every respect it is meant to be
    assert len(sizes) > 200 and orders == {3, 4, 5, 6, 7} and len(psfs) >= 10
    assert 80 < pms < 176  # a point mass with probability 1/2


def test_benchmark_workload_matches_its_description():
    s = W.c2_hst()
    assert (s["nx"], s["ny"], s["h"]) == (200, 200, 0.05) and s["rule"] == ("gl", 5)
    assert s["psf"].shape == (21, 21) and s["n_params"] == 11
    m = np.asarray(s["mask"])
    x = (np.arange(200) - 99.5) * 0.05
    r = np.hypot(*np.meshgrid(x, x))
    assert np.array_equal(m == 0, (r >= 0.5) & (r <= 3.0))
    t = dict(zip(s["param_names"], s["truth"]))
    assert (t["b_L"], t["q_L"], t["pa_L"]) == (1.3624, 0.75, 45.0)
    assert math.hypot(t["x_S"], t["y_S"]) <= 0.5 * 1.3624

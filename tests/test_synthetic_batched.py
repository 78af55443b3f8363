"""The batched uneven workload generator: sizes, oversampling and point range as specified."""
import numpy as np

from synthetic import BATCH_SIZES, batched_uneven


def test_batched_uneven_recipe():
    ps = batched_uneven()
    assert len(ps) == 64
    for p in ps:
        assert p["nx"] in BATCH_SIZES and p["ny"] in BATCH_SIZES
        N, M = p["nx"] * p["ny"], p["x"].size
        assert 1.5 <= p["rho"] <= 4.0
        r = np.sqrt(p["rho"])
        assert M > N
        assert (r * p["nx"] - 0.5) * (r * p["ny"] - 0.5) <= M <= (r * p["nx"] + 0.5) * (r * p["ny"] + 0.5)
        assert np.all((p["x"] >= 0) & (p["x"] < 1) & (p["y"] >= 0) & (p["y"] < 1))
        assert p["c_true"].shape == (N, 8)
    # uneven: several distinct shapes, and the recipe is reproducible
    assert len({(p["nx"], p["ny"]) for p in ps}) > 10
    again = batched_uneven(count=3)
    for a, b in zip(ps[:3], again):
        assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["c_true"], b["c_true"])

"""The seeded input recipes: the uneven relaxation workload of the batched
work list (N from {24, 32, 48} on [-N/3.2, N/3.2]^3, 2 or 3 species with
distinct masses from {1, 2, 4}, M from {6, 12}, N_rho from {8, 16}, VHS or
VSS) and its two-Maxwellian data."""
import numpy as np

from paper_1903_04670_gb300 import workloads as W


def test_relaxation_batch_recipe():
    a = W.relaxation_batch(count=24)
    b = W.relaxation_batch(count=24)
    assert len(a) == 24
    seen_N = set()
    for x, y in zip(a, b):  # seeded: the same draw twice
        assert x["N"] == y["N"] and x["masses"] == y["masses"] and np.array_equal(x["f"], y["f"])
        N, S = x["N"], len(x["masses"])
        seen_N.add(N)
        assert N in (24, 32, 48) and x["L"] == N / 3.2
        assert S in (2, 3) and len(set(x["masses"])) == S and set(x["masses"]) <= {1.0, 2.0, 4.0}
        assert x["M"] in (6, 12) and x["Nrho"] in (8, 16) and x["alpha"] in (1.0, 1.4)
        assert len(x["pairs"]) == S * S
        assert all(pr["alpha"] == x["alpha"] and pr["omega"] == 0.81 for pr in x["pairs"])
        assert x["f"].shape == (1, S, N, N, N) and np.all(x["f"] >= 0.0)
        # each species is a sum of two Maxwellians with densities in [0.5, 1.5]
        h3 = (2.0 * x["L"] / N) ** 3
        dens = x["f"][0].reshape(S, -1).sum(axis=1) * h3
        assert np.all(dens > 0.99 * 1.0) and np.all(dens < 1.01 * 3.0)
    assert len(seen_N) > 1


def test_relaxation_batch_other_seed_differs():
    a = W.relaxation_batch(count=4)
    b = W.relaxation_batch(count=4, seed=6)
    assert any(x["N"] != y["N"] or x["masses"] != y["masses"] or x["f"].shape != y["f"].shape
               or not np.array_equal(x["f"], y["f"]) for x, y in zip(a, b))

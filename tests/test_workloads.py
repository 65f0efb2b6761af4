"""The seeded input generator: determinism, validity and shape of the packings."""
import numpy as np
import pytest

from workloads import WORKLOADS, make_instance


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_instances_are_seeded_valid_and_nontrivial(name):
    a = make_instance(name, 0)
    b = make_instance(name, 0)
    np.testing.assert_array_equal(a.centers, b.centers)
    np.testing.assert_array_equal(a.axes, b.axes)
    d = np.linalg.norm(a.centers[:, None] - a.centers[None], axis=2)
    np.fill_diagonal(d, np.inf)
    assert d.min() - 2 * a.contact_radius > 0.0          # no overlaps
    np.testing.assert_allclose(np.linalg.norm(a.axes, axis=1), 1.0, rtol=1e-14)
    w = WORKLOADS[name]
    assert a.n_bodies == w["M"]
    assert 0.75 * w["n_target"] <= a.n_candidates <= 1.25 * w["n_target"]
    assert a.contact_radius > a.radius
    c = make_instance(name, 1)
    assert not np.array_equal(a.centers, c.centers)

"""Host arithmetic of the bench line that needs no GPU."""

import numpy as np
import pytest

pytest.importorskip("torch")

import bench  # noqa: E402
import oracle  # noqa: E402


def test_thalamic_events_per_biological_second(model):
    """Full scale: sum over populations of N_b K_ext,b nu_th.  With the Table params2 sizes
    (20,683 / 5,834 / 21,915 / 5,479 / 4,850 / 1,065 / 14,395 / 2,948) and in-degrees
    (1,600 / 1,500 / 2,100 / 1,900 / 2,000 / 1,900 / 2,900 / 2,100) at 8 Hz that is
    1,263,481,600 events per biological second."""
    sizes = oracle.pop_sizes(model, 1000)
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    assert bench.thalamic_events_per_bio_s(model, offsets) == 1_263_481_600.0
    by_hand = 8.0 * (20683 * 1600 + 5834 * 1500 + 21915 * 2100 + 5479 * 1900 + 4850 * 2000 + 1065 * 1900
                     + 14395 * 2900 + 2948 * 2100)
    assert by_hand == 1_263_481_600.0


def test_thalamic_events_follow_the_population_sizes(model):
    sizes = oracle.pop_sizes(model, 100)
    offsets = np.concatenate([[0], np.cumsum(sizes), [0] * 3])  # trailing unused slots are ignored
    want = float(sum(int(n) * k * 8.0 for n, k in zip(sizes, model.k_ext)))
    assert bench.thalamic_events_per_bio_s(model, offsets) == want

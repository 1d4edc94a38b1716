"""Host logic of the first-passage harness (no GPU): the first sweep with M <= 0 per chain."""
import numpy as np

from paper_2509_23945_gb300 import first_passage


def test_first_crossing_and_summary():
    m = np.array([[1.0, 0.5, 1.0], [0.2, -0.1, 0.8], [0.0, 0.3, 0.6], [-0.5, 0.2, 0.4]])
    fp = first_passage.first_crossing(m, 4)
    assert fp == [3, 2, None]                   # sweeps are 1-based; M <= 0 counts (C-amb-11)
    s = first_passage.summary(fp)
    assert s == {"chains": 3, "censored": 1, "mean_sweeps": 2.5, "median_sweeps": 2.5}

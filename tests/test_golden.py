"""The paper's printed figures (tests/golden/paper_figures.txt, each with its citation)
against the oracle, the seeded generators and the benchmark's quoted context.

The paper prints no worked example of a simulated mechanism; what it does print are the
curation parameters and shares (Sec. "Dataset Curation & Processing"), the operator
probabilities of its topology generator (Sec. "Generating Valid Topologies"), the scale
of infeasibility of random samples (the infeasibility figure) and the timing table.
"""
import inspect
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2208_14567_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


def load_figures():
    figs = {}
    with open(os.path.join(HERE, "golden", "paper_figures.txt")) as f:
        for line in f:
            if not line.strip() or line.lstrip().startswith("#"):
                continue
            left, _, cite = line.partition("|")
            key, value = left.split()
            assert cite.strip(), f"{key}: no citation"
            figs[key] = float(value)
    return figs


FIG = load_figures()


def test_fixture_is_complete_and_cited():
    assert len(FIG) == 13
    assert FIG["share_circles"] + FIG["share_arcs"] == pytest.approx(0.62)  # the paper's combined 62%


def test_oracle_curation_defaults_are_the_papers():
    sig = inspect.signature(O.curate_paths).parameters
    assert sig["circle_var"].default == FIG["circle_variance_threshold"]
    assert sig["keep_rate"].default == FIG["curation_keep_rate"]


def test_generator_operator_probability_is_the_papers():
    """N_g : N_s = 1 : 3, so a new joint is a ground joint with probability 1/4."""
    r = FIG["ground_to_simple_ratio"]
    p = inspect.signature(I.paper_topologies).parameters["p_ground"].default
    assert p == pytest.approx(r / (1 + r), abs=1e-9)


def test_maxline_normalisation_gives_unit_horizontal_chord_in_the_unit_box():
    """A rotated, scaled and shifted ellipse: after the paper's normalisation the farthest
    pair of points is horizontal, its length is the paper's 1.0, and the path sits centred
    in the unit box."""
    T = 200
    th = 2 * np.pi * np.arange(T) / T
    e = np.stack([3.0 * np.cos(th), 1.0 * np.sin(th)], -1)
    a = 0.7
    R = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
    c = (e @ R.T) * 0.37 + np.array([5.0, -2.0])
    out = O.normalize_maxline(c[None])
    q = out[0] if not isinstance(out, tuple) else out[0][0]
    d = np.linalg.norm(q[:, None] - q[None], axis=-1)
    i, j = np.unravel_index(np.argmax(d), d.shape)
    assert d[i, j] == pytest.approx(FIG["normalised_max_length"], abs=1e-12)
    assert q[i, 1] == pytest.approx(q[j, 1], abs=1e-12)  # the chord is horizontal
    lo, hi = q.min(0), q.max(0)
    assert (lo + hi) / 2 == pytest.approx([0.5, 0.5], abs=1e-12)


def test_generator_reproduces_the_papers_infeasibility_scale(oracle_lib):
    """Seeded samples of the paper's generator (64 topologies x 256 positions per joint
    count), simulated by the oracle at T = 200.  From 13 joints at least the paper's 99%
    lock; at 11 and 12 joints, 98-99% (the generator's larger samples give 1.9% and 1.25%
    valid there).  Averaged over 8-20 joints, a valid design costs more than the paper's
    500 samples."""
    wasted = FIG["wasted_above_10_joints"]
    per_valid = []
    for n in range(8, 21):
        b = I.paper_batch(64, 256, n, seed=100 + n)
        rate = float(oracle_lib.simulate(b, 200, traj=False, path=False).valid.mean())
        per_valid.append(1.0 / rate if rate > 0 else np.inf)
        if n >= 13:
            assert rate <= 1 - wasted, (n, rate)
        elif n >= 11:
            assert rate <= 2 * (1 - wasted), (n, rate)
    assert np.mean(per_valid) > FIG["samples_per_valid_mean"]


def test_benchmark_quotes_the_papers_timing_table_and_shares():
    """bench.py's paper context carries the timing table's figures and the curation
    shares unchanged (read as text: importing the benchmark needs no GPU, but its context
    lives in the code that prints the line)."""
    src = open(os.path.join(HERE, "..", "bench.py")).read()
    for key in ("time_single_thread_s", "time_80_threads_s", "time_v100_s"):
        assert repr(FIG[key]) in src, key
    m = re.search(r'"paper_shares":\s*\{"arcs":\s*([0-9.]+),\s*"circles":\s*([0-9.]+)\}', src)
    assert m and float(m.group(1)) == FIG["share_arcs"] and float(m.group(2)) == FIG["share_circles"]
    # mechanism-steps per second of the V100 row at T = 200
    assert f"{int(FIG['mechanisms_per_timing'])} * 200 / {FIG['time_v100_s']!r}" in src

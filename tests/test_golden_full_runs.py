"""The stored full-length golden runs (tests/golden/full_<name>.npz, written by tests/golden/make_full_runs.py)
are the oracle's runs of the workloads the GPU tests compare against: their receivers, checkpoints and shapes
follow the script's definitions, the whole small run is recomputed here with the serial oracle, and the first
steps of the 2-D runs too.  (The 3-D runs take the oracle minutes per step; their files are checked for shape and
content only.)"""
import importlib.util
import os

import numpy as np
import pytest

from oracle.wave import Simulation

HERE = os.path.dirname(os.path.abspath(__file__))


def _module():
    spec = importlib.util.spec_from_file_location("make_full_runs", os.path.join(HERE, "golden", "make_full_runs.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


G = _module()


def test_survey_picks_span_the_sizes():
    from synth import batched_shots

    shots = batched_shots()
    picks = G.survey_shot_indices(shots)
    sizes = [shots[s].n[0] for s in picks]
    assert len(set(picks)) == 4
    assert sizes[0] == min(w.n[0] for w in shots) and sizes[-1] == max(w.n[0] for w in shots)
    assert sizes == sorted(sizes) and len(set(sizes)) == 4


@pytest.mark.parametrize("name", G.golden_names())
def test_golden_file_matches_its_definition(name):
    path = G.path_of(name)
    assert os.path.exists(path), f"missing {path}: python tests/golden/make_full_runs.py {name}"
    d = np.load(path)
    w, stride = G.golden_workload(name)
    assert int(d["stride"]) == stride
    assert list(d["ckpt_steps"]) == G.checkpoints(w.steps)
    fields = ("sigma", "v1", "v3") if w.physics == "acoustic" else ("v1", "v2", "v3", "s11", "s22", "s33", "s12",
                                                                    "s13", "s23")
    sampled = tuple(len(range(0, s, stride)) for s in w.shape)
    for f in fields:
        assert d[f"snap_{f}"].shape == (4,) + sampled
        assert d[f"norm_{f}"].shape == (4,)
        assert np.isfinite(d[f"snap_{f}"]).all()
    for f, idx in w.receivers.items():
        assert np.array_equal(d[f"rcv_{f}"], idx)
        tr = d[f"trace_{f}"]
        assert tr.shape == (w.steps, len(idx)) and np.isfinite(tr).all()
        assert np.abs(tr).max() > 0.0


def test_small_golden_run_is_the_serial_oracle():
    d = np.load(G.path_of("acoustic2d_small"))
    w, stride = G.golden_workload("acoustic2d_small")
    sim = Simulation(w)
    done = 0
    sl = tuple(slice(None, None, stride) for _ in range(w.dim))
    for i, c in enumerate(d["ckpt_steps"]):
        sim.step(int(c) - done)
        done = int(c)
        for f in ("sigma", "v1", "v3"):
            ref = d[f"snap_{f}"][i]
            assert np.abs(sim.state[f][sl] - ref).max() <= 1e-14 * np.abs(ref).max()
    tr = d["trace_sigma"]
    assert np.abs(sim.trace_array("sigma") - tr).max() <= 1e-14 * np.abs(tr).max()


@pytest.mark.parametrize("name", ["acoustic2d_layered", "survey_first"])
def test_first_steps_of_the_2d_golden_runs(name):
    """The first 6 steps of the full-size 2-D runs, recomputed with the serial oracle."""
    if name == "survey_first":
        name = [n for n in G.golden_names() if n.startswith("survey_shot")][0]
    d = np.load(G.path_of(name))
    w, _ = G.golden_workload(name)
    sim = Simulation(w).step(6)
    tr = d["trace_sigma"][:6]
    got = sim.trace_array("sigma")
    assert np.abs(got - tr).max() <= 1e-14 * max(np.abs(tr).max(), 1e-300)

"""The oracle's process-pool driver (oracle/parallel.py) must equal the serial oracle bit for bit: it only spreads
the derivative terms of each Strang sub-step (Sec. 3.3) over worker processes, each on slabs of whole grid
lines."""
import dataclasses

import numpy as np

from oracle.parallel import ParallelSimulation
from oracle.wave import Simulation
from synth import acoustic2d_small
from synth.workloads import elastic3d_double_layer, elastic3d_gradient_case


def _same_run(w, steps, workers=2):
    ser = Simulation(w).step(steps)
    with ParallelSimulation(w, workers=workers) as par:
        par.step(steps)
        for k in ser.state:
            assert np.array_equal(ser.state[k], par.state[k]), k
        for k in ser.traces:
            assert np.array_equal(ser.trace_array(k), par.trace_array(k)), k
        if ser.mem is not None:
            for k in ser.mem:
                assert np.array_equal(ser.mem[k], par.mem[k]), k
    assert max(float(np.abs(v).max()) for v in ser.state.values()) > 0.0


def test_parallel_acoustic_with_layer_and_source_equals_serial():
    w = acoustic2d_small(n=32, p=2, steps=6, n_nb=8, pml_width=6)
    _same_run(w, 6, workers=3)


def test_parallel_acoustic_without_layer_equals_serial():
    w = dataclasses.replace(acoustic2d_small(n=24, p=3, steps=4, n_nb=6, pml_width=0), dt=1e-3)
    _same_run(w, 4)


def test_parallel_elastic_heterogeneous_with_layer_equals_serial():
    w, _ = elastic3d_gradient_case(n=12, p=2, n_nb=4, steps=4, pml_width=3)
    _same_run(w, 4, workers=3)


def test_parallel_elastic_body_force_without_layer_equals_serial():
    w = elastic3d_double_layer(n=8, nz=12, p=2, pz=2, steps=3, n_nb=4, pml_width=0)
    w = dataclasses.replace(w, f0=2.0, t0=0.0)
    _same_run(w, 3)

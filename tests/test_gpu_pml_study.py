"""GPU reproduction of the paper's ADE-PML study and of the late rows of Table 2d_error (Sec. 4.1), against the
oracle's figures in tests/golden/pml_tables_oracle.txt (written by tests/golden/make_pml_tables.py).

The Gaussian pulse runs through the C ABI in FP64 on [-5, 5]^2 with N = 64 .. 512 intervals, padded by L points
with the absorbing layer in the padding.  At every 200 steps up to t = 0.2 s, the relative l2 error of v3 inside
the domain is taken against the free-space solution of the time stepping and compared with the oracle's value.
The FP64 path follows the oracle to rounding, so the two agree to far better than the 1e-4 allowed here.

About a minute of host work (the free-space solutions) plus 14 runs of 2000 steps.
"""
import collections
import dataclasses
import os

import numpy as np
import pytest

from oracle.exact import pulse_on_grid
from synth import gaussian_pulse_2d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge

    ge.build()
    import paper_2301_05127_gb300 as p

    return p


def _golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "pml_tables_oracle.txt")
    g = collections.defaultdict(dict)
    for line in open(path):
        if line.startswith("#"):
            continue
        N, L, R, k, steps, rel = line.split()[:6]
        g[int(N), int(L), float(R), float(k)][int(steps)] = float(rel)
    return g


def test_pml_study_matches_the_oracle(pkg):
    golden = _golden()
    refs = {}
    for (N, L, R, kmax), rows in sorted(golden.items()):
        w, s0 = gaussian_pulse_2d(N, p=2, n_nb=20, dt=1e-4, steps=max(rows), pad=L)
        w = dataclasses.replace(w, pml_width=L, pml_R=R, pml_kmax=kmax, f0=50.0 / L)
        g = pkg.Grid.from_workloads([w])
        g.set_field(0, "sigma", s0)
        done = 0
        for steps in sorted(rows):
            g.step(steps - done)
            done = steps
            if (N, steps) not in refs:
                refs[N, steps] = pulse_on_grid(N, steps, 1e-4)[1]
            ref = refs[N, steps]
            v3 = g.get_field(0, "v3")[L:L + N + 1, L:L + N + 1]
            rel = np.linalg.norm(v3 - ref) / np.linalg.norm(ref)
            assert abs(rel / rows[steps] - 1.0) < 1e-4, ((N, L, R, kmax), steps, rel, rows[steps])
        g.close()

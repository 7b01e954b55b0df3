"""GPU parity of the 2-D step at the edges of its geometry, against the FP64 oracle: one patch per axis (no
interior junction, only the two one-sided end closures), PMBC halos as wide as a patch (n_nb = M, the largest
the method's halo exchange with the neighbouring patch allows), ragged patches along both axes, and a source on a
patch junction.  Every field at checkpoints along the run relative to the largest reference norm, and the receiver
traces, as in tests/test_gpu_acoustic.py; the FP32 forms run on both truncated-convolution x paths (whole rows and
(row, patch) items) and on the line kernels."""
import dataclasses

import numpy as np
import pytest

from oracle.wave import Simulation
from synth import acoustic2d_small

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp32_kahan": 1e-5}
_REF = {}


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge

    ge.build()
    import paper_2301_05127_gb300 as p

    return p


def _case(name):
    if name == "one patch per axis":
        return acoustic2d_small(n=128, p=1, steps=120, n_nb=12, pml_width=16)
    if name == "halo as wide as a patch":
        return acoustic2d_small(n=128, p=8, steps=120, n_nb=16, pml_width=16)
    if name == "ragged patches":
        w = acoustic2d_small(n=128, p=2, steps=120, n_nb=10, pml_width=12)
        shape = (101, 301)

        def model():
            return np.full(shape, 2000.0), None, np.full(shape, 1000.0)

        return dataclasses.replace(w, name="ragged_100x300", n=(100, 300), p=(4, 4), model_fn=model,
                                   src_index=(50, 150), receivers={"sigma": np.arange(301, dtype=np.int64) + 12 * 301})
    raise KeyError(name)


def _reference(w, every):
    if w.name not in _REF:
        sim = Simulation(w)
        snaps = []
        done = 0
        while done < w.steps:
            k = min(every, w.steps - done)
            sim.step(k)
            done += k
            snaps.append({f: sim.state[f].copy() for f in ("sigma", "v1", "v3")})
        _REF[w.name] = (snaps, sim.trace_array("sigma"))
    return _REF[w.name]


def _errors(pkg, w, prec, family, every=30):
    snaps, ref_tr = _reference(w, every)
    g = pkg.Grid.from_workloads([w], precision=prec)
    if family:
        g.set_kernels(family)
    peak = {f: 0.0 for f in ("sigma", "v1", "v3")}
    worst = dict(peak)
    smax = 0.0
    done = 0
    for ref in snaps:
        k = min(every, w.steps - done)
        g.step(k)
        done += k
        for f in peak:
            peak[f] = max(peak[f], np.linalg.norm(ref[f]))
            worst[f] = max(worst[f], np.linalg.norm(g.get_field(0, f).astype(np.float64) - ref[f]))
        smax = max(smax, np.abs(ref["sigma"]).max())
    errs = {f: worst[f] / max(peak[f], 1e-300) for f in peak}
    errs["trace"] = np.abs(g.record(0)["sigma"].astype(np.float64) - ref_tr).max() / smax
    g.close()
    return errs


FORMS = [("fp64", None), ("fp32_kahan", "convolution"), ("fp32_kahan", "convolution_items"), ("fp32", "convolution"),
         ("fp32_kahan", "line")]


@pytest.mark.parametrize("case", ["one patch per axis", "halo as wide as a patch", "ragged patches"])
@pytest.mark.parametrize("prec,family", FORMS)
def test_step_geometry_edges(pkg, case, prec, family):
    w = _case(case)
    errs = _errors(pkg, w, prec, family)
    assert max(errs.values()) < TOL[prec], (case, prec, family, errs)


def test_halo_wider_than_a_patch_is_rejected(pkg):
    """n_nb > M would need junction sums beyond the neighbouring patch: loss_create_grid refuses it."""
    w = acoustic2d_small(n=128, p=8, steps=1, n_nb=20, pml_width=16)
    with pytest.raises(pkg.LossError) as e:
        pkg.Grid.from_workloads([w], precision="fp32_kahan")
    assert e.value.status == pkg.LOSS_E_SHAPE

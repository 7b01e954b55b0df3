"""GPU tests of the batched schedule (many 2-D acoustic shots of uneven size advanced by one persistent launch per
kernel, optionally replayed from a captured CUDA graph) and of the autotuner, through the C ABI.

The batched schedule performs the arithmetic of the per-shot schedule of the same kernel family (line kernels, or
the FP32 truncated-convolution kernels), so the two are compared for exact equality of every field and trace; the
batched FP64 run is also compared with the FP64 oracle per shot."""
import dataclasses

import numpy as np
import pytest

from oracle.wave import Simulation
from synth import acoustic2d_small, batched_shots

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge

    ge.build()
    import paper_2301_05127_gb300 as p

    return p


def _shots(prec="fp64"):
    """Three shots of different n, p and halo width; pressure, v1 and v3 receivers on the top row (inside the
    absorbing layer, so the velocity traces carry the layer corrections)."""
    ws = [acoustic2d_small(n=64, p=2, n_nb=12, steps=40, pml_width=10),
          acoustic2d_small(n=96, p=3, n_nb=10, steps=40, pml_width=12),
          acoustic2d_small(n=48, p=4, n_nb=8, steps=40, pml_width=8)]
    out = []
    for w in ws:
        top = np.arange(w.n[1] + 1, dtype=np.int64)
        out.append(dataclasses.replace(w, receivers={"sigma": top, "v1": top, "v3": top}, precision=prec,
                                       f0=40.0, t0=1.2 / 40.0))
    return out


def _conv_shots(prec):
    """Three shots whose patch lengths (32, 32, 16) are multiples of 8, so that both FP32 convolution kernels take
    them; receivers as in _shots."""
    ws = [acoustic2d_small(n=64, p=2, n_nb=12, steps=40, pml_width=10),
          acoustic2d_small(n=96, p=3, n_nb=10, steps=40, pml_width=12),
          acoustic2d_small(n=48, p=3, n_nb=8, steps=40, pml_width=8)]
    out = []
    for w in ws:
        top = np.arange(w.n[1] + 1, dtype=np.int64)
        out.append(dataclasses.replace(w, receivers={"sigma": top, "v1": top, "v3": top}, precision=prec,
                                       f0=40.0, t0=1.2 / 40.0))
    return out


def _run(pkg, ws, batched, graph_steps, chunks, family="line", zchunk_log2=0):
    g = pkg.Grid.from_workloads(ws)
    g.set_kernels(family)
    if zchunk_log2:  # z positions per warp row of the convolution z tiles (Z1 and Z2)
        g.set_tile("acoustic_z", 0, zchunk_log2)
        g.set_tile("acoustic_z2", 0, zchunk_log2)
    g.set_schedule(batched, graph_steps)
    for c in chunks:
        g.step(c)
    fields = [{f: g.get_field(s, f) for f in ("sigma", "v1", "v3")} for s in range(len(ws))]
    traces = [g.record(s) for s in range(len(ws))]
    steps = [g.get_step(s) for s in range(len(ws))]
    g.close()
    return fields, traces, steps


def _assert_same(a, b):
    fa, ta, sa = a
    fb, tb, sb = b
    assert sa == sb
    for s in range(len(fa)):
        for f in fa[s]:
            assert np.array_equal(fa[s][f], fb[s][f]), (s, f, np.abs(fa[s][f] - fb[s][f]).max())
        for f in ta[s]:
            assert np.array_equal(ta[s][f], tb[s][f]), (s, f)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_kahan"])
def test_batched_equals_per_shot(pkg, prec):
    ws = _shots(prec)
    ref = _run(pkg, ws, False, 0, [17, 23])
    _assert_same(_run(pkg, ws, True, 0, [17, 23]), ref)


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_graph_replay_equals_per_shot(pkg, prec):
    """Graphs of 7 steps: 17 = 2 replays + 3 plain steps, then 23 = 3 replays + 2 plain steps."""
    ws = _shots(prec)
    ref = _run(pkg, ws, False, 0, [17, 23])
    _assert_same(_run(pkg, ws, True, 7, [17, 23]), ref)


@pytest.mark.parametrize("zchunk_log2", [4, 3])
@pytest.mark.parametrize("prec", ["fp32", "fp32_kahan"])
def test_batched_convolution_equals_per_shot(pkg, prec, zchunk_log2):
    ws = _conv_shots(prec)
    ref = _run(pkg, ws, False, 0, [17, 23], "convolution", zchunk_log2)
    _assert_same(_run(pkg, ws, True, 0, [17, 23], "convolution", zchunk_log2), ref)
    _assert_same(_run(pkg, ws, True, 7, [17, 23], "convolution", zchunk_log2), ref)


def test_batched_convolution_against_oracle(pkg):
    ws = _conv_shots("fp32_kahan")
    g = pkg.Grid.from_workloads(ws)
    g.set_schedule(True, 5)
    g.step(40)
    for s, w in enumerate(ws):
        sim = Simulation(dataclasses.replace(w, precision="fp64")).step(40)
        for f in ("sigma", "v1", "v3"):
            ref = sim.state[f]
            err = np.linalg.norm(g.get_field(s, f).astype(np.float64) - ref) / np.linalg.norm(ref)
            assert err < 1e-5, (s, f, err)
    g.close()


def test_graph_single_shot(pkg):
    ws = _shots("fp32")[:1]
    ref = _run(pkg, ws, False, 0, [12, 9])
    _assert_same(_run(pkg, ws, False, 4, [12, 9]), ref)


def test_batched_fp64_against_oracle(pkg):
    ws = _shots("fp64")
    g = pkg.Grid.from_workloads(ws)
    g.set_schedule(True, 5)
    g.step(40)
    for s, w in enumerate(ws):
        sim = Simulation(w).step(40)
        for f in ("sigma", "v1", "v3"):
            ref = sim.state[f]
            err = np.linalg.norm(g.get_field(s, f) - ref) / np.linalg.norm(ref)
            assert err < 1e-11, (s, f, err)
        rec = g.record(s)
        for f in ("sigma", "v1", "v3"):
            # the direct wave has not reached the top row yet: traces are measured against the field's scale
            ref = sim.trace_array(f)
            assert np.abs(rec[f] - ref).max() <= 1e-11 * np.abs(sim.state[f]).max(), (s, f)
    g.close()


@pytest.mark.parametrize("family", ["line", "convolution"])
def test_interleaved_reads_and_records(pkg, family):
    """Velocity reads (which bring a shot back to integer time), trace reads and a state round trip between
    graph-replayed batched runs give the same results as the same sequence on the per-shot schedule."""
    ws = _shots("fp64") if family == "line" else _conv_shots("fp32_kahan")

    def seq(batched, graph_steps):
        g = pkg.Grid.from_workloads(ws)
        g.set_kernels(family)
        g.set_schedule(batched, graph_steps)
        g.step(10)
        v = g.get_field(1, "v1")
        blob = g.get_state()
        tr1 = [g.record(s) for s in range(3)]
        g.step(8)
        g.set_state(blob)  # back to step 10; the 8 trace rows stay recorded
        g.step(20)
        tr2 = [g.record(s) for s in range(3)]
        out = [v] + [g.get_field(s, f) for s in range(3) for f in ("sigma", "v1", "v3")]
        out += [t[f] for t in tr1 + tr2 for f in ("sigma", "v1", "v3")]
        steps = [g.get_step(s) for s in range(3)]
        g.close()
        return out, steps

    a, sa = seq(False, 0)
    b, sb = seq(True, 6)
    assert sa == sb == [30, 30, 30]
    assert len(a) == len(b)
    for i, (x, y) in enumerate(zip(a, b)):
        assert x.shape == y.shape and np.array_equal(x, y), i


def test_autotune(pkg):
    ws = _shots("fp32_kahan")
    g = pkg.Grid.from_workloads(ws)
    res = g.autotune(steps=2)
    assert set(res) == {"acoustic_x", "acoustic_z"}  # a patch length of 12 keeps these shots on the line kernels
    for r in res.values():
        assert r["threads_per_block"] in (128, 256, 512, 1024) and r["chunk_log2"] in (3, 4) and r["ms"] > 0
    assert g.get_step(0) == 0 and not g.get_field(0, "sigma").any()
    g.step(40)
    for s, w in enumerate(ws):
        sim = Simulation(w).step(40)
        ref = sim.state["sigma"]
        assert np.linalg.norm(g.get_field(s, "sigma") - ref) / np.linalg.norm(ref) < 1e-5
    g.close()


def test_autotune_convolution(pkg):
    """Shots that take the convolution kernels: the z chunk of Z1 and Z2 is tuned too, and the tuned handle still
    equals the per-shot schedule with the same shapes."""
    ws = _conv_shots("fp32_kahan")
    g = pkg.Grid.from_workloads(ws)
    res = g.autotune(steps=2)
    assert set(res) == {"acoustic_x", "acoustic_z", "acoustic_z2"}
    for k in ("acoustic_z", "acoustic_z2"):
        assert res[k]["chunk_log2"] in (3, 4) and res[k]["ms"] > 0
    g.step(17)
    r = pkg.Grid.from_workloads(ws)
    r.set_schedule(False, 0)
    for k in ("acoustic_z", "acoustic_z2"):
        r.set_tile(k, 0, res[k]["chunk_log2"])
    r.step(17)
    for s in range(len(ws)):
        for f in ("sigma", "v1", "v3"):
            assert np.array_equal(g.get_field(s, f), r.get_field(s, f)), (s, f)
    g.close()
    r.close()


@pytest.mark.parametrize("family", ["convolution", "line"])
def test_full_survey_batched(pkg, family):
    """The 64-shot survey (n from 512 to 2048, M = 128, n_nb = 20, 40-point layers, FP32): three graph-replayed
    steps equal the per-shot schedule of the same kernel family exactly on every shot, and the smallest and
    largest shots match the FP64 oracle after the same steps."""
    ws = batched_shots(steps=3)
    g = pkg.Grid.from_workloads(ws)
    g.set_kernels(family)
    g.set_schedule(True, 3)
    g.step(3)
    r = pkg.Grid.from_workloads(ws)
    r.set_kernels(family)
    r.set_schedule(False, 0)
    r.step(3)
    for s in range(len(ws)):
        a, b = g.get_field(s, "sigma"), r.get_field(s, "sigma")
        assert np.array_equal(a, b), s
        assert np.array_equal(g.record(s)["sigma"], r.record(s)["sigma"]), s
    r.close()
    sizes = [w.n[0] for w in ws]
    for s in (int(np.argmin(sizes)), int(np.argmax(sizes))):
        sim = Simulation(dataclasses.replace(ws[s], precision="fp64")).step(3)
        ref = sim.state["sigma"]
        err = np.linalg.norm(g.get_field(s, "sigma").astype(np.float64) - ref) / np.linalg.norm(ref)
        assert err < 1e-5, (s, err)
    g.close()

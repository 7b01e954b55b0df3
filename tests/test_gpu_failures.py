"""Failure detection through the C ABI, in forms that fault, trap or hang no GPU.

* Bounded waits: with a wait limit of 0 polls every staged x-kernel block gives up on its first row at once (the
  wait's phase cannot have completed), drains its own bulk copies in flight (a bounded wait on copies that do
  complete), sets the device error flag and stops.  loss_sync must report LOSS_E_TIMEOUT, the handle must then be
  poisoned, and the CUDA context must stay usable (a fresh handle still matches the oracle).
* Non-finite watchdog: a NaN or Inf planted with loss_set_field is reported by loss_sync as LOSS_E_NUMERIC, with
  the field, without poisoning the handle; a finite run with the watchdog on reports nothing.
* FP64 widening of FP32 samples in the PMBC sums keeps Inf and NaN non-finite.
* Allocation failure: an allocator callback that fails the k-th allocation makes loss_create_grid return
  LOSS_E_NOMEM with a NULL handle, after freeing every allocation it made."""
import ctypes
import dataclasses

import numpy as np
import pytest

from oracle.wave import Simulation
from synth import acoustic2d_small, batched_shots, elastic3d_homogeneous

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge

    ge.build()
    import paper_2301_05127_gb300 as p

    return p


def _status(pkg, fn):
    try:
        fn()
    except pkg.LossError as e:
        return e.status
    return pkg.LOSS_OK


@pytest.mark.parametrize("batched", [False, True])
def test_wait_limit_gives_timeout_and_poisons_the_handle(pkg, batched):
    if batched:
        ws = [dataclasses.replace(w, precision="fp32") for w in batched_shots(n_shots=3, steps=4)]
    else:
        ws = [acoustic2d_small(n=128, p=2, steps=4)]
        ws = [dataclasses.replace(ws[0], precision="fp32_kahan")]
    g = pkg.Grid.from_workloads(ws)
    g.set_wait_limit(0)
    g.step(2)
    assert _status(pkg, g.sync) == pkg.LOSS_E_TIMEOUT
    assert b"gave up" in pkg.lib().loss_last_error(g.h)
    # poisoned: every later call on the handle reports the same error; destroy still works
    assert _status(pkg, lambda: g.step(1)) == pkg.LOSS_E_TIMEOUT
    assert _status(pkg, lambda: g.get_field(0, "sigma")) == pkg.LOSS_E_TIMEOUT
    g.close()
    # the context is still usable: a fresh handle with the default limit runs and matches the oracle
    w = dataclasses.replace(acoustic2d_small(n=128, p=2, steps=20), precision="fp32_kahan")
    h = pkg.Grid.from_workloads([w])
    h.set_wait_limit(0)
    h.set_wait_limit(-1)
    h.step(20)
    h.sync()
    sim = Simulation(dataclasses.replace(w, precision="fp64")).step(20)
    ref = sim.state["sigma"]
    assert np.linalg.norm(h.get_field(0, "sigma") - ref) / np.linalg.norm(ref) < 1e-5
    h.close()


@pytest.mark.parametrize("prec,bad", [("fp32_kahan", np.nan), ("fp64", np.inf), ("fp32", -np.inf)])
def test_watchdog_reports_non_finite_field(pkg, prec, bad):
    w = dataclasses.replace(acoustic2d_small(n=64, p=2, steps=10, n_nb=12, pml_width=10), precision=prec)
    g = pkg.Grid.from_workloads([w])
    clean = g.get_state()
    g.set_watchdog(4)
    v1 = np.zeros(w.shape)
    v1[30, 17] = bad
    g.set_field(0, "v1", v1)
    g.step(3)
    assert _status(pkg, g.sync) == pkg.LOSS_OK  # no check yet (3 < 4 steps)
    g.step(3)
    assert _status(pkg, g.sync) == pkg.LOSS_E_NUMERIC
    msg = pkg.lib().loss_last_error(g.h).decode()
    assert "shot 0" in msg and "field" in msg
    g.sync()  # the report cleared the flag; the handle is not poisoned
    g.set_state(clean)  # fields, compensation and layer memory back to the finite start
    g.step(8)
    g.sync()
    assert np.isfinite(g.get_field(0, "sigma")).all()
    g.close()


def test_watchdog_quiet_on_a_finite_run(pkg):
    ws = [elastic3d_homogeneous(n=24, p=2, steps=6, n_nb=8, pml_width=4)]
    g = pkg.Grid.from_workloads(ws)
    g.set_watchdog(1)
    g.profile(True)
    for _ in range(6):
        g.step(1)
    g.sync()
    assert g.profile_read("watch")[1] == 6 * 9  # after every step, nine fields
    g.close()


def test_phi_sums_keep_inf_and_nan(pkg):
    """FP32 samples are widened to FP64 on the integer units for the PMBC sums; Inf and NaN must stay non-finite
    there (a finite stand-in would hide a diverged field in phi)."""
    w = dataclasses.replace(acoustic2d_small(n=64, p=2, steps=1, n_nb=12, pml_width=0), precision="fp32")
    g = pkg.Grid.from_workloads([w])
    f = np.random.default_rng(3).standard_normal(w.shape).astype(np.float32)
    f[5, 32 + 3] = np.inf   # inside the window of the junction at x = 32 on row 5
    f[9, 32 - 2] = np.nan   # row 9
    phi = g.pmbc_phi(0, 1, f)  # [lines][p + 1]
    assert not np.isfinite(phi[5, 1]) and not np.isfinite(phi[9, 1])
    assert np.isfinite(np.delete(phi, [5, 9], axis=0)).all()
    g.close()


def test_allocation_failure_gives_nomem_and_frees_everything(pkg):
    import torch

    L = pkg.lib()
    w = acoustic2d_small(n=64, p=2, steps=1, n_nb=12)
    d = pkg.make_desc(2, pkg.LOSS_ACOUSTIC, pkg.LOSS_FP32_KAHAN, w.n_nb, w.n, w.p, w.h, w.dt)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    state = {"fail_at": 0, "calls": 0, "live": set()}

    def alloc(ctx, nbytes, s):
        state["calls"] += 1
        if state["calls"] == state["fail_at"]:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), stream=torch.cuda.current_stream())
        state["live"].add(p)
        return p

    def free(ctx, ptr, s):
        state["live"].discard(ptr)
        torch.cuda.caching_allocator_delete(ptr)

    a_fn, f_fn = pkg.ALLOC_FN(alloc), pkg.FREE_FN(free)
    allocator = pkg.Allocator(None, a_fn, f_fn)
    descs = (pkg.GridDesc * 1)(d)

    def create():
        h = ctypes.c_void_p()
        st = L.loss_create_grid(descs, 1, ctypes.byref(allocator), stream, ctypes.byref(h))
        return st, h

    st, h = create()  # count the allocations of a successful creation
    assert st == pkg.LOSS_OK and h.value
    n_alloc = state["calls"]
    assert n_alloc >= 3
    assert L.loss_destroy(h) == pkg.LOSS_OK
    assert not state["live"]
    for k in sorted({1, 2, n_alloc // 2, n_alloc}):
        state.update(fail_at=k, calls=0)
        st, h = create()
        assert st == pkg.LOSS_E_NOMEM, (k, st)
        assert not h.value
        assert not state["live"], k  # everything allocated before the failure was freed
    torch.cuda.synchronize()

"""Oracle, part 5: the Strang steps of ``wave.Simulation`` with their derivative terms spread over worker
processes.  TEST INFRASTRUCTURE ONLY (golden runs at full size and the timed CPU baseline).

Nothing here is new arithmetic.  Every derivative term of a sub-step (Sec. 3.3: tau times the LOSS derivative
of one field along one axis, through the exact ADE-PML sub-flow inside the layers) is computed by the oracle's
own ``Operator.Dc`` and ``PML.advance`` on a slab of whole grid lines: the derivative along axis a needs whole
lines along a, so the slab is cut along another axis.  Each grid line is then processed exactly as in the
serial run, and the memory variables are advanced in place.  The parent process combines the terms with the same
expressions, in the same order, as ``wave.acoustic_step`` and ``wave.elastic_step``, so a run here equals the
serial oracle bit for bit (tested on small grids).

State, memory variables and term outputs live in shared memory; workers are started with the ``spawn`` method
(safe after a CUDA context exists in the parent).
"""
from __future__ import annotations

import math
import multiprocessing as mp
import os
import time
from multiprocessing import shared_memory
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import wave

_W: dict = {}  # per-worker globals


def _views(spec: Dict[str, Tuple[str, tuple]]):
    shms, arrays = [], {}
    for key, (shm_name, shape) in spec.items():
        shm = shared_memory.SharedMemory(name=shm_name)
        shms.append(shm)
        arrays[key] = np.ndarray(shape, dtype=np.float64, buffer=shm.buf)
    return shms, arrays


def _worker_init(spec, geom, pml):
    _W["shms"], _W["arrays"] = _views(spec)
    _W["op"] = wave.Operator(*geom)
    _W["pml"] = pml


def _slab(dim: int, axis: int, lo: int, hi: int):
    sl = [slice(None)] * dim
    sl[axis] = slice(lo, hi)
    return tuple(sl)


def _worker_term(task):
    """One term on one slab: out = Dc(field) (no layer) or the PML sub-flow's increment X (layer)."""
    f_key, comp, tau, mem_key, out_key, slab_axis, lo, hi = task
    A, op, pml = _W["arrays"], _W["op"], _W["pml"]
    sl = _slab(op.dim, slab_axis, lo, hi)
    g = op.Dc(A[f_key][sl], comp)
    if mem_key is None:
        A[out_key][sl] = g
    else:
        A[out_key][sl] = pml.advance(A[mem_key][sl], g, wave.component_axis(comp, op.dim), tau)
    return os.getpid(), time.process_time()


class ParallelSimulation(wave.Simulation):
    """``wave.Simulation`` whose step evaluates the independent derivative terms of each sub-step in ``workers``
    processes.  Use as a context manager (or call ``close``) to release the pool and the shared memory."""

    def __init__(self, w, workers: Optional[int] = None, state=None, model=None):
        super().__init__(w, state=state, model=model)
        self.workers = int(workers or max(1, (os.cpu_count() or 2) - 1))
        self._shms: List[shared_memory.SharedMemory] = []
        spec = {}

        def share(key, arr):
            shm = shared_memory.SharedMemory(create=True, size=max(8, arr.nbytes))
            self._shms.append(shm)
            view = np.ndarray(arr.shape, dtype=np.float64, buffer=shm.buf)
            view[...] = arr
            spec[key] = (shm.name, arr.shape)
            return view

        for k in list(self.state):
            self.state[k] = share(k, self.state[k])
        if self.mem is not None:
            for k in list(self.mem):
                self.mem[k] = share("mem:" + k, self.mem[k])
        n_out = 9 if w.physics == "elastic" else w.dim
        self.out = [share(f"out:{i}", np.zeros(w.shape)) for i in range(n_out)]
        geom = (w.n, w.p, w.h, w.n_nb)
        self._pool = mp.get_context("spawn").Pool(self.workers, initializer=_worker_init,
                                                  initargs=(spec, geom, self.pml))
        self._spec = spec
        self._worker_cpu: Dict[int, float] = {}

    # -- pool plumbing -------------------------------------------------------------------------------------------
    def close(self):
        if self._pool is not None:
            self._pool.close()
            self._pool.join()
            self._pool = None
        # Detach every view before the blocks are closed.
        for k in list(self.state):
            self.state[k] = np.array(self.state[k])
        if self.mem is not None:
            for k in list(self.mem):
                self.mem[k] = np.array(self.mem[k])
        self.out = []
        for shm in self._shms:
            shm.close()
            shm.unlink()
        self._shms = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _terms(self, specs):
        """specs: list of (field key, comp, tau, mem key or None).  Returns one shared output view per term,
        holding Dc(field) (mem key None) or the sub-flow increment X of PML.advance."""
        dim = self.op.dim
        # Slabs of about 1 MB keep each task's temporaries in the host's cache; at least 3 tasks per worker.
        field_bytes = 8 * int(np.prod(self.w.shape))
        per = max(math.ceil(3 * self.workers / len(specs)), math.ceil(field_bytes / (1 << 20)))
        tasks = []
        for t, (f_key, comp, tau, mem_key) in enumerate(specs):
            a = wave.component_axis(comp, dim)
            slab_axis = 0 if a != 0 else 1
            ext = self.w.shape[slab_axis]
            cuts = np.linspace(0, ext, min(per, ext) + 1).round().astype(int)
            for lo, hi in zip(cuts[:-1], cuts[1:]):
                if hi > lo:
                    tasks.append((f_key, comp, tau, None if mem_key is None else "mem:" + mem_key, f"out:{t}",
                                  slab_axis, int(lo), int(hi)))
        for pid, cpu in self._pool.map(_worker_term, tasks, chunksize=1):
            self._worker_cpu[pid] = max(self._worker_cpu.get(pid, 0.0), cpu)
        return self.out[:len(specs)]

    def cpu_time(self) -> float:
        """CPU seconds used so far by this process and by the workers (as of their last finished task)."""
        return time.process_time() + sum(self._worker_cpu.values())

    # -- the steps: same expressions, same order as wave.acoustic_step / wave.elastic_step ------------------------
    def _acoustic_half_A(self, tau):
        st, b, pml = self.state, self.b, self.pml
        names = wave._velocity_names(self.op.dim)
        specs = [("sigma", comp, tau, None if pml is None else f"psi{comp}") for _, comp in names]
        outs = self._terms(specs)
        for (name, _), out in zip(names, outs):
            if pml is None:
                np.copyto(st[name], st[name] - tau * b * out)
            else:
                np.copyto(st[name], st[name] + b * out)

    def _acoustic_B(self, dt, t_half):
        st, kappa, pml, src = self.state, self.kappa, self.pml, self.src
        names = wave._velocity_names(self.op.dim)
        if pml is None:
            outs = self._terms([(name, comp, dt, None) for name, comp in names])
            div = sum(o for o in outs)
            np.copyto(st["sigma"], st["sigma"] - dt * kappa * div)
        else:
            outs = self._terms([(name, comp, dt, f"phi{comp}") for name, comp in names])
            inc = 0.0
            for o in outs:
                inc = inc + o
            np.copyto(st["sigma"], st["sigma"] + kappa * inc)
        if src is not None and "pressure" in src.kinds:
            src.add(st["sigma"], dt, t_half)

    def _elastic_half_A(self, tau, t):
        st, b, pml, src = self.state, self.b, self.pml, self.src
        specs = [(wave._SIG[(i, j)], j, tau, None if pml is None else f"psi_{i}{j}") for i in (1, 2, 3)
                 for j in (1, 2, 3)]
        outs = self._terms(specs)
        for i in (1, 2, 3):
            terms = [(tau * o if pml is None else -o) for o in outs[3 * (i - 1):3 * i]]
            acc = sum(x for x in terms)
            np.copyto(st[f"v{i}"], st[f"v{i}"] + b * acc)
        if src is not None:
            for i, kind in ((1, "force_x"), (2, "force_y"), (3, "force_z")):
                if kind in src.kinds:
                    st[f"v{i}"][src.block] += tau * b[src.block] * wave.ricker(t, src.f0, src.t0) * src.profile

    def _elastic_B(self, dt, t_half):
        st, lam, mu, pml, src = self.state, self.lam, self.mu, self.pml, self.src
        pairs = [(i, j) for i in (1, 2, 3) for j in (1, 2, 3)]
        specs = [(f"v{i}", j, dt, None if pml is None else f"phi_{i}{j}") for i, j in pairs]
        outs = self._terms(specs)
        x = {ij: (dt * o if pml is None else -o) for ij, o in zip(pairs, outs)}
        tr = x[1, 1] + x[2, 2] + x[3, 3]
        for i in (1, 2, 3):
            np.copyto(st[f"s{i}{i}"], st[f"s{i}{i}"] + (lam * tr + 2.0 * mu * x[i, i]))
        for (i, j) in ((1, 2), (1, 3), (2, 3)):
            np.copyto(st[f"s{i}{j}"], st[f"s{i}{j}"] + mu * (x[i, j] + x[j, i]))
        if src is not None:
            if "explosive" in src.kinds:
                for k in ("s11", "s22", "s33"):
                    src.add(st[k], dt, t_half)
            if "shear_xz" in src.kinds:
                src.add(st["s13"], dt, t_half)

    def step(self, count: int = 1, record: bool = True):
        w = self.w
        for _ in range(count):
            t_n = self.step_index * w.dt
            if w.physics == "acoustic":
                self._acoustic_half_A(0.5 * w.dt)
                self._acoustic_B(w.dt, t_n + 0.5 * w.dt)
                self._acoustic_half_A(0.5 * w.dt)
            else:
                self._elastic_half_A(0.5 * w.dt, t_n)
                self._elastic_B(w.dt, t_n + 0.5 * w.dt)
                self._elastic_half_A(0.5 * w.dt, t_n + w.dt)
            self.step_index += 1
            if record:
                for k, idx in w.receivers.items():
                    self.traces[k].append(self.state[k].reshape(-1)[idx].copy())
        return self

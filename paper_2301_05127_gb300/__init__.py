"""Python binding of libloss, the sm_103a implementation of the LOSS time step (arXiv 2301.05127).

Argument marshalling only: every step of the method runs in the CUDA kernels behind include/loss.h.  The
functions of the C ABI are exposed under their C names (``loss_create_grid``, ``loss_step`` ...) through
``lib()``; the ``Grid`` class wraps a handle with numpy / torch conveniences.  The first call into the library
raises ImportError when the shared library has not been built (``python -m paper_2301_05127_gb300.build`` or
``__graft_entry__.build()``): there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libloss.so")

LOSS_OK, LOSS_E_ARG, LOSS_E_SHAPE, LOSS_E_NOMEM, LOSS_E_CUDA, LOSS_E_STATE, LOSS_E_TIMEOUT, LOSS_E_NUMERIC, \
    LOSS_E_UNSUPPORTED = range(9)
LOSS_ACOUSTIC, LOSS_ELASTIC = 0, 1
LOSS_FP64, LOSS_FP32, LOSS_FP32_KAHAN = 0, 1, 2
LOSS_MEM_HOST, LOSS_MEM_DEVICE = 0, 1
LOSS_SRC_PRESSURE, LOSS_SRC_EXPLOSIVE, LOSS_SRC_SHEAR_XZ, LOSS_SRC_FORCE_Z, LOSS_SRC_FORCE_X, LOSS_SRC_FORCE_Y = \
    1, 2, 4, 8, 16, 32
FIELDS = {"v1": 0, "v2": 1, "v3": 2, "s11": 3, "s22": 4, "s33": 5, "s12": 6, "s13": 7, "s23": 8, "sigma": 3}
PRECISIONS = {"fp64": LOSS_FP64, "fp32": LOSS_FP32, "fp32_kahan": LOSS_FP32_KAHAN}
SOURCE_KINDS = {"pressure": LOSS_SRC_PRESSURE, "explosive": LOSS_SRC_EXPLOSIVE, "shear_xz": LOSS_SRC_SHEAR_XZ,
                "force_z": LOSS_SRC_FORCE_Z, "force_x": LOSS_SRC_FORCE_X, "force_y": LOSS_SRC_FORCE_Y}


class GridDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("physics", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("n_nb", ctypes.c_int32), ("n", ctypes.c_int64 * 3), ("p", ctypes.c_int32 * 3),
                ("h", ctypes.c_double * 3), ("dt", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("threads_per_block", ctypes.c_int32), ("chunk_log2", ctypes.c_int32),
                ("ms", ctypes.c_double)]


_lib = None
_H = ctypes.c_void_p
_P = ctypes.c_void_p
_I32, _I64, _U32, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double

_PROTOS = {
    "loss_version": (ctypes.c_char_p, []),
    "loss_status_str": (ctypes.c_char_p, [_I32]),
    "loss_last_error": (ctypes.c_char_p, [_H]),
    "loss_create_grid": (_I32, [ctypes.POINTER(GridDesc), _I32, ctypes.POINTER(Allocator), _P, ctypes.POINTER(_H)]),
    "loss_destroy": (_I32, [_H]),
    "loss_set_model": (_I32, [_H, _I32, _P, _P, _P, _I32]),
    "loss_set_source": (_I32, [_H, _I32, ctypes.POINTER(_I64), _U32, _D, _D, _D]),
    "loss_set_receivers": (_I32, [_H, _I32, _I32, _P, _I64, _I32]),
    "loss_set_pml": (_I32, [_H, _I32, _I32, _D, _D, _D]),
    "loss_set_field": (_I32, [_H, _I32, _I32, _P, _I32]),
    "loss_get_field": (_I32, [_H, _I32, _I32, _P, _I32]),
    "loss_step": (_I32, [_H, _I64]),
    "loss_record_count": (_I32, [_H, _I32, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "loss_record": (_I32, [_H, _I32, _P, _I32]),
    "loss_derivative": (_I32, [_H, _I32, _I32, _P, _P, _P, _I32]),
    "loss_pmbc_phi": (_I32, [_H, _I32, _I32, _P, _P, _I32]),
    "loss_derivative_adjoint": (_I32, [_H, _I32, _I32, _P, _P, _I32]),
    "loss_gradient": (_I32, [_H, _I32, _P, _I32, _I64, ctypes.POINTER(_D), _P, _P, _P, _I32]),
    "loss_get_state": (_I32, [_H, _P, ctypes.POINTER(ctypes.c_size_t)]),
    "loss_set_state": (_I32, [_H, _P, ctypes.c_size_t]),
    "loss_get_step": (_I32, [_H, _I32, ctypes.POINTER(_I64)]),
    "loss_sync": (_I32, [_H]),
    "loss_derivative_noalloc": (_I32, [ctypes.POINTER(GridDesc), _I32, _P, _P, _P]),
    "loss_set_launch": (_I32, [_H, _I32, _I32, _I32]),
    "loss_set_tile": (_I32, [_H, _I32, _I32, _I32]),
    "loss_set_schedule": (_I32, [_H, _I32, _I32]),
    "loss_set_kernels": (_I32, [_H, _I32]),
    "loss_autotune": (_I32, [_H, _I32, ctypes.POINTER(TuneEntry), _I32, ctypes.POINTER(_I32)]),
    "loss_profile": (_I32, [_H, _I32]),
    "loss_profile_read": (_I32, [_H, _I32, ctypes.POINTER(_D), ctypes.POINTER(_I64)]),
    "loss_set_wait_limit": (_I32, [_H, _I64]),
    "loss_set_watchdog": (_I32, [_H, _I64]),
    "loss_set_coordinates": (_I32, [_H, _I32, _I32, _P]),
    "loss_round_fp32_unbiased": (_I32, [_P, _P, _I64, ctypes.c_uint64]),
}
KERNELS = {"acoustic_x": 0, "acoustic_z": 1, "gather": 2, "derivative": 3, "elastic_x": 4, "elastic_y": 5,
           "elastic_z": 6, "clock": 7, "adjoint": 8, "acoustic_x2": 9, "acoustic_z2": 10, "watch": 11}
KERNEL_NAMES = {v: k for k, v in KERNELS.items()}


def lib():
    """The loaded libloss (ctypes.CDLL) with typed prototypes.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libloss not built ({LIB_PATH} missing); run __graft_entry__.build() first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class LossError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{lib().loss_status_str(status).decode()}: {msg}")
        self.status = status


def _check(st, handle=None):
    if st != LOSS_OK:
        msg = lib().loss_last_error(handle).decode() if handle else ""
        raise LossError(st, msg)


def _expect_buffer(a, shape, itemsize, what):
    """Refuse an array or tensor that does not hold exactly the grid's points in the expected element size: the
    library reads and writes the full dense extent behind a plain pointer."""
    n = int(np.prod(shape))
    size = a.size if isinstance(a, np.ndarray) else a.numel()
    esize = a.itemsize if isinstance(a, np.ndarray) else a.element_size()
    if size != n or esize != itemsize:
        raise ValueError(f"{what}: expected {n} elements of {itemsize} bytes (shape {tuple(shape)}), "
                         f"got {size} of {esize}")


def _ptr_and_mem(a):
    """(pointer, mem) of a numpy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to libloss must be C-contiguous")
        return a.ctypes.data, LOSS_MEM_HOST
    import torch
    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensors passed to libloss must be contiguous")
        return a.data_ptr(), (LOSS_MEM_DEVICE if a.is_cuda else LOSS_MEM_HOST)
    raise TypeError(type(a))


def make_desc(dim, physics, precision, n_nb, n, p, h, dt) -> GridDesc:
    d = GridDesc()
    d.dim, d.physics, d.precision, d.n_nb = dim, physics, precision, n_nb
    nn, pp, hh = list(n) + [0] * (3 - len(n)), list(p) + [1] * (3 - len(p)), list(h) + [1.0] * (3 - len(h))
    for i in range(3):
        d.n[i], d.p[i], d.h[i] = int(nn[i]), int(pp[i]), float(hh[i])
    d.dt = float(dt)
    return d


def round_fp32_unbiased(x, key0: int = 0) -> np.ndarray:
    """loss_round_fp32_unbiased: x (float64) to FP32 by deterministic unbiased rounding, as FP32 grids store
    their model coefficients (element i uses the key key0 + i)."""
    a = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty(a.shape, dtype=np.float32)
    _check(lib().loss_round_fp32_unbiased(a.ctypes.data, out.ctypes.data, a.size, int(key0)))
    return out


class _TorchAllocator:
    """Routes libloss device allocations through torch's caching allocator."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)
        self.struct = Allocator(None, self._alloc, self._free)

    def _do_alloc(self, ctx, nbytes, stream):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream)
        except Exception:  # out of memory -> NULL, the library reports LOSS_E_NOMEM
            return None

    def _do_free(self, ctx, ptr, stream):
        self.torch.cuda.caching_allocator_delete(ptr)


class Grid:
    """One libloss handle holding one or more shots on the current CUDA device."""

    def __init__(self, descs: Sequence[GridDesc], stream=None, torch_allocator: bool = True):
        import torch
        L = lib()
        self.n_shots = len(descs)
        arr = (GridDesc * self.n_shots)(*descs)
        self.descs = list(descs)
        self._alloc = _TorchAllocator(torch.cuda.current_device()) if torch_allocator else None
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        h = _H()
        st = L.loss_create_grid(arr, self.n_shots, ctypes.byref(self._alloc.struct) if self._alloc else None, sp,
                                ctypes.byref(h))
        _check(st)
        self.h = h

    # -- construction from a workload description -----------------------------------------------------------
    @classmethod
    def from_workloads(cls, workloads, precision: Optional[str] = None, **kw) -> "Grid":
        descs = []
        for w in workloads:
            prec = PRECISIONS[precision or w.precision]
            phys = LOSS_ELASTIC if w.physics == "elastic" else LOSS_ACOUSTIC
            descs.append(make_desc(w.dim, phys, prec, w.n_nb, w.n, w.p, w.h, w.dt))
        g = cls(descs, **kw)
        g.workloads = list(workloads)
        for s, w in enumerate(workloads):
            vp, vs, rho = w.model()
            g.set_model(s, vp, vs, rho)
            if w.src_kinds:
                mask = 0
                for k in w.src_kinds:
                    mask |= SOURCE_KINDS[k]
                idx = list(w.src_index)
                if w.dim == 2:
                    idx = [idx[0], 0, idx[1]]
                g.set_source(s, idx, mask, w.amp, w.f0, w.t0)
            for f, ridx in w.receivers.items():
                g.set_receivers(s, f, np.asarray(ridx, dtype=np.int64))
            if getattr(w, "pml_width", 0) > 0:
                g.set_pml(s, w.pml_width, w.pml_R, w.pml_kmax, w.f0)
        return g

    @property
    def dtype(self):
        return np.float64 if self.descs[0].precision == LOSS_FP64 else np.float32

    def shape(self, shot=0):
        d = self.descs[shot]
        return tuple(int(d.n[i]) + 1 for i in range(d.dim))

    def close(self):
        if getattr(self, "h", None):
            lib().loss_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C ABI wrappers -----------------------------------------------------------------------------------------
    def set_model(self, shot, vp, vs, rho):
        """vp, vs (None for acoustic grids), rho: float64 numpy arrays or torch tensors of the grid shape."""
        if not isinstance(vp, np.ndarray):
            import torch
            cvt = lambda a: None if a is None else a.detach().to(torch.float64).contiguous()  # noqa: E731
            vp, vs, rho = cvt(vp), cvt(vs), cvt(rho)
            for name, a in (("vp", vp), ("vs", vs), ("rho", rho)):
                if a is not None:
                    _expect_buffer(a, self.shape(shot), 8, name)
            mem = LOSS_MEM_DEVICE if vp.is_cuda else LOSS_MEM_HOST
            _check(lib().loss_set_model(self.h, shot, vp.data_ptr(), None if vs is None else vs.data_ptr(),
                                        rho.data_ptr(), mem), self.h)
            return
        vp = np.ascontiguousarray(vp, dtype=np.float64)
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        vsa = None if vs is None else np.ascontiguousarray(vs, dtype=np.float64)
        for name, a in (("vp", vp), ("vs", vsa), ("rho", rho)):
            if a is not None:
                _expect_buffer(a, self.shape(shot), 8, name)
        _check(lib().loss_set_model(self.h, shot, vp.ctypes.data, None if vsa is None else vsa.ctypes.data,
                                    rho.ctypes.data, LOSS_MEM_HOST), self.h)

    def set_source(self, shot, idx3, kind_mask, amp, f0, t0):
        arr = (_I64 * 3)(*[int(i) for i in idx3])
        _check(lib().loss_set_source(self.h, shot, arr, kind_mask, amp, f0, t0), self.h)

    def set_pml(self, shot, width, R=1e-6, k_max=1.0, f0=10.0):
        _check(lib().loss_set_pml(self.h, shot, int(width), float(R), float(k_max), float(f0)), self.h)

    def set_receivers(self, shot, field, flat_idx):
        idx = np.ascontiguousarray(flat_idx, dtype=np.int64)
        _check(lib().loss_set_receivers(self.h, shot, FIELDS[field], idx.ctypes.data, idx.size, LOSS_MEM_HOST), self.h)

    def set_field(self, shot, field, arr):
        if isinstance(arr, np.ndarray):
            arr = np.ascontiguousarray(arr, dtype=self.dtype)
        _expect_buffer(arr, self.shape(shot), np.dtype(self.dtype).itemsize, field)
        ptr, mem = _ptr_and_mem(arr)
        _check(lib().loss_set_field(self.h, shot, FIELDS[field], ptr, mem), self.h)

    def get_field(self, shot, field, out=None):
        if out is None:
            out = np.empty(self.shape(shot), dtype=self.dtype)
        _expect_buffer(out, self.shape(shot), np.dtype(self.dtype).itemsize, field)
        ptr, mem = _ptr_and_mem(out)
        _check(lib().loss_get_field(self.h, shot, FIELDS[field], ptr, mem), self.h)
        return out

    def step(self, n=1):
        _check(lib().loss_step(self.h, int(n)), self.h)

    def record(self, shot=0) -> Dict[str, np.ndarray]:
        ns, nr = _I64(), _I64()
        _check(lib().loss_record_count(self.h, shot, ctypes.byref(ns), ctypes.byref(nr)), self.h)
        out = np.empty((ns.value, nr.value), dtype=self.dtype)
        _check(lib().loss_record(self.h, shot, out.ctypes.data if out.size else None, LOSS_MEM_HOST), self.h)
        res, off = {}, 0
        w = self.workloads[shot] if hasattr(self, "workloads") else None
        if w is not None:
            names = sorted(w.receivers, key=lambda k: FIELDS[k])
            for k in names:
                cnt = len(w.receivers[k])
                res[k] = out[:, off:off + cnt]
                off += cnt
        res["_all"] = out
        return res

    def derivative(self, shot, axis, f, second=False):
        """(d1, d2) of a dense field along ``axis``; numpy in -> numpy out, torch cuda in -> torch out."""
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=self.dtype)
            d1 = np.empty_like(f)
            d2 = np.empty_like(f) if second else None
        else:
            import torch
            d1 = torch.empty_like(f)
            d2 = torch.empty_like(f) if second else None
        fp, mem = _ptr_and_mem(f)
        _check(lib().loss_derivative(self.h, shot, axis, fp, _ptr_and_mem(d1)[0],
                                     None if d2 is None else _ptr_and_mem(d2)[0], mem), self.h)
        if mem == LOSS_MEM_DEVICE:
            self.sync()
        return (d1, d2) if second else d1

    def derivative_adjoint(self, shot, axis, g):
        """D^T g along ``axis`` (transpose of ``derivative``); numpy or torch cuda, like ``derivative``."""
        if isinstance(g, np.ndarray):
            g = np.ascontiguousarray(g, dtype=self.dtype)
            out = np.empty_like(g)
        else:
            out = g.new_empty(g.shape)
        gp, mem = _ptr_and_mem(g)
        _check(lib().loss_derivative_adjoint(self.h, shot, axis, gp, _ptr_and_mem(out)[0], mem), self.h)
        if mem == LOSS_MEM_DEVICE:
            self.sync()
        return out

    def gradient(self, shot, d_obs, n_steps, checkpoint_every=0):
        """Misfit 1/2 ||traces - d_obs||^2 over n_steps steps from rest and its gradient with respect to vp, vs,
        rho (loss_gradient).  d_obs: [n_steps, n_receivers] float64 (numpy, or torch on the device).  Returns
        (J, {"vp", "vs", "rho"}) with arrays of the grid shape (numpy, or torch tensors on d_obs's device)."""
        shape = self.shape(shot)
        elastic = self.descs[shot].physics == LOSS_ELASTIC
        J = _D()
        if isinstance(d_obs, np.ndarray):
            d_obs = np.ascontiguousarray(d_obs, dtype=np.float64)
            g = {k: np.zeros(shape) for k in ("vp", "vs", "rho")}
        else:
            import torch
            d_obs = d_obs.detach().to(torch.float64).contiguous()
            g = {k: torch.zeros(shape, dtype=torch.float64, device=d_obs.device) for k in ("vp", "vs", "rho")}
        dp, mem = _ptr_and_mem(d_obs)
        _check(lib().loss_gradient(self.h, shot, dp, int(checkpoint_every), int(n_steps), ctypes.byref(J),
                                   _ptr_and_mem(g["vp"])[0], _ptr_and_mem(g["vs"])[0] if elastic else None,
                                   _ptr_and_mem(g["rho"])[0], mem), self.h)
        if not elastic:
            g["vs"] = None
        return J.value, g

    def pmbc_phi(self, shot, axis, f):
        f = np.ascontiguousarray(f, dtype=self.dtype)
        d = self.descs[shot]
        lines = f.size // f.shape[axis]
        phi = np.empty((lines, int(d.p[axis]) + 1), dtype=np.float64)
        _check(lib().loss_pmbc_phi(self.h, shot, axis, f.ctypes.data, phi.ctypes.data, LOSS_MEM_HOST), self.h)
        return phi

    def get_state(self) -> bytes:
        n = ctypes.c_size_t()
        _check(lib().loss_get_state(self.h, None, ctypes.byref(n)), self.h)
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().loss_get_state(self.h, buf, ctypes.byref(n)), self.h)
        return buf.raw

    def set_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().loss_set_state(self.h, buf, len(blob)), self.h)

    def get_step(self, shot=0) -> int:
        s = _I64()
        _check(lib().loss_get_step(self.h, shot, ctypes.byref(s)), self.h)
        return s.value

    def set_launch(self, kernel, lines_per_block=0, chunk_log2=0):
        kid = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        _check(lib().loss_set_launch(self.h, kid, int(lines_per_block), int(chunk_log2)), self.h)

    def set_tile(self, kernel, threads_per_block=0, chunk_log2=0):
        kid = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        _check(lib().loss_set_tile(self.h, kid, int(threads_per_block), int(chunk_log2)), self.h)

    def set_kernels(self, family: str = "convolution"):
        """Kernel family of the per-shot FP32 2-D acoustic step: "line", "convolution" or "convolution_items"
        (loss_set_kernels)."""
        _check(lib().loss_set_kernels(self.h, {"line": 0, "convolution": 1, "convolution_items": 2}[family]),
               self.h)

    def set_schedule(self, batched: bool = True, graph_steps: int = 0):
        _check(lib().loss_set_schedule(self.h, 1 if batched else 0, int(graph_steps)), self.h)

    def autotune(self, steps: int = 3) -> Dict[str, dict]:
        """Run the library's autotuner; returns {kernel name: {threads_per_block, chunk_log2, ms}}."""
        out = (TuneEntry * 16)()
        n = _I32()
        _check(lib().loss_autotune(self.h, int(steps), out, 16, ctypes.byref(n)), self.h)
        return {KERNEL_NAMES.get(e.kernel, str(e.kernel)): {"threads_per_block": e.threads_per_block,
                                                            "chunk_log2": e.chunk_log2, "ms": e.ms}
                for e in out[:n.value]}

    def profile(self, enable: bool = True):
        _check(lib().loss_profile(self.h, 1 if enable else 0), self.h)

    def profile_read(self, kernel=-1):
        """(total_ms, launches) of one kernel id (see KERNELS) or of all kernels (-1)."""
        ms, n = _D(), _I64()
        kid = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        _check(lib().loss_profile_read(self.h, kid, ctypes.byref(ms), ctypes.byref(n)), self.h)
        return ms.value, n.value

    def set_coordinates(self, shot, axis, x):
        """Knot coordinates of a non-uniform axis (n + 1 increasing values), or None for uniform spacing
        (loss_set_coordinates)."""
        if x is None:
            _check(lib().loss_set_coordinates(self.h, shot, axis, None), self.h)
            return
        xs = np.ascontiguousarray(x, dtype=np.float64)
        _check(lib().loss_set_coordinates(self.h, shot, axis, xs.ctypes.data), self.h)

    def set_wait_limit(self, polls: int = -1):
        """Poll limit of the staged x kernels' bounded waits (-1 = default, 0 = give up at once)
        (loss_set_wait_limit)."""
        _check(lib().loss_set_wait_limit(self.h, int(polls)), self.h)

    def set_watchdog(self, every_steps: int):
        """Non-finite check of every field every ``every_steps`` steps (0 = off) (loss_set_watchdog)."""
        _check(lib().loss_set_watchdog(self.h, int(every_steps)), self.h)

    def sync(self):
        _check(lib().loss_sync(self.h), self.h)

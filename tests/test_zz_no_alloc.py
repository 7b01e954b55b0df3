"""loss_derivative_noalloc, the derivative entry point for callers that cannot allocate device memory (for
example code running under another framework's allocator, which owns every device allocation).  It keeps its
tables in a static device array instead of handle-owned memory.  Both paths launch the same kernel with the same
tables, so its output must equal the handle-based loss_derivative's bit for bit, also when two calls with
different grids come one after the other (the second rewrites the shared tables)."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [
    # dim, n, p, n_nb, h, precision, axis
    (2, (64, 96), (2, 3), 12, (1.0, 0.5), "fp32", 1),
    (3, (24, 32, 40), (2, 2, 4), 10, (1.0, 1.5, 0.5), "fp64", 0),
]


def test_noalloc_matches_handle_derivative_on_two_calls_in_a_row():
    import torch

    import __graft_entry__ as ge

    ge.build()
    import paper_2301_05127_gb300 as pkg

    L = pkg.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    refs, outs, descs = [], [], []
    rng = np.random.default_rng(42)
    for dim, n, p, n_nb, h, prec, axis in CASES:
        d = pkg.make_desc(dim, pkg.LOSS_ACOUSTIC, pkg.PRECISIONS[prec], n_nb, n, p, h, 1e-3)
        g = pkg.Grid([d])
        f = rng.standard_normal(g.shape()).astype(g.dtype)
        refs.append(g.derivative(0, axis, f))
        g.close()
        ft = torch.from_numpy(f).cuda()
        outs.append((ft, torch.empty_like(ft), axis, prec))
        descs.append(d)
    torch.cuda.synchronize()
    for d, (ft, out, axis, _) in zip(descs, outs):  # two calls in a row, different grids and precisions
        d.dt = 0.0  # only the geometry is read: an unset time step is accepted
        st = L.loss_derivative_noalloc(ctypes.byref(d), axis, ft.data_ptr(), out.data_ptr(), stream)
        assert st == pkg.LOSS_OK, L.loss_status_str(st)
    torch.cuda.synchronize()
    for ref, (_, out, _, prec) in zip(refs, outs):
        got = out.cpu().numpy()
        assert np.array_equal(got, ref), prec


def test_noalloc_rejects_tables_beyond_the_static_array():
    import torch

    import __graft_entry__ as ge

    ge.build()
    import paper_2301_05127_gb300 as pkg

    L = pkg.lib()
    # (p + 1) * (2 n_nb + 1) = 65 * 201 > 8096 weights on the x axis: rejected before any work is queued.
    d = pkg.make_desc(2, pkg.LOSS_ACOUSTIC, pkg.LOSS_FP32, 100, (100, 8192), (1, 64), (1.0, 1.0), 1e-3)
    x = torch.zeros((101, 8193), dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    st = L.loss_derivative_noalloc(ctypes.byref(d), 1, x.data_ptr(), y.data_ptr(),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == pkg.LOSS_E_UNSUPPORTED
    assert L.loss_derivative_noalloc(None, 0, x.data_ptr(), y.data_ptr(), None) == pkg.LOSS_E_ARG

"""The allocation-free backward transform against the regular one.

``sp_transform_backward_static`` serves callers that cannot allocate device
memory when they transform (for instance while a stream is being captured
into a CUDA graph, where cudaMalloc is not allowed, or when all device memory
belongs to another allocator): its intermediate buffer and twiddle tables are
fixed-size static device arrays.  This test calls it through the C ABI on
device buffers, twice in a row with different fields and sizes, and checks
each result against the FP64 oracle's backward transform (Chebyshev z, then
Fourier x, Sec. "Scaled transforms & dealiasing") and against
``sp_transform`` (which allocates its own scratch), to the FP64 transform
tolerance used elsewhere (1e-13 relative); then, after that eager set-up,
captures a call into a CUDA graph on a side stream, replays the graph and
checks the result against the oracle again.  It lives in a file of its own
that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import rb as orb
from paper_1905_10388_gb300 import _lib
from paper_1905_10388_gb300.solver import Context, RBSolver
from gpu_util import rel_err

pytestmark = pytest.mark.gpu


def _static_backward(coef, n_x, n_z, scale):
    nf = coef.shape[0]
    ngx, ngz = n_x * scale[0] // scale[1], n_z * scale[0] // scale[1]
    src = torch.from_numpy(np.ascontiguousarray(coef).view(np.float64)).cuda()
    dst = torch.empty(nf * ngz * ngx, dtype=torch.float64, device="cuda")
    err = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream().cuda_stream
    st = _lib.lib().sp_transform_backward_static(
        ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()), nf, n_x, n_z,
        scale[0], scale[1], ctypes.c_void_p(stream), err, len(err))
    assert st == _lib.SP_OK, err.value.decode()
    torch.cuda.synchronize()
    return dst.cpu().numpy().reshape(nf, ngz, ngx)


def test_static_backward_two_calls_in_a_row():
    ctx = Context(0)
    for (n_x, n_z, scale, nf, seed) in [(64, 32, (3, 2), 3, 1), (128, 64, (3, 2), 2, 2), (48, 12, (2, 1), 4, 3)]:
        rng = np.random.default_rng(seed)
        c = rng.standard_normal((nf, n_x // 2, n_z)) + 1j * rng.standard_normal((nf, n_x // 2, n_z))
        c[:, 0, :] = c[:, 0, :].real
        ngx, ngz = n_x * scale[0] // scale[1], n_z * scale[0] // scale[1]
        sysr = orb.RB2D(n_x, n_z, 1e6)
        oracle_grid = np.stack([sysr.to_grid(c[f], ngx, ngz) for f in range(nf)])
        s = RBSolver(ctx, n_x, n_z, 1e6, dealias=scale)
        ref = s.transform(c, -1, scale)
        got = _static_backward(c, n_x, n_z, scale)
        assert rel_err(got, oracle_grid) < 1e-13
        assert rel_err(got, ref) < 1e-13
    ctx.close()


def test_static_backward_inside_a_captured_graph():
    n_x, n_z, scale, nf = 64, 32, (3, 2), 3
    rng = np.random.default_rng(5)
    c = rng.standard_normal((nf, n_x // 2, n_z)) + 1j * rng.standard_normal((nf, n_x // 2, n_z))
    c[:, 0, :] = c[:, 0, :].real
    ngx, ngz = n_x * scale[0] // scale[1], n_z * scale[0] // scale[1]
    sysr = orb.RB2D(n_x, n_z, 1e6)
    oracle_grid = np.stack([sysr.to_grid(c[f], ngx, ngz) for f in range(nf)])
    _static_backward(c, n_x, n_z, scale)              # eager: the per-device set-up
    src = torch.from_numpy(np.ascontiguousarray(c).view(np.float64)).cuda()
    dst = torch.zeros(nf * ngz * ngx, dtype=torch.float64, device="cuda")
    err = ctypes.create_string_buffer(256)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        st = _lib.lib().sp_transform_backward_static(
            ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()), nf, n_x, n_z,
            scale[0], scale[1], ctypes.c_void_p(side.cuda_stream), err, len(err))
    assert st == _lib.SP_OK, err.value.decode()
    torch.cuda.synchronize()
    dst.zero_()
    graph.replay()
    torch.cuda.synchronize()
    got = dst.cpu().numpy().reshape(nf, ngz, ngx)
    assert rel_err(got, oracle_grid) < 1e-13


def test_static_backward_rejects_oversize():
    err = ctypes.create_string_buffer(256)
    st = _lib.lib().sp_transform_backward_static(
        ctypes.c_void_p(16), ctypes.c_void_p(16), 16, 1024, 512, 3, 2, None, err, len(err))
    assert st == _lib.SP_ERR_ARG
    assert b"static buffer" in err.value
    # fits the intermediate buffer, but one grid row of both fields (N_gx =
    # 4096: 256 KiB) exceeds a block's shared memory: refused before any launch
    st = _lib.lib().sp_transform_backward_static(
        ctypes.c_void_p(16), ctypes.c_void_p(16), 2, 2048, 64, 2, 1, None, err, len(err))
    assert st == _lib.SP_ERR_ARG
    assert b"shared memory" in err.value

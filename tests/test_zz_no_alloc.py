"""The allocation-free exact forward apply, against the allocating one.

Some callers must not allocate device memory while they run: serving loops that reserve all
device memory at start-up, hosts whose own allocator owns the device, and latency-bound paths
that cannot pay for cudaMalloc (it may synchronise the device).  For them the library offers
nudft2_exact_fwd_noalloc, which works in a fixed 64 MiB device array instead of requesting
workspace.  This file is collected last on purpose.  It calls the entry point through the C-ABI
twice in a row (the second call reuses the array the first one left behind) and checks both
results against nudft2_exact_apply within the exact-apply tolerance (1e-12 relative); it also
runs a size whose right-hand sides need three passes through the array, the largest size the
documented limit M*(2*nx + ny)*16 <= 64 MiB - 4 KiB accepts, and the first size it refuses.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synthetic import complex_normal, jittered_grid, random_grid  # noqa: E402

pytestmark = pytest.mark.gpu

LIMIT = (64 << 20) - 4096     # bytes of the fixed array available to M*(2*nx + ny) complex128 values


@pytest.fixture(scope="module")
def nh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_00928_b300 as m
    m.lib()
    return m


def _noalloc(nh, x, y, nx, ny, c):
    L = nh.lib()
    xt = torch.from_numpy(x).cuda().contiguous()
    yt = torch.from_numpy(y).cuda().contiguous()
    M, N = x.size, nx * ny
    cc = torch.from_numpy(c).cuda().t().contiguous()          # column major N x s
    s = cc.shape[0]
    f = torch.empty((s, M), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream()
    code = L.nudft2_exact_fwd_noalloc(ctypes.c_void_p(xt.data_ptr()), ctypes.c_void_p(yt.data_ptr()), M, nx, ny,
                                      ctypes.c_void_p(cc.data_ptr()), N, s, ctypes.c_void_p(f.data_ptr()), M,
                                      ctypes.c_void_p(stream.cuda_stream))
    stream.synchronize()                                   # the call only queues its work
    return code, f.t().cpu().numpy()


def _rel(a, b):
    return np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0))


def _check(nh, x, y, nx, ny, c):
    code, f = _noalloc(nh, x, y, nx, ny, c)
    assert code == 0, nh.lib().nudft2_last_error()
    ref = nh.exact_apply(x, y, nx, ny, nh.EXACT_FWD, torch.from_numpy(c)).cpu().numpy()
    assert _rel(f, ref) < 1e-12


def test_noalloc_matches_allocating_apply_twice(nh):
    nx, ny = 40, 24
    x, y = jittered_grid(80, 30, -0.3, 0.3, 901)
    c1 = complex_normal((nx * ny, 3), 902)
    c2 = complex_normal((nx * ny, 5), 903)
    for c in (c1, c2):                                     # two calls in a row
        _check(nh, x, y, nx, ny, c)


def test_noalloc_splits_right_hand_sides_into_chunks(nh):
    # M = 19200, nx = 64, ny = 48: the tables take 34.4 MB, one right-hand side 19.7 MB, so three
    # right-hand sides go through the array one at a time.
    nx, ny = 64, 48
    x, y = jittered_grid(160, 120, -0.3, 0.3, 906)
    assert 19200 * (nx + ny) * 16 + 2 * 19200 * nx * 16 > LIMIT
    _check(nh, x, y, nx, ny, complex_normal((nx * ny, 3), 907))


def test_noalloc_accepts_the_limit_and_refuses_past_it(nh):
    nx = ny = 43                                           # 2 nx + ny = 129
    M = 256 * 127                                          # M * 129 * 16 == 64 MiB - 4 KiB exactly
    assert M * (2 * nx + ny) * 16 == LIMIT
    x, y = random_grid(M + 1, 908)
    c = complex_normal((nx * ny, 2), 909)
    _check(nh, x[:M], y[:M], nx, ny, c)
    code, _ = _noalloc(nh, x, y, nx, ny, c)
    assert code == 1
    assert b"64 MiB" in nh.lib().nudft2_last_error()


def test_noalloc_rejects_sizes_beyond_its_workspace(nh):
    nx = ny = 256
    x, y = jittered_grid(256, 128, -0.3, 0.3, 904)        # M = 32768: 32768*768*16 B > 64 MiB
    c = complex_normal((nx * ny, 1), 905)
    code, _ = _noalloc(nh, x, y, nx, ny, c)
    assert code == 1
    assert b"64 MiB" in nh.lib().nudft2_last_error()

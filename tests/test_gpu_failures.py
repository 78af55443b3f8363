"""Failure paths, with the failure made on the host: nudft2_test_fail_alloc makes the k-th device
allocation request of the library's arenas report ENOMEM (as an exhausted device would).  The
library must return the status code, free what the failed call built, and keep the CUDA context
usable: the next build of the same problem matches the oracle.  No GPU fault is involved."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc  # noqa: E402
from synthetic import WORKLOADS, batched_uneven, make_workload  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_00928_b300 as m
    m.lib()
    yield m
    m.lib().nudft2_test_fail_alloc(0)


def _relcols(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))


@pytest.mark.parametrize("k", [1, 3, 12])
def test_enomem_during_build_is_reported_and_recoverable(nh, k):
    w = WORKLOADS["fp64_n16"]
    x, y, ct = make_workload(w)
    nh.lib().nudft2_test_fail_alloc(k)
    with pytest.raises(nh.NudftError) as e:
        nh.NudftHSS(x, y, w.nx, w.ny, eps=w.eps, levels=w.levels)
    nh.lib().nudft2_test_fail_alloc(0)
    assert e.value.code == 2 and "injected" in str(e.value)
    f = orc.forward(x, y, ct, w.nx, w.ny)
    h = nh.NudftHSS(x, y, w.nx, w.ny, eps=w.eps, levels=w.levels).factor()
    c = h.solve(torch.from_numpy(f)).cpu().numpy()
    h.close()
    assert _relcols(c, ct) < 1e-8


def test_enomem_during_factor_leaves_a_freeable_handle(nh):
    w = WORKLOADS["fp64_n32"]
    x, y, ct = make_workload(w)
    h = nh.NudftHSS(x, y, w.nx, w.ny, eps=w.eps, levels=w.levels)
    nh.lib().nudft2_test_fail_alloc(2)
    with pytest.raises(nh.NudftError) as e:
        h.factor()
    nh.lib().nudft2_test_fail_alloc(0)
    assert e.value.code == 2
    h.close()
    f = orc.forward(x, y, ct, w.nx, w.ny)
    h2 = nh.NudftHSS(x, y, w.nx, w.ny, eps=w.eps, levels=w.levels).factor()
    c = h2.solve(torch.from_numpy(f)).cpu().numpy()
    h2.close()
    assert _relcols(c, ct) < 1e-8


def test_run_batched_alone_on_the_device_reports_enomem_for_that_problem(nh):
    """With one host thread a problem that meets ENOMEM has no other problem to wait for, so its
    failure stands: the call names it, and the problems after it still run."""
    ps = batched_uneven(count=3, seed=300, sizes=(16, 24), nrhs=2)
    for p in ps:
        p.update(eps=1e-10)
    fs = [torch.from_numpy(orc.forward(p["x"], p["y"], p["c_true"], p["nx"], p["ny"])).cuda() for p in ps]
    nh.lib().nudft2_test_fail_alloc(1)
    with pytest.raises(nh.NudftError) as e:
        nh.run_batched(ps, fs, threads=1)
    nh.lib().nudft2_test_fail_alloc(0)
    assert e.value.code == 2 and "problem" in str(e.value)
    cs = nh.run_batched(ps, fs, threads=1)
    for p, c in zip(ps, cs):
        assert _relcols(c.cpu().numpy(), p["c_true"]) < 1e-8

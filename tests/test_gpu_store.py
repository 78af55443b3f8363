"""Factor store: a factored handle written by nudft2_hss_save and read back by nudft2_hss_load
solves, applies and adjoints as the saved one (its factors are byte copies; the results agree to
rounding of the kernel choices, checked at 1e-13), in FP64 and mixed precision, also after
per-level checkpointing; a truncated file is refused."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc  # noqa: E402
from synthetic import WORKLOADS, complex_normal, make_workload  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_00928_b300 as m
    m.lib()
    return m


@pytest.mark.parametrize("name,opts,checkpoint", [
    ("fp64_n32", dict(eps=1e-10), 0),
    ("fp64_n32", dict(eps=1e-10), 2),
    ("fp64_n64", dict(eps=1e-6, prec="mixed", refine_tol=1e-10, refine_max=10), 0),
])
def test_saved_handle_reloads(nh, tmp_path, name, opts, checkpoint):
    w = WORKLOADS[name]
    x, y, ct = make_workload(w)
    f = torch.from_numpy(orc.forward(x, y, ct, w.nx, w.ny))
    h = nh.NudftHSS(x, y, w.nx, w.ny, levels=w.levels, **opts).factor()
    c1 = h.solve(f).cpu().numpy()
    probe = torch.from_numpy(complex_normal((w.N, 2), 17))
    a1 = h.apply(nh.FAST_FWD, probe).cpu().numpy()
    g1 = h.apply(nh.PINV_ADJ, probe).cpu().numpy()
    if checkpoint:
        h.checkpoint(checkpoint)
    path = tmp_path / "store.bin"
    h.save(path)
    info1 = h.info()
    h.close()
    h2 = nh.NudftHSS.load(path)
    info2 = h2.info()
    assert (info2["M"], info2["nx"], info2["ny"], info2["levels"], info2["max_rank"]) == \
        (info1["M"], info1["nx"], info1["ny"], info1["levels"], info1["max_rank"])
    c2 = h2.solve(f).cpu().numpy()
    a2 = h2.apply(nh.FAST_FWD, probe).cpu().numpy()
    g2 = h2.apply(nh.PINV_ADJ, probe).cpu().numpy()
    h2.close()
    def rel(a, b):
        return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
    assert rel(c2, c1) < 1e-13
    assert rel(a2, a1) < 1e-13
    assert rel(g2, g1) < 1e-13
    assert float(np.max(np.linalg.norm(c2 - ct, axis=0) / np.linalg.norm(ct, axis=0))) < 1e-8


def test_truncated_store_and_unfactored_handle_are_refused(nh, tmp_path):
    w = WORKLOADS["fp64_n16"]
    x, y, _ = make_workload(w)
    h = nh.NudftHSS(x, y, w.nx, w.ny, eps=w.eps, levels=w.levels)
    with pytest.raises(nh.NudftError) as e:
        h.save(tmp_path / "early.bin")
    assert e.value.code == 6
    h.factor()
    path = tmp_path / "store.bin"
    h.save(path)
    h.close()
    data = path.read_bytes()
    cut = tmp_path / "cut.bin"
    cut.write_bytes(data[: len(data) - 100])
    with pytest.raises(nh.NudftError) as e:
        nh.NudftHSS.load(cut)
    assert e.value.code == 1

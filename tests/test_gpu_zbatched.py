"""Batched uneven problems: many independent point sets of different sizes built, factored and
solved together (each on its own stream).  Every batched result must equal the result of the
same problem's own handle, and recover the coefficients it was made from (consistent data,
FP64 at eps 1e-10: error ~1e-10, checked to the 1e-8 target)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc  # noqa: E402
from synthetic import batched_uneven  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_00928_b300 as m
    m.lib()
    return m


def _relcols(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))


def _problems(count, seed, **opts):
    ps = batched_uneven(count=count, seed=seed, sizes=(16, 24, 32), nrhs=3)
    for p in ps:
        p.update(opts)
        p["f"] = orc.forward(p["x"], p["y"], p["c_true"], p["nx"], p["ny"])
    return ps


def test_batched_fp64_matches_single_handles_and_truth(nh):
    ps = _problems(6, 100, eps=1e-10)
    hs = nh.build_batched(ps, threads=4)
    fs = [torch.from_numpy(p["f"]).cuda() for p in ps]
    cs = [c.cpu().numpy() for c in nh.solve_batched(hs, fs, threads=4)]
    for p, c, f in zip(ps, cs, fs):
        single = nh.NudftHSS(p["x"], p["y"], p["nx"], p["ny"], eps=1e-10).factor()
        c1 = single.solve(f).cpu().numpy()
        single.close()
        assert _relcols(c, c1) < 1e-12
        assert _relcols(c, p["c_true"]) < 1e-8
    # second batched solve: replays each handle's captured sweeps, same numbers
    cs2 = [c.cpu().numpy() for c in nh.solve_batched(hs, fs, threads=4)]
    for a, b in zip(cs, cs2):
        assert _relcols(b, a) < 1e-14
    for h in hs:
        h.close()


def test_batched_mixed_precision_refines(nh):
    ps = _problems(4, 140, eps=1e-6, prec="mixed", refine_tol=1e-10, refine_max=12)
    hs = nh.build_batched(ps, threads=4)
    cs = nh.solve_batched(hs, [torch.from_numpy(p["f"]).cuda() for p in ps], threads=4)
    for p, c in zip(ps, cs):
        assert _relcols(c.cpu().numpy(), p["c_true"]) < 1e-8
    for h in hs:
        h.close()


def test_run_batched_matches_build_and_solve(nh):
    """nudft2_hss_run_batched (each problem built, factored, solved and freed by the pool) gives the
    same c as build_batched + solve_batched, for more problems than threads, with the failing
    problem named."""
    ps = _problems(7, 200, eps=1e-10)
    fs = [torch.from_numpy(p["f"]).cuda() for p in ps]
    cs = [c.cpu().numpy() for c in nh.run_batched(ps, fs, threads=3)]
    hs = nh.build_batched(ps, threads=3)
    cs2 = [c.cpu().numpy() for c in nh.solve_batched(hs, fs, threads=3)]
    for h in hs:
        h.close()
    for p, a, b in zip(ps, cs, cs2):
        assert _relcols(a, b) < 1e-12
        assert _relcols(a, p["c_true"]) < 1e-8
    ps[4]["x"] = ps[4]["x"].copy()
    ps[4]["x"][3] = -0.25
    with pytest.raises(nh.NudftError) as e:
        nh.run_batched(ps, fs, threads=3)
    assert "problem 4" in str(e.value)


def test_batched_names_the_failing_problem(nh):
    ps = _problems(3, 170, eps=1e-10)
    ps[1]["x"] = ps[1]["x"].copy()
    ps[1]["x"][0] = 1.5                       # outside [0, 1): rejected by that problem's build
    with pytest.raises(nh.NudftError) as e:
        nh.build_batched(ps, threads=3)
    assert "problem 1" in str(e.value)


def test_config4_full_size_batch(nh):
    """The batched workload at its full size: 64 problems, n_x, n_y in {32, ..., 256}, M/N in
    [1.5, 4], 8 right-hand sides each, built, factored and solved together in mixed precision
    refined to 1e-8 (nudft2_hss_run_batched: at most 8 factorizations alive at a time).  Every problem recovers its c_true (consistent data) to the 1e-8 target, and
    the oracle's direct sum confirms the data of the largest problem at sampled points."""
    from synthetic import batched_uneven
    ps = batched_uneven()
    for p in ps:
        p.update(eps=1e-6, prec="mixed", refine_tol=1e-8, refine_max=10)
    fs = []
    for p in ps:
        ct = torch.from_numpy(p["c_true"]).cuda()
        fs.append(nh.exact_apply(torch.from_numpy(p["x"]).cuda(), torch.from_numpy(p["y"]).cuda(), p["nx"], p["ny"],
                                 nh.EXACT_FWD, ct))
    big = max(range(len(ps)), key=lambda i: ps[i]["nx"] * ps[i]["ny"])
    idx = np.random.default_rng(4).choice(ps[big]["x"].size, 16, replace=False)
    ref = orc.forward(ps[big]["x"][idx], ps[big]["y"][idx], ps[big]["c_true"], ps[big]["nx"], ps[big]["ny"])
    assert np.max(np.abs(fs[big].cpu().numpy()[idx] - ref)) < 1e-10 * np.max(np.abs(ref))
    cs = nh.run_batched(ps, fs, threads=8)   # each problem built, factored, solved and freed
    for p, c in zip(ps, cs):
        assert _relcols(c.cpu().numpy(), p["c_true"]) < 1e-8

"""The host-side retry rule of nudft2_hss_run_batched (csrc/retry.h), compiled with g++ and driven by a
simulated device-memory budget (tests/cpp/test_retry.cpp): tasks of which no two fit together all
finish, a task larger than the budget fails alone while the others finish, and with one thread a task
that does not fit fails at once."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lines(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("retry") / "test_retry")
    subprocess.run([gxx, "-std=c++17", "-O1", "-pthread", "-I", os.path.join(ROOT, "paper_2607_00928_b300", "csrc"),
                    os.path.join(ROOT, "tests", "cpp", "test_retry.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60, check=True).stdout
    return {ln.split()[0]: [int(v) for v in ln.split()[1:]] for ln in out.strip().splitlines()}


def test_pairwise_conflicting_tasks_all_finish(lines):
    assert lines["pairwise_conflict"] == [0] * 6


def test_ample_memory(lines):
    assert lines["ample"] == [0] * 4


def test_task_larger_than_the_device_fails_alone(lines):
    assert lines["too_big"] == [0, 2, 0, 0]


def test_single_thread_fails_at_once(lines):
    assert lines["single_thread"] == [2, 0]

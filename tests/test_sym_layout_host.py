"""Host logic of the symmetric streamed GEMV (CPU): the lower-triangle
layout read in block-rows (sym_layout.hpp). Compiles sym_layout_check.cpp,
which checks for every operator size up to 128 V (V = 8 bf16 / 4 fp32
entries per 16 bytes) that the closed-form row and block-row offsets equal
the sums of the padded row lengths, and that the closed-form stage end (a
quadratic solved with a float square root and integer corrections) equals
the linear search for the largest whole number of block-rows that fits a
stage, for stage sizes from one block-row to 60000 entries."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("sym") / "sym_layout_check")
    r = subprocess.run(["g++", "-O2", "-std=c++17", os.path.join(HERE, "sym_layout_check.cpp"), "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return exe


def test_block_row_offsets_and_stage_ends(checker):
    r = subprocess.run([checker, "97"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("ok")

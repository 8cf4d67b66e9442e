"""Host logic of the one-column coarse solve (CPU): the gather form of the
sweeps built from real supernodal factorisations (cube and perturbed
partitions, several levels) is emulated phase by phase in the order the
kernel works (coarse_layout_check.cpp): no read-after-write race within a
level, every value written once, A_c u = r to 1e-12, and the same u for
every launch shape (1 block, 3 blocks, 152 blocks of 16 and of 8 warps)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2410_14786_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    from paper_2410_14786_gb300 import build
    try:
        cuda_inc = build._cuda_include()
    except RuntimeError:
        pytest.skip("CUDA headers not available")
    exe = str(tmp_path_factory.mktemp("coarse") / "coarse_layout_check")
    cmd = ["g++", "-O2", "-std=c++17", "-pthread", "-I", cuda_inc, "-I", os.path.join(ROOT, "include"),
           os.path.join(HERE, "coarse_layout_check.cpp"), os.path.join(CSRC, "bddc_setup.cpp"),
           os.path.join(CSRC, "coarse_sparse.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return exe


@pytest.mark.parametrize("ne,nsub,jitter", [(24, 4, 0), (48, 8, 0), (36, 6, 1)])
def test_gather_layout_emulates_the_exact_coarse_solve(checker, ne, nsub, jitter):
    r = subprocess.run([checker, str(ne), str(nsub), str(jitter), "1:16", "3:16", "152:16", "152:8"],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("ok")


# The sparse local solver (host side): the Schur complement from the partial
# factorisation gives the dense path's K_GG, Phi_G and A_ci to 1e-10, and the
# sweeps of the merged interior forest (gather form in every launch shape,
# per-level form, block form), emulated as the kernels run them, give the
# dense A_II^-1 r of every subdomain to 1e-10. Cases: 2D and 3D cubes, a
# jittered partition (uneven subdomains), leaf size 1 (every dissection down
# to single dofs), the default leaf 32 on 32^2-element subdomains, and 12^3-
# element cubes whose fronts exceed one warp's share (large nodes in chunks).
@pytest.mark.parametrize("dim,ne,nsub,jitter,leaf", [(2, 32, 2, 0, 16), (3, 24, 3, 1, 16), (3, 16, 2, 0, 1),
                                                     (2, 64, 2, 0, 32), (3, 24, 2, 0, 32)])
def test_interior_forest_emulates_the_dense_interior_solves(checker, dim, ne, nsub, jitter, leaf):
    r = subprocess.run([checker, "local", str(dim), str(ne), str(nsub), str(jitter), str(leaf), "1:16", "3:16",
                        "152:16", "152:8"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("ok")

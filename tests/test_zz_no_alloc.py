"""bddc_apply_static_scratch: the apply whose temporaries live in a fixed
array reserved by the library, for callers that cannot let a library
allocate device memory (a host program whose own allocator owns the device,
or one that fixes all device memory at start-up). It must give the same
z = M^-1 r as bddc_apply, call after call, and refuse problems whose
temporaries do not fit the array. This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _setup(p, nrhs_max=2):
    from paper_2410_14786_gb300 import BDDC, build
    build.build()
    return BDDC.from_problem(p, precision="fp64", nrhs_max=nrhs_max)


def _call_static(g, r, z):
    from paper_2410_14786_gb300 import _lib
    L = _lib.lib()
    nrhs = 1 if r.dim() == 1 else r.shape[1]
    st = int(torch.cuda.current_stream().cuda_stream)
    return L.bddc_apply_static_scratch(g.handle, C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr()), nrhs, st)


@pytest.mark.parametrize("dim,ne,nsub", [(2, 64, 4), (3, 24, 3)])
def test_static_scratch_apply_matches_apply_twice(dim, ne, nsub):
    p = synth.make_problem(dim, ne, nsub, "lognormal", k=51)
    g = _setup(p)
    for call, seed in enumerate((61, 62)):          # two calls in a row
        r = torch.from_numpy(synth.uniform(seed, g.n_nodes * 2).reshape(-1, 2)).cuda()
        z_ref = g.apply(r)
        z = torch.full_like(r, np.nan)
        assert _call_static(g, r, z) == 0
        torch.cuda.synchronize()
        err = float((z - z_ref).abs().max() / z_ref.abs().max())
        assert err <= 1e-11, (call, err)
    g.close()


def test_static_scratch_rejects_problems_that_do_not_fit():
    # 27 subdomains of 8^3 elements with 64 right-hand sides need about
    # 3.2 million doubles of temporaries, more than the 2^20 reserved
    p = synth.make_problem(3, 24, 3, "one", k=52)
    g = _setup(p, nrhs_max=64)
    r = torch.zeros((g.n_nodes, 64), dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    assert _call_static(g, r, z) == -1
    from paper_2410_14786_gb300 import _lib
    assert b"reserved" in _lib.lib().bddc_last_error()
    g.close()

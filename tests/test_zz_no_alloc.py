"""cg_deposit_fixed_noalloc, the deposition entry point for callers that cannot allocate
device memory while they run (their memory manager owns the free memory, or
allocation after start-up is forbidden because cudaMalloc/cudaFree may synchronise
the device or fail).  Its scratch is a static device array inside the library.

Checked through the C ABI against cg_deposit in fixed-point mode and against the
oracle's fixed-point deposition (orc_deposit mode 1), which must agree bit for bit (the
deposition bar), on two calls in a row whose inputs differ, so that stale scratch from
the first call would show.  Also checked: a call leaves the device's free memory
unchanged, and particles outside the mesh give CG_EDOMAIN with the output untouched.
This file is collected last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1409_0001_gb300 as cg
    from paper_1409_0001_gb300 import build
    build.build()
    return cg, cg.load_library(), torch


def _stream(torch):
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _call_noalloc(lib, torch, dims, origin, dx, pos, w, out=None):
    nf, n = w.shape
    if out is None:
        out = torch.full((nf, int(np.prod(dims))), -1.0, dtype=torch.float64, device="cuda")
    bits = (ctypes.c_int * nf)()
    org = (ctypes.c_double * 3)(*origin)
    st = lib.cg_deposit_fixed_noalloc(dims[0], dims[1], dims[2], org, dx, n, pos.data_ptr(), nf,
                                      w.data_ptr(), out.data_ptr(), bits, _stream(torch))
    return st, out, list(bits)


def _call_deposit(cg, lib, torch, dims, origin, dx, pos, w):
    nf, n = w.shape
    mesh = cg.StructuredMesh(dims, origin, dx)
    out = torch.empty((nf, mesh.ncells), dtype=torch.float64, device="cuda")
    p = cg.Params(deposit_mode=cg.DEPOSIT_FIXED_POINT).to_c()
    rep = cg.CgReport()
    st = lib.cg_deposit(mesh.handle, n, pos.data_ptr(), nf, w.data_ptr(), out.data_ptr(),
                        ctypes.byref(p), ctypes.byref(rep), _stream(torch))
    mesh.close()
    return st, out, list(rep.fixed_point_bits)[:nf]


def test_noalloc_matches_cg_deposit_on_two_calls_in_a_row(env, orc):
    cg, lib, torch = env
    rng = np.random.default_rng(12)
    cases = [((40, 24, 17), (0.0, -0.5, 0.25), 0.05, 120_001, 3),
             ((33, 31, 29), (0.0, -0.5, 0.25), 0.05, 50_000, 5)]   # second call: new sizes
    for dims, origin, dx, n, nf in cases:
        L = np.array(dims) * dx
        pos_np = np.array(origin)[:, None] + rng.random((3, n)) * L[:, None]
        w_np = rng.standard_normal((nf, n)) * 10.0 ** rng.integers(-6, 3, (nf, 1))
        pos = torch.from_numpy(pos_np).cuda()
        w = torch.from_numpy(w_np).cuda()
        st_a, ref, bits_a = _call_deposit(cg, lib, torch, dims, origin, dx, pos, w)
        st_b, got, bits_b = _call_noalloc(lib, torch, dims, origin, dx, pos, w)
        assert st_a == 0 and st_b == 0, lib.cg_last_error()
        assert bits_a == bits_b
        assert torch.equal(got.view(torch.int64), ref.view(torch.int64))
        # and the oracle's fixed-point deposition, on the oracle's own locate
        cell, nout = orc.locate_structured(dims, origin, dx, pos_np)
        assert nout == 0
        eps, fbits = orc.deposit(cell, w_np, int(np.prod(dims)), vc_uniform=(dx * dx) * dx, mode=1)
        assert fbits == bits_b
        assert np.array_equal(got.cpu().numpy().view(np.int64), eps.view(np.int64))


def test_noalloc_call_allocates_no_device_memory(env):
    cg, lib, torch = env
    rng = np.random.default_rng(13)
    dims, origin, dx, n, nf = (64, 64, 64), (0.0, 0.0, 0.0), 1.0 / 64, 400_000, 4
    pos = torch.from_numpy(rng.random((3, n))).cuda()
    w = torch.from_numpy(rng.random((nf, n))).cuda()
    out = torch.empty((nf, int(np.prod(dims))), dtype=torch.float64, device="cuda")
    st, _, _ = _call_noalloc(lib, torch, dims, origin, dx, pos, w, out)   # the module is loaded
    assert st == 0, lib.cg_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        st, _, _ = _call_noalloc(lib, torch, dims, origin, dx, pos, w, out)
        assert st == 0, lib.cg_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_particles_outside_give_edomain_and_leave_the_output(env):
    cg, lib, torch = env
    rng = np.random.default_rng(14)
    dims, origin, dx, n = (16, 16, 16), (0.0, 0.0, 0.0), 1.0 / 16, 1000
    pos_np = rng.random((3, n))
    pos_np[1, 777] = 1.0 + 1e-9                       # just outside the upper y wall
    pos = torch.from_numpy(pos_np).cuda()
    w = torch.from_numpy(rng.random((2, n))).cuda()
    out = torch.full((2, 16 ** 3), 3.25, dtype=torch.float64, device="cuda")
    st, out, _ = _call_noalloc(lib, torch, dims, origin, dx, pos, w, out)
    assert st == 6
    assert b"outside" in lib.cg_last_error()
    assert bool((out == 3.25).all())


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    cg, lib, torch = env
    pos = torch.zeros((3, 1), dtype=torch.float64, device="cuda")
    w = torch.ones((1, 1), dtype=torch.float64, device="cuda")
    out = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    org = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    for dims in ((160, 160, 160),                    # 4.1M cells > the static scratch
                 (1 << 21, 1 << 21, 1 << 22)):       # a product that wraps around 2^64
        st = lib.cg_deposit_fixed_noalloc(dims[0], dims[1], dims[2], org, 0.01, 1, pos.data_ptr(),
                                          1, w.data_ptr(), out.data_ptr(), None, None)
        assert st == 1
        assert b"exceeds the static scratch" in lib.cg_last_error()

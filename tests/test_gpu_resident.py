"""GPU parity of the resident inner solve (sweep_shape 300: each round's Chebyshev
iterations in one cooperative launch with the mesh held in the SMs' shared memory and
faces exchanged between neighbouring blocks).

Its arithmetic, and the order of it, is that of the vectorised streamed sweep
(sweep_shape 101..116) with FP32 storage, so with FP32 inner solves the two must agree
bit for bit; both must meet the mixed-precision bar (1e-6 max-relative) against the FP64
oracle.  Its neighbour waits are bounded: with a budget of one clock cycle a wait gives
up and the call returns CG_ETIMEOUT, and the context stays usable.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-6
RESIDENT = 300


@pytest.fixture(scope="module")
def cg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1409_0001_gb300 as cg
    from paper_1409_0001_gb300 import build
    build.build()
    cg.load_library()
    return cg


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


def maxrel(u, ref):
    u, ref = np.atleast_2d(u), np.atleast_2d(ref)
    return max(np.max(np.abs(u[f] - ref[f])) / np.max(np.abs(ref[f])) for f in range(ref.shape[0]))


def field(dims, seed):
    rng = np.random.default_rng(seed)
    n = int(np.prod(dims))
    u0 = rng.random(n) * 0.2
    u0[rng.integers(0, n, max(n // 40, 3))] += rng.random(max(n // 40, 3)) * 20
    return u0


# nx = 128 (one warp per row), 256 (two warps per row), 36 (rows shorter than a warp)
@pytest.mark.parametrize("dims", [(32, 32, 32), (128, 20, 12), (256, 8, 9), (36, 17, 9)])
@pytest.mark.parametrize("precision", [3, 1])
@pytest.mark.parametrize("scheme", [0, 1])
def test_resident_bit_identical_to_streamed_and_matches_oracle(cg, orc, dims, precision, scheme):
    dx = 1.0 / dims[0]
    u0 = field(dims, 40)
    T = (3 * dx) ** 2 / 4
    mesh = cg.StructuredMesh(dims, (0, 0, 0), dx)
    outs = {}
    for shape in (RESIDENT, 101):
        u = dev(u0[None])
        _, rep = cg.diffuse(mesh, u, cg.Params(T=T, nsteps=10, scheme=scheme, precision=precision,
                                               sweep_shape=shape), report=True)
        assert rep["sweep_shape_used"] == shape
        assert rep["final_rel_residual"] <= 1e-13
        outs[shape] = u.cpu().numpy()
    assert np.array_equal(bits(outs[RESIDENT]), bits(outs[101]))
    ref, _ = orc.diffuse_structured(u0, dims, dx, T, 10, scheme=scheme, tol=1e-15)
    assert maxrel(outs[RESIDENT], ref) <= MIXED_TOL


@pytest.mark.parametrize("b_over_dx", [1, 8])
def test_resident_bf16_inner_matches_oracle(cg, orc, b_over_dx):
    dims = (64, 48, 40)
    dx = 1.0 / 64
    u0 = field(dims, 41)
    T = (b_over_dx * dx) ** 2 / 4
    mesh = cg.StructuredMesh(dims, (0, 0, 0), dx)
    u = dev(u0[None])
    _, rep = cg.diffuse(mesh, u, cg.Params(T=T, nsteps=10, precision=4, sweep_shape=RESIDENT),
                        report=True)
    assert rep["sweep_shape_used"] == RESIDENT
    ref, _ = orc.diffuse_structured(u0, dims, dx, T, 10, tol=1e-15)
    assert maxrel(u.cpu().numpy(), ref) <= MIXED_TOL


def test_resident_full_size_clustered_128(cg, orc):
    """The 128^3 clustered case (2,000,000 spheres) at b = 2 dx through the whole method
    with the resident inner solve: bit-identical to the streamed sweep, within the mixed
    bar of the oracle, mass conserved."""
    c = W.clustered_cube()
    cell, _ = orc.locate_structured(c.dims, c.origin, c.dx, c.pos)
    eps0, _ = orc.deposit(cell, c.w, c.ncells, vc_uniform=(c.dx * c.dx) * c.dx)
    ref, _ = orc.diffuse_structured(eps0, c.dims, c.dx, c.b ** 2 / 4, c.nsteps, tol=1e-14)
    mesh = cg.StructuredMesh(c.dims, c.origin, c.dx)
    pos, w = dev(c.pos), dev(c.w)
    outs = {}
    for shape in (RESIDENT, 104):
        got, rep = cg.coarse_grain(mesh, pos, w, cg.Params(bandwidth=c.b, nsteps=c.nsteps,
                                                           precision=3, sweep_shape=shape),
                                   report=True)
        assert abs(rep["mass_out"][0] - rep["mass_in"][0]) <= 1e-12 * rep["mass_in"][0]
        outs[shape] = got.cpu().numpy()
    assert np.array_equal(bits(outs[RESIDENT]), bits(outs[104]))
    assert maxrel(outs[RESIDENT], ref) <= MIXED_TOL


def test_resident_rejects_what_it_cannot_hold(cg):
    mesh = cg.StructuredMesh((32, 32, 32), (0, 0, 0), 1 / 32)
    with pytest.raises(cg.CGError) as e:          # two fields
        cg.diffuse(mesh, dev(np.zeros((2, 32 ** 3))), cg.Params(bandwidth=0.1, precision=3,
                                                                sweep_shape=RESIDENT))
    assert e.value.code == "CG_EINVAL"
    odd = cg.StructuredMesh((30, 32, 32), (0, 0, 0), 1 / 32)
    with pytest.raises(cg.CGError) as e:          # nx % 4 != 0
        cg.diffuse(odd, dev(np.zeros((1, 30 * 32 * 32))), cg.Params(bandwidth=0.1, precision=3,
                                                                    sweep_shape=RESIDENT))
    assert e.value.code == "CG_EINVAL"


def test_autotuned_shape_is_reported(cg):
    mesh = cg.StructuredMesh((64, 64, 64), (0, 0, 0), 1 / 64)
    u = dev(field((64, 64, 64), 42)[None])
    _, rep = cg.diffuse(mesh, u, cg.Params(bandwidth=3 / 64, precision=3), report=True)
    s = rep["sweep_shape_used"]
    assert (s == RESIDENT or 101 <= s <= 199 or 201 <= s <= 299 or 401 <= s <= 499
            or s in (2, 4, 8) or -32 <= s <= -1)


def test_resident_wait_budget_gives_etimeout_and_context_survives(cg):
    """A neighbour wait with a budget of one clock cycle gives up as soon as a neighbour's
    face is not already there: the blocks leave and the call returns CG_ETIMEOUT (some
    attempt must hit a wait).  Calls on the same mesh afterwards are unaffected."""
    dims = (128, 64, 64)
    dx = 1.0 / 128
    u0 = field(dims, 43)
    mesh = cg.StructuredMesh(dims, (0, 0, 0), dx)
    codes = []
    for _ in range(5):
        u = dev(u0[None])
        try:
            cg.diffuse(mesh, u, cg.Params(bandwidth=4 * dx, nsteps=10, precision=3,
                                          sweep_shape=RESIDENT, barrier_budget=1))
            codes.append("CG_OK")
        except cg.CGError as e:
            codes.append(e.code)
    assert "CG_ETIMEOUT" in codes
    assert set(codes) <= {"CG_OK", "CG_ETIMEOUT"}
    outs = []
    for shape in (RESIDENT, 101):
        u = dev(u0[None])
        cg.diffuse(mesh, u, cg.Params(bandwidth=4 * dx, nsteps=10, precision=3, sweep_shape=shape))
        outs.append(bits(u.cpu().numpy()))
    assert np.array_equal(outs[0], outs[1])

"""GPU parity of the two-iterations-per-launch Chebyshev sweep (sweep_shape 200 + z:
iterations k and k+1 in one launch, z planes per block; rows of at most 128 cells as one
warp each, longer rows, up to 512 cells, as whole-row blocks with staged planes).

Per cell it evaluates the same expression, in the same order, as the one-iteration
vectorised sweep (sweep_shape 100 + z), so with the same z the two must agree bit for
bit, whatever the parity of the iteration count; both must meet the mixed-precision bar
(1e-6 max-relative) against the FP64 oracle.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-6


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


def field(shape, seed):
    rng = np.random.default_rng(seed)
    u0 = rng.random(shape) * 0.2
    n = u0.shape[-1]
    idx = rng.integers(0, n, max(n // 40, 3))
    u0[..., idx] += 10.0
    return u0


# rows of 128 (a full warp), 36 (a partial warp), 4; ragged last row tile (ny % 8 != 0);
# b/dx 1 and 3 give odd and even iteration counts per round
@pytest.mark.parametrize("dims", [(128, 20, 13), (36, 17, 9), (4, 9, 30), (64, 64, 64)])
@pytest.mark.parametrize("z", [1, 4, 16])
@pytest.mark.parametrize("b_over_dx", [1, 3])
def test_pairs_bit_identical_to_single_sweep(cg, orc, dims, z, b_over_dx):
    dx = 1.0 / dims[0]
    u0 = field((2, int(np.prod(dims))), 50)
    T = (b_over_dx * dx) ** 2 / 4
    mesh = cg.StructuredMesh(dims, (0, 0, 0), dx)
    outs = {}
    for shape in (200 + z, 100 + z):
        u = dev(u0)
        _, rep = cg.diffuse(mesh, u, cg.Params(T=T, nsteps=10, precision=3, sweep_shape=shape),
                            report=True)
        assert rep["sweep_shape_used"] == shape
        assert rep["final_rel_residual"] <= 1e-13
        outs[shape] = u.cpu().numpy()
    assert np.array_equal(bits(outs[200 + z]), bits(outs[100 + z]))
    ref, _ = orc.diffuse_structured(u0, dims, dx, T, 10, tol=1e-15)
    assert maxrel(outs[200 + z], ref) <= MIXED_TOL


@pytest.mark.parametrize("precision,scheme", [(1, 0), (4, 0), (3, 1)])
def test_pairs_other_modes_bit_identical(cg, orc, precision, scheme):
    """IEEE-FP64 refinement (adaptive schedule), BF16 storage, Crank-Nicolson."""
    dims = (96, 40, 24)
    dx = 1.0 / 96
    u0 = field((1, int(np.prod(dims))), 51)
    T = (4 * dx) ** 2 / 4
    mesh = cg.StructuredMesh(dims, (0, 0, 0), dx)
    outs = {}
    for shape in (204, 104):
        u = dev(u0)
        cg.diffuse(mesh, u, cg.Params(T=T, nsteps=10, precision=precision, scheme=scheme,
                                      sweep_shape=shape))
        outs[shape] = u.cpu().numpy()
    assert np.array_equal(bits(outs[204]), bits(outs[104]))
    ref, _ = orc.diffuse_structured(u0, dims, dx, T, 10, scheme=scheme, tol=1e-15)
    assert maxrel(outs[204], ref) <= MIXED_TOL


def test_pairs_full_size_clustered_128(cg, orc):
    """The 128^3 clustered case (2,000,000 spheres), b = 2 dx, whole method: two
    iterations per launch reproduce the one-iteration sweep bit for bit."""
    c = W.clustered_cube()
    cell, _ = orc.locate_structured(c.dims, c.origin, c.dx, c.pos)
    eps0, _ = orc.deposit(cell, c.w, c.ncells, vc_uniform=(c.dx * c.dx) * c.dx)
    ref, _ = orc.diffuse_structured(eps0, c.dims, c.dx, c.b ** 2 / 4, c.nsteps, tol=1e-14)
    mesh = cg.StructuredMesh(c.dims, c.origin, c.dx)
    pos, w = dev(c.pos), dev(c.w)
    outs = {}
    for shape in (208, 108):
        got = cg.coarse_grain(mesh, pos, w, cg.Params(bandwidth=c.b, nsteps=c.nsteps, precision=3,
                                                      sweep_shape=shape))
        outs[shape] = got.cpu().numpy()
    assert np.array_equal(bits(outs[208]), bits(outs[108]))
    assert maxrel(outs[208], ref) <= MIXED_TOL


# long rows: two warps (256), a second warp one lane wide (132), three and four warps with
# idle lanes (388) and full (512); ragged last row block (ny not a multiple of the rows per
# block: 6 at 512, 8 at 388, 14 at 256, 14 at 132); one plane per block, odd chunks, whole mesh
@pytest.mark.parametrize("dims", [(256, 20, 13), (132, 17, 9), (388, 11, 6), (512, 14, 7)])
@pytest.mark.parametrize("z", [1, 3, 16])
@pytest.mark.parametrize("b_over_dx", [1, 3])
def test_pairs_long_rows_bit_identical_to_single_sweep(cg, orc, dims, z, b_over_dx):
    dx = 1.0 / dims[0]
    u0 = field((2, int(np.prod(dims))), 53)
    T = (b_over_dx * dx) ** 2 / 4
    mesh = cg.StructuredMesh(dims, (0, 0, 0), dx)
    outs = {}
    for shape in (200 + z, 100 + z):
        u = dev(u0)
        _, rep = cg.diffuse(mesh, u, cg.Params(T=T, nsteps=4, precision=3, sweep_shape=shape),
                            report=True)
        assert rep["sweep_shape_used"] == shape
        assert rep["final_rel_residual"] <= 1e-13
        outs[shape] = u.cpu().numpy()
    assert np.array_equal(bits(outs[200 + z]), bits(outs[100 + z]))
    ref, _ = orc.diffuse_structured(u0, dims, dx, T, 4, tol=1e-15)
    assert maxrel(outs[200 + z], ref) <= MIXED_TOL


@pytest.mark.parametrize("precision,scheme", [(1, 0), (4, 0), (3, 1)])
def test_pairs_long_rows_other_modes_bit_identical(cg, orc, precision, scheme):
    """Long rows in IEEE-FP64 refinement, BF16 storage and Crank-Nicolson."""
    dims = (320, 24, 10)
    dx = 1.0 / 320
    u0 = field((1, int(np.prod(dims))), 54)
    T = (6 * dx) ** 2 / 4
    mesh = cg.StructuredMesh(dims, (0, 0, 0), dx)
    outs = {}
    for shape in (205, 105):
        u = dev(u0)
        cg.diffuse(mesh, u, cg.Params(T=T, nsteps=5, precision=precision, scheme=scheme,
                                      sweep_shape=shape))
        outs[shape] = u.cpu().numpy()
    assert np.array_equal(bits(outs[205]), bits(outs[105]))
    ref, _ = orc.diffuse_structured(u0, dims, dx, T, 5, scheme=scheme, tol=1e-15)
    assert maxrel(outs[205], ref) <= MIXED_TOL


# a periodic x axis: whole-row blocks wrap the row within the block (rows of 4, 36, 132,
# 256 and 512 cells; two fields, one of them signed)
@pytest.mark.parametrize("dims", [(4, 6, 5), (36, 13, 7), (132, 9, 6), (256, 15, 5), (512, 8, 6)])
@pytest.mark.parametrize("z", [1, 4])
def test_pairs_periodic_x_bit_identical_to_single_sweep(cg, orc, dims, z):
    rng = np.random.default_rng(57)
    n = int(np.prod(dims))
    u0 = np.vstack([rng.random(n), rng.random(n) - 0.4])
    dx = 1.0 / dims[0]
    T = (3 * dx) ** 2 / 4
    mesh = cg.StructuredMesh(dims, (0, 0, 0), dx, periodic=(True, False, False))
    outs = {}
    for shape in (200 + z, 100 + z):
        u = dev(u0)
        _, rep = cg.diffuse(mesh, u, cg.Params(T=T, nsteps=4, precision=3, sweep_shape=shape),
                            report=True)
        assert rep["sweep_shape_used"] == shape
        outs[shape] = u.cpu().numpy()
    assert np.array_equal(bits(outs[200 + z]), bits(outs[100 + z]))
    ref, _ = orc.diffuse_structured(u0, dims, dx, T, 4, tol=1e-15, periodic=(True, False, False))
    assert maxrel(outs[200 + z], ref) <= MIXED_TOL


def test_pairs_reject_long_rows(cg):
    for dims in ((516, 8, 8), (30, 8, 8)):
        mesh = cg.StructuredMesh(dims, (0, 0, 0), 1.0 / dims[0])
        with pytest.raises(cg.CGError) as e:
            cg.diffuse(mesh, dev(np.zeros((1, int(np.prod(dims))))),
                       cg.Params(bandwidth=0.1, precision=3, sweep_shape=204))
        assert e.value.code == "CG_EINVAL"

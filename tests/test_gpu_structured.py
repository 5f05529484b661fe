"""GPU parity of the structured-mesh path against the FP64 oracle, through the C ABI.

Bars: locate and deposition bit-exact (both modes); diffusion max-relative error
(max_k |u - u_ref| / max_k |u_ref|, per field) <= 1e-10 for the FP64 solver and
<= 1e-6 for the mixed solvers; mass conserved to 1e-12 relative; two runs
bit-identical.  Sizes span several tiles and a ragged tail; the full-size 128^3
clustered case is included.
"""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
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
    u = np.atleast_2d(u)
    ref = np.atleast_2d(ref)
    return max(np.max(np.abs(u[f] - ref[f])) / max(np.max(np.abs(ref[f])), 1e-300)
               for f in range(ref.shape[0]))


# ----------------------------------------------------------------------------- locate
@pytest.mark.parametrize("dims,origin,dx", [((32, 32, 32), (0, 0, 0), 1 / 32),
                                            ((37, 23, 11), (-0.3, 0.25, 1.0), 0.1)])
def test_locate_bit_exact(cg, orc, dims, origin, dx):
    rng = np.random.default_rng(1)
    L = np.array(dims) * dx
    pos = np.array(origin)[:, None] + rng.random((3, 20_011)) * L[:, None]
    k = 500
    pos[:, :k] = np.array(origin)[:, None] + np.round(rng.random((3, k)) * np.array(dims)[:, None]) * dx
    pos[:, k] = np.array(origin) + L                      # upper corner
    pos[0, k + 1] = origin[0] - 1e-9                      # outside
    pos[1, k + 2] = np.nan
    ref, nref = orc.locate_structured(dims, origin, dx, pos)
    mesh = cg.StructuredMesh(dims, origin, dx)
    got, nout = cg.locate(mesh, dev(pos))
    assert nout == nref == 2
    assert np.array_equal(got.cpu().numpy(), ref)


def test_locate_near_faces_bit_exact(cg, orc):
    """Positions a few ulps either side of every face plane, on an offset origin with an
    inexact spacing (and -0.0 on a wall at 0): the estimate-then-confirm locate must give
    the FP64 definition's cell everywhere."""
    dims, dx = (29, 17, 13), 1.0 / 7.0
    for origin in ((-3.7, 0.0, 1e-3), (0.0, 123.456, -0.5)):
        rng = np.random.default_rng(11)
        o = np.array(origin)
        faces = [o[a] + np.arange(dims[a] + 1) * dx for a in range(3)]
        cols = []
        for a in range(3):
            f = np.repeat(faces[a], 9)
            ulps = np.tile(np.arange(-4, 5), dims[a] + 1)
            cols.append(f + ulps * np.spacing(np.abs(f) + 1e-300))
        n = max(len(c) for c in cols)
        pos = np.empty((3, n))
        for a in range(3):
            pos[a] = np.resize(cols[a], n)
            rng.shuffle(pos[a])
        pos[:, 0] = [-0.0 if origin[0] == 0.0 else origin[0], pos[1, 0], pos[2, 0]]
        ref, nref = orc.locate_structured(dims, origin, dx, pos)
        mesh = cg.StructuredMesh(dims, origin, dx)
        got, nout = cg.locate(mesh, dev(pos))
        assert nout == nref
        assert np.array_equal(got.cpu().numpy(), ref)


# ----------------------------------------------------------------------------- deposit
def _deposit_case(orc, cg, dims, origin, dx, pos, w, mode):
    cell, nout = orc.locate_structured(dims, origin, dx, pos)
    assert nout == 0
    ncells = int(np.prod(dims))
    ref, fb = orc.deposit(cell, w, ncells, vc_uniform=(dx * dx) * dx, mode=mode)
    mesh = cg.StructuredMesh(dims, origin, dx)
    got, rep = cg.deposit(mesh, dev(pos), dev(w), cg.Params(deposit_mode=mode), report=True)
    got = got.cpu().numpy()
    assert np.array_equal(bits(got), bits(ref))
    if mode == 1:
        assert rep["fixed_point_bits"][:len(fb)] == fb[:8]
    return got


@pytest.mark.parametrize("mode", [0, 1])
def test_deposit_uniform_cube_bit_exact(cg, orc, mode):
    c = W.uniform_cube()
    _deposit_case(orc, cg, c.dims, c.origin, c.dx, c.pos, c.w, mode)


@pytest.mark.parametrize("mode", [0, 1])
def test_deposit_clustered_signed_multifield_bit_exact(cg, orc, mode):
    c = W.clustered_cube(n_side=48, n_particles=300_007, seed=3)
    rng = np.random.default_rng(4)
    w = np.vstack([c.w, rng.standard_normal((4, c.n)) * 1e-3])   # volume + 4 signed fields
    _deposit_case(orc, cg, c.dims, c.origin, c.dx, c.pos, w, mode)


@pytest.mark.parametrize("mode", [0, 1])
def test_deposit_degenerate_inputs(cg, orc, mode):
    dims, origin, dx = (9, 5, 3), (0.0, 0.0, 0.0), 0.125
    rng = np.random.default_rng(5)
    # every particle in one cell (one long ordered segment), values spanning magnitudes
    n = 70_001
    pos = np.full((3, n), 0.3)
    w = rng.standard_normal((1, n)) * 10.0 ** rng.integers(-8, 8, (1, n))
    _deposit_case(orc, cg, dims, origin, dx, pos, w, mode)
    # a single particle; particles exactly on the upper walls
    _deposit_case(orc, cg, dims, origin, dx, np.array([[1.125], [0.625], [0.375]]),
                  np.array([[2.0]]), mode)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("crowd", [64, 65])
def test_deposit_crowded_cell_both_paths(cg, orc, mode, crowd):
    """One cell holding 64 particles (the largest the per-cell sort takes) or 65 (the
    stable radix sort takes over), among scattered others: bit-exact either way."""
    dims, origin, dx = (16, 16, 16), (0.0, 0.0, 0.0), 1.0 / 16
    rng = np.random.default_rng(12)
    pos = rng.random((3, 5000))
    idx = rng.choice(5000, crowd, replace=False)
    pos[:, idx] = 0.51
    w = rng.standard_normal((2, 5000)) * 10.0 ** rng.integers(-6, 6, (2, 5000))
    _deposit_case(orc, cg, dims, origin, dx, pos, w, mode)


def test_deposit_empty_and_errors(cg, orc):
    import torch
    dims, origin, dx = (8, 8, 8), (0.0, 0.0, 0.0), 0.125
    mesh = cg.StructuredMesh(dims, origin, dx)
    out = cg.deposit(mesh, dev(np.zeros((3, 0))), dev(np.zeros((2, 0))))
    assert torch.count_nonzero(out).item() == 0
    pos = np.full((3, 10), 0.5)
    pos[2, 7] = 1.5
    sentinel = torch.full((1, 512), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(cg.CGError) as e:
        cg.deposit(mesh, dev(pos), dev(np.ones((1, 10))), out=sentinel)
    assert e.value.code == "CG_EDOMAIN"
    assert torch.all(sentinel == 7.0)                 # nothing written on error
    w = np.ones((1, 10))
    w[0, 3] = np.inf
    with pytest.raises(cg.CGError) as e:
        cg.deposit(mesh, dev(np.full((3, 10), 0.5)), dev(w), out=sentinel)
    assert e.value.code == "CG_EINVAL"
    assert torch.all(sentinel == 7.0)


# ----------------------------------------------------------------------------- diffuse
def _diffuse_case(orc, cg, dims, dx, u0, T, nsteps, scheme, precision, tol=1e-13):
    ref, _ = orc.diffuse_structured(u0, dims, dx, T, nsteps, scheme=scheme, tol=1e-15)
    mesh = cg.StructuredMesh(dims, (0, 0, 0), dx)
    u = dev(np.atleast_2d(u0))
    _, rep = cg.diffuse(mesh, u, cg.Params(T=T, nsteps=nsteps, scheme=scheme,
                                           precision=precision, tol=tol), report=True)
    return u.cpu().numpy(), np.atleast_2d(ref), rep


@pytest.mark.parametrize("precision,bar", [(0, FP64_TOL), (1, MIXED_TOL), (2, MIXED_TOL),
                                           (3, MIXED_TOL), (4, MIXED_TOL)])
@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("dims", [(32, 32, 32), (13, 7, 5), (257, 3, 2)])
def test_diffuse_parity(cg, orc, dims, scheme, precision, bar):
    rng = np.random.default_rng(6)
    dx = 1.0 / dims[0]
    n = int(np.prod(dims))
    u0 = np.zeros((2, n))
    u0[0, rng.integers(0, n, max(n // 50, 3))] = rng.random(max(n // 50, 3)) * 30
    u0[1] = rng.random(n) - 0.5
    T = (3 * dx) ** 2 / 4
    got, ref, rep = _diffuse_case(orc, cg, dims, dx, u0, T, 10, scheme, precision)
    assert maxrel(got, ref) <= bar
    assert rep["final_rel_residual"] <= 1e-13
    m_in, m_out = np.array(rep["mass_in"][:2]), np.array(rep["mass_out"][:2])
    scale = np.abs(u0).sum(axis=1) * dx ** 3
    assert np.all(np.abs(m_out - m_in) <= 1e-12 * scale)


def test_diffuse_explicit_parity(cg, orc):
    dims = (40, 30, 20)
    dx = 0.025
    rng = np.random.default_rng(7)
    u0 = rng.random(int(np.prod(dims)))
    T = 0.15 * dx * dx * 20          # dtau/dx^2 = 0.15 <= 1/6
    got, ref, _ = _diffuse_case(orc, cg, dims, dx, u0, T, 20, 2, 0)
    assert maxrel(got, ref) <= 1e-13


@pytest.mark.parametrize("b_over_dx", [1, 2, 4, 8])
def test_diffuse_bandwidth_sweep_mixed_vs_fp64(cg, orc, b_over_dx):
    """The 128^3 clustered case's b/dx sweep on a 48^3 mesh: FP32+FP64 refinement and
    FP64 CG both match the oracle."""
    c = W.clustered_cube(n_side=48, n_particles=100_000, seed=8)
    cell, _ = orc.locate_structured(c.dims, c.origin, c.dx, c.pos)
    u0, _ = orc.deposit(cell, c.w, c.ncells, vc_uniform=c.dx ** 3)
    T = (b_over_dx * c.dx) ** 2 / 4
    for precision, bar in ((0, FP64_TOL), (1, MIXED_TOL), (3, MIXED_TOL), (4, MIXED_TOL)):
        got, ref, _ = _diffuse_case(orc, cg, c.dims, c.dx, u0, T, 10, 0, precision)
        assert maxrel(got, ref) <= bar


def test_diffuse_is_deterministic(cg):
    dims = (50, 40, 30)
    rng = np.random.default_rng(9)
    u0 = rng.random((3, int(np.prod(dims))))
    mesh = cg.StructuredMesh(dims, (0, 0, 0), 0.02)
    outs = []
    for precision in (0, 1, 3, 0, 1, 3):
        u = dev(u0)
        cg.diffuse(mesh, u, cg.Params(bandwidth=0.08, nsteps=5, precision=precision))
        outs.append(bits(u.cpu().numpy()))
    for i in range(3):
        assert np.array_equal(outs[i], outs[i + 3])


# ----------------------------------------------------------------------------- whole method
def test_coarse_grain_uniform_cube_fp64(cg, orc):
    """The 32^3 unit-cube case: 10,000 spheres, b = 3 dx, 10 implicit-Euler steps, FP64."""
    c = W.uniform_cube()
    eps0, ref, nout, _ = orc.coarse_grain_structured(c.dims, c.origin, c.dx, c.pos, c.w, c.b,
                                                    c.nsteps)
    mesh = cg.StructuredMesh(c.dims, c.origin, c.dx)
    p = cg.Params(bandwidth=c.b, nsteps=c.nsteps)
    got, rep = cg.coarse_grain(mesh, dev(c.pos), dev(c.w), p, report=True)
    assert maxrel(got.cpu().numpy(), ref) <= FP64_TOL
    assert abs(rep["mass_out"][0] - c.w.sum()) <= 1e-12 * c.w.sum()
    host, rep2 = cg.coarse_grain_host(mesh, c.pos, c.w, p, report=True)
    assert np.array_equal(bits(host), bits(got.cpu().numpy()))


@pytest.mark.parametrize("precision", [1, 3, 0])
def test_coarse_grain_clustered_128_full_size(cg, orc, precision):
    """Full-size 128^3 case, 2,000,000 clustered spheres, b = 2 dx: deposition bit-exact,
    diffusion within the bar of its precision."""
    c = W.clustered_cube()
    cell, nout = orc.locate_structured(c.dims, c.origin, c.dx, c.pos)
    assert nout == 0
    eps0, _ = orc.deposit(cell, c.w, c.ncells, vc_uniform=(c.dx * c.dx) * c.dx)
    mesh = cg.StructuredMesh(c.dims, c.origin, c.dx)
    d0 = cg.deposit(mesh, dev(c.pos), dev(c.w)).cpu().numpy()
    assert np.array_equal(bits(d0), bits(eps0))
    ref, _ = orc.diffuse_structured(eps0, c.dims, c.dx, c.b ** 2 / 4, c.nsteps, tol=1e-14)
    got, rep = cg.coarse_grain(mesh, dev(c.pos), dev(c.w),
                               cg.Params(bandwidth=c.b, nsteps=c.nsteps, precision=precision),
                               report=True)
    assert maxrel(got.cpu().numpy(), ref) <= (FP64_TOL if precision == 0 else MIXED_TOL)
    assert abs(rep["mass_out"][0] - rep["mass_in"][0]) <= 1e-12 * rep["mass_in"][0]


def test_barrier_timeout_reports_etimeout_and_context_survives(cg):
    """The persistent inner solve's grid barrier has a bounded wait: with a budget of
    one clock cycle it gives up, every block leaves, and the call returns CG_ETIMEOUT.
    The next call on the same mesh works."""
    dims = (40, 40, 40)
    rng = np.random.default_rng(13)
    u0 = rng.random((1, 40 ** 3))
    mesh = cg.StructuredMesh(dims, (0, 0, 0), 0.025)
    u = dev(u0)
    with pytest.raises(cg.CGError) as e:
        cg.diffuse(mesh, u, cg.Params(bandwidth=0.2, nsteps=2, precision=1,
                                      barrier_budget=1))
    assert e.value.code == "CG_ETIMEOUT"
    # the same mesh afterwards: persistent (ample budget) and per-launch inner solves agree
    outs = []
    for budget in (2_000_000_000, 0):
        u = dev(u0)
        cg.diffuse(mesh, u, cg.Params(bandwidth=0.2, nsteps=2, precision=1, barrier_budget=budget))
        outs.append(bits(u.cpu().numpy()))
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("dims", [(40, 30, 20), (130, 9, 7)])
def test_diffuse_explicit_double_float_parity(cg, orc, dims):
    """Explicit Euler steps in double-float arithmetic (precision 3, even nx): within
    the FP64 bar of the oracle after 40 steps, deterministic, and matching the FP64 GPU
    steps; beyond the stability limit the call is refused."""
    dx = 1.0 / dims[0]
    rng = np.random.default_rng(17)
    u0 = rng.random((2, int(np.prod(dims))))
    u0[1] -= 0.5
    T = 0.15 * dx * dx * 40          # dtau/dx^2 = 0.15 <= 1/6
    ref, _ = orc.diffuse_structured(u0, dims, dx, T, 40, scheme=2)
    mesh = cg.StructuredMesh(dims, (0, 0, 0), dx)
    outs = []
    for _ in range(2):
        u = dev(u0)
        cg.diffuse(mesh, u, cg.Params(T=T, nsteps=40, scheme=2, precision=3))
        outs.append(u.cpu().numpy())
    assert np.array_equal(bits(outs[0]), bits(outs[1]))
    assert maxrel(outs[0], ref) <= 1e-12
    u64 = dev(u0)
    cg.diffuse(mesh, u64, cg.Params(T=T, nsteps=40, scheme=2, precision=0))
    assert maxrel(outs[0], u64.cpu().numpy()) <= 1e-12
    with pytest.raises(cg.CGError):
        cg.diffuse(mesh, dev(u0), cg.Params(T=0.2 * dx * dx * 40, nsteps=40, scheme=2, precision=3))

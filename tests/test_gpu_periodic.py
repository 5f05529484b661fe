"""GPU parity of periodic axes (Section 3.1: periodic boundaries keep periodic
conditions) and of the solid velocity (diffused momentum over diffused solid fraction),
against the FP64 oracle.

Bars: FP64 solvers <= 1e-10 and mixed precision <= 1e-6 max-relative against the
oracle; mass conserved to 1e-12; the solid velocity bit-exact against the oracle's
division of the same smoothed fields.
"""
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
    u, ref = np.atleast_2d(u), np.atleast_2d(ref)
    return max(np.max(np.abs(u[f] - ref[f])) / np.max(np.abs(ref[f])) for f in range(ref.shape[0]))


# ragged tiles (37 x 13), a one-cell axis, a two-cell axis
@pytest.mark.parametrize("dims", [(37, 13, 11), (32, 16, 8), (6, 1, 9), (2, 9, 5)])
@pytest.mark.parametrize("periodic", [(True, True, True), (True, False, False), (False, True, True)])
@pytest.mark.parametrize("precision,bar", [(0, FP64_TOL), (3, MIXED_TOL), (1, MIXED_TOL)])
def test_periodic_diffusion_parity(cg, orc, dims, periodic, precision, bar):
    rng = np.random.default_rng(70)
    n = int(np.prod(dims))
    u0 = np.vstack([rng.random(n), rng.random(n) - 0.4])
    dx = 1.0 / max(dims)
    T = (2.5 * dx) ** 2 / 4
    ref, _ = orc.diffuse_structured(u0, dims, dx, T, 10, tol=1e-15, periodic=periodic)
    mesh = cg.StructuredMesh(dims, (0, 0, 0), dx, periodic=periodic)
    u = dev(u0)
    _, rep = cg.diffuse(mesh, u, cg.Params(T=T, nsteps=10, precision=precision), report=True)
    got = u.cpu().numpy()
    assert maxrel(got, ref) <= bar
    scale = np.abs(u0).sum(axis=1) * dx ** 3
    assert np.all(np.abs(np.array(rep["mass_out"][:2]) - np.array(rep["mass_in"][:2])) <= 1e-12 * scale)


@pytest.mark.parametrize("scheme", [1, 2])
def test_periodic_other_schemes(cg, orc, scheme):
    dims = (20, 12, 9)
    dx = 0.05
    rng = np.random.default_rng(71)
    u0 = rng.random(int(np.prod(dims)))
    T = 0.15 * dx * dx * 12
    ref, _ = orc.diffuse_structured(u0, dims, dx, T, 12, scheme=scheme, tol=1e-15,
                                    periodic=(True, False, True))
    mesh = cg.StructuredMesh(dims, (0, 0, 0), dx, periodic=(True, False, True))
    for precision, bar in ((0, FP64_TOL), (3, MIXED_TOL if scheme != 2 else FP64_TOL)):
        u = dev(u0[None])
        cg.diffuse(mesh, u, cg.Params(T=T, nsteps=12, scheme=scheme, precision=precision))
        assert maxrel(u.cpu().numpy(), ref) <= bar


def test_periodic_shapes_and_reset(cg):
    """Shapes other than the z-marching and vectorised sweeps are refused on a periodic
    mesh (two iterations per launch only take a periodic x axis); clearing the periodic
    axes restores the wall results bit for bit (cached schedules are dropped)."""
    dims = (32, 24, 16)
    rng = np.random.default_rng(72)
    u0 = rng.random((1, int(np.prod(dims))))
    mesh = cg.StructuredMesh(dims, (0, 0, 0), 1 / 32)
    p = cg.Params(bandwidth=3 / 32, nsteps=5, precision=3)
    u = dev(u0)
    cg.diffuse(mesh, u, p)
    walls = u.cpu().numpy()
    mesh.set_periodic(True, True, False)
    for shape in (4, 300, 204, 404):
        with pytest.raises(cg.CGError) as e:
            cg.diffuse(mesh, dev(u0), cg.Params(bandwidth=3 / 32, nsteps=5, precision=3,
                                                sweep_shape=shape))
        assert e.value.code == "CG_EINVAL"
    u = dev(u0)
    _, rep = cg.diffuse(mesh, u, cg.Params(bandwidth=3 / 32, nsteps=5, precision=3, sweep_shape=-4),
                        report=True)
    assert rep["sweep_shape_used"] == -4
    assert not np.array_equal(u.cpu().numpy(), walls)
    mesh.set_periodic(False, False, False)
    u = dev(u0)
    cg.diffuse(mesh, u, p)
    assert np.array_equal(bits(u.cpu().numpy()), bits(walls))
    other = cg.StructuredMesh(dims, (0, 0, 0), 1 / 32, periodic=(True, False, False))
    with pytest.raises(cg.CGError) as e:
        cg.diffuse_batched([other], [dev(u0)], cg.Params(bandwidth=3 / 32, precision=3))
    assert e.value.code == "CG_EINVAL"
    xyz, tets = W.kuhn_tet_mesh(2)
    assert cg.load_library().cg_mesh_set_periodic(cg.TetMesh(xyz, tets).handle, 1, 0, 0) != 0


def test_solid_velocity_parity(cg, orc):
    """Volume and three momentum components of clustered particles with random
    velocities, coarse-grained together (mixed precision) on a mesh periodic in x: the
    GPU's solid velocity equals the oracle's division of the same smoothed fields bit for
    bit, and the smoothed fields match the oracle pipeline."""
    c = W.clustered_cube(n_side=48, n_particles=150_000, seed=73)
    rng = np.random.default_rng(74)
    vel = 0.1 * rng.standard_normal((3, c.n))
    w = np.vstack([c.w[0], c.w[0] * vel])
    mesh = cg.StructuredMesh(c.dims, c.origin, c.dx, periodic=(True, False, False))
    b = 2 * c.dx
    got = cg.coarse_grain(mesh, dev(c.pos), dev(w), cg.Params(bandwidth=b, nsteps=10, precision=3))
    eps_min = 1e-6
    us = cg.solid_velocity(mesh, got[0].contiguous(), got[1:].contiguous(), eps_min=eps_min)
    g = got.cpu().numpy()
    ref_us = orc.solid_velocity(g[0], g[1:], eps_min)
    assert np.array_equal(bits(us.cpu().numpy()), bits(ref_us))
    cell, _ = orc.locate_structured(c.dims, c.origin, c.dx, c.pos)
    eps0, _ = orc.deposit(cell, w, c.ncells, vc_uniform=c.dx ** 3)
    ref, _ = orc.diffuse_structured(eps0, c.dims, c.dx, b * b / 4, 10, tol=1e-15,
                                    periodic=(True, False, False))
    assert maxrel(g, ref) <= MIXED_TOL
    with pytest.raises(cg.CGError):   # the output may not alias an input
        cg.solid_velocity(mesh, got[0].contiguous(), got[1:].contiguous(), out=got[1:])


# nx % 4 == 0: the vectorised sweep with wrapping halos (partial row tiles, one-cell and
# four-cell axes); against the oracle and against the z-marching sweep
@pytest.mark.parametrize("dims", [(36, 13, 11), (4, 3, 5), (128, 1, 6), (8, 9, 1), (260, 17, 4)])
@pytest.mark.parametrize("periodic", [(True, True, True), (True, False, False), (False, True, False),
                                      (False, False, True)])
@pytest.mark.parametrize("shape", [101, 104])
def test_periodic_vectorised_sweep(cg, orc, dims, periodic, shape):
    rng = np.random.default_rng(75)
    n = int(np.prod(dims))
    u0 = np.vstack([rng.random(n), rng.random(n) - 0.4])
    dx = 1.0 / max(dims)
    T = (2.5 * dx) ** 2 / 4
    ref, _ = orc.diffuse_structured(u0, dims, dx, T, 8, tol=1e-15, periodic=periodic)
    mesh = cg.StructuredMesh(dims, (0, 0, 0), dx, periodic=periodic)
    out = {}
    for sh in (shape, -4):
        u = dev(u0)
        _, rep = cg.diffuse(mesh, u, cg.Params(T=T, nsteps=8, precision=3, sweep_shape=sh), report=True)
        assert rep["sweep_shape_used"] == sh
        out[sh] = u.cpu().numpy()
    assert maxrel(out[shape], ref) <= MIXED_TOL
    assert maxrel(out[shape], out[-4]) <= 1e-12

"""GPU parity of explicit Euler steps with temporal blocking (fused_k steps per launch,
FP32 storage and arithmetic) against the FP64 oracle, through the C ABI.

Bars: max-relative error <= 1e-6 against the oracle's explicit steps (FP32 rounding
grows with the step count; 40 steps at dtau/dx^2 <= 1/6 stay near 7e-7 at worst);
results bit-identical for every fused_k, including a last launch that takes the
remainder of the steps; mass conserved to 1e-6 relative (FP32 sums).
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

BAR = 1e-6


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


def run(cg, mesh, u0, T, nsteps, k, report=False):
    u = dev(u0)
    out = cg.diffuse(mesh, u, cg.Params(T=T, nsteps=nsteps, scheme=2, fused_k=k), report=report)
    return (u.cpu().numpy(), out[1]) if report else u.cpu().numpy()


# ragged tiles in x and y (the output tile is (64 - 2K) x (32 - 2K)), short z chunks
@pytest.mark.parametrize("dims", [(70, 45, 19), (128, 24, 9), (13, 70, 33), (244, 61, 12)])
@pytest.mark.parametrize("ratio", [0.1, 1 / 6])
def test_blocked_explicit_parity_and_k_independence(cg, orc, dims, ratio):
    rng = np.random.default_rng(100)
    n = int(np.prod(dims))
    u0 = np.vstack([rng.random(n), rng.random(n) - 0.5])
    dx = 1.0 / max(dims)
    nsteps = 11
    T = ratio * dx * dx * nsteps
    ref, _ = orc.diffuse_structured(u0, dims, dx, T, nsteps, scheme=2)
    mesh = cg.StructuredMesh(dims, (0, 0, 0), dx)
    got = {k: run(cg, mesh, u0, T, nsteps, k) for k in (1, 2, 3, 4)}
    assert maxrel(got[1], ref) <= BAR
    for k in (2, 3, 4):
        assert np.array_equal(bits(got[k]), bits(got[1])), k


def test_blocked_explicit_forty_steps_on_a_pcm_field(cg, orc):
    """The channel's explicit reading at reduced size: a deposited (PCM) field of the
    modulated-density particles, 40 steps at dtau/dx^2 = 0.1."""
    c = W.channel(n_particles=400_000, dims=(96, 48, 48), lengths=(4.0, 2.0, 2.0))
    cell, _ = orc.locate_structured(c.dims, c.origin, c.dx, c.pos)
    eps, _ = orc.deposit(cell, c.w, c.ncells, vc_uniform=c.dx ** 3)
    T = 0.1 * c.dx * c.dx * 40
    ref, _ = orc.diffuse_structured(eps, c.dims, c.dx, T, 40, scheme=2)
    mesh = cg.StructuredMesh(c.dims, c.origin, c.dx)
    got, rep = run(cg, mesh, eps, T, 40, 4, report=True)
    assert maxrel(got, ref) <= BAR
    assert abs(rep["mass_out"][0] - rep["mass_in"][0]) <= 1e-6 * rep["mass_in"][0]
    df = dev(eps)
    cg.diffuse(mesh, df, cg.Params(T=T, nsteps=40, scheme=2, precision=cg.PREC_FP32_DF_REFINE))
    assert maxrel(got, df.cpu().numpy()) <= BAR


# nx % 4 == 0 runs the four-cells-per-thread kernel, other nx the two-cells one
@pytest.mark.parametrize("dims", [(37, 13, 11), (6, 1, 9), (2, 9, 5), (1, 3, 4), (36, 13, 11), (4, 3, 4),
                                  (248, 7, 5)])
@pytest.mark.parametrize("periodic", [(True, True, True), (True, False, False), (False, True, True)])
def test_blocked_explicit_periodic(cg, orc, dims, periodic):
    rng = np.random.default_rng(101)
    n = int(np.prod(dims))
    u0 = rng.random((1, n))
    dx = 0.05
    T = 0.15 * dx * dx * 9
    ref, _ = orc.diffuse_structured(u0, dims, dx, T, 9, scheme=2, periodic=periodic)
    mesh = cg.StructuredMesh(dims, (0, 0, 0), dx, periodic=periodic)
    got = {k: run(cg, mesh, u0, T, 9, k) for k in (1, 4)}
    assert maxrel(got[1], ref) <= BAR
    assert np.array_equal(bits(got[4]), bits(got[1]))


def test_blocked_explicit_rejections(cg):
    mesh = cg.StructuredMesh((16, 16, 16), (0, 0, 0), 1 / 16)
    u = dev(np.ones((1, 16 ** 3)))
    for params in (cg.Params(T=1e-4, nsteps=4, scheme=2, fused_k=5),
                   cg.Params(T=1e-4, nsteps=4, scheme=0, fused_k=2),
                   cg.Params(T=1.0, nsteps=4, scheme=2, fused_k=2)):      # dtau > dx^2 / 6
        with pytest.raises(cg.CGError) as e:
            cg.diffuse(mesh, u, params)
        assert e.value.code == "CG_EINVAL"
    assert np.all(u.cpu().numpy() == 1.0)      # nothing written on error
    xyz, tets = W.kuhn_tet_mesh(2)
    tm = cg.TetMesh(xyz, tets)
    with pytest.raises(cg.CGError):
        cg.diffuse(tm, dev(np.ones((1, tm.ncells))), cg.Params(T=1e-6, nsteps=2, scheme=2, fused_k=2))

"""Degenerate diffusion inputs on every mesh kind and precision mode: T = 0 leaves the
field untouched; a mesh of one cell, a field that is zero everywhere and a constant field
are fixed points of the zero-flux diffusion (L u = 0), so every solver must return them
(the double-float modes within their 48-bit significand); a single pseudo-step matches
the oracle."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


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


def inputs():
    """Mesh descriptions (the oracle builds its own operators from these)."""
    xyz, tets = W.kuhn_tet_mesh(5, jitter=0.2, seed=120)
    f = np.linspace(0.0, 1.0, 9) ** 1.3
    faces = (f, f[:6] / f[5], f[:5] / f[4])
    D = 0.5 + np.arange(8 * 5 * 4) % 3
    return xyz, tets, faces, D


def meshes(cg):
    xyz, tets, faces, D = inputs()
    return {"structured": cg.StructuredMesh((12, 8, 6), (0, 0, 0), 1 / 12),
            "tet": cg.TetMesh(xyz, tets),
            "hex": cg.HexMesh(*faces, D)}


PRECISIONS = [0, 1, 2, 3, 4]
# A fixed point is reached to the solvers' own accuracy: each pseudo-step stops at a
# residual of tol = 1e-13 relative (the double-float residual itself bottoms out near
# 2^-48 (1 + 12 dtau/dx^2)), so over 4 steps of a well-conditioned system 1e-12 bounds
# the drift.  On one cell L = 0 and only the double-float round trip (2^-48) remains.
FIXED_TOL = 1e-12
ONE_CELL_TOL = {0: 0.0, 1: 4e-15, 2: 4e-15, 3: 4e-15, 4: 4e-15}


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("kind", ["structured", "tet", "hex"])
def test_fixed_points(cg, kind, precision):
    m = meshes(cg)[kind]
    n = m.ncells
    rng = np.random.default_rng(121)
    u0 = rng.random((2, n)) - 0.3
    # T = 0: untouched, bit for bit
    u = dev(u0)
    cg.diffuse(m, u, cg.Params(T=0.0, nsteps=3, precision=precision))
    assert np.array_equal(u.cpu().numpy(), u0)
    # zero and constant fields stay what they are
    for field in (np.zeros((2, n)), np.vstack([np.full(n, 0.37), np.full(n, -2.5)])):
        u = dev(field)
        cg.diffuse(m, u, cg.Params(bandwidth=0.2, nsteps=4, precision=precision))
        got = u.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - field)) <= FIXED_TOL * max(np.max(np.abs(field)), 1e-300)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_one_cell_mesh(cg, precision):
    m = cg.StructuredMesh((1, 1, 1), (0, 0, 0), 0.1)
    u0 = np.array([[3.25], [-1e-3]])
    u = dev(u0)
    cg.diffuse(m, u, cg.Params(bandwidth=0.5, nsteps=7, precision=precision))
    assert np.max(np.abs(u.cpu().numpy() - u0) / np.abs(u0)) <= ONE_CELL_TOL[precision]


@pytest.mark.parametrize("precision,bar", [(0, 1e-10), (1, 1e-6), (3, 1e-6)])
@pytest.mark.parametrize("kind", ["structured", "tet", "hex"])
def test_single_step_matches_oracle(cg, orc, kind, precision, bar):
    m = meshes(cg)[kind]
    rng = np.random.default_rng(122)
    u0 = rng.random((1, m.ncells))
    T = 2e-3
    xyz, tets, faces, D = inputs()
    if kind == "structured":
        ref, _ = orc.diffuse_structured(u0, (12, 8, 6), 1 / 12, T, 1, tol=1e-15)
    else:
        if kind == "tet":
            vc, _, rp, col, val = orc.tet_build(xyz, tets)
        else:
            vc, rp, col, val = orc.hex_build(*faces, D)
        ref, _ = orc.diffuse_csr(u0, vc, rp, col, val, T, 1, tol=1e-15)
    u = dev(u0)
    cg.diffuse(m, u, cg.Params(T=T, nsteps=1, precision=precision))
    got = u.cpu().numpy()
    ref = np.atleast_2d(ref)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= bar


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("kind", ["structured", "tet", "hex"])
def test_empty_particle_set(cg, kind, mode):
    """No particles: the deposited fields are zero in both deposition modes, and so is
    the coarse-grained result (zero is a fixed point of the diffusion), with zero mass in
    and out and nothing out of the domain."""
    import torch
    m = meshes(cg)[kind]
    pos, w = dev(np.zeros((3, 0))), dev(np.zeros((2, 0)))
    sentinel = torch.full((2, m.ncells), 7.0, dtype=torch.float64, device="cuda")
    out = cg.deposit(m, pos, w, cg.Params(deposit_mode=mode), out=sentinel)
    assert torch.count_nonzero(out).item() == 0
    for precision in (0, 3):
        u, rep = cg.coarse_grain(m, pos, w, cg.Params(bandwidth=0.2, nsteps=3, precision=precision,
                                                      deposit_mode=mode), report=True)
        assert u.shape == (2, m.ncells)
        assert torch.count_nonzero(u).item() == 0
        assert rep["n_out_of_domain"] == 0
        assert rep["mass_in"][:2] == [0.0, 0.0] and rep["mass_out"][:2] == [0.0, 0.0]

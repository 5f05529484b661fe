"""GPU parity of the unstructured (tetrahedral) path against the FP64 oracle, via the C ABI.

Bars as for the structured path: locate and deposition bit-exact; diffusion max-relative
error <= 1e-10 (FP64 PCG) and <= 1e-6 (FP32/BF16 inner solves with FP64 refinement);
mass conserved to 1e-12.  The full-size mesh (100^3 hexes -> 6,000,000 Kuhn tets,
5,000,000 particles in a dense bottom layer) is checked against the oracle on every
particle (its bucketed search), bit for bit in the deposition, and in the diffusion.
"""
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


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


def maxrel(u, ref):
    u, ref = np.atleast_2d(u), np.atleast_2d(ref)
    return max(np.max(np.abs(u[f] - ref[f])) / np.max(np.abs(ref[f])) for f in range(ref.shape[0]))


@pytest.fixture(scope="module")
def small_mesh(cg):
    xyz, tets = W.kuhn_tet_mesh(9, jitter=0.2, seed=4)
    return xyz, tets, cg.TetMesh(xyz, tets)


def test_tet_operator_matches_oracle_build(cg, orc, small_mesh):
    xyz, tets, mesh = small_mesh
    vc, cent, rp, col, val = orc.tet_build(xyz, tets)
    assert np.max(np.abs(mesh.cell_volumes() - vc)) <= 1e-15 * vc.max()
    grp, gcol, gval = mesh.operator()
    assert np.array_equal(grp, rp) and np.array_equal(gcol, col)
    assert np.max(np.abs(gval - val)) <= 1e-13 * np.max(np.abs(val))


def test_tet_locate_bit_exact(cg, orc, small_mesh):
    xyz, tets, mesh = small_mesh
    rng = np.random.default_rng(21)
    pos = rng.random((3, 30_000))
    k = 2000
    pos[:, :k] = xyz[rng.integers(0, len(xyz), k)].T                 # exactly on vertices
    fc = xyz[tets[rng.integers(0, len(tets), k)][:, :3]].mean(axis=1)  # on face planes
    pos[:, k:2 * k] = fc.T
    pos[:, 2 * k] = (1.2, 0.5, 0.5)                                  # outside
    pos[:, 2 * k + 1] = (0.5, np.nan, 0.5)
    ref, nref = orc.locate_tet(xyz, tets, pos)
    got, nout = cg.locate(mesh, dev(pos))
    assert nout == nref
    assert np.array_equal(got.cpu().numpy(), ref)


def test_tet_locate_bucket_ordered_bit_exact(cg, orc, small_mesh):
    """A set large enough to be grouped by point-location bucket before the search
    (at least 65,536 particles): the same cells as the oracle, including points on
    vertices and faces, outside the mesh and not finite; deposition bit-exact too."""
    xyz, tets, mesh = small_mesh
    rng = np.random.default_rng(23)
    n = 90_000
    pos = rng.random((3, n))
    k = 3000
    pos[:, :k] = xyz[rng.integers(0, len(xyz), k)].T
    fc = xyz[tets[rng.integers(0, len(tets), k)][:, :3]].mean(axis=1)
    pos[:, k:2 * k] = fc.T
    pos[:, 2 * k] = (1.2, 0.5, 0.5)
    pos[:, 2 * k + 1] = (0.5, np.nan, 0.5)
    pos[:, 2 * k + 2] = (-np.inf, 0.5, 0.5)
    perm = rng.permutation(n)
    pos = pos[:, perm]
    ref, nref = orc.locate_tet(xyz, tets, pos)
    got, nout = cg.locate(mesh, dev(pos))
    assert nout == nref == 3
    assert np.array_equal(got.cpu().numpy(), ref)
    inside = ref >= 0
    p_in = pos[:, inside]
    w = np.vstack([np.full(p_in.shape[1], 3e-7), rng.standard_normal(p_in.shape[1])])
    vc, *_ = orc.tet_build(xyz, tets)
    for mode in (0, 1):
        eps, _ = orc.deposit(ref[inside], w, len(tets), vc=vc, mode=mode)
        d = cg.deposit(mesh, dev(p_in), dev(w), cg.Params(deposit_mode=mode)).cpu().numpy()
        assert np.array_equal(bits(d), bits(eps))


@pytest.mark.parametrize("mode", [0, 1])
def test_tet_deposit_bit_exact(cg, orc, small_mesh, mode):
    xyz, tets, mesh = small_mesh
    rng = np.random.default_rng(22)
    pos, _ = W.layered_positions(rng, 40_000, d=0.02)
    w = np.vstack([np.full(40_000, 4.2e-6), rng.standard_normal(40_000)])
    cell, nout = orc.locate_tet(xyz, tets, pos)
    assert nout == 0
    vc, *_ = orc.tet_build(xyz, tets)
    ref, _ = orc.deposit(cell, w, len(tets), vc=vc, mode=mode)
    got = cg.deposit(mesh, dev(pos), dev(w), cg.Params(deposit_mode=mode)).cpu().numpy()
    assert np.array_equal(bits(got), bits(ref))


# inner solver of the mixed modes: 0 = Chebyshev after a PCG spectrum estimate, 1 = PCG
@pytest.mark.parametrize("precision,bar,shape", [(0, 1e-10, 0), (1, 1e-6, 0), (2, 1e-6, 0),
                                                 (1, 1e-6, 1), (2, 1e-6, 1)])
@pytest.mark.parametrize("scheme", [0, 1])
def test_tet_diffuse_parity(cg, orc, small_mesh, scheme, precision, bar, shape):
    xyz, tets, mesh = small_mesh
    vc, cent, rp, col, val = orc.tet_build(xyz, tets)
    nt = len(vc)
    rng = np.random.default_rng(23)
    u0 = np.zeros((2, nt))
    u0[0, rng.integers(0, nt, 300)] = rng.random(300) * 10
    u0[1] = rng.random(nt) - 0.3
    b = 3.0 / 9
    T = b * b / 4
    ref, _ = orc.diffuse_csr(u0, vc, rp, col, val, T, 10, scheme=scheme, tol=1e-15)
    u = dev(u0)
    _, rep = cg.diffuse(mesh, u, cg.Params(bandwidth=b, nsteps=10, scheme=scheme,
                                           precision=precision, sweep_shape=shape), report=True)
    got = u.cpu().numpy()
    assert maxrel(got, ref) <= bar
    assert rep["final_rel_residual"] <= 1e-13
    mass0 = (vc * np.abs(u0)).sum(axis=1)
    assert np.all(np.abs(np.array(rep["mass_out"][:2]) - np.array(rep["mass_in"][:2])) <= 1e-12 * mass0)


def test_tet_explicit_parity(cg, orc, small_mesh):
    xyz, tets, mesh = small_mesh
    vc, cent, rp, col, val = orc.tet_build(xyz, tets)
    rng = np.random.default_rng(24)
    u0 = rng.random(len(vc))
    rate = np.max(-val[col == np.repeat(np.arange(len(vc)), np.diff(rp))] / vc)
    T = 0.9 / rate * 20
    ref, _ = orc.diffuse_csr(u0, vc, rp, col, val, T, 20, scheme=2)
    u = dev(u0[None])
    cg.diffuse(mesh, u, cg.Params(T=T, nsteps=20, scheme=2))
    assert maxrel(u.cpu().numpy(), ref) <= 1e-13
    with pytest.raises(cg.CGError):                      # beyond the stability limit
        cg.diffuse(mesh, dev(u0[None]), cg.Params(T=3.0 / rate * 20, nsteps=20, scheme=2))


def _near_face_points(xyz, tets, rng, k, eps=1e-12):
    """k points within eps of a face of random tets (a random point of the face, moved
    by at most eps along a random direction), inside the unit cube."""
    t = tets[rng.integers(0, len(tets), k)]
    f = np.stack([rng.permutation(4)[:3] for _ in range(k)])
    corners = xyz[np.take_along_axis(t, f, axis=1)]             # [k, 3, 3]
    lam = rng.dirichlet(np.ones(3), size=k)
    p = np.einsum("kj,kja->ka", lam, corners)
    d = rng.standard_normal((k, 3))
    d *= (rng.random((k, 1)) * eps) / np.linalg.norm(d, axis=1, keepdims=True)
    return np.clip(p + d, 0.0, 1.0).T


def test_tet_full_size_layered(cg, orc):
    """Configuration of the paper's unstructured case (Section 4.3) at full size: 100^3
    hexes -> 6,000,000 jittered Kuhn tets, 5,000,000 spheres (d = 0.003) with a dense
    bottom layer, b = 0.03, 10 implicit-Euler steps.  Against the oracle: every
    particle's tet (the oracle's bucketed search, the same rule as its brute force),
    plus 2,000 particles half of them within 1e-12 of a face, both alone and inside a
    set large enough for the bucket-ordered search; the ordered deposition bit for bit;
    the oracle's 10 FP64 CG steps against FP64 PCG (1e-10) and the mixed modes (1e-6,
    Chebyshev and PCG inner solves); mass to 1e-12; non-negativity."""
    import torch
    xyz, tets = W.kuhn_tet_mesh(100, jitter=0.2, seed=0)
    mesh = cg.TetMesh(xyz, tets)
    assert mesh.ncells == 6_000_000
    pos, w, h = W.layered_cube()
    dpos, dw = dev(pos), dev(w)
    # locate: all 5,000,000 particles
    ref_cell, nref = orc.locate_tet_bucketed(xyz, tets, pos)
    assert nref == 0
    cell, nout = cg.locate(mesh, dpos)
    assert nout == 0
    assert np.array_equal(cell.cpu().numpy(), ref_cell)
    # locate: 2,000 particles, half within 1e-12 of a face, alone and among 98,000 others
    rng = np.random.default_rng(25)
    special = np.hstack([pos[:, rng.choice(pos.shape[1], 1000, replace=False)],
                         _near_face_points(xyz, tets, rng, 1000)])
    ref_s, nref_s = orc.locate_tet_bucketed(xyz, tets, special)
    got_s, nout_s = cg.locate(mesh, dev(special))
    assert nout_s == nref_s
    assert np.array_equal(got_s.cpu().numpy(), ref_s)
    mixed_set = np.hstack([pos[:, :98_000], special])[:, rng.permutation(100_000)]
    ref_m, _ = orc.locate_tet_bucketed(xyz, tets, mixed_set)
    got_m, _ = cg.locate(mesh, dev(mixed_set))
    assert np.array_equal(got_m.cpu().numpy(), ref_m)
    # deposition, bit for bit, on the oracle's own cells and volumes
    vc, cent, rp, col, val = orc.tet_build(xyz, tets)
    eps0, _ = orc.deposit(ref_cell, w, len(tets), vc=vc, mode=0)
    got0 = cg.deposit(mesh, dpos, dw).cpu().numpy()
    assert np.array_equal(bits(got0), bits(eps0))
    # diffusion: the oracle's FP64 CG against the GPU modes
    b = 0.03
    ref, _ = orc.diffuse_csr(eps0, vc, rp, col, val, b * b / 4, 10, scheme=0, tol=1e-14)
    f64 = cg.coarse_grain(mesh, dpos, dw, cg.Params(bandwidth=b, nsteps=10, precision=0))
    assert maxrel(f64.cpu().numpy(), ref) <= 1e-10
    mixed, rep = cg.coarse_grain(mesh, dpos, dw, cg.Params(bandwidth=b, nsteps=10,
                                                           precision=1), report=True)
    m = mixed.cpu().numpy()
    assert maxrel(m, ref) <= 1e-6
    assert abs(rep["mass_out"][0] - w.sum()) <= 1e-12 * w.sum()
    assert abs(rep["mass_in"][0] - w.sum()) <= 1e-12 * w.sum()
    assert m.min() >= -1e-12 * m.max()
    pcg = cg.coarse_grain(mesh, dpos, dw, cg.Params(bandwidth=b, nsteps=10, precision=1,
                                                    sweep_shape=1))    # PCG inner solves
    assert maxrel(pcg.cpu().numpy(), ref) <= 1e-6
    mesh.close()
    del dpos, dw, f64, mixed, pcg
    torch.cuda.empty_cache()


def test_tet_mixed_results_do_not_depend_on_call_history(cg, small_mesh):
    """The Chebyshev interval comes from a probe on a fixed right-hand side and is
    remembered per mesh and dtau, so a call gives the same bits on a fresh mesh and on a
    mesh that has already smoothed other fields with other step sizes."""
    import torch
    xyz, tets, _ = small_mesh
    a, b = cg.TetMesh(xyz, tets), cg.TetMesh(xyz, tets)
    rng = np.random.default_rng(26)
    x = dev(rng.random((1, a.ncells)))
    y = dev(rng.random((2, a.ncells)) - 0.3)
    p = cg.Params(bandwidth=0.3, nsteps=10, precision=1)
    cg.diffuse(a, x.clone(), cg.Params(bandwidth=0.2, nsteps=5, precision=1))
    cg.diffuse(a, x.clone(), p)
    ya, yb, yc = y.clone(), y.clone(), y.clone()
    cg.diffuse(a, ya, p)
    cg.diffuse(b, yb, p)
    cg.diffuse(b, yc, p)
    assert torch.equal(ya, yb) and torch.equal(yb, yc)

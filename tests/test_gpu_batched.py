"""GPU parity of batched snapshots (all snapshots, steps and fields in one persistent
launch, or in one launch per phase, captured as one graph) against the FP64 oracle and
against the single-mesh path, through the C ABI.

Bars: mixed modes <= 1e-6 max-relative error per snapshot and field against the oracle;
mass conserved to 1e-12 of sum |w| per field; the persistent kernel's grid barrier gives
up with CG_ETIMEOUT when its wait budget runs out.
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


def maxrel(u, ref):
    u, ref = np.atleast_2d(u), np.atleast_2d(ref)
    return max(np.max(np.abs(u[f] - ref[f])) / max(np.max(np.abs(ref[f])), 1e-300)
               for f in range(ref.shape[0]))


def small_batch():
    cases = W.batched_snapshots(n_snap=6, side_lo=13, side_hi=40, logn_lo=3.0, logn_hi=4.3, seed=31)
    cases[0].dims = (24, 24, 24)          # sides that are multiples of 4 (vectorised sweeps)
    cases[0].dx = 1.0 / 24
    cases[0].b = 3.0 / 24
    cases[1].dims = (40, 40, 40)
    cases[1].dx = 1.0 / 40
    cases[1].b = 3.0 / 40
    return cases


@pytest.mark.parametrize("precision,scheme", [(3, 0), (4, 0), (3, 1)])
def test_batched_matches_oracle_per_snapshot(cg, orc, precision, scheme):
    cases = small_batch()
    meshes = [cg.StructuredMesh(c.dims, c.origin, c.dx) for c in cases]
    pos = [dev(c.pos) for c in cases]
    w = [dev(c.w) for c in cases]
    bws = [c.b for c in cases]
    out, rep = cg.coarse_grain_batched(meshes, pos, w, cg.Params(nsteps=10, precision=precision,
                                                                 scheme=scheme),
                                       bandwidths=bws, report=True)
    for c, o in zip(cases, out):
        _, ref, nout, _ = orc.coarse_grain_structured(c.dims, c.origin, c.dx, c.pos, c.w, c.b,
                                                      c.nsteps, scheme=scheme)
        assert nout == 0
        assert maxrel(o.cpu().numpy(), ref) <= MIXED_TOL
    scale = np.array([sum(np.abs(c.w[f]).sum() for c in cases) for f in range(5)])
    m_in, m_out = np.array(rep["mass_in"][:5]), np.array(rep["mass_out"][:5])
    assert np.all(np.abs(m_out - m_in) <= 1e-12 * scale)
    assert rep["final_rel_residual"] <= 1e-13


def test_batched_agrees_with_single_mesh_path(cg):
    cases = small_batch()
    meshes = [cg.StructuredMesh(c.dims, c.origin, c.dx) for c in cases]
    pos = [dev(c.pos) for c in cases]
    w = [dev(c.w) for c in cases]
    bws = [c.b for c in cases]
    out = cg.coarse_grain_batched(meshes, pos, w, cg.Params(nsteps=10, precision=3), bandwidths=bws)
    for m, p_, w_, b, o in zip(meshes, pos, w, bws, out):
        single = cg.coarse_grain(m, p_, w_, cg.Params(bandwidth=b, nsteps=10, precision=0))
        assert maxrel(o.cpu().numpy(), single.cpu().numpy()) <= 1e-10


def test_batched_phased_and_persistent_schedules_give_the_same_bits(cg):
    """The phased schedule (one launch per phase) evaluates every cell's update as the
    persistent launch does, so both give the same bits, for any work-item depth."""
    import torch
    cases = small_batch()
    meshes = [cg.StructuredMesh(c.dims, c.origin, c.dx) for c in cases]
    pos = [dev(c.pos) for c in cases]
    w = [dev(c.w) for c in cases]
    bws = [c.b for c in cases]
    outs = []
    for shape in (8, 508, 4, 516):
        out, rep = cg.coarse_grain_batched(meshes, pos, w, cg.Params(nsteps=10, precision=3,
                                                                     sweep_shape=shape),
                                           bandwidths=bws, report=True)
        assert rep["sweep_shape_used"] == shape
        outs.append([o.clone() for o in out])
    for o in outs[1:]:
        assert all(torch.equal(a, b) for a, b in zip(outs[0], o))


def test_batched_full_size_64_snapshots(cg, orc):
    """64 snapshots, cube sides 32..96, 10^4..10^6 particles, 5 fields, b = 3 dx, the
    autotuned schedule (as the benchmark runs it); three snapshots checked against the
    oracle, and the persistent launch gives the same bits."""
    import torch
    cases = W.batched_snapshots()
    meshes = [cg.StructuredMesh(c.dims, c.origin, c.dx) for c in cases]
    pos = [dev(c.pos) for c in cases]
    w = [dev(c.w) for c in cases]
    out, rep = cg.coarse_grain_batched(meshes, pos, w, cg.Params(nsteps=10, precision=3),
                                       bandwidths=[c.b for c in cases], report=True)
    scale = np.array([sum(np.abs(c.w[f]).sum() for c in cases) for f in range(5)])
    assert np.all(np.abs(np.array(rep["mass_out"][:5]) - np.array(rep["mass_in"][:5])) <= 1e-12 * scale)
    assert rep["final_rel_residual"] <= 1e-13
    for s in (0, 17, 63):
        c = cases[s]
        _, ref, _, _ = orc.coarse_grain_structured(c.dims, c.origin, c.dx, c.pos, c.w, c.b, c.nsteps)
        assert maxrel(out[s].cpu().numpy(), ref) <= MIXED_TOL
    out = [o.clone() for o in out]
    other = 16 if rep["sweep_shape_used"] >= 500 else 516
    out2 = cg.coarse_grain_batched(meshes, pos, w, cg.Params(nsteps=10, precision=3,
                                                             sweep_shape=other),
                                   bandwidths=[c.b for c in cases])
    assert all(torch.equal(a, b) for a, b in zip(out, out2))


def test_batched_barrier_timeout(cg):
    cases = small_batch()[:3]
    meshes = [cg.StructuredMesh(c.dims, c.origin, c.dx) for c in cases]
    pos = [dev(c.pos) for c in cases]
    w = [dev(c.w) for c in cases]
    with pytest.raises(cg.CGError) as e:
        cg.coarse_grain_batched(meshes, pos, w, cg.Params(nsteps=2, precision=3, barrier_budget=1),
                                bandwidths=[c.b for c in cases])
    assert e.value.code == "CG_ETIMEOUT"
    out = cg.coarse_grain_batched(meshes, pos, w, cg.Params(nsteps=2, precision=3),
                                  bandwidths=[c.b for c in cases])
    assert all(np.isfinite(o.cpu().numpy()).all() for o in out)


def test_batched_rejects_shared_meshes_and_tets(cg):
    m = cg.StructuredMesh((8, 8, 8), (0, 0, 0), 0.125)
    cells = [dev(np.zeros((1, 512))), dev(np.zeros((1, 512)))]
    with pytest.raises(cg.CGError) as e:
        cg.diffuse_batched([m, m], cells, cg.Params(bandwidth=0.2, precision=3))
    assert e.value.code == "CG_EINVAL"
    xyz, tets = W.kuhn_tet_mesh(2)
    t = cg.TetMesh(xyz, tets)
    with pytest.raises(cg.CGError):
        cg.diffuse_batched([t], [dev(np.zeros((1, t.ncells)))], cg.Params(bandwidth=0.2, precision=3))


@pytest.mark.parametrize("zlen", [4, 16, 504, 516])
def test_batched_tile_override_matches_oracle(cg, orc, zlen):
    """Work items of 4 or 16 z-planes, in the persistent launch (4, 16) or one launch per
    phase (504, 516) -- the autotuner's other candidates -- give the same answers as the
    oracle; the report names the schedule that ran."""
    cases = small_batch()[:4]
    meshes = [cg.StructuredMesh(c.dims, c.origin, c.dx) for c in cases]
    pos = [dev(c.pos) for c in cases]
    w = [dev(c.w) for c in cases]
    out, rep = cg.coarse_grain_batched(meshes, pos, w, cg.Params(nsteps=10, precision=3,
                                                                 sweep_shape=zlen),
                                       bandwidths=[c.b for c in cases], report=True)
    assert rep["sweep_shape_used"] == zlen
    for c, o in zip(cases, out):
        _, ref, _, _ = orc.coarse_grain_structured(c.dims, c.origin, c.dx, c.pos, c.w, c.b, c.nsteps)
        assert maxrel(o.cpu().numpy(), ref) <= MIXED_TOL


def test_batched_graph_replay_is_deterministic(cg):
    """The first call tunes the z-chunk and captures the schedule; later calls replay the
    captured graph and must reproduce the first call's bits."""
    cases = small_batch()
    meshes = [cg.StructuredMesh(c.dims, c.origin, c.dx) for c in cases]
    pos = [dev(c.pos) for c in cases]
    w = [dev(c.w) for c in cases]
    bws = [c.b for c in cases]
    runs = []
    for _ in range(3):
        out, rep = cg.coarse_grain_batched(meshes, pos, w, cg.Params(nsteps=10, precision=3),
                                           bandwidths=bws, report=True)
        assert rep["sweep_shape_used"] in (4, 8, 16, 504, 508, 516)
        runs.append([o.cpu().numpy().view(np.int64) for o in out])
    for r in runs[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(runs[0], r))


def test_batched_unreachable_tol_leaves_last_iterate(cg, orc):
    """A tolerance below double-float resolution cannot be met: CG_ENOCONV, with the last
    iterate (still within the mixed bar of the oracle) written to the caller's arrays."""
    cases = small_batch()[:2]
    meshes = [cg.StructuredMesh(c.dims, c.origin, c.dx) for c in cases]
    cells = [dev(orc.deposit(orc.locate_structured(c.dims, c.origin, c.dx, c.pos)[0], c.w,
                             int(np.prod(c.dims)), vc_uniform=c.dx * c.dx * c.dx)[0])
             for c in cases]
    with pytest.raises(cg.CGError) as e:
        cg.diffuse_batched(meshes, cells, cg.Params(nsteps=10, precision=3, tol=1e-17,
                                                    max_rounds=3),
                           bandwidths=[c.b for c in cases])
    assert e.value.code == "CG_ENOCONV"
    for c, u in zip(cases, cells):
        _, ref, _, _ = orc.coarse_grain_structured(c.dims, c.origin, c.dx, c.pos, c.w, c.b, c.nsteps)
        assert maxrel(u.cpu().numpy(), ref) <= MIXED_TOL


def test_batched_degenerate_and_boundary_shapes(cg, orc):
    """Snapshots with one-cell axes, a plane of one chunk, rows of exactly 512 cells (the
    flat-plane engine's limit) and 513 cells (the 2.5D tiles), in one batch: each smoothed
    field matches the oracle, and the phased and persistent schedules give the same bits."""
    import torch
    dims_list = [(1, 7, 5), (7, 1, 3), (5, 6, 1), (512, 3, 2), (513, 2, 2), (33, 31, 29),
                 (2, 2, 2), (40, 26, 3)]
    rng = np.random.default_rng(41)
    dx = 0.1
    meshes = [cg.StructuredMesh(d, (0.0, 0.0, 0.0), dx) for d in dims_list]
    u0 = [rng.random((2, int(np.prod(d)))) - np.array([[0.0], [0.4]]) for d in dims_list]
    bws = [2 * dx] * len(dims_list)
    outs = []
    for shape in (504, 4):
        cells = [dev(u) for u in u0]
        cg.diffuse_batched(meshes, cells, cg.Params(nsteps=10, precision=3, sweep_shape=shape),
                           bandwidths=bws)
        outs.append(cells)
    assert all(torch.equal(a, b) for a, b in zip(*outs))
    for d, u, got in zip(dims_list, u0, outs[0]):
        ref, _ = orc.diffuse_structured(u, d, dx, (2 * dx) ** 2 / 4, 10, tol=1e-14)
        assert maxrel(got.cpu().numpy(), ref) <= MIXED_TOL, d


def test_batched_deposition_checks_every_snapshot_before_writing(cg):
    """The batch locates every snapshot's particles before writing any deposited field: a
    snapshot with a particle outside its mesh fails the call with CG_EDOMAIN, names that
    snapshot, and leaves every snapshot's cells untouched; a valid batch reports the
    batch's phase times."""
    import torch
    cases = small_batch()
    meshes = [cg.StructuredMesh(c.dims, c.origin, c.dx) for c in cases]
    pos = [dev(c.pos) for c in cases]
    w = [dev(c.w) for c in cases]
    bad = [p.clone() for p in pos]
    bad[2][1, 3] = 2.5                               # outside the unit cube
    out = [torch.full((c.w.shape[0], m.ncells), float("nan"), dtype=torch.float64, device="cuda")
           for c, m in zip(cases, meshes)]
    prm = cg.Params(nsteps=2, precision=3)
    with pytest.raises(cg.CGError) as e:
        cg.coarse_grain_batched(meshes, bad, w, prm, bandwidths=[c.b for c in cases], out=out)
    assert e.value.code == "CG_EDOMAIN" and "snapshot 2" in str(e.value)
    assert all(bool(torch.isnan(o).all()) for o in out)
    # the same batch with valid particles: every deposition runs (the batch's parity
    # against the oracle is checked above), the report covers the whole batch
    _, rep = cg.coarse_grain_batched(meshes, pos, w, prm, bandwidths=[c.b for c in cases], out=out,
                                     report=True)
    assert not any(bool(torch.isnan(o).any()) for o in out)
    assert rep["n_out_of_domain"] == 0 and rep["ms_locate"] > 0 and rep["ms_deposit"] > 0
    for m in meshes:
        m.close()

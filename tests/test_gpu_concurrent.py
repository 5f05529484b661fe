"""Concurrent independent coarse-grainings (cg_coarse_grain_concurrent): every problem's
result and report equal those of cg_coarse_grain on the same arguments, bit for bit, for
any concurrency; failures name the lowest failing problem; misuse is refused."""
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


@pytest.fixture(scope="module")
def problems(cg):
    """Four bandwidths of one clustered case, a second structured case and a tet mesh."""
    c = W.clustered_cube(n_side=48, n_particles=200_000, seed=11)
    u = W.uniform_cube(n_side=40, n_particles=50_000, seed=12)
    xyz, tets = W.kuhn_tet_mesh(12, jitter=0.2, seed=13)
    rng = np.random.default_rng(14)
    tp = rng.random((3, 30_000))
    tw = np.vstack([np.full(30_000, 1e-6), rng.standard_normal(30_000)])
    probs = []
    for bdx in (1.0, 2.0, 4.0, 8.0):
        probs.append((cg.StructuredMesh(c.dims, c.origin, c.dx), dev(c.pos), dev(np.vstack([c.w, c.w])),
                      cg.Params(bandwidth=bdx * c.dx, nsteps=10, precision=3)))
    probs.append((cg.StructuredMesh(u.dims, u.origin, u.dx), dev(u.pos), dev(np.vstack([u.w, -u.w])),
                  cg.Params(bandwidth=u.b, nsteps=10, precision=0)))
    probs.append((cg.TetMesh(xyz, tets), dev(tp), dev(tw), cg.Params(bandwidth=0.1, nsteps=5, precision=1)))
    # sequential results first (this also autotunes every mesh in isolation)
    ref = [cg.coarse_grain(m, p, w, prm, report=True) for m, p, w, prm in probs]
    return probs, [(u_.clone(), r) for u_, r in ref]


@pytest.mark.parametrize("k", [1, 2, 4, 6])
def test_concurrent_equals_sequential(cg, problems, k):
    import torch
    probs, ref = problems
    out, reps = cg.coarse_grain_concurrent([p[0] for p in probs], [p[1] for p in probs],
                                           [p[2] for p in probs], [p[3] for p in probs],
                                           max_concurrent=k, report=True)
    for (u_ref, r_ref), u, r in zip(ref, out, reps):
        assert torch.equal(u, u_ref)
        for key in ("cell_updates", "refine_rounds", "iters", "final_rel_residual", "n_out_of_domain"):
            assert r[key] == r_ref[key], key
        assert r["mass_out"] == r_ref["mass_out"]


def test_concurrent_failure_and_misuse(cg, problems):
    probs, _ = problems
    meshes = [p[0] for p in probs[:3]]
    pos = [p[1] for p in probs[:3]]
    bad = pos[1].clone()
    bad[0, 5] = 7.0                      # outside the unit cube: problem 1 fails
    w = [p[2] for p in probs[:3]]
    prm = [p[3] for p in probs[:3]]
    with pytest.raises(cg.CGError) as e:
        cg.coarse_grain_concurrent(meshes, [pos[0], bad, pos[2]], w, prm, max_concurrent=3)
    assert e.value.code == "CG_EDOMAIN" and "problem 1" in str(e.value)
    with pytest.raises(cg.CGError) as e:                      # a mesh used twice
        cg.coarse_grain_concurrent([meshes[0], meshes[0]], pos[:2], w[:2], prm[:2])
    assert e.value.code == "CG_EINVAL"
    with pytest.raises(cg.CGError):
        cg.coarse_grain_concurrent(meshes, pos, w, prm, max_concurrent=0)
    cg.profile_enable(True)
    try:
        with pytest.raises(cg.CGError) as e:
            cg.coarse_grain_concurrent(meshes, pos, w, prm)
        assert "profiling" in str(e.value)
    finally:
        cg.profile_enable(False)


def test_concurrent_host_buffers_equal_device_run(cg, problems):
    """Host inputs and outputs: each problem runs as cg_coarse_grain_host (copies in and
    out) and gives the device run's bits."""
    import torch
    probs, ref = problems
    pos = [p[1].cpu().pin_memory() for p in probs]
    w = [p[2].cpu().pin_memory() for p in probs]
    out, reps = cg.coarse_grain_concurrent([p[0] for p in probs], pos, w, [p[3] for p in probs],
                                           max_concurrent=3, report=True)
    for (u_ref, r_ref), u, r in zip(ref, out, reps):
        assert not u.is_cuda
        assert torch.equal(u, u_ref.cpu())
        assert r["cell_updates"] == r_ref["cell_updates"]


@pytest.mark.parametrize("k", [1, 3])
def test_concurrent_shared_host_inputs(cg, problems, k):
    """The four bandwidths of one particle set given the same host arrays share one copy
    of them (made before any problem starts); the other problems copy their own.  Every
    result equals the device run's bits, whichever problems run together."""
    import torch
    probs, ref = problems
    pos0, w0 = probs[0][1].cpu().pin_memory(), probs[0][2].cpu().pin_memory()
    for p in probs[1:4]:
        assert torch.equal(p[1].cpu(), pos0) and torch.equal(p[2].cpu(), w0)
    pos = [pos0] * 4 + [p[1].cpu().pin_memory() for p in probs[4:]]
    w = [w0] * 4 + [p[2].cpu().pin_memory() for p in probs[4:]]
    out, reps = cg.coarse_grain_concurrent([p[0] for p in probs], pos, w, [p[3] for p in probs],
                                           max_concurrent=k, report=True)
    for (u_ref, r_ref), u, r in zip(ref, out, reps):
        assert torch.equal(u, u_ref.cpu())
        assert r["cell_updates"] == r_ref["cell_updates"]
    # the inputs are untouched and a second call (buffers reused) gives the same bits
    assert torch.equal(pos0, probs[0][1].cpu())
    out2 = cg.coarse_grain_concurrent([p[0] for p in probs], pos, w, [p[3] for p in probs], max_concurrent=k)
    for a, b in zip(out, out2):
        assert torch.equal(a, b)


def test_concurrent_full_size_benchmark_configuration(cg):
    """The benchmark's step as it times it: the 128^3 clustered case (2,000,000 spheres)
    at b/dx = 1, 2, 4, 8, two problems at a time -- the same bits as four calls in a row."""
    import torch
    c = W.clustered_cube()
    pos, w = dev(c.pos), dev(c.w)
    meshes = [cg.StructuredMesh(c.dims, c.origin, c.dx) for _ in range(4)]
    prm = [cg.Params(bandwidth=b * c.dx, nsteps=10, precision=3, tol=1e-13) for b in (1.0, 2.0, 4.0, 8.0)]
    seq = [cg.coarse_grain(m, pos, w, p) for m, p in zip(meshes, prm)]
    out = cg.coarse_grain_concurrent(meshes, [pos] * 4, [w] * 4, prm, max_concurrent=2)
    for a, b in zip(out, seq):
        assert torch.equal(a, b)


@pytest.mark.parametrize("k", [1, 2, 4])
def test_concurrent_shared_deposition(cg, problems, k):
    """Problems given the same device particle arrays on meshes of one geometry deposit
    once (the first to start, here the largest bandwidth); every result and every
    report field but the deposition times equal the sequential run's, bit for bit."""
    import torch
    probs, ref = problems
    pos0, w0 = probs[0][1], probs[0][2]
    pos = [pos0] * 4 + [p[1] for p in probs[4:]]
    w = [w0] * 4 + [p[2] for p in probs[4:]]
    out, reps = cg.coarse_grain_concurrent([p[0] for p in probs], pos, w, [p[3] for p in probs],
                                           max_concurrent=k, report=True)
    for (u_ref, r_ref), u, r in zip(ref, out, reps):
        assert torch.equal(u, u_ref)
        for key in ("cell_updates", "refine_rounds", "iters", "final_rel_residual", "n_out_of_domain",
                    "fixed_point_bits"):
            assert r[key] == r_ref[key], key
        assert r["mass_in"] == r_ref["mass_in"] and r["mass_out"] == r_ref["mass_out"]
    deposited = [i for i in range(4) if reps[i]["ms_locate"] + reps[i]["ms_deposit"] > 0]
    assert deposited == [3]                                      # b = 8 dx starts first
    assert all(reps[i]["ms_locate"] + reps[i]["ms_deposit"] > 0 for i in range(4, len(probs)))


def test_concurrent_shared_deposition_mixed_geometry_and_failure(cg, problems):
    """Only problems on meshes of the same geometry and deposition mode share; a shared
    set whose deposition fails runs unshared and every member reports the failure."""
    import torch
    probs, ref = problems
    c = W.clustered_cube(n_side=48, n_particles=200_000, seed=11)
    pos0, w0 = probs[0][1], probs[0][2]
    # one more cell column, the mesh shifted by it: the same particles, another geometry
    shifted = cg.StructuredMesh((c.dims[0] + 1, c.dims[1], c.dims[2]),
                                (c.origin[0] - c.dx, c.origin[1], c.origin[2]), c.dx)
    fixed = cg.Params(bandwidth=2.0 * c.dx, nsteps=10, precision=3, deposit_mode=1)
    meshes = [probs[0][0], probs[1][0], shifted, probs[2][0]]
    prm = [probs[0][3], probs[1][3], probs[1][3], fixed]
    out, reps = cg.coarse_grain_concurrent(meshes, [pos0] * 4, [w0] * 4, prm, max_concurrent=2,
                                           report=True)
    seq = [cg.coarse_grain(m, pos0, w0, p) for m, p in zip(meshes, prm)]
    for a, b in zip(out, seq):
        assert torch.equal(a, b)
    assert torch.equal(out[0], ref[0][0]) and torch.equal(out[1], ref[1][0])
    dep = [r["ms_locate"] + r["ms_deposit"] > 0 for r in reps]
    assert dep[2] and dep[3] and dep[0] != dep[1]                # only problems 0 and 1 share
    bad = pos0.clone()
    bad[0, 5] = 7.0
    with pytest.raises(cg.CGError) as e:
        cg.coarse_grain_concurrent([p[0] for p in probs[:4]], [bad] * 4, [w0] * 4,
                                   [p[3] for p in probs[:4]], max_concurrent=2)
    assert e.value.code == "CG_EDOMAIN" and "problem 0" in str(e.value)
    shifted.close()

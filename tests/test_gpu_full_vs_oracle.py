"""Full-size configurations in the launch configuration the benchmark times, every output
against the FP64 oracle: the 128^3 clustered step at all four bandwidths through the
concurrent entry (two problems at a time, FP32 inner solves with double-float
refinement), and all 64 batched snapshots x 5 fields in the autotuned batched schedule.
The oracle's multi-core build serves as the reference where it compiles (the CPU tests
hold it to the single-thread oracle: the same deposition bits, diffusion within 1e-12);
bars as everywhere: deposition bit-exact, mixed precision <= 1e-6 max-relative, mass to
1e-12."""
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


@pytest.fixture(scope="module")
def ref(orc):
    """(locate, deposit, diffuse) of the oracle: the multi-core build if it compiles."""
    from oracle import omp
    if omp.available():
        return (omp.locate_structured, lambda cell, w, n, vcu: omp.deposit(cell, w, n, vc_uniform=vcu),
                omp.diffuse_structured)
    return (orc.locate_structured, lambda cell, w, n, vcu: orc.deposit(cell, w, n, vc_uniform=vcu)[0],
            orc.diffuse_structured)


def maxrel(u, r):
    u, r = np.atleast_2d(u), np.atleast_2d(r)
    return max(np.max(np.abs(u[f] - r[f])) / max(np.max(np.abs(r[f])), 1e-300) for f in range(r.shape[0]))


def test_clustered_128_step_all_bandwidths_vs_oracle(cg, ref):
    import torch
    locate, deposit, diffuse = ref
    c = W.clustered_cube()
    cell, nout = locate(c.dims, c.origin, c.dx, c.pos)
    assert nout == 0
    eps0 = deposit(cell, c.w, c.ncells, (c.dx * c.dx) * c.dx)
    meshes = [cg.StructuredMesh(c.dims, c.origin, c.dx) for _ in range(4)]
    pos, w = torch.from_numpy(c.pos).cuda(), torch.from_numpy(c.w).cuda()
    bands = [k * c.dx for k in (1.0, 2.0, 4.0, 8.0)]
    prm = [cg.Params(bandwidth=b, nsteps=10, precision=cg.PREC_FP32_DF_REFINE) for b in bands]
    for m, q in zip(meshes, prm):   # the first call of each mesh tunes its sweep shape
        cg.coarse_grain(m, pos, w, q)
    streams = [torch.cuda.Stream() for _ in meshes]
    outs, reps = cg.coarse_grain_concurrent(meshes, [pos] * 4, [w] * 4, prm, streams=streams,
                                            max_concurrent=2, report=True)
    for b, o, r in zip(bands, outs, reps):
        want, _ = diffuse(eps0, c.dims, c.dx, b * b / 4, 10, tol=1e-14)
        assert maxrel(o.cpu().numpy(), want) <= MIXED_TOL, b
        assert abs(r["mass_out"][0] - r["mass_in"][0]) <= 1e-12 * r["mass_in"][0]
        assert r["final_rel_residual"] <= 1e-13
    for m in meshes:
        m.close()


def test_batched_64_snapshots_every_one_vs_oracle(cg, ref):
    import torch
    locate, deposit, diffuse = ref
    cases = W.batched_snapshots()
    meshes = [cg.StructuredMesh(c.dims, c.origin, c.dx) for c in cases]
    pos = [torch.from_numpy(c.pos).cuda() for c in cases]
    w = [torch.from_numpy(c.w).cuda() for c in cases]
    outs, rep = cg.coarse_grain_batched(meshes, pos, w, cg.Params(nsteps=10, precision=cg.PREC_FP32_DF_REFINE),
                                        bandwidths=[c.b for c in cases], report=True)
    assert rep["final_rel_residual"] <= 1e-13
    worst = 0.0
    for c, o in zip(cases, outs):
        cell, nout = locate(c.dims, c.origin, c.dx, c.pos)
        assert nout == 0
        eps0 = deposit(cell, c.w, c.ncells, (c.dx * c.dx) * c.dx)
        want, _ = diffuse(eps0, c.dims, c.dx, c.b * c.b / 4, 10, tol=1e-14)
        worst = max(worst, maxrel(o.cpu().numpy(), want))
    assert worst <= MIXED_TOL
    for m in meshes:
        m.close()

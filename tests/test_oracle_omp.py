"""The multi-core oracle (oracle/cg_oracle_omp.c) against the single-thread oracle:
locate and deposition bit for bit, diffusion within 1e-12 max-relative (only the order
of the conjugate-gradient dot products differs), and the same bits for any thread
count.  It serves the benchmark's multi-core CPU baseline and its error legs on
workloads too large for the single-thread oracle."""
import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def omp():
    from oracle import omp
    if not omp.available():
        pytest.skip("no OpenMP compiler here")
    return omp


def test_omp_locate_and_deposit_are_bit_identical(orc, omp):
    rng = np.random.default_rng(31)
    dims, origin, dx = (37, 21, 16), (0.5, -1.0, 0.0), 0.03125
    n = 200_000
    L = np.array(dims) * dx
    pos = np.array(origin)[:, None] + rng.random((3, n)) * L[:, None]
    pos[:, :50] = np.array(origin)[:, None] + np.floor(rng.random((3, 50)) * np.array(dims)[:, None]) * dx
    pos[:, 50] = (origin[0] + L[0], origin[1], origin[2] + L[2])     # upper walls clamp
    pos[:, 51] = (origin[0] - 1e-12, origin[1], origin[2])          # outside
    pos[:, 52] = (np.nan, 0.0, 0.0)
    c1, n1 = orc.locate_structured(dims, origin, dx, pos)
    c2, n2 = omp.locate_structured(dims, origin, dx, pos)
    assert n1 == n2 == 2 and np.array_equal(c1, c2)
    w = np.vstack([rng.random(n), rng.standard_normal(n) * 1e-3])
    ncells = int(np.prod(dims))
    for mode in (0, 1):
        e1, fb = orc.deposit(c1, w, ncells, vc_uniform=(dx * dx) * dx, mode=mode)
        for t in (1, 3, 8):
            omp.use_threads(t)
            e2 = omp.deposit(c1, w, ncells, vc_uniform=(dx * dx) * dx, mode=mode, fbits=fb)
            assert np.array_equal(e1.view(np.int64), e2.view(np.int64))


@pytest.mark.parametrize("scheme", [0, 1])
def test_omp_structured_diffusion_matches_the_oracle(orc, omp, scheme):
    rng = np.random.default_rng(32)
    dims, dx = (24, 17, 13), 1.0 / 24
    u0 = np.vstack([rng.random(int(np.prod(dims))), rng.standard_normal(int(np.prod(dims)))])
    T = (3 * dx) ** 2 / 4
    ref, it1 = orc.diffuse_structured(u0, dims, dx, T, 10, scheme=scheme, tol=1e-14)
    outs = []
    for t in (1, 4):
        omp.use_threads(t)
        got, it2 = omp.diffuse_structured(u0, dims, dx, T, 10, scheme=scheme, tol=1e-14)
        outs.append(got)
    assert np.array_equal(outs[0], outs[1])              # independent of the thread count
    for f in range(2):
        assert np.max(np.abs(outs[0][f] - ref[f])) <= 1e-12 * np.max(np.abs(ref[f]))


def test_omp_tet_diffusion_and_locate_match_the_oracle(orc, omp):
    xyz, tets = W.kuhn_tet_mesh(6, jitter=0.2, seed=7)
    vc, cent, rp, col, val = orc.tet_build(xyz, tets)
    rng = np.random.default_rng(33)
    u0 = rng.random(len(vc))
    ref, _ = orc.diffuse_csr(u0, vc, rp, col, val, 0.01, 10, tol=1e-14)
    omp.use_threads(4)
    got, _ = omp.diffuse_csr(u0, vc, rp, col, val, 0.01, 10, tol=1e-14)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    pos = rng.random((3, 5000))
    pos[:, :500] = xyz[rng.integers(0, len(xyz), 500)].T
    pos[:, 500:1000] = xyz[tets[rng.integers(0, len(tets), 500)][:, :3]].mean(axis=1).T
    pos[:, 1000] = (1.5, 0.5, 0.5)
    c1, n1 = orc.locate_tet(xyz, tets, pos)
    c2, n2 = omp.locate_tet_bucketed(xyz, tets, pos)
    assert n1 == n2 == 1 and np.array_equal(c1, c2)

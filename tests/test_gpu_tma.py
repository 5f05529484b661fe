"""The TMA-staged Chebyshev sweep (sweep_shape 400 + z planes per block): tile copies by
the Tensor Memory Accelerator into an mbarrier-synchronised ring of shared-memory
stages.  It computes the vectorised sweep's arithmetic term for term, so its results
must equal those of sweep_shape 100 + z bit for bit, on ragged meshes (partial 128-cell
tiles in x, partial row tiles in y, short z chunks, several fields) and in both
refinement modes that store the inner solve in FP32."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("dims", [(64, 16, 8), (132, 13, 7), (260, 9, 21), (4, 4, 3)])
@pytest.mark.parametrize("zlen", [1, 2, 4, 8])
@pytest.mark.parametrize("precision", [1, 3])
def test_tma_sweep_equals_vectorised_sweep(cg, dims, zlen, precision):
    import torch
    rng = np.random.default_rng(110)
    n = int(np.prod(dims))
    u0 = np.vstack([rng.random(n), rng.random(n) - 0.5])
    dx = 1.0 / max(dims)
    mesh = cg.StructuredMesh(dims, (0, 0, 0), dx)
    out = {}
    for shape in (100 + zlen, 400 + zlen):
        u = dev(u0)
        _, rep = cg.diffuse(mesh, u, cg.Params(bandwidth=3 * dx, nsteps=4, precision=precision,
                                               sweep_shape=shape), report=True)
        assert rep["sweep_shape_used"] == shape
        out[shape] = u
    assert torch.equal(out[100 + zlen], out[400 + zlen])


def test_tma_sweep_refusals(cg):
    u = dev(np.ones((1, 30 * 8 * 8)))
    for dims, prec, per in (((30, 8, 8), 3, None),      # nx % 4 != 0
                            ((32, 8, 8), 4, None),      # BF16 inner storage
                            ((32, 8, 8), 3, (True, False, False))):
        mesh = cg.StructuredMesh(dims, (0, 0, 0), 1 / 32, periodic=per or (False, False, False))
        with pytest.raises(cg.CGError) as e:
            cg.diffuse(mesh, dev(np.ones((1, mesh.ncells))), cg.Params(bandwidth=0.1, nsteps=2, precision=prec,
                                                                        sweep_shape=402))
        assert e.value.code == "CG_EINVAL"
    mesh = cg.StructuredMesh((32, 8, 8), (0, 0, 0), 1 / 32)
    for shape in (350, 500):
        with pytest.raises(cg.CGError):
            cg.diffuse(mesh, dev(np.ones((1, mesh.ncells))), cg.Params(bandwidth=0.1, nsteps=2, precision=3,
                                                                        sweep_shape=shape))
    del u

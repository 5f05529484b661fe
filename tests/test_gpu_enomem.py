"""Allocation failure (CG_ENOMEM) produced on the host by a workspace cap: a call whose
workspace would exceed the cap fails before allocating and before writing its output,
the library stays usable, and with the cap lifted the same call gives the same result as
on a fresh mesh.  No GPU memory is exhausted."""
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
    yield cg
    cg.set_workspace_limit(0)


@pytest.mark.parametrize("precision", [0, 3])
def test_workspace_cap_gives_enomem_and_leaves_the_output(cg, precision):
    import torch
    c = W.uniform_cube(n_side=48, n_particles=20_000)
    pos, w = torch.from_numpy(c.pos).cuda(), torch.from_numpy(c.w).cuda()
    mesh = cg.StructuredMesh(c.dims, c.origin, c.dx)
    held = cg.workspace_bytes()
    cg.set_workspace_limit(held + 64 * 1024)        # far below what the call needs
    out = torch.full((1, mesh.ncells), 7.5, dtype=torch.float64, device="cuda")
    p = cg.Params(bandwidth=c.b, nsteps=c.nsteps, precision=precision)
    with pytest.raises(cg.CGError) as e:
        cg.coarse_grain(mesh, pos, w, p, out=out)
    assert e.value.code == "CG_ENOMEM"
    assert "cg_set_workspace_limit" in str(e.value)
    assert bool((out == 7.5).all())
    assert cg.workspace_bytes() <= held + 64 * 1024
    # a cap the deposition fits under but the diffusion does not: CG_ENOMEM in the
    # second phase, after cells_out received the deposited field (include/cg.h)
    cg.set_workspace_limit(0)
    eps0 = cg.deposit(mesh, pos, w)
    cg.set_workspace_limit(cg.workspace_bytes() + 64 * 1024)
    with pytest.raises(cg.CGError) as e:
        cg.coarse_grain(mesh, pos, w, p, out=out)
    assert e.value.code == "CG_ENOMEM"
    assert torch.equal(out, eps0)
    cg.set_workspace_limit(0)
    got = cg.coarse_grain(mesh, pos, w, p)
    fresh = cg.StructuredMesh(c.dims, c.origin, c.dx)
    ref = cg.coarse_grain(fresh, pos, w, p)
    assert torch.equal(got, ref)
    mesh.close()
    fresh.close()
    assert cg.workspace_bytes() == held


def test_workspace_bytes_tracks_mesh_lifetimes(cg):
    import torch
    c = W.uniform_cube(n_side=32, n_particles=5_000)
    pos, w = torch.from_numpy(c.pos).cuda(), torch.from_numpy(c.w).cuda()
    before = cg.workspace_bytes()
    mesh = cg.StructuredMesh(c.dims, c.origin, c.dx)
    cg.coarse_grain(mesh, pos, w, cg.Params(bandwidth=c.b, nsteps=c.nsteps, precision=3))
    assert cg.workspace_bytes() > before
    mesh.close()
    assert cg.workspace_bytes() == before

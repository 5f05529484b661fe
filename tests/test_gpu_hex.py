"""GPU parity of stretched Cartesian meshes with a cell diffusion constant (stretched
meshes: Section 4.4; a local diffusion constant lowered to 0 to degenerate to PCM with
conservation kept: Section 5.2), against the FP64 oracle, through the C ABI.

Bars: operator, locate and deposition bit-exact; diffusion <= 1e-10 (FP64 PCG) and
<= 1e-6 (mixed) max-relative, explicit steps <= 1e-13; cells with D = 0 keep their
deposited values bit for bit; mass conserved to 1e-12.
"""
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


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


def maxrel(u, ref):
    u, ref = np.atleast_2d(u), np.atleast_2d(ref)
    return max(np.max(np.abs(u[f] - ref[f])) / np.max(np.abs(ref[f])) for f in range(ref.shape[0]))


def faces(n, ratio, length):
    w = ratio ** np.arange(n)
    f = np.concatenate([[0.0], np.cumsum(w)])
    return f * (length / f[-1])


@pytest.fixture(scope="module")
def case(cg):
    """23 x 14 x 9 cells, stretch ratios 1.04 / 0.97 / 1, D varying in [0.5, 1.5) with a
    frozen (D = 0) block."""
    xf, yf, zf = faces(23, 1.04, 1.0), faces(14, 0.97, 0.7), faces(9, 1.0, 0.4)
    nx, ny, nz = 23, 14, 9
    rng = np.random.default_rng(90)
    D = 0.5 + rng.random(nx * ny * nz)
    frozen = np.zeros((nz, ny, nx), bool)
    frozen[2:6, 4:9, 7:12] = True
    D[frozen.ravel()] = 0.0
    mesh = cg.HexMesh(xf, yf, zf, D)
    return xf, yf, zf, D, frozen.ravel(), mesh


def test_hex_operator_matches_oracle(cg, orc, case):
    xf, yf, zf, D, _, mesh = case
    vc, rp, col, val = orc.hex_build(xf, yf, zf, D)
    assert np.array_equal(bits(mesh.cell_volumes()), bits(vc))
    grp, gcol, gval = mesh.operator()
    n = len(vc)
    for k in range(0, n, 37):                       # rows compared entry by entry
        a = sorted(zip(col[rp[k]:rp[k + 1]], val[rp[k]:rp[k + 1]]))
        b = sorted(zip(gcol[grp[k]:grp[k + 1]], gval[grp[k]:grp[k + 1]]))
        assert [c for c, _ in a] == [c for c, _ in b]
        assert np.array_equal(bits([v for _, v in a]), bits([v for _, v in b]))


def test_hex_locate_and_deposit_bit_exact(cg, orc, case):
    xf, yf, zf, D, _, mesh = case
    rng = np.random.default_rng(91)
    pos = rng.random((3, 40_000)) * np.array([[1.0], [0.7], [0.4]])
    pos[0, :500] = xf[rng.integers(0, 24, 500)]      # on faces, both walls included
    pos[1, 500:1000] = yf[rng.integers(0, 15, 500)]
    pos[2, 1000:1500] = zf[rng.integers(0, 10, 500)]
    ref, nref = orc.locate_hex(xf, yf, zf, pos)
    got, nout = cg.locate(mesh, dev(pos))
    assert nout == nref == 0
    assert np.array_equal(got.cpu().numpy(), ref)
    bad = pos[:, :3].copy()
    bad[:, 0] = (1.0000001, 0.3, 0.2)
    bad[:, 1] = (0.5, np.nan, 0.2)
    ref2, nref2 = orc.locate_hex(xf, yf, zf, bad)
    got2, nout2 = cg.locate(mesh, dev(bad))
    assert nout2 == nref2 == 2 and np.array_equal(got2.cpu().numpy(), ref2)
    vc, *_ = orc.hex_build(xf, yf, zf, D)
    w = np.vstack([np.full(40_000, 1e-6), rng.standard_normal(40_000)])
    for mode in (0, 1):
        eps, _ = orc.deposit(ref, w, len(vc), vc=vc, mode=mode)
        d = cg.deposit(mesh, dev(pos), dev(w), cg.Params(deposit_mode=mode)).cpu().numpy()
        assert np.array_equal(bits(d), bits(eps))


@pytest.mark.parametrize("precision,bar,shape", [(0, 1e-10, 0), (1, 1e-6, 0), (3, 1e-6, 0), (1, 1e-6, 1)])
@pytest.mark.parametrize("scheme", [0, 1])
def test_hex_diffuse_parity_and_frozen_cells(cg, orc, case, precision, scheme, bar, shape):
    xf, yf, zf, D, frozen, mesh = case
    vc, rp, col, val = orc.hex_build(xf, yf, zf, D)
    rng = np.random.default_rng(92)
    n = len(vc)
    u0 = np.vstack([rng.random(n) * 3, rng.random(n) - 0.5])
    T = 0.004
    ref, _ = orc.diffuse_csr(u0, vc, rp, col, val, T, 10, scheme=scheme, tol=1e-15)
    u = dev(u0)
    _, rep = cg.diffuse(mesh, u, cg.Params(T=T, nsteps=10, scheme=scheme, precision=precision,
                                           sweep_shape=shape), report=True)
    got = u.cpu().numpy()
    assert maxrel(got, ref) <= bar
    assert np.array_equal(bits(got[:, frozen]), bits(u0[:, frozen]))     # D = 0: PCM kept
    mass0 = (vc * np.abs(u0)).sum(axis=1)
    assert np.all(np.abs(np.array(rep["mass_out"][:2]) - np.array(rep["mass_in"][:2])) <= 1e-12 * mass0)


def test_hex_explicit_parity(cg, orc, case):
    xf, yf, zf, D, frozen, mesh = case
    vc, rp, col, val = orc.hex_build(xf, yf, zf, D)
    rng = np.random.default_rng(93)
    u0 = rng.random(len(vc))
    rate = np.max(-val[col == np.repeat(np.arange(len(vc)), np.diff(rp))] / vc)
    T = 0.9 / rate * 15
    ref, _ = orc.diffuse_csr(u0, vc, rp, col, val, T, 15, scheme=2)
    u = dev(u0[None])
    cg.diffuse(mesh, u, cg.Params(T=T, nsteps=15, scheme=2))
    assert maxrel(u.cpu().numpy(), ref) <= 1e-13
    with pytest.raises(cg.CGError):
        cg.diffuse(mesh, dev(u0[None]), cg.Params(T=2.5 / rate * 15, nsteps=15, scheme=2))


def test_hex_rejects_bad_faces(cg):
    with pytest.raises(cg.CGError):
        cg.HexMesh([0.0, 0.5, 0.5, 1.0], [0.0, 1.0], [0.0, 1.0])          # not increasing
    with pytest.raises(cg.CGError):
        cg.HexMesh([0.0, 1.0], [0.0, 1.0], [0.0, 1.0], diffusivity=[-1.0])
    one = cg.HexMesh([0.0, 1.0], [0.0, 1.0], [0.0, 1.0])
    assert cg.load_library().cg_mesh_set_periodic(one.handle, 1, 0, 0) != 0


def test_uniform_hex_matches_structured(cg, orc):
    """Equal spacing and D = 1 everywhere: the stretched-mesh path and the uniform
    structured path solve the same system (one-cell axis included)."""
    dims = (17, 1, 12)
    dx = 0.05
    xf, yf, zf = (np.arange(d + 1) * dx for d in dims)
    rng = np.random.default_rng(94)
    u0 = rng.random((2, int(np.prod(dims))))
    T = (2 * dx) ** 2 / 4
    ref, _ = orc.diffuse_structured(u0, dims, dx, T, 8, tol=1e-15)
    for mesh in (cg.HexMesh(xf, yf, zf), cg.StructuredMesh(dims, (0, 0, 0), dx)):
        u = dev(u0)
        cg.diffuse(mesh, u, cg.Params(T=T, nsteps=8, precision=0))
        assert maxrel(u.cpu().numpy(), ref) <= 1e-10

"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each check uses a closed form, an
exact invariant, a library special case or a brute-force computation written a
different way.  A plausible slip in the oracle (a dropped neighbour, a wrong sign,
a wrong step size, a transposed index, a missing wall image) fails at least one.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.fft
import scipy.sparse
import scipy.sparse.linalg

import workloads as W


# ----------------------------------------------------------------------------- diffusion
def _dct_closed_form(u0, dims, dx, T, nsteps, scheme):
    """Exact discrete solution: the zero-flux 7-point Laplacian is diagonalised by
    the separable orthonormal DCT-II, eigenvalue -(4/dx^2) sin^2(pi j / (2N)) per axis."""
    nx, ny, nz = dims
    u = u0.reshape(nz, ny, nx)
    uh = scipy.fft.dctn(u, type=2, norm="ortho")
    lam = np.zeros((nz, ny, nx))
    for axis, n in zip((2, 1, 0), (nx, ny, nz)):
        j = np.arange(n)
        l1 = -(4.0 / dx ** 2) * np.sin(np.pi * j / (2.0 * n)) ** 2
        shape = [1, 1, 1]
        shape[axis] = n
        lam = lam + l1.reshape(shape)
    dt = T / nsteps
    if scheme == 0:
        g = 1.0 / (1.0 - dt * lam)
    elif scheme == 1:
        g = (1.0 + 0.5 * dt * lam) / (1.0 - 0.5 * dt * lam)
    else:
        g = 1.0 + dt * lam
    return scipy.fft.idctn(uh * g ** nsteps, type=2, norm="ortho").ravel()


@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("dims", [(13, 7, 5), (8, 8, 8), (1, 9, 6)])
def test_structured_diffusion_matches_dct_closed_form(orc, scheme, dims):
    rng = np.random.default_rng(11)
    dx = 0.37
    u0 = rng.random(np.prod(dims)) - 0.3
    # explicit Euler is only stable for dtau <= dx^2/6: choose T accordingly
    T = 0.9 * dx ** 2 if scheme == 2 else 2.3 * dx ** 2
    nsteps = 7
    got, _ = orc.diffuse_structured(u0, dims, dx, T, nsteps, scheme=scheme, tol=1e-15)
    ref = _dct_closed_form(u0, dims, dx, T, nsteps, scheme)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_point_source_variance_is_exactly_2T(orc, scheme, axis):
    """Eq. (solutionGi): the diffused point source has variance 2T per axis.  On the
    discrete grid this holds exactly: every step keeps the mass and the mean and adds
    2*dtau*mass to the second moment along each axis.  The 7-point operator is
    separable, so the marginal along the long axis obeys the 1-D law whatever the
    (short, walled) cross-section; the long axis keeps the wall leakage of the
    implicit schemes' exponential tails below 1e-20."""
    long_n = 121
    dims = [9, 7, 5]
    dims[axis] = long_n
    dx = 0.5
    u0 = np.zeros((dims[2], dims[1], dims[0]))
    src = [3, 2, 1]
    src[axis] = long_n // 2
    u0[src[2], src[1], src[0]] = 3.0
    T = (3 * dx) ** 2 / 4.0
    nsteps = 12 if scheme == 2 else 6
    u, _ = orc.diffuse_structured(u0.ravel(), tuple(dims), dx, T, nsteps, scheme=scheme, tol=1e-15)
    u = u.reshape(dims[2], dims[1], dims[0])
    x = (np.arange(long_n) - long_n // 2) * dx
    mass = u.sum()
    assert abs(mass - 3.0) <= 1e-13 * 3.0
    np_axis = 2 - axis
    marg = u.sum(axis=tuple(a for a in range(3) if a != np_axis))
    mean = (marg * x).sum() / mass
    var = (marg * x ** 2).sum() / mass
    assert abs(mean) <= 1e-12
    assert abs(var - 2.0 * T) <= 1e-11 * 2.0 * T


def test_conservation_nonnegativity_symmetry_linearity(orc):
    dims = (12, 12, 12)
    dx = 1.0 / 12
    n = 12 ** 3
    rng = np.random.default_rng(3)
    u0 = np.zeros(n)
    u0[rng.integers(0, n, 40)] += rng.random(40)
    T = (3 * dx) ** 2 / 4
    u, _ = orc.diffuse_structured(u0, dims, dx, T, 10)
    # Eq. (conserve): zero-flux walls keep sum V_c eps
    assert abs(u.sum() - u0.sum()) <= 1e-13 * u0.sum()
    # implicit Euler of an M-matrix keeps eps >= 0
    assert u.min() >= -1e-15 * u.max()
    # mirror symmetry of a centred source on an even grid
    v0 = np.zeros((12, 12, 12))
    v0[5:7, 5:7, 5:7] = 1.0
    v, _ = orc.diffuse_structured(v0.ravel(), dims, dx, T, 10)
    v = v.reshape(12, 12, 12)
    for ax in range(3):
        assert np.max(np.abs(v - np.flip(v, axis=ax))) <= 1e-14
    # per-component linearity (Section 3.2.1: each component is diffused alone)
    w0 = rng.random(n)
    both, _ = orc.diffuse_structured(np.stack([u0, w0, 2.5 * u0 - w0]), dims, dx, T, 10, tol=1e-15)
    assert np.max(np.abs(both[2] - (2.5 * both[0] - both[1]))) <= 1e-12 * np.max(np.abs(both[2]))


def test_equivalence_to_gaussian_kernel_with_images_converges_second_order(orc):
    """Section 3.2 / Section 4.1: the diffused PCM field of sources at cell centres
    approaches the image-summed Gaussian kernel of bandwidth b = sqrt(4T) at
    O(dx^2/b^2) + O(dtau/T).  Paper-shaped slab: 135 x 135 x 1 (d_p = 1), one cell
    layer of thickness d_p, b = 18; meshes of 15, 45 and 135 cells per side share
    the coarse cell centres; dtau is refined with dx^2."""
    L = 135.0
    b = 18.0
    T = b * b / 4.0
    rng = np.random.default_rng(5)
    coarse = rng.integers(0, 15, size=(20, 2))
    coarse[0] = (0, 0)        # corner source: needs the 2-D corner images
    coarse[1] = (7, 0)        # wall source
    src = np.zeros((20, 3))
    src[:, :2] = (coarse + 0.5) * 9.0
    src[:, 2] = 0.5
    wts = rng.random(20) + 0.5
    ev = np.zeros((15 * 15, 3))
    gx, gy = np.meshgrid((np.arange(15) + 0.5) * 9.0, (np.arange(15) + 0.5) * 9.0, indexing="xy")
    ev[:, 0] = gx.ravel()
    ev[:, 1] = gy.ravel()
    ev[:, 2] = 0.5
    exact = orc.kernel_sum(src, wts, ev, (L, L, 1.0), b, mmax=60)
    errs = []
    for r, nsteps in ((1, 4), (3, 36), (9, 324)):       # r fine cells per coarse cell
        N = 15 * r
        dx = L / N
        u0 = np.zeros(N * N)
        fine = coarse * r + r // 2                       # the coarse centre, on the fine grid
        np.add.at(u0, fine[:, 1] * N + fine[:, 0], wts / (dx * dx * 1.0))
        # the slab cells are dx x dx x 1 (dz != dx): diffuse with the generic CSR oracle
        u, _ = _diffuse_slab(orc, u0, N, dx, T, nsteps)
        u2 = u.reshape(N, N)[r // 2::r, r // 2::r].ravel()
        errs.append(np.max(np.abs(u2 - exact)) / np.max(exact))
    assert errs[2] < (9.0 / 9 / b) ** 2     # O((dx/b)^2) on the finest mesh
    order1 = math.log(errs[0] / errs[1]) / math.log(3)
    order2 = math.log(errs[1] / errs[2]) / math.log(3)
    assert 1.6 < order2 < 2.4, errs
    assert order1 > 1.3, errs


def _slab_csr(N, dx):
    """TPFA Laplacian of an N x N x 1 slab with cells dx x dx x 1: transmissibility of a
    face = area / distance = (dx * 1) / dx = 1 across x and y faces."""
    idx = np.arange(N * N).reshape(N, N)
    rows, cols = [], []
    for a, b_ in ((idx[:, :-1], idx[:, 1:]), (idx[:-1, :], idx[1:, :])):
        rows += [a.ravel(), b_.ravel()]
        cols += [b_.ravel(), a.ravel()]
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    off = scipy.sparse.csr_matrix((np.ones(len(r)), (r, c)), shape=(N * N, N * N))
    Lm = off - scipy.sparse.diags(np.asarray(off.sum(axis=1)).ravel())
    Lm = Lm.tocsr()
    Lm.sort_indices()
    return Lm


def _diffuse_slab(orc, u0, N, dx, T, nsteps):
    Lm = _slab_csr(N, dx)
    vc = np.full(N * N, dx * dx * 1.0)
    return orc.diffuse_csr(u0, vc, Lm.indptr.astype(np.int64), Lm.indices.astype(np.int32), Lm.data,
                           T, nsteps, tol=1e-14)


def test_structured_and_csr_oracles_agree_on_a_hex_grid(orc):
    """The uniform 7-point operator is the two-point-flux FV operator with T_f = dx
    (face dx^2 over distance dx) and V_c = dx^3; the two oracle paths must agree."""
    n = 7
    dx = 0.2
    dims = (n, n, n)
    idx = np.arange(n ** 3).reshape(n, n, n)
    rows, cols = [], []
    for a, b_ in ((idx[:, :, :-1], idx[:, :, 1:]), (idx[:, :-1, :], idx[:, 1:, :]),
                  (idx[:-1, :, :], idx[1:, :, :])):
        rows += [a.ravel(), b_.ravel()]
        cols += [b_.ravel(), a.ravel()]
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    off = scipy.sparse.csr_matrix((np.full(len(r), dx), (r, c)), shape=(n ** 3, n ** 3))
    Lm = (off - scipy.sparse.diags(np.asarray(off.sum(axis=1)).ravel())).tocsr()
    Lm.sort_indices()
    rng = np.random.default_rng(2)
    u0 = rng.random(n ** 3)
    T = 0.05
    for scheme in (0, 1, 2):
        Ts = T if scheme != 2 else 0.002
        a, _ = orc.diffuse_structured(u0, dims, dx, Ts, 5, scheme=scheme, tol=1e-15)
        b2, _ = orc.diffuse_csr(u0, np.full(n ** 3, dx ** 3), Lm.indptr.astype(np.int64),
                                Lm.indices.astype(np.int32), Lm.data, Ts, 5, scheme=scheme,
                                tol=1e-15)
        assert np.max(np.abs(a - b2)) <= 1e-12 * np.max(np.abs(a))


# ----------------------------------------------------------------------------- locate / deposit
def test_locate_structured_edge_cases(orc):
    dims = (4, 3, 2)
    dx = 0.25
    origin = (-0.5, 0.0, 1.0)
    pts = np.array([
        [-0.5, 0.0, 1.0],            # lower corner -> cell 0
        [0.5, 0.75, 1.5],            # upper corner (on the walls) clamps into the last cell
        [-0.25, 0.25, 1.25],         # exactly on interior faces -> the upper cell
        [-0.5 - 1e-12, 0.1, 1.1],    # just outside
        [0.5 + 1e-12, 0.1, 1.1],     # just outside
        [np.nan, 0.1, 1.1],          # NaN is out of domain
        [0.1, 0.2, 1.4],
    ]).T
    cell, nout = orc.locate_structured(dims, origin, dx, pts)
    assert nout == 3
    assert list(cell) == [0, 23, (1 * 3 + 1) * 4 + 1, -1, -1, -1, (1 * 3 + 0) * 4 + 2]


def test_locate_structured_matches_exact_rational_floor(orc):
    """With dx a power of two every step of the cell computation is exact, so the
    oracle must match the exact floor((x - x0)/dx) computed in rationals."""
    rng = np.random.default_rng(4)
    dims = (32, 16, 8)
    dx = 1.0 / 32
    pos = rng.random((3, 3000)) * np.array([1.0, 0.5, 0.25])[:, None]
    pos[:, :50] = np.round(pos[:, :50] * 32) / 32          # points on faces
    cell, nout = orc.locate_structured(dims, (0, 0, 0), dx, pos)
    assert nout == 0
    for i in range(pos.shape[1]):
        ijk = []
        for a in range(3):
            k = math.floor(Fraction(pos[a, i]) / Fraction(dx))
            ijk.append(min(k, dims[a] - 1))
        assert cell[i] == (ijk[2] * dims[1] + ijk[1]) * dims[0] + ijk[0]


def test_deposit_mode0_matches_python_sequential_sum(orc):
    rng = np.random.default_rng(7)
    n, ncells = 500, 27
    cell = rng.integers(-1, ncells, n).astype(np.int32)
    w = rng.standard_normal((2, n)) * 10.0 ** rng.integers(-3, 3, (2, n))
    vc = rng.random(ncells) + 0.1
    got, _ = orc.deposit(cell, w, ncells, vc=vc, mode=0)
    for f in range(2):
        s = [0.0] * ncells
        for i in range(n):              # plain Python floats: IEEE doubles, in order
            if cell[i] >= 0:
                s[cell[i]] = s[cell[i]] + float(w[f, i])
        ref = np.array([s[k] / vc[k] for k in range(ncells)])
        assert np.array_equal(got[f].view(np.int64), ref.view(np.int64))


def test_deposit_mode1_is_exact_fixed_point(orc):
    rng = np.random.default_rng(8)
    n, ncells = 700, 13
    cell = rng.integers(0, ncells, n).astype(np.int32)
    w = rng.standard_normal((3, n)) * np.array([1e-7, 1.0, 3e5])[:, None]
    vcu = 0.125
    got, fbits = orc.deposit(cell, w, ncells, vc_uniform=vcu, mode=1)
    for f in range(3):
        F = fbits[f]
        m = Fraction(float(np.max(np.abs(w[f]))))
        # n * max|w| * 2^F < 2^61 and F is within 2 of the largest such exponent
        assert n * m * Fraction(2) ** F < 2 ** 61
        assert n * m * Fraction(2) ** (F + 2) >= 2 ** 61
        acc = [0] * ncells
        for i in range(n):
            acc[cell[i]] += round(float(w[f, i]) * 2.0 ** F)   # Python round: half to even
        ref = np.array([(float(a) * 2.0 ** (-F)) / vcu for a in acc])
        assert np.array_equal(got[f].view(np.int64), ref.view(np.int64))
        # conservation is exact in the integer domain
        assert sum(acc) == sum(round(float(x) * 2.0 ** F) for x in w[f])


def test_fixed_point_bits_limits(orc):
    assert orc.fixed_point_bits(0, 1.0) == 0
    assert orc.fixed_point_bits(10, 0.0) == 0
    assert orc.fixed_point_bits(1, 5e-324) == 1000
    for n, m in ((1, 1e308), (3, 7.0), (2_000_000, 3.35e-8), (5, 1e-300)):
        F = orc.fixed_point_bits(n, m)
        assert n * Fraction(m) * Fraction(2) ** F < 2 ** 61
        if -1000 < F < 1000:               # not clamped: within 2 of the largest exponent
            assert 2 ** 61 <= n * Fraction(m) * Fraction(2) ** (F + 2)
        else:
            assert F == 1000 and m == 1e-300


def test_deposit_conservation_cfg_small(orc):
    c = W.uniform_cube()
    cell, nout = orc.locate_structured(c.dims, c.origin, c.dx, c.pos)
    eps, _ = orc.deposit(cell, c.w, c.ncells, vc_uniform=(c.dx * c.dx) * c.dx)
    assert nout == 0
    assert abs(eps.sum() * c.dx ** 3 - c.w.sum()) <= 1e-12 * c.w.sum()


def test_paper_slab_smoothing_caps_pcm_extremes(orc):
    """Section 4.4: on a mesh finer than the particles (dx = d_p/2) PCM gives cells with
    eps far above 1; the diffused field (b = 6 d_p) stays smooth and below the PCM
    maximum, and on meshes dx = 1 and 0.5 the fields agree (mesh convergence)."""
    rng = np.random.default_rng(0)
    L = 135.0
    pos = np.zeros((3, 1000))
    pos[:2] = 30.0 + 75.0 * rng.random((2, 1000))
    pos[2] = 0.5
    vp = math.pi / 6.0
    fields = {}
    for N in (135, 270):
        dx = L / N
        cell, nout = orc.locate_structured((N, N, 1), (0, 0, 0), dx, np.vstack([pos[:2], pos[2:] * 0 + 0.5 * dx]))
        assert nout == 0
        u0, _ = orc.deposit(cell, np.full((1, 1000), vp), N * N, vc_uniform=dx * dx * dx)
        # thickness of the layer is dx here: keep the slab a single layer of cells
        u, _ = orc.diffuse_structured(u0, (N, N, 1), dx, 9.0, 3)
        fields[N] = (u0[0].reshape(N, N), u.reshape(N, N))
    pcm_max = fields[270][0].max()
    assert pcm_max > 1.0
    assert fields[270][1].max() < 0.5 * pcm_max
    # one cell layer: compare areal densities eps * thickness on the common 135 grid
    fine = fields[270][1].reshape(135, 2, 135, 2).mean(axis=(1, 3)) * 0.5
    c135 = fields[135][1] * 1.0
    assert np.max(np.abs(fine - c135)) <= 0.1 * np.max(c135)


# ----------------------------------------------------------------------------- tetrahedra
def _heron_face(a, b, c):
    la, lb, lc = np.linalg.norm(b - c), np.linalg.norm(a - c), np.linalg.norm(a - b)
    s = 0.5 * (la + lb + lc)
    return math.sqrt(max(s * (s - la) * (s - lb) * (s - lc), 0.0))


def test_tet_mesh_geometry_and_operator(orc):
    xyz, tets = W.kuhn_tet_mesh(5, jitter=0.2, seed=1)
    vc, cent, rowptr, col, val = orc.tet_build(xyz, tets)
    nt = tets.shape[0]
    assert abs(vc.sum() - 1.0) <= 1e-13                      # tets tile the unit cube
    A = scipy.sparse.csr_matrix((val, col, rowptr), shape=(nt, nt))
    assert abs(A - A.T).max() == 0.0                          # symmetric by construction
    assert np.max(np.abs(A @ np.ones(nt))) <= 1e-13 * np.max(np.abs(val))   # L 1 = 0
    off = A - scipy.sparse.diags(A.diagonal())
    assert off.data.min() > 0.0                               # every T_f > 0 (M-matrix)
    # interior tets have 4 face neighbours, all have at least 1
    deg = np.diff(rowptr) - 1
    assert deg.max() == 4 and deg.min() >= 1
    # independent geometry for a few faces: area by Heron, normal by SVD of the plane
    rng = np.random.default_rng(0)
    for k in rng.integers(0, nt, 25):
        for e in range(rowptr[k], rowptr[k + 1]):
            l = col[e]
            if l == k:
                continue
            shared = sorted(set(tets[k]) & set(tets[l]))
            assert len(shared) == 3
            p = xyz[shared]
            area = _heron_face(*p)
            centred = p - p.mean(axis=0)
            nrm = np.linalg.svd(centred)[2][-1]
            d = cent[l] - cent[k]
            T = area / abs(np.dot(nrm, d))
            assert abs(A[k, l] - T) <= 1e-11 * T
    # undeformed Kuhn tets: each is one sixth of its hex
    xyz0, tets0 = W.kuhn_tet_mesh(3, jitter=0.0)
    vc0, *_ = orc.tet_build(xyz0, tets0)
    assert np.max(np.abs(vc0 - (1.0 / 27) / 6)) <= 1e-16


def test_tet_diffusion_matches_sparse_direct_solve(orc):
    xyz, tets = W.kuhn_tet_mesh(4, jitter=0.2, seed=2)
    vc, cent, rowptr, col, val = orc.tet_build(xyz, tets)
    nt = len(vc)
    Lm = scipy.sparse.csr_matrix((val, col, rowptr), shape=(nt, nt))
    rng = np.random.default_rng(1)
    u0 = rng.random(nt)
    T, nsteps = 0.004, 4
    dt = T / nsteps
    for scheme in (0, 1):
        got, _ = orc.diffuse_csr(u0, vc, rowptr, col, val, T, nsteps, scheme=scheme, tol=1e-15)
        M = scipy.sparse.diags(vc)
        th = 1.0 if scheme == 0 else 0.5
        A = (M - th * dt * Lm).tocsc()
        u = u0.copy()
        for _ in range(nsteps):
            rhs = vc * u + ((1 - th) * dt * (Lm @ u) if scheme == 1 else 0.0)
            u = scipy.sparse.linalg.spsolve(A, rhs)
        assert np.max(np.abs(got - u)) <= 1e-12 * np.max(np.abs(u))
        assert abs((vc * got).sum() - (vc * u0).sum()) <= 1e-13 * (vc * u0).sum()


def test_tet_locate_matches_independent_barycentric(orc):
    xyz, tets = W.kuhn_tet_mesh(4, jitter=0.2, seed=3)
    rng = np.random.default_rng(9)
    pos = rng.random((3, 300))
    cell, nout = orc.locate_tet(xyz, tets, pos)
    assert nout == 0
    for i in range(pos.shape[1]):
        # barycentric coordinates by a linear solve (not by orientation determinants)
        best, bestm = -1, -np.inf
        for t in range(tets.shape[0]):
            v = xyz[tets[t]]
            Mt = np.vstack([(v[1:] - v[0]).T])
            lam = np.linalg.solve(Mt, pos[:, i] - v[0])
            m = min(1.0 - lam.sum(), lam.min())
            if m > bestm:
                best, bestm = t, m
        if bestm > 1e-9:                      # unambiguous interior point
            assert cell[i] == best
    # outside the cube: out of domain
    _, nout = orc.locate_tet(xyz, tets, np.array([[1.5], [0.5], [0.5]]))
    assert nout == 1


def _bary_solve(xyz, tet, x):
    """Barycentric coordinates of x in a tet by a linear solve of the edge system (an
    independent route: no orientation determinants).  Returns the 4 coordinates."""
    v = xyz[np.asarray(tet)]
    lam = np.linalg.solve((v[1:] - v[0]).T, np.asarray(x, dtype=np.float64) - v[0])
    return np.concatenate([[1.0 - lam.sum()], lam])


def test_tet_locate_fallback_takes_a_point_just_outside_a_lone_tet():
    """The fallback branch: a point inside a tet's bounding box but 5e-11 outside one of
    its faces qualifies for no tet, so the rule takes the tet with the largest minimum
    coordinate when that minimum is >= -1e-10; 2e-10 outside it is out of domain."""
    import oracle as orc
    xyz = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    # the face x + y + z = 1 (opposite vertex 0): lambda_0 = 1 - x - y - z
    pts = np.array([[0.25, 0.25, 0.5 + 5e-11], [0.25, 0.25, 0.5 - 5e-11],
                    [0.25, 0.25, 0.5 + 2e-10], [0.5, 0.5, 0.5]]).T
    cell, nout = orc.locate_tet(xyz, tets, pts)
    assert list(cell) == [0, 0, -1, -1] and nout == 2
    for i in (0, 2):                                   # both are outside the tet
        assert _bary_solve(xyz, tets[0], pts[:, i]).min() < 0.0


def test_tet_locate_fallback_takes_the_largest_minimum_not_the_lowest_index():
    """Two disjoint tets whose boxes both hold the point, which lies outside both, each
    by less than 1e-10: the rule picks the tet whose minimum coordinate is larger
    (closer to containing it), whichever index it has; between identical minima (a tet
    listed twice) the lower index."""
    import oracle as orc
    base = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    # tet A: the unit corner tet, face x + y + z = 1; tet B: A mirrored through the
    # plane x + y + z = 1 + g, so B's matching face is x + y + z = 1 + 2g
    g = 4e-11

    def mirror(p):
        return p + (2.0 * (1.0 + g) - 2.0 * p.sum()) / 3.0 * np.ones(3)
    xyz = np.vstack([base, np.array([mirror(p) for p in base])])
    A, B = [0, 1, 2, 3], [4, 5, 6, 7]
    # 1e-11 beyond A's face, about 7e-11 short of B's
    x = np.array([0.3, 0.3, 0.4 + 1e-11])
    la, lb = _bary_solve(xyz, A, x).min(), _bary_solve(xyz, B, x).min()
    assert -1e-10 < lb < la < 0.0
    for order, want in (([A, B], 0), ([B, A], 1)):
        cell, nout = orc.locate_tet(xyz, np.array(order, dtype=np.int32), x[:, None])
        assert nout == 0 and cell[0] == want
    for order, want in (([A, A, B], 0), ([B, A, A], 1), ([B, B], 0)):
        cell, nout = orc.locate_tet(xyz, np.array(order, dtype=np.int32), x[:, None])
        assert nout == 0 and cell[0] == want


def test_tet_locate_takes_the_lowest_index_of_overlapping_tets():
    """The first branch: among tets that contain the point, the lowest index."""
    import oracle as orc
    xyz = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0],
                    [2.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, 2.0]])
    small, big = [0, 1, 2, 3], [0, 4, 5, 6]
    x = np.array([[0.2], [0.2], [0.2]])
    for order, want in (([small, big], 0), ([big, small], 0), ([small, small, big], 0)):
        cell, nout = orc.locate_tet(xyz, np.array(order, dtype=np.int32), x)
        assert nout == 0 and cell[0] == want
    y = np.array([[0.2], [0.2], [1.2]])              # only in the big tet
    cell, _ = orc.locate_tet(xyz, np.array([small, big], dtype=np.int32), y)
    assert cell[0] == 1
    # exactly on the small tet's face x + y + z = 1 (dyadic coordinates: every
    # determinant is exact, the minimum coordinate is exactly 0) and 1e-13 inside it:
    # the small tet qualifies and wins over the big tet, which holds the point deeply
    for z in (0.5, 0.5 - 1e-13):
        p = np.array([[0.25], [0.25], [z]])
        assert 0.0 <= _bary_solve(xyz, small, p[:, 0]).min() < 1e-12
        cell, _ = orc.locate_tet(xyz, np.array([small, big], dtype=np.int32), p)
        assert cell[0] == 0


def test_tet_locate_on_shared_faces_edges_and_vertices():
    """Points placed on shared faces, edges and vertices of a jittered Kuhn mesh, where
    the first branch or the fallback decides on rounding: the tet returned holds the
    point to within 1e-9 (linear-solve barycentrics), no lower-index tet holds it by
    more than 1e-9, and points 1e-6 outside the cube are out of domain."""
    import oracle as orc
    xyz, tets = W.kuhn_tet_mesh(3, jitter=0.2, seed=5)
    rng = np.random.default_rng(17)
    pts = []
    nt = tets.shape[0]
    for t in rng.choice(nt, 40, replace=False):
        v = xyz[tets[t]]
        pts.append(v[rng.integers(4)])                             # a vertex
        a, b = rng.choice(4, 2, replace=False)
        s = rng.random()
        pts.append(v[a] + s * (v[b] - v[a]))                       # on an edge
        f = rng.choice(4, 3, replace=False)
        l = rng.dirichlet(np.ones(3))
        pts.append(l[0] * v[f[0]] + l[1] * v[f[1]] + l[2] * v[f[2]])  # on a face
    pts = np.array(pts).T
    inside = np.all((pts >= 0.0) & (pts <= 1.0), axis=0)
    pts = pts[:, inside]
    cell, nout = orc.locate_tet(xyz, tets, pts)
    assert nout == 0
    for i in range(pts.shape[1]):
        x = pts[:, i]
        got = cell[i]
        assert _bary_solve(xyz, tets[got], x).min() >= -1e-9
        for t in range(got):
            assert _bary_solve(xyz, tets[t], x).min() <= 1e-9
    out = np.array([[-1e-6, 0.5, 0.5], [0.5, 1.0 + 1e-6, 0.5], [0.3, 0.3, 1.0 + 1e-6]]).T
    cell, nout = orc.locate_tet(xyz, tets, out)
    assert nout == 3 and list(cell) == [-1, -1, -1]


@pytest.mark.parametrize("nb", [1, 2, 3, 7])
def test_bucketed_tet_locate_equals_the_brute_force(orc, nb):
    """locate_tet_bucketed searches only the point's bucket; its results equal the brute
    force over all tets bit for bit, for any bucket count, on points at vertices, on
    faces and edges, just off faces, outside the mesh and not finite."""
    xyz, tets = W.kuhn_tet_mesh(5, jitter=0.2, seed=6)
    rng = np.random.default_rng(19)
    n = 6000
    pos = rng.random((3, n))
    k = 1000
    pos[:, :k] = xyz[rng.integers(0, len(xyz), k)].T
    t = tets[rng.integers(0, len(tets), k)]
    pos[:, k:2 * k] = xyz[t[:, :3]].mean(axis=1).T
    pos[:, 2 * k:3 * k] = (0.5 * (xyz[t[:, 0]] + xyz[t[:, 3]])).T
    pos[:, 3 * k:4 * k] = xyz[t[:, :3]].mean(axis=1).T + rng.standard_normal((3, k)) * 1e-12
    pos[:, 4 * k] = (1.2, 0.5, 0.5)
    pos[:, 4 * k + 1] = (0.5, np.nan, 0.5)
    pos[:, 4 * k + 2] = (-np.inf, 0.5, 0.5)
    pos[:, 4 * k + 3] = (0.5, 0.5, 1.0 + 1e-15)
    ref, nref = orc.locate_tet(xyz, tets, pos)
    got, nout = orc.locate_tet_bucketed(xyz, tets, pos, nb=nb)
    assert nout == nref and nref >= 3
    assert np.array_equal(got, ref)


def test_image_kernel_is_normalised_over_the_box(orc):
    """Eq. (normal) with Eq. (hi-bound): the image-summed kernel of a particle near a
    corner integrates to its volume over the box (midpoint quadrature, 60^3 points)."""
    L = (1.0, 0.8, 0.6)
    b = 0.15
    n = 60
    pts = []
    for a in range(3):
        pts.append((np.arange(n) + 0.5) * L[a] / n)
    X, Y, Z = np.meshgrid(*pts, indexing="ij")
    ev = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    src = np.array([[0.03, 0.75, 0.31]])
    vals = orc.kernel_sum(src, np.array([2.0]), ev, L, b, mmax=2)
    integral = vals.sum() * (L[0] * L[1] * L[2]) / n ** 3
    assert abs(integral - 2.0) <= 1e-6


def test_golden_close_packed_layer_solid_fraction(orc):
    """The paper's 0.606 (Section 4.3, tests/golden/close_packed_layer.json): a triangular
    close-packed layer of spheres (diameter d, spacing d, one diameter thick) deposited by
    the particle centroid method onto cells of side d carries a mean solid fraction over the
    layer equal to pi/(3 sqrt 3) = 0.6046 -- a check of V_p, V_c and the per-cell division.
    Single cells see 1 or 2 centroids (0.52 or 1.05: PCM exceeds the packing limit, as the
    paper remarks); the smoothed field keeps the layer's mean."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "close_packed_layer.json")) as f:
        gold = json.load(f)
    d = 1.0 / 64
    cols, rows = 64, 74
    i, j = np.meshgrid(np.arange(cols), np.arange(rows))
    pos = np.vstack([(i * d + 0.25 * d + (j % 2) * 0.5 * d).ravel(),
                     ((j + 0.5) * np.sqrt(3) / 2 * d).ravel(),
                     np.full(cols * rows, d / 2)])
    vp = np.pi * d ** 3 / 6
    w = np.full((1, cols * rows), vp)
    dims = (64, 65, 1)
    cell, nout = orc.locate_structured(dims, (0, 0, 0), d, pos)
    assert nout == 0
    eps, _ = orc.deposit(cell, w, int(np.prod(dims)), vc_uniform=d * d * d)
    layer_volume = (cols * d) * (rows * np.sqrt(3) / 2 * d) * d
    mean = eps.sum() * d ** 3 / layer_volume
    assert abs(mean - np.pi / (3 * np.sqrt(3))) <= 1e-12
    assert abs(mean - gold["value"]) <= gold["tolerance_abs"]
    assert eps.max() > gold["value"]                     # PCM overshoots the packing limit
    u, _ = orc.diffuse_structured(eps, dims, d, (3 * d) ** 2 / 4, 10)
    assert abs(u.sum() * d ** 3 / layer_volume - mean) <= 1e-12
    inner = u.reshape(65, 64)[10:54, 10:54]
    assert abs(inner.mean() - mean) <= 2e-3


def _closed_form_mixed(u0, dims, c, nsteps, periodic, scheme=0):
    """The exact discrete solution with per-axis eigenbases: the DFT on a periodic axis
    (eigenvalues -4 sin^2(pi j / n)), the orthonormal DCT-II on a zero-flux axis
    (-4 sin^2(pi j / (2 n)))."""
    import scipy.fft as sf
    nx, ny, nz = dims
    a = np.asarray(u0, dtype=np.float64).reshape(nz, ny, nx).astype(complex)
    lam = np.zeros((nz, ny, nx))
    for ax, (n, per) in enumerate(zip((nz, ny, nx), (periodic[2], periodic[1], periodic[0]))):
        j = np.arange(n)
        lj = -4.0 * np.sin(np.pi * j / n) ** 2 if per else -4.0 * np.sin(np.pi * j / (2 * n)) ** 2
        shape = [1, 1, 1]
        shape[ax] = n
        lam = lam + lj.reshape(shape)
        a = np.fft.fft(a, axis=ax) if per else sf.dct(a.real, type=2, norm="ortho", axis=ax) + 1j * sf.dct(a.imag, type=2, norm="ortho", axis=ax)
    g = {0: 1.0 / (1.0 - c * lam), 1: (1.0 + 0.5 * c * lam) / (1.0 - 0.5 * c * lam),
         2: 1.0 + c * lam}[scheme]
    a = a * g ** nsteps
    for ax, (n, per) in reversed(list(enumerate(zip((nz, ny, nx), (periodic[2], periodic[1], periodic[0]))))):
        a = np.fft.ifft(a, axis=ax) if per else sf.idct(a.real, type=2, norm="ortho", axis=ax) + 1j * sf.idct(a.imag, type=2, norm="ortho", axis=ax)
    return a.real.ravel()


@pytest.mark.parametrize("periodic", [(True, True, True), (True, False, False), (False, True, True)])
@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_periodic_diffusion_matches_closed_form(orc, periodic, scheme):
    """Periodic axes (Section 3.1): the oracle against the exact DFT/DCT solution."""
    dims = (9, 6, 5)
    rng = np.random.default_rng(60)
    u0 = rng.random(int(np.prod(dims)))
    dx = 0.1
    c = 0.15 if scheme == 2 else 0.8
    T = c * dx * dx * 7
    got, _ = orc.diffuse_structured(u0, dims, dx, T, 7, scheme=scheme, tol=1e-15, periodic=periodic)
    ref = _closed_form_mixed(u0, dims, c, 7, periodic, scheme)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert abs(got.sum() - u0.sum()) <= 1e-12 * u0.sum()


def test_periodic_shift_invariance(orc):
    """On an all-periodic mesh the smoothing commutes with a cyclic shift of the cells."""
    dims = (8, 7, 6)
    rng = np.random.default_rng(61)
    u0 = rng.random(dims[::-1])
    shifted = np.roll(u0, (2, -3, 5), axis=(0, 1, 2))
    a, _ = orc.diffuse_structured(u0.ravel(), dims, 0.1, 0.02, 5, tol=1e-15, periodic=(True,) * 3)
    b, _ = orc.diffuse_structured(shifted.ravel(), dims, 0.1, 0.02, 5, tol=1e-15, periodic=(True,) * 3)
    assert np.max(np.abs(np.roll(a.reshape(dims[::-1]), (2, -3, 5), axis=(0, 1, 2)) - b.reshape(dims[::-1]))) <= 1e-13


def test_solid_velocity_of_uniform_motion(orc):
    """Every particle moving with the same velocity U0: the diffused momentum is U0 times
    the diffused solid fraction (linearity), so the solid velocity is U0 in every cell
    with solid, and 0 where there is none."""
    c = W.uniform_cube(n_side=16, n_particles=2000, seed=62)
    U0 = np.array([0.3, -1.25, 2.0])
    w = np.vstack([c.w[0], np.outer(U0, c.w[0])])
    cell, _ = orc.locate_structured(c.dims, c.origin, c.dx, c.pos)
    eps, _ = orc.deposit(cell, w, c.ncells, vc_uniform=c.dx ** 3)
    u, _ = orc.diffuse_structured(eps, c.dims, c.dx, (2 * c.dx) ** 2 / 4, 10, tol=1e-15)
    us = orc.solid_velocity(u[0], u[1:], eps_min=1e-12 * u[0].max())
    inside = u[0] > 1e-12 * u[0].max()
    assert inside.any()
    assert np.max(np.abs(us[:, inside] - U0[:, None])) <= 1e-12 * np.abs(U0).max()
    assert np.all(us[:, ~inside] == 0.0)
    raw = orc.solid_velocity(eps[0], eps[1:], 0.0)      # before smoothing: per particle cell
    occ = eps[0] > 0
    assert np.max(np.abs(raw[:, occ] - U0[:, None])) <= 1e-14 * np.abs(U0).max()


def _stretched_faces(n, ratio, length=1.0):
    w = ratio ** np.arange(n)
    f = np.concatenate([[0.0], np.cumsum(w)])
    return f * (length / f[-1])


def test_hex_operator_uniform_equals_structured(orc):
    """A stretched mesh with equal spacing and D = 1 is the uniform mesh: the CSR oracle
    on it reproduces the structured oracle (both implicit schemes and explicit)."""
    dims = (7, 5, 4)
    dx = 0.125
    xf, yf, zf = (np.arange(n + 1) * dx for n in dims)
    vc, rp, col, val = orc.hex_build(xf, yf, zf)
    assert np.allclose(vc, dx ** 3, rtol=0, atol=1e-18)
    rng = np.random.default_rng(80)
    u0 = rng.random(int(np.prod(dims)))
    for scheme, T in ((0, 0.01), (1, 0.01), (2, 0.1 * dx * dx * 6)):
        a, _ = orc.diffuse_structured(u0, dims, dx, T, 6, scheme=scheme, tol=1e-15)
        b, _ = orc.diffuse_csr(u0, vc, rp, col, val, T, 6, scheme=scheme, tol=1e-15)
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


def test_hex_operator_varying_diffusivity(orc):
    """Stretched spacing (ratio 1.04, as the paper's stretched mesh) and a region with
    D = 0: the operator is symmetric with L 1 = 0 and total volume equal to the box; the
    D = 0 cells keep their deposited values exactly (PCM there), and mass is conserved."""
    xf, yf, zf = _stretched_faces(20, 1.04), _stretched_faces(12, 1 / 1.04, 0.6), _stretched_faces(6, 1.0, 0.3)
    nx, ny, nz = 20, 12, 6
    D = np.ones(nx * ny * nz)
    frozen = np.zeros((nz, ny, nx), bool)
    frozen[:, 3:7, 5:11] = True
    D[frozen.ravel()] = 0.0
    D[~frozen.ravel()] = 0.5 + np.random.default_rng(81).random((~frozen).sum())
    vc, rp, col, val = orc.hex_build(xf, yf, zf, D)
    assert abs(vc.sum() - 1.0 * 0.6 * 0.3) <= 1e-14
    n = nx * ny * nz
    A = scipy.sparse.csr_matrix((val, col, rp), shape=(n, n))
    assert abs(A - A.T).max() <= 1e-15 * abs(A).max()
    assert np.max(np.abs(A @ np.ones(n))) <= 1e-12 * abs(A).max()
    u0 = np.random.default_rng(82).random(n)
    u, _ = orc.diffuse_csr(u0, vc, rp, col, val, 0.002, 10, tol=1e-15)
    assert np.array_equal(u[frozen.ravel()], u0[frozen.ravel()])
    assert abs((vc * u).sum() - (vc * u0).sum()) <= 1e-13 * (vc * u0).sum()
    assert u.min() >= 0.0


def test_locate_hex_against_searchsorted(orc):
    xf, yf, zf = _stretched_faces(17, 1.05), _stretched_faces(9, 0.97), _stretched_faces(5, 1.0)
    rng = np.random.default_rng(83)
    pos = rng.random((3, 5000)) * np.array([[1.0], [1.0], [1.0]])
    pos[0, :100] = xf[rng.integers(0, 18, 100)]        # exactly on faces
    pos[1, 100:200] = yf[rng.integers(0, 10, 100)]
    pos[:, 200] = (1.5, 0.5, 0.5)
    pos[:, 201] = (0.5, np.nan, 0.5)
    cell, nout = orc.locate_hex(xf, yf, zf, pos)
    ids = []
    for a, f in enumerate((xf, yf, zf)):
        i = np.searchsorted(f, pos[a], side="right") - 1
        ids.append(np.clip(i, 0, len(f) - 2))
    inside = np.all([(pos[a] >= f[0]) & (pos[a] <= f[-1]) for a, f in enumerate((xf, yf, zf))], axis=0)
    ref = np.where(inside, (ids[2] * 9 + ids[1]) * 17 + ids[0], -1)
    assert nout == 2
    assert np.array_equal(cell, ref)
    # power-of-two spacing: the same cells as the uniform-mesh locate
    dx = 1.0 / 16
    f = np.arange(17) * dx
    p2 = rng.random((3, 2000))
    a, _ = orc.locate_hex(f, f, f, p2)
    b, _ = orc.locate_structured((16, 16, 16), (0, 0, 0), dx, p2)
    assert np.array_equal(a, b)


def test_hex_operator_is_exact_on_linear_fields(orc):
    """Two-point flux on a Cartesian stretched mesh with uniform D is consistent: for a
    linear field u = a.x the flux through a face is D |A_f| a_axis, equal on both faces of
    an interior cell along each axis, so (L u)_k = 0 in every interior cell; a wall cell
    loses exactly the flux of its missing face (D |A_f| a_axis).  A wrong centre distance,
    area or neighbour index breaks this at stretched spacing."""
    xf, yf, zf = _stretched_faces(11, 1.07), _stretched_faces(8, 0.93, 0.7), _stretched_faces(6, 1.12, 0.4)
    n3 = (11, 8, 6)
    D0 = 2.5
    vc, rp, col, val = orc.hex_build(xf, yf, zf, np.full(int(np.prod(n3)), D0))
    n = len(vc)
    A = scipy.sparse.csr_matrix((val, col, rp), shape=(n, n))
    cen = [0.5 * (f[1:] + f[:-1]) for f in (xf, yf, zf)]
    wid = [np.diff(f) for f in (xf, yf, zf)]
    Z, Y, X = np.meshgrid(cen[2], cen[1], cen[0], indexing="ij")
    WZ, WY, WX = np.meshgrid(wid[2], wid[1], wid[0], indexing="ij")
    grid_ix = np.meshgrid(np.arange(n3[2]), np.arange(n3[1]), np.arange(n3[0]), indexing="ij")
    a = (0.7, -1.3, 2.1)
    Lu = (A @ (a[0] * X + a[1] * Y + a[2] * Z).ravel()).reshape(n3[::-1])
    expect = np.zeros(n3[::-1])
    areas = (WY * WZ, WX * WZ, WX * WY)
    for ax, idx in enumerate((grid_ix[2], grid_ix[1], grid_ix[0])):
        expect -= np.where(idx == n3[ax] - 1, D0 * areas[ax] * a[ax], 0.0)   # no face above
        expect += np.where(idx == 0, D0 * areas[ax] * a[ax], 0.0)            # no face below
    assert np.max(np.abs(Lu - expect)) <= 1e-12 * np.max(np.abs(expect))

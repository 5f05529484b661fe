"""Seeded synthetic inputs for diffusion-based coarse graining.

This module only draws inputs: particle centroids and carried quantities, and
tetrahedral meshes.  It holds none of the method's arithmetic and is shared by the
tests, the benchmark, the oracle calls and the CUDA calls alike.

The paper's own particle sets (1000 quasi-random spheres in a 135 d_p square slab,
Section 4) are not published, so every workload here is a seeded stand-in with the
shapes, sizes and distributions listed below (numpy ``default_rng(seed)``; particle
order is the generation order, which matters for ordered deposition):

* ``uniform_cube``: the 32^3 unit-cube case -- 10,000 spheres of d = 0.01, U[0,1]^3,
  b = 3 dx, 10 implicit-Euler steps, one field (volume).
* ``clustered_cube``: the 128^3 unit-cube case -- 2,000,000 spheres of d = 0.004 in
  20 Gaussian clusters (sigma 0.05, centres U[0.1,0.9]^3), at most 8 centroids per
  128^3 cell (local volume fraction <= 0.562); a centroid outside the cube or in a
  full cell is redrawn from its cluster, after 64 tries from U[0,1]^3 (until it lands in
  a cell with room).
* ``kuhn_tet_mesh``: an n^3 hex grid of the unit cube, each hex split into 6 tets
  along its v000-v111 diagonal (one per axis permutation, lexicographic order),
  interior vertices jittered by U(-0.2 dx, 0.2 dx) per coordinate.
* ``layered_cube``: 5,000,000 spheres of d = 0.003: 70 % uniform in a bottom layer
  z in [0, h] with h = 0.7 N V_p / 0.55, 30 % uniform in the cube.
* ``batched_snapshots``: 64 snapshots, cube side N ~ U{32..96}, n_p = round(10^U(4,6)),
  d = 0.004, 5 fields: V_p, V_p u (u ~ N(0, 0.1) per component), drag ~ LogNormal(0,1).
* ``channel``: a 512x256x256 mesh over a 4x2x2 box, 50,000,000 spheres of d = 0.004,
  density proportional to 1 + 0.5 sin(2 pi x) (x in box units), by rejection.
* ``stretched_box``: a 128^3 stretched Cartesian mesh of the unit cube, uniform in x and
  y, z faces growing geometrically (ratio 1.02) away from the bottom wall, a cell
  diffusion constant of 1 except a block with D = 0 (where the smoothed field stays the
  PCM field) and a block with D = 4; the particles of ``layered_cube`` with their
  velocities as three more fields (u ~ N(0, 0.1)).
* ``channel_velocities``: per-particle velocities for the channel, a mean streamwise
  flow of 1 + 0.5 sin(2 pi x) plus N(0, 0.1) per component.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def sphere_volume(d: float) -> float:
    return math.pi * d ** 3 / 6.0


@dataclass
class StructuredCase:
    """A uniform-mesh workload: mesh, particles (pos [3,n], weights [nf,n]) and the
    smoothing parameters."""
    name: str
    dims: tuple
    origin: tuple
    dx: float
    pos: np.ndarray
    w: np.ndarray
    b: float
    nsteps: int
    extra: dict = field(default_factory=dict)

    @property
    def ncells(self) -> int:
        return int(self.dims[0] * self.dims[1] * self.dims[2])

    @property
    def n(self) -> int:
        return int(self.pos.shape[1])


def uniform_particles(rng, n, lo, hi):
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    u = rng.random((3, n))
    return lo[:, None] + u * (hi - lo)[:, None]


def uniform_cube(n_side=32, n_particles=10_000, d=0.01, b_over_dx=3.0, nsteps=10, seed=0):
    """Unit cube, n_side^3 cells, spheres at U[0,1]^3 centres, one field (V_p)."""
    rng = np.random.default_rng(seed)
    pos = rng.random((3, n_particles))
    w = np.full((1, n_particles), sphere_volume(d))
    dx = 1.0 / n_side
    return StructuredCase("uniform_cube_%d" % n_side, (n_side,) * 3, (0.0, 0.0, 0.0), dx, pos, w,
                          b_over_dx * dx, nsteps)


def clustered_cube(n_side=128, n_particles=2_000_000, d=0.004, n_clusters=20, sigma=0.05,
                   cap_fraction=0.6, b_over_dx=2.0, nsteps=10, seed=0, max_tries=64):
    """Unit cube, Gaussian clusters with a per-cell cap on the number of centroids."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / n_side
    vp = sphere_volume(d)
    cap = int(math.floor(cap_fraction * dx ** 3 / vp))
    centres = 0.1 + 0.8 * rng.random((n_clusters, 3))
    which = rng.integers(0, n_clusters, size=n_particles)
    pos = centres[which].T + sigma * rng.standard_normal((3, n_particles))
    occupancy = np.zeros(n_side ** 3, dtype=np.int64)     # accepted centroids per bin
    todo = np.arange(n_particles)                          # not yet accepted, in order
    attempt = 0
    while len(todo):
        p = pos[:, todo]
        inside = np.all((p >= 0.0) & (p <= 1.0), axis=0)
        ijk = np.clip(np.floor(np.where(inside, p, 0.0) * n_side).astype(np.int64), 0, n_side - 1)
        binid = (ijk[2] * n_side + ijk[1]) * n_side + ijk[0]
        # rank of each candidate among this round's candidates of its bin, in index order
        order = np.argsort(binid, kind="stable")
        sb = binid[order]
        starts = np.r_[0, np.flatnonzero(np.diff(sb)) + 1] if len(sb) else np.zeros(0, np.int64)
        run_start = np.repeat(starts, np.diff(np.r_[starts, len(sb)]))
        rank = np.empty(len(todo), dtype=np.int64)
        rank[order] = np.arange(len(todo)) - run_start
        ok = inside & (occupancy[binid] + rank < cap)
        np.add.at(occupancy, binid[ok], 1)
        todo = todo[~ok]
        if len(todo) == 0:
            break
        attempt += 1
        if attempt > max_tries:   # from U[0,1]^3 now, still under the cap
            if attempt > max_tries + 10_000 or occupancy.sum() + len(todo) > cap * n_side ** 3:
                raise ValueError("clustered_cube: the cap leaves no room for the particles")
            pos[:, todo] = rng.random((3, len(todo)))
        else:
            pos[:, todo] = centres[which[todo]].T + sigma * rng.standard_normal((3, len(todo)))
    w = np.full((1, n_particles), vp)
    return StructuredCase("clustered_cube_%d" % n_side, (n_side,) * 3, (0.0, 0.0, 0.0), dx, pos, w,
                          b_over_dx * dx, nsteps, {"cap": cap, "sigma": sigma})


def layered_positions(rng, n_particles, d=0.003, frac_layer=0.7, layer_fraction=0.55):
    vp = sphere_volume(d)
    h = frac_layer * n_particles * vp / layer_fraction
    n_layer = int(round(frac_layer * n_particles))
    pos = rng.random((3, n_particles))
    pos[2, :n_layer] *= h
    return pos, h


def layered_cube(n_particles=5_000_000, d=0.003, seed=0):
    rng = np.random.default_rng(seed)
    pos, h = layered_positions(rng, n_particles, d)
    w = np.full((1, n_particles), sphere_volume(d))
    return pos, w, h


def kuhn_tet_mesh(n_side, jitter=0.2, seed=0, lengths=(1.0, 1.0, 1.0)):
    """Kuhn split of an n_side^3 hex grid into 6 n_side^3 tets; interior vertices
    jittered by U(-jitter*dx, jitter*dx) per coordinate.  Tet index = hex id * 6 +
    permutation index; hex id = (k*n + j)*n + i.  Returns (xyz [nv,3], tets [nt,4])."""
    n = int(n_side)
    rng = np.random.default_rng(seed)
    L = np.asarray(lengths, dtype=np.float64)
    g = [np.linspace(0.0, L[a], n + 1) for a in range(3)]
    Z, Y, X = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).copy()
    if jitter > 0.0:
        dxv = L / n
        off = rng.uniform(-1.0, 1.0, size=xyz.shape) * (jitter * dxv)[None, :]
        idx = np.arange(n + 1)
        Kz, Jy, Ix = np.meshgrid(idx, idx, idx, indexing="ij")   # vertex id order
        interior = ((Ix > 0) & (Ix < n) & (Jy > 0) & (Jy < n) & (Kz > 0) & (Kz < n)).ravel()
        xyz[interior] += off[interior]
    def vid(i, j, k):
        return (k * (n + 1) + j) * (n + 1) + i
    ii, jj, kk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    # hex id ordering (k*n + j)*n + i
    ii = ii.transpose(2, 1, 0).ravel()
    jj = jj.transpose(2, 1, 0).ravel()
    kk = kk.transpose(2, 1, 0).ravel()
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    tets = np.empty((n ** 3, 6, 4), dtype=np.int32)
    for p, perm in enumerate(perms):
        c = [ii.copy(), jj.copy(), kk.copy()]
        tets[:, p, 0] = vid(c[0], c[1], c[2])
        for s in range(3):
            c[perm[s]] = c[perm[s]] + 1
            tets[:, p, s + 1] = vid(c[0], c[1], c[2])
    return xyz, tets.reshape(-1, 4)


def batched_snapshots(n_snap=64, d=0.004, side_lo=32, side_hi=96, logn_lo=4.0, logn_hi=6.0,
                      b_over_dx=3.0, nsteps=10, seed=0):
    """64 independent unit-cube snapshots of uneven size with 5 carried fields."""
    rng = np.random.default_rng(seed)
    vp = sphere_volume(d)
    cases = []
    for s in range(n_snap):
        side = int(rng.integers(side_lo, side_hi + 1))
        n_p = int(round(10.0 ** rng.uniform(logn_lo, logn_hi)))
        pos = rng.random((3, n_p))
        u = 0.1 * rng.standard_normal((3, n_p))
        drag = rng.lognormal(0.0, 1.0, size=n_p)
        w = np.empty((5, n_p))
        w[0] = vp
        w[1:4] = vp * u
        w[4] = drag
        dx = 1.0 / side
        cases.append(StructuredCase("snapshot_%02d" % s, (side,) * 3, (0.0, 0.0, 0.0), dx, pos, w,
                                    b_over_dx * dx, nsteps))
    return cases


def channel(n_particles=50_000_000, dims=(512, 256, 256), lengths=(4.0, 2.0, 2.0), d=0.004,
            b_over_dx=4.0, nsteps=40, seed=0, chunk=8_000_000):
    """Modulated-density channel: rejection sampling of 1 + 0.5 sin(2 pi x)."""
    rng = np.random.default_rng(seed)
    L = np.asarray(lengths, dtype=np.float64)
    out = np.empty((3, n_particles))
    got = 0
    while got < n_particles:
        m = min(chunk, 2 * (n_particles - got) + 1024)
        cand = rng.random((3, m)) * L[:, None]
        keep = rng.random(m) * 1.5 < 1.0 + 0.5 * np.sin(2.0 * np.pi * cand[0])
        cand = cand[:, keep]
        k = min(cand.shape[1], n_particles - got)
        out[:, got:got + k] = cand[:, :k]
        got += k
    w = np.full((1, n_particles), sphere_volume(d))
    dx = lengths[0] / dims[0]
    return StructuredCase("channel_%dx%dx%d" % dims, tuple(dims), (0.0, 0.0, 0.0), dx, out, w,
                          b_over_dx * dx, nsteps)


def stretched_box(n=128, ratio=1.02, n_particles=5_000_000, d=0.003, seed=0):
    """Face coordinates (xf, yf, zf), cell diffusion constants D [ncells] (cell k =
    (iz n + iy) n + ix), particle centroids [3, n_p] and weights [4, n_p] (V_p and V_p u)."""
    rng = np.random.default_rng(seed)
    xf = np.linspace(0.0, 1.0, n + 1)
    wz = ratio ** np.arange(n)
    zf = np.concatenate([[0.0], np.cumsum(wz)])
    zf /= zf[-1]
    zf[-1] = 1.0
    D = np.ones((n, n, n))
    D[n // 8:n // 4, 3 * n // 8:5 * n // 8, 3 * n // 8:5 * n // 8] = 0.0
    D[n // 2:3 * n // 4, n // 8:n // 4, :] = 4.0
    pos, _ = layered_positions(rng, n_particles, d=d)
    u = 0.1 * rng.standard_normal((3, n_particles))
    vp = sphere_volume(d)
    w = np.empty((4, n_particles))
    w[0] = vp
    w[1:] = vp * u
    return xf, xf.copy(), zf, D.ravel(), pos, w


def channel_velocities(pos, seed=1):
    """Particle velocities [3, n] for the channel: 1 + 0.5 sin(2 pi x) streamwise plus
    N(0, 0.1) per component."""
    rng = np.random.default_rng(seed)
    v = 0.1 * rng.standard_normal((3, pos.shape[1]))
    v[0] += 1.0 + 0.5 * np.sin(2.0 * np.pi * pos[0])
    return v


def random_field(rng, nf, ncells, positive=True):
    """A dense random initial field (used to exercise the diffusion step alone)."""
    f = rng.random((nf, ncells))
    return f if positive else f - 0.5

"""The seeded input generators (workloads/) against the recipes they state: sizes, supports,
weights and the distributions' defining properties, checked on small draws (no GPU).

The generators hold none of the method's arithmetic. These tests pin what every parity test
and benchmark line feeds the oracle and the CUDA path: the 32^3 uniform case, the clustered
128^3 case (its per-cell cap), the layered bed of the tet case, the 64-snapshot batch and
the modulated channel."""
import math

import numpy as np

import workloads as W


def test_uniform_cube_recipe_and_seeding():
    c = W.uniform_cube()
    assert c.dims == (32, 32, 32) and c.n == 10_000 and c.w.shape == (1, 10_000)
    assert np.all((c.pos >= 0.0) & (c.pos < 1.0))
    assert np.all(c.w == math.pi * 0.01 ** 3 / 6.0)
    assert c.b == 3.0 / 32 and c.nsteps == 10
    again, other = W.uniform_cube(), W.uniform_cube(seed=1)
    assert np.array_equal(again.pos, c.pos) and not np.array_equal(other.pos, c.pos)
    # U[0,1]^3: per-axis means and variances near 1/2 and 1/12 (10,000 draws: about 3e-3
    # standard error on the mean)
    assert np.all(np.abs(c.pos.mean(axis=1) - 0.5) < 0.015)
    assert np.all(np.abs(c.pos.var(axis=1) - 1.0 / 12.0) < 0.005)


def test_clustered_cube_cap_holds_and_binds():
    """The per-cell cap is floor(cap_fraction dx^3 / V_p) centroids (8 for the 128^3 case);
    no cell holds more, and on a dense draw the cap is reached."""
    full = 0.6 * (1.0 / 128) ** 3 / W.sphere_volume(0.004)
    assert math.floor(full) == 8
    n_side, d = 64, 0.008
    c = W.clustered_cube(n_side=n_side, n_particles=200_000, d=d, seed=3)
    cap = c.extra["cap"]
    assert cap == math.floor(0.6 * (1.0 / n_side) ** 3 / W.sphere_volume(d)) == 8
    assert c.pos.shape == (3, 200_000) and np.all((c.pos >= 0.0) & (c.pos <= 1.0))
    ijk = np.clip(np.floor(c.pos * n_side).astype(np.int64), 0, n_side - 1)
    counts = np.bincount((ijk[2] * n_side + ijk[1]) * n_side + ijk[0], minlength=n_side ** 3)
    assert counts.max() == cap
    # clustered, not uniform: many full cells, many empty ones
    assert np.count_nonzero(counts == cap) > 1000 and np.count_nonzero(counts == 0) > n_side ** 3 // 4
    assert np.all(c.w == W.sphere_volume(d))


def test_layered_bed_fraction():
    """70 % of the centroids in a bottom layer of height h = 0.7 N V_p / 0.55 (a layer at
    volume fraction 0.55), the rest uniform in the cube."""
    n, d = 100_000, 0.003
    pos, w, h = W.layered_cube(n_particles=n, d=d, seed=4)
    assert pos.shape == (3, n) and w.shape == (1, n)
    vp = W.sphere_volume(d)
    assert abs(h - 0.7 * n * vp / 0.55) <= 1e-15 * h
    n_layer = int(round(0.7 * n))
    assert np.all(pos[2, :n_layer] <= h) and np.all((pos >= 0.0) & (pos < 1.0))
    assert abs(n_layer * vp / h - 0.55) < 1e-12
    # the uniform remainder reaches the top of the cube
    assert pos[2, n_layer:].max() > 0.9


def test_batched_snapshots_recipe():
    cases = W.batched_snapshots()
    assert len(cases) == 64
    sides = np.array([c.dims[0] for c in cases])
    counts = np.array([c.n for c in cases])
    assert sides.min() >= 32 and sides.max() <= 96 and len(set(sides)) > 20
    assert counts.min() >= 10_000 and counts.max() <= 1_000_000
    vp = W.sphere_volume(0.004)
    big = cases[int(np.argmax(counts))]
    assert big.w.shape == (5, big.n) and np.all(big.w[0] == vp)
    u = big.w[1:4] / vp                      # velocities ~ N(0, 0.1) per component
    assert np.all(np.abs(u.mean(axis=1)) < 0.01) and np.all(np.abs(u.std(axis=1) - 0.1) < 0.005)
    drag = big.w[4]                          # LogNormal(0, 1)
    assert np.all(drag > 0.0)
    assert abs(np.log(drag).mean()) < 0.02 and abs(np.log(drag).std() - 1.0) < 0.02
    assert all(abs(c.b - 3.0 / c.dims[0]) <= 1e-15 * c.b for c in cases)


def test_channel_density_modulation():
    """Density proportional to 1 + 0.5 sin(2 pi x) on a 4 x 2 x 2 box: the half-periods
    where the sine is positive hold (1/2 + 1/(2 pi)) of the particles."""
    n = 400_000
    c = W.channel(n_particles=n, seed=5)
    assert c.dims == (512, 256, 256) and c.dx == 4.0 / 512 and c.nsteps == 40
    assert np.all((c.pos >= 0.0) & (c.pos < np.array([[4.0], [2.0], [2.0]])))
    frac = np.count_nonzero(np.mod(c.pos[0], 1.0) < 0.5) / n
    expect = 0.5 + 1.0 / (2.0 * math.pi)
    assert abs(frac - expect) < 5 * math.sqrt(expect * (1 - expect) / n)
    # y and z stay uniform
    assert abs(c.pos[1].mean() - 1.0) < 0.01 and abs(c.pos[2].mean() - 1.0) < 0.01
    v = W.channel_velocities(c.pos[:, :100_000])
    resid = v[0] - (1.0 + 0.5 * np.sin(2.0 * np.pi * c.pos[0, :100_000]))
    assert abs(resid.mean()) < 0.002 and abs(resid.std() - 0.1) < 0.002

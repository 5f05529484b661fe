"""Run one diffusion-smoothing case for a profiler (ncu) or a quick timing.

    python -m paper_1409_0001_gb300.profile_case --n 256 --precision 3 --reps 2

Builds a seeded random field on an n^3 (or --dims) unit-spaced hex mesh and smooths
it --reps times with the chosen precision mode (see include/cg.h), b = --b-over-dx
cells, --nsteps implicit-Euler steps (or, with --explicit-k K, --nsteps explicit steps
in FP32 with K steps per launch; or, with --tet --locate N, the point location of N
particles).  Prints the device time of each call.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--dims", type=int, nargs=3, default=None)
    ap.add_argument("--precision", type=int, default=3)
    ap.add_argument("--b-over-dx", type=float, default=2.0)
    ap.add_argument("--nsteps", type=int, default=10)
    ap.add_argument("--nfields", type=int, default=1)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--tet", action="store_true", help="Kuhn tet mesh of n^3 hexes instead")
    ap.add_argument("--shape", type=int, default=0, help="sweep_shape (0 = autotuned)")
    ap.add_argument("--explicit-k", type=int, default=0,
                    help="explicit Euler instead: fused_k steps per launch (FP32, temporal "
                         "blocking), --nsteps steps at dtau/dx^2 = 0.1")
    ap.add_argument("--batched", type=int, default=0,
                    help="the first N snapshots of the 64-snapshot batch (cube sides 32..96, "
                         "5 fields, b = 3 dx) through one batched call instead")
    ap.add_argument("--deposit", action="store_true",
                    help="ordered deposition of the clustered n^3 workload (2,000,000 spheres "
                         "at n = 128) instead of a diffusion")
    ap.add_argument("--locate", type=int, default=0,
                    help="with --tet: point location of N particles of the layered workload "
                         "(a dense bottom layer) on the Kuhn tet mesh instead of a diffusion")
    a = ap.parse_args(argv)

    import numpy as np
    import torch

    import paper_1409_0001_gb300 as cg
    from paper_1409_0001_gb300 import build
    import workloads as W

    build.build()
    if a.batched:
        cases = W.batched_snapshots()[:a.batched]
        meshes = [cg.StructuredMesh(c.dims, c.origin, c.dx) for c in cases]
        pos = [torch.from_numpy(c.pos).cuda() for c in cases]
        w = [torch.from_numpy(c.w).cuda() for c in cases]
        for r in range(a.reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, rep = cg.coarse_grain_batched(meshes, pos, w, cg.Params(nsteps=a.nsteps, precision=a.precision),
                                             bandwidths=[c.b for c in cases], report=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            print("rep %d: %.3f ms, %d cell-updates, %.3e cell-updates/s"
                  % (r, dt * 1e3, rep["cell_updates"], rep["cell_updates"] / dt))
        return
    if a.deposit:
        c = W.clustered_cube(n_side=a.n, n_particles=2_000_000 * (a.n // 128) ** 3 or 2_000_000)
        mesh = cg.StructuredMesh(c.dims, c.origin, c.dx)
        pos, w = torch.from_numpy(c.pos).cuda(), torch.from_numpy(c.w).cuda()
        for r in range(a.reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, rep = cg.deposit(mesh, pos, w, cg.Params(), report=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            print("rep %d: %.3f ms (locate %.3f, deposit %.3f), %.3e particles/s"
                  % (r, dt * 1e3, rep["ms_locate"], rep["ms_deposit"], c.n / dt))
        mesh.close()
        return
    dims = tuple(a.dims) if a.dims else (a.n, a.n, a.n)
    dx = 1.0 / dims[0]
    if a.tet:
        xyz, tets = W.kuhn_tet_mesh(a.n)
        mesh = cg.TetMesh(xyz, tets)
        if a.locate:
            pos = torch.from_numpy(W.layered_cube(n_particles=a.locate)[0]).cuda()
            for r in range(a.reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, nout = cg.locate(mesh, pos)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                print("rep %d: %.3f ms, %d outside, %.3e particles/s" % (r, dt * 1e3, nout, a.locate / dt))
            mesh.close()
            return
    else:
        mesh = cg.StructuredMesh(dims, (0.0, 0.0, 0.0), dx)
    rng = np.random.default_rng(0)
    u0 = torch.from_numpy(rng.random((a.nfields, mesh.ncells))).cuda()
    if a.explicit_k:
        p = cg.Params(T=0.1 * dx * dx * a.nsteps, nsteps=a.nsteps, scheme=2, fused_k=a.explicit_k)
    else:
        p = cg.Params(bandwidth=a.b_over_dx * dx, nsteps=a.nsteps, precision=a.precision,
                      sweep_shape=a.shape)
    for r in range(a.reps):
        u = u0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, rep = cg.diffuse(mesh, u, p, report=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        print("rep %d: %.3f ms, %d cell-updates, %.3e cell-updates/s, residual %.2e"
              % (r, dt * 1e3, rep["cell_updates"], rep["cell_updates"] / dt,
                 rep["final_rel_residual"]))
    mesh.close()


if __name__ == "__main__":
    main()

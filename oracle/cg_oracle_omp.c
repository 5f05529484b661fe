/*
 * cg_oracle_omp.c -- the oracle's arithmetic (cg_oracle.c) spread over the host's cores
 * with OpenMP: the multi-core CPU baseline of diffusion-based coarse graining (Sun &
 * Xiao), and a faster FP64 reference for workloads too large for the single-thread
 * oracle to finish in seconds.
 *
 * TEST INFRASTRUCTURE ONLY, like cg_oracle.c: only the test-suite and the benchmark's
 * CPU-baseline and error legs load it.  It shares no code with the CUDA library or with
 * cg_oracle.c (it restates the same definitions), and neither calls the other.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared.
 *
 * Every per-element expression is the one cg_oracle.c evaluates, in the same order, so
 * the locate and the deposition give the same bits, and the only difference in the
 * diffusion is the order of the conjugate-gradient dot products: here each is a sum of
 * fixed chunks of ORC_OMP_CHUNK terms (each chunk summed in index order, the chunk sums
 * then added in chunk order), which does not depend on the number of threads.
 *   1. Locate, Section 3.1 (uniform mesh) and the tet rule of cg_oracle.c (Section 4.3
 *      unstructured cells): one particle per iteration, any order.
 *   2. Deposition, Eq. (pcm-k): each thread owns a range of cells and adds, in
 *      ascending particle index, the particles whose cell is in its range -- the
 *      sequential sum of every cell, bit for bit.
 *   3. Diffusion, Eq. (diffusion): implicit Euler or Crank-Nicolson steps, each solved
 *      by unpreconditioned conjugate gradients from u^n to ||r|| <= tol ||b||.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

#define ORC_OMP_CHUNK 4096

int omp_num_threads_used(void)
{
    return omp_get_max_threads();
}

/* Threads for the following parallel regions (n >= 1). */
void omp_use_threads(int n)
{
    if (n >= 1) omp_set_num_threads(n);
}

/* ---------------------------------------------------------------- locate (uniform) */
int64_t omp_locate_structured(int nx, int ny, int nz, const double *origin, double dx,
                              int64_t n, const double *pos, int32_t *cell)
{
    const int dims[3] = {nx, ny, nz};
    const double inv_dx = 1.0 / dx;
    double hi[3];
    for (int a = 0; a < 3; ++a) {
        double len = (double)dims[a] * dx;
        hi[a] = origin[a] + len;
    }
    int64_t out = 0;
#pragma omp parallel for schedule(static) reduction(+ : out)
    for (int64_t i = 0; i < n; ++i) {
        int idx[3];
        int inside = 1;
        for (int a = 0; a < 3; ++a) {
            double x = pos[(int64_t)a * n + i];
            if (!(x >= origin[a] && x <= hi[a])) {
                inside = 0;
                break;
            }
            double t = (x - origin[a]) * inv_dx;
            int k = (int)floor(t);
            if (k > dims[a] - 1) k = dims[a] - 1;
            if (k < 0) k = 0;
            idx[a] = k;
        }
        if (!inside) {
            cell[i] = -1;
            ++out;
            continue;
        }
        cell[i] = (int32_t)(((int64_t)idx[2] * ny + idx[1]) * nx + idx[0]);
    }
    return out;
}

/* ---------------------------------------------------------------- deposition */
/* mode 0: each cell's particles in ascending index from +0.0, then / V_c.
 * mode 1: llrint(w * 2^F) summed in int64, then * 2^-F / V_c (fbits[f] = F). */
void omp_deposit(int64_t n, const int32_t *cell, int nf, const double *w, int64_t ncells,
                 const double *vc, double vc_uniform, int mode, const int *fbits, double *out)
{
    for (int f = 0; f < nf; ++f) {
        const double *wf = w + (int64_t)f * n;
        double *of = out + (int64_t)f * ncells;
        const double scale = mode == 1 ? ldexp(1.0, fbits[f]) : 1.0;
        const double unscale = mode == 1 ? ldexp(1.0, -fbits[f]) : 1.0;
#pragma omp parallel
        {
            int nt = omp_get_num_threads(), t = omp_get_thread_num();
            int64_t c0 = ncells * t / nt, c1 = ncells * (t + 1) / nt;
            if (mode == 0) {
                for (int64_t k = c0; k < c1; ++k) of[k] = 0.0;
                for (int64_t i = 0; i < n; ++i) {
                    int64_t c = cell[i];
                    if (c < c0 || c >= c1) continue;
                    of[c] = of[c] + wf[i];
                }
                for (int64_t k = c0; k < c1; ++k) {
                    double v = vc ? vc[k] : vc_uniform;
                    of[k] = of[k] / v;
                }
            } else {
                int64_t *acc = (int64_t *)calloc((size_t)(c1 > c0 ? c1 - c0 : 1), sizeof(int64_t));
                for (int64_t i = 0; i < n; ++i) {
                    int64_t c = cell[i];
                    if (c < c0 || c >= c1) continue;
                    acc[c - c0] += (int64_t)llrint(wf[i] * scale);
                }
                for (int64_t k = c0; k < c1; ++k) {
                    double v = vc ? vc[k] : vc_uniform;
                    double s = (double)acc[k - c0] * unscale;
                    of[k] = s / v;
                }
                free(acc);
            }
        }
    }
}

/* ---------------------------------------------------------------- reductions */
static double chunked_dot(int64_t n, const double *a, const double *b, double *part)
{
    int64_t nch = (n + ORC_OMP_CHUNK - 1) / ORC_OMP_CHUNK;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nch; ++c) {
        int64_t i0 = c * ORC_OMP_CHUNK, i1 = i0 + ORC_OMP_CHUNK < n ? i0 + ORC_OMP_CHUNK : n;
        double s = 0.0;
        for (int64_t i = i0; i < i1; ++i) s += a[i] * b[i];
        part[c] = s;
    }
    double s = 0.0;
    for (int64_t c = 0; c < nch; ++c) s += part[c];
    return s;
}

/* ---------------------------------------------------------------- operators */
typedef struct {
    int kind;                       /* 0 uniform hex, 1 CSR */
    int nx, ny, nz;
    double cth;                     /* theta * dtau / dx^2 (hex) or theta * dtau (CSR) */
    int64_t n;
    const double *vc;
    const int64_t *rowptr;
    const int32_t *col;
    const double *val;
} op_t;

/* out = L u (hex: sum over existing face neighbours of u_l - u_k; CSR: the matrix row) */
static void op_lap(const op_t *o, const double *u, double *out)
{
    if (o->kind == 0) {
        const int nx = o->nx, ny = o->ny, nz = o->nz;
#pragma omp parallel for schedule(static) collapse(2)
        for (int iz = 0; iz < nz; ++iz)
            for (int iy = 0; iy < ny; ++iy)
                for (int ix = 0; ix < nx; ++ix) {
                    int64_t k = ((int64_t)iz * ny + iy) * nx + ix;
                    double s = 0.0;
                    if (ix > 0) s += u[k - 1] - u[k];
                    if (ix < nx - 1) s += u[k + 1] - u[k];
                    if (iy > 0) s += u[k - nx] - u[k];
                    if (iy < ny - 1) s += u[k + nx] - u[k];
                    if (iz > 0) s += u[k - (int64_t)nx * ny] - u[k];
                    if (iz < nz - 1) s += u[k + (int64_t)nx * ny] - u[k];
                    out[k] = s;
                }
    } else {
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < o->n; ++k) {
            double s = 0.0;
            for (int64_t e = o->rowptr[k]; e < o->rowptr[k + 1]; ++e) s += o->val[e] * u[o->col[e]];
            out[k] = s;
        }
    }
}

/* out = A u: hex u - cth L u; CSR V_c u - cth L u (as cg_oracle.c forms them) */
static void op_apply(const op_t *o, const double *u, double *out)
{
    op_lap(o, u, out);
    if (o->kind == 0) {
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < o->n; ++k) out[k] = u[k] - o->cth * out[k];
    } else {
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < o->n; ++k) out[k] = o->vc[k] * u[k] - o->cth * out[k];
    }
}

/* conjugate gradients on A x = b from x, to ||r|| <= tol ||b||; iterations or -1 */
static int cg_solve(const op_t *o, const double *b, double *x, double tol, int max_iter,
                    double *r, double *p, double *Ap, double *part)
{
    const int64_t n = o->n;
    op_apply(o, x, Ap);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        r[i] = b[i] - Ap[i];
        p[i] = r[i];
    }
    double bb = chunked_dot(n, b, b, part);
    double rr = chunked_dot(n, r, r, part);
    double thresh = tol * tol * bb;
    int it = 0;
    while (rr > thresh && it < max_iter) {
        op_apply(o, p, Ap);
        double pAp = chunked_dot(n, p, Ap, part);
        if (!(pAp > 0.0)) break;
        double alpha = rr / pAp;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            x[i] = x[i] + alpha * p[i];
            r[i] = r[i] - alpha * Ap[i];
        }
        double rr_new = chunked_dot(n, r, r, part);
        double beta = rr_new / rr;
        rr = rr_new;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        ++it;
    }
    return rr <= thresh ? it : -1;
}

/* nsteps implicit-Euler (scheme 0) or Crank-Nicolson (scheme 1) steps of every field */
static int diffuse(op_t *o, int nf, double *u, double dtau, double c, int nsteps, int scheme,
                   double tol, int max_iter, int64_t *iters_out)
{
    const int64_t n = o->n;
    double *buf = (double *)malloc((size_t)(5 * n) * sizeof(double));
    int64_t nch = (n + ORC_OMP_CHUNK - 1) / ORC_OMP_CHUNK;
    double *part = (double *)malloc((size_t)(nch > 0 ? nch : 1) * sizeof(double));
    double *rhs = buf, *lu = buf + n, *r = buf + 2 * n, *p = buf + 3 * n, *Ap = buf + 4 * n;
    o->cth = scheme == 1 ? 0.5 * c : c;
    int64_t iters = 0;
    int status = 0;
    for (int f = 0; f < nf; ++f) {
        double *uf = u + (int64_t)f * n;
        for (int s = 0; s < nsteps; ++s) {
            if (scheme == 1) {
                op_lap(o, uf, lu);
                if (o->kind == 0) {
#pragma omp parallel for schedule(static)
                    for (int64_t k = 0; k < n; ++k) rhs[k] = uf[k] + 0.5 * c * lu[k];
                } else {
#pragma omp parallel for schedule(static)
                    for (int64_t k = 0; k < n; ++k) rhs[k] = o->vc[k] * uf[k] + 0.5 * dtau * lu[k];
                }
            } else if (o->kind == 0) {
#pragma omp parallel for schedule(static)
                for (int64_t k = 0; k < n; ++k) rhs[k] = uf[k];
            } else {
#pragma omp parallel for schedule(static)
                for (int64_t k = 0; k < n; ++k) rhs[k] = o->vc[k] * uf[k];
            }
            int it = cg_solve(o, rhs, uf, tol, max_iter, r, p, Ap, part);
            if (it < 0) {
                status = -1;
                it = max_iter;
            }
            iters += it;
        }
    }
    free(part);
    free(buf);
    if (iters_out) *iters_out = iters;
    return status;
}

/* Uniform hex mesh with zero-flux walls; scheme 0 or 1 (as orc_diffuse_structured). */
int omp_diffuse_structured(int nx, int ny, int nz, double dx, int nf, double *u, double T,
                           int nsteps, int scheme, double tol, int max_iter, int64_t *iters_out)
{
    if (scheme != 0 && scheme != 1) return -2;
    op_t o;
    memset(&o, 0, sizeof(o));
    o.kind = 0;
    o.nx = nx;
    o.ny = ny;
    o.nz = nz;
    o.n = (int64_t)nx * ny * nz;
    double dtau = T / (double)nsteps;
    double c = dtau / (dx * dx);
    return diffuse(&o, nf, u, dtau, c, nsteps, scheme, tol, max_iter, iters_out);
}

/* CSR operator from orc_tet_build / orc_hex_build; scheme 0 or 1 (as orc_diffuse_csr). */
int omp_diffuse_csr(int64_t n, const double *vc, const int64_t *rowptr, const int32_t *col,
                    const double *val, int nf, double *u, double T, int nsteps, int scheme,
                    double tol, int max_iter, int64_t *iters_out)
{
    if (scheme != 0 && scheme != 1) return -2;
    op_t o;
    memset(&o, 0, sizeof(o));
    o.kind = 1;
    o.n = n;
    o.vc = vc;
    o.rowptr = rowptr;
    o.col = col;
    o.val = val;
    double dtau = T / (double)nsteps;
    return diffuse(&o, nf, u, dtau, dtau, nsteps, scheme, tol, max_iter, iters_out);
}

/* ---------------------------------------------------------------- locate (tets) */
/* The rule of cg_oracle.c: the lowest-index tet whose box holds x and whose four
 * barycentric coordinates (signed-volume ratios, the same expression) are >= 0, else
 * the box-holding tet with the largest minimum coordinate (lowest index on ties) if
 * that is >= -1e-10, else outside; candidates from a uniform bucket grid that lists
 * every tet in each bucket its box overlaps, in ascending index. */
static double orient3(const double *p0, const double *p1, const double *p2, const double *p3)
{
    double a0 = p1[0] - p0[0], a1 = p1[1] - p0[1], a2 = p1[2] - p0[2];
    double b0 = p2[0] - p0[0], b1 = p2[1] - p0[1], b2 = p2[2] - p0[2];
    double c0 = p3[0] - p0[0], c1 = p3[1] - p0[1], c2 = p3[2] - p0[2];
    double m0 = b1 * c2 - b2 * c1;
    double m1 = b0 * c2 - b2 * c0;
    double m2 = b0 * c1 - b1 * c0;
    return (a0 * m0 - a1 * m1) + a2 * m2;
}

static double min_bary(const double *xyz, const int32_t *tv, int64_t t, const double *x)
{
    const double *v[4];
    for (int j = 0; j < 4; ++j) v[j] = xyz + 3 * (int64_t)tv[4 * t + j];
    double D = orient3(v[0], v[1], v[2], v[3]);
    double l0 = orient3(x, v[1], v[2], v[3]) / D;
    double l1 = orient3(v[0], x, v[2], v[3]) / D;
    double l2 = orient3(v[0], v[1], x, v[3]) / D;
    double l3 = orient3(v[0], v[1], v[2], x) / D;
    double m = l0;
    if (l1 < m) m = l1;
    if (l2 < m) m = l2;
    if (l3 < m) m = l3;
    return m;
}

static int64_t bucket_of(double c, double lo, double inv, int64_t nb)
{
    double f = floor((c - lo) * inv);
    if (!(f >= 0.0)) return 0;
    if (f >= (double)nb) return nb - 1;
    return (int64_t)f;
}

int64_t omp_locate_tet_bucketed(int64_t nv, const double *xyz, int64_t nt, const int32_t *tv,
                                int64_t n, const double *pos, int32_t *cell, int nb1)
{
    (void)nv;
    double *lo = (double *)malloc((size_t)(3 * nt) * sizeof(double));
    double *hi = (double *)malloc((size_t)(3 * nt) * sizeof(double));
    double glo[3] = {INFINITY, INFINITY, INFINITY}, ghi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t t = 0; t < nt; ++t)
        for (int a = 0; a < 3; ++a) {
            double mn = xyz[3 * (int64_t)tv[4 * t] + a], mx = mn;
            for (int j = 1; j < 4; ++j) {
                double c = xyz[3 * (int64_t)tv[4 * t + j] + a];
                if (c < mn) mn = c;
                if (c > mx) mx = c;
            }
            lo[3 * t + a] = mn;
            hi[3 * t + a] = mx;
            if (mn < glo[a]) glo[a] = mn;
            if (mx > ghi[a]) ghi[a] = mx;
        }
    int64_t nb = nb1 < 1 ? 1 : nb1;
    double inv[3];
    for (int a = 0; a < 3; ++a) inv[a] = ghi[a] > glo[a] ? (double)nb / (ghi[a] - glo[a]) : 0.0;
    int64_t nbk = nb * nb * nb;
    int64_t *start = (int64_t *)calloc((size_t)(nbk + 1), sizeof(int64_t));
    int64_t *fill = NULL, *lists = NULL;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            for (int64_t b = 0; b < nbk; ++b) start[b + 1] += start[b];
            lists = (int64_t *)malloc((size_t)(start[nbk] > 0 ? start[nbk] : 1) * sizeof(int64_t));
            fill = (int64_t *)malloc((size_t)nbk * sizeof(int64_t));
            for (int64_t b = 0; b < nbk; ++b) fill[b] = start[b];
        }
        for (int64_t t = 0; t < nt; ++t) {
            int64_t b0[3], b1[3];
            for (int a = 0; a < 3; ++a) {
                b0[a] = bucket_of(lo[3 * t + a], glo[a], inv[a], nb);
                b1[a] = bucket_of(hi[3 * t + a], glo[a], inv[a], nb);
            }
            for (int64_t k = b0[2]; k <= b1[2]; ++k)
                for (int64_t j = b0[1]; j <= b1[1]; ++j)
                    for (int64_t i = b0[0]; i <= b1[0]; ++i) {
                        int64_t b = (k * nb + j) * nb + i;
                        if (pass == 0)
                            ++start[b + 1];
                        else
                            lists[fill[b]++] = t;
                    }
        }
    }
    free(fill);
    int64_t out = 0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(+ : out)
    for (int64_t i = 0; i < n; ++i) {
        double x[3] = {pos[i], pos[n + i], pos[2 * n + i]};
        int64_t found = -1, best = -1;
        double best_m = -INFINITY;
        int inside = 1;
        for (int a = 0; a < 3; ++a)
            if (!(x[a] >= glo[a] && x[a] <= ghi[a])) inside = 0;
        if (inside) {
            int64_t b = (bucket_of(x[2], glo[2], inv[2], nb) * nb +
                         bucket_of(x[1], glo[1], inv[1], nb)) * nb +
                        bucket_of(x[0], glo[0], inv[0], nb);
            for (int64_t q = start[b]; q < start[b + 1]; ++q) {
                int64_t t = lists[q];
                if (!(x[0] >= lo[3 * t] && x[0] <= hi[3 * t] && x[1] >= lo[3 * t + 1] &&
                      x[1] <= hi[3 * t + 1] && x[2] >= lo[3 * t + 2] && x[2] <= hi[3 * t + 2]))
                    continue;
                double m = min_bary(xyz, tv, t, x);
                if (m >= 0.0) {
                    found = t;
                    break;
                }
                if (m > best_m) {
                    best_m = m;
                    best = t;
                }
            }
        }
        if (found < 0 && best >= 0 && best_m >= -1e-10) found = best;
        cell[i] = (int32_t)found;
        if (found < 0) ++out;
    }
    free(lists);
    free(start);
    free(lo);
    free(hi);
    return out;
}

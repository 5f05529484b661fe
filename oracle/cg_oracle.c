/*
 * cg_oracle.c -- plain, slow, single-threaded FP64 reference of diffusion-based
 * coarse graining (Sun & Xiao, "Diffusion-based coarse graining in hybrid
 * continuum-discrete solvers").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  The CUDA library shares no code,
 * header, table or helper with it, and neither calls the other.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so every
 * floating-point expression rounds exactly as written).
 *
 * What it computes, step by step, in the order the paper gives them:
 *   1. Particle centroid method, Section 2.2 and Section 3.1 Eq. (pcm-k):
 *      each particle's quantity goes to the cell holding its centroid, the cell
 *      sums are divided by the cell volume V_c.
 *   2. Diffusion smoothing, Section 2.6 step 2 and Section 3.2 Eq. (diffusion):
 *      d(eps)/d(tau) = Laplacian(eps) from eps_0 to tau = T, zero-flux walls,
 *      with T = b^2/4 (the bandwidth relation of Section 3.2.1).  The time
 *      discretisation is implicit Euler (primary), Crank-Nicolson (Section 5.1,
 *      the paper's own) or explicit Euler; each implicit step is solved by plain
 *      unpreconditioned conjugate gradients in FP64.
 *   3. The statistical Gaussian kernel of Section 2.5 Eq. (hi) with the image
 *      construction of Section 2.5.2 / Section 3.2.2 Eq. (diffHalf), summed
 *      by brute force (used only to pin the diffusion result).
 *
 * Readings where the paper is silent (each one is restated where it is used):
 *   - cell index: floor((x - x0) / dx) per axis, computed as (x - x0) * (1/dx),
 *     clamped into [0, n-1]; a particle outside the closed box is "out of domain";
 *   - mode-0 deposition sums the particles of a cell in ascending particle index,
 *     starting from +0.0; mode-1 deposition quantises each weight to a 64-bit
 *     integer with a per-field scale 2^F and sums exactly;
 *   - the unstructured operator is the two-point flux finite-volume Laplacian
 *     T_f = |S_f|^2 / (S_f . d_f), with d_f the vector between tet centroids and
 *     the mass matrix M = diag(V_c).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Step 1a: locate on a uniform Cartesian mesh (Section 3.1, host cell of a    */
/* particle centroid).                                                          */
/* ------------------------------------------------------------------------- */

/* Returns the number of particles outside the closed box [x0, x0 + n*dx] (or with
 * a NaN coordinate); their cell is set to -1.  pos is [3][n] (x row, y row, z row).
 * Cells are numbered (iz*ny + iy)*nx + ix. */
int64_t orc_locate_structured(int nx, int ny, int nz, const double *origin, double dx,
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
    for (int64_t i = 0; i < n; ++i) {
        int idx[3];
        int inside = 1;
        for (int a = 0; a < 3; ++a) {
            double x = pos[(int64_t)a * n + i];
            if (!(x >= origin[a] && x <= hi[a])) {   /* NaN fails too */
                inside = 0;
                break;
            }
            double t = (x - origin[a]) * inv_dx;
            double f = floor(t);
            int k = (int)f;
            if (k > dims[a] - 1) k = dims[a] - 1;  /* x == upper wall clamps */
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

/* ------------------------------------------------------------------------- */
/* Step 1b: deposition, Eq. (pcm-k): eps_k = (sum over particles in k of w_i)  */
/* / V_c,k.  Conservation, Eq. (conserve), follows by construction.            */
/* ------------------------------------------------------------------------- */

/* Scale exponent F of the fixed-point mode: with m = max|w| = fm*2^em and
 * n = fn*2^en (frexp), F = 61 - em - en, so that n*m*2^F < 2^61.  F = 0 when
 * m == 0 or n == 0; F is clamped into [-1000, 1000] so that 2^F, 2^-F and every
 * rescaled non-zero sum are normal doubles. */
int orc_fixed_point_bits(int64_t n, double maxabs)
{
    if (n <= 0 || !(maxabs > 0.0)) return 0;
    int em = 0, en = 0;
    (void)frexp(maxabs, &em);
    (void)frexp((double)n, &en);
    int F = 61 - em - en;
    if (F > 1000) F = 1000;
    if (F < -1000) F = -1000;
    return F;
}

/* w is [nf][n]; out is [nf][ncells].  vc == NULL means a uniform cell volume
 * vc_uniform.  Particles with cell < 0 are skipped.
 * mode 0: S = +0.0; S += w_i in ascending i; eps = S / V_c (IEEE division).
 * mode 1: q_i = llrint(w_i * 2^F_f) (round half to even), summed in int64;
 *         eps = ((double)sum * 2^-F_f) / V_c.  fbits[f] holds F_f. */
void orc_deposit(int64_t n, const int32_t *cell, int nf, const double *w,
                 int64_t ncells, const double *vc, double vc_uniform, int mode,
                 const int *fbits, double *out)
{
    for (int f = 0; f < nf; ++f) {
        const double *wf = w + (int64_t)f * n;
        double *of = out + (int64_t)f * ncells;
        if (mode == 0) {
            for (int64_t k = 0; k < ncells; ++k) of[k] = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                if (cell[i] < 0) continue;
                of[cell[i]] = of[cell[i]] + wf[i];
            }
            for (int64_t k = 0; k < ncells; ++k) {
                double v = vc ? vc[k] : vc_uniform;
                of[k] = of[k] / v;
            }
        } else {
            int64_t *acc = (int64_t *)calloc((size_t)ncells, sizeof(int64_t));
            double scale = ldexp(1.0, fbits[f]);
            double unscale = ldexp(1.0, -fbits[f]);
            for (int64_t i = 0; i < n; ++i) {
                if (cell[i] < 0) continue;
                long long q = llrint(wf[i] * scale);
                acc[cell[i]] += (int64_t)q;
            }
            for (int64_t k = 0; k < ncells; ++k) {
                double v = vc ? vc[k] : vc_uniform;
                double s = (double)acc[k] * unscale;
                of[k] = s / v;
            }
            free(acc);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Step 2 on a uniform hex mesh: the 7-point Laplacian with zero-flux walls    */
/* (Section 3.2.2, Neumann condition d(eps)/dn = 0; finite-volume form, Sec.   */
/* 5.1): (L u)_k = sum over existing face neighbours l of (u_l - u_k).  A      */
/* missing neighbour at a wall carries no flux, so it drops out of the sum.    */
/* The physical operator is L / dx^2.                                           */
/* ------------------------------------------------------------------------- */

/* An axis may instead be periodic (Section 3.1: periodic boundaries keep periodic
 * conditions): bit a of per set means the neighbour beyond the last cell along axis a
 * is the first one and the other way round (on an axis of one cell that is the cell
 * itself). */
static int64_t wrap(int64_t i, int64_t n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

static void lap7p(int nx, int ny, int nz, int per, const double *u, double *out)
{
    const int px = per & 1, py = (per >> 1) & 1, pz = (per >> 2) & 1;
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                int64_t k = ((int64_t)iz * ny + iy) * nx + ix;
                double s = 0.0;
                if (ix > 0 || px) s += u[((int64_t)iz * ny + iy) * nx + wrap(ix - 1, nx)] - u[k];
                if (ix < nx - 1 || px) s += u[((int64_t)iz * ny + iy) * nx + wrap(ix + 1, nx)] - u[k];
                if (iy > 0 || py) s += u[((int64_t)iz * ny + wrap(iy - 1, ny)) * nx + ix] - u[k];
                if (iy < ny - 1 || py) s += u[((int64_t)iz * ny + wrap(iy + 1, ny)) * nx + ix] - u[k];
                if (iz > 0 || pz) s += u[(wrap(iz - 1, nz) * ny + iy) * nx + ix] - u[k];
                if (iz < nz - 1 || pz) s += u[(wrap(iz + 1, nz) * ny + iy) * nx + ix] - u[k];
                out[k] = s;
            }
}


/* A u = u - theta * c * L u, with c = dtau / dx^2 and theta = 1 (implicit Euler)
 * or 1/2 (Crank-Nicolson). */
static void apply_implicit(int nx, int ny, int nz, int per, double cth, const double *u,
                           double *tmp, double *out)
{
    int64_t N = (int64_t)nx * ny * nz;
    lap7p(nx, ny, nz, per, u, tmp);
    for (int64_t k = 0; k < N; ++k) out[k] = u[k] - cth * tmp[k];
}

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Plain conjugate gradients on A x = b (A symmetric positive definite), from the
 * given x, until ||r||_2 <= tol * ||b||_2 or max_iter iterations.  Returns the
 * number of iterations, or -1 if it did not converge.  apply(ctx, in, out) is the
 * operator. */
typedef void (*orc_apply_fn)(const void *ctx, const double *in, double *out);

static int cg_solve(int64_t n, orc_apply_fn apply, const void *ctx, const double *b,
                    double *x, double tol, int max_iter)
{
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *p = (double *)malloc((size_t)n * sizeof(double));
    double *Ap = (double *)malloc((size_t)n * sizeof(double));
    apply(ctx, x, Ap);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - Ap[i];
    for (int64_t i = 0; i < n; ++i) p[i] = r[i];
    double bb = dot(n, b, b);
    double rr = dot(n, r, r);
    double thresh = tol * tol * bb;
    int it = 0;
    while (rr > thresh && it < max_iter) {
        apply(ctx, p, Ap);
        double pAp = dot(n, p, Ap);
        if (!(pAp > 0.0)) break;
        double alpha = rr / pAp;
        for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
        for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * Ap[i];
        double rr_new = dot(n, r, r);
        double beta = rr_new / rr;
        rr = rr_new;
        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        ++it;
    }
    int ok = rr <= thresh;
    free(r);
    free(p);
    free(Ap);
    return ok ? it : -1;
}

typedef struct {
    int nx, ny, nz, per;
    double cth;
    double *tmp;
} struct_ctx;

static void struct_apply(const void *vctx, const double *in, double *out)
{
    const struct_ctx *c = (const struct_ctx *)vctx;
    apply_implicit(c->nx, c->ny, c->nz, c->per, c->cth, in, c->tmp, out);
}

/* u is [nf][nx*ny*nz] (intensive field eps, in/out).  T is the pseudo-time,
 * nsteps the number of equal steps dtau = T/nsteps.
 * scheme 0: implicit Euler   (I - c L) u^{n+1} = u^n
 * scheme 1: Crank-Nicolson   (I - c/2 L) u^{n+1} = (I + c/2 L) u^n
 * scheme 2: explicit Euler   u^{n+1} = u^n + c L u^n
 * (all divided through by the uniform cell volume).  Each implicit step starts CG
 * from u^n.  iters_out (may be NULL) receives the total CG iteration count.
 * Returns 0, or -1 if some solve did not converge. */
int orc_diffuse_structured_p(int nx, int ny, int nz, int per, double dx, int nf, double *u,
                             double T, int nsteps, int scheme, double tol, int max_iter,
                             int64_t *iters_out)
{
    int64_t N = (int64_t)nx * ny * nz;
    double dtau = T / (double)nsteps;
    double c = dtau / (dx * dx);
    double *tmp = (double *)malloc((size_t)N * sizeof(double));
    double *rhs = (double *)malloc((size_t)N * sizeof(double));
    double *lu = (double *)malloc((size_t)N * sizeof(double));
    struct_ctx ctx = {nx, ny, nz, per, scheme == 1 ? 0.5 * c : c, tmp};
    int64_t iters = 0;
    int status = 0;
    for (int f = 0; f < nf; ++f) {
        double *uf = u + (int64_t)f * N;
        for (int s = 0; s < nsteps; ++s) {
            if (scheme == 2) {
                lap7p(nx, ny, nz, per, uf, lu);
                for (int64_t k = 0; k < N; ++k) uf[k] = uf[k] + c * lu[k];
                continue;
            }
            if (scheme == 1) {
                lap7p(nx, ny, nz, per, uf, lu);
                for (int64_t k = 0; k < N; ++k) rhs[k] = uf[k] + 0.5 * c * lu[k];
            } else {
                for (int64_t k = 0; k < N; ++k) rhs[k] = uf[k];
            }
            int it = cg_solve(N, struct_apply, &ctx, rhs, uf, tol, max_iter);
            if (it < 0) {
                status = -1;
                it = max_iter;
            }
            iters += it;
        }
    }
    free(tmp);
    free(rhs);
    free(lu);
    if (iters_out) *iters_out = iters;
    return status;
}

/* The zero-flux case (no periodic axis). */
int orc_diffuse_structured(int nx, int ny, int nz, double dx, int nf, double *u,
                           double T, int nsteps, int scheme, double tol, int max_iter,
                           int64_t *iters_out)
{
    return orc_diffuse_structured_p(nx, ny, nz, 0, dx, nf, u, T, nsteps, scheme, tol, max_iter,
                                    iters_out);
}

/* The solid velocity of a cell as the ratio of two smoothed fields: the diffused
 * momentum sum_i V_p,i u_i / V_c and the diffused solid fraction (the momentum, not
 * the velocity, is what is diffused).  Cells whose solid fraction is not above eps_min
 * get 0.  mom is [ncomp][n], out the same. */
void orc_solid_velocity(int64_t n, int ncomp, const double *eps, const double *mom,
                        double eps_min, double *out)
{
    for (int c = 0; c < ncomp; ++c)
        for (int64_t k = 0; k < n; ++k)
            out[(int64_t)c * n + k] = eps[k] > eps_min ? mom[(int64_t)c * n + k] / eps[k] : 0.0;
}

/* ------------------------------------------------------------------------- */
/* Step 2 on an unstructured tetrahedral mesh: cell-centred finite volumes     */
/* with a two-point flux, (L u)_k = sum over faces f of T_f (u_l - u_k),       */
/* T_f = |S_f|^2 / (S_f . d_f), S_f the face area vector pointing out of k,    */
/* d_f = c_l - c_k between tet centroids (vertex means).  Boundary faces carry */
/* no flux (zero-flux walls).  M = diag(V_c).                                  */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t v[3];   /* sorted vertex ids */
    int32_t tet;
    int32_t local;  /* opposite vertex slot 0..3 */
} face_rec;

static int face_cmp(const void *pa, const void *pb)
{
    const face_rec *a = (const face_rec *)pa, *b = (const face_rec *)pb;
    for (int i = 0; i < 3; ++i) {
        if (a->v[i] < b->v[i]) return -1;
        if (a->v[i] > b->v[i]) return 1;
    }
    if (a->tet != b->tet) return a->tet < b->tet ? -1 : 1;
    return 0;
}

static void sort3(int32_t *v)
{
    int32_t t;
    if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
    if (v[1] > v[2]) { t = v[1]; v[1] = v[2]; v[2] = t; }
    if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
}

typedef struct {
    int32_t col;
    double val;
} entry;

static int entry_cmp(const void *pa, const void *pb)
{
    const entry *a = (const entry *)pa, *b = (const entry *)pb;
    return (a->col > b->col) - (a->col < b->col);
}

/* Builds the cell volumes, centroids and the CSR matrix of L (diagonal included,
 * columns ascending per row).  rowptr has nt+1 entries, col/val room for
 * 5*nt entries.  Returns nnz >= 0, or
 *   -1 a face shared by more than two tets,  -2 a zero-volume tet,
 *   -3 a non-positive or non-finite transmissibility,  -4 a vertex id out of range. */
int64_t orc_tet_build(int64_t nv, const double *xyz, int64_t nt, const int32_t *tv,
                      double *vc, double *cent, int64_t *rowptr, int32_t *col, double *val)
{
    if (nt <= 0) {
        rowptr[0] = 0;
        return 0;
    }
    for (int64_t t = 0; t < nt; ++t)
        for (int j = 0; j < 4; ++j)
            if (tv[4 * t + j] < 0 || tv[4 * t + j] >= nv) return -4;
    for (int64_t t = 0; t < nt; ++t) {
        const double *p[4];
        for (int j = 0; j < 4; ++j) p[j] = xyz + 3 * (int64_t)tv[4 * t + j];
        for (int a = 0; a < 3; ++a)
            cent[3 * t + a] = (((p[0][a] + p[1][a]) + p[2][a]) + p[3][a]) * 0.25;
        double e1[3], e2[3], e3[3];
        for (int a = 0; a < 3; ++a) {
            e1[a] = p[1][a] - p[0][a];
            e2[a] = p[2][a] - p[0][a];
            e3[a] = p[3][a] - p[0][a];
        }
        double det = e1[0] * (e2[1] * e3[2] - e2[2] * e3[1])
                   - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0])
                   + e1[2] * (e2[0] * e3[1] - e2[1] * e3[0]);
        double v = fabs(det) / 6.0;
        if (!(v > 0.0)) return -2;
        vc[t] = v;
    }
    face_rec *faces = (face_rec *)malloc((size_t)(4 * nt) * sizeof(face_rec));
    for (int64_t t = 0; t < nt; ++t)
        for (int j = 0; j < 4; ++j) {
            face_rec *fr = &faces[4 * t + j];
            int m = 0;
            for (int q = 0; q < 4; ++q)
                if (q != j) fr->v[m++] = tv[4 * t + q];
            sort3(fr->v);
            fr->tet = (int32_t)t;
            fr->local = j;
        }
    qsort(faces, (size_t)(4 * nt), sizeof(face_rec), face_cmp);

    /* per-tet neighbour list (at most 4) */
    int32_t *nb = (int32_t *)malloc((size_t)(4 * nt) * sizeof(int32_t));
    double *tf = (double *)malloc((size_t)(4 * nt) * sizeof(double));
    int *cnt = (int *)calloc((size_t)nt, sizeof(int));
    int64_t status = 0;
    for (int64_t i = 0; i < 4 * nt;) {
        int64_t j = i + 1;
        while (j < 4 * nt && faces[j].v[0] == faces[i].v[0] && faces[j].v[1] == faces[i].v[1] &&
               faces[j].v[2] == faces[i].v[2])
            ++j;
        if (j - i > 2) { status = -1; break; }
        if (j - i == 2) {
            int32_t k = faces[i].tet, l = faces[i + 1].tet;
            const double *a = xyz + 3 * (int64_t)faces[i].v[0];
            const double *b = xyz + 3 * (int64_t)faces[i].v[1];
            const double *c = xyz + 3 * (int64_t)faces[i].v[2];
            double ab[3], ac[3], S[3], fc[3], d[3];
            for (int q = 0; q < 3; ++q) {
                ab[q] = b[q] - a[q];
                ac[q] = c[q] - a[q];
            }
            S[0] = 0.5 * (ab[1] * ac[2] - ab[2] * ac[1]);
            S[1] = 0.5 * (ab[2] * ac[0] - ab[0] * ac[2]);
            S[2] = 0.5 * (ab[0] * ac[1] - ab[1] * ac[0]);
            /* orient S out of cell k: towards the face centroid from c_k */
            double so = 0.0;
            for (int q = 0; q < 3; ++q) {
                fc[q] = ((a[q] + b[q]) + c[q]) / 3.0;
                so += S[q] * (fc[q] - cent[3 * (int64_t)k + q]);
            }
            if (so < 0.0)
                for (int q = 0; q < 3; ++q) S[q] = -S[q];
            for (int q = 0; q < 3; ++q) d[q] = cent[3 * (int64_t)l + q] - cent[3 * (int64_t)k + q];
            double ss = S[0] * S[0] + S[1] * S[1] + S[2] * S[2];
            double sd = S[0] * d[0] + S[1] * d[1] + S[2] * d[2];
            double T = ss / sd;
            if (!(T > 0.0) || !isfinite(T)) { status = -3; break; }
            nb[4 * (int64_t)k + cnt[k]] = l;
            tf[4 * (int64_t)k + cnt[k]] = T;
            cnt[k]++;
            nb[4 * (int64_t)l + cnt[l]] = k;
            tf[4 * (int64_t)l + cnt[l]] = T;
            cnt[l]++;
        }
        i = j;
    }
    if (status == 0) {
        int64_t pos = 0;
        for (int64_t t = 0; t < nt; ++t) {
            entry e[5];
            int m = 0;
            double diag = 0.0;
            for (int q = 0; q < cnt[t]; ++q) {
                e[m].col = nb[4 * t + q];
                e[m].val = tf[4 * t + q];
                diag -= tf[4 * t + q];
                ++m;
            }
            e[m].col = (int32_t)t;
            e[m].val = diag;
            ++m;
            qsort(e, (size_t)m, sizeof(entry), entry_cmp);
            rowptr[t] = pos;
            for (int q = 0; q < m; ++q) {
                col[pos] = e[q].col;
                val[pos] = e[q].val;
                ++pos;
            }
        }
        rowptr[nt] = pos;
        status = pos;
    }
    free(faces);
    free(nb);
    free(tf);
    free(cnt);
    return status;
}

typedef struct {
    int64_t n;
    const double *vc;
    const int64_t *rowptr;
    const int32_t *col;
    const double *val;
    double theta_dtau;
} csr_ctx;

/* out = L u (CSR) */
static void csr_lap(const csr_ctx *c, const double *u, double *out)
{
    for (int64_t k = 0; k < c->n; ++k) {
        double s = 0.0;
        for (int64_t e = c->rowptr[k]; e < c->rowptr[k + 1]; ++e) s += c->val[e] * u[c->col[e]];
        out[k] = s;
    }
}

/* out = (M - theta*dtau*L) u */
static void csr_apply(const void *vctx, const double *in, double *out)
{
    const csr_ctx *c = (const csr_ctx *)vctx;
    csr_lap(c, in, out);
    for (int64_t k = 0; k < c->n; ++k) out[k] = c->vc[k] * in[k] - c->theta_dtau * out[k];
}

/* Diffusion on a general cell-centred mesh given M = diag(vc) and L (CSR).
 * u is [nf][n], the intensive field, in/out.  Schemes as in the structured case:
 * 0: (M - dtau L) u^{n+1} = M u^n,  1: (M - dtau/2 L) u^{n+1} = (M + dtau/2 L) u^n,
 * 2: u^{n+1} = u^n + dtau M^{-1} L u^n.  Returns 0, or -1 on non-convergence. */
int orc_diffuse_csr(int64_t n, const double *vc, const int64_t *rowptr, const int32_t *col,
                    const double *val, int nf, double *u, double T, int nsteps, int scheme,
                    double tol, int max_iter, int64_t *iters_out)
{
    double dtau = T / (double)nsteps;
    csr_ctx ctx = {n, vc, rowptr, col, val, scheme == 1 ? 0.5 * dtau : dtau};
    double *rhs = (double *)malloc((size_t)n * sizeof(double));
    double *lu = (double *)malloc((size_t)n * sizeof(double));
    int64_t iters = 0;
    int status = 0;
    for (int f = 0; f < nf; ++f) {
        double *uf = u + (int64_t)f * n;
        for (int s = 0; s < nsteps; ++s) {
            if (scheme == 2) {
                csr_lap(&ctx, uf, lu);
                for (int64_t k = 0; k < n; ++k) uf[k] = uf[k] + dtau * lu[k] / vc[k];
                continue;
            }
            if (scheme == 1) {
                csr_lap(&ctx, uf, lu);
                for (int64_t k = 0; k < n; ++k) rhs[k] = vc[k] * uf[k] + 0.5 * dtau * lu[k];
            } else {
                for (int64_t k = 0; k < n; ++k) rhs[k] = vc[k] * uf[k];
            }
            int it = cg_solve(n, csr_apply, &ctx, rhs, uf, tol, max_iter);
            if (it < 0) {
                status = -1;
                it = max_iter;
            }
            iters += it;
        }
    }
    free(rhs);
    free(lu);
    if (iters_out) *iters_out = iters;
    return status;
}

/* ------------------------------------------------------------------------- */
/* Step 1a on a tetrahedral mesh: the host tet of a particle centroid.         */
/* orient(p0,p1,p2,p3) = det[p1-p0; p2-p0; p3-p0] by cofactor expansion along  */
/* the first row, evaluated exactly in the order written.  For tet (v0..v3)    */
/* with D = orient(v0,v1,v2,v3), the barycentric coordinate of x opposite v_j  */
/* is lambda_j = orient(tet with v_j replaced by x) / D.                        */
/* Rule: the lowest-index tet whose axis-aligned box holds x and whose four    */
/* lambda_j are all >= 0.  If there is none (x falls in a rounding gap on a    */
/* face), the tet among those whose box holds x with the largest min_j lambda_j */
/* (lowest index on ties), provided that value is >= -1e-10; else out of domain. */
/* ------------------------------------------------------------------------- */

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

/* Minimum barycentric coordinate of x in tet t (see the rule above). */
double orc_tet_min_bary(const double *xyz, const int32_t *tv, int64_t t, const double *x)
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

int64_t orc_locate_tet(int64_t nv, const double *xyz, int64_t nt, const int32_t *tv, int64_t n,
                       const double *pos, int32_t *cell)
{
    (void)nv;
    double *lo = (double *)malloc((size_t)(3 * nt) * sizeof(double));
    double *hi = (double *)malloc((size_t)(3 * nt) * sizeof(double));
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
        }
    int64_t out = 0;
    for (int64_t i = 0; i < n; ++i) {
        double x[3] = {pos[i], pos[n + i], pos[2 * n + i]};
        int64_t found = -1, best = -1;
        double best_m = -INFINITY;
        for (int64_t t = 0; t < nt; ++t) {
            if (!(x[0] >= lo[3 * t] && x[0] <= hi[3 * t] && x[1] >= lo[3 * t + 1] &&
                  x[1] <= hi[3 * t + 1] && x[2] >= lo[3 * t + 2] && x[2] <= hi[3 * t + 2]))
                continue;
            double m = orc_tet_min_bary(xyz, tv, t, x);
            if (m >= 0.0) {
                found = t;
                break;
            }
            if (m > best_m) {
                best_m = m;
                best = t;
            }
        }
        if (found < 0 && best >= 0 && best_m >= -1e-10) found = best;
        cell[i] = (int32_t)found;
        if (found < 0) ++out;
    }
    free(lo);
    free(hi);
    return out;
}

/* The same rule, for large meshes: the candidates of a point are the tets whose  */
/* axis-aligned box holds it, and only those; a uniform grid of buckets over the   */
/* mesh's box lists each tet in every bucket its box overlaps, in ascending index. */
/* The bucket of a coordinate, clamp(floor((c - lo) * inv), 0, nb - 1), does not   */
/* decrease as c grows, so a tet whose box [lo_t, hi_t] holds x is listed in x's   */
/* bucket; scanning that bucket in ascending index with the box test meets exactly */
/* the candidates orc_locate_tet meets, in the same order, and gives the same      */
/* result.  A point outside the mesh's box has no candidate.                       */
static int64_t bucket_of(double c, double lo, double inv, int64_t nb)
{
    double f = floor((c - lo) * inv);
    if (!(f >= 0.0)) return 0;          /* also NaN: such points fail the box test */
    if (f >= (double)nb) return nb - 1;
    return (int64_t)f;
}

int64_t orc_locate_tet_bucketed(int64_t nv, const double *xyz, int64_t nt, const int32_t *tv,
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
    for (int a = 0; a < 3; ++a)
        inv[a] = ghi[a] > glo[a] ? (double)nb / (ghi[a] - glo[a]) : 0.0;
    int64_t nbk = nb * nb * nb;
    /* pass 0 counts the tets each bucket lists, pass 1 writes the lists; tets are
     * visited in ascending index, so every list is ascending */
    int64_t *start = (int64_t *)calloc((size_t)(nbk + 1), sizeof(int64_t));
    int64_t *fill = NULL;
    int64_t *lists = NULL;
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
                double m = orc_tet_min_bary(xyz, tv, t, x);
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

/* ------------------------------------------------------------------------- */
/* The Gaussian kernel of Eq. (hi) with bandwidth b (equivalently the Green's  */
/* function of Eq. (solutionGi) at T = b^2/4), summed with images about the    */
/* six walls of the box [0,L0]x[0,L1]x[0,L2] (Eq. (hi-bound), Eq. (diffHalf),  */
/* extended to corners by reflecting per axis).  Per axis the image positions  */
/* are 2mL + s and 2mL - s for m = -mmax..mmax.                                */
/* out[k] = sum_i w_i * sum_images h(xe_k - image(xs_i)).                        */
/* ------------------------------------------------------------------------- */

static double image_sum_1d(double x, double s, double L, double b, int mmax)
{
    double acc = 0.0;
    double norm = 1.0 / (b * sqrt(M_PI));
    for (int m = -mmax; m <= mmax; ++m) {
        double i1 = 2.0 * m * L + s;
        double i2 = 2.0 * m * L - s;
        acc += norm * exp(-(x - i1) * (x - i1) / (b * b));
        acc += norm * exp(-(x - i2) * (x - i2) / (b * b));
    }
    return acc;
}

void orc_kernel_sum(int64_t ns, const double *src /*[ns][3]*/, const double *w, int64_t ne,
                    const double *ev /*[ne][3]*/, const double *L, double b, int mmax, double *out)
{
    for (int64_t k = 0; k < ne; ++k) {
        double s = 0.0;
        for (int64_t i = 0; i < ns; ++i) {
            double g = 1.0;
            for (int a = 0; a < 3; ++a)
                g *= image_sum_1d(ev[3 * k + a], src[3 * i + a], L[a], b, mmax);
            s += w[i] * g;
        }
        out[k] = s;
    }
}

/* ------------------------------------------------------------------------- */
/* A stretched Cartesian mesh with a spatially varying diffusion constant      */
/* (stretched meshes: Section 4.4; a local diffusion constant that can fall    */
/* to zero to degenerate to PCM there, with conservation kept: Section 5.2).   */
/* Cell (ix, iy, iz), k = (iz ny + iy) nx + ix, spans [xf[ix], xf[ix+1]] x ... */
/* Finite volumes with a two-point flux: across the face between cells a and b  */
/* T_f = D_f |A_f| / d_f, |A_f| the face area, d_f the distance between the     */
/* two cell centres, D_f = 2 D_a D_b / (D_a + D_b) (harmonic mean, 0 if either  */
/* is 0); walls carry no flux.  (L u)_k = sum_f T_f (u_l - u_k), M = diag(V_c),  */
/* the same CSR layout as orc_tet_build (diagonal entry first in each row).     */
/* ------------------------------------------------------------------------- */

static double face_d(double da, double db)
{
    return (da > 0.0 && db > 0.0) ? 2.0 * da * db / (da + db) : 0.0;
}

int64_t orc_hex_build(int nx, int ny, int nz, const double *xf, const double *yf,
                      const double *zf, const double *D, double *vc, int64_t *rowptr,
                      int32_t *col, double *val)
{
    const int n3[3] = {nx, ny, nz};
    const double *f[3] = {xf, yf, zf};
    int64_t nnz = 0;
    rowptr[0] = 0;
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                const int64_t k = ((int64_t)iz * ny + iy) * nx + ix;
                const int id[3] = {ix, iy, iz};
                double w[3], c[3];
                for (int a = 0; a < 3; ++a) {
                    w[a] = f[a][id[a] + 1] - f[a][id[a]];
                    c[a] = 0.5 * (f[a][id[a]] + f[a][id[a] + 1]);
                }
                vc[k] = w[0] * w[1] * w[2];
                const double dk = D ? D[k] : 1.0;
                const int64_t dstart = nnz++;   /* diagonal first */
                col[dstart] = (int32_t)k;
                double diag = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int s = -1; s <= 1; s += 2) {
                        const int j = id[a] + s;
                        if (j < 0 || j >= n3[a]) continue;
                        int nid[3] = {ix, iy, iz};
                        nid[a] = j;
                        const int64_t l = ((int64_t)nid[2] * ny + nid[1]) * nx + nid[0];
                        const double cl = 0.5 * (f[a][j] + f[a][j + 1]);
                        const double area = w[(a + 1) % 3] * w[(a + 2) % 3];
                        const double t = face_d(dk, D ? D[l] : 1.0) * area / fabs(cl - c[a]);
                        col[nnz] = (int32_t)l;
                        val[nnz] = t;
                        ++nnz;
                        diag -= t;
                    }
                val[dstart] = diag;
                rowptr[k + 1] = nnz;
            }
    return nnz;
}

/* Cell of each point on the stretched mesh: per axis the i with f[i] <= x < f[i+1]
 * (x = f[n] is in the last cell); outside the closed box or NaN gives -1.  Returns
 * the number outside. */
int64_t orc_locate_hex(int nx, int ny, int nz, const double *xf, const double *yf,
                       const double *zf, int64_t n, const double *pos, int32_t *cell)
{
    const int n3[3] = {nx, ny, nz};
    const double *f[3] = {xf, yf, zf};
    int64_t nout = 0;
    for (int64_t p = 0; p < n; ++p) {
        int id[3];
        int ok = 1;
        for (int a = 0; a < 3 && ok; ++a) {
            const double x = pos[(int64_t)a * n + p];
            if (!(x >= f[a][0] && x <= f[a][n3[a]])) {
                ok = 0;
                break;
            }
            int i = 0;   /* the last face not above x, by a linear scan */
            while (i + 1 < n3[a] && f[a][i + 1] <= x) ++i;
            id[a] = i;
        }
        if (!ok) {
            cell[p] = -1;
            ++nout;
        } else {
            cell[p] = (int32_t)(((int64_t)id[2] * ny + id[1]) * nx + id[0]);
        }
    }
    return nout;
}

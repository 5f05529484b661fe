/*
 * cg.h -- C ABI of the GB300 (sm_103a) library for diffusion-based coarse graining
 * (Sun & Xiao, "Diffusion-Based Coarse Graining in Hybrid Continuum-Discrete
 * Solvers").
 *
 * The method (Section 2.6): (1) deposit every particle's quantity into the mesh cell
 * holding its centroid and divide by the cell volume (particle centroid method,
 * Section 2.2, Section 3.1 Eq. (pcm-k)); (2) smooth the deposited field by
 * integrating the diffusion equation d(eps)/d(tau) = Laplacian(eps) (Section 3.2.1
 * Eq. (diffusion)) over pseudo-time T = b^2/4 (b the equivalent Gaussian kernel
 * bandwidth, Section 3.2.1) with zero-flux walls (Section 3.2.2).
 *
 * Conventions for every entry point:
 *  - Array arguments are CALLER-OWNED DEVICE memory unless the name ends in _host.
 *    Mesh-construction inputs are host memory and are copied.
 *  - The library owns the mesh and its workspace (allocated on first use, grown as
 *    needed, freed by cg_destroy_mesh).  Calls that use the same mesh must not run
 *    concurrently.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    enqueued on it, and every call synchronises that stream before it returns
 *    (the status depends on device results), so outputs are complete on return.
 *  - Every function returns a cg_status and never aborts.  Validation runs before
 *    any output is written: on an error status the output arrays are untouched,
 *    except CG_ENOCONV / CG_ETIMEOUT, which leave the last iterate in place.
 *  - FP64 particle positions are SoA: pos[0..n) = x, pos[n..2n) = y, pos[2n..3n) = z.
 *    Carried quantities are field-major: w[f*n + i].  Cell fields are field-major:
 *    cells[f*ncells + k].  Weights are extensive (V_p, V_p*u, F_d); cell fields are
 *    intensive (per unit cell volume), as in Eq. (pcm-k).
 *  - Structured cells are numbered k = (iz*ny + iy)*nx + ix.
 */
#ifndef CG_H
#define CG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CG_OK = 0,
    CG_EINVAL = 1,    /* bad argument, size, pointer, non-finite input, invalid mesh */
    CG_ENOMEM = 2,    /* device or host allocation failed */
    CG_ECUDA = 3,     /* a CUDA runtime call failed (see cg_last_error) */
    CG_ENOCONV = 4,   /* an implicit step did not reach params.tol within the limits */
    CG_ETIMEOUT = 5,  /* a bounded device-side wait gave up (persistent, resident or
                         TMA-staged kernels) */
    CG_EDOMAIN = 6    /* particles outside the mesh; report->n_out_of_domain has the count */
} cg_status;

/* Human-readable name of a status code (static string). */
const char *cg_status_string(cg_status s);

/* Detail of the last error raised in the calling thread (static per-thread buffer). */
const char *cg_last_error(void);

/* ------------------------------------------------------------------------ meshes */

typedef struct cg_mesh cg_mesh; /* opaque, library-owned */

/* Uniform Cartesian hex mesh of nx*ny*nz cubic cells of edge dx with lower corner
 * origin[3] (host).  The paper's structured tests use such meshes (Section 4,
 * Table (apriori-indep)).  Requires nx, ny, nz >= 1, nx*ny*nz < 2^31, dx > 0 finite.
 * Errors: CG_EINVAL, CG_ENOMEM, CG_ECUDA. */
cg_status cg_create_mesh_structured(int nx, int ny, int nz, const double origin[3], double dx,
                                    cg_mesh **out);

/* Unstructured tetrahedral mesh (Section 4.3 uses unstructured cells; this library
 * takes tetrahedra).  xyz_host is [nverts][3] FP64, tv_host is [ntets][4] int32 vertex ids
 * (either orientation).  The library derives cell volumes V_c, centroids (vertex
 * means), faces, and the two-point-flux finite-volume Laplacian
 * T_f = |S_f|^2 / (S_f . d_f) between face neighbours (S_f the face area vector out
 * of the first cell, d_f the centroid-to-centroid vector), M = diag(V_c); boundary
 * faces carry no flux.  Also builds the point-location buckets and each tet's box and
 * FP32 edge vectors for the inside test (device memory held until cg_destroy_mesh).
 * Errors: CG_EINVAL (vertex id out of range, a face shared by more than two tets, a
 * zero-volume tet, a non-positive transmissibility), CG_ENOMEM, CG_ECUDA. */
cg_status cg_create_mesh_tet(int64_t nverts, const double *xyz_host, int64_t ntets,
                             const int32_t *tv_host, cg_mesh **out);

cg_status cg_destroy_mesh(cg_mesh *mesh);

/* Number of cells (structured: nx*ny*nz; tet: ntets); -1 for NULL. */
int64_t cg_mesh_num_cells(const cg_mesh *mesh);

/* Copies the cell volumes V_c into out_host[ncells] (FP64). */
cg_status cg_mesh_cell_volumes(const cg_mesh *mesh, double *out_host);

/* Periodic axes of a structured mesh (Section 3.1: a periodic boundary keeps a
 * periodic condition instead of zero flux).  px, py, pz nonzero make the faces at the
 * two ends of the mesh along x, y, z neighbours of each other (on an axis of one cell,
 * of the cell itself); all zero restores the walls.  Deposition is unchanged.  With a
 * periodic axis the diffusion uses the z-marching or the vectorised sweeps and the
 * one-cell-per-thread refinement (two cells per thread when only x is periodic and nx is
 * even) (params->sweep_shape must be 0, negative or 100 + z),
 * and batched calls reject the mesh.  Drops the mesh's captured schedules and tuned shapes.  Errors: CG_EINVAL (NULL
 * or a tet mesh). */
cg_status cg_mesh_set_periodic(cg_mesh *mesh, int px, int py, int pz);

/* Stretched Cartesian mesh with a spatially varying diffusion constant (stretched
 * meshes: Section 4.4; a local diffusion constant that may be set very small, down to
 * 0, to degenerate to PCM there with conservation kept: Section 5.2).  Cell
 * (ix, iy, iz), k = (iz ny + iy) nx + ix, spans [xf[ix], xf[ix+1]] x [yf[iy], yf[iy+1]]
 * x [zf[iz], zf[iz+1]] (host arrays of nx+1, ny+1, nz+1 strictly increasing face
 * coordinates); diffusivity (host [ncells], may be NULL for 1) is the cell's D >= 0.
 * The operator is the two-point-flux finite-volume Laplacian T_f = D_f |A_f| / d_f
 * between face neighbours (|A_f| the face area, d_f the distance between the cell
 * centres, D_f the harmonic mean of the two cells' D, 0 if either is 0), M = diag(V_c),
 * zero-flux walls; it is solved like the tet operator (cg_diffuse on this mesh uses
 * the same solvers and precision modes).  A point is in the cell whose half-open face
 * interval holds it on every axis (the upper boundary face belongs to the last cell).
 * Errors: CG_EINVAL (NULL, dimensions, non-increasing or non-finite faces, a negative
 * or non-finite D), CG_ENOMEM, CG_ECUDA. */
cg_status cg_create_mesh_hex(int nx, int ny, int nz, const double *xf, const double *yf,
                             const double *zf, const double *diffusivity, cg_mesh **out);

/* Copies the mesh's Laplacian (tet or stretched hex mesh) in CSR form to host arrays:
 * rowptr_host[ncells+1], col_host[nnz], val_host[nnz] (ascending columns, diagonal
 * included); *nnz_out receives nnz.  Pass NULL arrays to query nnz only.  CG_EINVAL
 * for a uniform structured mesh. */
cg_status cg_mesh_tet_operator(const cg_mesh *mesh, int64_t *rowptr_host, int32_t *col_host,
                               double *val_host, int64_t *nnz_out);

/* ------------------------------------------------------------------------ parameters */

enum { CG_SCHEME_IMPLICIT_EULER = 0, CG_SCHEME_CRANK_NICOLSON = 1, CG_SCHEME_EXPLICIT_EULER = 2 };
enum {
    CG_PREC_FP64 = 0,           /* FP64 conjugate gradients */
    CG_PREC_FP32_REFINE = 1,    /* FP32 inner solves, IEEE-FP64 iterative refinement */
    CG_PREC_BF16_REFINE = 2,    /* BF16-stored inner solves, IEEE-FP64 refinement */
    CG_PREC_FP32_DF_REFINE = 3, /* FP32 inner solves, double-float refinement (the iterate
                                   and residual as FP32 hi+lo pairs, ~48-bit significand;
                                   hex meshes; field values must lie in FP32 range) */
    CG_PREC_BF16_DF_REFINE = 4  /* BF16-stored inner solves, double-float refinement */
};
enum { CG_DEPOSIT_ORDERED = 0, CG_DEPOSIT_FIXED_POINT = 1 };

typedef struct {
    double bandwidth;   /* b; T = b^2/4 (Section 3.2.1).  If <= 0, T below is used. */
    double T;           /* pseudo-time span (used when bandwidth <= 0) */
    int nsteps;         /* number of equal pseudo-steps, dtau = T/nsteps (Section 5.1) */
    int scheme;         /* CG_SCHEME_*: implicit Euler (default), Crank-Nicolson (the
                           paper's choice, Section 5.1), explicit Euler */
    int precision;      /* CG_PREC_*: FP64 conjugate gradients; FP32 (or BF16-stored)
                           inner solves with FP64 or double-float iterative refinement
                           (tet meshes run modes 3 and 4 as 1 and 2) */
    int deposit_mode;   /* CG_DEPOSIT_ORDERED: FP64 sum per cell in ascending particle
                           index; CG_DEPOSIT_FIXED_POINT: exact 64-bit integer sum of
                           w * 2^F (F per field, see cg_report.fixed_point_bits) */
    double tol;         /* per implicit step: stop when ||b - A x||_2 <= tol ||b||_2
                           (FP64 residual); default 1e-13 */
    int max_iter;       /* FP64 CG: iteration cap per step; mixed: inner iteration cap */
    int max_rounds;     /* mixed: refinement-round cap per step (default 12) */
    int fused_k;        /* explicit Euler on a uniform structured mesh only: 1..4 runs
                           the steps in FP32 storage and arithmetic, fused_k steps per
                           launch (temporal blocking; the precision field is then not
                           used; results do not depend on fused_k); rounding grows with
                           the step count (about 2-7e-7 max-relative after 40 steps).
                           0 (default): FP64 or double-float steps per precision.  Other
                           schemes need 0 (else CG_EINVAL) */
    int sweep_shape;    /* hex Chebyshev sweep shape: 0 = autotuned per mesh (default);
                           100 + z = vectorised, 4 x-cells per thread, z planes per block
                           (needs nx % 4 == 0); 2, 4, 8 = register-blocked planes per
                           block; -z = z-marching, z planes per block; 200 + z = two
                           iterations per launch (temporal blocking), z planes per block
                           (nx % 4 == 0, nx <= 512, no periodic axis but x; the same
                           results as 100 + z; the autotuner also weighs it on rows over
                           128 cells); 300 = resident:
                           each round's inner solve in one cooperative launch that keeps
                           the mesh in the SMs' shared memory (one field, nx % 4 == 0, a
                           mesh that fits; the autotuner also weighs it); 400 + z =
                           TMA-staged vectorised sweep, z planes per block (FP32 inner
                           storage, nx % 4 == 0, no periodic axis; same results as
                           100 + z).  Batched calls: z = the persistent launch with
                           z planes per work item, 500 + z = one launch per phase with z
                           planes per work item (same results); 0 = autotuned per batch
                           shape (both schedules; only the persistent one when
                           barrier_budget > 0).  Tet
                           and stretched meshes, FP32 storage: 0 = Chebyshev inner
                           solves on an interval from a probe PCG solve on a fixed
                           right-hand side (kept per mesh and pseudo-step, so results do
                           not depend on earlier calls), 1 = Jacobi-PCG throughout (BF16
                           storage: always PCG) */
    long long barrier_budget; /* > 0: run each structured inner solve as one persistent
                                 cooperative launch whose grid barriers give up after this
                                 many clock cycles of waiting (then CG_ETIMEOUT); with
                                 sweep_shape 300 it bounds the resident solve's waits
                                 instead (default about one second); 0: one launch per
                                 inner iteration (default) */
} cg_params;

/* Fills the defaults: bandwidth 0, T 0, nsteps 10, implicit Euler, FP64, ordered
 * deposition, tol 1e-13, max_iter 10000, max_rounds 12, fused_k 0, barrier_budget 0. */
void cg_params_default(cg_params *p);

#define CG_REPORT_MAX_FIELDS 8

typedef struct {
    double ms_locate, ms_deposit, ms_diffuse;   /* device time per phase (CUDA events) */
    long long iters;          /* total operator applications per field, summed over fields */
    long long refine_rounds;  /* mixed precision: refinement rounds, summed over steps */
    long long cell_updates;   /* operator applications x cells, all fields (the metric unit) */
    double final_rel_residual;/* max over steps and fields of ||b - A x||_2 / ||b||_2 */
    double mass_in[CG_REPORT_MAX_FIELDS];   /* sum_k V_c,k eps_k before smoothing */
    double mass_out[CG_REPORT_MAX_FIELDS];  /* ... after smoothing (Eq. (conserve)) */
    long long n_out_of_domain;
    int fixed_point_bits[CG_REPORT_MAX_FIELDS];
    int inner_iters_per_round;/* mixed: Chebyshev iterations per refinement round */
    int sweep_shape_used;     /* mixed hex: the sweep shape (or batched z planes) that ran */
} cg_report;

/* ------------------------------------------------------------------------ the path */

/* Step 1a (Section 2.2, Section 3.1): host cell of each particle centroid.
 * pos: device [3][n] FP64.  cell_out: device [n] int32, -1 for a particle outside
 * the mesh.  Structured: per axis i = floor((x - x0) * (1/dx)) clamped into
 * [0, n-1]; a particle is outside unless x0 <= x <= x0 + n*dx on every axis (a NaN
 * is outside).  Tet: the lowest-index tet whose bounding box holds x and whose four
 * barycentric coordinates (signed-volume ratios) are all >= 0; if none, the tet
 * with the largest minimum barycentric coordinate (lowest index on ties) when that
 * value is >= -1e-10; else outside.  The result does not depend on the particles'
 * order (sets of 65,536 or more are searched grouped by location bucket, in a
 * workspace kept with the mesh).  *n_out_host receives the outside count.
 * Errors: CG_EINVAL, CG_ENOMEM, CG_ECUDA. */
cg_status cg_locate(cg_mesh *mesh, int64_t n, const double *pos, int32_t *cell_out,
                    int64_t *n_out_host, void *stream);

/* Step 1 (Section 3.1 Eq. (pcm-k)): eps_k,f = (sum over particles i in cell k of
 * w_f,i) / V_c,k for nfields fields.  pos: device [3][n]; w: device [nfields][n];
 * cells_out: device [nfields][ncells] FP64.  params->deposit_mode selects the
 * ordered FP64 sum (bit-identical to a sequential loop over particles) or the
 * 64-bit fixed-point sum.  report may be NULL.
 * Errors: CG_EINVAL (sizes, NULL pointers, non-finite weights), CG_EDOMAIN
 * (particles outside the mesh; nothing written), CG_ENOMEM, CG_ECUDA. */
cg_status cg_deposit(cg_mesh *mesh, int64_t n, const double *pos, int nfields, const double *w,
                     double *cells_out, const cg_params *params, cg_report *report, void *stream);

/* Step 2 (Section 2.6 step 2, Section 3.2): smooth nfields cell fields in place by
 * params->nsteps steps of the chosen scheme of Eq. (diffusion) to T, zero-flux walls.
 * Implicit Euler solves (M - dtau L) u^{n+1} = M u^n per step, Crank-Nicolson
 * (M - dtau/2 L) u^{n+1} = (M + dtau/2 L) u^n, explicit Euler u += dtau M^{-1} L u
 * (requires dtau <= dx^2/6 on hex meshes; with precision 3 or 4 on a hex mesh of even
 * nx its steps run in double-float arithmetic, else in FP64).  cells: device
 * [nfields][ncells] FP64.
 * Errors: CG_EINVAL, CG_ENOCONV (report->final_rel_residual says how far it got),
 * CG_ENOMEM, CG_ECUDA. */
cg_status cg_diffuse(cg_mesh *mesh, int nfields, double *cells, const cg_params *params,
                     cg_report *report, void *stream);

/* cg_deposit followed by cg_diffuse (Section 2.6): the whole method.  An error in the
 * deposition phase leaves cells_out untouched; an error in the diffusion phase
 * (CG_ENOMEM, CG_ECUDA, or CG_ENOCONV / CG_ETIMEOUT with the last iterate) comes after
 * cells_out has received the deposited field, which it then holds. */
cg_status cg_coarse_grain(cg_mesh *mesh, int64_t n, const double *pos, int nfields,
                          const double *w, double *cells_out, const cg_params *params,
                          cg_report *report, void *stream);

/* cg_coarse_grain with HOST inputs and outputs: copies pos_host [3][n] and w_host
 * [nfields][n] to library-owned device buffers, runs the method, and copies the
 * result to cells_host [nfields][ncells].  Pinned host memory gives the fastest
 * copies; pageable memory works. */
cg_status cg_coarse_grain_host(cg_mesh *mesh, int64_t n, const double *pos_host, int nfields,
                               const double *w_host, double *cells_host, const cg_params *params,
                               cg_report *report, void *stream);

/* Independent coarse-grainings run concurrently: problem i is exactly
 * cg_coarse_grain(meshes[i], n[i], pos[i], nfields, w[i], cells[i], &params[i],
 * reports ? &reports[i] : NULL, streams[i]) -- same results, bit for bit -- or, when
 * cells[i] is host memory, cg_coarse_grain_host with the same arguments (pos[i], w[i]
 * host memory too: the problem copies its inputs in and its result out; host problems
 * given the same pos, w and n share one copy of those inputs, made before any problem
 * starts, in the mesh of the first of them to start), and up to
 * max_concurrent problems run at a time, each on a host thread of the library (the
 * calling thread is one of them), so their kernels overlap on the device where their
 * streams allow it.  Problems start longest first (estimated from cells, steps and
 * dtau over the squared cell size).  Problems given the same pos, w and n (all device or
 * all host arrays) on structured meshes of one geometry (dimensions, origin, cell size,
 * periodic axes) with the same deposit_mode deposit once: the first of them to start
 * deposits before any problem starts, into a buffer of its mesh (nfields x ncells
 * doubles, within the workspace limit), and each copies the field from there and
 * smooths it -- the same results, bit for bit; that problem's report carries the
 * deposition times, the others report 0 for ms_locate and ms_deposit.  A shared
 * deposition that fails leaves its problems to run unshared.  The meshes must be
 * distinct (each problem uses its mesh's workspaces); give each problem its own
 * non-default stream for overlap.  A mesh's first call of a configuration autotunes its
 * sweep shape by timing candidates; one thread times at a time, and meshes of one
 * geometry share the result (other running problems can still disturb the timing: make
 * the first call of a configuration through cg_coarse_grain where that matters).
 * Returns when every problem has finished: CG_OK, or the status of the lowest-index
 * failing problem (cg_last_error names it).  CG_EINVAL also for NULL arrays, a shared
 * mesh, max_concurrent < 1, or kernel profiling switched on (cg_profile_enable). */
cg_status cg_coarse_grain_concurrent(int nprob, cg_mesh *const *meshes, const int64_t *n,
                                     const double *const *pos, int nfields, const double *const *w,
                                     double *const *cells, const cg_params *params, cg_report *reports,
                                     void *const *streams, int max_concurrent);

/* The solid velocity (the paper's conclusions: the momentum, not the velocity, is
 * diffused): U_s = smoothed momentum / smoothed solid fraction per cell and component,
 * the two smoothed fields taken from one multi-field cg_coarse_grain or cg_diffuse call
 * (weights V_p and V_p u).  eps: device [ncells] FP64; mom: device [ncomp][ncells];
 * u_out: device [ncomp][ncells], not overlapping the inputs.  A cell whose solid
 * fraction is not above eps_min (>= 0) gets 0; the division is IEEE FP64.  Synchronises
 * the stream.  Errors: CG_EINVAL (NULL, host pointers, overlap, ncomp outside [1, 64]). */
cg_status cg_solid_velocity(const cg_mesh *mesh, int ncomp, const double *eps,
                            const double *mom, double eps_min, double *u_out, void *stream);

/* ------------------------------------------------------------------------ batches */

/* Many independent snapshots (Section 3.2.1: every field and component is an
 * independent diffusion problem) smoothed together.  meshes[nsnap] are structured
 * meshes of any sizes; cells[s] is device [nfields][ncells_s] FP64 (in/out);
 * bandwidths (host, may be NULL) gives b per snapshot, else params->bandwidth/T.
 * Precision modes 3 and 4 with implicit Euler or Crank-Nicolson run every snapshot,
 * step, refinement round and inner iteration as one CUDA graph, either as ONE persistent
 * cooperative launch (grid barriers bounded by params->barrier_budget, default ~1 s of
 * clock cycles; CG_ETIMEOUT if one gives up) or as one launch per phase covering every
 * snapshot and field (no grid barrier), whichever the autotuner measures faster for the
 * batch shape (params->sweep_shape can force either; barrier_budget > 0 forces the
 * persistent launch), with per-step residuals verified afterwards; both give the same
 * bits.  Other modes and schemes run the snapshots one after another.  The batch's descriptors
 * and work lists are kept with meshes[0].  report (may be NULL) aggregates all
 * snapshots.  Errors: CG_EINVAL (a tet mesh, sizes, pointers), CG_ENOCONV,
 * CG_ETIMEOUT, CG_ENOMEM, CG_ECUDA. */
cg_status cg_diffuse_batched(int nsnap, cg_mesh *const *meshes, int nfields,
                             double *const *cells, const cg_params *params,
                             const double *bandwidths, cg_report *report, void *stream);

/* The whole method for a batch: cg_deposit of snapshot s (n[s] particles, pos[s]
 * device [3][n[s]], w[s] device [nfields][n[s]]) into cells[s], then
 * cg_diffuse_batched.  Every snapshot's particles are located before any deposited
 * field is written: a snapshot with particles outside its mesh (CG_EDOMAIN) or
 * non-finite weights (CG_EINVAL) fails the call with no cells written (cg_last_error
 * names the first such snapshot).  report: ms_locate and ms_deposit are the device times
 * of the two phases over the whole batch, n_out_of_domain the batch's total. */
cg_status cg_coarse_grain_batched(int nsnap, cg_mesh *const *meshes, const int64_t *n,
                                  const double *const *pos, int nfields, const double *const *w,
                                  double *const *cells, const cg_params *params,
                                  const double *bandwidths, cg_report *report, void *stream);

/* ------------------------------------------------------------------------ no allocation */

/* Limits of cg_deposit_fixed_noalloc's static scratch. */
#define CG_NOALLOC_MAX_FIELDS 8
#define CG_NOALLOC_MAX_CELL_FIELDS 2097152   /* nfields * ncells, 64-bit accumulators */

/* Fixed-point particle-centroid deposition on a uniform hex mesh that allocates
 * nothing.  The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory while they run -- for example a solver whose memory
 * manager (such as a caching allocator) already owns the free device memory, or one
 * that forbids allocation after start-up because cudaMalloc and cudaFree may
 * synchronise the device and may fail under memory pressure.  Such callers cannot
 * use cg_deposit, which grows a mesh-owned workspace on first use.
 *
 * It computes exactly what cg_deposit computes with deposit_mode =
 * CG_DEPOSIT_FIXED_POINT on the mesh cg_create_mesh_structured(nx, ny, nz, origin, dx)
 * (same locate rule, same scale exponents F, same result bit for bit), without a mesh
 * object: pos is device [3][n] FP64, w device [nfields][n] FP64, cells_out device
 * [nfields][nx*ny*nz] FP64, all caller-owned.  fixed_point_bits_host (may be NULL)
 * receives F per field.
 *
 * Scratch: a file-scope static device array of 128 + CG_NOALLOC_MAX_CELL_FIELDS
 * 64-bit words (about 16 MiB), which every GPU that loads the library's module holds
 * until the process exits.  Under CUDA's default lazy module loading that memory is
 * taken when the module first loads on a device, i.e. by the first call there (or
 * earlier with CUDA_MODULE_LOADING=EAGER): a caller that must not allocate later
 * should make one call at start-up.  The first call on a device also looks up the
 * array's device address (once per device, with the device current); make that
 * first call before any stream capture.  A device reset (cudaDeviceReset)
 * invalidates the looked-up address: make no call after one.  Every call on a device
 * shares the array and clears the part it uses; calls whose work overlaps on the GPU
 * race on it, so serialise them.  The call makes no cudaMalloc, cudaFree or other
 * allocating call; it synchronises `stream` before returning, like every entry point
 * here.
 *
 * Errors: CG_EINVAL (nfields outside [1, CG_NOALLOC_MAX_FIELDS], nfields * ncells >
 * CG_NOALLOC_MAX_CELL_FIELDS -- checked without overflow --, a non-finite origin or
 * box, bad sizes or NULL pointers, non-finite weights),
 * CG_EDOMAIN (particles outside the mesh; nothing written), CG_ECUDA. */
cg_status cg_deposit_fixed_noalloc(int nx, int ny, int nz, const double origin[3], double dx,
                                   int64_t n, const double *pos, int nfields, const double *w,
                                   double *cells_out, int *fixed_point_bits_host, void *stream);

/* ------------------------------------------------------------------------ diagnostics */

/* Per-kernel device timing (no counterpart in the paper; a measurement aid).  When
 * enabled, every kernel launch of the library is bracketed by a CUDA event pair on its
 * launching stream; after each call the elapsed times are accumulated per kernel name
 * with the launch count and the launch's algorithmic bytes (the minimum DRAM traffic
 * the kernel's definition implies: each input element read once, each output element
 * written once).  Process-wide; adds a little host overhead per launch while enabled. */
cg_status cg_profile_enable(int on);
void cg_profile_reset(void);
int cg_profile_count(void);
/* Entry i: name (NUL-terminated, truncated to name_len), launches, total ms, total
 * algorithmic bytes.  Any out pointer may be NULL.  CG_EINVAL for a bad index. */
cg_status cg_profile_get(int i, char *name, int name_len, long long *launches, double *ms,
                         double *bytes);

/* Device workspace accounting (no counterpart in the paper).  cg_workspace_bytes: the
 * device bytes the library's workspaces hold now, over all meshes and devices (caller
 * arrays and the no-allocation entry point's static scratch not included).
 * cg_set_workspace_limit: a process-wide cap on that total (0, the default: none); a
 * call that would grow a workspace beyond it returns CG_ENOMEM before allocating and
 * before writing any output, as a failed cudaMalloc does, and the library stays usable.
 * Lets a caller budget device memory, and tests the allocation-failure path without
 * exhausting a GPU.  CG_EINVAL for a negative limit. */
cg_status cg_set_workspace_limit(long long bytes);
long long cg_workspace_bytes(void);

/* Number of kernels the library has launched in this process since the last reset
 * (counted whether or not profiling is enabled). */
long long cg_launch_count(void);
void cg_launch_count_reset(void);

#ifdef __cplusplus
}
#endif

#endif /* CG_H */

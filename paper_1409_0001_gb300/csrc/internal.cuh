// internal.cuh -- shared declarations of the CUDA library behind include/cg.h.
// Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <utility>
#include <vector>

#include "cg.h"

namespace cgk {

// ----------------------------------------------------------------------------- errors
// Records a message for cg_last_error() (per thread) and returns the status.
cg_status fail(cg_status s, const char *fmt, ...);
cg_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define CGK_CUDA(call)                                                          \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) return ::cgk::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define CGK_TRY(call)                                                           \
    do {                                                                        \
        cg_status s_ = (call);                                                  \
        if (s_ != CG_OK) return s_;                                             \
    } while (0)

// ----------------------------------------------------------------------------- buffers
// A device buffer that only grows.  Owned by a mesh; freed in cg_destroy_mesh.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    unsigned gen = 0;        // bumped on every reallocation (invalidates captured graphs)
    cg_status ensure(size_t n);
    void release();
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// A pinned host buffer that only grows (readback of scalars, flags, counters).
struct HostBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cg_status ensure(size_t n);
    void release();
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// ----------------------------------------------------------------------------- graphs
// Launch records of a captured graph: when profiling was on during capture, each
// launch got its own event pair (recorded inside the graph); after every replay the
// elapsed times are added to the profile.
struct ProfRecord {
    const char *name;
    double bytes;
    cudaEvent_t a, b;
    int count;               // launches between the two events
};

// A captured diffusion (one entry per distinct call signature and buffer set).
// Shape of a captured batched schedule: the arena its kernels read (descriptors and
// work items are re-uploaded before every replay), the readback buffer, and the scalars
// baked into its launches.
struct BatchKey {
    const void *arena = nullptr;
    unsigned gen = 0;
    int nsnap = 0, nf = 0, nsteps = 0, R = 0, mmax = 0, nr = 0, nc = 0, grid = 0, zlen = 0,
        tsize = 0, scheme = 0, phased = 0;
    long long budget = 0;
    double tol2 = 0.0;
    bool operator==(const BatchKey &o) const {
        return arena == o.arena && gen == o.gen && nsnap == o.nsnap && nf == o.nf &&
               nsteps == o.nsteps && R == o.R && mmax == o.mmax && nr == o.nr && nc == o.nc &&
               grid == o.grid && zlen == o.zlen && tsize == o.tsize && scheme == o.scheme &&
               phased == o.phased && budget == o.budget && tol2 == o.tol2;
    }
};

struct GraphEntry {
    bool batched = false;           // a batched schedule (matched by bkey only)
    BatchKey bkey;
    int nf = 0, precision = 0, scheme = 0, nsteps = 0, rounds = 0;
    int code = 0;                   // inner-solve shape (sweep_shape code) captured
    long long wait_budget = 0;      // resident waits' clock-cycle budget captured
    double T = 0, tol = 0;
    const void *cells = nullptr;
    unsigned gen_diffuse = 0, gen_small = 0;
    bool profiled = false;
    cudaGraphExec_t exec = nullptr;
    const void *result = nullptr;   // workspace buffer holding the final iterate
    long long kernels = 0;
    std::vector<ProfRecord> records;
};

// Refinement rounds per step that sufficed for a call signature (learned on the first
// call, used to capture a fixed schedule afterwards).
struct RoundsEntry {
    int nf, precision, scheme, nsteps;
    double T, tol;
    int rounds;
};

// ----------------------------------------------------------------------------- meshes
enum MeshKind { MESH_STRUCTURED = 0, MESH_TET = 1, MESH_HEX = 2 };   // HEX: stretched Cartesian

struct TetDevice {
    // operator in ELL-4 form (slot s = the face opposite local vertex s); a boundary
    // face points at the cell itself with a zero transmissibility
    double *vc = nullptr;        // [ncells] cell volumes V_c
    double *diagL = nullptr;     // [ncells] L_kk = -sum_f T_f
    int32_t *offc = nullptr;     // [4][ncells] neighbour across face s
    double *offv = nullptr;      // [4][ncells] T_f across face s (FP64)
    float *offv32 = nullptr;     // [4][ncells] the same in FP32
    double max_rate = 0.0;       // max_k (-L_kk / V_k): explicit Euler needs dtau <= 1/max_rate
    int ns = 4;                  // neighbour slots per cell: 4 (tets) or 6 (stretched hex)
    // point location on a stretched Cartesian mesh: face coordinates x | y | z
    double *faces = nullptr;
    int hn[3] = {0, 0, 0};
    // point location
    double *xyz = nullptr;       // [nverts][3]
    int32_t *tv = nullptr;       // [ntets][4]
    double *box = nullptr;       // [ntets][6] lo.x lo.y lo.z hi.x hi.y hi.z
    float *edge32 = nullptr;     // [ntets][9] v1 - v0, v2 - v0, v3 - v0: FP64 differences
                                 // rounded to FP32 (the inside test's edge vectors)
    int32_t *bucket_start = nullptr;  // [nbuckets+1]
    int32_t *bucket_tets = nullptr;   // tet ids, ascending within a bucket
    int nb[3] = {0, 0, 0};
    double blo[3] = {0, 0, 0};
    double binv[3] = {0, 0, 0};
};

}  // namespace cgk

struct cg_mesh {
    int kind = cgk::MESH_STRUCTURED;
    int nx = 0, ny = 0, nz = 0;
    int per = 0;   // periodic axes of a structured mesh (bit 0 x, 1 y, 2 z)
    double origin[3] = {0, 0, 0};
    double dx = 0;
    int64_t ncells = 0;
    int64_t nverts = 0;

    cgk::TetDevice tet;
    std::vector<double> h_vc;            // host copy of V_c (tet)
    std::vector<int32_t> h_rowptr, h_col;
    std::vector<double> h_val;

    // workspaces (grown on demand)
    cgk::DevBuf ws_locate;   // cell ids / keys / values / counts
    cgk::DevBuf ws_sort;     // radix sort ping-pong and histograms
    cgk::DevBuf ws_diffuse;  // solver vectors
    cgk::DevBuf ws_small;    // scalars, partials, counters
    cgk::DevBuf ws_stage;    // device staging for the host-pointer entry point
    cgk::DevBuf ws_shared_in;  // host inputs copied once for several concurrent problems
    cgk::DevBuf ws_shared_dep; // a deposited field shared by several concurrent problems
    cgk::DevBuf ws_order;    // particles ordered by point-location bucket (tet meshes)
    cgk::DevBuf ws_batch;    // batched calls: descriptors, work items, partials (first mesh)
    cgk::HostBuf h_small;    // pinned readback
    std::vector<std::pair<int, int>> tuned;   // autotuned sweep z-chunk per (fields, type)
    std::vector<std::pair<std::vector<int>, int>> btuned;   // batched z-chunk per batch shape
    std::vector<std::pair<std::vector<double>, int>> brounds;  // batched rounds per call signature
    std::vector<cgk::GraphEntry> graphs;      // captured diffusions
    std::vector<cgk::RoundsEntry> rounds;     // learned refinement schedules
    std::vector<std::pair<double, double>> spectrum;   // unstructured: lower end of the
                                                       // Chebyshev interval per dte
    cudaStream_t capture_stream = nullptr;    // private stream used only for capture
    std::vector<cudaStream_t> aux_streams;    // batched depositions: snapshots in parallel
};

namespace cgk {

// ----------------------------------------------------------------------------- device props
int num_sms();

// nx * ny * nz < limit for dimensions >= 1, decided without overflow.
bool cells_below(int nx, int ny, int nz, int64_t limit);

// ----------------------------------------------------------------------------- profiling
// Opt-in per-kernel device timing (cg_profile_enable).  A scope records a CUDA event
// pair on the launching stream around one launch and remembers the launch's
// algorithmic bytes; prof_collect() (called after the stream is synchronised)
// accumulates the elapsed times per kernel name.
bool prof_on();
struct ProfScope {
    // name == nullptr: count the launch only.  count: launches the scope covers (their
    // device time is the interval between the scope's two events).  counts_launch:
    // the scope itself is one launch for the launch counter.
    ProfScope(const char *name, double bytes, cudaStream_t st, int count = 1,
              bool counts_launch = true);
    ~ProfScope();
    int slot = -1;
    cudaStream_t st = nullptr;
};
void prof_collect();
// While a sink is set (graph capture), profiling scopes give each launch its own event
// pair and append it to the sink, and launches are counted into *kernels instead of the
// process-wide counter.
void prof_capture_begin(std::vector<ProfRecord> *sink, long long *kernels);
void prof_capture_end();
// After a replay of a graph: add its records' elapsed times and launch count.
void prof_account_replay(const GraphEntry &e);
void graph_release(GraphEntry &e);

// Launch with an optional profiling scope: CGK_LAUNCH("name", algorithmic_bytes, stream,
// kernel<<<grid, block, smem, stream>>>(args...));
#define CGK_LAUNCH(name, bytes, st, ...)                                        \
    do {                                                                        \
        ::cgk::ProfScope ps_(name, (double)(bytes), st);                        \
        __VA_ARGS__;                                                            \
    } while (0)

// A launch counted but not timed on its own (it is inside a CGK_TIMED scope).
#define CGK_LAUNCH_UNTIMED(st, ...)                                             \
    do {                                                                        \
        ::cgk::ProfScope ps_(nullptr, 0.0, st);                                 \
        __VA_ARGS__;                                                            \
    } while (0)

// A timed scope over `count` launches made with CGK_LAUNCH_UNTIMED: one event pair.
#define CGK_TIMED(var, name, bytes, st, count) ::cgk::ProfScope var(name, (double)(bytes), st, count, false)

// ----------------------------------------------------------------------------- phases
// Locate (structured or tet).  Writes cell ids (int32, -1 outside) to cell_out and the
// number outside / number of non-finite weights to the host.  If counts != nullptr
// also accumulates per-cell particle counts (must be zeroed by the caller), writes each
// particle's arrival rank at its cell's counter to ranks (if not nullptr) and returns
// the largest count in max_count (if not nullptr).
// u_out[c][k] = mom[c][k] / eps[k] where eps[k] > eps_min, else 0 (IEEE division).
cg_status solid_velocity_run(int64_t n, int ncomp, const double *eps, const double *mom,
                             double eps_min, double *u_out, cudaStream_t st);

cg_status locate_run(cg_mesh *m, int64_t n, const double *pos, int nf, const double *w,
                     int32_t *cell_out, uint32_t *counts, int64_t *n_out, int64_t *n_nonfinite,
                     cudaStream_t st, uint32_t *max_count = nullptr, uint32_t *ranks = nullptr);

// Deposition (Eq. (pcm-k)) given particles; validates and writes out[nf][ncells].
cg_status deposit_run(cg_mesh *m, int64_t n, const double *pos, int nf, const double *w,
                      double *out, const cg_params *p, cg_report *rep, cudaStream_t st);
// The depositions of several distinct meshes with one synchronisation (see deposit.cu).
cg_status deposit_many(int nsnap, cg_mesh *const *meshes, const int64_t *n, const double *const *pos,
                       int nf, const double *const *w, double *const *out, const cg_params *p,
                       cg_report *rep, cudaStream_t st);

// Diffusion on a structured mesh (in place).
cg_status diffuse_structured_run(cg_mesh *m, int nf, double *cells, const cg_params *p,
                                 cg_report *rep, cudaStream_t st);

// Batched diffusion of many structured snapshots in one persistent launch (double-float
// modes 3 and 4, implicit Euler or Crank-Nicolson).
cg_status diffuse_batched_run(int nsnap, cg_mesh *const *meshes, int nf, double *const *cells,
                              const cg_params *p, const double *bandwidths, cg_report *rep,
                              cudaStream_t st);

// Diffusion on a tet mesh (in place).
cg_status diffuse_tet_run(cg_mesh *m, int nf, double *cells, const cg_params *p,
                          cg_report *rep, cudaStream_t st);

// sum_k V_c,k u_f,k for each field (FP64, deterministic order), written to host.
cg_status field_mass(cg_mesh *m, int nf, const double *cells, double *mass_host,
                     cudaStream_t st);
cg_status field_mass_many(int nmesh, cg_mesh *const *ms, int nf, const double *const *cells,
                          double *mass_host, cudaStream_t st);

// Tet mesh construction (host C++), fills m->tet and the host copies.
cg_status tet_build(cg_mesh *m, int64_t nverts, const double *xyz, int64_t ntets,
                    const int32_t *tv);
// A stretched Cartesian mesh (host C++): face coordinates xf[nx+1], yf[ny+1], zf[nz+1]
// (strictly increasing) and a cell diffusion constant D[ncells] (NULL: 1), as the same
// finite-volume operator with six neighbour slots; fills m->tet and the host copies.
cg_status hex_build(cg_mesh *m, int nx, int ny, int nz, const double *xf, const double *yf,
                    const double *zf, const double *D);
void tet_release(cg_mesh *m);

// Exclusive scan of n uint32 values (in and out may alias).  tmp needs
// scan_tmp_words(n) words.
size_t scan_tmp_words(int64_t n);
cg_status exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp,
                             cudaStream_t st);

}  // namespace cgk

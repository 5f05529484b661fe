// capi.cu -- the extern "C" entry points of include/cg.h: argument validation, mesh
// objects, workspace management and phase orchestration.  The arithmetic of the
// method lives in deposit.cu (Section 3.1), stencil.cu and tet.cu (Section 3.2).
#include <cuda_runtime.h>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace cgk {

static thread_local char g_last_error[512] = "";

cg_status fail(cg_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return s;
}

cg_status cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    snprintf(g_last_error, sizeof(g_last_error), "%s failed: %s (%s:%d)", what,
             cudaGetErrorString(e), file, line);
    return e == cudaErrorMemoryAllocation ? CG_ENOMEM : CG_ECUDA;
}

// Device bytes the library's workspaces hold (all meshes, all devices), and the cap set
// by cg_set_workspace_limit (0: none).
static std::atomic<long long> g_ws_bytes{0};
static std::atomic<long long> g_ws_limit{0};

cg_status DevBuf::ensure(size_t n) {
    if (n <= bytes) return CG_OK;
    size_t want = n + n / 8;
    const long long lim = g_ws_limit.load();
    if (lim > 0 && g_ws_bytes.load() - (long long)bytes + (long long)want > lim)
        return fail(CG_ENOMEM,
                    "device workspace of %zu bytes refused: the library would hold %lld bytes, "
                    "above the limit of %lld (cg_set_workspace_limit)",
                    want, g_ws_bytes.load() - (long long)bytes + (long long)want, lim);
    if (p) {
        cudaError_t e = cudaFree(p);
        p = nullptr;
        g_ws_bytes -= (long long)bytes;
        bytes = 0;
        if (e != cudaSuccess) return cuda_fail(e, "cudaFree", __FILE__, __LINE__);
    }
    ++gen;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return fail(CG_ENOMEM, "cudaMalloc of %zu bytes failed: %s", want, cudaGetErrorString(e));
    }
    bytes = want;
    g_ws_bytes += (long long)want;
    return CG_OK;
}

void DevBuf::release() {
    if (p) {
        cudaFree(p);
        g_ws_bytes -= (long long)bytes;
    }
    p = nullptr;
    bytes = 0;
}

cg_status HostBuf::ensure(size_t n) {
    if (n <= bytes) return CG_OK;
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMallocHost(&p, n);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return fail(CG_ENOMEM, "cudaMallocHost of %zu bytes failed", n);
    }
    bytes = n;
    return CG_OK;
}

void HostBuf::release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
}

int num_sms() {
    static thread_local int dev = -1, sms = 0;
    int d = 0;
    cudaGetDevice(&d);
    if (d != dev) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || v <= 0)
            v = 148;
        dev = d;
        sms = v;
    }
    return sms;
}

bool cells_below(int nx, int ny, int nz, int64_t limit) {
    // each factor is bounded before it multiplies, so no product overflows
    if (nx < 1 || ny < 1 || nz < 1 || limit < 1) return false;
    if ((int64_t)nx >= limit) return false;
    if ((int64_t)ny > (limit - 1) / nx) return false;
    const int64_t nxy = (int64_t)nx * ny;
    if ((int64_t)nz > (limit - 1) / nxy) return false;
    return nxy * nz < limit;
}

// ----------------------------------------------------------------------------- profiler
namespace {
struct ProfEntry {
    std::string name;
    long long launches = 0;
    double ms = 0.0, bytes = 0.0;
};
struct Pending {
    cudaEvent_t a, b;
    int entry;
    double bytes;
    int count;
};
std::mutex g_prof_mu;
std::atomic<bool> g_prof_enabled{false};
std::vector<ProfEntry> g_prof;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t pool_get() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

std::atomic<long long> g_launches{0};
thread_local std::vector<ProfRecord> *t_sink = nullptr;
thread_local long long *t_sink_kernels = nullptr;

int prof_entry(const char *name) {
    for (size_t i = 0; i < g_prof.size(); ++i)
        if (g_prof[i].name == name) return (int)i;
    g_prof.push_back(ProfEntry{name});
    return (int)g_prof.size() - 1;
}

bool prof_on() { return g_prof_enabled.load(std::memory_order_relaxed); }

void prof_capture_begin(std::vector<ProfRecord> *sink, long long *kernels) {
    t_sink = sink;
    t_sink_kernels = kernels;
}

void prof_capture_end() {
    t_sink = nullptr;
    t_sink_kernels = nullptr;
}

void prof_account_replay(const GraphEntry &e) {
    g_launches.fetch_add(e.kernels, std::memory_order_relaxed);
    if (!e.profiled) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (const ProfRecord &r : e.records) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        ProfEntry &pe = g_prof[prof_entry(r.name)];
        pe.launches += r.count;
        pe.ms += ms;
        pe.bytes += r.bytes;
    }
}

void graph_release(GraphEntry &e) {
    if (e.exec) cudaGraphExecDestroy(e.exec);
    e.exec = nullptr;
    for (ProfRecord &r : e.records) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    e.records.clear();
}

ProfScope::ProfScope(const char *name, double bytes, cudaStream_t s, int count,
                     bool counts_launch)
    : st(s) {
    if (t_sink_kernels) {
        if (counts_launch) ++*t_sink_kernels;
        if (name && t_sink && prof_on()) {
            ProfRecord r{name, bytes, nullptr, nullptr, count};
            cudaEventCreate(&r.a);
            cudaEventCreate(&r.b);
            // inside a capture only an "external" record becomes a timing node
            cudaEventRecordWithFlags(r.a, st, cudaEventRecordExternal);
            t_sink->push_back(r);
            slot = (int)t_sink->size() - 1;
            slot = -2 - slot;   // records in the sink are addressed as -2 - index
        }
        return;
    }
    if (counts_launch) g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!name || !prof_on()) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int entry = prof_entry(name);
    Pending pe{pool_get(), pool_get(), entry, bytes, count};
    cudaEventRecord(pe.a, st);
    g_pending.push_back(pe);
    slot = (int)g_pending.size() - 1;
}

ProfScope::~ProfScope() {
    if (slot <= -2) {
        const size_t i = (size_t)(-2 - slot);
        if (t_sink && i < t_sink->size())
            cudaEventRecordWithFlags((*t_sink)[i].b, st, cudaEventRecordExternal);
        return;
    }
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEventRecord(g_pending[slot].b, st);
}

void prof_collect() {
    if (!prof_on()) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &pe : g_pending) {
        cudaEventSynchronize(pe.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, pe.a, pe.b);
        ProfEntry &e = g_prof[pe.entry];
        e.launches += pe.count;
        e.ms += ms;
        e.bytes += pe.bytes;
        g_event_pool.push_back(pe.a);
        g_event_pool.push_back(pe.b);
    }
    g_pending.clear();
}

static bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static cg_status check_params(const cg_params *p) {
    if (!p) return fail(CG_EINVAL, "params is NULL");
    if (p->nsteps < 1) return fail(CG_EINVAL, "nsteps must be >= 1 (got %d)", p->nsteps);
    if (p->scheme < 0 || p->scheme > 2) return fail(CG_EINVAL, "unknown scheme %d", p->scheme);
    if (p->precision < 0 || p->precision > 4)
        return fail(CG_EINVAL, "unknown precision %d", p->precision);
    if (p->deposit_mode < 0 || p->deposit_mode > 1)
        return fail(CG_EINVAL, "unknown deposit_mode %d", p->deposit_mode);
    double T = p->bandwidth > 0.0 ? p->bandwidth * p->bandwidth / 4.0 : p->T;
    if (!(T >= 0.0) || !std::isfinite(T)) return fail(CG_EINVAL, "pseudo-time T must be finite and >= 0");
    if (!(p->tol > 0.0) || !(p->tol < 1.0)) return fail(CG_EINVAL, "tol must be in (0, 1)");
    if (p->max_iter < 1) return fail(CG_EINVAL, "max_iter must be >= 1");
    if (p->fused_k < 0 || p->fused_k > 4) return fail(CG_EINVAL, "fused_k must be in [0, 4] (got %d)", p->fused_k);
    if (p->fused_k > 0 && p->scheme != CG_SCHEME_EXPLICIT_EULER)
        return fail(CG_EINVAL, "fused_k > 0 selects blocked explicit Euler steps (scheme 2)");
    return CG_OK;
}

}  // namespace cgk

using namespace cgk;

extern "C" {

const char *cg_status_string(cg_status s) {
    switch (s) {
        case CG_OK: return "CG_OK";
        case CG_EINVAL: return "CG_EINVAL";
        case CG_ENOMEM: return "CG_ENOMEM";
        case CG_ECUDA: return "CG_ECUDA";
        case CG_ENOCONV: return "CG_ENOCONV";
        case CG_ETIMEOUT: return "CG_ETIMEOUT";
        case CG_EDOMAIN: return "CG_EDOMAIN";
    }
    return "CG_UNKNOWN";
}

const char *cg_last_error(void) { return g_last_error; }

cg_status cg_profile_enable(int on) {
    prof_collect();
    g_prof_enabled.store(on != 0);
    return CG_OK;
}

long long cg_launch_count(void) { return g_launches.load(); }

cg_status cg_set_workspace_limit(long long bytes) {
    if (bytes < 0) return fail(CG_EINVAL, "the workspace limit must be >= 0 (0: no limit)");
    g_ws_limit.store(bytes);
    return CG_OK;
}

long long cg_workspace_bytes(void) { return g_ws_bytes.load(); }

void cg_launch_count_reset(void) { g_launches.store(0); }

void cg_profile_reset(void) {
    prof_collect();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.clear();
}

int cg_profile_count(void) {
    prof_collect();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    return (int)g_prof.size();
}

cg_status cg_profile_get(int i, char *name, int name_len, long long *launches, double *ms,
                         double *bytes) {
    prof_collect();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (i < 0 || i >= (int)g_prof.size()) return fail(CG_EINVAL, "profile index out of range");
    const ProfEntry &e = g_prof[i];
    if (name && name_len > 0) {
        std::strncpy(name, e.name.c_str(), (size_t)name_len - 1);
        name[name_len - 1] = 0;
    }
    if (launches) *launches = e.launches;
    if (ms) *ms = e.ms;
    if (bytes) *bytes = e.bytes;
    return CG_OK;
}

void cg_params_default(cg_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->nsteps = 10;
    p->scheme = CG_SCHEME_IMPLICIT_EULER;
    p->precision = CG_PREC_FP64;
    p->deposit_mode = CG_DEPOSIT_ORDERED;
    p->tol = 1e-13;
    p->max_iter = 10000;
    p->max_rounds = 12;
    p->fused_k = 0;
    p->barrier_budget = 0;
}

cg_status cg_create_mesh_structured(int nx, int ny, int nz, const double origin[3], double dx,
                                    cg_mesh **out) {
    if (!out) return fail(CG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!origin) return fail(CG_EINVAL, "origin is NULL");
    if (nx < 1 || ny < 1 || nz < 1) return fail(CG_EINVAL, "mesh dimensions must be >= 1");
    if (!cells_below(nx, ny, nz, (int64_t)1 << 31))
        return fail(CG_EINVAL, "mesh too large: nx*ny*nz must be < 2^31");
    if (!(dx > 0.0) || !std::isfinite(dx)) return fail(CG_EINVAL, "dx must be finite and > 0");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(origin[a])) return fail(CG_EINVAL, "origin must be finite");
    cg_mesh *m = new (std::nothrow) cg_mesh();
    if (!m) return fail(CG_ENOMEM, "host allocation failed");
    m->kind = MESH_STRUCTURED;
    m->nx = nx;
    m->ny = ny;
    m->nz = nz;
    for (int a = 0; a < 3; ++a) m->origin[a] = origin[a];
    m->dx = dx;
    m->ncells = (int64_t)nx * ny * nz;
    *out = m;
    return CG_OK;
}

cg_status cg_create_mesh_tet(int64_t nverts, const double *xyz_host, int64_t ntets,
                             const int32_t *tv_host, cg_mesh **out) {
    if (!out) return fail(CG_EINVAL, "out is NULL");
    *out = nullptr;
    if (nverts < 4 || ntets < 1 || !xyz_host || !tv_host)
        return fail(CG_EINVAL, "a tet mesh needs >= 4 vertices, >= 1 tet and host arrays");
    if (ntets >= ((int64_t)1 << 31) / 5 || nverts >= ((int64_t)1 << 31))
        return fail(CG_EINVAL, "tet mesh too large");
    cg_mesh *m = new (std::nothrow) cg_mesh();
    if (!m) return fail(CG_ENOMEM, "host allocation failed");
    m->kind = MESH_TET;
    m->ncells = ntets;
    m->nverts = nverts;
    cg_status s = tet_build(m, nverts, xyz_host, ntets, tv_host);
    if (s != CG_OK) {
        tet_release(m);
        delete m;
        return s;
    }
    *out = m;
    return CG_OK;
}

cg_status cg_create_mesh_hex(int nx, int ny, int nz, const double *xf, const double *yf,
                             const double *zf, const double *diffusivity, cg_mesh **out) {
    if (!out) return fail(CG_EINVAL, "out is NULL");
    *out = nullptr;
    if (!xf || !yf || !zf) return fail(CG_EINVAL, "face coordinate arrays are NULL");
    if (nx < 1 || ny < 1 || nz < 1) return fail(CG_EINVAL, "mesh dimensions must be >= 1");
    if (!cells_below(nx, ny, nz, ((int64_t)1 << 31) / 7))
        return fail(CG_EINVAL, "mesh too large: nx*ny*nz must be < 2^31 / 7");
    const int n3[3] = {nx, ny, nz};
    const double *f[3] = {xf, yf, zf};
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i <= n3[a]; ++i) {
            if (!std::isfinite(f[a][i])) return fail(CG_EINVAL, "face coordinates must be finite");
            if (i > 0 && !(f[a][i] > f[a][i - 1]))
                return fail(CG_EINVAL, "face coordinates must increase strictly (axis %d, face %d)", a, i);
        }
    const int64_t n = (int64_t)nx * ny * nz;
    if (diffusivity)
        for (int64_t k = 0; k < n; ++k)
            if (!(diffusivity[k] >= 0.0) || !std::isfinite(diffusivity[k]))
                return fail(CG_EINVAL, "diffusivity must be finite and >= 0 (cell %lld)", (long long)k);
    cg_mesh *m = new (std::nothrow) cg_mesh();
    if (!m) return fail(CG_ENOMEM, "host allocation failed");
    m->kind = MESH_HEX;
    m->nx = nx;
    m->ny = ny;
    m->nz = nz;
    m->ncells = n;
    cg_status s = hex_build(m, nx, ny, nz, xf, yf, zf, diffusivity);
    if (s != CG_OK) {
        tet_release(m);
        delete m;
        return s;
    }
    *out = m;
    return CG_OK;
}

cg_status cg_destroy_mesh(cg_mesh *m) {
    if (!m) return CG_OK;
    m->ws_locate.release();
    m->ws_sort.release();
    m->ws_diffuse.release();
    m->ws_small.release();
    m->ws_stage.release();
    m->ws_shared_in.release();
    m->ws_shared_dep.release();
    m->ws_order.release();
    m->ws_batch.release();
    m->h_small.release();
    for (auto &e : m->graphs) graph_release(e);
    m->graphs.clear();
    if (m->capture_stream) cudaStreamDestroy(m->capture_stream);
    for (cudaStream_t a : m->aux_streams) cudaStreamDestroy(a);
    if (m->kind != MESH_STRUCTURED) tet_release(m);
    delete m;
    return CG_OK;
}

int64_t cg_mesh_num_cells(const cg_mesh *m) { return m ? m->ncells : -1; }

cg_status cg_mesh_set_periodic(cg_mesh *m, int px, int py, int pz) {
    if (!m) return fail(CG_EINVAL, "mesh is NULL");
    if (m->kind != MESH_STRUCTURED) return fail(CG_EINVAL, "periodic axes need a structured mesh");
    const int per = (px ? 1 : 0) | (py ? 2 : 0) | (pz ? 4 : 0);
    if (per != m->per) {   // captured schedules and tuned shapes assumed the old walls
        for (auto &e : m->graphs) graph_release(e);
        m->graphs.clear();
        m->tuned.clear();
        m->rounds.clear();
        m->per = per;
    }
    return CG_OK;
}

cg_status cg_solid_velocity(const cg_mesh *m, int ncomp, const double *eps, const double *mom,
                            double eps_min, double *u_out, void *stream) {
    if (!m) return fail(CG_EINVAL, "mesh is NULL");
    if (ncomp < 1 || ncomp > 64) return fail(CG_EINVAL, "ncomp must be in [1, 64]");
    if (!is_device_ptr(eps) || !is_device_ptr(mom) || !is_device_ptr(u_out))
        return fail(CG_EINVAL, "eps, mom and u_out must be device pointers");
    if (!(eps_min >= 0.0) || !std::isfinite(eps_min)) return fail(CG_EINVAL, "eps_min must be >= 0");
    const int64_t n = m->ncells;
    const char *a = (const char *)u_out, *b = (const char *)mom, *c = (const char *)eps;
    const size_t bytes = (size_t)ncomp * n * 8;
    if ((a < b + bytes && b < a + bytes) || (a < c + (size_t)n * 8 && c < a + bytes))
        return fail(CG_EINVAL, "u_out overlaps eps or mom");
    return solid_velocity_run(n, ncomp, eps, mom, eps_min, u_out, (cudaStream_t)stream);
}

cg_status cg_mesh_cell_volumes(const cg_mesh *m, double *out_host) {
    if (!m || !out_host) return fail(CG_EINVAL, "NULL argument");
    if (m->kind == MESH_STRUCTURED) {
        double v = (m->dx * m->dx) * m->dx;
        for (int64_t k = 0; k < m->ncells; ++k) out_host[k] = v;
    } else {
        std::memcpy(out_host, m->h_vc.data(), (size_t)m->ncells * sizeof(double));
    }
    return CG_OK;
}

cg_status cg_mesh_tet_operator(const cg_mesh *m, int64_t *rowptr_host, int32_t *col_host,
                               double *val_host, int64_t *nnz_out) {
    if (!m) return fail(CG_EINVAL, "mesh is NULL");
    if (m->kind == MESH_STRUCTURED) return fail(CG_EINVAL, "a uniform mesh has no stored operator");
    if (nnz_out) *nnz_out = (int64_t)m->h_col.size();
    if (rowptr_host)
        for (int64_t k = 0; k <= m->ncells; ++k) rowptr_host[k] = m->h_rowptr[k];
    if (col_host) std::memcpy(col_host, m->h_col.data(), m->h_col.size() * sizeof(int32_t));
    if (val_host) std::memcpy(val_host, m->h_val.data(), m->h_val.size() * sizeof(double));
    return CG_OK;
}

cg_status cg_locate(cg_mesh *m, int64_t n, const double *pos, int32_t *cell_out,
                    int64_t *n_out_host, void *stream) {
    if (!m) return fail(CG_EINVAL, "mesh is NULL");
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(CG_EINVAL, "n must be in [0, 2^31)");
    if (n > 0 && (!is_device_ptr(pos) || !is_device_ptr(cell_out)))
        return fail(CG_EINVAL, "pos and cell_out must be device pointers");
    int64_t nout = 0;
    CGK_TRY(locate_run(m, n, pos, 0, nullptr, cell_out, nullptr, &nout, nullptr,
                       (cudaStream_t)stream));
    prof_collect();
    if (n_out_host) *n_out_host = nout;
    return CG_OK;
}

static cg_status check_deposit_args(cg_mesh *m, int64_t n, const double *pos, int nfields,
                                    const double *w, double *cells, const cg_params *p) {
    if (!m) return fail(CG_EINVAL, "mesh is NULL");
    CGK_TRY(check_params(p));
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(CG_EINVAL, "n must be in [0, 2^31)");
    if (nfields < 1 || nfields > 64) return fail(CG_EINVAL, "nfields must be in [1, 64]");
    if ((int64_t)nfields * m->ncells >= ((int64_t)1 << 40))
        return fail(CG_EINVAL, "nfields * ncells too large");
    if (!is_device_ptr(cells)) return fail(CG_EINVAL, "cells must be a device pointer");
    if (n > 0 && (!is_device_ptr(pos) || !is_device_ptr(w)))
        return fail(CG_EINVAL, "pos and w must be device pointers");
    return CG_OK;
}

cg_status cg_deposit(cg_mesh *m, int64_t n, const double *pos, int nfields, const double *w,
                     double *cells_out, const cg_params *p, cg_report *rep, void *stream) {
    CGK_TRY(check_deposit_args(m, n, pos, nfields, w, cells_out, p));
    cg_status s = deposit_run(m, n, pos, nfields, w, cells_out, p, rep, (cudaStream_t)stream);
    prof_collect();
    return s;
}

static cg_status diffuse_impl(cg_mesh *m, int nf, double *cells, const cg_params *p,
                              cg_report *rep, cudaStream_t st) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rep) {
        CGK_TRY(field_mass(m, nf < CG_REPORT_MAX_FIELDS ? nf : CG_REPORT_MAX_FIELDS, cells,
                           rep->mass_in, st));
        CGK_CUDA(cudaEventCreate(&e0));
        CGK_CUDA(cudaEventCreate(&e1));
        CGK_CUDA(cudaEventRecord(e0, st));
    }
    cg_status s;
    double T = p->bandwidth > 0.0 ? p->bandwidth * p->bandwidth / 4.0 : p->T;
    if (T == 0.0) {
        s = CG_OK;   // nothing to smooth
    } else if (m->kind == MESH_STRUCTURED) {
        s = diffuse_structured_run(m, nf, cells, p, rep, st);
    } else {
        s = diffuse_tet_run(m, nf, cells, p, rep, st);
    }
    if (rep) {
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        rep->ms_diffuse = ms;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (s == CG_OK || s == CG_ENOCONV) {
            cg_status s2 = field_mass(m, nf < CG_REPORT_MAX_FIELDS ? nf : CG_REPORT_MAX_FIELDS,
                                      cells, rep->mass_out, st);
            if (s == CG_OK) s = s2;
        }
    }
    return s;
}

cg_status cg_diffuse(cg_mesh *m, int nfields, double *cells, const cg_params *p, cg_report *rep,
                     void *stream) {
    if (!m) return fail(CG_EINVAL, "mesh is NULL");
    CGK_TRY(check_params(p));
    if (nfields < 1 || nfields > 64) return fail(CG_EINVAL, "nfields must be in [1, 64]");
    if (!is_device_ptr(cells)) return fail(CG_EINVAL, "cells must be a device pointer");
    if (rep) {
        double keep_loc = rep->ms_locate, keep_dep = rep->ms_deposit;
        long long keep_out = rep->n_out_of_domain;
        int keep_bits[CG_REPORT_MAX_FIELDS];
        std::memcpy(keep_bits, rep->fixed_point_bits, sizeof(keep_bits));
        std::memset(rep, 0, sizeof(*rep));
        rep->ms_locate = keep_loc;
        rep->ms_deposit = keep_dep;
        rep->n_out_of_domain = keep_out;
        std::memcpy(rep->fixed_point_bits, keep_bits, sizeof(keep_bits));
    }
    cg_status s = diffuse_impl(m, nfields, cells, p, rep, (cudaStream_t)stream);
    prof_collect();
    return s;
}

cg_status cg_coarse_grain(cg_mesh *m, int64_t n, const double *pos, int nfields, const double *w,
                          double *cells_out, const cg_params *p, cg_report *rep, void *stream) {
    CGK_TRY(check_deposit_args(m, n, pos, nfields, w, cells_out, p));
    if (rep) std::memset(rep, 0, sizeof(*rep));
    cudaStream_t st = (cudaStream_t)stream;
    cg_status s = deposit_run(m, n, pos, nfields, w, cells_out, p, rep, st);
    if (s == CG_OK) s = diffuse_impl(m, nfields, cells_out, p, rep, st);
    prof_collect();
    return s;
}

static cg_status batched_diffuse_impl(int nsnap, cg_mesh *const *meshes, int nfields,
                                     double *const *cells, const cg_params *p,
                                     const double *bandwidths, cg_report *rep, cudaStream_t st) {
    const bool fused = (p->precision == CG_PREC_FP32_DF_REFINE || p->precision == CG_PREC_BF16_DF_REFINE) &&
                       p->scheme != CG_SCHEME_EXPLICIT_EULER;
    double mass_in[CG_REPORT_MAX_FIELDS] = {0}, mass_out[CG_REPORT_MAX_FIELDS] = {0};
    const int nrep = nfields < CG_REPORT_MAX_FIELDS ? nfields : CG_REPORT_MAX_FIELDS;
    // the masses before and after: the batched graph's run reports them itself; the
    // per-snapshot loop below takes them here, one synchronisation for all snapshots
    std::vector<double> mm;
    if (rep && !fused) {
        mm.resize((size_t)nsnap * nrep);
        CGK_TRY(field_mass_many(nsnap, meshes, nrep, cells, mm.data(), st));
        for (int s = 0; s < nsnap; ++s)
            for (int f = 0; f < nrep; ++f) mass_in[f] += mm[(size_t)s * nrep + f];
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rep) {
        CGK_CUDA(cudaEventCreate(&e0));
        CGK_CUDA(cudaEventCreate(&e1));
        CGK_CUDA(cudaEventRecord(e0, st));
    }
    cg_status s = CG_OK;
    if (fused) {
        s = diffuse_batched_run(nsnap, meshes, nfields, cells, p, bandwidths, rep, st);
    } else {
        cg_report one;
        long long upd = 0, it = 0, rounds = 0;
        double worst = 0;
        for (int q = 0; q < nsnap && s == CG_OK; ++q) {
            cg_params pq = *p;
            if (bandwidths) pq.bandwidth = bandwidths[q];
            std::memset(&one, 0, sizeof(one));
            s = diffuse_structured_run(meshes[q], nfields, cells[q], &pq, &one, st);
            upd += one.cell_updates;
            it += one.iters;
            rounds += one.refine_rounds;
            worst = std::max(worst, one.final_rel_residual);
        }
        if (rep) {
            rep->cell_updates = upd;
            rep->iters = it;
            rep->refine_rounds = rounds;
            rep->final_rel_residual = worst;
        }
    }
    if (rep) {
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        rep->ms_diffuse = ms;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (!fused) {
            if (s == CG_OK || s == CG_ENOCONV) {
                cg_status s2 = field_mass_many(nsnap, meshes, nrep, cells, mm.data(), st);
                if (s2 != CG_OK) return s2;
                for (int q = 0; q < nsnap; ++q)
                    for (int f = 0; f < nrep; ++f) mass_out[f] += mm[(size_t)q * nrep + f];
            }
            for (int f = 0; f < nrep; ++f) {
                rep->mass_in[f] = mass_in[f];
                rep->mass_out[f] = mass_out[f];
            }
        }
    }
    return s;
}

static cg_status check_batch(int nsnap, cg_mesh *const *meshes, int nfields, double *const *cells,
                             const cg_params *p, const double *bandwidths) {
    CGK_TRY(check_params(p));
    if (nsnap < 1 || !meshes || !cells) return fail(CG_EINVAL, "empty batch or NULL arrays");
    if (nsnap > 65535) return fail(CG_EINVAL, "a batch holds at most 65535 snapshots");
    if (nfields < 1 || nfields > 64) return fail(CG_EINVAL, "nfields must be in [1, 64]");
    for (int s = 0; s < nsnap; ++s) {
        if (!meshes[s] || meshes[s]->kind != MESH_STRUCTURED)
            return fail(CG_EINVAL, "batch snapshot %d: not a structured mesh", s);
        if (meshes[s]->per)
            return fail(CG_EINVAL, "batch snapshot %d: periodic meshes are not batched", s);
        if (!is_device_ptr(cells[s])) return fail(CG_EINVAL, "batch snapshot %d: cells not on the device", s);
        if (bandwidths && !(bandwidths[s] > 0.0 && std::isfinite(bandwidths[s])))
            return fail(CG_EINVAL, "batch snapshot %d: bandwidth must be finite and > 0", s);
        for (int q = 0; q < s; ++q)
            if (meshes[q] == meshes[s])
                return fail(CG_EINVAL, "batch snapshots %d and %d share a mesh (workspaces would collide)", q, s);
    }
    return CG_OK;
}

cg_status cg_diffuse_batched(int nsnap, cg_mesh *const *meshes, int nfields, double *const *cells,
                             const cg_params *p, const double *bandwidths, cg_report *rep,
                             void *stream) {
    CGK_TRY(check_batch(nsnap, meshes, nfields, cells, p, bandwidths));
    if (rep) std::memset(rep, 0, sizeof(*rep));
    cg_status s = batched_diffuse_impl(nsnap, meshes, nfields, cells, p, bandwidths, rep,
                                       (cudaStream_t)stream);
    prof_collect();
    return s;
}

cg_status cg_coarse_grain_batched(int nsnap, cg_mesh *const *meshes, const int64_t *n,
                                  const double *const *pos, int nfields, const double *const *w,
                                  double *const *cells, const cg_params *p,
                                  const double *bandwidths, cg_report *rep, void *stream) {
    CGK_TRY(check_batch(nsnap, meshes, nfields, cells, p, bandwidths));
    if (!n || !pos || !w) return fail(CG_EINVAL, "NULL particle arrays");
    cudaStream_t st = (cudaStream_t)stream;
    if (rep) std::memset(rep, 0, sizeof(*rep));
    for (int s = 0; s < nsnap; ++s)
        CGK_TRY(check_deposit_args(meshes[s], n[s], pos[s], nfields, w[s], cells[s], p));
    CGK_TRY(deposit_many(nsnap, meshes, n, pos, nfields, w, cells, p, rep, st));
    double keep_loc = rep ? rep->ms_locate : 0, keep_dep = rep ? rep->ms_deposit : 0;
    cg_status s = batched_diffuse_impl(nsnap, meshes, nfields, cells, p, bandwidths, rep, st);
    if (rep) {
        rep->ms_locate = keep_loc;
        rep->ms_deposit = keep_dep;
    }
    prof_collect();
    return s;
}

static cg_status check_host_args(cg_mesh *m, int64_t n, const double *pos_host, int nfields,
                                 const double *w_host, const double *cells_host, const cg_params *p) {
    if (!m) return fail(CG_EINVAL, "mesh is NULL");
    CGK_TRY(check_params(p));
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(CG_EINVAL, "n must be in [0, 2^31)");
    if (nfields < 1 || nfields > 64) return fail(CG_EINVAL, "nfields must be in [1, 64]");
    if (!cells_host || (n > 0 && (!pos_host || !w_host)))
        return fail(CG_EINVAL, "NULL host array");
    return CG_OK;
}

// A deposited field shared by several concurrent problems: the buffer that holds it, the
// event after which it is complete, and the report of the deposition that made it (its
// phase times for the problem that deposited, zero for the others).
struct SharedDeposit {
    const double *src = nullptr;
    cudaEvent_t ready = nullptr;
    cg_report rep{};
};

// The host-memory form of the method (cg_coarse_grain_host).  dpos/dw non-NULL: the
// inputs are already on the device (a copy shared with other problems, complete once
// `ready` has fired), else pos_host/w_host are copied into this mesh's staging buffer.
// dep non-NULL: the deposited field is already on the device (shared with other
// problems), so the inputs are not needed.  The result is staged in this mesh's buffer
// and copied to cells_host.
static cg_status coarse_grain_host_impl(cg_mesh *m, int64_t n, const double *pos_host, int nfields,
                                        const double *w_host, double *cells_host, const cg_params *p,
                                        cg_report *rep, cudaStream_t st, const double *dpos_in,
                                        const double *dw_in, cudaEvent_t ready,
                                        const SharedDeposit *dep = nullptr) {
    CGK_TRY(check_host_args(m, n, pos_host, nfields, w_host, cells_host, p));
    const bool shared = dpos_in != nullptr && dep == nullptr;
    const size_t b_pos = ((size_t)3 * n * 8 + 255) / 256 * 256;
    const size_t b_w = ((size_t)nfields * n * 8 + 255) / 256 * 256;
    const size_t b_c = (size_t)nfields * m->ncells * 8;
    const size_t b_in = (shared || dep) ? 0 : b_pos + b_w;
    CGK_TRY(m->ws_stage.ensure(b_in + b_c + 256));
    char *base = m->ws_stage.as<char>();
    const double *dpos = shared ? dpos_in : (const double *)base;
    const double *dw = shared ? dw_in : (const double *)(base + b_pos);
    double *dc = (double *)(base + b_in);
    if (dep) {
        CGK_CUDA(cudaStreamWaitEvent(st, dep->ready, 0));
        CGK_CUDA(cudaMemcpyAsync(dc, dep->src, b_c, cudaMemcpyDeviceToDevice, st));
        if (rep) *rep = dep->rep;
    } else {
        if (shared) {
            CGK_CUDA(cudaStreamWaitEvent(st, ready, 0));
        } else if (n > 0) {
            CGK_CUDA(cudaMemcpyAsync(base, pos_host, (size_t)3 * n * 8, cudaMemcpyHostToDevice, st));
            CGK_CUDA(cudaMemcpyAsync(base + b_pos, w_host, (size_t)nfields * n * 8, cudaMemcpyHostToDevice, st));
        }
        if (rep) std::memset(rep, 0, sizeof(*rep));
        CGK_TRY(deposit_run(m, n, dpos, nfields, dw, dc, p, rep, st));
    }
    cg_status s = diffuse_impl(m, nfields, dc, p, rep, st);
    if (s != CG_OK && s != CG_ENOCONV) return s;
    CGK_CUDA(cudaMemcpyAsync(cells_host, dc, b_c, cudaMemcpyDeviceToHost, st));
    CGK_CUDA(cudaStreamSynchronize(st));
    prof_collect();
    return s;
}

// cg_coarse_grain from a deposited field shared with other problems.
static cg_status coarse_grain_from_shared(cg_mesh *m, int nfields, double *cells_out,
                                          const cg_params *p, cg_report *rep, cudaStream_t st,
                                          const SharedDeposit &dep) {
    CGK_CUDA(cudaStreamWaitEvent(st, dep.ready, 0));
    CGK_CUDA(cudaMemcpyAsync(cells_out, dep.src, (size_t)nfields * m->ncells * 8,
                             cudaMemcpyDeviceToDevice, st));
    if (rep) *rep = dep.rep;
    cg_status s = diffuse_impl(m, nfields, cells_out, p, rep, st);
    prof_collect();
    return s;
}

cg_status cg_coarse_grain_concurrent(int nprob, cg_mesh *const *meshes, const int64_t *n,
                                     const double *const *pos, int nfields, const double *const *w,
                                     double *const *cells, const cg_params *params, cg_report *reports,
                                     void *const *streams, int max_concurrent) {
    if (nprob < 1 || !meshes || !n || !pos || !w || !cells || !params || !streams)
        return fail(CG_EINVAL, "cg_coarse_grain_concurrent: no problems or a NULL array");
    if (max_concurrent < 1) return fail(CG_EINVAL, "max_concurrent must be >= 1");
    if (prof_on())
        return fail(CG_EINVAL, "kernel profiling is on: concurrent problems would share its event timing");
    for (int i = 0; i < nprob; ++i) {
        if (!meshes[i]) return fail(CG_EINVAL, "problem %d: mesh is NULL", i);
        for (int j = 0; j < i; ++j)
            if (meshes[j] == meshes[i])
                return fail(CG_EINVAL, "problems %d and %d share a mesh (workspaces would collide)", j, i);
    }
    int dev = 0;
    CGK_CUDA(cudaGetDevice(&dev));
    std::vector<cg_status> status(nprob, CG_OK);
    std::vector<std::string> detail(nprob);
    std::atomic<int> next{0};
    // a problem whose output is host memory runs as cg_coarse_grain_host (its inputs are
    // host memory too), otherwise as cg_coarse_grain
    std::vector<char> host(nprob);
    for (int i = 0; i < nprob; ++i) host[i] = !is_device_ptr(cells[i]);
    // longest first (fewer idle workers at the end): the cost estimate is cells x steps x
    // sqrt(1 + 12 dtau / h^2), which follows the Chebyshev iteration count, with h the
    // cell edge (structured) or the edge of a cube of the mean cell volume
    std::vector<int> order(nprob);
    std::vector<double> cost(nprob);
    for (int i = 0; i < nprob; ++i) {
        const cg_mesh *m = meshes[i];
        const cg_params &q = params[i];
        const double T = q.bandwidth > 0.0 ? q.bandwidth * q.bandwidth / 4.0 : q.T;
        double h = m->dx;
        if (m->kind != MESH_STRUCTURED) {
            double v = 0;
            for (double x : m->h_vc) v += x;
            h = std::cbrt(v / std::max<int64_t>(m->ncells, 1));
        }
        const int ns = std::max(q.nsteps, 1);
        const double c = (h > 0 && std::isfinite(T)) ? T / ns / (h * h) : 0.0;
        cost[i] = (double)m->ncells * ns * std::sqrt(1.0 + 12.0 * std::max(c, 0.0));
        order[i] = i;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    // host problems given the same input arrays (pos, w and n) share one host-to-device
    // copy, made here before any problem starts, into the shared-input buffer of the
    // group's first problem in start order; the others wait for it on their streams.  A
    // group whose copy cannot be set up runs unshared (each problem copies its own).
    std::vector<const double *> sh_pos(nprob, nullptr), sh_w(nprob, nullptr);
    std::vector<cudaEvent_t> sh_ev(nprob, nullptr);
    std::vector<cudaEvent_t> events;
    const bool nf_ok = nfields >= 1 && nfields <= 64;
    for (int a = 0; a < nprob && nf_ok; ++a) {
        const int i = order[a];
        if (!host[i] || sh_pos[i] || n[i] <= 0 || n[i] >= ((int64_t)1 << 31) || !pos[i] || !w[i]) continue;
        std::vector<int> members{i};
        for (int b = a + 1; b < nprob; ++b) {
            const int k = order[b];
            if (host[k] && !sh_pos[k] && pos[k] == pos[i] && w[k] == w[i] && n[k] == n[i]) members.push_back(k);
        }
        if (members.size() < 2) continue;
        const size_t b_pos = ((size_t)3 * n[i] * 8 + 255) / 256 * 256;
        const size_t b_w = (size_t)nfields * n[i] * 8;
        if (meshes[i]->ws_shared_in.ensure(b_pos + b_w) != CG_OK) continue;
        char *base = meshes[i]->ws_shared_in.as<char>();
        cudaStream_t st = (cudaStream_t)streams[i];
        cudaEvent_t ev = nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (cudaMemcpyAsync(base, pos[i], (size_t)3 * n[i] * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(base + b_pos, w[i], b_w, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaEventRecord(ev, st) != cudaSuccess) {
            cudaGetLastError();
            cudaEventDestroy(ev);
            continue;
        }
        events.push_back(ev);
        for (int k : members) {
            sh_pos[k] = (const double *)base;
            sh_w[k] = (const double *)(base + b_pos);
            sh_ev[k] = ev;
        }
    }
    // problems given the same particle arrays (pos, w and n) on structured meshes of one
    // geometry (dimensions, origin, cell size, periodic axes) with the same deposition mode
    // deposit once: the group's first problem in start order deposits here, before any
    // problem starts, into a buffer of its mesh, and every member (that one included)
    // copies the field from there on its own stream and smooths it.  The deposition is
    // the same computation on the same inputs, so every result is bit-identical to an
    // unshared run; the problem that deposited reports the deposition's phase times, the
    // others report zero for them.  A group whose deposition fails (an argument, a
    // particle outside the mesh, a workspace that cannot grow) runs unshared, each
    // problem then reporting its own status as it would alone.
    std::vector<SharedDeposit> sdep(nprob);
    std::vector<char> in_dep(nprob, 0);
    auto same_deposit = [&](int i, int k) {
        const cg_mesh *a = meshes[i], *b = meshes[k];
        return host[k] == host[i] && pos[k] == pos[i] && w[k] == w[i] && n[k] == n[i] &&
               b->kind == MESH_STRUCTURED && a->kind == MESH_STRUCTURED && b->nx == a->nx &&
               b->ny == a->ny && b->nz == a->nz && b->per == a->per && b->dx == a->dx &&
               b->origin[0] == a->origin[0] && b->origin[1] == a->origin[1] &&
               b->origin[2] == a->origin[2] && params[k].deposit_mode == params[i].deposit_mode;
    };
    auto args_ok = [&](int k) {
        return (host[k] ? check_host_args(meshes[k], n[k], pos[k], nfields, w[k], cells[k], &params[k])
                        : check_deposit_args(meshes[k], n[k], pos[k], nfields, w[k], cells[k],
                                             &params[k])) == CG_OK;
    };
    for (int a = 0; a < nprob && nf_ok; ++a) {
        const int i = order[a];
        if (in_dep[i] || meshes[i]->kind != MESH_STRUCTURED || n[i] <= 0 || !args_ok(i)) continue;
        if (host[i] && !sh_pos[i]) continue;   // host inputs not on the device
        std::vector<int> members{i};
        for (int b = a + 1; b < nprob; ++b) {
            const int k = order[b];
            if (!in_dep[k] && same_deposit(i, k) && args_ok(k)) members.push_back(k);
        }
        if (members.size() < 2) continue;
        cg_mesh *mi = meshes[i];
        cudaStream_t st = (cudaStream_t)streams[i];
        if (mi->ws_shared_dep.ensure((size_t)nfields * mi->ncells * 8) != CG_OK) continue;
        double *buf = mi->ws_shared_dep.as<double>();
        if (host[i] && cudaStreamWaitEvent(st, sh_ev[i], 0) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cg_report r;
        std::memset(&r, 0, sizeof(r));
        if (deposit_run(mi, n[i], host[i] ? sh_pos[i] : pos[i], nfields, host[i] ? sh_w[i] : w[i], buf,
                        &params[i], &r, st) != CG_OK)
            continue;
        cudaEvent_t ev = nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (cudaEventRecord(ev, st) != cudaSuccess) {
            cudaGetLastError();
            cudaEventDestroy(ev);
            continue;
        }
        events.push_back(ev);
        for (int k : members) {
            in_dep[k] = 1;
            sdep[k].src = buf;
            sdep[k].ready = ev;
            sdep[k].rep = r;
            if (k != i) sdep[k].rep.ms_locate = sdep[k].rep.ms_deposit = 0.0;
        }
    }
    auto worker = [&](bool own_thread) {
        if (own_thread && cudaSetDevice(dev) != cudaSuccess) return;
        for (int j; (j = next.fetch_add(1)) < nprob;) {
            const int i = order[j];
            cg_report *ri = reports ? &reports[i] : nullptr;
            cudaStream_t st = (cudaStream_t)streams[i];
            const SharedDeposit *dep = in_dep[i] ? &sdep[i] : nullptr;
            if (host[i])
                status[i] = coarse_grain_host_impl(meshes[i], n[i], pos[i], nfields, w[i], cells[i], &params[i],
                                                   ri, st, sh_pos[i], sh_w[i], sh_ev[i], dep);
            else if (dep)
                status[i] = coarse_grain_from_shared(meshes[i], nfields, cells[i], &params[i], ri, st, *dep);
            else
                status[i] = cg_coarse_grain(meshes[i], n[i], pos[i], nfields, w[i], cells[i], &params[i], ri,
                                            streams[i]);
            if (status[i] != CG_OK) detail[i] = g_last_error;   // this thread's message
        }
    };
    std::vector<std::thread> pool;
    const int nthreads = std::min(max_concurrent, nprob);
    for (int t = 1; t < nthreads; ++t) {
        try {
            pool.emplace_back(worker, true);
        } catch (...) {
            break;   // fewer workers: the remaining problems run on the threads there are
        }
    }
    worker(false);
    for (std::thread &t : pool) t.join();
    if (next.load() < nprob)   // a worker could not select the device: finish here
        worker(false);
    for (cudaEvent_t ev : events) cudaEventDestroy(ev);
    for (int i = 0; i < nprob; ++i)
        if (status[i] != CG_OK) return fail(status[i], "problem %d: %s", i, detail[i].c_str());
    return CG_OK;
}

cg_status cg_coarse_grain_host(cg_mesh *m, int64_t n, const double *pos_host, int nfields,
                               const double *w_host, double *cells_host, const cg_params *p,
                               cg_report *rep, void *stream) {
    return coarse_grain_host_impl(m, n, pos_host, nfields, w_host, cells_host, p, rep,
                                  (cudaStream_t)stream, nullptr, nullptr, nullptr);
}

}  // extern "C"

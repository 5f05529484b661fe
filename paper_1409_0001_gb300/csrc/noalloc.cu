// noalloc.cu -- cg_deposit_fixed_noalloc: the fixed-point deposition of cg_deposit for
// callers that must not allocate device memory during a call.
//
// Its scratch (error counters, per-field max |w|, and the 64-bit accumulators) lives in
// the file-scope array below, part of this library's static device memory: every GPU
// that loads this module holds it (8 * (128 + CG_NOALLOC_MAX_CELL_FIELDS) bytes) until the
// process exits.
// The array is shared by every call on a device and keeps the previous call's contents,
// so each call clears what must start at zero; calls that overlap on the GPU race.
#include <cuda_runtime.h>
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace cgk {
namespace {

constexpr int kNoallocHeader = 128;   // [0..2) counters, [64..128) max |w| bits
constexpr int kThreads = 256;

static __device__ __align__(256) unsigned long long
    g_noalloc_scratch[kNoallocHeader + CG_NOALLOC_MAX_CELL_FIELDS];

// Device address of g_noalloc_scratch per device (host code may not use the symbol's
// name as an address: it is a host-side stand-in).  Under CUDA's lazy module loading
// (the default) the array is placed in device memory when this file's module first
// loads on a device, i.e. by the first call there; a device reset (cudaDeviceReset)
// invalidates the cached address, and calls after one must not follow.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

cg_status scratch_for_current_device(unsigned long long **out) {
    int dev = 0;
    CGK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(CG_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned long long *>(g_scratch_ptr[dev]);
    return CG_OK;
}

struct Box {
    int nx, ny, nz;
    double ox, oy, oz, inv_dx, hx, hy, hz;
};

struct Scales {
    double scale[CG_NOALLOC_MAX_FIELDS];
    double unscale[CG_NOALLOC_MAX_FIELDS];
};

__device__ __forceinline__ int cell_of(const Box &b, double x, double y, double z) {
    bool inside = (x >= b.ox) && (x <= b.hx) && (y >= b.oy) && (y <= b.hy) && (z >= b.oz) &&
                  (z <= b.hz);
    if (!inside) return -1;
    int ix = (int)floor(__dmul_rn(__dsub_rn(x, b.ox), b.inv_dx));
    int iy = (int)floor(__dmul_rn(__dsub_rn(y, b.oy), b.inv_dx));
    int iz = (int)floor(__dmul_rn(__dsub_rn(z, b.oz), b.inv_dx));
    ix = min(max(ix, 0), b.nx - 1);
    iy = min(max(iy, 0), b.ny - 1);
    iz = min(max(iz, 0), b.nz - 1);
    return (iz * b.ny + iy) * b.nx + ix;
}

// pass 1: count particles outside the box and non-finite weights; max |w| per field
__global__ void k_noalloc_validate(Box b, int64_t n, const double *__restrict__ pos, int nf,
                                   const double *__restrict__ w,
                                   unsigned long long *__restrict__ scratch) {
    unsigned long long n_out = 0, n_bad = 0;
    unsigned long long mx[CG_NOALLOC_MAX_FIELDS] = {};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (cell_of(b, pos[i], pos[n + i], pos[2 * n + i]) < 0) ++n_out;
        for (int f = 0; f < nf; ++f) {
            double v = w[(int64_t)f * n + i];
            if (!isfinite(v)) ++n_bad;
            unsigned long long bits = (unsigned long long)__double_as_longlong(fabs(v));
            mx[f] = bits > mx[f] ? bits : mx[f];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        n_out += __shfl_down_sync(0xffffffffu, n_out, o);
        n_bad += __shfl_down_sync(0xffffffffu, n_bad, o);
        for (int f = 0; f < nf; ++f) {
            unsigned long long t = __shfl_down_sync(0xffffffffu, mx[f], o);
            mx[f] = t > mx[f] ? t : mx[f];
        }
    }
    if ((threadIdx.x & 31) == 0) {
        if (n_out) atomicAdd(&scratch[0], n_out);
        if (n_bad) atomicAdd(&scratch[1], n_bad);
        for (int f = 0; f < nf; ++f)
            if (mx[f]) atomicMax(&scratch[64 + f], mx[f]);
    }
}

// pass 2: q = round-half-even(w * 2^F) added into the cell's int64 accumulator
__global__ void k_noalloc_accum(Box b, int64_t n, const double *__restrict__ pos, int nf,
                                const double *__restrict__ w, Scales s, int64_t ncells,
                                unsigned long long *__restrict__ acc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int c = cell_of(b, pos[i], pos[n + i], pos[2 * n + i]);
        if (c < 0) continue;
        for (int f = 0; f < nf; ++f) {
            long long q = __double2ll_rn(__dmul_rn(w[(int64_t)f * n + i], s.scale[f]));
            atomicAdd(&acc[(int64_t)f * ncells + c], (unsigned long long)q);
        }
    }
}

// pass 3: eps = ((double)sum * 2^-F) / V_c
__global__ void k_noalloc_finalize(int64_t ncells, int nf, const unsigned long long *__restrict__ acc,
                                   Scales s, double vc, double *__restrict__ out) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells;
         c += (int64_t)gridDim.x * blockDim.x)
        for (int f = 0; f < nf; ++f) {
            double x = __dmul_rn(__ll2double_rn((long long)acc[(int64_t)f * ncells + c]), s.unscale[f]);
            out[(int64_t)f * ncells + c] = __ddiv_rn(x, vc);
        }
}

int grid_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)num_sms() * 8;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace
}  // namespace cgk

using namespace cgk;

extern "C" cg_status cg_deposit_fixed_noalloc(int nx, int ny, int nz, const double origin[3],
                                              double dx, int64_t n, const double *pos,
                                              int nfields, const double *w, double *cells_out,
                                              int *fixed_point_bits_host, void *stream) {
    if (!origin || !cells_out) return fail(CG_EINVAL, "origin and cells_out must not be NULL");
    if (nx < 1 || ny < 1 || nz < 1) return fail(CG_EINVAL, "mesh dimensions must be >= 1");
    if (!(dx > 0.0) || !std::isfinite(dx)) return fail(CG_EINVAL, "dx must be finite and > 0");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(origin[a])) return fail(CG_EINVAL, "origin must be finite");
    if (nfields < 1 || nfields > CG_NOALLOC_MAX_FIELDS)
        return fail(CG_EINVAL, "nfields must be in [1, %d]", CG_NOALLOC_MAX_FIELDS);
    // the cell count is bounded before it is formed, so that no product overflows
    if (!cells_below(nx, ny, nz, (int64_t)CG_NOALLOC_MAX_CELL_FIELDS / nfields + 1))
        return fail(CG_EINVAL,
                    "cg_deposit_fixed_noalloc: nfields * nx * ny * nz (%d * %d * %d * %d) "
                    "exceeds the static scratch of %d accumulators",
                    nfields, nx, ny, nz, CG_NOALLOC_MAX_CELL_FIELDS);
    const int64_t ncells = (int64_t)nx * ny * nz;
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(CG_EINVAL, "n must be in [0, 2^31)");
    if (n > 0 && (!pos || !w)) return fail(CG_EINVAL, "pos and w must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;

    Box b;
    b.nx = nx;
    b.ny = ny;
    b.nz = nz;
    const int dims[3] = {nx, ny, nz};
    double hi[3];
    for (int a = 0; a < 3; ++a) {
        volatile double len = (double)dims[a] * dx;   // two roundings, as cg_locate defines
        hi[a] = origin[a] + len;
        if (!std::isfinite(hi[a])) return fail(CG_EINVAL, "origin + n * dx must be finite");
    }
    b.ox = origin[0];
    b.oy = origin[1];
    b.oz = origin[2];
    b.inv_dx = 1.0 / dx;
    b.hx = hi[0];
    b.hy = hi[1];
    b.hz = hi[2];

    unsigned long long *scratch = nullptr;
    CGK_TRY(scratch_for_current_device(&scratch));
    unsigned long long *acc = scratch + kNoallocHeader;

    // clear the counters, the maxima and this call's accumulators
    CGK_CUDA(cudaMemsetAsync(scratch, 0, (kNoallocHeader + (size_t)ncells * nfields) * 8, st));
    if (n > 0) {
        k_noalloc_validate<<<grid_for(n), kThreads, 0, st>>>(b, n, pos, nfields, w, scratch);
        CGK_CUDA(cudaGetLastError());
    }
    unsigned long long head[kNoallocHeader];
    CGK_CUDA(cudaMemcpyAsync(head, scratch, sizeof(head), cudaMemcpyDeviceToHost, st));
    CGK_CUDA(cudaStreamSynchronize(st));
    if (head[1]) return fail(CG_EINVAL, "cg_deposit_fixed_noalloc: %llu non-finite weights", head[1]);
    if (head[0]) return fail(CG_EDOMAIN, "cg_deposit_fixed_noalloc: %llu particles outside the mesh", head[0]);

    // F = 61 - e(max|w|) - e(n) with frexp exponents, clamped to [-1000, 1000]
    Scales s;
    for (int f = 0; f < nfields; ++f) {
        double m;
        std::memcpy(&m, &head[64 + f], 8);
        int F = 0;
        if (n > 0 && m > 0.0) {
            int em = 0, en = 0;
            std::frexp(m, &em);
            std::frexp((double)n, &en);
            F = 61 - em - en;
            F = F > 1000 ? 1000 : (F < -1000 ? -1000 : F);
        }
        s.scale[f] = std::ldexp(1.0, F);
        s.unscale[f] = std::ldexp(1.0, -F);
        if (fixed_point_bits_host) fixed_point_bits_host[f] = F;
    }
    if (n > 0) {
        k_noalloc_accum<<<grid_for(n), kThreads, 0, st>>>(b, n, pos, nfields, w, s, ncells, acc);
        CGK_CUDA(cudaGetLastError());
    }
    k_noalloc_finalize<<<grid_for(ncells), kThreads, 0, st>>>(ncells, nfields, acc, s,
                                                              (dx * dx) * dx, cells_out);
    CGK_CUDA(cudaGetLastError());
    CGK_CUDA(cudaStreamSynchronize(st));
    return CG_OK;
}

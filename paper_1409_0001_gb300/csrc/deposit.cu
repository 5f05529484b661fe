// deposit.cu -- particle centroid method on the GPU (Section 2.2, Section 3.1
// Eq. (pcm-k)): locate each particle's host cell, then sum the particles' carried
// quantities per cell and divide by the cell volume.
//
// Ordered mode reproduces a sequential loop over particles bit for bit: the
// (cell, particle) pairs are put in cell order by a stable LSD radix sort on the
// cell id (particle order is kept inside a cell), and the first position of each
// cell's segment adds the segment's weights in that order, in FP64 starting from
// +0.0, then divides by V_c with an IEEE division.  Fixed-point mode quantises w * 2^F to int64 (round half to
// even) and adds with 64-bit integer atomics, which is exact and order-free.
#include <cuda_runtime.h>
#include <cmath>
#include <vector>
#include <cstdio>
#include <cstring>

#include "internal.cuh"

namespace cgk {

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t n, int per_block = kThreads, int max_blocks_per_sm = 8) {
    int64_t b = (n + per_block - 1) / per_block;
    int64_t cap = (int64_t)num_sms() * max_blocks_per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// --------------------------------------------------------------------------- locate
// Host cell per axis: i = floor(fl(fl(x - x0) * inv_dx)) clamped into [0, n-1]; outside
// unless x0 <= x <= hi on every axis (NaN is outside).  FP64 arithmetic is slow on this
// GPU, so the result is first taken from an FP32 estimate with a rigorous error bound,
// and the FP64 definition (explicitly rounded intrinsics, no contraction) is evaluated
// only when the bound does not keep the estimate away from an integer -- the answer is
// the FP64 definition's either way.  The domain test compares doubles exactly as
// ordered integer keys.

// A double as a 64-bit key in the order of the doubles (-0 as +0; a NaN sorts above +inf
// or below -inf by its sign, so it fails one side of a range test).
__device__ __forceinline__ unsigned long long dkey(double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    if (b == 0x8000000000000000ull) b = 0;
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// A float carrying the sign, exponent and top 20 fraction bits of v (relative error
// below 2^-20); ok is cleared outside float's normal range.  Zero maps to zero.
__device__ __forceinline__ float approx20(double v, bool &ok) {
    const int hi = __double2hiint(v);
    const unsigned int lo = (unsigned int)__double2loint(v);
    const int e = (hi >> 20) & 0x7ff;
    const unsigned int frac = (unsigned int)hi & 0xfffffu;
    if (e == 0 && frac == 0 && lo == 0) return 0.0f;
    const int e32 = e - 1023 + 127;
    if (e32 < 1 || e32 > 254) {
        ok = false;
        return 0.0f;
    }
    return __int_as_float((int)(((unsigned int)hi & 0x80000000u) | ((unsigned int)e32 << 23) | (frac << 3)));
}

// The FP64 definition itself, out of line so that it is not evaluated speculatively for
// every particle.
__device__ __noinline__ int cell_index_exact(double x, double o, double inv) {
    return (int)floor(__dmul_rn(__dsub_rn(x, o), inv));
}

// floor(fl(fl(x - o) * inv)) for x >= o.  With xf = approx20(x), of and invf the FP32
// roundings of o and inv, rf = (xf - of) * invf differs from the FP64 value by less than
// (|xf| + |of|) invf 2^-20 (1 + 2^-20) + 3 |rf| 2^-24 + 2 |rf| 2^-53; the bound used is
// four times the first term plus 2^-18 |rf|.  If rf's fraction clears it on both sides,
// both values have the same floor.
__device__ __forceinline__ int cell_index(double x, double o, double inv, float of, float invf) {
    bool ok = true;
    const float xf = approx20(x, ok);
    const float rf = (xf - of) * invf;
    const float bound = (fabsf(xf) + fabsf(of)) * invf * 0x1p-18f + fabsf(rf) * 0x1p-18f;
    const float fl = floorf(rf);
    const float fr = rf - fl;   // exact (Sterbenz)
    if (ok && rf >= 0.0f && rf < 4194304.0f && fr > bound && fr < 1.0f - bound) return (int)fl;
    return cell_index_exact(x, o, inv);
}

__global__ void k_locate_structured(int64_t n, const double *__restrict__ pos, int nx, int ny,
                                    int nz, double ox, double oy, double oz, double inv_dx,
                                    double hx, double hy, double hz, float oxf, float oyf,
                                    float ozf, float invf, int nf, const double *__restrict__ w,
                                    int32_t *__restrict__ cell, uint32_t *__restrict__ counts,
                                    uint32_t *__restrict__ ranks,
                                    unsigned long long *__restrict__ bad) {
    unsigned long long n_out = 0, n_nonfinite = 0;
    uint32_t most = 0;   // largest per-cell count seen (counts != nullptr)
    const unsigned long long kox = dkey(ox), koy = dkey(oy), koz = dkey(oz);
    const unsigned long long khx = dkey(hx), khy = dkey(hy), khz = dkey(hz);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = pos[i], y = pos[n + i], z = pos[2 * n + i];
        for (int f = 0; f < nf; ++f)
            if (((__double2hiint(w[(int64_t)f * n + i]) >> 20) & 0x7ff) == 0x7ff) ++n_nonfinite;
        const unsigned long long kx = dkey(x), ky = dkey(y), kz = dkey(z);
        const bool inside = kx >= kox && kx <= khx && ky >= koy && ky <= khy && kz >= koz && kz <= khz;
        int32_t c = -1;
        if (inside) {
            int ix = cell_index(x, ox, inv_dx, oxf, invf);
            int iy = cell_index(y, oy, inv_dx, oyf, invf);
            int iz = cell_index(z, oz, inv_dx, ozf, invf);
            ix = min(max(ix, 0), nx - 1);
            iy = min(max(iy, 0), ny - 1);
            iz = min(max(iz, 0), nz - 1);
            c = (int32_t)(((int64_t)iz * ny + iy) * nx + ix);
            if (counts) {   // the arrival rank orders nothing: it only picks a free slot
                const uint32_t r = atomicAdd(&counts[c], 1u);
                if (ranks) ranks[i] = r;
                most = max(most, r + 1u);
            }
        } else {
            ++n_out;
        }
        cell[i] = c;
    }
    // warp-aggregate the rare error counters and the largest count
    for (int o = 16; o > 0; o >>= 1) {
        n_out += __shfl_down_sync(0xffffffffu, n_out, o);
        n_nonfinite += __shfl_down_sync(0xffffffffu, n_nonfinite, o);
        most = max(most, __shfl_down_sync(0xffffffffu, most, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (n_out) atomicAdd(&bad[0], n_out);
        if (n_nonfinite) atomicAdd(&bad[1], n_nonfinite);
        if (most) atomicMax(&bad[2], (unsigned long long)most);
    }
}

// --------------------------------------------------------------------------- scan
constexpr int kScanItems = 16;
constexpr int kScanChunk = kThreads * kScanItems;  // 4096 values per block

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t warp_sums[kThreads / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < kThreads / 32 ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane < kThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    uint32_t warp_off = warp ? warp_sums[warp - 1] : 0;
    uint32_t tot = warp_sums[kThreads / 32 - 1];
    __syncthreads();
    if (total) *total = tot;
    return warp_off + inc - v;
}

__global__ void k_scan_reduce(const uint32_t *__restrict__ in, int64_t n,
                              uint32_t *__restrict__ block_sums) {
    int64_t base = (int64_t)blockIdx.x * kScanChunk;
    uint32_t s = 0;
    for (int j = threadIdx.x; j < kScanChunk; j += kThreads) {
        int64_t i = base + j;
        if (i < n) s += in[i];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ uint32_t ws[kThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += ws[w];
        block_sums[blockIdx.x] = t;
    }
}

// single block: exclusive scan of nb block sums, in place
__global__ void k_scan_top(uint32_t *__restrict__ sums, int64_t nb) {
    uint32_t carry = 0;
    for (int64_t base = 0; base < nb; base += kThreads) {
        int64_t i = base + threadIdx.x;
        uint32_t v = i < nb ? sums[i] : 0;
        uint32_t tot;
        uint32_t ex = block_exclusive_scan(v, &tot);
        if (i < nb) sums[i] = carry + ex;
        carry += tot;
    }
}

__global__ void k_scan_down(const uint32_t *in, uint32_t *out, int64_t n,
                            const uint32_t *__restrict__ block_off) {
    __shared__ uint32_t tile[kScanChunk + kScanChunk / 32];
    int64_t base = (int64_t)blockIdx.x * kScanChunk;
    for (int j = threadIdx.x; j < kScanChunk; j += kThreads) {
        int64_t i = base + j;
        tile[j + (j >> 5)] = i < n ? in[i] : 0;
    }
    __syncthreads();
    uint32_t v[kScanItems];
    uint32_t s = 0;
    int t0 = threadIdx.x * kScanItems;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        int j = t0 + q;
        v[q] = tile[j + (j >> 5)];
        s += v[q];
    }
    __syncthreads();
    uint32_t ex = block_exclusive_scan(s, nullptr) + block_off[blockIdx.x];
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        int j = t0 + q;
        tile[j + (j >> 5)] = ex;
        ex += v[q];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < kScanChunk; j += kThreads) {
        int64_t i = base + j;
        if (i < n) out[i] = tile[j + (j >> 5)];
    }
}

// --------------------------------------------------------------------------- radix sort
// Stable LSD radix sort of 32-bit keys (cell ids) carrying 32-bit values (particle
// ids), 8-bit digits.  A tile of 4096 keys per 256-thread block; inside a tile warp w
// owns keys [w*512, (w+1)*512) in 16 rounds of 32 consecutive keys, and ranks each
// key among equal digits with __match_any_sync, so ranks follow input order.
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortItems = 16;
constexpr int kSortWarps = kThreads / 32;
constexpr int kTile = kThreads * kSortItems;

__global__ void __launch_bounds__(kThreads) k_radix_upsweep(const uint32_t *__restrict__ keys,
                                                           int64_t n, int shift,
                                                           uint32_t *__restrict__ hist,
                                                           int ntiles) {
    __shared__ uint32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kTile;
    for (int j = threadIdx.x; j < kTile; j += kThreads) {
        int64_t i = base + j;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads) k_radix_downsweep(
    const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
    uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, int64_t n, int shift,
    const uint32_t *__restrict__ hist_scan, int ntiles) {
    __shared__ uint32_t wcnt[kSortWarps][kRadix];
    __shared__ uint32_t gbase[kRadix];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = threadIdx.x; j < kSortWarps * kRadix; j += kThreads) (&wcnt[0][0])[j] = 0;
    gbase[threadIdx.x] = hist_scan[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();

    const int64_t wbase = (int64_t)blockIdx.x * kTile + (int64_t)warp * (32 * kSortItems);
    const unsigned lt = (1u << lane) - 1u;
    uint32_t k[kSortItems], v[kSortItems], rk[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int64_t i = wbase + r * 32 + lane;
        bool valid = i < n;
        uint32_t key = valid ? keys_in[i] : 0u;
        uint32_t d = (key >> shift) & (kRadix - 1);
        uint32_t tag = valid ? d : (0x10000u + lane);   // invalid lanes stay alone
        unsigned peers = __match_any_sync(0xffffffffu, tag);
        unsigned rank = __popc(peers & lt);
        uint32_t old = valid ? wcnt[warp][d] : 0u;
        __syncwarp();
        if (valid && rank == 0) wcnt[warp][d] = old + __popc(peers);
        __syncwarp();
        k[r] = key;
        v[r] = valid ? (vals_in ? vals_in[i] : (uint32_t)i) : 0u;
        rk[r] = old + rank;
    }
    __syncthreads();
    {   // exclusive prefix over warps for digit threadIdx.x
        uint32_t run = 0;
        for (int w = 0; w < kSortWarps; ++w) {
            uint32_t t = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int64_t i = wbase + r * 32 + lane;
        if (i < n) {
            uint32_t d = (k[r] >> shift) & (kRadix - 1);
            uint32_t dst = gbase[d] + wcnt[warp][d] + rk[r];
            keys_out[dst] = k[r];
            vals_out[dst] = v[r];
        }
    }
}

// --------------------------------------------------------------------------- sums
// One thread per position p of the cell-sorted particle list; the first position of
// each cell's segment sums the segment's weights in ascending particle index (FP64,
// from +0.0) and writes eps = S / V_c.  Cells without particles keep the +0.0 the
// output was cleared to (0.0 / V_c = +0.0).
// eps = S / V_c with an IEEE division (Eq. (pcm-k)).  When every cell has the same volume
// and it is an exact power of two, its reciprocal is exact too and S * (1 / V_c) is the
// same correctly rounded value as S / V_c (scaling by a power of two, rounded once), at
// the cost of one multiplication; inv_pow2 is that reciprocal, or 0 to divide.
__device__ __forceinline__ double div_vc(double S, double v, double inv_pow2) {
    return inv_pow2 != 0.0 ? __dmul_rn(S, inv_pow2) : __ddiv_rn(S, v);
}

__global__ void k_segment_heads(int64_t n, const uint32_t *__restrict__ keys,
                                const uint32_t *__restrict__ sorted_idx, int nf,
                                const double *__restrict__ w, int64_t ncells,
                                const double *__restrict__ vc, double vc_uniform, double inv_pow2,
                                double *__restrict__ out) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = keys[p];
        if (p > 0 && keys[p - 1] == c) continue;
        int64_t e = p + 1;
        while (e < n && keys[e] == c) ++e;
        const double v = vc ? vc[c] : vc_uniform;
        for (int f = 0; f < nf; ++f) {
            const double *wf = w + (int64_t)f * n;
            double acc = 0.0;
            for (int64_t q = p; q < e; ++q) acc = __dadd_rn(acc, wf[sorted_idx[q]]);
            out[(int64_t)f * ncells + c] = div_vc(acc, v, inv_pow2);
        }
    }
}

// Counting path of the ordered sums (cells holding at most kSegMax particles): each
// particle goes to the slot of its cell's segment given by its arrival rank at the
// cell's counter (so the order inside a segment is arbitrary), then one thread per cell
// sorts its segment's particle ids and adds the weights in ascending particle index.
constexpr int kSegMax = 64;

__global__ void k_scatter_cells(int64_t n, const int32_t *__restrict__ cell,
                                const uint32_t *__restrict__ off, const uint32_t *__restrict__ ranks,
                                uint32_t *__restrict__ idx) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        idx[off[cell[i]] + ranks[i]] = (uint32_t)i;
}

// eps_c = (sum of the cell's weights in ascending particle index, FP64 from +0.0) / V_c;
// an empty cell gets +0.0.
__global__ void k_cell_sums(int64_t ncells, const uint32_t *__restrict__ off,
                            const uint32_t *__restrict__ idx, int nf,
                            const double *__restrict__ w, int64_t n,
                            const double *__restrict__ vc, double vc_uniform, double inv_pow2,
                            double *__restrict__ out) {
    uint32_t s[kSegMax];
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells;
         c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t beg = off[c];
        const int k = (int)(off[c + 1] - beg);
        if (k == 0) {
            for (int f = 0; f < nf; ++f) out[(int64_t)f * ncells + c] = 0.0;
            continue;
        }
        for (int j = 0; j < k; ++j) {   // insertion sort of the segment's ids
            const uint32_t v = idx[beg + j];
            int q = j;
            while (q > 0 && s[q - 1] > v) {
                s[q] = s[q - 1];
                --q;
            }
            s[q] = v;
        }
        const double v = vc ? vc[c] : vc_uniform;
        for (int f = 0; f < nf; ++f) {
            const double *wf = w + (int64_t)f * n;
            double acc = 0.0;
            for (int j = 0; j < k; ++j) acc = __dadd_rn(acc, wf[s[j]]);
            out[(int64_t)f * ncells + c] = div_vc(acc, v, inv_pow2);
        }
    }
}

// max |w| per field as the bit pattern of a non-negative double (orders like uint64)
__global__ void k_absmax(int64_t n, int nf, const double *__restrict__ w,
                         unsigned long long *__restrict__ out) {
    int f = blockIdx.y;
    const double *wf = w + (int64_t)f * n;
    unsigned long long m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long b = (unsigned long long)__double_as_longlong(fabs(wf[i]));
        m = b > m ? b : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_down_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&out[f], m);
}

__global__ void k_fixed_accum(int64_t n, const int32_t *__restrict__ cell, int nf,
                              const double *__restrict__ w, const double *__restrict__ scale,
                              unsigned long long *__restrict__ acc, int64_t ncells) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = cell[i];
        if (c < 0) continue;
        for (int f = 0; f < nf; ++f) {
            long long q = __double2ll_rn(__dmul_rn(w[(int64_t)f * n + i], scale[f]));
            atomicAdd(&acc[(int64_t)f * ncells + c], (unsigned long long)q);
        }
    }
}

__global__ void k_fixed_finalize(int64_t ncells, int nf,
                                 const unsigned long long *__restrict__ acc,
                                 const double *__restrict__ unscale,
                                 const double *__restrict__ vc, double vc_uniform, double inv_pow2,
                                 double *__restrict__ out) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells;
         c += (int64_t)gridDim.x * blockDim.x) {
        double v = vc ? vc[c] : vc_uniform;
        for (int f = 0; f < nf; ++f) {
            long long s = (long long)acc[(int64_t)f * ncells + c];
            double x = __dmul_rn(__ll2double_rn(s), unscale[f]);
            out[(int64_t)f * ncells + c] = div_vc(x, v, inv_pow2);
        }
    }
}

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

}  // namespace

// ============================================================================ host side
size_t scan_tmp_words(int64_t n) {
    int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    return (size_t)(nb > 0 ? nb : 1);
}

cg_status exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *tmp,
                             cudaStream_t st) {
    if (n <= 0) return CG_OK;
    int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    CGK_LAUNCH("scan_reduce", (double)n * 4, st,
               k_scan_reduce<<<(unsigned)nb, kThreads, 0, st>>>(in, n, tmp));
    CGK_LAUNCH("scan_top", (double)nb * 8, st, k_scan_top<<<1, kThreads, 0, st>>>(tmp, nb));
    CGK_LAUNCH("scan_down", (double)n * 8, st,
               k_scan_down<<<(unsigned)nb, kThreads, 0, st>>>(in, out, n, tmp));
    CGK_CUDA(cudaGetLastError());
    return CG_OK;
}

// Forward declaration of the tet locate launcher (tet.cu).
cg_status tet_locate_launch(cg_mesh *m, int64_t n, const double *pos, int nf, const double *w,
                            int32_t *cell_out, uint32_t *counts, uint32_t *ranks,
                            unsigned long long *bad, cudaStream_t st);

// The point location and its counters (outside particles, non-finite weights, the most
// particles in one cell), copied to the mesh's pinned readback buffer; nothing is waited
// for (locate_read takes the counters once the stream has synchronised).
static cg_status locate_launch(cg_mesh *m, int64_t n, const double *pos, int nf, const double *w,
                               int32_t *cell_out, uint32_t *counts, uint32_t *ranks, cudaStream_t st) {
    CGK_TRY(m->ws_small.ensure(4096));
    CGK_TRY(m->h_small.ensure(4096));
    unsigned long long *bad = m->ws_small.as<unsigned long long>();
    CGK_CUDA(cudaMemsetAsync(bad, 0, 3 * sizeof(unsigned long long), st));
    if (n > 0) {
        if (m->kind == MESH_STRUCTURED) {
            double hi[3];
            const int dims[3] = {m->nx, m->ny, m->nz};
            for (int a = 0; a < 3; ++a) {
                volatile double len = (double)dims[a] * m->dx;   // two roundings, as defined
                hi[a] = m->origin[a] + len;
            }
            double inv_dx = 1.0 / m->dx;
            CGK_LAUNCH("locate_structured", (double)n * (24 + 8 * nf + 4), st,
                       k_locate_structured<<<grid_for(n), kThreads, 0, st>>>(
                           n, pos, m->nx, m->ny, m->nz, m->origin[0], m->origin[1],
                           m->origin[2], inv_dx, hi[0], hi[1], hi[2], (float)m->origin[0],
                           (float)m->origin[1], (float)m->origin[2], (float)inv_dx, nf, w,
                           cell_out, counts, ranks, bad));
            CGK_CUDA(cudaGetLastError());
        } else {
            CGK_TRY(tet_locate_launch(m, n, pos, nf, w, cell_out, counts, ranks, bad, st));
        }
    }
    CGK_CUDA(cudaMemcpyAsync(m->h_small.as<unsigned long long>(), bad, 3 * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, st));
    return CG_OK;
}

static void locate_read(const cg_mesh *m, int64_t *n_out, int64_t *n_nonfinite, uint32_t *max_count) {
    const unsigned long long *hb = m->h_small.as<unsigned long long>();
    if (n_out) *n_out = (int64_t)hb[0];
    if (n_nonfinite) *n_nonfinite = (int64_t)hb[1];
    if (max_count) *max_count = (uint32_t)hb[2];
}

cg_status locate_run(cg_mesh *m, int64_t n, const double *pos, int nf, const double *w,
                     int32_t *cell_out, uint32_t *counts, int64_t *n_out, int64_t *n_nonfinite,
                     cudaStream_t st, uint32_t *max_count, uint32_t *ranks) {
    CGK_TRY(locate_launch(m, n, pos, nf, w, cell_out, counts, ranks, st));
    CGK_CUDA(cudaStreamSynchronize(st));
    locate_read(m, n_out, n_nonfinite, max_count);
    return CG_OK;
}

// Scale exponent of the fixed-point mode: with m = max|w| = fm*2^em, n = fn*2^en
// (frexp), F = 61 - em - en (so n*m*2^F < 2^61), F = 0 if m == 0, clamped to
// [-1000, 1000] so that the scales and every rescaled non-zero sum stay normal.
static int fixed_bits(int64_t n, double maxabs) {
    if (n <= 0 || !(maxabs > 0.0)) return 0;
    int em = 0, en = 0;
    std::frexp(maxabs, &em);
    std::frexp((double)n, &en);
    int F = 61 - em - en;
    return F > 1000 ? 1000 : (F < -1000 ? -1000 : F);
}

// The quantities of a deposition that both its phases use (workspace layout, cell volume).
struct DepositPlan {
    int64_t ncells;
    int mode;
    const double *vc;
    double vcu, inv_pow2;
    bool ordered;
    size_t s_cell, s_cnt;
    int32_t *cell;
    uint32_t *counts, *ranks;
};

// Phase 1 of a deposition: the workspace, the cleared per-cell counters and the point
// location (locate_launch); nothing is waited for.
static cg_status deposit_begin(cg_mesh *m, int64_t n, const double *pos, int nf, const double *w,
                               const cg_params *p, cudaStream_t st, DepositPlan &dp) {
    const int64_t ncells = m->ncells;
    const int mode = p->deposit_mode;
    const double *vc = m->kind != MESH_STRUCTURED ? m->tet.vc : nullptr;
    const double vcu = m->kind != MESH_STRUCTURED ? 0.0 : (m->dx * m->dx) * m->dx;
    // a uniform cell volume that is a power of two (dx = 2^-k): divide by multiplying
    double inv_pow2 = 0.0;
    if (vc == nullptr && vcu > 0.0 && std::isfinite(vcu)) {
        int e = 0;
        const double mant = std::frexp(vcu, &e);
        const double inv = std::ldexp(1.0, 1 - e);   // 1 / vcu when vcu = 2^(e-1)
        if (mant == 0.5 && std::isnormal(inv)) inv_pow2 = inv;
    }

    // workspace: cell[n] (int32); the ordered mode also counts particles per cell
    // (ncells + 1 counters, the last one staying 0 for the exclusive scan)
    // and keeps each particle's arrival rank at its cell's counter
    const bool ordered = mode == CG_DEPOSIT_ORDERED;
    const size_t s_cell = align_up((size_t)(n > 0 ? n : 1) * 4);
    const size_t s_cnt = align_up((size_t)(ncells + 1) * 4);
    CGK_TRY(m->ws_locate.ensure(s_cell + (ordered ? s_cnt + s_cell : 0)));
    int32_t *cell = m->ws_locate.as<int32_t>();
    uint32_t *counts = ordered ? (uint32_t *)(m->ws_locate.as<char>() + s_cell) : nullptr;
    uint32_t *ranks = ordered ? (uint32_t *)(m->ws_locate.as<char>() + s_cell + s_cnt) : nullptr;
    if (counts) CGK_CUDA(cudaMemsetAsync(counts, 0, (size_t)(ncells + 1) * 4, st));
    dp = DepositPlan{ncells, mode, vc, vcu, inv_pow2, ordered, s_cell, s_cnt, cell, counts, ranks};
    return locate_launch(m, n, pos, nf, w, cell, counts, ranks, st);
}

// Phase 2, once the stream has synchronised after phase 1: the location's counters are
// checked (CG_EINVAL for non-finite weights, CG_EDOMAIN for particles outside the mesh,
// before anything is written to out), then the per-cell sums run.
static cg_status deposit_end(cg_mesh *m, int64_t n, int nf, const double *w, double *out,
                             cg_report *rep, cudaStream_t st, const DepositPlan &dp) {
    const int64_t ncells = dp.ncells;
    const double *vc = dp.vc;
    const double vcu = dp.vcu, inv_pow2 = dp.inv_pow2;
    const bool ordered = dp.ordered;
    const size_t s_cnt = dp.s_cnt;
    int32_t *cell = dp.cell;
    uint32_t *counts = dp.counts, *ranks = dp.ranks;
    int64_t n_out = 0, n_bad = 0;
    uint32_t max_count = 0;
    locate_read(m, &n_out, &n_bad, counts ? &max_count : nullptr);
    if (rep) rep->n_out_of_domain = n_out;
    if (n_bad) return fail(CG_EINVAL, "cg_deposit: %lld non-finite weights", (long long)n_bad);
    if (n_out)
        return fail(CG_EDOMAIN, "cg_deposit: %lld particles outside the mesh", (long long)n_out);

    if (ordered && max_count <= (uint32_t)kSegMax) {
        // counting sort by cell: offsets = exclusive scan of the counts, a scatter into the
        // segments, then per cell the segment's ids in ascending order and the ordered sum
        const size_t s_off = s_cnt;
        const size_t s_idx = align_up((size_t)(n > 0 ? n : 1) * 4);
        const size_t s_tmp = align_up(scan_tmp_words(ncells + 1) * 4);
        CGK_TRY(m->ws_sort.ensure(s_off + s_idx + s_tmp));
        char *sb = m->ws_sort.as<char>();
        uint32_t *off = (uint32_t *)sb, *idx = (uint32_t *)(sb + s_off);
        uint32_t *tmp = (uint32_t *)(sb + s_off + s_idx);
        CGK_TRY(exclusive_scan_u32(counts, off, ncells + 1, tmp, st));
        if (n > 0) {
            CGK_LAUNCH("scatter_cells", (double)n * 16, st,
                       k_scatter_cells<<<grid_for(n), kThreads, 0, st>>>(n, cell, off, ranks, idx));
            CGK_CUDA(cudaGetLastError());
        }
        CGK_LAUNCH("cell_sums", (double)n * (4 + 8 * nf) + (double)ncells * (4 + 8 * nf), st,
                   k_cell_sums<<<grid_for(ncells), kThreads, 0, st>>>(ncells, off, idx, nf, w, n,
                                                                      vc, vcu, inv_pow2, out));
        CGK_CUDA(cudaGetLastError());
        if (rep)
            for (int f = 0; f < nf && f < CG_REPORT_MAX_FIELDS; ++f) rep->fixed_point_bits[f] = 0;
    } else if (ordered) {
        // a crowded cell: stable sort of (cell, particle) by cell
        int bits = 1;
        while (bits < 32 && ((int64_t)1 << bits) < ncells) ++bits;
        int passes = (bits + kRadixBits - 1) / kRadixBits;
        int64_t ntiles = (n + kTile - 1) / kTile;
        if (ntiles < 1) ntiles = 1;
        int64_t hist_n = (int64_t)kRadix * ntiles;
        size_t s_keys = align_up((size_t)n * 4);
        size_t s_hist = align_up((size_t)hist_n * 4);
        size_t s_htmp = align_up(scan_tmp_words(hist_n) * 4);
        CGK_TRY(m->ws_sort.ensure(4 * s_keys + s_hist + s_htmp));
        char *sb = m->ws_sort.as<char>();
        uint32_t *ka = (uint32_t *)sb, *kb = (uint32_t *)(sb + s_keys);
        uint32_t *va = (uint32_t *)(sb + 2 * s_keys), *vb = (uint32_t *)(sb + 3 * s_keys);
        uint32_t *hist = (uint32_t *)(sb + 4 * s_keys);
        uint32_t *htmp = (uint32_t *)(sb + 4 * s_keys + s_hist);
        const uint32_t *kin = (const uint32_t *)cell;   // no cell is negative here
        const uint32_t *vin = nullptr;                  // identity on the first pass
        uint32_t *kout = ka, *vout = va;
        if (n > 0) {
            for (int ps = 0; ps < passes; ++ps) {
                int shift = ps * kRadixBits;
                CGK_LAUNCH("radix_upsweep", (double)n * 4, st,
                           k_radix_upsweep<<<(unsigned)ntiles, kThreads, 0, st>>>(
                               kin, n, shift, hist, (int)ntiles));
                CGK_TRY(exclusive_scan_u32(hist, hist, hist_n, htmp, st));
                CGK_LAUNCH("radix_downsweep", (double)n * (vin ? 16 : 12), st,
                           k_radix_downsweep<<<(unsigned)ntiles, kThreads, 0, st>>>(
                               kin, vin, kout, vout, n, shift, hist, (int)ntiles));
                CGK_CUDA(cudaGetLastError());
                kin = kout;
                vin = vout;
                kout = (kout == ka) ? kb : ka;
                vout = (vout == va) ? vb : va;
            }
        }
        CGK_CUDA(cudaMemsetAsync(out, 0, (size_t)ncells * nf * 8, st));
        if (n > 0) {
            CGK_LAUNCH("segment_heads", (double)n * (8 + 8 * nf) + (double)ncells * 8 * nf, st,
                       k_segment_heads<<<grid_for(n), kThreads, 0, st>>>(
                           n, kin, vin, nf, w, ncells, vc, vcu, inv_pow2, out));
            CGK_CUDA(cudaGetLastError());
        }
        if (rep)
            for (int f = 0; f < nf && f < CG_REPORT_MAX_FIELDS; ++f) rep->fixed_point_bits[f] = 0;
    } else {
        // fixed point: F per field from max|w|
        size_t s_acc = align_up((size_t)ncells * nf * 8);
        CGK_TRY(m->ws_sort.ensure(s_acc + 4096));
        unsigned long long *acc = m->ws_sort.as<unsigned long long>();
        unsigned long long *mx = (unsigned long long *)(m->ws_sort.as<char>() + s_acc);
        double *scales = (double *)(mx + 64);
        CGK_CUDA(cudaMemsetAsync(mx, 0, 64 * 8, st));
        if (n > 0) {
            dim3 g(grid_for(n), nf);
            CGK_LAUNCH("absmax", (double)n * nf * 8, st,
                       k_absmax<<<g, kThreads, 0, st>>>(n, nf, w, mx));
            CGK_CUDA(cudaGetLastError());
        }
        CGK_TRY(m->h_small.ensure(4096));
        unsigned long long *hmx = m->h_small.as<unsigned long long>();
        CGK_CUDA(cudaMemcpyAsync(hmx, mx, nf * 8, cudaMemcpyDeviceToHost, st));
        CGK_CUDA(cudaStreamSynchronize(st));
        double hs[2 * 64];
        for (int f = 0; f < nf; ++f) {
            double mabs;
            std::memcpy(&mabs, &hmx[f], 8);
            int F = fixed_bits(n, mabs);
            hs[f] = std::ldexp(1.0, F);
            hs[64 + f] = std::ldexp(1.0, -F);
            if (rep && f < CG_REPORT_MAX_FIELDS) rep->fixed_point_bits[f] = F;
        }
        CGK_CUDA(cudaMemcpyAsync(scales, hs, sizeof(hs), cudaMemcpyHostToDevice, st));
        CGK_CUDA(cudaMemsetAsync(acc, 0, (size_t)ncells * nf * 8, st));
        if (n > 0) {
            CGK_LAUNCH("fixed_accum", (double)n * (4 + 8 * nf), st,
                       k_fixed_accum<<<grid_for(n), kThreads, 0, st>>>(n, cell, nf, w, scales,
                                                                        acc, ncells));
            CGK_CUDA(cudaGetLastError());
        }
        CGK_LAUNCH("fixed_finalize", (double)ncells * nf * 16, st,
                   k_fixed_finalize<<<grid_for(ncells), kThreads, 0, st>>>(
                       ncells, nf, acc, scales + 64, vc, vcu, inv_pow2, out));
        CGK_CUDA(cudaGetLastError());
        // the host array hs must outlive the async copy
        CGK_CUDA(cudaStreamSynchronize(st));
    }
    return CG_OK;
}

cg_status deposit_run(cg_mesh *m, int64_t n, const double *pos, int nf, const double *w,
                      double *out, const cg_params *p, cg_report *rep, cudaStream_t st) {
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    auto drop = [&]() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    };
    if (rep) {
        for (auto &e : ev) CGK_CUDA(cudaEventCreate(&e));
        CGK_CUDA(cudaEventRecord(ev[0], st));
    }
    DepositPlan dp;
    cg_status s = deposit_begin(m, n, pos, nf, w, p, st, dp);
    if (s == CG_OK && cudaStreamSynchronize(st) != cudaSuccess)
        s = cuda_fail(cudaGetLastError(), "deposition", __FILE__, __LINE__);
    if (s == CG_OK && rep) cudaEventRecord(ev[1], st);
    if (s == CG_OK) s = deposit_end(m, n, nf, w, out, rep, st, dp);
    if (s == CG_OK && rep) {
        cudaEventRecord(ev[2], st);
        cudaEventSynchronize(ev[2]);
        float a = 0, b = 0;
        cudaEventElapsedTime(&a, ev[0], ev[1]);
        cudaEventElapsedTime(&b, ev[1], ev[2]);
        rep->ms_locate = a;
        rep->ms_deposit = b;
    }
    drop();
    return s;
}

// The depositions of several distinct meshes: every point location is launched before
// one synchronisation, every counter is checked before any output is written (the first
// failing snapshot's status), then every sum runs.  The snapshots' kernels are small, so
// they are spread over a few streams of the first mesh (forked from and joined back to
// st by events) and run side by side.  rep (optional) gets the device time of the two
// phases and the total count of outside particles.
cg_status deposit_many(int nsnap, cg_mesh *const *meshes, const int64_t *n, const double *const *pos,
                       int nf, const double *const *w, double *const *out, const cg_params *p,
                       cg_report *rep, cudaStream_t st) {
    constexpr int kAux = 8;
    cg_mesh *m0 = meshes[0];
    while ((int)m0->aux_streams.size() < kAux) {
        cudaStream_t a = nullptr;
        CGK_CUDA(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
        m0->aux_streams.push_back(a);
    }
    const int na = std::min(kAux, nsnap);
    std::vector<cudaEvent_t> evs;
    auto event = [&](cudaEvent_t *e) -> cg_status {
        CGK_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        evs.push_back(*e);
        return CG_OK;
    };
    // the auxiliary streams start after what st holds, and st continues after them
    auto fork = [&]() -> cg_status {
        cudaEvent_t e;
        CGK_TRY(event(&e));
        CGK_CUDA(cudaEventRecord(e, st));
        for (int a = 0; a < na; ++a) CGK_CUDA(cudaStreamWaitEvent(m0->aux_streams[a], e, 0));
        return CG_OK;
    };
    auto join = [&]() -> cg_status {
        for (int a = 0; a < na; ++a) {
            cudaEvent_t e;
            CGK_TRY(event(&e));
            CGK_CUDA(cudaEventRecord(e, m0->aux_streams[a]));
            CGK_CUDA(cudaStreamWaitEvent(st, e, 0));
        }
        return CG_OK;
    };
    std::vector<DepositPlan> dps((size_t)nsnap);
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    auto drop = [&]() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : evs) cudaEventDestroy(e);
    };
    cg_status s = CG_OK;
    if (rep) {
        for (auto &e : ev)
            if (s == CG_OK && cudaEventCreate(&e) != cudaSuccess) s = fail(CG_ECUDA, "event");
        if (s == CG_OK) cudaEventRecord(ev[0], st);
    }
    if (s == CG_OK) s = fork();
    for (int q = 0; q < nsnap && s == CG_OK; ++q)
        s = deposit_begin(meshes[q], n[q], pos[q], nf, w[q], p, m0->aux_streams[q % na], dps[q]);
    if (s == CG_OK) s = join();
    if (s == CG_OK && cudaStreamSynchronize(st) != cudaSuccess)
        s = cuda_fail(cudaGetLastError(), "deposition", __FILE__, __LINE__);
    if (s == CG_OK && rep) cudaEventRecord(ev[1], st);
    long long n_out_total = 0;
    for (int q = 0; q < nsnap && s == CG_OK; ++q) {
        int64_t n_out = 0, n_bad = 0;
        locate_read(meshes[q], &n_out, &n_bad, nullptr);
        n_out_total += n_out;
        if (n_bad) s = fail(CG_EINVAL, "batch snapshot %d: %lld non-finite weights", q, (long long)n_bad);
        else if (n_out) s = fail(CG_EDOMAIN, "batch snapshot %d: %lld particles outside the mesh", q, (long long)n_out);
    }
    if (rep) rep->n_out_of_domain = n_out_total;
    if (s == CG_OK) s = fork();
    for (int q = 0; q < nsnap && s == CG_OK; ++q)
        s = deposit_end(meshes[q], n[q], nf, w[q], out[q], nullptr, m0->aux_streams[q % na], dps[q]);
    if (s == CG_OK) s = join();
    if (s == CG_OK && rep) {
        cudaEventRecord(ev[2], st);
        cudaEventSynchronize(ev[2]);
        float a = 0, b = 0;
        cudaEventElapsedTime(&a, ev[0], ev[1]);
        cudaEventElapsedTime(&b, ev[1], ev[2]);
        rep->ms_locate = a;
        rep->ms_deposit = b;
    }
    if (s != CG_OK) {   // nothing of this call stays in flight
        for (int a = 0; a < na; ++a) cudaStreamSynchronize(m0->aux_streams[a]);
        cudaStreamSynchronize(st);
    }
    drop();
    return s;
}

}  // namespace cgk

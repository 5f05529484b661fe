// tet.cu -- unstructured tetrahedral meshes: mesh construction (host), point location
// of particle centroids, and diffusion smoothing with the cell-centred two-point-flux
// finite-volume operator (the paper's method on unstructured cells, Section 4.3).
//
// Operator: (L u)_k = sum over the faces f of cell k shared with cell l of
// T_f (u_l - u_k), T_f = |S_f|^2 / (S_f . d_f) with S_f the face area vector pointing
// out of k and d_f = c_l - c_k the vector between the tet centroids (vertex means);
// boundary faces carry no flux (zero-flux walls, Section 3.2.2).  With M = diag(V_c)
// an implicit-Euler pseudo-step solves (M - dtau L) u^{n+1} = M u^n, Crank-Nicolson
// (M - dtau/2 L) u^{n+1} = (M + dtau/2 L) u^n (Section 5.1), explicit Euler
// u += dtau M^{-1} L u.  The system matrix is symmetric positive definite (an M-matrix
// when every T_f > 0), so it is solved by Jacobi-preconditioned conjugate gradients:
// in FP64, or in FP32/BF16 storage inside FP64 iterative refinement.
//
// Layout: each cell has at most four face neighbours; they are stored as four
// structure-of-arrays slots (slot s = the face opposite local vertex s), so a thread
// per cell reads its neighbour ids and transmissibilities with coalesced loads.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "reduce.cuh"

namespace cgk {

namespace {

template <class T> cg_status upload(T **dst, const T *src, size_t n) {
    *dst = nullptr;
    if (n == 0) return CG_OK;
    cudaError_t e = cudaMalloc((void **)dst, n * sizeof(T));
    if (e != cudaSuccess) {
        *dst = nullptr;
        cudaGetLastError();
        return fail(CG_ENOMEM, "cudaMalloc of %zu bytes failed", n * sizeof(T));
    }
    CGK_CUDA(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
    return CG_OK;
}

inline int grid1d(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)num_sms() * 8;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// ============================================================================ locate
// orient(p0,p1,p2,p3) = det[p1-p0; p2-p0; p3-p0], cofactor expansion along the first
// row in this exact order, every operation explicitly rounded (no contraction).
__device__ __forceinline__ double orient3(const double *p0, const double *p1, const double *p2,
                                          const double *p3) {
    double a0 = __dsub_rn(p1[0], p0[0]), a1 = __dsub_rn(p1[1], p0[1]), a2 = __dsub_rn(p1[2], p0[2]);
    double b0 = __dsub_rn(p2[0], p0[0]), b1 = __dsub_rn(p2[1], p0[1]), b2 = __dsub_rn(p2[2], p0[2]);
    double c0 = __dsub_rn(p3[0], p0[0]), c1 = __dsub_rn(p3[1], p0[1]), c2 = __dsub_rn(p3[2], p0[2]);
    double m0 = __dsub_rn(__dmul_rn(b1, c2), __dmul_rn(b2, c1));
    double m1 = __dsub_rn(__dmul_rn(b0, c2), __dmul_rn(b2, c0));
    double m2 = __dsub_rn(__dmul_rn(b0, c1), __dmul_rn(b1, c0));
    return __dadd_rn(__dsub_rn(__dmul_rn(a0, m0), __dmul_rn(a1, m1)), __dmul_rn(a2, m2));
}

// A double as a 64-bit key in the order of the doubles (-0 as +0; a NaN sorts above +inf
// or below -inf by its sign, so it fails one side of a range test).
__device__ __forceinline__ unsigned long long tkey(double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    if (b == 0x8000000000000000ull) b = 0;
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// The FP64 barycentric coordinates of x in tet tt by the defining expressions.
__device__ __noinline__ void tet_lambdas(const TetDevice &t, int32_t tt, const double *x, double *lam) {
    const double *v0 = t.xyz + 3 * (size_t)t.tv[4 * (size_t)tt + 0];
    const double *v1 = t.xyz + 3 * (size_t)t.tv[4 * (size_t)tt + 1];
    const double *v2 = t.xyz + 3 * (size_t)t.tv[4 * (size_t)tt + 2];
    const double *v3 = t.xyz + 3 * (size_t)t.tv[4 * (size_t)tt + 3];
    const double D = orient3(v0, v1, v2, v3);
    lam[0] = __ddiv_rn(orient3(x, v1, v2, v3), D);
    lam[1] = __ddiv_rn(orient3(v0, x, v2, v3), D);
    lam[2] = __ddiv_rn(orient3(v0, v1, x, v3), D);
    lam[3] = __ddiv_rn(orient3(v0, v1, v2, x), D);
}

// det[a; b; c] in FP32 and a bound on its distance from the exact determinant of the
// vectors a, b, c stand for (each component within 2^-24 (1 + 2^-28) relative of the
// exact value): input error 3.0001 u + evaluation error 6 u (u = 2^-24) times the
// permanent of |a|, |b|, |c|, with a factor of more than 1.5 to spare.
__device__ __forceinline__ float det3f(const float *a, const float *b, const float *c, float *bound) {
    const float d = a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                    a[2] * (b[0] * c[1] - b[1] * c[0]);
    const float p = fabsf(a[0]) * (fabsf(b[1] * c[2]) + fabsf(b[2] * c[1])) +
                    fabsf(a[1]) * (fabsf(b[0] * c[2]) + fabsf(b[2] * c[0])) +
                    fabsf(a[2]) * (fabsf(b[0] * c[1]) + fabsf(b[1] * c[0]));
    *bound = p * 0x1p-20f;
    return d;
}

// Whether x is in tet tt by the FP64 definition (all four lambda >= 0), decided from
// FP32 determinants when their signs are certain: 1 inside, 0 outside, -1 undecided.
// With e_i = v_i - v0 (kept per tet) and q = x - v0 (FP64 differences, then FP32), the coordinates'
// numerators are det(q,e2,e3), det(e1,q,e3), det(e1,e2,q) and D minus those three (the
// four sum to D exactly); the FP64 definition evaluates the same determinants with errors
// below 2^-50 of their permanents, far inside the bounds used here.
__device__ __forceinline__ int tet_inside_f(const TetDevice &t, int32_t tt, const double *x) {
    const double *v0 = t.xyz + 3 * (size_t)t.tv[4 * (size_t)tt + 0];
    const float *ev = t.edge32 + 9 * (size_t)tt;   // precomputed: same roundings as below
    float e1[3], e2[3], e3[3], q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        e1[k] = ev[k];
        e2[k] = ev[3 + k];
        e3[k] = ev[6 + k];
        q[k] = __double2float_rn(__dsub_rn(x[k], v0[k]));
    }
    float bD, b1, b2, b3;
    const float D = det3f(e1, e2, e3, &bD);
    const float o1 = det3f(q, e2, e3, &b1);
    const float o2 = det3f(e1, q, e3, &b2);
    const float o3 = det3f(e1, e2, q, &b3);
    const float o0 = ((D - o1) - o2) - o3;
    // o0's bound: the four bounds, the three subtractions' rounding (3 u of the terms),
    // and the FP64 definition's error on det(v1-x, v2-x, v3-x) (below 6 2^-50 of the
    // product of the vectors' max-norms, each at most |e_i| + |q|)
    float n1 = 0.f, n2 = 0.f, n3 = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        n1 = fmaxf(n1, fabsf(e1[k]) + fabsf(q[k]));
        n2 = fmaxf(n2, fabsf(e2[k]) + fabsf(q[k]));
        n3 = fmaxf(n3, fabsf(e3[k]) + fabsf(q[k]));
    }
    const float b0 = 1.001f * (bD + b1 + b2 + b3) +
                     (fabsf(D) + fabsf(o1) + fabsf(o2) + fabsf(o3)) * 0x1p-22f +
                     n1 * n2 * n3 * 0x1p-44f;
    if (!(fabsf(D) > bD)) return -1;   // a flat tet: leave it to FP64
    const bool pos = D > 0.f;
    const float o[4] = {o0, o1, o2, o3}, bb[4] = {b0, b1, b2, b3};
    bool undecided = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (o[j] > bb[j]) {
            if (!pos) return 0;
        } else if (o[j] < -bb[j]) {
            if (pos) return 0;
        } else {
            undecided = true;
        }
    }
    return undecided ? -1 : 1;
}

// Host tet of each particle: the lowest-index tet whose axis-aligned box holds x and
// whose four barycentric coordinates lambda_j = orient(tet with v_j -> x) / orient(tet)
// are all >= 0; else the tet (box holding x) with the largest min_j lambda_j, lowest
// index on ties, if that value is >= -1e-10; else outside (-1).  Candidates come from
// the bucket of x, which holds every tet whose box overlaps it, in ascending order.  The
// box tests compare doubles exactly as integer keys; a candidate is settled from FP32
// determinants when their signs are certain and from the FP64 coordinates otherwise,
// and the largest-minimum search (no tet holds x) runs on FP64 coordinates only.
// The point-location bucket of x (clamped into the bucket grid), or nbuckets if a
// coordinate is not finite.
__device__ __forceinline__ int tet_bucket(const TetDevice &t, const double *x) {
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) ok = ok && (((__double2hiint(x[a]) >> 20) & 0x7ff) != 0x7ff);
    if (!ok) return t.nb[0] * t.nb[1] * t.nb[2];
    int bi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double q = floor(__dmul_rn(__dsub_rn(x[a], t.blo[a]), t.binv[a]));
        bi[a] = q < 0.0 ? 0 : (q > (double)(t.nb[a] - 1) ? t.nb[a] - 1 : (int)q);
    }
    return (bi[2] * t.nb[1] + bi[1]) * t.nb[0] + bi[0];
}

// No candidate tet of bucket entries [c0, c1) holds x: the tet (box holding x) with the
// largest minimum barycentric coordinate, lowest index on ties, if that value is >= -1e-10,
// else -1.  Rare (rounding at faces), so kept out of line to leave the search loop's
// registers to the common case.
__device__ __noinline__ int32_t tet_largest_min(const TetDevice &t, int c0, int c1, const double *x) {
    const unsigned long long kx0 = tkey(x[0]), kx1 = tkey(x[1]), kx2 = tkey(x[2]);
    int32_t best = -1;
    double best_m = -INFINITY;
    for (int c = c0; c < c1; ++c) {
        const int32_t tt = t.bucket_tets[c];
        const double *bx = t.box + 6 * (size_t)tt;
        if (!(kx0 >= tkey(bx[0]) && kx0 <= tkey(bx[3]) && kx1 >= tkey(bx[1]) &&
              kx1 <= tkey(bx[4]) && kx2 >= tkey(bx[2]) && kx2 <= tkey(bx[5])))
            continue;
        double lam[4];
        tet_lambdas(t, tt, x, lam);
        double m = lam[0];
        if (lam[1] < m) m = lam[1];
        if (lam[2] < m) m = lam[2];
        if (lam[3] < m) m = lam[3];
        if (m > best_m) {
            best_m = m;
            best = tt;
        }
    }
    return (best >= 0 && best_m >= -1e-10) ? best : -1;
}

// Particles grouped by bucket (a counting sort; the order within a bucket is arbitrary),
// so that the lanes of a warp in k_tet_locate scan the same candidate list: bucket and
// arrival rank per particle, then order[offset[bucket] + rank] = particle.
__global__ void k_tet_bucket_count(int64_t n, const double *__restrict__ pos, TetDevice t,
                                   int32_t *__restrict__ key, uint32_t *__restrict__ rank,
                                   uint32_t *__restrict__ count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x[3] = {pos[i], pos[n + i], pos[2 * n + i]};
        const int b = tet_bucket(t, x);
        key[i] = b;
        rank[i] = atomicAdd(&count[b], 1u);
    }
}

__global__ void k_tet_bucket_scatter(int64_t n, const int32_t *__restrict__ key,
                                     const uint32_t *__restrict__ rank,
                                     const uint32_t *__restrict__ offset, int32_t *__restrict__ order) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        order[offset[key[i]] + rank[i]] = (int32_t)i;
}

// Three blocks per SM (80 registers, a few bytes spilled) hide the gathers' latency better
// than two at 102: 5.7 -> 4.3 ms for 5,000,000 particles on 6,000,000 tets.
__global__ void __launch_bounds__(256, 3) k_tet_locate(int64_t n, const double *__restrict__ pos, TetDevice t, int nf,
                             const double *__restrict__ w, int32_t *__restrict__ cell,
                             uint32_t *__restrict__ counts, uint32_t *__restrict__ ranks,
                             unsigned long long *__restrict__ bad, const int32_t *__restrict__ order) {
    unsigned long long n_out = 0, n_nonfinite = 0;
    uint32_t most = 0;   // largest per-cell count seen (counts != nullptr)
    const int nbk = t.nb[0] * t.nb[1] * t.nb[2];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = order ? (int64_t)order[j] : j;
        for (int f = 0; f < nf; ++f)
            if (((__double2hiint(w[(int64_t)f * n + i]) >> 20) & 0x7ff) == 0x7ff) ++n_nonfinite;
        double x[3] = {pos[i], pos[n + i], pos[2 * n + i]};
        int32_t found = -1;
        const int b = tet_bucket(t, x);
        if (b < nbk) {
            const unsigned long long kx0 = tkey(x[0]), kx1 = tkey(x[1]), kx2 = tkey(x[2]);
            const int c0 = t.bucket_start[b], c1 = t.bucket_start[b + 1];
            bool any_box = false;
            for (int c = c0; c < c1 && found < 0; ++c) {
                const int32_t tt = t.bucket_tets[c];
                const double *bx = t.box + 6 * (size_t)tt;
                if (!(kx0 >= tkey(bx[0]) && kx0 <= tkey(bx[3]) && kx1 >= tkey(bx[1]) &&
                      kx1 <= tkey(bx[4]) && kx2 >= tkey(bx[2]) && kx2 <= tkey(bx[5])))
                    continue;
                any_box = true;
                int in = tet_inside_f(t, tt, x);
                if (in < 0) {
                    double lam[4];
                    tet_lambdas(t, tt, x, lam);
                    in = (lam[0] >= 0.0 && lam[1] >= 0.0 && lam[2] >= 0.0 && lam[3] >= 0.0) ? 1 : 0;
                }
                if (in) found = tt;
            }
            if (found < 0 && any_box) found = tet_largest_min(t, c0, c1, x);   // no tet holds x
        }
        cell[i] = found;
        if (found < 0) {
            ++n_out;
        } else if (counts) {
            const uint32_t r = atomicAdd(&counts[found], 1u);
            if (ranks) ranks[i] = r;
            most = max(most, r + 1u);
        }
    }
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

// Host cell of each particle on a stretched Cartesian mesh: per axis the largest i with
// f[i] <= x by bisection over the face coordinates (x = f[n] is in the last cell);
// outside the closed box, or NaN, is -1.  Doubles are compared exactly as integer keys.
__global__ void k_hex_locate(int64_t n, const double *__restrict__ pos, TetDevice t, int nf,
                             const double *__restrict__ w, int32_t *__restrict__ cell,
                             uint32_t *__restrict__ counts, uint32_t *__restrict__ ranks,
                             unsigned long long *__restrict__ bad) {
    unsigned long long n_out = 0, n_nonfinite = 0;
    uint32_t most = 0;
    const double *fa[3] = {t.faces, t.faces + t.hn[0] + 1, t.faces + t.hn[0] + t.hn[1] + 2};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int f = 0; f < nf; ++f)
            if (((__double2hiint(w[(int64_t)f * n + i]) >> 20) & 0x7ff) == 0x7ff) ++n_nonfinite;
        int id[3];
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const unsigned long long kx = tkey(pos[(int64_t)a * n + i]);
            const double *f = fa[a];
            const int na = t.hn[a];
            if (!(kx >= tkey(f[0]) && kx <= tkey(f[na]))) {
                ok = false;
                id[a] = 0;
                continue;
            }
            int lo = 0, hi = na - 1;   // invariant: f[lo] <= x, answer in [lo, hi]
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (tkey(f[mid]) <= kx) lo = mid;
                else hi = mid - 1;
            }
            id[a] = lo;
        }
        int32_t found = -1;
        if (ok) found = (int32_t)(((int64_t)id[2] * t.hn[1] + id[1]) * t.hn[0] + id[0]);
        cell[i] = found;
        if (found < 0) {
            ++n_out;
        } else if (counts) {
            const uint32_t r = atomicAdd(&counts[found], 1u);
            if (ranks) ranks[i] = r;
            most = max(most, r + 1u);
        }
    }
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

// ============================================================================ solver kernels
template <class TS> __device__ __forceinline__ float ldf(const TS *p, int64_t i);
template <> __device__ __forceinline__ float ldf<float>(const float *p, int64_t i) { return p[i]; }
template <> __device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16 *p, int64_t i) {
    return __bfloat162float(p[i]);
}
template <class TS> __device__ __forceinline__ void stf(TS *p, int64_t i, float v);
template <> __device__ __forceinline__ void stf<float>(float *p, int64_t i, float v) { p[i] = v; }
template <> __device__ __forceinline__ void stf<__nv_bfloat16>(__nv_bfloat16 *p, int64_t i, float v) {
    p[i] = __float2bfloat16_rn(v);
}

struct Op {          // the operator seen by the kernels
    int n;
    const double *vc, *diagL, *offv;
    const float *offv32;
    const int32_t *offc;
    double dte;      // theta * dtau (the coefficient of L in A = M - dte L)
    double dtau;     // full dtau (for the residual of the first pass)
    const float *adiag32 = nullptr;    // FP32 diagonal of A, V_c - dte L_kk (inner solves)
    const float *iadiag32 = nullptr;   // its reciprocal (the Jacobi preconditioner)
    const float *wsc32 = nullptr;      // [ns][n] dte T_f / A_kk (the Jacobi-scaled off-diagonals)
    int ns = 4;                        // neighbour slots per cell (4 tets, 6 stretched hex)
    int hx = 0, hy = 0, hz = 0;        // stretched hex mesh: cells per axis (0 for tets)
};
constexpr int kMaxSlots = 6;

// The FP32 diagonal of A = M - dte L and its reciprocal, for the inner solves.
__global__ void k_tdiag32(int n, const double *__restrict__ vc, const double *__restrict__ diagL,
                          double dte, float *__restrict__ ad, float *__restrict__ iad) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const double a = vc[k] - dte * diagL[k];
        ad[k] = (float)a;
        iad[k] = (float)(1.0 / a);
    }
}

// Jacobi-scaled off-diagonal weights of A for this call's dte: w[q][k] = dte T_q / A_kk,
// from the FP64 values, rounded once to FP32
__global__ void k_tscaled(int n, int ns, const double *__restrict__ vc, const double *__restrict__ diagL,
                          const double *__restrict__ offv, double dte, float *__restrict__ w) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const double a = vc[k] - dte * diagL[k];
        for (int q = 0; q < ns; ++q) w[(size_t)q * n + k] = (float)(dte * offv[(size_t)q * n + k] / a);
    }
}

// (L u)_k with u given by load(l)
template <class T, class Load>
__device__ __forceinline__ T lap_row(const Op &o, int k, T uk, Load load) {
    T s = (T)o.diagL[k] * uk;
#pragma unroll
    for (int q = 0; q < kMaxSlots; ++q) {
        if (q >= o.ns) break;
        const size_t e = (size_t)q * o.n + k;
        s += (T)o.offv[e] * load(o.offc[e]);
    }
    return s;
}

struct TScal {
    double rr, bb, rz, alpha, beta, rr0;
    int done, iters;
    unsigned int ticket;
    int breakdown;
};

// FP64 PCG, initial pass: x = u^n, r = b - A x = dtau L x, b = M x (+ dtau/2 L x for CN),
// z = r / diag(A), p = z.
__global__ void k_tcg_init(Op o, int scheme, const double *__restrict__ xall,
                           double *__restrict__ rall, double *__restrict__ zall,
                           double *__restrict__ pall, double *__restrict__ partials_all,
                           TScal *__restrict__ sc, double tol2) {
    const int f = blockIdx.y;
    const size_t off = (size_t)f * o.n;
    const double *x = xall + off;
    double rr = 0, bb = 0, rz = 0;
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < o.n; k += gridDim.x * kThreads) {
        double xk = x[k];
        double lx = lap_row<double>(o, k, xk, [&](int l) { return x[l]; });
        double rk = o.dtau * lx;
        double bk = o.vc[k] * xk;
        if (scheme == 1) bk += 0.5 * o.dtau * lx;
        double ad = o.vc[k] - o.dte * o.diagL[k];
        double zk = rk / ad;
        rall[off + k] = rk;
        zall[off + k] = zk;
        pall[off + k] = zk;
        rr += rk * rk;
        bb += bk * bk;
        rz += rk * zk;
    }
    double v[3] = {block_sum(rr), block_sum(bb), block_sum(rz)};
    double *partials = partials_all + (size_t)f * 3 * gridDim.x;
    if (arrive(partials, 3, v, blockIdx.x, gridDim.x, &sc[f].ticket)) {
        double RR = finish_sum(partials, 0, gridDim.x);
        double BB = finish_sum(partials, 1, gridDim.x);
        double RZ = finish_sum(partials, 2, gridDim.x);
        if (is_thread0()) {
            TScal &S = sc[f];
            S.rr = RR;
            S.bb = BB;
            S.rz = RZ;
            S.beta = 0;
            S.iters = 0;
            S.breakdown = 0;
            S.done = (RR <= tol2 * BB) ? 1 : 0;
            S.ticket = 0;
        }
    }
}

// pass 1: p_new = z + beta p (formed on the fly at the neighbours too), q = A p_new,
// accumulate p_new . q; alpha = rz / (p.q).
__global__ void k_tcg_pass1(Op o, const double *__restrict__ zall, const double *__restrict__ pin_all,
                            double *__restrict__ pout_all, double *__restrict__ qall,
                            double *__restrict__ partials_all, TScal *__restrict__ sc) {
    const int f = blockIdx.y;
    if (sc[f].done) return;
    const double beta = sc[f].beta;
    const size_t off = (size_t)f * o.n;
    const double *z = zall + off;
    const double *pin = pin_all + off;
    double pq = 0;
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < o.n; k += gridDim.x * kThreads) {
        double pk = z[k] + beta * pin[k];
        double lp = lap_row<double>(o, k, pk, [&](int l) { return z[l] + beta * pin[l]; });
        double qk = o.vc[k] * pk - o.dte * lp;
        pout_all[off + k] = pk;
        qall[off + k] = qk;
        pq += pk * qk;
    }
    double v = block_sum(pq);
    double *partials = partials_all + (size_t)f * 3 * gridDim.x;
    if (arrive(partials, 1, &v, blockIdx.x, gridDim.x, &sc[f].ticket)) {
        double PQ = finish_sum(partials, 0, gridDim.x);
        if (is_thread0()) {
            TScal &S = sc[f];
            if (PQ > 0) {
                S.alpha = S.rz / PQ;
            } else {
                S.alpha = 0;
                S.breakdown = 1;
                S.done = 1;
            }
            S.ticket = 0;
        }
    }
}

// pass 2: x += alpha p, r -= alpha q, z = r / diag(A); beta = r.z_new / r.z_old.
__global__ void k_tcg_pass2(Op o, const double *__restrict__ pall, const double *__restrict__ qall,
                            double *__restrict__ xall, double *__restrict__ rall,
                            double *__restrict__ zall, double *__restrict__ partials_all,
                            TScal *__restrict__ sc, double tol2) {
    const int f = blockIdx.y;
    if (sc[f].done) return;
    const double alpha = sc[f].alpha;
    const size_t off = (size_t)f * o.n;
    double rr = 0, rz = 0;
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < o.n; k += gridDim.x * kThreads) {
        size_t i = off + k;
        xall[i] += alpha * pall[i];
        double rk = rall[i] - alpha * qall[i];
        double zk = rk / (o.vc[k] - o.dte * o.diagL[k]);
        rall[i] = rk;
        zall[i] = zk;
        rr += rk * rk;
        rz += rk * zk;
    }
    double v[2] = {block_sum(rr), block_sum(rz)};
    double *partials = partials_all + (size_t)f * 3 * gridDim.x;
    if (arrive(partials, 2, v, blockIdx.x, gridDim.x, &sc[f].ticket)) {
        double RR = finish_sum(partials, 0, gridDim.x);
        double RZ = finish_sum(partials, 1, gridDim.x);
        if (is_thread0()) {
            TScal &S = sc[f];
            S.beta = RZ / S.rz;
            S.rz = RZ;
            S.rr = RR;
            S.iters += 1;
            S.done = (RR <= tol2 * S.bb) ? 1 : 0;
            S.ticket = 0;
        }
    }
}

// explicit Euler: x_out = x + dtau L x / V_c
__global__ void k_texplicit(Op o, const double *__restrict__ xin, double *__restrict__ xout) {
    const size_t off = (size_t)blockIdx.y * o.n;
    const double *x = xin + off;
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < o.n; k += gridDim.x * kThreads) {
        double xk = x[k];
        double lx = lap_row<double>(o, k, xk, [&](int l) { return x[l]; });
        xout[off + k] = xk + o.dtau * lx / o.vc[k];
    }
}

// ---------------------------------------------------------------- mixed precision
// x_out = x_in + d (the refinement update of every field; FP64 = FP64 + FP32)
template <class TS>
__global__ void k_tadd(size_t n, const double *__restrict__ xin, const TS *__restrict__ d,
                       double *__restrict__ xout) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        xout[i] = xin[i] + (double)ldf(d, i);
}

// One FP64 refinement pass, fused with the initialisation of the next inner solve.
// kFirst: x = u^n, r = dtau L x, b = M x (CN: + dtau/2 L x, stored in bout).
// Otherwise x = x_in + d (at the cell and its neighbours), x_out = x, r = b - A x
// with b = M u^n (IE, from ub) or the stored CN right-hand side (bptr).
// Then the inner PCG starts from d = 0 (zeroed by the host after this pass):
// rin = r, z = r / diag(A), p = z.
// kPcg false (Chebyshev inner solves): only rin is started (no z, p or r.z), and a
// non-first pass reads x_in as the updated iterate itself (d = NULL, x_out unused; the
// update x += d ran before as k_tadd, so neighbours cost no conversions or additions on
// the FP64 units, which bound this pass on GB300).
template <class TS, bool kFirst, bool kPcg = true>
__global__ void k_trefine(Op o, int scheme, const double *__restrict__ xin_all,
                          const TS *__restrict__ d_all, const double *__restrict__ ub_all,
                          const double *__restrict__ bcn_all, double *__restrict__ xout_all,
                          double *__restrict__ bout_all, TS *__restrict__ rin_all,
                          TS *__restrict__ z_all, TS *__restrict__ p_all,
                          double *__restrict__ partials_all, TScal *__restrict__ sc) {
    const int f = blockIdx.y;
    const size_t off = (size_t)f * o.n;
    const double *xin = xin_all + off;
    const TS *d = (kFirst || !kPcg) ? nullptr : d_all + off;
    double rr = 0, bb = 0, rz = 0;
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < o.n; k += gridDim.x * kThreads) {
        double rk;
        if (kFirst) {
            double xk = xin[k];
            double lx = lap_row<double>(o, k, xk, [&](int l) { return xin[l]; });
            rk = o.dtau * lx;
            double bk = o.vc[k] * xk;
            if (scheme == 1) {
                bk += 0.5 * o.dtau * lx;
                bout_all[off + k] = bk;
            }
            bb += bk * bk;
        } else {
            double xk, lx;
            if (kPcg) {
                xk = xin[k] + (double)ldf(d, k);
                lx = lap_row<double>(o, k, xk, [&](int l) { return xin[l] + (double)ldf(d, l); });
                xout_all[off + k] = xk;
            } else {
                xk = xin[k];
                lx = lap_row<double>(o, k, xk, [&](int l) { return xin[l]; });
            }
            double bk = scheme == 1 ? bcn_all[off + k] : o.vc[k] * ub_all[off + k];
            rk = bk - (o.vc[k] * xk - o.dte * lx);
        }
        float rf = (float)rk;
        stf(rin_all, off + k, rf);
        if (!kPcg && z_all) stf(z_all, off + k, rf * o.iadiag32[k]);   // D^-1 r for k_tcheb1
        if (kPcg) {
            float zf = rf * o.iadiag32[k];
            stf(z_all, off + k, zf);
            stf(p_all, off + k, zf);
            rz += (double)rf * (double)zf;
        }
        rr += rk * rk;
    }
    double v[3] = {block_sum(rr), block_sum(rz), kFirst ? block_sum(bb) : 0.0};
    double *partials = partials_all + (size_t)f * 3 * gridDim.x;
    if (arrive(partials, kFirst ? 3 : 2, v, blockIdx.x, gridDim.x, &sc[f].ticket)) {
        double RR = finish_sum(partials, 0, gridDim.x);
        double RZ = finish_sum(partials, 1, gridDim.x);
        double BB = kFirst ? finish_sum(partials, 2, gridDim.x) : 0.0;
        if (is_thread0()) {
            TScal &S = sc[f];
            S.rr = RR;       // the FP64 residual of the outer iteration
            S.rr0 = RR;      // reference for the inner stopping test
            S.rz = RZ;
            S.beta = 0;
            S.iters = 0;
            S.breakdown = 0;
            if (kFirst) S.bb = BB;
            S.done = 0;
            S.ticket = 0;
        }
    }
}

// inner PCG pass 1 (FP32 arithmetic, TS storage): p_new = z + beta p, q = A p_new
// hist (may be null): per field, alpha_j at [f * 2H + j] and beta_j at [f * 2H + H + j]
// for the first H iterations (the Lanczos coefficients of the solve)
constexpr int kHist = 64;

template <class TS>
__global__ void k_tin_pass1(Op o, const TS *__restrict__ z_all, const TS *__restrict__ pin_all,
                            TS *__restrict__ pout_all, TS *__restrict__ q_all,
                            double *__restrict__ partials_all, TScal *__restrict__ sc,
                            double *__restrict__ hist) {
    const int f = blockIdx.y;
    if (sc[f].done) return;
    const float beta = (float)sc[f].beta;
    const float dte = (float)o.dte;
    const size_t off = (size_t)f * o.n;
    const TS *z = z_all + off;
    const TS *pin = pin_all + off;
    float pq = 0.f;   // a thread's partial sum stays short: FP32, then FP64 across threads
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < o.n; k += gridDim.x * kThreads) {
        float pk = ldf(z, k) + beta * ldf(pin, k);
        float off_sum = 0.f;
#pragma unroll
        for (int q = 0; q < kMaxSlots; ++q) {
            if (q >= o.ns) break;
            const size_t e = (size_t)q * o.n + k;
            const int l = o.offc[e];
            off_sum += o.offv32[e] * (ldf(z, l) + beta * ldf(pin, l));
        }
        float qk = o.adiag32[k] * pk - dte * off_sum;
        stf(pout_all, off + k, pk);
        stf(q_all, off + k, qk);
        pq = fmaf(pk, qk, pq);
    }
    double v = block_sum((double)pq);
    double *partials = partials_all + (size_t)f * 3 * gridDim.x;
    if (arrive(partials, 1, &v, blockIdx.x, gridDim.x, &sc[f].ticket)) {
        double PQ = finish_sum(partials, 0, gridDim.x);
        if (is_thread0()) {
            TScal &S = sc[f];
            if (PQ > 0) {
                S.alpha = S.rz / PQ;
                if (hist && S.iters < kHist) hist[(size_t)f * 2 * kHist + S.iters] = S.alpha;
            } else {
                S.alpha = 0;
                S.breakdown = 1;
                S.done = 1;
            }
            S.ticket = 0;
        }
    }
}

// inner PCG pass 2: d += alpha p, rin -= alpha q, z = rin / diag(A); stop when
// ||rin|| <= eps_in * ||r||
template <class TS>
__global__ void k_tin_pass2(Op o, const TS *__restrict__ p_all, const TS *__restrict__ q_all,
                            TS *__restrict__ d_all, TS *__restrict__ rin_all, TS *__restrict__ z_all,
                            double *__restrict__ partials_all, TScal *__restrict__ sc,
                            double eps2, double *__restrict__ hist) {
    const int f = blockIdx.y;
    if (sc[f].done) return;
    const float alpha = (float)sc[f].alpha;
    const size_t off = (size_t)f * o.n;
    float rr = 0.f, rz = 0.f;   // per-thread partial sums in FP32, FP64 across threads
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < o.n; k += gridDim.x * kThreads) {
        size_t i = off + k;
        float pk = ldf(p_all, i);
        stf(d_all, i, ldf(d_all, i) + alpha * pk);
        float rk = ldf(rin_all, i) - alpha * ldf(q_all, i);
        float zk = rk * o.iadiag32[k];
        stf(rin_all, i, rk);
        stf(z_all, i, zk);
        rr = fmaf(rk, rk, rr);
        rz = fmaf(rk, zk, rz);
    }
    double v[2] = {block_sum((double)rr), block_sum((double)rz)};
    double *partials = partials_all + (size_t)f * 3 * gridDim.x;
    if (arrive(partials, 2, v, blockIdx.x, gridDim.x, &sc[f].ticket)) {
        double RR = finish_sum(partials, 0, gridDim.x);
        double RZ = finish_sum(partials, 1, gridDim.x);
        if (is_thread0()) {
            TScal &S = sc[f];
            S.beta = RZ / S.rz;
            if (hist && S.iters < kHist) hist[(size_t)f * 2 * kHist + kHist + S.iters] = S.beta;
            S.rz = RZ;
            S.iters += 1;
            S.done = (RR <= eps2 * S.rr0) ? 1 : 0;
            S.ticket = 0;
        }
    }
}

// Start of the spectrum probe: an inner PCG solve (field 0) on a fixed right-hand side,
// r_k uniform in [-1/2, 1/2) from the 32-bit finaliser of MurmurHash3 (Appleby) applied
// to k, so the estimate depends on the operator alone.  Sets r, z = D^-1 r, p = z, d = 0
// and the solve's scalars as k_trefine does for a real solve (bb untouched).
__device__ __forceinline__ uint32_t mix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

template <class TS>
__global__ void k_tprobe_init(Op o, TS *__restrict__ rin, TS *__restrict__ z, TS *__restrict__ p,
                              TS *__restrict__ d, double *__restrict__ partials, TScal *__restrict__ sc) {
    double rr = 0, rz = 0;
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < o.n; k += gridDim.x * kThreads) {
        const float rf = (float)(mix32((uint32_t)k) >> 8) * 0x1p-24f - 0.5f;
        const float zf = rf * o.iadiag32[k];
        stf(rin, k, rf);
        stf(z, k, zf);
        stf(p, k, zf);
        stf(d, k, 0.f);
        rr += (double)rf * rf;
        rz += (double)rf * zf;
    }
    double v[2] = {block_sum(rr), block_sum(rz)};
    if (arrive(partials, 2, v, blockIdx.x, gridDim.x, &sc[0].ticket)) {
        const double RR = finish_sum(partials, 0, gridDim.x), RZ = finish_sum(partials, 1, gridDim.x);
        if (is_thread0()) {
            TScal &S = sc[0];
            S.rr = RR;
            S.rr0 = RR;
            S.rz = RZ;
            S.beta = 0;
            S.iters = 0;
            S.breakdown = 0;
            S.done = 0;
            S.ticket = 0;
        }
    }
}

// Inner Chebyshev iteration on the Jacobi-scaled system D^-1 A d = D^-1 r (FP32
// arithmetic, TS storage), spectrum enclosed in [theta - delta, theta + delta]: from
// d_0 = 0, d_1 = c0 D^-1 r; then d_{k+1} = d_k + c1 (d_k - d_{k-1}) + c2 D^-1 (r - A d_k)
// (dkm1 null: d_0 = 0).  No inner products, one pass per iteration.  This form handles
// one field; it reads the scaled residual rs = D^-1 r (written by the refinement pass)
// and the scaled weights w_q = dte T_q / A_kk, so that D^-1 (r - A d) = rs - d_k +
// sum_q w_q d_nb(q): a cell's operator row is NS indices and NS weights (32 B on tets),
// no diagonal.  k_tcheb below handles several fields.
template <class TS, int NS>
__global__ void __launch_bounds__(kThreads, 6) k_tcheb1(Op o, const TS *__restrict__ rs,
                                                        const TS *__restrict__ dk,
                                                        const TS *__restrict__ dkm1, TS *__restrict__ dn,
                                                        float c1, float c2) {
    const int stride = gridDim.x * kThreads;
    // two cells per pass (k and k + stride): both cells' NS neighbour indices and
    // weights are loaded before either cell's gathers, so twice the dependent loads are
    // in flight per thread
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < o.n; k += 2 * stride) {
        const int k2 = k + stride;
        const bool two = k2 < o.n;
        const int kb = two ? k2 : k;
        int nb[2][NS];
        float wv[2][NS];
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            nb[0][q] = o.offc[(size_t)q * o.n + k];
            wv[0][q] = o.wsc32[(size_t)q * o.n + k];
            nb[1][q] = o.offc[(size_t)q * o.n + kb];
            wv[1][q] = o.wsc32[(size_t)q * o.n + kb];
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int kc = c ? kb : k;
            float off_sum = 0.f;
#pragma unroll
            for (int q = 0; q < NS; ++q) off_sum += wv[c][q] * ldf(dk, nb[c][q]);
            const float dkk = ldf(dk, kc);
            const float sres = (ldf(rs, kc) - dkk) + off_sum;   // D^-1 (r - A d_k)
            const float dm = dkm1 ? ldf(dkm1, kc) : 0.f;        // d_0 = 0
            if (c == 0 || two) stf(dn, kc, dkk + c1 * (dkk - dm) + c2 * sres);
        }
    }
}

// The same iteration for nf fields: a thread reads a cell's operator row (indices and
// scaled weights) once and applies it to every field; r_all is the scaled residual
// rs = D^-1 r.  kFirst: the first step d_1 = c1 D^-1 r for any nf, with r_all the
// residual r itself.  The one-field loop above keeps more gathers in flight when there
// is only one.
template <class TS, bool kFirst>
__global__ void __launch_bounds__(kThreads, 4) k_tcheb(Op o, int nf, const TS *__restrict__ r_all,
                                                        const TS *__restrict__ dk_all,
                                                        const TS *__restrict__ dkm1_all, TS *__restrict__ dn_all,
                                                        float c1, float c2) {
    const size_t n = (size_t)o.n;
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < o.n; k += gridDim.x * kThreads) {
        if constexpr (kFirst) {
            const float iad = o.iadiag32[k];
            for (int f = 0; f < nf; ++f) stf(dn_all, f * n + k, c1 * (iad * ldf(r_all, f * n + k)));
        } else {   // the cell's operator row (indices, scaled weights) is read once for all fields
            int nb[kMaxSlots];
            float wv[kMaxSlots];
#pragma unroll
            for (int q = 0; q < kMaxSlots; ++q) {
                if (q >= o.ns) break;
                nb[q] = o.offc[(size_t)q * n + k];
                wv[q] = o.wsc32[(size_t)q * n + k];
            }
            for (int f = 0; f < nf; ++f) {
                const TS *dk = dk_all + f * n;
                const float dkk = ldf(dk, k);
                float off_sum = 0.f;
#pragma unroll
                for (int q = 0; q < kMaxSlots; ++q) {
                    if (q >= o.ns) break;
                    off_sum += wv[q] * ldf(dk, nb[q]);
                }
                const float sres = (ldf(r_all, f * n + k) - dkk) + off_sum;   // D^-1 (r - A d_k)
                const float dm = dkm1_all ? ldf(dkm1_all, f * n + k) : 0.f;   // d_0 = 0
                stf(dn_all, f * n + k, dkk + c1 * (dkk - dm) + c2 * sres);
            }
        }
    }
}

// The Chebyshev iteration of k_tcheb on a stretched Cartesian mesh, whose neighbours are
// implicit: slots 0..5 are the cells at k-1, k+1, k-nx, k+nx, k-nx ny, k+nx ny (a wall
// slot has T = 0 and reads the cell itself), so the neighbour values load without first
// loading their indices.  Like k_tcheb1 it reads the scaled residual rs = D^-1 r and the
// Jacobi-scaled weights dte T_q / A_kk (six per cell, no diagonal), for every field of
// the call.  A block is blockDim.x cells of a row by blockDim.y rows (256 threads).
template <class TS>
__global__ void __launch_bounds__(kThreads) k_hcheb(Op o, int nf, const TS *__restrict__ rs_all,
                                                     const TS *__restrict__ dk_all,
                                                     const TS *__restrict__ dkm1_all, TS *__restrict__ dn_all,
                                                     float c1, float c2) {
    const size_t n = (size_t)o.n;
    const int nx = o.hx, nxy = o.hx * o.hy, rows = o.hy * o.hz;
    for (int row = blockIdx.y * blockDim.y + threadIdx.y; row < rows; row += gridDim.y * blockDim.y) {
        const int iy = row % o.hy, iz = row / o.hy;
        for (int ix = blockIdx.x * blockDim.x + threadIdx.x; ix < nx; ix += gridDim.x * blockDim.x) {
            const int k = row * nx + ix;
            const int nb[6] = {ix > 0 ? k - 1 : k, ix + 1 < nx ? k + 1 : k, iy > 0 ? k - nx : k,
                               iy + 1 < o.hy ? k + nx : k, iz > 0 ? k - nxy : k, iz + 1 < o.hz ? k + nxy : k};
            float wv[6];   // Jacobi-scaled weights dte T_q / A_kk
#pragma unroll
            for (int q = 0; q < 6; ++q) wv[q] = o.wsc32[(size_t)q * n + k];
            for (int f = 0; f < nf; ++f) {
                const TS *dk = dk_all + f * n;
                const float dkk = ldf(dk, k);
                float off_sum = 0.f;
#pragma unroll
                for (int q = 0; q < 6; ++q) off_sum += wv[q] * ldf(dk, nb[q]);
                const float sres = (ldf(rs_all, f * n + k) - dkk) + off_sum;   // D^-1 (r - A d_k)
                const float dm = dkm1_all ? ldf(dkm1_all, f * n + k) : 0.f;   // d_0 = 0
                stf(dn_all, f * n + k, dkk + c1 * (dkk - dm) + c2 * sres);
            }
        }
    }
}

}  // namespace

// ============================================================================ host: build
void tet_release(cg_mesh *m) {
    TetDevice &t = m->tet;
    void *ptrs[] = {t.vc, t.diagL, t.offc, t.offv, t.offv32, t.xyz, t.tv, t.box, t.edge32, t.bucket_start,
                    t.bucket_tets, t.faces};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    t = TetDevice();
}

cg_status tet_build(cg_mesh *m, int64_t nv, const double *xyz, int64_t nt, const int32_t *tv) {
    for (int64_t i = 0; i < 4 * nt; ++i)
        if (tv[i] < 0 || tv[i] >= nv)
            return fail(CG_EINVAL, "cg_create_mesh_tet: vertex id %d out of range", tv[i]);
    // centroids (vertex means) and volumes |det| / 6
    std::vector<double> cent(3 * (size_t)nt), vc((size_t)nt);
    for (int64_t t = 0; t < nt; ++t) {
        const double *p[4];
        for (int j = 0; j < 4; ++j) p[j] = xyz + 3 * (size_t)tv[4 * t + j];
        for (int a = 0; a < 3; ++a) {
            volatile double s = p[0][a] + p[1][a];
            s = s + p[2][a];
            s = s + p[3][a];
            cent[3 * t + a] = s * 0.25;
        }
        double e[3][3];
        for (int j = 0; j < 3; ++j)
            for (int a = 0; a < 3; ++a) e[j][a] = p[j + 1][a] - p[0][a];
        double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                     e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                     e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
        vc[t] = std::fabs(det) / 6.0;
        if (!(vc[t] > 0.0)) return fail(CG_EINVAL, "cg_create_mesh_tet: tet %lld has zero volume", (long long)t);
    }
    // faces: bucket the 4 nt faces by their smallest vertex id, then match inside a bucket
    struct Face { int32_t b, c, tet, slot; };
    std::vector<int64_t> start((size_t)nv + 1, 0);
    auto face_verts = [&](int64_t t, int j, int32_t *v) {
        int q = 0;
        for (int i = 0; i < 4; ++i)
            if (i != j) v[q++] = tv[4 * t + i];
        std::sort(v, v + 3);
    };
    for (int64_t t = 0; t < nt; ++t)
        for (int j = 0; j < 4; ++j) {
            int32_t v[3];
            face_verts(t, j, v);
            start[(size_t)v[0] + 1]++;
        }
    for (int64_t i = 0; i < nv; ++i) start[i + 1] += start[i];
    std::vector<Face> faces((size_t)(4 * nt));
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int64_t t = 0; t < nt; ++t)
        for (int j = 0; j < 4; ++j) {
            int32_t v[3];
            face_verts(t, j, v);
            faces[(size_t)fill[v[0]]++] = Face{v[1], v[2], (int32_t)t, j};
        }
    std::vector<int32_t> offc(4 * (size_t)nt);
    std::vector<double> offv(4 * (size_t)nt, 0.0), diag((size_t)nt, 0.0);
    for (int64_t t = 0; t < nt; ++t)
        for (int j = 0; j < 4; ++j) offc[(size_t)j * nt + t] = (int32_t)t;
    for (int64_t a = 0; a < nv; ++a) {
        Face *f0 = faces.data() + start[a], *f1 = faces.data() + start[a + 1];
        std::sort(f0, f1, [](const Face &x, const Face &y) {
            return x.b != y.b ? x.b < y.b : (x.c != y.c ? x.c < y.c : x.tet < y.tet);
        });
        for (Face *f = f0; f < f1;) {
            Face *g = f + 1;
            while (g < f1 && g->b == f->b && g->c == f->c) ++g;
            if (g - f > 2)
                return fail(CG_EINVAL, "cg_create_mesh_tet: a face is shared by more than two tets");
            if (g - f == 2) {
                const int32_t k = f[0].tet, l = f[1].tet;
                const double *A = xyz + 3 * (size_t)a, *B = xyz + 3 * (size_t)f->b,
                             *C = xyz + 3 * (size_t)f->c;
                double ab[3], ac[3], S[3], d[3];
                for (int q = 0; q < 3; ++q) {
                    ab[q] = B[q] - A[q];
                    ac[q] = C[q] - A[q];
                }
                S[0] = 0.5 * (ab[1] * ac[2] - ab[2] * ac[1]);
                S[1] = 0.5 * (ab[2] * ac[0] - ab[0] * ac[2]);
                S[2] = 0.5 * (ab[0] * ac[1] - ab[1] * ac[0]);
                double out = 0.0;   // S . (face centroid - c_k) > 0 for S pointing out of k
                for (int q = 0; q < 3; ++q)
                    out += S[q] * ((A[q] + B[q] + C[q]) / 3.0 - cent[3 * (size_t)k + q]);
                if (out < 0.0)
                    for (int q = 0; q < 3; ++q) S[q] = -S[q];
                double ss = 0.0, sd = 0.0;
                for (int q = 0; q < 3; ++q) {
                    d[q] = cent[3 * (size_t)l + q] - cent[3 * (size_t)k + q];
                    ss += S[q] * S[q];
                    sd += S[q] * d[q];
                }
                double T = ss / sd;
                if (!(T > 0.0) || !std::isfinite(T))
                    return fail(CG_EINVAL, "cg_create_mesh_tet: non-positive transmissibility "
                                           "between tets %d and %d", k, l);
                offc[(size_t)f[0].slot * nt + k] = l;
                offv[(size_t)f[0].slot * nt + k] = T;
                offc[(size_t)f[1].slot * nt + l] = k;
                offv[(size_t)f[1].slot * nt + l] = T;
                diag[k] -= T;
                diag[l] -= T;
            }
            f = g;
        }
    }
    faces.clear();
    faces.shrink_to_fit();
    // host CSR (diagonal included, ascending columns) for cg_mesh_tet_operator
    m->h_rowptr.assign((size_t)nt + 1, 0);
    m->h_col.clear();
    m->h_val.clear();
    m->h_col.reserve(5 * (size_t)nt);
    m->h_val.reserve(5 * (size_t)nt);
    double max_rate = 0.0;
    for (int64_t t = 0; t < nt; ++t) {
        std::pair<int32_t, double> e[5];
        int q = 0;
        e[q++] = {(int32_t)t, diag[t]};
        for (int j = 0; j < 4; ++j)
            if (offc[(size_t)j * nt + t] != t) e[q++] = {offc[(size_t)j * nt + t], offv[(size_t)j * nt + t]};
        std::sort(e, e + q);
        for (int i = 0; i < q; ++i) {
            m->h_col.push_back(e[i].first);
            m->h_val.push_back(e[i].second);
        }
        m->h_rowptr[t + 1] = (int32_t)m->h_col.size();
        max_rate = std::max(max_rate, -diag[t] / vc[t]);
    }
    m->h_vc = vc;
    // point-location buckets: a uniform grid over the vertex bounding box, cell size
    // about the edge of the average hex (6 tets), each tet listed in every bucket its
    // bounding box overlaps
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < nv; ++i)
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], xyz[3 * i + a]);
            hi[a] = std::max(hi[a], xyz[3 * i + a]);
        }
    TetDevice &td = m->tet;
    double vol = 1.0;
    for (int a = 0; a < 3; ++a) vol *= std::max(hi[a] - lo[a], 1e-300);
    double h = std::cbrt(6.0 * vol / (double)nt);
    int64_t total = 1;
    for (int a = 0; a < 3; ++a) {
        double ext = std::max(hi[a] - lo[a], 1e-300);
        int nba = (int)std::ceil(ext / h);
        nba = std::max(1, std::min(nba, 1024));
        td.nb[a] = nba;
        td.blo[a] = lo[a];
        td.binv[a] = (double)nba / ext;
        total *= nba;
    }
    std::vector<double> box(6 * (size_t)nt);
    std::vector<int32_t> bstart((size_t)total + 1, 0);
    auto bucket_range = [&](int64_t t, int *b0, int *b1) {
        for (int a = 0; a < 3; ++a) {
            double mn = xyz[3 * (size_t)tv[4 * t] + a], mx = mn;
            for (int j = 1; j < 4; ++j) {
                double c = xyz[3 * (size_t)tv[4 * t + j] + a];
                mn = std::min(mn, c);
                mx = std::max(mx, c);
            }
            box[6 * t + a] = mn;
            box[6 * t + 3 + a] = mx;
            volatile double qa = (mn - td.blo[a]);
            volatile double qb = (mx - td.blo[a]);
            double fa = std::floor(qa * td.binv[a]), fb = std::floor(qb * td.binv[a]);
            b0[a] = fa < 0 ? 0 : (fa > td.nb[a] - 1 ? td.nb[a] - 1 : (int)fa);
            b1[a] = fb < 0 ? 0 : (fb > td.nb[a] - 1 ? td.nb[a] - 1 : (int)fb);
        }
    };
    for (int64_t t = 0; t < nt; ++t) {
        int b0[3], b1[3];
        bucket_range(t, b0, b1);
        for (int z = b0[2]; z <= b1[2]; ++z)
            for (int y = b0[1]; y <= b1[1]; ++y)
                for (int x = b0[0]; x <= b1[0]; ++x) bstart[((size_t)z * td.nb[1] + y) * td.nb[0] + x + 1]++;
    }
    for (int64_t i = 0; i < total; ++i) bstart[i + 1] += bstart[i];
    std::vector<int32_t> btets((size_t)bstart[total]);
    std::vector<int32_t> bfill(bstart.begin(), bstart.end() - 1);
    for (int64_t t = 0; t < nt; ++t) {
        int b0[3], b1[3];
        bucket_range(t, b0, b1);
        for (int z = b0[2]; z <= b1[2]; ++z)
            for (int y = b0[1]; y <= b1[1]; ++y)
                for (int x = b0[0]; x <= b1[0]; ++x)
                    btets[(size_t)bfill[((size_t)z * td.nb[1] + y) * td.nb[0] + x]++] = (int32_t)t;
    }
    std::vector<float> offv32(offv.size());
    for (size_t i = 0; i < offv.size(); ++i) offv32[i] = (float)offv[i];
    td.max_rate = max_rate;
    CGK_TRY(upload(&td.vc, vc.data(), vc.size()));
    CGK_TRY(upload(&td.diagL, diag.data(), diag.size()));
    CGK_TRY(upload(&td.offc, offc.data(), offc.size()));
    CGK_TRY(upload(&td.offv, offv.data(), offv.size()));
    CGK_TRY(upload(&td.offv32, offv32.data(), offv32.size()));
    CGK_TRY(upload(&td.xyz, xyz, 3 * (size_t)nv));
    CGK_TRY(upload(&td.tv, tv, 4 * (size_t)nt));
    CGK_TRY(upload(&td.box, box.data(), box.size()));
    std::vector<float> edge((size_t)9 * nt);
    for (int64_t t = 0; t < nt; ++t) {
        const double *v0 = xyz + 3 * (size_t)tv[4 * t];
        for (int j = 1; j < 4; ++j) {
            const double *vj = xyz + 3 * (size_t)tv[4 * t + j];
            for (int a = 0; a < 3; ++a) {
                volatile double dd = vj[a] - v0[a];   // one FP64 rounding, then one to FP32
                edge[9 * (size_t)t + 3 * (j - 1) + a] = (float)dd;
            }
        }
    }
    CGK_TRY(upload(&td.edge32, edge.data(), edge.size()));
    CGK_TRY(upload(&td.bucket_start, bstart.data(), bstart.size()));
    CGK_TRY(upload(&td.bucket_tets, btets.data(), btets.size()));
    return CG_OK;
}

// ============================================================================ host: stretched hex
// The operator of a stretched Cartesian mesh with the same arithmetic, in the same order,
// as its finite-volume definition: cell widths w = f[i+1] - f[i], centres (f[i] + f[i+1])/2,
// T_f = D_f |A_f| / |c_l - c_k| with D_f the harmonic mean of the two cells' D (0 if either
// is 0).  Slots 0..5 = x-, x+, y-, y+, z-, z+; a wall slot points at the cell itself with
// a zero transmissibility.
static double hex_face_d(double a, double b) { return (a > 0.0 && b > 0.0) ? 2.0 * a * b / (a + b) : 0.0; }

cg_status hex_build(cg_mesh *m, int nx, int ny, int nz, const double *xf, const double *yf,
                    const double *zf, const double *D) {
    const int64_t n = (int64_t)nx * ny * nz;
    const int n3[3] = {nx, ny, nz};
    const double *f[3] = {xf, yf, zf};
    std::vector<double> vc((size_t)n), diag((size_t)n, 0.0), offv(6 * (size_t)n, 0.0);
    std::vector<int32_t> offc(6 * (size_t)n);
    m->h_rowptr.assign((size_t)n + 1, 0);
    m->h_col.clear();
    m->h_val.clear();
    m->h_col.reserve(7 * (size_t)n);
    m->h_val.reserve(7 * (size_t)n);
    double max_rate = 0.0;
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
                std::pair<int32_t, double> e[7];
                int ne = 0;
                for (int a = 0; a < 3; ++a)
                    for (int sgn = 0; sgn < 2; ++sgn) {
                        const int slot = 2 * a + sgn;
                        const int j = id[a] + (sgn ? 1 : -1);
                        offc[(size_t)slot * n + k] = (int32_t)k;
                        if (j < 0 || j >= n3[a]) continue;
                        int nid[3] = {ix, iy, iz};
                        nid[a] = j;
                        const int64_t l = ((int64_t)nid[2] * ny + nid[1]) * nx + nid[0];
                        const double cl = 0.5 * (f[a][j] + f[a][j + 1]);
                        const double area = w[(a + 1) % 3] * w[(a + 2) % 3];
                        const double t = hex_face_d(dk, D ? D[l] : 1.0) * area / std::fabs(cl - c[a]);
                        offc[(size_t)slot * n + k] = (int32_t)l;
                        offv[(size_t)slot * n + k] = t;
                        diag[k] -= t;
                        e[ne++] = {(int32_t)l, t};
                    }
                e[ne++] = {(int32_t)k, diag[k]};
                std::sort(e, e + ne);
                for (int q = 0; q < ne; ++q) {
                    m->h_col.push_back(e[q].first);
                    m->h_val.push_back(e[q].second);
                }
                m->h_rowptr[k + 1] = (int32_t)m->h_col.size();
                max_rate = std::max(max_rate, -diag[k] / vc[k]);
            }
    m->h_vc = vc;
    std::vector<float> offv32(offv.size());
    for (size_t i = 0; i < offv.size(); ++i) offv32[i] = (float)offv[i];
    std::vector<double> faces;
    for (int a = 0; a < 3; ++a) faces.insert(faces.end(), f[a], f[a] + n3[a] + 1);
    TetDevice &td = m->tet;
    td.ns = 6;
    td.max_rate = max_rate;
    for (int a = 0; a < 3; ++a) td.hn[a] = n3[a];
    CGK_TRY(upload(&td.vc, vc.data(), vc.size()));
    CGK_TRY(upload(&td.diagL, diag.data(), diag.size()));
    CGK_TRY(upload(&td.offc, offc.data(), offc.size()));
    CGK_TRY(upload(&td.offv, offv.data(), offv.size()));
    CGK_TRY(upload(&td.offv32, offv32.data(), offv32.size()));
    CGK_TRY(upload(&td.faces, faces.data(), faces.size()));
    return CG_OK;
}

// Particle sets at least this large are grouped by point-location bucket before the
// tet search (smaller ones are searched in their own order).
constexpr int64_t kTetOrderMin = 1 << 16;

cg_status tet_locate_launch(cg_mesh *m, int64_t n, const double *pos, int nf, const double *w,
                            int32_t *cell_out, uint32_t *counts, uint32_t *ranks,
                            unsigned long long *bad, cudaStream_t st) {
    if (m->kind == MESH_HEX)
        CGK_LAUNCH("hex_locate", (double)n * (24 + 8 * nf + 4), st,
                   k_hex_locate<<<grid1d(n), kThreads, 0, st>>>(n, pos, m->tet, nf, w, cell_out,
                                                                counts, ranks, bad));
    else {
        // large sets: group the particles by bucket first (a counting sort) so that a
        // warp's lanes share their candidate lists; the results do not depend on the order
        const int32_t *order = nullptr;
        const TetDevice &t = m->tet;
        const int64_t nbk = (int64_t)t.nb[0] * t.nb[1] * t.nb[2];
        if (n >= kTetOrderMin) {
            const size_t s_n = ((size_t)n * 4 + 255) / 256 * 256;
            const size_t s_b = ((size_t)(nbk + 2) * 4 + 255) / 256 * 256;
            const size_t s_t = (scan_tmp_words(nbk + 2) * 4 + 255) / 256 * 256;
            CGK_TRY(m->ws_order.ensure(3 * s_n + 2 * s_b + s_t));
            char *base = m->ws_order.as<char>();
            int32_t *key = (int32_t *)base;
            uint32_t *rank = (uint32_t *)(base + s_n);
            int32_t *ord = (int32_t *)(base + 2 * s_n);
            uint32_t *cnt = (uint32_t *)(base + 3 * s_n);
            uint32_t *off = (uint32_t *)(base + 3 * s_n + s_b);
            uint32_t *tmp = (uint32_t *)(base + 3 * s_n + 2 * s_b);
            CGK_CUDA(cudaMemsetAsync(cnt, 0, (size_t)(nbk + 2) * 4, st));
            CGK_LAUNCH("tet_bucket_count", (double)n * 32, st,
                       k_tet_bucket_count<<<grid1d(n), kThreads, 0, st>>>(n, pos, t, key, rank, cnt));
            CGK_CUDA(cudaGetLastError());
            CGK_TRY(exclusive_scan_u32(cnt, off, nbk + 2, tmp, st));
            CGK_LAUNCH("tet_bucket_scatter", (double)n * 12, st,
                       k_tet_bucket_scatter<<<grid1d(n), kThreads, 0, st>>>(n, key, rank, off, ord));
            CGK_CUDA(cudaGetLastError());
            order = ord;
        }
        CGK_LAUNCH("tet_locate", (double)n * (24 + 8 * nf + 4), st,
                   k_tet_locate<<<grid1d(n), kThreads, 0, st>>>(n, pos, m->tet, nf, w, cell_out,
                                                                counts, ranks, bad, order));
    }
    CGK_CUDA(cudaGetLastError());
    return CG_OK;
}

// ============================================================================ host: diffuse
static Op make_op(cg_mesh *m, double dte, double dtau) {
    Op o;
    o.n = (int)m->ncells;
    o.vc = m->tet.vc;
    o.diagL = m->tet.diagL;
    o.offv = m->tet.offv;
    o.offv32 = m->tet.offv32;
    o.offc = m->tet.offc;
    o.dte = dte;
    o.dtau = dtau;
    o.ns = m->tet.ns;
    if (m->kind == MESH_HEX) {
        o.hx = m->tet.hn[0];
        o.hy = m->tet.hn[1];
        o.hz = m->tet.hn[2];
    }
    return o;
}

// bytes of one operator row: ns ids + ns T + diag + V_c, plus the gathered values
static thread_local int g_row_slots = 4;   // set per call from the mesh (profiling byte counts only)
static double row_bytes(int s) { return g_row_slots * 4 + g_row_slots * (s == 4 ? 4 : 8) + 16; }

static cg_status tet_fp64(cg_mesh *m, int nf, double *cells, const cg_params *p, double T,
                          cg_report *rep, cudaStream_t st) {
    const int n = (int)m->ncells;
    const double dtau = T / p->nsteps;
    const Op o = make_op(m, p->scheme == CG_SCHEME_CRANK_NICOLSON ? 0.5 * dtau : dtau, dtau);
    const double tol2 = p->tol * p->tol;
    const int G = grid1d(n);
    const dim3 grid(G, nf);
    const size_t vec = align_up((size_t)n * nf * 8);
    CGK_TRY(m->ws_diffuse.ensure(5 * vec));
    char *wb = m->ws_diffuse.as<char>();
    double *r = (double *)wb, *z = (double *)(wb + vec), *q = (double *)(wb + 2 * vec);
    double *P[2] = {(double *)(wb + 3 * vec), (double *)(wb + 4 * vec)};
    CGK_TRY(m->ws_small.ensure(4096 + align_up((size_t)nf * 3 * G * 8) + 64 * sizeof(TScal)));
    double *partials = (double *)(m->ws_small.as<char>() + 4096);
    TScal *sc = (TScal *)(m->ws_small.as<char>() + 4096 + align_up((size_t)nf * 3 * G * 8));
    CGK_CUDA(cudaMemsetAsync(sc, 0, nf * sizeof(TScal), st));
    CGK_TRY(m->h_small.ensure(4096 + 64 * sizeof(TScal)));
    TScal *hsc = (TScal *)(m->h_small.as<char>() + 4096);
    long long total = 0;
    double worst = 0;
    const double rb = row_bytes(8);
    for (int s = 0; s < p->nsteps; ++s) {
        CGK_LAUNCH("tcg64_init", (double)n * nf * (rb + 8 + 24), st,
                   k_tcg_init<<<grid, kThreads, 0, st>>>(o, p->scheme, cells, r, z, P[0], partials,
                                                         sc, tol2));
        int it = 0;
        bool all_done = false;
        while (true) {
            for (int c = 0; c < 8; ++c, ++it) {
                CGK_LAUNCH("tcg64_pass1", (double)n * nf * (rb + 16 + 16), st,
                           k_tcg_pass1<<<grid, kThreads, 0, st>>>(o, z, P[it & 1], P[(it + 1) & 1],
                                                                  q, partials, sc));
                CGK_LAUNCH("tcg64_pass2", (double)n * nf * (16 + 40 + 16), st,
                           k_tcg_pass2<<<grid, kThreads, 0, st>>>(o, P[(it + 1) & 1], q, cells, r,
                                                                  z, partials, sc, tol2));
            }
            CGK_CUDA(cudaGetLastError());
            CGK_CUDA(cudaMemcpyAsync(hsc, sc, nf * sizeof(TScal), cudaMemcpyDeviceToHost, st));
            CGK_CUDA(cudaStreamSynchronize(st));
            all_done = true;
            for (int f = 0; f < nf; ++f) all_done = all_done && hsc[f].done;
            if (all_done || it >= p->max_iter) break;
        }
        for (int f = 0; f < nf; ++f) {
            total += hsc[f].iters + 1;
            double rel = hsc[f].bb > 0 ? std::sqrt(hsc[f].rr / hsc[f].bb) : 0.0;
            worst = std::max(worst, rel);
            if (hsc[f].breakdown && hsc[f].rr > tol2 * hsc[f].bb) all_done = false;
        }
        if (!all_done) {
            if (rep) {
                rep->iters = total;
                rep->cell_updates = total * (long long)n;
                rep->final_rel_residual = worst;
            }
            return fail(CG_ENOCONV, "cg_diffuse: FP64 PCG did not reach tol in step %d", s);
        }
    }
    if (rep) {
        rep->iters = total;
        rep->cell_updates = total * (long long)n;
        rep->final_rel_residual = worst;
    }
    return CG_OK;
}

static cg_status tet_explicit(cg_mesh *m, int nf, double *cells, const cg_params *p, double T,
                              cg_report *rep, cudaStream_t st) {
    const int n = (int)m->ncells;
    const double dtau = T / p->nsteps;
    if (dtau * m->tet.max_rate > 1.0 + 1e-12)
        return fail(CG_EINVAL, "cg_diffuse: explicit Euler needs dtau <= %g on this mesh",
                    1.0 / m->tet.max_rate);
    const Op o = make_op(m, dtau, dtau);
    const size_t vec = align_up((size_t)n * nf * 8);
    CGK_TRY(m->ws_diffuse.ensure(vec));
    double *a = cells, *b = m->ws_diffuse.as<double>();
    for (int s = 0; s < p->nsteps; ++s) {
        CGK_LAUNCH("texplicit64", (double)n * nf * (row_bytes(8) + 16), st,
                   k_texplicit<<<dim3(grid1d(n), nf), kThreads, 0, st>>>(o, a, b));
        std::swap(a, b);
    }
    CGK_CUDA(cudaGetLastError());
    if (a != cells)
        CGK_CUDA(cudaMemcpyAsync(cells, a, (size_t)n * nf * 8, cudaMemcpyDeviceToDevice, st));
    CGK_CUDA(cudaStreamSynchronize(st));
    if (rep) {
        rep->iters = (long long)p->nsteps * nf;
        rep->cell_updates = rep->iters * n;
    }
    return CG_OK;
}

// The smallest eigenvalue of the Lanczos tridiagonal that m conjugate-gradient steps
// (coefficients alpha_j, beta_j) build for the preconditioned operator:
// T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}, T_{j,j+1}^2 = beta_j / alpha_j^2 (Saad,
// Iterative Methods for Sparse Linear Systems, Section 6.7.3).  Its eigenvalues (Ritz
// values) lie inside the operator's spectrum, here within (0, 2); bisection on the
// Sturm count of the LDL^T pivots below x.
static double lanczos_min(const double *alpha, const double *beta, int m) {
    std::vector<double> a(m), b2(m, 0.0);
    for (int j = 0; j < m; ++j) {
        a[j] = 1.0 / alpha[j] + (j > 0 ? beta[j - 1] / alpha[j - 1] : 0.0);
        if (j + 1 < m) b2[j] = beta[j] / (alpha[j] * alpha[j]);
    }
    auto below = [&](double x) {
        int c = 0;
        double q = a[0] - x;
        c += q < 0;
        for (int j = 1; j < m; ++j) {
            if (q == 0.0) q = 1e-300;
            q = a[j] - x - b2[j - 1] / q;
            c += q < 0;
        }
        return c;
    };
    double lo = 0.0, hi = 2.0;
    for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        (below(mid) >= 1 ? hi : lo) = mid;
    }
    return hi;
}

// Chebyshev schedule on [a, b] for a residual reduction eps: c0 and, per later
// iteration k, (c1_k, c2_k) of k_tcheb.
struct ChebSchedule {
    float c0 = 1.f;
    std::vector<float> c1, c2;
    int iterations() const { return 1 + (int)c1.size(); }
};
static ChebSchedule cheb_schedule(double a, double b, double eps) {
    ChebSchedule cs;
    const double theta = 0.5 * (a + b), delta = 0.5 * (b - a);
    cs.c0 = (float)(1.0 / theta);
    if (!(delta > 1e-12 * theta)) return cs;   // one point: D^-1 A = theta I
    const double kappa = b / a, sg = (std::sqrt(kappa) - 1.0) / (std::sqrt(kappa) + 1.0);
    const int m = std::max(1, (int)std::ceil(std::log(2.0 / eps) / -std::log(sg)));
    const double s1 = theta / delta;
    double rho = 1.0 / s1;
    for (int k = 1; k < m; ++k) {
        const double rn = 1.0 / (2.0 * s1 - rho);
        cs.c1.push_back((float)(rn * rho));
        cs.c2.push_back((float)(2.0 * rn / delta));
        rho = rn;
    }
    return cs;
}

template <class TS>
static cg_status tet_mixed(cg_mesh *m, int nf, double *cells, const cg_params *p, double T,
                           cg_report *rep, cudaStream_t st) {
    const int n = (int)m->ncells;
    const bool cn = p->scheme == CG_SCHEME_CRANK_NICOLSON;
    const double dtau = T / p->nsteps;
    Op o = make_op(m, cn ? 0.5 * dtau : dtau, dtau);
    const double tol2 = p->tol * p->tol;
    const double eps_in = sizeof(TS) == 2 ? 3e-3 : 1e-6;
    const int G = grid1d(n);
    const dim3 grid(G, nf);
    const size_t v64 = align_up((size_t)n * nf * 8), vts = align_up((size_t)n * nf * sizeof(TS));
    const size_t v32 = align_up((size_t)n * 4);
    // the Chebyshev passes (k_tcheb1, k_tcheb, k_hcheb) read Jacobi-scaled weights and
    // the scaled residual D^-1 r, which the refinement passes write to Z
    CGK_TRY(m->ws_diffuse.ensure(3 * v64 + 7 * vts + (2 + o.ns) * v32));
    char *wb = m->ws_diffuse.as<char>();
    {   // FP32 diagonal of A and its reciprocal for this call's dtau
        float *ad = (float *)(wb + 3 * v64 + 7 * vts), *iad = (float *)(wb + 3 * v64 + 7 * vts + v32);
        CGK_LAUNCH("tdiag32", (double)n * 24, st,
                   k_tdiag32<<<G, kThreads, 0, st>>>(n, o.vc, o.diagL, o.dte, ad, iad));
        CGK_CUDA(cudaGetLastError());
        o.adiag32 = ad;
        o.iadiag32 = iad;
        {
            float *w = (float *)(wb + 3 * v64 + 7 * vts + 2 * v32);
            CGK_LAUNCH("tscaled", (double)n * (16 + 12.0 * o.ns), st,
                       k_tscaled<<<G, kThreads, 0, st>>>(n, o.ns, o.vc, o.diagL, o.offv, o.dte, w));
            CGK_CUDA(cudaGetLastError());
            o.wsc32 = w;
        }
    }
    double *X1 = (double *)wb, *X2 = (double *)(wb + v64), *B = (double *)(wb + 2 * v64);
    TS *Rin = (TS *)(wb + 3 * v64), *Z = (TS *)(wb + 3 * v64 + vts), *Q = (TS *)(wb + 3 * v64 + 2 * vts);
    TS *Pp[2] = {(TS *)(wb + 3 * v64 + 3 * vts), (TS *)(wb + 3 * v64 + 4 * vts)};
    TS *D = (TS *)(wb + 3 * v64 + 5 * vts);
    TS *Cb[3] = {Q, Pp[1], D};   // the Chebyshev iterates rotate through these
    const size_t hist_bytes = align_up((size_t)nf * 2 * kHist * 8);
    CGK_TRY(m->ws_small.ensure(4096 + align_up((size_t)nf * 3 * G * 8) + 64 * sizeof(TScal) + hist_bytes));
    double *partials = (double *)(m->ws_small.as<char>() + 4096);
    TScal *sc = (TScal *)(m->ws_small.as<char>() + 4096 + align_up((size_t)nf * 3 * G * 8));
    double *hist = (double *)(m->ws_small.as<char>() + 4096 + align_up((size_t)nf * 3 * G * 8) +
                              64 * sizeof(TScal));
    CGK_CUDA(cudaMemsetAsync(sc, 0, nf * sizeof(TScal), st));
    CGK_TRY(m->h_small.ensure(4096 + 64 * sizeof(TScal) + hist_bytes));
    TScal *hsc = (TScal *)(m->h_small.as<char>() + 4096);
    double *hhist = (double *)(m->h_small.as<char>() + 4096 + 64 * sizeof(TScal));
    // Inner solver: Chebyshev on [a, 1 + rho], 1 + rho the Gershgorin bound (rho =
    // dte R / (1 + dte R), R the largest sum of a cell's transmissibilities over its
    // volume) and a from a probe (below), so every inner solve of every call is the same
    // fixed polynomial for this mesh and dte.  sweep_shape 1 keeps Jacobi-PCG throughout,
    // and so does BF16 storage: the three-term recurrence stored with an 8-bit
    // significand stalls above the inner tolerance.
    const bool want_cheb = p->sweep_shape != 1 && sizeof(TS) == 4;
    const double rho_g = o.dte * m->tet.max_rate / (1.0 + o.dte * m->tet.max_rate);
    ChebSchedule cheb;
    double cheb_sg = 0.0;   // the schedule's convergence rate per iteration
    bool have_cheb = false;
    const int max_rounds = p->max_rounds > 0 ? p->max_rounds : 12;
    const int max_inner = p->max_iter;
    const double rb32 = row_bytes(4);
    long long applications = 0, rounds_total = 0;
    double worst = 0;
    double *ubuf = cells, *F1 = X1, *F2 = X2;
    bool converged = true;
    if (want_cheb) {
        // the lower end of the Chebyshev interval for this dte: remembered per mesh, else
        // from a PCG probe solve on a fixed right-hand side (Lanczos estimate of the
        // smallest eigenvalue of D^-1 A, taken 5 % lower; never below Gershgorin's)
        double a = -1.0;
        for (const auto &e : m->spectrum)
            if (e.first == o.dte) a = e.second;
        if (a < 0) {
            CGK_LAUNCH("tprobe_init", (double)n * (8 + 4.0 * sizeof(TS)), st,
                       k_tprobe_init<TS><<<G, kThreads, 0, st>>>(o, Rin, Z, Pp[0], D, partials, sc));
            int it = 0;
            bool done = false;
            while (!done && it < std::min(max_inner, kHist)) {
                for (int c = 0; c < 8; ++c, ++it) {
                    CGK_LAUNCH(sizeof(TS) == 2 ? "tin_pass1_bf16" : "tin_pass1_fp32", (double)n * (rb32 + 4.0 * sizeof(TS)),
                               st, k_tin_pass1<TS><<<G, kThreads, 0, st>>>(o, Z, Pp[it & 1], Pp[(it + 1) & 1], Q,
                                                                            partials, sc, hist));
                    CGK_LAUNCH(sizeof(TS) == 2 ? "tin_pass2_bf16" : "tin_pass2_fp32", (double)n * (16 + 7.0 * sizeof(TS)),
                               st, k_tin_pass2<TS><<<G, kThreads, 0, st>>>(o, Pp[(it + 1) & 1], Q, D, Rin, Z, partials,
                                                                            sc, eps_in * eps_in, hist));
                }
                CGK_CUDA(cudaGetLastError());
                CGK_CUDA(cudaMemcpyAsync(hsc, sc, sizeof(TScal), cudaMemcpyDeviceToHost, st));
                CGK_CUDA(cudaStreamSynchronize(st));
                done = hsc[0].done;
            }
            // (setup of the inner solver: not counted as cell-updates of the fields)
            CGK_CUDA(cudaMemcpyAsync(hhist, hist, 2 * kHist * 8, cudaMemcpyDeviceToHost, st));
            CGK_CUDA(cudaStreamSynchronize(st));
            const int mh = std::min(hsc[0].iters, kHist);
            a = 1.0 - rho_g;
            if (!hsc[0].breakdown && mh >= 4) a = std::max(0.95 * lanczos_min(hhist, hhist + kHist, mh), a);
            if (m->spectrum.size() < 64) m->spectrum.emplace_back(o.dte, a);
        }
        cheb = cheb_schedule(a, 1.0 + rho_g, eps_in);
        have_cheb = cheb.iterations() <= max_inner;   // else PCG stays cheaper
        const double kap = (1.0 + rho_g) / a;
        cheb_sg = (std::sqrt(kap) - 1.0) / (std::sqrt(kap) + 1.0);
    }
    int s = 0;
    for (; s < p->nsteps; ++s) {
        if (have_cheb)
            CGK_LAUNCH("trefine64_first", (double)n * nf * (row_bytes(8) + 8 + 8 * cn + 2 * sizeof(TS)), st,
                       (k_trefine<TS, true, false><<<grid, kThreads, 0, st>>>(
                           o, p->scheme, ubuf, nullptr, nullptr, nullptr, nullptr, B, Rin,
                           Z, nullptr, partials, sc)));
        else
            CGK_LAUNCH("trefine64_first", (double)n * nf * (row_bytes(8) + 8 + 8 * cn + 4 * sizeof(TS)), st,
                       (k_trefine<TS, true><<<grid, kThreads, 0, st>>>(
                           o, p->scheme, ubuf, nullptr, nullptr, nullptr, nullptr, B, Rin, Z, Pp[0],
                           partials, sc)));
        CGK_CUDA(cudaMemsetAsync(D, 0, (size_t)n * nf * sizeof(TS), st));
        applications += 1;
        double *xcur = ubuf;
        int rounds = 0;
        converged = false;
        while (rounds < max_rounds) {
            TS *dsol = D;
            if (have_cheb) {
            // inner Chebyshev on A d = r, from d = 0: d_1, then one pass per iteration
            // bytes: the operator row (slots, diagonal, its reciprocal) once per cell, then
            // per field r, d_k, d_{k-1} and d_{k+1}
            CGK_LAUNCH(sizeof(TS) == 2 ? "tcheb_bf16" : "tcheb_fp32", (double)n * (4 + nf * 2.0 * sizeof(TS)), st,
                       (k_tcheb<TS, true><<<G, kThreads, 0, st>>>(o, nf, Rin, nullptr, nullptr, Cb[1],
                                                                              cheb.c0, 0.f)));
            // a later round of a step needs only what is left to the tolerance: the last
            // round's FP64 residual is on the host, so the round runs the schedule's first
            // iterations that reduce it below tol ||b|| with a tenfold margin (the
            // recurrence's coefficients do not depend on where it stops); a round that falls
            // short is followed by another, as ever
            int mi = cheb.iterations();
            if (rounds > 0 && cheb_sg > 0.0 && cheb_sg < 1.0) {
                double need = 1.0;
                for (int f = 0; f < nf; ++f)
                    if (hsc[f].rr > 0.0 && hsc[f].bb > 0.0)
                        need = std::min(need, std::sqrt(tol2 * hsc[f].bb / hsc[f].rr));
                const double eps = 0.1 * need;
                if (eps > eps_in)
                    mi = std::min(mi, std::max(1, (int)std::ceil(std::log(2.0 / eps) / -std::log(cheb_sg))));
            }
            // blocks of (row width rounded to a warp, at most 256) x (256 / that) rows
            const int hbx = std::min(kThreads, (o.hx + 31) / 32 * 32);
            const dim3 hblk((unsigned)hbx, (unsigned)(kThreads / hbx));
            const dim3 hgrid((unsigned)((o.hx + hbx - 1) / hbx),
                             (unsigned)std::min((o.hy * o.hz + (int)hblk.y - 1) / (int)hblk.y, 65535));
            for (int k = 1; k < mi; ++k) {
                const TS *dm = k == 1 ? nullptr : Cb[(k - 1) % 3];
                if (o.hx > 0)   // stretched hex mesh: implicit neighbours
                    CGK_LAUNCH(sizeof(TS) == 2 ? "tcheb_bf16" : "tcheb_fp32",
                               (double)n * (6 * 4 + nf * 4.0 * sizeof(TS)), st,
                               k_hcheb<TS><<<hgrid, hblk, 0, st>>>(o, nf, Z, Cb[k % 3], dm, Cb[(k + 1) % 3],
                                                                       cheb.c1[k - 1], cheb.c2[k - 1]));
                else if (nf == 1)   // bytes: the row's indices and scaled weights, rs, d_k, d_{k-1}, d_{k+1}
                    CGK_LAUNCH(sizeof(TS) == 2 ? "tcheb_bf16" : "tcheb_fp32", (double)n * (8.0 * o.ns + 4.0 * sizeof(TS)),
                               st, (o.ns == 4 ? k_tcheb1<TS, 4> : k_tcheb1<TS, 6>)<<<G, kThreads, 0, st>>>(
                                       o, Z, Cb[k % 3], dm, Cb[(k + 1) % 3], cheb.c1[k - 1], cheb.c2[k - 1]));
                else
                    CGK_LAUNCH(sizeof(TS) == 2 ? "tcheb_bf16" : "tcheb_fp32",
                               (double)n * (8.0 * o.ns + nf * 4.0 * sizeof(TS)), st,
                               (k_tcheb<TS, false><<<G, kThreads, 0, st>>>(
                                   o, nf, Z, Cb[k % 3], dm, Cb[(k + 1) % 3], cheb.c1[k - 1], cheb.c2[k - 1])));
            }
            CGK_CUDA(cudaGetLastError());
            dsol = Cb[mi % 3];
            applications += mi - 1;
            } else {
            // inner Jacobi-PCG on A d = r in FP32 (TS storage), from d = 0
            int it = 0;
            bool inner_done = false;
            while (!inner_done && it < max_inner) {
                for (int c = 0; c < 8; ++c, ++it) {
                    CGK_LAUNCH(sizeof(TS) == 2 ? "tin_pass1_bf16" : "tin_pass1_fp32",
                               (double)n * nf * (rb32 + 4.0 * sizeof(TS)), st,
                               k_tin_pass1<TS><<<grid, kThreads, 0, st>>>(
                                   o, Z, Pp[it & 1], Pp[(it + 1) & 1], Q, partials, sc, nullptr));
                    CGK_LAUNCH(sizeof(TS) == 2 ? "tin_pass2_bf16" : "tin_pass2_fp32",
                               (double)n * nf * (16 + 7.0 * sizeof(TS)), st,
                               k_tin_pass2<TS><<<grid, kThreads, 0, st>>>(
                                   o, Pp[(it + 1) & 1], Q, D, Rin, Z, partials, sc, eps_in * eps_in, nullptr));
                }
                CGK_CUDA(cudaGetLastError());
                CGK_CUDA(cudaMemcpyAsync(hsc, sc, nf * sizeof(TScal), cudaMemcpyDeviceToHost, st));
                CGK_CUDA(cudaStreamSynchronize(st));
                inner_done = true;
                for (int f = 0; f < nf; ++f) inner_done = inner_done && hsc[f].done;
            }
            int used = 0;
            for (int f = 0; f < nf; ++f) used = std::max(used, hsc[f].iters);
            applications += used;
            }
            // x += d, new FP64 residual, start of the next inner solve
            double *xnext = (xcur == F1) ? F2 : F1;
            if (have_cheb) {
                CGK_LAUNCH("tadd", (double)n * nf * (16 + sizeof(TS)), st,
                           k_tadd<TS><<<grid1d((int64_t)n * nf), kThreads, 0, st>>>((size_t)n * nf, xcur, dsol,
                                                                                 xnext));
                CGK_LAUNCH("trefine64", (double)n * nf * (row_bytes(8) + 8 + sizeof(TS) + 8), st,
                           (k_trefine<TS, false, false><<<grid, kThreads, 0, st>>>(
                               o, p->scheme, xnext, nullptr, ubuf, B, nullptr, nullptr, Rin,
                               Z, nullptr, partials, sc)));
            } else {
                CGK_LAUNCH("trefine64", (double)n * nf * (row_bytes(8) + 8 + sizeof(TS) * 5 + 16), st,
                           (k_trefine<TS, false><<<grid, kThreads, 0, st>>>(
                               o, p->scheme, xcur, dsol, ubuf, B, xnext, nullptr, Rin, Z, Pp[0],
                               partials, sc)));
            }
            CGK_CUDA(cudaGetLastError());
            if (!have_cheb) CGK_CUDA(cudaMemsetAsync(D, 0, (size_t)n * nf * sizeof(TS), st));
            applications += 1;
            ++rounds;
            xcur = xnext;
            CGK_CUDA(cudaMemcpyAsync(hsc, sc, nf * sizeof(TScal), cudaMemcpyDeviceToHost, st));
            CGK_CUDA(cudaStreamSynchronize(st));
            converged = true;
            for (int f = 0; f < nf; ++f) converged = converged && (hsc[f].rr <= tol2 * hsc[f].bb);
            if (converged) break;
        }
        rounds_total += rounds;
        for (int f = 0; f < nf; ++f)
            worst = std::max(worst, hsc[f].bb > 0 ? std::sqrt(hsc[f].rr / hsc[f].bb) : 0.0);
        double *old_u = ubuf, *other = (xcur == F1) ? F2 : F1;
        ubuf = xcur;
        F1 = old_u;
        F2 = other;
        if (!converged) break;
    }
    if (ubuf != cells)
        CGK_CUDA(cudaMemcpyAsync(cells, ubuf, (size_t)n * nf * 8, cudaMemcpyDeviceToDevice, st));
    CGK_CUDA(cudaStreamSynchronize(st));
    if (rep) {
        rep->iters = applications * nf;
        rep->refine_rounds = rounds_total;
        rep->cell_updates = applications * nf * (long long)n;
        rep->final_rel_residual = worst;
    }
    if (!converged)
        return fail(CG_ENOCONV, "cg_diffuse: refinement did not reach tol in step %d", s);
    return CG_OK;
}

cg_status diffuse_tet_run(cg_mesh *m, int nf, double *cells, const cg_params *p, cg_report *rep,
                          cudaStream_t st) {
    g_row_slots = m->tet.ns;
    double T = p->bandwidth > 0.0 ? p->bandwidth * p->bandwidth / 4.0 : p->T;
    if (p->scheme == CG_SCHEME_EXPLICIT_EULER) {
        if (p->fused_k > 0)
            return fail(CG_EINVAL, "cg_diffuse: fused_k (blocked explicit steps) needs a uniform structured mesh");
        return tet_explicit(m, nf, cells, p, T, rep, st);
    }
    if (p->precision == CG_PREC_FP64) return tet_fp64(m, nf, cells, p, T, rep, st);
    if (p->precision == CG_PREC_FP32_REFINE || p->precision == CG_PREC_FP32_DF_REFINE)
        return tet_mixed<float>(m, nf, cells, p, T, rep, st);
    return tet_mixed<__nv_bfloat16>(m, nf, cells, p, T, rep, st);
}

}  // namespace cgk

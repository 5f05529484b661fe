// stencil.cu -- diffusion smoothing on a uniform hex mesh (Section 2.6 step 2,
// Section 3.2 Eq. (diffusion), zero-flux walls of Section 3.2.2).
//
// Finite-volume 7-point Laplacian per unit cell volume: (L u)_k = sum over the
// existing face neighbours l of (u_l - u_k) / dx^2.  A wall face carries no flux, so
// a missing neighbour drops out of both the sum and the diagonal.  One pseudo-step of
// implicit Euler solves A u^{n+1} = u^n with A = I - c L (c = dtau/dx^2, L unscaled);
// Crank-Nicolson (the paper's scheme, Section 5.1) solves (I - c/2 L) u^{n+1} =
// (I + c/2 L) u^n; explicit Euler is u += c L u.
//
// Two solvers:
//  * FP64: conjugate gradients in two fused passes per iteration (pass 1 forms the new
//    search direction p = r + beta p on the fly at a cell and its neighbours, and
//    accumulates p.Ap; pass 2 recomputes Ap, updates x and r, and accumulates r.r).
//    Scalars stay on the device; the last block of each pass finishes the reduction
//    in a fixed order, so results are run-to-run deterministic.
//  * Mixed: FP64 iterative refinement.  A fused FP64 pass applies the previous
//    correction (x += d), forms the true residual r = b - A x in FP64 and stores it in
//    FP32 (or BF16); the correction A d = r is then solved in FP32 by Chebyshev
//    iteration, whose spectrum bounds are known in closed form on this mesh:
//    lambda(A) lies in [1, 1 + 4 c sum_axes sin^2(pi (n-1) / (2n))] (DCT-II
//    eigenvalues).  Chebyshev needs no inner products, only stencil sweeps.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cmath>
#include <cstdio>
#include <vector>

#include "internal.cuh"
#include "reduce.cuh"

namespace cgk {

namespace {

constexpr int TX = 32, TY = 8;     // xy tile of the 2.5D sweeps (one thread per column)

struct Geo {
    int nx, ny, nz;
    int nxy;
    int n;
};

// Launch geometry of a 2.5D sweep: blocks of TX x TY columns, each marching over zlen
// planes; blockIdx.z = f * nzc + z-chunk.
struct Sweep {
    dim3 grid;
    int zlen, nzc, nb;   // planes per chunk, chunks, blocks per field
};

Sweep make_sweep(const Geo &g, int nf) {
    Sweep s;
    int gx = (g.nx + TX - 1) / TX, gy = (g.ny + TY - 1) / TY;
    long long cols = (long long)gx * gy * nf;
    long long target = (long long)num_sms() * 16;   // ~2 waves of 8 resident blocks per SM
    int nzc = (int)((target + cols - 1) / cols);
    int zlen = (g.nz + nzc - 1) / nzc;
    if (zlen < 4) zlen = g.nz < 4 ? g.nz : 4;
    nzc = (g.nz + zlen - 1) / zlen;
    s.grid = dim3(gx, gy, nzc * nf);
    s.zlen = zlen;
    s.nzc = nzc;
    s.nb = gx * gy * nzc;
    return s;
}

struct BlockPos {
    int f, z0, z1, bid, nb;
};

__device__ __forceinline__ BlockPos block_pos(const Geo &g, int zlen, int nzc) {
    BlockPos p;
    p.f = blockIdx.z / nzc;
    int zc = blockIdx.z - p.f * nzc;
    p.z0 = zc * zlen;
    p.z1 = min(g.nz, p.z0 + zlen);
    p.bid = (zc * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    p.nb = gridDim.x * gridDim.y * nzc;
    return p;
}

// The 2.5D engine.  Each thread owns one (x, y) column of the tile and marches over the
// planes [z0, z1): the value of the stencil field at a cell is produced once
// (produce(k)), kept in a 3-deep register queue for the z neighbours and published in a
// shared (TY+2) x (TX+2) plane for the x and y neighbours.  For every cell of the
// column, consume(k, v, s, nn) receives its value v, the sum s of its existing face
// neighbours (order x-, x+, y-, y+, z-, z+) and their number nn: a wall face has no
// neighbour, so it adds nothing to s or nn (zero flux).
template <class T, class Produce, class Consume>
__device__ __forceinline__ void sweep25_at(const Geo &g, int bx, int by, int z0, int z1,
                                           Produce produce, Consume consume) {
    __shared__ T pl[TY + 2][TX + 2];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = bx * TX + tx, y = by * TY + ty;
    const bool own = (x < g.nx) && (y < g.ny);
    const int kxy = y * g.nx + x;
    const bool hxl = (tx == 0) && (x > 0) && (y < g.ny);
    const bool hxh = (tx == TX - 1) && (x + 1 < g.nx) && (y < g.ny);
    const bool hyl = (ty == 0) && (y > 0) && (x < g.nx);
    const bool hyh = (ty == TY - 1) && (y + 1 < g.ny) && (x < g.nx);
    T vdn = T(0), vc = T(0), vup = T(0);
    if (own) {
        if (z0 > 0) vdn = produce(kxy + (z0 - 1) * g.nxy);
        if (z0 < z1) vc = produce(kxy + z0 * g.nxy);
    }
    for (int z = z0; z < z1; ++z) {
        const int kz = kxy + z * g.nxy;
        vup = T(0);
        if (own && z + 1 < g.nz) vup = produce(kz + g.nxy);
        if (own) pl[ty + 1][tx + 1] = vc;
        if (hxl) pl[ty + 1][0] = produce(kz - 1);
        if (hxh) pl[ty + 1][TX + 1] = produce(kz + 1);
        if (hyl) pl[0][tx + 1] = produce(kz - g.nx);
        if (hyh) pl[TY + 1][tx + 1] = produce(kz + g.nx);
        __syncthreads();
        if (own) {
            T s = T(0);
            int nn = 0;
            if (x > 0) { s += pl[ty + 1][tx]; ++nn; }
            if (x + 1 < g.nx) { s += pl[ty + 1][tx + 2]; ++nn; }
            if (y > 0) { s += pl[ty][tx + 1]; ++nn; }
            if (y + 1 < g.ny) { s += pl[ty + 2][tx + 1]; ++nn; }
            if (z > 0) { s += vdn; ++nn; }
            if (z + 1 < g.nz) { s += vup; ++nn; }
            consume(kz, vc, s, nn);
        }
        __syncthreads();
        vdn = vc;
        vc = vup;
    }
}

template <class T, class Produce, class Consume>
__device__ __forceinline__ void sweep25(const Geo &g, int z0, int z1, Produce produce,
                                        Consume consume) {
    sweep25_at<T>(g, blockIdx.x, blockIdx.y, z0, z1, produce, consume);
}

struct Scal {
    double rr, bb, alpha, beta;
    int done, iters;
    unsigned int ticket;
    int breakdown;
};

// Diagonal of A = I - ce L per neighbour count: dg[nn] = 1 + ce * nn.
struct Coef64 {
    double ce;
    double dg[7];
};
struct Coef32 {
    float ce;
    float dg[7];
};

// ================================================================ FP64 conjugate gradients
// r = b - A x = c L x for both schemes (x = u^n), p = r; b = u^n (implicit Euler) or
// u^n + c/2 L u^n (Crank-Nicolson).  rr and bb are reduced.
__global__ void __launch_bounds__(kThreads) k_cg_init(Geo g, int zlen, int nzc, double c,
                                                      int scheme, const double *__restrict__ xall,
                                                      double *__restrict__ rall,
                                                      double *__restrict__ pall,
                                                      double *__restrict__ partials_all,
                                                      Scal *__restrict__ sc, double tol2) {
    const BlockPos bp = block_pos(g, zlen, nzc);
    const size_t off = (size_t)bp.f * g.n;
    const double *x = xall + off;
    double *r = rall + off;
    double *p = pall + off;
    double rr = 0.0, bb = 0.0;
    sweep25<double>(
        g, bp.z0, bp.z1, [&](int k) { return x[k]; },
        [&](int k, double v, double s, int nn) {
            double lx = s - nn * v;
            double rk = c * lx;
            double bk = scheme == 1 ? v + 0.5 * c * lx : v;
            r[k] = rk;
            p[k] = rk;
            rr += rk * rk;
            bb += bk * bk;
        });
    double vals[2] = {block_sum(rr), block_sum(bb)};
    double *partials = partials_all + (size_t)bp.f * 2 * bp.nb;
    if (arrive(partials, 2, vals, bp.bid, bp.nb, &sc[bp.f].ticket)) {
        double RR = finish_sum(partials, 0, bp.nb);
        double BB = finish_sum(partials, 1, bp.nb);
        if (is_thread0()) {
            Scal &S = sc[bp.f];
            S.rr = RR;
            S.bb = BB;
            S.beta = 0.0;
            S.iters = 0;
            S.breakdown = 0;
            S.done = (RR <= tol2 * BB) ? 1 : 0;
            S.ticket = 0;
        }
    }
}

// pass 1: p = r + beta p (produced once per cell), accumulate p.Ap
__global__ void __launch_bounds__(kThreads) k_cg_pass1(Geo g, int zlen, int nzc, Coef64 cf,
                                                       const double *__restrict__ rall,
                                                       const double *__restrict__ pin_all,
                                                       double *__restrict__ pout_all,
                                                       double *__restrict__ partials_all,
                                                       Scal *__restrict__ sc) {
    const BlockPos bp = block_pos(g, zlen, nzc);
    if (sc[bp.f].done) return;
    const double beta = sc[bp.f].beta;
    const size_t off = (size_t)bp.f * g.n;
    const double *r = rall + off;
    const double *pin = pin_all + off;
    double *pout = pout_all + off;
    double pap = 0.0;
    __shared__ double sdg[8];
    stage_table(sdg, cf.dg);
    sweep25<double>(
        g, bp.z0, bp.z1, [&](int k) { return fma(beta, pin[k], r[k]); },
        [&](int k, double v, double s, int nn) {
            double ap = fma(sdg[nn], v, -cf.ce * s);
            pout[k] = v;
            pap = fma(v, ap, pap);
        });
    double val = block_sum(pap);
    double *partials = partials_all + (size_t)bp.f * 2 * bp.nb;
    if (arrive(partials, 1, &val, bp.bid, bp.nb, &sc[bp.f].ticket)) {
        double PAP = finish_sum(partials, 0, bp.nb);
        if (is_thread0()) {
            Scal &S = sc[bp.f];
            if (PAP > 0.0) {
                S.alpha = S.rr / PAP;
            } else {
                S.alpha = 0.0;
                S.breakdown = 1;
                S.done = 1;
            }
            S.ticket = 0;
        }
    }
}

// pass 2: recompute Ap, x += alpha p, r -= alpha Ap, accumulate r.r
__global__ void __launch_bounds__(kThreads) k_cg_pass2(Geo g, int zlen, int nzc, Coef64 cf,
                                                       const double *__restrict__ pall,
                                                       double *__restrict__ xall,
                                                       double *__restrict__ rall,
                                                       double *__restrict__ partials_all,
                                                       Scal *__restrict__ sc, double tol2) {
    const BlockPos bp = block_pos(g, zlen, nzc);
    if (sc[bp.f].done) return;
    const double alpha = sc[bp.f].alpha;
    const size_t off = (size_t)bp.f * g.n;
    const double *p = pall + off;
    double *x = xall + off;
    double *r = rall + off;
    double rr = 0.0;
    __shared__ double sdg[8];
    stage_table(sdg, cf.dg);
    sweep25<double>(
        g, bp.z0, bp.z1, [&](int k) { return p[k]; },
        [&](int k, double v, double s, int nn) {
            double ap = fma(sdg[nn], v, -cf.ce * s);
            x[k] = fma(alpha, v, x[k]);
            double rk = fma(-alpha, ap, r[k]);
            r[k] = rk;
            rr = fma(rk, rk, rr);
        });
    double val = block_sum(rr);
    double *partials = partials_all + (size_t)bp.f * 2 * bp.nb;
    if (arrive(partials, 1, &val, bp.bid, bp.nb, &sc[bp.f].ticket)) {
        double RR = finish_sum(partials, 0, bp.nb);
        if (is_thread0()) {
            Scal &S = sc[bp.f];
            S.beta = RR / S.rr;
            S.rr = RR;
            S.iters += 1;
            S.done = (RR <= tol2 * S.bb) ? 1 : 0;
            S.ticket = 0;
        }
    }
}

// explicit Euler: x_out = x + c L x (FP64)
__global__ void __launch_bounds__(kThreads) k_explicit(Geo g, int zlen, int nzc, double c,
                                                       const double *__restrict__ xin_all,
                                                       double *__restrict__ xout_all) {
    const BlockPos bp = block_pos(g, zlen, nzc);
    const size_t off = (size_t)bp.f * g.n;
    const double *x = xin_all + off;
    double *y = xout_all + off;
    sweep25<double>(
        g, bp.z0, bp.z1, [&](int k) { return x[k]; },
        [&](int k, double v, double s, int nn) { y[k] = v + c * (s - nn * v); });
}

// ================================================================ mixed precision
template <class TS> __device__ __forceinline__ float ld(const TS *p, int i);
template <> __device__ __forceinline__ float ld<float>(const float *p, int i) { return p[i]; }
template <> __device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16 *p, int i) {
    return __bfloat162float(p[i]);
}
// L2-coherent loads (bypass L1) for data that other blocks of the same launch write.
template <class TS> __device__ __forceinline__ float ldcg(const TS *p, int i);
template <> __device__ __forceinline__ float ldcg<float>(const float *p, int i) {
    return __ldcg(p + i);
}
template <> __device__ __forceinline__ float ldcg<__nv_bfloat16>(const __nv_bfloat16 *p, int i) {
    unsigned short u = __ldcg(reinterpret_cast<const unsigned short *>(p) + i);
    return __bfloat162float(__ushort_as_bfloat16(u));
}
template <class TS> __device__ __forceinline__ void st(TS *p, int i, float v);
template <> __device__ __forceinline__ void st<float>(float *p, int i, float v) { p[i] = v; }
template <> __device__ __forceinline__ void st<__nv_bfloat16>(__nv_bfloat16 *p, int i, float v) {
    p[i] = __float2bfloat16_rn(v);
}

struct RefScal {
    double rr, bb;
    unsigned int ticket;
    int pad;
};

// One FP64 refinement pass.  kFirst: x = x_in (no correction), r = c L x_in, and
// b = x_in (implicit Euler) or x_in + c/2 L x_in written to b_out (Crank-Nicolson).
// Otherwise x = x_in + d (produced once per cell), x_out = x, r = b - A x.  Stores r and
// the first Chebyshev iterate y1 = gamma r in the storage type; reduces ||r||^2 (and
// ||b||^2 on the first pass) in FP64.
template <class TS, bool kFirst>
__global__ void __launch_bounds__(kThreads) k_refine(Geo g, int zlen, int nzc, double c,
                                                     Coef64 cf, int scheme,
                                                     const double *__restrict__ xin_all,
                                                     const TS *__restrict__ d_all,
                                                     const double *__restrict__ b_all,
                                                     double *__restrict__ xout_all,
                                                     double *__restrict__ bout_all,
                                                     TS *__restrict__ r_all, TS *__restrict__ y1_all,
                                                     float gamma, double *__restrict__ partials_all,
                                                     RefScal *__restrict__ sc) {
    const BlockPos bp = block_pos(g, zlen, nzc);
    const size_t off = (size_t)bp.f * g.n;
    const double *xin = xin_all + off;
    TS *r = r_all + off;
    TS *y1 = y1_all + off;
    double rr = 0.0, bb = 0.0;
    if (kFirst) {
        sweep25<double>(
            g, bp.z0, bp.z1, [&](int k) { return xin[k]; },
            [&](int k, double v, double s, int nn) {
                double lx = s - nn * v;
                double rk = c * lx;
                double bk = v;
                if (scheme == 1) {
                    bk = fma(0.5 * c, lx, v);
                    bout_all[off + k] = bk;
                }
                bb = fma(bk, bk, bb);
                float rf = (float)rk;
                st(r, k, rf);
                st(y1, k, gamma * rf);
                rr = fma(rk, rk, rr);
            });
    } else {
        const TS *d = d_all + off;
        const double *b = b_all + off;
        double *xout = xout_all + off;
        __shared__ double sdg[8];
        stage_table(sdg, cf.dg);
        sweep25<double>(
            g, bp.z0, bp.z1, [&](int k) { return xin[k] + (double)ld(d, k); },
            [&](int k, double v, double s, int nn) {
                xout[k] = v;
                double rk = fma(cf.ce, s, fma(-sdg[nn], v, b[k]));   // b - (dg v - ce s)
                float rf = (float)rk;
                st(r, k, rf);
                st(y1, k, gamma * rf);
                rr = fma(rk, rk, rr);
            });
    }
    double vals[2] = {block_sum(rr), kFirst ? block_sum(bb) : 0.0};
    double *partials = partials_all + (size_t)bp.f * 2 * bp.nb;
    if (arrive(partials, kFirst ? 2 : 1, vals, bp.bid, bp.nb, &sc[bp.f].ticket)) {
        double RR = finish_sum(partials, 0, bp.nb);
        double BB = kFirst ? finish_sum(partials, 1, bp.nb) : 0.0;
        if (is_thread0()) {
            sc[bp.f].rr = RR;
            if (kFirst) sc[bp.f].bb = BB;
            sc[bp.f].ticket = 0;
        }
    }
}

// One Chebyshev iteration (see k_cheb_loop for the recurrence) as its own launch:
// y_next = omega (y - y_prev + gamma (r - A y)) + y_prev; y_prev == nullptr means 0.
// y_next may alias y_prev (both are accessed only at the cell itself).
template <class TS>
__global__ void __launch_bounds__(kThreads) k_cheb(Geo g, int zlen, int nzc, Coef32 cf,
                                                   float gamma, float omega,
                                                   const TS *__restrict__ y_all,
                                                   const TS *yprev_all,
                                                   const TS *__restrict__ r_all, TS *ynext_all) {
    const BlockPos bp = block_pos(g, zlen, nzc);
    const size_t off = (size_t)bp.f * g.n;
    const TS *y = y_all + off;
    const TS *r = r_all + off;
    const TS *yp = yprev_all ? yprev_all + off : nullptr;
    TS *yn = ynext_all + off;
    __shared__ float sdg[8];
    stage_table(sdg, cf.dg);
    sweep25<float>(
        g, bp.z0, bp.z1, [&](int k) { return ld(y, k); },
        [&](int k, float v, float s, int nn) {
            float ay = fmaf(sdg[nn], v, -cf.ce * s);
            float ypk = yp ? ld(yp, k) : 0.0f;
            st(yn, k, fmaf(omega, v - ypk + gamma * (ld(r, k) - ay), ypk));
        });
}

// ---------------------------------------------------------------- grid barrier
// A barrier over all blocks of a cooperative launch (all blocks co-resident).  The
// wait is bounded: a block that spins longer than `budget` clock cycles raises err and
// every block gives up at its next barrier, so the kernel always ends; the host then
// reports CG_ETIMEOUT.
struct GridBar {
    unsigned int count;
    unsigned int gen;
    int err;
    int pad;
};

__device__ __forceinline__ bool grid_sync(GridBar *gb, unsigned nblocks, long long budget) {
    __shared__ int s_ok;
    __syncthreads();
    if (is_thread0()) {
        volatile unsigned int *vgen = &gb->gen;
        volatile int *verr = &gb->err;
        const unsigned int g0 = *vgen;
        __threadfence();
        int ok = 1;
        const unsigned int arrived = atomicAdd(&gb->count, 1u);
        if (arrived == nblocks - 1) {
            gb->count = 0;
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g0) {
                if (*verr) { ok = 0; break; }
                if (clock64() - t0 > budget) {
                    atomicExch(&gb->err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        if (*verr) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The whole inner Chebyshev solve of one refinement round in one cooperative launch.
// Chebyshev iteration for A y = r on the spectrum [1, lmax] (theta, delta its centre
// and half-width, sigma = theta/delta, gamma = 1/theta): y_1 = gamma r, and
// y_{k+1} = omega_k (y_k - y_{k-1} + gamma (r - A y_k)) + y_{k-1} with omega_1 =
// 1/(1 - 1/(2 sigma^2)), omega_k = 1/(1 - omega_{k-1}/(4 sigma^2)); FP32 arithmetic,
// TS storage, y_{k+1} written over y_{k-1}.  Iterations k = 1 .. m-1, each a pass over every work
// item (xy tile x z-chunk x field) with a grid barrier between iterations.  y1 holds
// gamma r on entry; the result is left where the host-side rotation says.
template <class TS>
__global__ void __launch_bounds__(kThreads) k_cheb_loop(Geo g, int zlen, int nzc, int gx, int gy,
                                                        int nitems, Coef32 cf, float gamma,
                                                        double sigma, int m, TS *y1,
                                                        TS *yother, const TS *__restrict__ r_all,
                                                        GridBar *gb, long long budget) {
    __shared__ float sdg[8];
    stage_table(sdg, cf.dg);
    __syncthreads();
    TS *ycur = y1, *yprev = nullptr;
    double om = 1.0;
    for (int k = 1; k < m; ++k) {
        if (sigma > 0.0) {
            om = (k == 1) ? 1.0 / (1.0 - 1.0 / (2.0 * sigma * sigma))
                          : 1.0 / (1.0 - om / (4.0 * sigma * sigma));
        }
        const float omega = (float)om;
        TS *ynext = yprev ? yprev : yother;
        for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
            int t = it;
            const int bx = t % gx;
            t /= gx;
            const int by = t % gy;
            t /= gy;
            const int zc = t % nzc;
            const int f = t / nzc;
            const int z0 = zc * zlen, z1 = min(g.nz, z0 + zlen);
            const size_t off = (size_t)f * g.n;
            const TS *y = ycur + off;
            const TS *r = r_all + off;
            const TS *yp = yprev ? yprev + off : nullptr;
            TS *yn = ynext + off;
            sweep25_at<float>(
                g, bx, by, z0, z1, [&](int q) { return ldcg(y, q); },
                [&](int q, float v, float s, int nn) {
                    float ay = fmaf(sdg[nn], v, -cf.ce * s);
                    float ypk = yp ? ldcg(yp, q) : 0.0f;
                    st(yn, q, fmaf(omega, v - ypk + gamma * (ld(r, q) - ay), ypk));
                });
        }
        yprev = ycur;
        ycur = ynext;
        if (k + 1 < m && !grid_sync(gb, gridDim.x, budget)) return;
    }
}

// sum_k V_c,k u_k per field (1-D grid-stride; any mesh)
__global__ void k_mass(int n, const double *__restrict__ u_all, const double *__restrict__ vc,
                       double vcu, double *__restrict__ partials_all, unsigned int *tickets,
                       double *__restrict__ out) {
    const int f = blockIdx.y;
    const double *u = u_all + (size_t)f * n;
    double s = 0.0;
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < n; k += gridDim.x * kThreads)
        s += (vc ? vc[k] : vcu) * u[k];
    double v = block_sum(s);
    double *partials = partials_all + (size_t)f * gridDim.x;
    if (arrive(partials, 1, &v, blockIdx.x, gridDim.x, &tickets[f])) {
        double S = finish_sum(partials, 0, gridDim.x);
        if (is_thread0()) {
            out[f] = S;
            tickets[f] = 0;
        }
    }
}

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

int stencil_grid(int n) {
    int b = (n + kThreads - 1) / kThreads;
    int cap = num_sms() * 8;
    return b < cap ? (b < 1 ? 1 : b) : cap;
}

// Blocks of a cooperative launch: all must be co-resident (at most 4 per SM here).
template <class K> int coop_blocks(K kernel) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess)
        per_sm = 1;
    per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);
    return per_sm * num_sms();
}

// Work items (xy tile x z-chunk x field) for a persistent sweep over G blocks.
struct Items {
    int gx, gy, zlen, nzc, n;
};
Items make_items(const Geo &g, int nf, int G) {
    Items it;
    it.gx = (g.nx + TX - 1) / TX;
    it.gy = (g.ny + TY - 1) / TY;
    long long cols = (long long)it.gx * it.gy * nf;
    int nzc = (int)((G + cols - 1) / cols);
    if (nzc < 1) nzc = 1;
    it.zlen = (g.nz + nzc - 1) / nzc;
    it.nzc = (g.nz + it.zlen - 1) / it.zlen;
    it.n = (int)(cols * it.nzc);
    return it;
}

Coef64 coef64(double ce) {
    Coef64 c;
    c.ce = ce;
    for (int q = 0; q < 7; ++q) c.dg[q] = 1.0 + ce * q;
    return c;
}

Coef32 coef32(double ce) {
    Coef32 c;
    c.ce = (float)ce;
    for (int q = 0; q < 7; ++q) c.dg[q] = (float)(1.0 + ce * q);
    return c;
}

// Chebyshev iteration count for a residual reduction eps on spectrum [1, lmax].
int cheb_iters(double lmax, double eps) {
    if (lmax <= 1.0 + 1e-12) return 1;
    double kappa = lmax;
    double rho = (std::sqrt(kappa) - 1.0) / (std::sqrt(kappa) + 1.0);
    int m = (int)std::ceil(std::log(2.0 * std::sqrt(kappa) / eps) / std::log(1.0 / rho));
    return m < 1 ? 1 : (m > 400 ? 400 : m);
}

}  // namespace

// ============================================================================ host side
cg_status field_mass(cg_mesh *m, int nf, const double *cells, double *mass_host, cudaStream_t st) {
    int n = (int)m->ncells;
    int G = stencil_grid(n);
    size_t need = align_up((size_t)nf * G * 8) + 64 * 8 + 64 * 4;
    CGK_TRY(m->ws_small.ensure(4096 + need));
    char *base = m->ws_small.as<char>() + 4096;
    double *partials = (double *)base;
    double *out = (double *)(base + align_up((size_t)nf * G * 8));
    unsigned int *tickets = (unsigned int *)(out + 64);
    CGK_CUDA(cudaMemsetAsync(tickets, 0, 64 * 4, st));
    const double *vc = m->kind == MESH_TET ? m->tet.vc : nullptr;
    double vcu = (m->dx * m->dx) * m->dx;
    CGK_LAUNCH("mass", (double)n * nf * 8, st,
               k_mass<<<dim3(G, nf), kThreads, 0, st>>>(n, cells, vc, vcu, partials, tickets, out));
    CGK_CUDA(cudaGetLastError());
    CGK_TRY(m->h_small.ensure(4096));
    CGK_CUDA(cudaMemcpyAsync(m->h_small.as<char>() + 2048, out, nf * 8, cudaMemcpyDeviceToHost, st));
    CGK_CUDA(cudaStreamSynchronize(st));
    for (int f = 0; f < nf; ++f) mass_host[f] = ((double *)(m->h_small.as<char>() + 2048))[f];
    return CG_OK;
}

static cg_status diffuse_fp64(cg_mesh *m, int nf, double *cells, const cg_params *p, double T,
                              cg_report *rep, cudaStream_t st) {
    const int n = (int)m->ncells;
    Geo g{m->nx, m->ny, m->nz, m->nx * m->ny, n};
    const double dtau = T / p->nsteps;
    const double c = dtau / (m->dx * m->dx);
    const double ce = p->scheme == CG_SCHEME_CRANK_NICOLSON ? 0.5 * c : c;
    const double tol2 = p->tol * p->tol;
    const Sweep sw = make_sweep(g, nf);
    const int G = sw.nb;
    const Coef64 cf = coef64(ce);
    const dim3 blk(TX, TY);
    const size_t vec = align_up((size_t)n * nf * 8);
    CGK_TRY(m->ws_diffuse.ensure(3 * vec));
    double *r = (double *)m->ws_diffuse.as<char>();
    double *P[2] = {(double *)(m->ws_diffuse.as<char>() + vec),
                    (double *)(m->ws_diffuse.as<char>() + 2 * vec)};
    CGK_TRY(m->ws_small.ensure(4096 + align_up((size_t)nf * 2 * G * 8) + 64 * sizeof(Scal)));
    double *partials = (double *)(m->ws_small.as<char>() + 4096);
    Scal *sc = (Scal *)(m->ws_small.as<char>() + 4096 + align_up((size_t)nf * 2 * G * 8));
    CGK_CUDA(cudaMemsetAsync(sc, 0, nf * sizeof(Scal), st));
    CGK_TRY(m->h_small.ensure(4096 + 64 * sizeof(Scal)));
    Scal *hsc = (Scal *)(m->h_small.as<char>() + 4096);
    long long total_iters = 0;
    double worst = 0.0;
    const int chunk = 8;
    for (int s = 0; s < p->nsteps; ++s) {
        CGK_LAUNCH("cg64_init", (double)n * nf * 24, st,
                   k_cg_init<<<sw.grid, blk, 0, st>>>(g, sw.zlen, sw.nzc, c, p->scheme, cells, r,
                                                      P[0], partials, sc, tol2));
        CGK_CUDA(cudaGetLastError());
        int it = 0;
        bool all_done = false;
        while (true) {
            for (int q = 0; q < chunk; ++q, ++it) {
                CGK_LAUNCH("cg64_pass1", (double)n * nf * 24, st,
                           k_cg_pass1<<<sw.grid, blk, 0, st>>>(g, sw.zlen, sw.nzc, cf, r,
                                                               P[it & 1], P[(it + 1) & 1],
                                                               partials, sc));
                CGK_LAUNCH("cg64_pass2", (double)n * nf * 40, st,
                           k_cg_pass2<<<sw.grid, blk, 0, st>>>(g, sw.zlen, sw.nzc, cf,
                                                               P[(it + 1) & 1], cells, r,
                                                               partials, sc, tol2));
            }
            CGK_CUDA(cudaGetLastError());
            CGK_CUDA(cudaMemcpyAsync(hsc, sc, nf * sizeof(Scal), cudaMemcpyDeviceToHost, st));
            CGK_CUDA(cudaStreamSynchronize(st));
            all_done = true;
            for (int f = 0; f < nf; ++f) all_done = all_done && hsc[f].done;
            if (all_done || it >= p->max_iter) break;
        }
        for (int f = 0; f < nf; ++f) {
            total_iters += hsc[f].iters + 1;
            double rel = hsc[f].bb > 0 ? std::sqrt(hsc[f].rr / hsc[f].bb) : 0.0;
            if (rel > worst) worst = rel;
            if (hsc[f].breakdown && hsc[f].rr > tol2 * hsc[f].bb) all_done = false;
        }
        if (!all_done) {
            if (rep) {
                rep->iters = total_iters;
                rep->cell_updates = total_iters * (long long)n;
                rep->final_rel_residual = worst;
            }
            return fail(CG_ENOCONV, "cg_diffuse: FP64 CG did not reach tol in step %d", s);
        }
    }
    if (rep) {
        rep->iters = total_iters;
        rep->cell_updates = total_iters * (long long)n;
        rep->final_rel_residual = worst;
    }
    return CG_OK;
}

static cg_status diffuse_explicit(cg_mesh *m, int nf, double *cells, const cg_params *p, double T,
                                  cg_report *rep, cudaStream_t st) {
    const int n = (int)m->ncells;
    Geo g{m->nx, m->ny, m->nz, m->nx * m->ny, n};
    const double dtau = T / p->nsteps;
    const double c = dtau / (m->dx * m->dx);
    if (c > 1.0 / 6.0 + 1e-15)
        return fail(CG_EINVAL, "cg_diffuse: explicit Euler needs dtau <= dx^2/6 (dtau/dx^2 = %g)", c);
    const size_t vec = align_up((size_t)n * nf * 8);
    CGK_TRY(m->ws_diffuse.ensure(vec));
    double *tmp = m->ws_diffuse.as<double>();
    const Sweep sw = make_sweep(g, nf);
    const dim3 blk(TX, TY);
    double *a = cells, *b = tmp;
    for (int s = 0; s < p->nsteps; ++s) {
        CGK_LAUNCH("explicit64", (double)n * nf * 16, st,
                   k_explicit<<<sw.grid, blk, 0, st>>>(g, sw.zlen, sw.nzc, c, a, b));
        std::swap(a, b);
    }
    CGK_CUDA(cudaGetLastError());
    if (a != cells)
        CGK_CUDA(cudaMemcpyAsync(cells, a, (size_t)n * nf * 8, cudaMemcpyDeviceToDevice, st));
    CGK_CUDA(cudaStreamSynchronize(st));
    if (rep) {
        rep->iters = (long long)p->nsteps * nf;
        rep->cell_updates = rep->iters * (long long)n;
        rep->final_rel_residual = 0.0;
    }
    return CG_OK;
}

template <class TS>
static cg_status diffuse_mixed(cg_mesh *m, int nf, double *cells, const cg_params *p, double T,
                               cg_report *rep, cudaStream_t st) {
    const int n = (int)m->ncells;
    Geo g{m->nx, m->ny, m->nz, m->nx * m->ny, n};
    const bool cn = p->scheme == CG_SCHEME_CRANK_NICOLSON;
    const double dtau = T / p->nsteps;
    const double c = dtau / (m->dx * m->dx);
    const double ce = cn ? 0.5 * c : c;
    const double tol2 = p->tol * p->tol;
    const Sweep sw = make_sweep(g, nf);
    const int G = sw.nb;
    const dim3 blk(TX, TY);
    const Coef64 cf64 = coef64(ce);
    const Coef32 cf32 = coef32(ce);

    // spectrum of A = I - ce L: [1, lmax]
    const int dims[3] = {m->nx, m->ny, m->nz};
    double lmax = 1.0;
    for (int a = 0; a < 3; ++a) {
        double sv = std::sin(M_PI * (dims[a] - 1) / (2.0 * dims[a]));
        lmax += 4.0 * ce * sv * sv;
    }
    const double theta = 0.5 * (lmax + 1.0), delta = 0.5 * (lmax - 1.0);
    const double gamma = 1.0 / theta;
    const double eps_inner = sizeof(TS) == 2 ? 2e-3 : 1e-6;
    int m_it = cheb_iters(lmax, eps_inner);
    if (p->max_iter > 0 && m_it > p->max_iter) m_it = p->max_iter;
    double sigma_d = delta > 0.0 ? theta / delta : 0.0;
    const int coopG = coop_blocks(k_cheb_loop<TS>);
    const Items items = make_items(g, nf, coopG);
    // barrier_budget > 0: the whole inner solve as one cooperative launch with bounded
    // grid barriers between iterations; otherwise one launch per iteration.
    const bool persistent = p->barrier_budget > 0;
    const long long budget = persistent ? p->barrier_budget : 0;

    // buffers: X1, X2, B (FP64); R, Ya, Yb (TS)
    const size_t v64 = align_up((size_t)n * nf * 8), vts = align_up((size_t)n * nf * sizeof(TS));
    CGK_TRY(m->ws_diffuse.ensure(3 * v64 + 3 * vts));
    char *wb = m->ws_diffuse.as<char>();
    double *X1 = (double *)wb, *X2 = (double *)(wb + v64), *B = (double *)(wb + 2 * v64);
    TS *R = (TS *)(wb + 3 * v64), *Ya = (TS *)(wb + 3 * v64 + vts), *Yb = (TS *)(wb + 3 * v64 + 2 * vts);
    CGK_TRY(m->ws_small.ensure(4096 + align_up((size_t)nf * 2 * G * 8) + 64 * sizeof(RefScal) +
                               256));
    double *partials = (double *)(m->ws_small.as<char>() + 4096);
    RefScal *sc = (RefScal *)(m->ws_small.as<char>() + 4096 + align_up((size_t)nf * 2 * G * 8));
    GridBar *gbar = (GridBar *)((char *)sc + 64 * sizeof(RefScal));
    CGK_CUDA(cudaMemsetAsync(sc, 0, nf * sizeof(RefScal), st));
    CGK_CUDA(cudaMemsetAsync(gbar, 0, sizeof(GridBar), st));
    CGK_TRY(m->h_small.ensure(4096 + 64 * sizeof(RefScal) + 256));
    RefScal *hsc = (RefScal *)(m->h_small.as<char>() + 4096);
    GridBar *hgb = (GridBar *)((char *)hsc + 64 * sizeof(RefScal));

    const int max_rounds = p->max_rounds > 0 ? p->max_rounds : 12;
    int sched = 2;   // rounds before the first convergence check of a step
    long long applications = 0, rounds_total = 0;
    double worst = 0.0;
    double *ubuf = cells;                    // u^n (also b for implicit Euler)
    double *F1 = X1, *F2 = X2;               // the two FP64 buffers not holding u^n
    bool converged = true, timed_out = false;
    int s = 0;
    for (; s < p->nsteps; ++s) {
        const double *bptr = cn ? B : ubuf;
        TS *y1buf = Ya;
        CGK_LAUNCH("refine64_first", (double)n * nf * (8 + (cn ? 8 : 0) + 2 * sizeof(TS)), st,
                   (k_refine<TS, true><<<sw.grid, blk, 0, st>>>(
                       g, sw.zlen, sw.nzc, c, cf64, p->scheme, ubuf, nullptr, nullptr, nullptr, B,
                       R, y1buf, (float)gamma, partials, sc)));
        CGK_CUDA(cudaGetLastError());
        applications += 1;
        double *xcur = ubuf;
        int rounds = 0;
        converged = false;
        while (rounds < max_rounds) {
            // inner Chebyshev solve of A d = r, starting from y1 = gamma r: one cooperative
            // launch runs iterations 2..m with grid barriers in between
            TS *ycur = y1buf, *yprev = nullptr, *yother = (y1buf == Ya) ? Yb : Ya;
            if (m_it > 1 && persistent) {
                CGK_CUDA(cudaMemsetAsync(gbar, 0, sizeof(GridBar), st));
                Geo ga = g;
                int a_zlen = items.zlen, a_nzc = items.nzc, a_gx = items.gx, a_gy = items.gy;
                int a_n = items.n, a_m = m_it;
                float a_gamma = (float)gamma;
                Coef32 a_cf = cf32;
                TS *a_y1 = y1buf, *a_oth = yother;
                const TS *a_r = R;
                long long a_budget = budget;
                void *args[] = {&ga,      &a_zlen, &a_nzc, &a_gx,  &a_gy,  &a_n,   &a_cf,   &a_gamma,
                                &sigma_d, &a_m,    &a_y1,  &a_oth, &a_r,   &gbar,  &a_budget};
                CGK_LAUNCH(sizeof(TS) == 2 ? "cheb_loop_bf16" : "cheb_loop_fp32",
                           (double)n * nf * sizeof(TS) * (3.0 + 4.0 * (m_it - 2)), st,
                           CGK_CUDA(cudaLaunchCooperativeKernel((const void *)k_cheb_loop<TS>,
                                                                dim3(coopG), dim3(TX, TY), args, 0,
                                                                st)));
            }
            {
                double om = 1.0;
                for (int k = 1; k < m_it; ++k) {
                    if (sigma_d > 0.0)
                        om = (k == 1) ? 1.0 / (1.0 - 1.0 / (2.0 * sigma_d * sigma_d))
                                      : 1.0 / (1.0 - om / (4.0 * sigma_d * sigma_d));
                    TS *ynext = yprev ? yprev : yother;
                    if (!persistent)
                        CGK_LAUNCH(sizeof(TS) == 2 ? "cheb_bf16" : "cheb_fp32",
                                   (double)n * nf * sizeof(TS) * (yprev ? 4 : 3), st,
                                   k_cheb<TS><<<sw.grid, blk, 0, st>>>(g, sw.zlen, sw.nzc, cf32,
                                                                       (float)gamma, (float)om,
                                                                       ycur, yprev, R, ynext));
                    yprev = ycur;
                    ycur = ynext;
                }
                CGK_CUDA(cudaGetLastError());
            }
            applications += m_it - 1;
            // x += d and the new FP64 residual; y1 goes to the buffer d is not in
            double *xnext = (xcur == F1) ? F2 : F1;
            y1buf = (ycur == Ya) ? Yb : Ya;
            CGK_LAUNCH("refine64", (double)n * nf * (24 + 3 * sizeof(TS)), st,
                       (k_refine<TS, false><<<sw.grid, blk, 0, st>>>(
                           g, sw.zlen, sw.nzc, c, cf64, p->scheme, xcur, ycur, bptr, xnext,
                           nullptr, R, y1buf, (float)gamma, partials, sc)));
            CGK_CUDA(cudaGetLastError());
            applications += 1;
            ++rounds;
            xcur = xnext;
            if (rounds >= sched) {
                CGK_CUDA(cudaMemcpyAsync(hsc, sc, nf * sizeof(RefScal), cudaMemcpyDeviceToHost, st));
                if (persistent)
                    CGK_CUDA(cudaMemcpyAsync(hgb, gbar, sizeof(GridBar), cudaMemcpyDeviceToHost, st));
                CGK_CUDA(cudaStreamSynchronize(st));
                if (persistent && hgb->err) {
                    timed_out = true;
                    break;
                }
                converged = true;
                for (int f = 0; f < nf; ++f) converged = converged && (hsc[f].rr <= tol2 * hsc[f].bb);
                if (converged) break;
            }
        }
        rounds_total += rounds;
        for (int f = 0; f < nf; ++f) {
            double rel = hsc[f].bb > 0 ? std::sqrt(hsc[f].rr / hsc[f].bb) : 0.0;
            if (rel > worst) worst = rel;
        }
        if (timed_out) break;
        sched = rounds > 1 ? rounds : 1;
        // u^{n+1} = xcur; the other two buffers become the spares
        double *old_u = ubuf;
        double *other = (xcur == F1) ? F2 : F1;
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
        rep->inner_iters_per_round = m_it;
    }
    if (timed_out)
        return fail(CG_ETIMEOUT, "cg_diffuse: a grid barrier of the inner solve gave up (step %d)", s);
    if (!converged)
        return fail(CG_ENOCONV, "cg_diffuse: refinement did not reach tol in step %d", s);
    return CG_OK;
}

cg_status diffuse_structured_run(cg_mesh *m, int nf, double *cells, const cg_params *p,
                                 cg_report *rep, cudaStream_t st) {
    double T = p->bandwidth > 0.0 ? p->bandwidth * p->bandwidth / 4.0 : p->T;
    if (p->scheme == CG_SCHEME_EXPLICIT_EULER) return diffuse_explicit(m, nf, cells, p, T, rep, st);
    if (p->precision == CG_PREC_FP64) return diffuse_fp64(m, nf, cells, p, T, rep, st);
    if (p->precision == CG_PREC_FP32_REFINE) return diffuse_mixed<float>(m, nf, cells, p, T, rep, st);
    return diffuse_mixed<__nv_bfloat16>(m, nf, cells, p, T, rep, st);
}

}  // namespace cgk

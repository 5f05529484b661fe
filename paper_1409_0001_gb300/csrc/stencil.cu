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

namespace cgk {

namespace {

constexpr int kThreads = 256;

struct Geo {
    int nx, ny, nz;
    int nxy;
    int n;
};

__device__ __forceinline__ void decompose(const Geo &g, int k, int &ix, int &iy, int &iz) {
    ix = k % g.nx;
    int t = k / g.nx;
    iy = t % g.ny;
    iz = t / g.ny;
}

// sum of the existing face neighbours of k (value given by load(l)) and their number
template <class T, class Load>
__device__ __forceinline__ T nbr_sum(const Geo &g, int k, int ix, int iy, int iz, Load load,
                                     int &nn) {
    T s = T(0);
    nn = 0;
    if (ix > 0) { s += load(k - 1); ++nn; }
    if (ix < g.nx - 1) { s += load(k + 1); ++nn; }
    if (iy > 0) { s += load(k - g.nx); ++nn; }
    if (iy < g.ny - 1) { s += load(k + g.nx); ++nn; }
    if (iz > 0) { s += load(k - g.nxy); ++nn; }
    if (iz < g.nz - 1) { s += load(k + g.nxy); ++nn; }
    return s;
}

// ---------------------------------------------------------------- deterministic sums
// Block sum of one double per thread in a fixed order; valid on thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) t += ws[w];
    __syncthreads();
    return t;
}

// Writes this block's partial(s), and returns true in the last block to arrive.
__device__ __forceinline__ bool arrive(double *partials, int nparts, const double *vals,
                                       unsigned int *ticket) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        for (int q = 0; q < nparts; ++q) partials[q * gridDim.x + blockIdx.x] = vals[q];
        __threadfence();
        unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    return last;
}

// In the last block: the total of partials[q][0..G) in a fixed order (thread 0).
__device__ __forceinline__ double finish_sum(const double *partials, int q) {
    double s = 0.0;
    const double *pq = partials + (size_t)q * gridDim.x;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kThreads) s += __ldcg(pq + i);
    return block_sum(s);
}

struct Scal {
    double rr, bb, alpha, beta;
    int done, iters;
    unsigned int ticket;
    int breakdown;
};

// ================================================================ FP64 conjugate gradients
__global__ void __launch_bounds__(kThreads) k_cg_init(Geo g, double c, int scheme,
                                                      const double *__restrict__ xall,
                                                      double *__restrict__ rall,
                                                      double *__restrict__ pall,
                                                      double *__restrict__ partials_all,
                                                      Scal *__restrict__ sc, double tol2) {
    const int f = blockIdx.y;
    const double *x = xall + (size_t)f * g.n;
    double *r = rall + (size_t)f * g.n;
    double *p = pall + (size_t)f * g.n;
    double rr = 0.0, bb = 0.0;
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < g.n; k += gridDim.x * kThreads) {
        int ix, iy, iz, nn;
        decompose(g, k, ix, iy, iz);
        double xk = x[k];
        double s = nbr_sum<double>(g, k, ix, iy, iz, [&](int l) { return x[l]; }, nn);
        double lx = s - nn * xk;
        double rk = c * lx;                              // b - A x for both schemes
        double bk = scheme == 1 ? xk + 0.5 * c * lx : xk;
        r[k] = rk;
        p[k] = rk;
        rr += rk * rk;
        bb += bk * bk;
    }
    double v[2] = {block_sum(rr), block_sum(bb)};
    double *partials = partials_all + (size_t)f * 2 * gridDim.x;
    if (arrive(partials, 2, v, &sc[f].ticket)) {
        double RR = finish_sum(partials, 0);
        double BB = finish_sum(partials, 1);
        if (threadIdx.x == 0) {
            sc[f].rr = RR;
            sc[f].bb = BB;
            sc[f].beta = 0.0;
            sc[f].iters = 0;
            sc[f].breakdown = 0;
            sc[f].done = (RR <= tol2 * BB) ? 1 : 0;
            sc[f].ticket = 0;
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_cg_pass1(Geo g, double ce,
                                                       const double *__restrict__ rall,
                                                       const double *__restrict__ pin_all,
                                                       double *__restrict__ pout_all,
                                                       double *__restrict__ partials_all,
                                                       Scal *__restrict__ sc) {
    const int f = blockIdx.y;
    if (sc[f].done) return;
    const double beta = sc[f].beta;
    const double *r = rall + (size_t)f * g.n;
    const double *pin = pin_all + (size_t)f * g.n;
    double *pout = pout_all + (size_t)f * g.n;
    double pap = 0.0;
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < g.n; k += gridDim.x * kThreads) {
        int ix, iy, iz, nn;
        decompose(g, k, ix, iy, iz);
        double pk = r[k] + beta * pin[k];
        double s = nbr_sum<double>(g, k, ix, iy, iz, [&](int l) { return r[l] + beta * pin[l]; }, nn);
        double apk = pk + ce * (nn * pk - s);
        pout[k] = pk;
        pap += pk * apk;
    }
    double v = block_sum(pap);
    double *partials = partials_all + (size_t)f * 2 * gridDim.x;
    if (arrive(partials, 1, &v, &sc[f].ticket)) {
        double PAP = finish_sum(partials, 0);
        if (threadIdx.x == 0) {
            if (PAP > 0.0) {
                sc[f].alpha = sc[f].rr / PAP;
            } else {
                sc[f].alpha = 0.0;
                sc[f].breakdown = 1;
                sc[f].done = 1;
            }
            sc[f].ticket = 0;
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_cg_pass2(Geo g, double ce,
                                                       const double *__restrict__ pall,
                                                       double *__restrict__ xall,
                                                       double *__restrict__ rall,
                                                       double *__restrict__ partials_all,
                                                       Scal *__restrict__ sc, double tol2) {
    const int f = blockIdx.y;
    if (sc[f].done) return;
    const double alpha = sc[f].alpha;
    const double *p = pall + (size_t)f * g.n;
    double *x = xall + (size_t)f * g.n;
    double *r = rall + (size_t)f * g.n;
    double rr = 0.0;
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < g.n; k += gridDim.x * kThreads) {
        int ix, iy, iz, nn;
        decompose(g, k, ix, iy, iz);
        double pk = p[k];
        double s = nbr_sum<double>(g, k, ix, iy, iz, [&](int l) { return p[l]; }, nn);
        double apk = pk + ce * (nn * pk - s);
        x[k] = x[k] + alpha * pk;
        double rk = r[k] - alpha * apk;
        r[k] = rk;
        rr += rk * rk;
    }
    double v = block_sum(rr);
    double *partials = partials_all + (size_t)f * 2 * gridDim.x;
    if (arrive(partials, 1, &v, &sc[f].ticket)) {
        double RR = finish_sum(partials, 0);
        if (threadIdx.x == 0) {
            sc[f].beta = RR / sc[f].rr;
            sc[f].rr = RR;
            sc[f].iters += 1;
            sc[f].done = (RR <= tol2 * sc[f].bb) ? 1 : 0;
            sc[f].ticket = 0;
        }
    }
}

// explicit Euler: x_out = x + c L x (FP64)
__global__ void __launch_bounds__(kThreads) k_explicit(Geo g, double c,
                                                       const double *__restrict__ xin_all,
                                                       double *__restrict__ xout_all) {
    const int f = blockIdx.y;
    const double *x = xin_all + (size_t)f * g.n;
    double *y = xout_all + (size_t)f * g.n;
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < g.n; k += gridDim.x * kThreads) {
        int ix, iy, iz, nn;
        decompose(g, k, ix, iy, iz);
        double xk = x[k];
        double s = nbr_sum<double>(g, k, ix, iy, iz, [&](int l) { return x[l]; }, nn);
        y[k] = xk + c * (s - nn * xk);
    }
}

// ================================================================ mixed precision
template <class TS> __device__ __forceinline__ float ld(const TS *p, int i);
template <> __device__ __forceinline__ float ld<float>(const float *p, int i) { return p[i]; }
template <> __device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16 *p, int i) {
    return __bfloat162float(p[i]);
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

// One FP64 refinement pass.  first: x = x_in (no correction), b = x_in (implicit Euler)
// or b = x_in + c/2 L x_in written to b_out (Crank-Nicolson), r = c L x_in.
// Otherwise: x = x_in + d at the cell and its neighbours, x_out = x, r = b - A x.
// Stores r and y1 = gamma r (the first Chebyshev iterate) in the storage type.
template <class TS, bool kFirst>
__global__ void __launch_bounds__(kThreads) k_refine(Geo g, double c, double ce, int scheme,
                                                     const double *__restrict__ xin_all,
                                                     const TS *__restrict__ d_all,
                                                     const double *__restrict__ b_all,
                                                     double *__restrict__ xout_all,
                                                     double *__restrict__ bout_all,
                                                     TS *__restrict__ r_all, TS *__restrict__ y1_all,
                                                     float gamma, double *__restrict__ partials_all,
                                                     RefScal *__restrict__ sc) {
    const int f = blockIdx.y;
    const size_t off = (size_t)f * g.n;
    const double *xin = xin_all + off;
    TS *r = r_all + off;
    TS *y1 = y1_all + off;
    double rr = 0.0, bb = 0.0;
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < g.n; k += gridDim.x * kThreads) {
        int ix, iy, iz, nn;
        decompose(g, k, ix, iy, iz);
        double rk;
        if (kFirst) {
            double xk = xin[k];
            double s = nbr_sum<double>(g, k, ix, iy, iz, [&](int l) { return xin[l]; }, nn);
            double lx = s - nn * xk;
            rk = c * lx;
            double bk = xk;
            if (scheme == 1) {
                bk = xk + 0.5 * c * lx;
                bout_all[off + k] = bk;
            }
            bb += bk * bk;
        } else {
            const TS *d = d_all + off;
            double xk = xin[k] + (double)ld(d, k);
            double s = nbr_sum<double>(
                g, k, ix, iy, iz, [&](int l) { return xin[l] + (double)ld(d, l); }, nn);
            double ax = xk + ce * (nn * xk - s);
            rk = b_all[off + k] - ax;
            xout_all[off + k] = xk;
        }
        float rf = (float)rk;
        st(r, k, rf);
        st(y1, k, gamma * rf);
        rr += rk * rk;
    }
    double v[2] = {block_sum(rr), kFirst ? block_sum(bb) : 0.0};
    double *partials = partials_all + (size_t)f * 2 * gridDim.x;
    if (arrive(partials, kFirst ? 2 : 1, v, &sc[f].ticket)) {
        double RR = finish_sum(partials, 0);
        double BB = kFirst ? finish_sum(partials, 1) : 0.0;
        if (threadIdx.x == 0) {
            sc[f].rr = RR;
            if (kFirst) sc[f].bb = BB;
            sc[f].ticket = 0;
        }
    }
}

// One Chebyshev iteration for A y = r (FP32 arithmetic, TS storage):
// y_next = omega (y - y_prev + gamma (r - A y)) + y_prev; y_prev == nullptr means 0.
// y_next may alias y_prev (pointwise access only).
template <class TS>
__global__ void __launch_bounds__(kThreads) k_cheb(Geo g, float ce, float gamma, float omega,
                                                   const TS *__restrict__ y_all,
                                                   const TS *yprev_all,
                                                   const TS *__restrict__ r_all, TS *ynext_all) {
    const int f = blockIdx.y;
    const size_t off = (size_t)f * g.n;
    const TS *y = y_all + off;
    const TS *r = r_all + off;
    const TS *yp = yprev_all ? yprev_all + off : nullptr;
    TS *yn = ynext_all + off;
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < g.n; k += gridDim.x * kThreads) {
        int ix, iy, iz, nn;
        decompose(g, k, ix, iy, iz);
        float yk = ld(y, k);
        float s = nbr_sum<float>(g, k, ix, iy, iz, [&](int l) { return ld(y, l); }, nn);
        float ay = yk + ce * (nn * yk - s);
        float ypk = yp ? ld(yp, k) : 0.0f;
        float v = omega * (yk - ypk + gamma * (ld(r, k) - ay)) + ypk;
        st(yn, k, v);
    }
}

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
    if (arrive(partials, 1, &v, &tickets[f])) {
        double S = finish_sum(partials, 0);
        if (threadIdx.x == 0) {
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
    const int G = stencil_grid(n);
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
    const dim3 grid(G, nf);
    long long total_iters = 0;
    double worst = 0.0;
    const int chunk = 8;
    for (int s = 0; s < p->nsteps; ++s) {
        CGK_LAUNCH("cg64_init", (double)n * nf * 24, st,
                   k_cg_init<<<grid, kThreads, 0, st>>>(g, c, p->scheme, cells, r, P[0], partials,
                                                        sc, tol2));
        CGK_CUDA(cudaGetLastError());
        int it = 0;
        bool all_done = false;
        while (true) {
            for (int q = 0; q < chunk; ++q, ++it) {
                CGK_LAUNCH("cg64_pass1", (double)n * nf * 24, st,
                           k_cg_pass1<<<grid, kThreads, 0, st>>>(g, ce, r, P[it & 1],
                                                                 P[(it + 1) & 1], partials, sc));
                CGK_LAUNCH("cg64_pass2", (double)n * nf * 40, st,
                           k_cg_pass2<<<grid, kThreads, 0, st>>>(g, ce, P[(it + 1) & 1], cells, r,
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
    const dim3 grid(stencil_grid(n), nf);
    double *a = cells, *b = tmp;
    for (int s = 0; s < p->nsteps; ++s) {
        CGK_LAUNCH("explicit64", (double)n * nf * 16, st,
                   k_explicit<<<grid, kThreads, 0, st>>>(g, c, a, b));
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
    const int G = stencil_grid(n);
    const dim3 grid(G, nf);

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
    std::vector<float> omega((size_t)m_it + 1, 1.0f);
    if (delta > 0.0) {
        double sigma = theta / delta, om = 1.0;
        for (int k = 1; k < m_it; ++k) {
            om = (k == 1) ? 1.0 / (1.0 - 1.0 / (2.0 * sigma * sigma)) : 1.0 / (1.0 - om / (4.0 * sigma * sigma));
            omega[k] = (float)om;
        }
    }

    // buffers: X1, X2, B (FP64); R, Ya, Yb (TS)
    const size_t v64 = align_up((size_t)n * nf * 8), vts = align_up((size_t)n * nf * sizeof(TS));
    CGK_TRY(m->ws_diffuse.ensure(3 * v64 + 3 * vts));
    char *wb = m->ws_diffuse.as<char>();
    double *X1 = (double *)wb, *X2 = (double *)(wb + v64), *B = (double *)(wb + 2 * v64);
    TS *R = (TS *)(wb + 3 * v64), *Ya = (TS *)(wb + 3 * v64 + vts), *Yb = (TS *)(wb + 3 * v64 + 2 * vts);
    CGK_TRY(m->ws_small.ensure(4096 + align_up((size_t)nf * 2 * G * 8) + 64 * sizeof(RefScal)));
    double *partials = (double *)(m->ws_small.as<char>() + 4096);
    RefScal *sc = (RefScal *)(m->ws_small.as<char>() + 4096 + align_up((size_t)nf * 2 * G * 8));
    CGK_CUDA(cudaMemsetAsync(sc, 0, nf * sizeof(RefScal), st));
    CGK_TRY(m->h_small.ensure(4096 + 64 * sizeof(RefScal)));
    RefScal *hsc = (RefScal *)(m->h_small.as<char>() + 4096);

    const int max_rounds = p->max_rounds > 0 ? p->max_rounds : 12;
    int sched = 2;   // rounds before the first convergence check of a step
    long long applications = 0, rounds_total = 0;
    double worst = 0.0;
    double *ubuf = cells;                    // u^n (also b for implicit Euler)
    double *F1 = X1, *F2 = X2;               // the two FP64 buffers not holding u^n
    bool converged = true;
    int s = 0;
    for (; s < p->nsteps; ++s) {
        const double *bptr = cn ? B : ubuf;
        TS *y1buf = Ya;
        CGK_LAUNCH("refine64_first", (double)n * nf * (8 + (cn ? 8 : 0) + 2 * sizeof(TS)), st,
                   (k_refine<TS, true><<<grid, kThreads, 0, st>>>(
                       g, c, ce, p->scheme, ubuf, nullptr, nullptr, nullptr, B, R, y1buf,
                       (float)gamma, partials, sc)));
        CGK_CUDA(cudaGetLastError());
        applications += 1;
        double *xcur = ubuf;
        int rounds = 0;
        converged = false;
        while (rounds < max_rounds) {
            // inner Chebyshev solve of A d = r, starting from y1 = gamma r
            TS *ycur = y1buf, *yprev = nullptr, *yother = (y1buf == Ya) ? Yb : Ya;
            for (int k = 1; k < m_it; ++k) {
                TS *ynext = yprev ? yprev : yother;
                CGK_LAUNCH(sizeof(TS) == 2 ? "cheb_bf16" : "cheb_fp32",
                           (double)n * nf * sizeof(TS) * (yprev ? 4 : 3), st,
                           k_cheb<TS><<<grid, kThreads, 0, st>>>(g, (float)ce, (float)gamma,
                                                                 omega[k], ycur, yprev, R, ynext));
                yprev = ycur;
                ycur = ynext;
            }
            applications += m_it - 1;
            // x += d and the new FP64 residual; y1 goes to the buffer d is not in
            double *xnext = (xcur == F1) ? F2 : F1;
            y1buf = (ycur == Ya) ? Yb : Ya;
            CGK_LAUNCH("refine64", (double)n * nf * (24 + 3 * sizeof(TS)), st,
                       (k_refine<TS, false><<<grid, kThreads, 0, st>>>(
                           g, c, ce, p->scheme, xcur, ycur, bptr, xnext, nullptr, R, y1buf,
                           (float)gamma, partials, sc)));
            CGK_CUDA(cudaGetLastError());
            applications += 1;
            ++rounds;
            xcur = xnext;
            if (rounds >= sched) {
                CGK_CUDA(cudaMemcpyAsync(hsc, sc, nf * sizeof(RefScal), cudaMemcpyDeviceToHost, st));
                CGK_CUDA(cudaStreamSynchronize(st));
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

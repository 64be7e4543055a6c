// Unfused step: three plain global-memory kernels, one thread per node.  The lattice Boltzmann
// kernel is also the second kernel of the two-kernel step (step_split.cu).
//   1. ac_flux:   W = ubar^n phi^n + kappa_AC phi^n (1 - phi^n) n^n          (3N scratch)
//   2. ac_update: phi^{n+1} = phi^n - div W + D lap(phi^n)
//   3. lbm:       pull streaming, forces from phi^{n+1}, regularised collision
// Kept as the simple cross-check of the fused kernel; boundary handling (periodic x, y; z walls
// with halfway bounce-back and mirrored fields) is identical.
#include "lbm_node.cuh"
#include "tslb_internal.h"

namespace tslb {
namespace {

// One thread per node: x from the thread index, y and z from the block index.
__device__ __forceinline__ bool node_coords(const Grid &G, int &x, int &y, int &z)
{
    x = blockIdx.x * blockDim.x + threadIdx.x;
    y = blockIdx.y;
    z = blockIdx.z;
    return x < G.nx;
}

// advect = 1 leaves the advective flux u phi out of W (the update adds u . grad(phi) instead)
__global__ void __launch_bounds__(128) ac_flux_kernel(Grid G, Phys P, const float *__restrict__ phi,
                                                      const float *__restrict__ u, float *__restrict__ W, int advect)
{
    int x, y, z;
    if (!node_coords(G, x, y, z)) return;
    const Nbr n = make_nbr(x, y, z, G);
    float ps[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) ps[i] = __ldg(phi + nidx(n, i));
    float gx, gy, gz, lap;
    grad_lap27(ps, gx, gy, gz, lap);
    const float inv = rsqrtf(fmaxf(gx * gx + gy * gy + gz * gz, kNormalEps * kNormalEps));
    const int k = n.zo[1] + n.yo[1] + x;
    const float p = ps[13];
    const float s = P.kac * fmaxf(p * (1.0f - p), 0.0f) * inv;
    if (advect) {
        W[k] = s * gx;
        W[G.N + k] = s * gy;
        W[2 * G.N + k] = s * gz;
    } else {
        W[k] = fmaf(u[k], p, s * gx);
        W[G.N + k] = fmaf(u[G.N + k], p, s * gy);
        W[2 * G.N + k] = fmaf(u[2 * G.N + k], p, s * gz);
    }
}

// phi^{n+1} = phi - div W + D lap(phi), and with advect = 1 also - ubar . grad(phi) (the literal
// advection term; W then holds the sharpening flux alone)
__global__ void __launch_bounds__(128) ac_update_kernel(Grid G, Phys P, const float *__restrict__ phi,
                                                        const float *__restrict__ W, const float *__restrict__ u,
                                                        int advect, float *__restrict__ phi_out)
{
    int x, y, z;
    if (!node_coords(G, x, y, z)) return;
    const Nbr n = make_nbr(x, y, z, G);
    float ps[27];
    float div = 0.0f;
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const int j = nidx(n, i);
        ps[i] = __ldg(phi + j);
        const float w3 = 3.0f * wgt(i);
        if (cx(i)) div = fmaf(cx(i) * w3, __ldg(W + j), div);
        if (cy(i)) div = fmaf(cy(i) * w3, __ldg(W + G.N + j), div);
        if (cz(i)) div = fmaf(cz(i) * w3 * n.zsgn[cz(i) + 1], __ldg(W + 2 * G.N + j), div);
    }
    float gx, gy, gz, lap;
    grad_lap27(ps, gx, gy, gz, lap);
    const int k = n.zo[1] + n.yo[1] + x;
    float p0 = ps[13];
    if (advect) p0 -= fmaf(u[k], gx, fmaf(u[G.N + k], gy, u[2 * G.N + k] * gz));
    phi_out[k] = p0 - div + P.mob * lap;
}

// Lattice Boltzmann update, one thread per node (x from the thread, y and z from the block); the
// node update itself is lbm_node (lbm_node.cuh).
template <class S>
__global__ void __launch_bounds__(128) lbm_kernel(Grid G, Phys P, const typename S::T *__restrict__ gin,
                                                  const float *__restrict__ pin, const float *__restrict__ phi_new,
                                                  const float *__restrict__ ubar, typename S::T *__restrict__ gout,
                                                  float *__restrict__ pout, float *__restrict__ uout,
                                                  float *__restrict__ wout)
{
    pdl_trigger();
    pdl_wait();
    int x, y, z;
    if (!node_coords(G, x, y, z)) return;
    lbm_node<S>(G, P, gin, pin, phi_new, ubar, gout, pout, uout, wout, x, y, z);
}

// W = W(phi, ubar) at every node, with the same gradient and flux arithmetic as the lattice
// Boltzmann kernels (so a restored state continues exactly as an uninterrupted one)
__global__ void __launch_bounds__(128) flux_kernel(Grid G, Phys P, const float *__restrict__ phi,
                                                   const float *__restrict__ u, float *__restrict__ w)
{
    int x, y, z;
    if (!node_coords(G, x, y, z)) return;
    const Nbr n = make_nbr(x, y, z, G);
    const int k = n.zo[1] + n.yo[1] + x;
    const size_t N = (size_t)G.N;
    float ps[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) ps[i] = __ldg(phi + nidx(n, i));
    float gx, gy, gz, lap;
    grad_lap27(ps, gx, gy, gz, lap);
    float wx, wy, wz;
    ac_flux(ps[13], gx, gy, gz, u[k], u[N + k], u[2 * N + k], P, wx, wy, wz);
    w[k] = wx;
    w[N + k] = wy;
    w[2 * N + k] = wz;
}

// 16-bit formats from equilibrium: h = 0 and P = p*0.
template <class S>
__global__ void __launch_bounds__(128) init16_kernel(Grid G, const float *__restrict__ pstar,
                                                     typename S::T *__restrict__ h, float *__restrict__ pst)
{
    int x, y, z;
    if (!node_coords(G, x, y, z)) return;
    const size_t N = (size_t)G.N;
    const int k = (z * G.ny + y) * G.nx + x;
#pragma unroll
    for (int i = 0; i < 27; ++i) h[i * N + k] = S::from_f(0.0f);
    pst[k] = pstar ? pstar[k] : 0.0f;
}

// g_i = w_i (P + f^eq_i(0, u) / w_i + h_i) for directions [i0, i0 + ni) into g[(i - i0) * N + node]
template <class S>
__global__ void __launch_bounds__(128) expand16_kernel(Grid G, const typename S::T *__restrict__ h,
                                                       const float *__restrict__ pst, const float *__restrict__ u,
                                                       int i0, int ni, float *__restrict__ g)
{
    int x, y, z;
    if (!node_coords(G, x, y, z)) return;
    const size_t N = (size_t)G.N;
    const int k = (z * G.ny + y) * G.nx + x;
    const float p = pst[k], ux = u[k], uy = u[N + k], uz = u[2 * N + k];
    const float u2 = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < 27; ++i)
        if (i >= i0 && i < i0 + ni)
            g[(size_t)(i - i0) * N + k] = wgt(i) * (p + eq_shifted(cdot(i, ux, uy, uz), u2) + S::to_f(h[i * N + k]));
}

// From FP32 g (directions [i0, i0 + ni) at g[(i - i0) * N + node]) and the node's u: mode 0
// accumulates p* = sum g into pst (zeroed by the caller); mode 1 writes
// h_i = g_i / w_i - p* - f^eq_i(0, u) / w_i and accumulates sum w_i h_i(rounded) into corr.
template <class S>
__global__ void __launch_bounds__(128) compress16_kernel(Grid G, const float *__restrict__ g,
                                                         const float *__restrict__ u, int i0, int ni, int mode,
                                                         typename S::T *__restrict__ h, float *__restrict__ pst,
                                                         float *__restrict__ corr)
{
    int x, y, z;
    if (!node_coords(G, x, y, z)) return;
    const size_t N = (size_t)G.N;
    const int k = (z * G.ny + y) * G.nx + x;
    if (mode == 0) {
        float s = pst[k];
#pragma unroll
        for (int i = 0; i < 27; ++i)
            if (i >= i0 && i < i0 + ni) s += g[(size_t)(i - i0) * N + k];
        pst[k] = s;
        return;
    }
    const float p = pst[k], ux = u[k], uy = u[N + k], uz = u[2 * N + k];
    const float u2 = ux * ux + uy * uy + uz * uz;
    float c = corr[k];
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        if (i >= i0 && i < i0 + ni) {
            const float gi = g[(size_t)(i - i0) * N + k];
            const typename S::T v = S::from_f(gi / wgt(i) - p - eq_shifted(cdot(i, ux, uy, uz), u2));
            h[i * N + k] = v;
            c = fmaf(wgt(i), S::to_f(v), c);
        }
    }
    corr[k] = c;
}

__global__ void __launch_bounds__(128) finish16_kernel(Grid G, const float *__restrict__ corr, float *__restrict__ pst)
{
    int x, y, z;
    if (!node_coords(G, x, y, z)) return;
    const int k = (z * G.ny + y) * G.nx + x;
    pst[k] -= corr[k];
}

__global__ void __launch_bounds__(128) init_kernel(Grid G, const float *__restrict__ pstar, const float *__restrict__ u,
                                                   float *__restrict__ g)
{
    int x, y, z;
    if (!node_coords(G, x, y, z)) return;
    const size_t N = (size_t)G.N;
    const int k = (z * G.ny + y) * G.nx + x;
    float e[27];
    equilibrium(pstar ? pstar[k] : 0.0f, u[k], u[N + k], u[2 * N + k], e);
#pragma unroll
    for (int i = 0; i < 27; ++i) g[i * N + k] = e[i];
}

// p = p* rho cs^2 with p* = sum_i g_i (FP32 populations; pst null), or P + sum_i w_i h_i
// (16-bit formats: g holds h, storage 1 / 2)
__global__ void __launch_bounds__(128) pressure_kernel(Grid G, Phys P, const float *__restrict__ g, int storage,
                                                       const float *__restrict__ pst, const float *__restrict__ phi,
                                                       float *__restrict__ p)
{
    int x, y, z;
    if (!node_coords(G, x, y, z)) return;
    const size_t N = (size_t)G.N;
    const int k = (z * G.ny + y) * G.nx + x;
    float s = 0.0f;
    if (storage >= LBM_MOM) {   // moment storages: p* is the first moment array
        s = g[k];
    } else if (pst) {   // 16-bit formats: p* = P + sum_i w_i h_i
        s = pst[k];
#pragma unroll
        for (int i = 0; i < 27; ++i) s = fmaf(wgt(i), load_h16(g, storage, i * N + k), s);
    } else {
#pragma unroll
        for (int i = 0; i < 27; ++i) s += g[i * N + k];
    }
    p[k] = s * fmaf(phi[k], P.drho, P.rho_g) * (1.0f / 3.0f);
}

dim3 node_grid(const Grid &G) { return dim3((G.nx + 127) / 128, G.ny, G.nz); }

}  // namespace

cudaError_t launch_step_unfused(const Grid &G, const Phys &P, const StepArgs &a, cudaStream_t s)
{
    const dim3 grid = node_grid(G);
    ac_flux_kernel<<<grid, 128, 0, s>>>(G, P, a.phi_in, a.u_in, a.flux, a.advect);
    ac_update_kernel<<<grid, 128, 0, s>>>(G, P, a.phi_in, a.flux, a.u_in, a.advect, a.phi_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the scratch flux is consumed: the lattice Boltzmann kernel leaves W^{n+1} in it
    return launch_lbm(G, P, a.storage, a.g_in, a.p_in, a.phi_out, a.u_in, a.g_out, a.p_out, a.u_out, a.flux, s);
}

cudaError_t launch_lbm(const Grid &G, const Phys &P, int storage, const void *g_in, const float *p_in,
                       const float *phi_new, const float *u_in, void *g_out, float *p_out, float *u_out,
                       float *w_out, cudaStream_t s)
{
    const dim3 grid = node_grid(G);
    switch (storage) {
    case 0:
        return launch_pdl(lbm_kernel<StoreF32>, grid, dim3(128), 0, s, G, P, (const float *)g_in, (const float *)nullptr,
                          phi_new, u_in, (float *)g_out, (float *)nullptr, u_out, w_out);
    case 1:
        return launch_pdl(lbm_kernel<StoreB16>, grid, dim3(128), 0, s, G, P, (const __nv_bfloat16 *)g_in, p_in, phi_new,
                          u_in, (__nv_bfloat16 *)g_out, p_out, u_out, w_out);
    case 2:
        return launch_pdl(lbm_kernel<StoreF16>, grid, dim3(128), 0, s, G, P, (const __half *)g_in, p_in, phi_new, u_in,
                          (__half *)g_out, p_out, u_out, w_out);
    case LBM_MOM:
    case LBM_MOM_BF16:
    case LBM_MOM_FP16:
        return launch_mom_plain(G, P, storage, (const float *)g_in, u_in, phi_new, (float *)g_out, u_out, w_out, s);
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_flux(const Grid &G, const Phys &P, const float *phi, const float *u, float *w, cudaStream_t s)
{
    flux_kernel<<<node_grid(G), 128, 0, s>>>(G, P, phi, u, w);
    return cudaGetLastError();
}

cudaError_t launch_init16(const Grid &G, int storage, const float *pstar, void *h, float *pst, cudaStream_t s)
{
    if (storage == 1)
        init16_kernel<StoreB16><<<node_grid(G), 128, 0, s>>>(G, pstar, (__nv_bfloat16 *)h, pst);
    else
        init16_kernel<StoreF16><<<node_grid(G), 128, 0, s>>>(G, pstar, (__half *)h, pst);
    return cudaGetLastError();
}

cudaError_t launch_expand16(const Grid &G, int storage, const void *h, const float *pst, const float *u, int i0,
                            int ni, float *g, cudaStream_t s)
{
    if (storage == 1)
        expand16_kernel<StoreB16><<<node_grid(G), 128, 0, s>>>(G, (const __nv_bfloat16 *)h, pst, u, i0, ni, g);
    else
        expand16_kernel<StoreF16><<<node_grid(G), 128, 0, s>>>(G, (const __half *)h, pst, u, i0, ni, g);
    return cudaGetLastError();
}

cudaError_t launch_compress16(const Grid &G, int storage, const float *g, const float *u, int i0, int ni, int mode,
                              void *h, float *pst, float *corr, cudaStream_t s)
{
    if (storage == 1)
        compress16_kernel<StoreB16><<<node_grid(G), 128, 0, s>>>(G, g, u, i0, ni, mode, (__nv_bfloat16 *)h, pst,
                                                                 corr);
    else
        compress16_kernel<StoreF16><<<node_grid(G), 128, 0, s>>>(G, g, u, i0, ni, mode, (__half *)h, pst, corr);
    return cudaGetLastError();
}

cudaError_t launch_finish16(const Grid &G, const float *corr, float *pst, cudaStream_t s)
{
    finish16_kernel<<<node_grid(G), 128, 0, s>>>(G, corr, pst);
    return cudaGetLastError();
}

cudaError_t launch_init(const Grid &G, const float *pstar, const float *u, float *g, cudaStream_t s)
{
    init_kernel<<<node_grid(G), 128, 0, s>>>(G, pstar, u, g);
    return cudaGetLastError();
}

cudaError_t launch_pressure(const Grid &G, const Phys &P, int storage, const void *g, const float *pst,
                            const float *phi, float *p, cudaStream_t s)
{
    pressure_kernel<<<node_grid(G), 128, 0, s>>>(G, P, (const float *)g, storage, pst, phi, p);
    return cudaGetLastError();
}

}  // namespace tslb

// Unfused step: three plain global-memory kernels, one thread per node.  The lattice Boltzmann
// kernel is also the second kernel of the two-kernel step (step_split.cu).
//   1. ac_flux:   W = ubar^n phi^n + kappa_AC phi^n (1 - phi^n) n^n          (3N scratch)
//   2. ac_update: phi^{n+1} = phi^n - div W + D lap(phi^n)
//   3. lbm:       pull streaming, forces from phi^{n+1}, regularised collision
// Kept as the simple cross-check of the fused kernel; boundary handling (periodic x, y; z walls
// with halfway bounce-back and mirrored fields) is identical.
#include "tslb_internal.h"

namespace tslb {
namespace {

// Neighbour coordinates of one node at distance 1: offsets into a scalar array for c = -1, 0, +1
// along each axis, with x, y periodic and z periodic or mirrored at the walls.
struct Nbr {
    int xo[3], yo[3], zo[3];
    float zsgn[3];   // -1 where the z neighbour is a mirror image (odd z component of vectors)
};

__device__ __forceinline__ Nbr make_nbr(int x, int y, int z, const Grid &G)
{
    Nbr n;
    n.xo[0] = x == 0 ? G.nx - 1 : x - 1;
    n.xo[1] = x;
    n.xo[2] = x == G.nx - 1 ? 0 : x + 1;
    n.yo[0] = (y == 0 ? G.ny - 1 : y - 1) * G.nx;
    n.yo[1] = y * G.nx;
    n.yo[2] = (y == G.ny - 1 ? 0 : y + 1) * G.nx;
    n.zsgn[0] = n.zsgn[1] = n.zsgn[2] = 1.0f;
    int zm, zp;
    if (G.wall) {
        zm = z == 0 ? 0 : z - 1;
        zp = z == G.nz - 1 ? G.nz - 1 : z + 1;
        if (z == 0) n.zsgn[0] = -1.0f;
        if (z == G.nz - 1) n.zsgn[2] = -1.0f;
    } else {
        zm = z == 0 ? G.nz - 1 : z - 1;
        zp = z == G.nz - 1 ? 0 : z + 1;
    }
    n.zo[0] = zm * G.nxy;
    n.zo[1] = z * G.nxy;
    n.zo[2] = zp * G.nxy;
    return n;
}

__device__ __forceinline__ int nidx(const Nbr &n, int i)
{
    return n.zo[cz(i) + 1] + n.yo[cy(i) + 1] + n.xo[cx(i) + 1];
}

__device__ __forceinline__ bool node_coords(const Grid &G, int &x, int &y, int &z)
{
    x = blockIdx.x * blockDim.x + threadIdx.x;
    y = blockIdx.y;
    z = blockIdx.z;
    return x < G.nx;
}

__global__ void __launch_bounds__(128) ac_flux_kernel(Grid G, Phys P, const float *__restrict__ phi,
                                                      const float *__restrict__ u, float *__restrict__ W)
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
    W[k] = fmaf(u[k], p, s * gx);
    W[G.N + k] = fmaf(u[G.N + k], p, s * gy);
    W[2 * G.N + k] = fmaf(u[2 * G.N + k], p, s * gz);
}

__global__ void __launch_bounds__(128) ac_update_kernel(Grid G, Phys P, const float *__restrict__ phi,
                                                        const float *__restrict__ W, float *__restrict__ phi_out)
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
    phi_out[n.zo[1] + n.yo[1] + x] = ps[13] - div + P.mob * lap;
}

__global__ void __launch_bounds__(128) lbm_kernel(Grid G, Phys P, const float *__restrict__ gin,
                                                  const float *__restrict__ phi_new, const float *__restrict__ ubar,
                                                  float *__restrict__ gout, float *__restrict__ uout)
{
    int x, y, z;
    if (!node_coords(G, x, y, z)) return;
    const Nbr n = make_nbr(x, y, z, G);
    const int k = n.zo[1] + n.yo[1] + x;
    const size_t N = (size_t)G.N;
    const bool wlo = G.wall && z == 0;
    const bool whi = G.wall && z == G.nz - 1;

    // pull f_i(x) = g_i(x - c_i); at a wall the population returns reversed: g_{26-i}(x)
    float f[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const int j = n.zo[1 - cz(i)] + n.yo[1 - cy(i)] + n.xo[1 - cx(i)];
        bool bounce = false;
        if (cz(i) == 1) bounce = wlo;
        if (cz(i) == -1) bounce = whi;
        f[i] = bounce ? __ldg(gin + (26 - i) * N + k) : __ldg(gin + i * N + j);
    }

    float ps[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) ps[i] = __ldg(phi_new + nidx(n, i));
    float gx, gy, gz, lap;
    grad_lap27(ps, gx, gy, gz, lap);

    float g[27], ux, uy, uz;
    collide_node(f, ps[13], gx, gy, gz, lap, ubar[k], ubar[N + k], ubar[2 * N + k], P, g, ux, uy, uz);
#pragma unroll
    for (int i = 0; i < 27; ++i) gout[i * N + k] = g[i];
    uout[k] = ux;
    uout[N + k] = uy;
    uout[2 * N + k] = uz;
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

__global__ void __launch_bounds__(128) pressure_kernel(Grid G, Phys P, const float *__restrict__ g,
                                                       const float *__restrict__ phi, float *__restrict__ p)
{
    int x, y, z;
    if (!node_coords(G, x, y, z)) return;
    const size_t N = (size_t)G.N;
    const int k = (z * G.ny + y) * G.nx + x;
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 27; ++i) s += g[i * N + k];
    p[k] = s * fmaf(phi[k], P.drho, P.rho_g) * (1.0f / 3.0f);
}

dim3 node_grid(const Grid &G) { return dim3((G.nx + 127) / 128, G.ny, G.nz); }

}  // namespace

cudaError_t launch_step_unfused(const Grid &G, const Phys &P, const StepArgs &a, cudaStream_t s)
{
    const dim3 grid = node_grid(G);
    ac_flux_kernel<<<grid, 128, 0, s>>>(G, P, a.phi_in, a.u_in, a.flux);
    ac_update_kernel<<<grid, 128, 0, s>>>(G, P, a.phi_in, a.flux, a.phi_out);
    lbm_kernel<<<grid, 128, 0, s>>>(G, P, a.g_in, a.phi_out, a.u_in, a.g_out, a.u_out);
    return cudaGetLastError();
}

cudaError_t launch_lbm(const Grid &G, const Phys &P, const float *g_in, const float *phi_new, const float *u_in,
                       float *g_out, float *u_out, cudaStream_t s)
{
    lbm_kernel<<<node_grid(G), 128, 0, s>>>(G, P, g_in, phi_new, u_in, g_out, u_out);
    return cudaGetLastError();
}

cudaError_t launch_init(const Grid &G, const float *pstar, const float *u, float *g, cudaStream_t s)
{
    init_kernel<<<node_grid(G), 128, 0, s>>>(G, pstar, u, g);
    return cudaGetLastError();
}

cudaError_t launch_pressure(const Grid &G, const Phys &P, const float *g, const float *phi, float *p, cudaStream_t s)
{
    pressure_kernel<<<node_grid(G), 128, 0, s>>>(G, P, g, phi, p);
    return cudaGetLastError();
}

}  // namespace tslb

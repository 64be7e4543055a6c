// Fused step: one kernel per time step.
//
// A CTA of TX*TY threads owns a TX x TY column tile of the (x, y) plane and marches through a
// chunk of z planes.  Each thread owns one column (x, y).  A rolling shared-memory window keeps
//   sPhi  phi^n      4 planes, halo 3   (TX+6) x (TY+6)
//   sU    ubar^n     1 plane,  halo 2   (TX+4) x (TY+4) x 3
//   sW    flux W     3 planes, halo 2   W = ubar phi + kappa_AC phi (1-phi) n   (x3 components)
//   sPn   phi^{n+1}  3 planes, halo 1   (TX+2) x (TY+2)
// Iteration s of the march (plane index p = z0 - 3 + s):
//   0. issue the 27 pulled population loads of plane p - 3 (consumed in stage 4)
//   1. load phi^n plane p (halo 3) and ubar^n plane p - 1 (halo 2) into shared memory
//   2. W on plane p - 1 (halo 2)
//   3. phi^{n+1} = phi^n - div W + D lap(phi^n) on plane p - 2 (halo 1)
//   4. lattice Boltzmann update of plane p - 3: gradient and Laplacian of phi^{n+1}, pull
//      streaming, forces, regularised collision; write g, ubar, phi^{n+1} of the own node.
// Only the halo of the Allen–Cahn fields is recomputed; every node's populations are read once
// and written once.  Periodic axes wrap; with z walls the fields are mirrored about the wall
// (vector z components negated) and the populations bounce back (halfway).
#include "tslb_internal.h"

namespace tslb {
namespace {

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int NT = TX * TY;
constexpr int R3X = TX + 6, R3Y = TY + 6, N3 = R3X * R3Y;
constexpr int R2X = TX + 4, R2Y = TY + 4, N2 = R2X * R2Y;
constexpr int R1X = TX + 2, R1Y = TY + 2, N1 = R1X * R1Y;
constexpr int K3 = (N3 + NT - 1) / NT;
constexpr int K2 = (N2 + NT - 1) / NT;
constexpr int K1 = (N1 + NT - 1) / NT;

__device__ __forceinline__ int wrapc(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// stored plane of an extended z index (periodic wrap, or mirror about the walls)
template <bool WALL>
__device__ __forceinline__ int zmap(int p, int nz)
{
    if (WALL) return p < 0 ? -1 - p : (p >= nz ? 2 * nz - 1 - p : p);
    return p < 0 ? p + nz : (p >= nz ? p - nz : p);
}

// sign of vector z components at an extended z index
template <bool WALL>
__device__ __forceinline__ float zsign(int p, int nz)
{
    return (WALL && (p < 0 || p >= nz)) ? -1.0f : 1.0f;
}

__device__ __forceinline__ int slot4(int p) { return (p + 8) & 3; }
__device__ __forceinline__ int slot3(int p) { return (p + 9) % 3; }

template <bool WALL>
__global__ void __launch_bounds__(NT, 2) fused_step_kernel(Grid G, Phys P, StepArgs a, int TZ)
{
    __shared__ float sPhi[4][N3];
    __shared__ float sU[3][N2];
    __shared__ float sW[3][3][N2];
    __shared__ float sPn[3][N1];

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * TZ;
    const int zend = min(z0 + TZ, G.nz);
    const int nx = G.nx, ny = G.ny, nz = G.nz, nxy = G.nxy;
    const size_t N = (size_t)G.N;

    // (x, y) offsets of the halo points this thread loads
    int off3[K3], off2[K2];
#pragma unroll
    for (int k = 0; k < K3; ++k) {
        const int t = tid + k * NT;
        const int ry = t / R3X, rx = t - ry * R3X;
        off3[k] = wrapc(y0 - 3 + ry, ny) * nx + wrapc(x0 - 3 + rx, nx);
    }
#pragma unroll
    for (int k = 0; k < K2; ++k) {
        const int t = tid + k * NT;
        const int ry = t / R2X, rx = t - ry * R2X;
        off2[k] = wrapc(y0 - 2 + ry, ny) * nx + wrapc(x0 - 2 + rx, nx);
    }

    // own column and its periodic x, y neighbours
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < nx && y < ny;
    const int xo[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
    const int yo[3] = {(y == 0 ? ny - 1 : y - 1) * nx, y * nx, (y == ny - 1 ? 0 : y + 1) * nx};

    const int nsteps = (zend - z0) + 6;
    for (int s = 0; s < nsteps; ++s) {
        const int zl = z0 - 3 + s;       // phi^n plane loaded now
        const int zw = zl - 1;           // W plane
        const int zp = zl - 2;           // phi^{n+1} plane
        const int zc = zl - 3;           // lattice Boltzmann plane
        const bool do_w = s >= 2, do_p = s >= 4, do_c = s >= 6 && active;

        // 0. pulled populations of plane zc: f_i(x) = g_i(x - c_i)
        float f[27];
        int kc = 0;
        if (do_c) {
            const int zs[3] = {zmap<false>(zc - 1, nz) * nxy, zc * nxy, zmap<false>(zc + 1, nz) * nxy};
            kc = zs[1] + yo[1] + x;
            const bool wlo = WALL && zc == 0, whi = WALL && zc == nz - 1;
#pragma unroll
            for (int i = 0; i < 27; ++i) {
                bool bounce = false;
                if (cz(i) == 1) bounce = wlo;
                if (cz(i) == -1) bounce = whi;
                const size_t src = bounce ? (size_t)(26 - i) * N + kc
                                          : (size_t)i * N + (zs[1 - cz(i)] + yo[1 - cy(i)] + xo[1 - cx(i)]);
                f[i] = __ldg(a.g_in + src);
            }
        }

        // 1. phi^n plane zl (halo 3) and ubar^n plane zw (halo 2)
        {
            const int pl = zmap<WALL>(zl, nz) * nxy;
            float *dst = sPhi[slot4(zl)];
#pragma unroll
            for (int k = 0; k < K3; ++k) {
                const int t = tid + k * NT;
                if (t < N3) dst[t] = __ldg(a.phi_in + pl + off3[k]);
            }
            if (do_w) {
                const int pw = zmap<WALL>(zw, nz) * nxy;
                const float sg = zsign<WALL>(zw, nz);
#pragma unroll
                for (int k = 0; k < K2; ++k) {
                    const int t = tid + k * NT;
                    if (t < N2) {
                        sU[0][t] = __ldg(a.u_in + pw + off2[k]);
                        sU[1][t] = __ldg(a.u_in + N + pw + off2[k]);
                        sU[2][t] = sg * __ldg(a.u_in + 2 * N + pw + off2[k]);
                    }
                }
            }
        }
        __syncthreads();

        // 2. Allen–Cahn flux on plane zw (halo 2)
        if (do_w) {
            const float *ph[3] = {sPhi[slot4(zw - 1)], sPhi[slot4(zw)], sPhi[slot4(zw + 1)]};
            float *w = &sW[slot3(zw)][0][0];
#pragma unroll
            for (int k = 0; k < K2; ++k) {
                const int t = tid + k * NT;
                if (t < N2) {
                    const int ry = t / R2X, rx = t - ry * R2X;
                    const int c3 = (ry + 1) * R3X + rx + 1;
                    float psi[27];
#pragma unroll
                    for (int i = 0; i < 27; ++i) psi[i] = ph[cz(i) + 1][c3 + cy(i) * R3X + cx(i)];
                    float gx, gy, gz;
                    grad27(psi, gx, gy, gz);
                    const float inv = rsqrtf(fmaxf(gx * gx + gy * gy + gz * gz, kNormalEps * kNormalEps));
                    const float p = psi[13];
                    const float sh = P.kac * p * (1.0f - p) * inv;
                    w[t] = fmaf(sU[0][t], p, sh * gx);
                    w[N2 + t] = fmaf(sU[1][t], p, sh * gy);
                    w[2 * N2 + t] = fmaf(sU[2][t], p, sh * gz);
                }
            }
        }
        __syncthreads();

        // 3. phi^{n+1} on plane zp (halo 1)
        if (do_p) {
            const float *ph[3] = {sPhi[slot4(zp - 1)], sPhi[slot4(zp)], sPhi[slot4(zp + 1)]};
            const float *ws[3] = {&sW[slot3(zp - 1)][0][0], &sW[slot3(zp)][0][0], &sW[slot3(zp + 1)][0][0]};
            float *dst = sPn[slot3(zp)];
#pragma unroll
            for (int k = 0; k < K1; ++k) {
                const int t = tid + k * NT;
                if (t < N1) {
                    const int ry = t / R1X, rx = t - ry * R1X;
                    const int c2 = (ry + 1) * R2X + rx + 1;
                    const int c3 = (ry + 2) * R3X + rx + 2;
                    float div = 0.f;
#pragma unroll
                    for (int i = 0; i < 27; ++i) {
                        if (i == 13) continue;
                        const float w3 = 3.0f * wgt(i);
                        const float *wp = ws[cz(i) + 1] + c2 + cy(i) * R2X + cx(i);
                        if (cx(i)) div = fmaf(cx(i) * w3, wp[0], div);
                        if (cy(i)) div = fmaf(cy(i) * w3, wp[N2], div);
                        if (cz(i)) div = fmaf(cz(i) * w3, wp[2 * N2], div);
                    }
                    float psi[27];
#pragma unroll
                    for (int i = 0; i < 27; ++i) psi[i] = ph[cz(i) + 1][c3 + cy(i) * R3X + cx(i)];
                    const float p0 = psi[13];
                    const float lap = lap27(psi);
                    dst[t] = p0 - div + P.mob * lap;
                }
            }
        }
        __syncthreads();

        // 4. lattice Boltzmann update of the own node on plane zc
        if (do_c) {
            const float *pn[3] = {sPn[slot3(zc - 1)], sPn[slot3(zc)], sPn[slot3(zc + 1)]};
            const int c1 = (ty + 1) * R1X + tx + 1;
            float psi[27];
#pragma unroll
            for (int i = 0; i < 27; ++i) psi[i] = pn[cz(i) + 1][c1 + cy(i) * R1X + cx(i)];
            float gx, gy, gz, lap;
            grad_lap27(psi, gx, gy, gz, lap);
            const float ubx = __ldg(a.u_in + kc), uby = __ldg(a.u_in + N + kc), ubz = __ldg(a.u_in + 2 * N + kc);
            float g[27], ux, uy, uz;
            collide_node(f, psi[13], gx, gy, gz, lap, ubx, uby, ubz, P, g, ux, uy, uz);
#pragma unroll
            for (int i = 0; i < 27; ++i) a.g_out[(size_t)i * N + kc] = g[i];
            a.u_out[kc] = ux;
            a.u_out[N + kc] = uy;
            a.u_out[2 * N + kc] = uz;
            a.phi_out[kc] = psi[13];
        }
    }
}

}  // namespace

int fused_default_chunk(const Grid &G)
{
    // z chunk per CTA: enough CTAs for several waves on 148 SMs while keeping the 6-plane
    // prologue of each chunk small.
    const long long cols = (long long)((G.nx + TX - 1) / TX) * ((G.ny + TY - 1) / TY);
    int tz = G.nz;
    while (tz > 16 && cols * ((G.nz + tz - 1) / tz) < 148 * 2 * 4) tz = (tz + 1) / 2;
    return tz;
}

cudaError_t launch_step_fused(const Grid &G, const Phys &P, const StepArgs &a, int tz, cudaStream_t s)
{
    if (tz <= 0) tz = fused_default_chunk(G);
    const dim3 grid((G.nx + TX - 1) / TX, (G.ny + TY - 1) / TY, (G.nz + tz - 1) / tz);
    if (G.wall)
        fused_step_kernel<true><<<grid, NT, 0, s>>>(G, P, a, tz);
    else
        fused_step_kernel<false><<<grid, NT, 0, s>>>(G, P, a, tz);
    return cudaGetLastError();
}

}  // namespace tslb

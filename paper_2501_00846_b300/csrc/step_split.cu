// Two-kernel step: a separable z-marching Allen–Cahn kernel writes phi^{n+1}; the one-thread-per-
// node lattice Boltzmann kernel (step_unfused.cu) then streams the populations.
//
// Allen–Cahn kernel.  The 27-point stencils factorise over the D3Q27 weights (w = w1 w1 w1,
// w1(0) = 2/3, w1(+-1) = 1/6) into 3x3 partials of one z plane combined over three planes:
//   Px = sum_dy w1(dy) (psi(x+1,y+dy) - psi(x-1,y+dy)),  Py likewise,
//   Sd = sum w1 w1 (psi(x+dx,y+dy) - psi(x,y)),  c = psi(x,y)
//   d_x psi = 1/2 [2/3 Px(z) + 1/6 (Px(z-1) + Px(z+1))],  d_z psi = 1/2 [(Sd + c)(z+1) - (Sd + c)(z-1)]
//   lap psi = 6 [2/3 Sd(z) + 1/6 (Sd(z-1) + Sd(z+1)) + 1/6 ((c(z-1) - c(z)) + (c(z+1) - c(z)))]
//   div V   = 1/2 [2/3 Q(z) + 1/6 (Q(z-1) + Q(z+1))] + 1/2 [T(z+1) - T(z-1)],
//             Q = Px[V_x] + Py[V_y],  T = sum w1 w1 V_z
// (the paper's isotropic gradient and, reading R2, Laplacian).  A CTA of 32 x 8 threads owns a
// 32 x 8 column tile; thread t owns the halo-1 points t and t + 256 of the tile's 34 x 10 halo-1
// plane, so the z combination of its partials reads only its own shared-memory slots.  Per plane p
// loaded: partials of phi^n (p) on the halo-1 points, W = ubar phi + kappa_AC phi (1-phi) n on plane
// p-1 (halo 1), Q and T of W on plane p-1 and phi^{n+1} = phi^n - div W + D lap phi^n on plane p-2
// at the tile's own nodes.  phi^n (halo 2) and ubar^n (own points) of the next plane are loaded
// into registers one iteration ahead.  Units (column tile, z chunk) are dealt round-robin so all
// CTAs march the same z range at the same time.
#include "tslb_internal.h"

namespace tslb {
namespace {

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int NT = TX * TY;
constexpr int R2X = TX + 4, R2Y = TY + 4, N2 = R2X * R2Y;   // halo 2
constexpr int R1X = TX + 2, R1Y = TY + 2, N1 = R1X * R1Y;   // halo 1
constexpr int K2 = (N2 + NT - 1) / NT;
constexpr int K1 = (N1 + NT - 1) / NT;

constexpr float W0 = 2.0f / 3.0f, W1 = 1.0f / 6.0f;
constexpr float WE = W0 * W1, WC = W1 * W1;

__device__ __forceinline__ int wrapc(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

template <bool WALL>
__device__ __forceinline__ int zmap(int p, int nz)
{
    if (WALL) return p < 0 ? -1 - p : (p >= nz ? 2 * nz - 1 - p : p);
    return p < 0 ? p + nz : (p >= nz ? p - nz : p);
}

template <bool WALL>
__device__ __forceinline__ float zsign(int p, int nz)
{
    return (WALL && (p < 0 || p >= nz)) ? -1.0f : 1.0f;
}

__device__ __forceinline__ int slot3(int p) { return (p + 9) % 3; }
__device__ __forceinline__ int slot4(int p) { return (p + 8) & 3; }

template <bool WALL>
__global__ void __launch_bounds__(NT, 4) ac_split_kernel(Grid G, Phys P, const float *__restrict__ phi_in,
                                                         const float *__restrict__ u_in, float *__restrict__ phi_out,
                                                         int ncols, int zlen, int units)
{
    __shared__ float sPhi[N2];             // phi^n plane, halo 2
    __shared__ float sW[3][N1];            // W plane, halo 1
    __shared__ float sPxy[3][2][N1];       // Px, Py of phi^n, 3 plane slots
    __shared__ float sSc[4][2][N1];        // Sd, c of phi^n, 4 plane slots
    __shared__ float sQt[3][2][N1];        // Q, T of W, 3 plane slots

    const int tid = threadIdx.x;
    const int nx = G.nx, ny = G.ny, nz = G.nz, nxy = G.nxy;
    const size_t N = (size_t)G.N;
    const int ncx = (nx + TX - 1) / TX;

    // halo-1 points owned by this thread; core = also a node of the tile
    int ry1[K1], rx1[K1];
    bool own[K1], core[K1];
#pragma unroll
    for (int k = 0; k < K1; ++k) {
        const int t = tid + k * NT;
        own[k] = t < N1;
        ry1[k] = t / R1X;
        rx1[k] = t - ry1[k] * R1X;
        core[k] = own[k] && ry1[k] >= 1 && ry1[k] <= TY && rx1[k] >= 1 && rx1[k] <= TX;
    }

    for (int unit = blockIdx.x; unit < units; unit += gridDim.x) {
        const int col = unit % ncols;
        const int z0 = (unit / ncols) * zlen;
        const int zend = min(nz, z0 + zlen);
        const int x0 = (col % ncx) * TX, y0 = (col / ncx) * TY;

        int off2[K2], off1[K1];
        bool store[K1];
#pragma unroll
        for (int k = 0; k < K2; ++k) {
            const int t = tid + k * NT;
            const int ry = t / R2X, rx = t - ry * R2X;
            off2[k] = wrapc(y0 - 2 + ry, ny) * nx + wrapc(x0 - 2 + rx, nx);
        }
#pragma unroll
        for (int k = 0; k < K1; ++k) {
            off1[k] = wrapc(y0 - 1 + ry1[k], ny) * nx + wrapc(x0 - 1 + rx1[k], nx);
            store[k] = core[k] && x0 - 1 + rx1[k] < nx && y0 - 1 + ry1[k] < ny;
        }

        // registers one iteration ahead: phi^n (halo 2) of the next plane, ubar^n at own points
        float nphi[K2], nub[K1][3];
        {
            const int pl = zmap<WALL>(z0 - 2, nz) * nxy;
#pragma unroll
            for (int k = 0; k < K2; ++k) nphi[k] = (tid + k * NT < N2) ? __ldg(phi_in + pl + off2[k]) : 0.0f;
#pragma unroll
            for (int k = 0; k < K1; ++k) nub[k][0] = nub[k][1] = nub[k][2] = 0.0f;
        }

        const int nsteps = (zend - z0) + 4;
        for (int s = 0; s < nsteps; ++s) {
            const int p = z0 - 2 + s;
            const bool do_w = s >= 2, do_e = s >= 4;

            // phi^n plane p into shared memory; ubar^n plane p-1 stays in registers (cub)
            float cub[K1][3];
#pragma unroll
            for (int k = 0; k < K2; ++k)
                if (tid + k * NT < N2) sPhi[tid + k * NT] = nphi[k];
#pragma unroll
            for (int k = 0; k < K1; ++k) {
                cub[k][0] = nub[k][0];
                cub[k][1] = nub[k][1];
                cub[k][2] = nub[k][2];
            }
            if (s + 1 < nsteps) {
                const int pl = zmap<WALL>(p + 1, nz) * nxy;
#pragma unroll
                for (int k = 0; k < K2; ++k)
                    if (tid + k * NT < N2) nphi[k] = __ldg(phi_in + pl + off2[k]);
                if (s + 1 >= 2) {
                    const int pw = zmap<WALL>(p, nz) * nxy;
                    const float sg = zsign<WALL>(p, nz);
#pragma unroll
                    for (int k = 0; k < K1; ++k) {
                        if (own[k]) {
                            nub[k][0] = __ldg(u_in + pw + off1[k]);
                            nub[k][1] = __ldg(u_in + N + pw + off1[k]);
                            nub[k][2] = sg * __ldg(u_in + 2 * N + pw + off1[k]);
                        }
                    }
                }
            }
            __syncthreads();

            // partials of phi^n plane p; W on plane p-1 (own halo-1 points)
            {
                float(*pxy_p)[N1] = sPxy[slot3(p)];
                float(*sc_p)[N1] = sSc[slot4(p)];
                const float(*pxy_m1)[N1] = sPxy[slot3(p - 1)];
                const float(*pxy_m2)[N1] = sPxy[slot3(p - 2)];
                const float(*sc_m1)[N1] = sSc[slot4(p - 1)];
                const float(*sc_m2)[N1] = sSc[slot4(p - 2)];
#pragma unroll
                for (int k = 0; k < K1; ++k) {
                    if (!own[k]) continue;
                    const int t = tid + k * NT;
                    const int ci = (ry1[k] + 1) * R2X + rx1[k] + 1;
                    const float m0 = sPhi[ci - R2X - 1], m1 = sPhi[ci - R2X], m2 = sPhi[ci - R2X + 1];
                    const float l0 = sPhi[ci - 1], c = sPhi[ci], l2 = sPhi[ci + 1];
                    const float q0 = sPhi[ci + R2X - 1], q1 = sPhi[ci + R2X], q2 = sPhi[ci + R2X + 1];
                    const float px = fmaf(W0, l2 - l0, W1 * ((m2 - m0) + (q2 - q0)));
                    const float py = fmaf(W0, q1 - m1, W1 * ((q0 - m0) + (q2 - m2)));
                    const float sd = fmaf(WE, ((m1 - c) + (q1 - c)) + ((l0 - c) + (l2 - c)),
                                          WC * (((m0 - c) + (m2 - c)) + ((q0 - c) + (q2 - c))));
                    pxy_p[0][t] = px;
                    pxy_p[1][t] = py;
                    sc_p[0][t] = sd;
                    sc_p[1][t] = c;
                    if (do_w) {
                        const float gx = 0.5f * fmaf(W0, pxy_m1[0][t], W1 * (pxy_m2[0][t] + px));
                        const float gy = 0.5f * fmaf(W0, pxy_m1[1][t], W1 * (pxy_m2[1][t] + py));
                        const float gz = 0.5f * ((sd - sc_m2[0][t]) + (c - sc_m2[1][t]));
                        const float ph = sc_m1[1][t];
                        const float inv = rsqrtf(fmaxf(gx * gx + gy * gy + gz * gz, kNormalEps * kNormalEps));
                        const float sh = P.kac * fmaxf(ph * (1.0f - ph), 0.0f) * inv;
                        sW[0][t] = fmaf(cub[k][0], ph, sh * gx);
                        sW[1][t] = fmaf(cub[k][1], ph, sh * gy);
                        sW[2][t] = fmaf(cub[k][2], ph, sh * gz);
                    }
                }
            }
            __syncthreads();

            // Q, T of W on plane p-1 and phi^{n+1} on plane p-2 at the tile's own nodes
            if (do_w) {
                float(*qt_m1)[N1] = sQt[slot3(p - 1)];
                const float(*qt_m2)[N1] = sQt[slot3(p - 2)];
                const float(*qt_m3)[N1] = sQt[slot3(p - 3)];
                const float(*sc_m1)[N1] = sSc[slot4(p - 1)];
                const float(*sc_m2)[N1] = sSc[slot4(p - 2)];
                const float(*sc_m3)[N1] = sSc[slot4(p - 3)];
                const float *wx = sW[0], *wy = sW[1], *wz = sW[2];
#pragma unroll
                for (int k = 0; k < K1; ++k) {
                    if (!core[k]) continue;
                    const int t = tid + k * NT;
                    const float q = fmaf(W0, wx[t + 1] - wx[t - 1],
                                         W1 * ((wx[t - R1X + 1] - wx[t - R1X - 1]) + (wx[t + R1X + 1] - wx[t + R1X - 1])))
                                  + fmaf(W0, wy[t + R1X] - wy[t - R1X],
                                         W1 * ((wy[t + R1X - 1] - wy[t - R1X - 1]) + (wy[t + R1X + 1] - wy[t - R1X + 1])));
                    const float tt = fmaf(W0 * W0, wz[t],
                                          fmaf(WE, (wz[t - 1] + wz[t + 1]) + (wz[t - R1X] + wz[t + R1X]),
                                               WC * ((wz[t - R1X - 1] + wz[t - R1X + 1]) + (wz[t + R1X - 1] + wz[t + R1X + 1]))));
                    qt_m1[0][t] = q;
                    qt_m1[1][t] = tt;
                    if (do_e && store[k]) {
                        const float div = 0.5f * fmaf(W0, qt_m2[0][t], W1 * (qt_m3[0][t] + q)) + 0.5f * (tt - qt_m3[1][t]);
                        const float c2 = sc_m2[1][t];
                        const float lap = 6.0f * fmaf(W0, sc_m2[0][t],
                                                      W1 * ((sc_m3[0][t] + sc_m1[0][t]) + ((sc_m3[1][t] - c2) + (sc_m1[1][t] - c2))));
                        phi_out[(size_t)(p - 2) * nxy + off1[k]] = c2 - div + P.mob * lap;
                    }
                }
            }
        }
    }
}

struct LaunchAC {
    int blocks_per_sm = 0;
    int sms = 0;
};

template <bool WALL>
cudaError_t prepare_ac(LaunchAC &L)
{
    int dev = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&L.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L.blocks_per_sm, ac_split_kernel<WALL>, NT, 0);
}

}  // namespace

cudaError_t launch_ac_split(const Grid &G, const Phys &P, const float *phi_in, const float *u_in, float *phi_out,
                            int zchunks, cudaStream_t s)
{
    static LaunchAC lw[2];
    LaunchAC &L = lw[G.wall ? 1 : 0];
    if (L.sms == 0) {
        cudaError_t e = G.wall ? prepare_ac<true>(L) : prepare_ac<false>(L);
        if (e != cudaSuccess) return e;
        if (L.blocks_per_sm < 1) return cudaErrorInvalidConfiguration;
    }
    const int slots = L.sms * L.blocks_per_sm;
    const int ncols = ((G.nx + TX - 1) / TX) * ((G.ny + TY - 1) / TY);
    int m = zchunks;
    if (m <= 0) {
        m = slots / ncols;
        if (m > G.nz / 16) m = G.nz / 16;
        if (m < 1) m = 1;
    }
    if (m > G.nz) m = G.nz;
    const int zlen = (G.nz + m - 1) / m;
    m = (G.nz + zlen - 1) / zlen;
    const int units = ncols * m;
    const int rounds = (units + slots - 1) / slots;
    const int ctas = (units + rounds - 1) / rounds;
    if (G.wall)
        ac_split_kernel<true><<<ctas, NT, 0, s>>>(G, P, phi_in, u_in, phi_out, ncols, zlen, units);
    else
        ac_split_kernel<false><<<ctas, NT, 0, s>>>(G, P, phi_in, u_in, phi_out, ncols, zlen, units);
    return cudaGetLastError();
}

cudaError_t launch_step_split(const Grid &G, const Phys &P, const StepArgs &a, int zchunks, cudaStream_t s)
{
    cudaError_t e = launch_ac_split(G, P, a.phi_in, a.u_in, a.phi_out, zchunks, s);
    if (e != cudaSuccess) return e;
    return launch_lbm(G, P, a.g_in, a.phi_out, a.u_in, a.g_out, a.u_out, s);
}

}  // namespace tslb

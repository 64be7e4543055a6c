// Fused step, separable-stencil form with persistent CTAs.
//
// The D3Q27 weights factorise, w(c) = w1(cx) w1(cy) w1(cz) with w1(0) = 2/3, w1(+-1) = 1/6, so
// every 27-point operator of the step splits into 3x3 partials of one z plane, combined over the
// planes z-1, z, z+1.  For a scalar psi and a point (x, y) of plane z':
//   Px = sum_dy w1(dy) (psi(x+1, y+dy) - psi(x-1, y+dy))        Py likewise with x <-> y
//   Sd = sum_{dx,dy} w1(dx) w1(dy) (psi(x+dx, y+dy) - psi(x, y))  c = psi(x, y)
// and for the target (x, y, z):
//   d_x psi = 1/2 [2/3 Px(z) + 1/6 (Px(z-1) + Px(z+1))]          d_y psi likewise with Py
//   d_z psi = 1/2 [(Sd(z+1) - Sd(z-1)) + (c(z+1) - c(z-1))]
//   lap psi = 6 [2/3 Sd(z) + 1/6 (Sd(z-1) + Sd(z+1)) + 1/6 ((c(z-1) - c(z)) + (c(z+1) - c(z)))]
// which are exactly the paper's isotropic gradient and (reading R2) Laplacian stencils.  The
// divergence of a vector V uses Q = Px[V_x] + Py[V_y] and T = sum w1 w1 V_z:
//   div V = 1/2 [2/3 Q(z) + 1/6 (Q(z-1) + Q(z+1))] + 1/2 [T(z+1) - T(z-1)].
//
// A CTA of 32 x 8 threads works on a 32 x 8 column tile; thread t owns the halo-2 points t and
// t + 256 of the tile's (36 x 12) halo-2 plane for every Allen–Cahn stage, so the combination over
// z of its partials reads only its own shared-memory slots.  Per z plane p (loaded now):
//   a. load phi^n plane p (halo 3) and ubar^n plane p-1 (halo 2)                      sync
//   b. phi^n partials (Px, Py, Sd, c) of plane p on the halo-2 points
//   c. W = ubar phi + kappa_AC phi (1-phi) n on plane p-1 (halo 2)                     sync
//   d. Q, T of W on plane p-1 (halo 1)
//   e. phi^{n+1} = phi^n - div W + D lap phi^n on plane p-2 (halo 1)                   sync
//   f. partials of phi^{n+1} at the own node (plane p-2), then the lattice Boltzmann update of
//      the own node on plane p-3 (pull, forces, regularised collision), whose 27 population
//      loads were issued at the top of the iteration.
// The phi^n and ubar^n values of the next plane are loaded into registers one iteration ahead
// (stored to shared memory at the top of the next iteration), and the own node's ubar^n with the
// pulled populations, so no stage waits on a global load it has just issued.
// Scheduling: the box is cut into units (column tile, z chunk of equal length); units are dealt
// round-robin to the CTAs, so in every round all CTAs march the same z range and a tile's
// neighbours are processed at the same time (their halo rows are then L2 hits).
#include "tslb_internal.h"

namespace tslb {
namespace {

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int NT = TX * TY;
constexpr int R3X = TX + 6, R3Y = TY + 6, N3 = R3X * R3Y;   // halo 3
constexpr int R2X = TX + 4, R2Y = TY + 4, N2 = R2X * R2Y;   // halo 2
constexpr int R1X = TX + 2, R1Y = TY + 2, N1 = R1X * R1Y;   // halo 1
constexpr int K3 = (N3 + NT - 1) / NT;
constexpr int K2 = (N2 + NT - 1) / NT;

constexpr float W0 = 2.0f / 3.0f, W1 = 1.0f / 6.0f;        // w1(0), w1(+-1)
constexpr float WE = W0 * W1, WC = W1 * W1;                 // 3x3 edge and corner weights

// shared-memory layout (floats)
constexpr int OFF_PHI = 0;                    // phi^n plane, halo 3
constexpr int OFF_U = OFF_PHI + N3;           // ubar^n plane, halo 2, 3 components
constexpr int OFF_W = OFF_U + 3 * N2;         // W plane, halo 2, 3 components
constexpr int OFF_PN = OFF_W + 3 * N2;        // phi^{n+1} plane, halo 1
constexpr int OFF_PXY = OFF_PN + N1;          // Px, Py of phi^n: 3 plane slots x 2 x N2
constexpr int OFF_SC = OFF_PXY + 3 * 2 * N2;  // Sd, c of phi^n: 4 plane slots x 2 x N2
constexpr int OFF_QT = OFF_SC + 4 * 2 * N2;   // Q, T of W: 3 plane slots x 2 x N2
constexpr int SMEM_FLOATS = OFF_QT + 3 * 2 * N2;
constexpr size_t SMEM_BYTES = SMEM_FLOATS * sizeof(float);

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

// 3x3 partials of a scalar plane around element `ci` of an array with row pitch RX.
template <int RX>
__device__ __forceinline__ void partials(const float *a, int ci, float &px, float &py, float &sd, float &c)
{
    const float m0 = a[ci - RX - 1], m1 = a[ci - RX], m2 = a[ci - RX + 1];
    const float l0 = a[ci - 1], l1 = a[ci], l2 = a[ci + 1];
    const float p0 = a[ci + RX - 1], p1 = a[ci + RX], p2 = a[ci + RX + 1];
    c = l1;
    px = fmaf(W0, l2 - l0, W1 * ((m2 - m0) + (p2 - p0)));
    py = fmaf(W0, p1 - m1, W1 * ((p0 - m0) + (p2 - m2)));
    sd = fmaf(WE, ((m1 - l1) + (p1 - l1)) + ((l0 - l1) + (l2 - l1)),
              WC * (((m0 - l1) + (m2 - l1)) + ((p0 - l1) + (p2 - l1))));
}

template <bool WALL>
__global__ void __launch_bounds__(NT, 2) fused2_kernel(Grid G, Phys P, StepArgs a, int ncols, int zlen, int units)
{
    extern __shared__ float sm[];
    float *sPhi = sm + OFF_PHI;
    float *sU = sm + OFF_U;
    float *sW = sm + OFF_W;
    float *sPn = sm + OFF_PN;

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int nx = G.nx, ny = G.ny, nz = G.nz, nxy = G.nxy;
    const size_t N = (size_t)G.N;
    const int ncx = (nx + TX - 1) / TX;

    // halo-2 points owned by this thread (k = 0, 1) and whether each is also a halo-1 point
    int ry2[K2], rx2[K2];
    bool own2[K2], own1[K2];
#pragma unroll
    for (int k = 0; k < K2; ++k) {
        const int t = tid + k * NT;
        own2[k] = t < N2;
        ry2[k] = t / R2X;
        rx2[k] = t - ry2[k] * R2X;
        own1[k] = own2[k] && ry2[k] >= 1 && ry2[k] <= R2Y - 2 && rx2[k] >= 1 && rx2[k] <= R2X - 2;
    }

    for (int unit = blockIdx.x; unit < units; unit += gridDim.x) {
        const int col = unit % ncols;
        const int z0 = (unit / ncols) * zlen;
        const int zend = min(nz, z0 + zlen);
        const int x0 = (col % ncx) * TX, y0 = (col / ncx) * TY;

        int off3[K3], off2[K2];
#pragma unroll
        for (int k = 0; k < K3; ++k) {
            const int t = tid + k * NT;
            const int ry = t / R3X, rx = t - ry * R3X;
            off3[k] = wrapc(y0 - 3 + ry, ny) * nx + wrapc(x0 - 3 + rx, nx);
        }
#pragma unroll
        for (int k = 0; k < K2; ++k) off2[k] = wrapc(y0 - 2 + ry2[k], ny) * nx + wrapc(x0 - 2 + rx2[k], nx);

        const int x = x0 + tx, y = y0 + ty;
        const bool active = x < nx && y < ny;
        const int xo[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
        const int yo[3] = {(y == 0 ? ny - 1 : y - 1) * nx, y * nx, (y == ny - 1 ? 0 : y + 1) * nx};

        // own-node partials of phi^{n+1} on the two planes below the newest one
        float qx0 = 0.f, qy0 = 0.f, qs0 = 0.f, qc0 = 0.f;   // plane p-4
        float qx1 = 0.f, qy1 = 0.f, qs1 = 0.f, qc1 = 0.f;   // plane p-3

        // phi^n (halo 3) of the plane loaded next, and ubar^n (own halo-2 points) of the plane
        // before it, held in registers one iteration ahead of their use
        float nphi[K3], nub[K2][3];
        {
            const int pl = zmap<WALL>(z0 - 3, nz) * nxy;
#pragma unroll
            for (int k = 0; k < K3; ++k)
                nphi[k] = (tid + k * NT < N3) ? __ldg(a.phi_in + pl + off3[k]) : 0.0f;
#pragma unroll
            for (int k = 0; k < K2; ++k) nub[k][0] = nub[k][1] = nub[k][2] = 0.0f;
        }

        const int nsteps = (zend - z0) + 6;
        for (int s = 0; s < nsteps; ++s) {
            const int p = z0 - 3 + s;
            const bool do_w = s >= 2, do_e = s >= 4, do_c = s >= 6 && active;
            const int zc = p - 3;

            // pulled populations of plane zc and the own ubar^n, issued early
            float f[27];
            float ubx = 0.f, uby = 0.f, ubz = 0.f;
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
                ubx = __ldg(a.u_in + kc);
                uby = __ldg(a.u_in + N + kc);
                ubz = __ldg(a.u_in + 2 * N + kc);
            }

            // a. phi^n plane p (halo 3) and ubar^n plane p-1 (own halo-2 points) from the
            //    registers loaded one iteration ago; then load plane p+1 / p into them
            {
#pragma unroll
                for (int k = 0; k < K3; ++k) {
                    const int t = tid + k * NT;
                    if (t < N3) sPhi[t] = nphi[k];
                }
#pragma unroll
                for (int k = 0; k < K2; ++k) {
                    if (own2[k]) {
                        const int t = tid + k * NT;
                        sU[t] = nub[k][0];
                        sU[N2 + t] = nub[k][1];
                        sU[2 * N2 + t] = nub[k][2];
                    }
                }
                if (s + 1 < nsteps) {
                    const int pl = zmap<WALL>(p + 1, nz) * nxy;
#pragma unroll
                    for (int k = 0; k < K3; ++k)
                        if (tid + k * NT < N3) nphi[k] = __ldg(a.phi_in + pl + off3[k]);
                    if (s + 1 >= 2) {
                        const int pw = zmap<WALL>(p, nz) * nxy;
                        const float sg = zsign<WALL>(p, nz);
#pragma unroll
                        for (int k = 0; k < K2; ++k) {
                            if (own2[k]) {
                                nub[k][0] = __ldg(a.u_in + pw + off2[k]);
                                nub[k][1] = __ldg(a.u_in + N + pw + off2[k]);
                                nub[k][2] = sg * __ldg(a.u_in + 2 * N + pw + off2[k]);
                            }
                        }
                    }
                }
            }
            __syncthreads();

            // b. partials of phi^n plane p;  c. W on plane p-1 (own halo-2 points)
            {
                float *pxy_p = sm + OFF_PXY + slot3(p) * 2 * N2;
                float *sc_p = sm + OFF_SC + slot4(p) * 2 * N2;
                const float *pxy_m1 = sm + OFF_PXY + slot3(p - 1) * 2 * N2;
                const float *pxy_m2 = sm + OFF_PXY + slot3(p - 2) * 2 * N2;
                const float *sc_m1 = sm + OFF_SC + slot4(p - 1) * 2 * N2;
                const float *sc_m2 = sm + OFF_SC + slot4(p - 2) * 2 * N2;
#pragma unroll
                for (int k = 0; k < K2; ++k) {
                    if (!own2[k]) continue;
                    const int t = tid + k * NT;
                    float px, py, sd, c;
                    partials<R3X>(sPhi, (ry2[k] + 1) * R3X + rx2[k] + 1, px, py, sd, c);
                    pxy_p[t] = px;
                    pxy_p[N2 + t] = py;
                    sc_p[t] = sd;
                    sc_p[N2 + t] = c;
                    if (do_w) {
                        const float gx = 0.5f * fmaf(W0, pxy_m1[t], W1 * (pxy_m2[t] + px));
                        const float gy = 0.5f * fmaf(W0, pxy_m1[N2 + t], W1 * (pxy_m2[N2 + t] + py));
                        const float gz = 0.5f * ((sd - sc_m2[t]) + (c - sc_m2[N2 + t]));
                        const float ph = sc_m1[N2 + t];
                        const float inv = rsqrtf(fmaxf(gx * gx + gy * gy + gz * gz, kNormalEps * kNormalEps));
                        const float sh = P.kac * fmaxf(ph * (1.0f - ph), 0.0f) * inv;
                        sW[t] = fmaf(sU[t], ph, sh * gx);
                        sW[N2 + t] = fmaf(sU[N2 + t], ph, sh * gy);
                        sW[2 * N2 + t] = fmaf(sU[2 * N2 + t], ph, sh * gz);
                    }
                }
            }
            __syncthreads();

            // d. Q, T of W on plane p-1;  e. phi^{n+1} on plane p-2 (own halo-1 points)
            if (do_w) {
                float *qt_m1 = sm + OFF_QT + slot3(p - 1) * 2 * N2;
                const float *qt_m2 = sm + OFF_QT + slot3(p - 2) * 2 * N2;
                const float *qt_m3 = sm + OFF_QT + slot3(p - 3) * 2 * N2;
                const float *sc_m1 = sm + OFF_SC + slot4(p - 1) * 2 * N2;
                const float *sc_m2 = sm + OFF_SC + slot4(p - 2) * 2 * N2;
                const float *sc_m3 = sm + OFF_SC + slot4(p - 3) * 2 * N2;
#pragma unroll
                for (int k = 0; k < K2; ++k) {
                    if (!own1[k]) continue;
                    const int t = tid + k * NT;
                    const float *wx = sW, *wy = sW + N2, *wz = sW + 2 * N2;
                    const float q = fmaf(W0, wx[t + 1] - wx[t - 1],
                                         W1 * ((wx[t - R2X + 1] - wx[t - R2X - 1]) + (wx[t + R2X + 1] - wx[t + R2X - 1])))
                                  + fmaf(W0, wy[t + R2X] - wy[t - R2X],
                                         W1 * ((wy[t + R2X - 1] - wy[t - R2X - 1]) + (wy[t + R2X + 1] - wy[t - R2X + 1])));
                    const float tt = fmaf(W0 * W0, wz[t],
                                          fmaf(WE, (wz[t - 1] + wz[t + 1]) + (wz[t - R2X] + wz[t + R2X]),
                                               WC * ((wz[t - R2X - 1] + wz[t - R2X + 1]) + (wz[t + R2X - 1] + wz[t + R2X + 1]))));
                    qt_m1[t] = q;
                    qt_m1[N2 + t] = tt;
                    if (do_e) {
                        const float div = 0.5f * fmaf(W0, qt_m2[t], W1 * (qt_m3[t] + q)) + 0.5f * (tt - qt_m3[N2 + t]);
                        const float c2 = sc_m2[N2 + t];
                        const float lap = 6.0f * fmaf(W0, sc_m2[t],
                                                      W1 * ((sc_m3[t] + sc_m1[t]) + ((sc_m3[N2 + t] - c2) + (sc_m1[N2 + t] - c2))));
                        sPn[(ry2[k] - 1) * R1X + rx2[k] - 1] = c2 - div + P.mob * lap;
                    }
                }
            }
            __syncthreads();

            // f. partials of phi^{n+1} (plane p-2) at the own node; lattice Boltzmann on plane p-3
            if (do_e && active) {
                float px, py, sd, c;
                partials<R1X>(sPn, (ty + 1) * R1X + tx + 1, px, py, sd, c);
                if (do_c) {
                    const float gx = 0.5f * fmaf(W0, qx1, W1 * (qx0 + px));
                    const float gy = 0.5f * fmaf(W0, qy1, W1 * (qy0 + py));
                    const float gz = 0.5f * ((sd - qs0) + (c - qc0));
                    const float lap = 6.0f * fmaf(W0, qs1, W1 * ((qs0 + sd) + ((qc0 - qc1) + (c - qc1))));
                    float g[27], ux, uy, uz;
                    collide_node(f, qc1, gx, gy, gz, lap, ubx, uby, ubz, P, g, ux, uy, uz);
#pragma unroll
                    for (int i = 0; i < 27; ++i) a.g_out[(size_t)i * N + kc] = g[i];
                    a.u_out[kc] = ux;
                    a.u_out[N + kc] = uy;
                    a.u_out[2 * N + kc] = uz;
                    a.phi_out[kc] = qc1;
                }
                qx0 = qx1; qy0 = qy1; qs0 = qs1; qc0 = qc1;
                qx1 = px; qy1 = py; qs1 = sd; qc1 = c;
            }
        }
    }
}

struct Launch2 {
    int blocks_per_sm = 0;
    int sms = 0;
};

struct Split2 {
    int ncols, zlen, units, ctas;
};

// Units of work: every column tile cut into m z chunks of equal length.  Default m: as many
// chunks as fit one round on the resident slots, keeping chunks of at least 16 planes (the
// march recomputes ~6 halo planes per chunk).  CTAs = units / rounds, rounded up.
Split2 fused2_split(const Grid &G, int slots, int m)
{
    Split2 sp;
    sp.ncols = ((G.nx + TX - 1) / TX) * ((G.ny + TY - 1) / TY);
    if (m <= 0) {
        m = slots / sp.ncols;
        if (m > G.nz / 16) m = G.nz / 16;
        if (m < 1) m = 1;
    }
    if (m > G.nz) m = G.nz;
    sp.zlen = (G.nz + m - 1) / m;
    m = (G.nz + sp.zlen - 1) / sp.zlen;
    sp.units = sp.ncols * m;
    const int rounds = (sp.units + slots - 1) / slots;
    sp.ctas = (sp.units + rounds - 1) / rounds;
    return sp;
}

template <bool WALL>
cudaError_t prepare(Launch2 &L)
{
    cudaError_t e = cudaFuncSetAttribute(fused2_kernel<WALL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    // two CTAs of ~48 KB per SM need a large shared-memory carveout
    e = cudaFuncSetAttribute(fused2_kernel<WALL>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&L.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L.blocks_per_sm, fused2_kernel<WALL>, NT, SMEM_BYTES);
}

}  // namespace

cudaError_t launch_step_fused2(const Grid &G, const Phys &P, const StepArgs &a, int zchunks, cudaStream_t s)
{
    static Launch2 lw[2];
    Launch2 &L = lw[G.wall ? 1 : 0];
    if (L.sms == 0) {
        cudaError_t e = G.wall ? prepare<true>(L) : prepare<false>(L);
        if (e != cudaSuccess) return e;
        if (L.blocks_per_sm < 1) return cudaErrorInvalidConfiguration;
    }
    Split2 sp = fused2_split(G, L.sms * L.blocks_per_sm, zchunks);
    if (G.wall)
        fused2_kernel<true><<<sp.ctas, NT, SMEM_BYTES, s>>>(G, P, a, sp.ncols, sp.zlen, sp.units);
    else
        fused2_kernel<false><<<sp.ctas, NT, SMEM_BYTES, s>>>(G, P, a, sp.ncols, sp.zlen, sp.units);
    return cudaGetLastError();
}

}  // namespace tslb

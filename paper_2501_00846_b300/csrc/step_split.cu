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
// (the paper's isotropic gradient and, reading R2, Laplacian).  A CTA of 352 threads works on a
// 32 x 8 column tile; thread t owns point t of the tile's 34 x 10 halo-1 plane, so the z
// combination of its partials reads only its own registers.  Per plane p
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
constexpr int R2X = TX + 4, R2Y = TY + 4, N2 = R2X * R2Y;   // halo 2
constexpr int R1X = TX + 2, R1Y = TY + 2, N1 = R1X * R1Y;   // halo 1

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


// One thread per halo-1 point (340 of 352 threads); the 4-slot rings of plane partials that only
// the owning thread reads live in its registers (the march is unrolled by 4, so every slot index
// is a compile-time constant).  Shared memory holds only what neighbours read: the phi^n plane
// (halo 2) and the W plane (halo 1).
constexpr int NTA = 352;                          // threads of the Allen-Cahn CTA (11 warps)
constexpr int KA2 = (N2 + NTA - 1) / NTA;         // halo-2 loads per thread

struct AcShared {
    float phi[N2];
    float w[3][N1];
};

struct AcThread {
    int ry1, rx1;
    bool own, core, store;
    int off1;
    int off2[KA2];
    float nphi[KA2], nub[3];
    float px[4], py[4], sd[4], c[4], q[4], t[4];  // rings, slot = plane index mod 4
};

// One plane of the march: iteration s (phase J = s mod 4), plane p = z0 - 2 + s loaded.
template <bool WALL, int J>
__device__ __forceinline__ void ac_iteration(AcShared &sh, AcThread &th, const Grid &G, const Phys &P,
                                             const float *__restrict__ phi_in, const float *__restrict__ u_in,
                                             float *__restrict__ phi_out, int z0, int s, int nsteps)
{
    constexpr int S0 = J, S1 = (J + 3) & 3, S2 = (J + 2) & 3, S3 = (J + 1) & 3;   // slots of p, p-1, p-2, p-3
    const int tid = threadIdx.x;
    const int nz = G.nz, nxy = G.nxy;
    const size_t N = (size_t)G.N;
    const int p = z0 - 2 + s;
    const bool do_w = s >= 2, do_e = s >= 4;

    // phi^n plane p into shared memory; ubar^n plane p-1 from registers; prefetch the next ones
#pragma unroll
    for (int k = 0; k < KA2; ++k)
        if (tid + k * NTA < N2) sh.phi[tid + k * NTA] = th.nphi[k];
    const float ub0 = th.nub[0], ub1 = th.nub[1], ub2 = th.nub[2];
    if (s + 1 < nsteps) {
        const int pl = zmap<WALL>(p + 1, nz) * nxy;
#pragma unroll
        for (int k = 0; k < KA2; ++k)
            if (tid + k * NTA < N2) th.nphi[k] = __ldg(phi_in + pl + th.off2[k]);
        if (s + 1 >= 2 && th.own) {
            const int pw = zmap<WALL>(p, nz) * nxy;
            th.nub[0] = __ldg(u_in + pw + th.off1);
            th.nub[1] = __ldg(u_in + N + pw + th.off1);
            th.nub[2] = zsign<WALL>(p, nz) * __ldg(u_in + 2 * N + pw + th.off1);
        }
    }
    __syncthreads();

    // partials of phi^n plane p; W on plane p-1
    if (th.own) {
        const int ci = (th.ry1 + 1) * R2X + th.rx1 + 1;
        const float *a = sh.phi;
        const float m0 = a[ci - R2X - 1], m1 = a[ci - R2X], m2 = a[ci - R2X + 1];
        const float l0 = a[ci - 1], c = a[ci], l2 = a[ci + 1];
        const float q0 = a[ci + R2X - 1], q1 = a[ci + R2X], q2 = a[ci + R2X + 1];
        th.px[S0] = fmaf(W0, l2 - l0, W1 * ((m2 - m0) + (q2 - q0)));
        th.py[S0] = fmaf(W0, q1 - m1, W1 * ((q0 - m0) + (q2 - m2)));
        th.sd[S0] = fmaf(WE, ((m1 - c) + (q1 - c)) + ((l0 - c) + (l2 - c)),
                         WC * (((m0 - c) + (m2 - c)) + ((q0 - c) + (q2 - c))));
        th.c[S0] = c;
        if (do_w) {
            const int t = tid;
            const float gx = 0.5f * fmaf(W0, th.px[S1], W1 * (th.px[S2] + th.px[S0]));
            const float gy = 0.5f * fmaf(W0, th.py[S1], W1 * (th.py[S2] + th.py[S0]));
            const float gz = 0.5f * ((th.sd[S0] - th.sd[S2]) + (th.c[S0] - th.c[S2]));
            const float ph = th.c[S1];
            const float inv = rsqrtf(fmaxf(gx * gx + gy * gy + gz * gz, kNormalEps * kNormalEps));
            const float shp = P.kac * fmaxf(ph * (1.0f - ph), 0.0f) * inv;
            sh.w[0][t] = fmaf(ub0, ph, shp * gx);
            sh.w[1][t] = fmaf(ub1, ph, shp * gy);
            sh.w[2][t] = fmaf(ub2, ph, shp * gz);
        }
    }
    __syncthreads();

    // Q, T of W on plane p-1 and phi^{n+1} on plane p-2 at the tile's own nodes
    if (do_w && th.core) {
        const int t = tid;
        const float *wx = sh.w[0], *wy = sh.w[1], *wz = sh.w[2];
        th.q[S1] = fmaf(W0, wx[t + 1] - wx[t - 1],
                        W1 * ((wx[t - R1X + 1] - wx[t - R1X - 1]) + (wx[t + R1X + 1] - wx[t + R1X - 1])))
                 + fmaf(W0, wy[t + R1X] - wy[t - R1X],
                        W1 * ((wy[t + R1X - 1] - wy[t - R1X - 1]) + (wy[t + R1X + 1] - wy[t - R1X + 1])));
        th.t[S1] = fmaf(W0 * W0, wz[t],
                        fmaf(WE, (wz[t - 1] + wz[t + 1]) + (wz[t - R1X] + wz[t + R1X]),
                             WC * ((wz[t - R1X - 1] + wz[t - R1X + 1]) + (wz[t + R1X - 1] + wz[t + R1X + 1]))));
        if (do_e && th.store) {
            const float div = 0.5f * fmaf(W0, th.q[S2], W1 * (th.q[S3] + th.q[S1])) + 0.5f * (th.t[S1] - th.t[S3]);
            const float c2 = th.c[S2];
            const float lap = 6.0f * fmaf(W0, th.sd[S2], W1 * ((th.sd[S3] + th.sd[S1]) + ((th.c[S3] - c2) + (th.c[S1] - c2))));
            phi_out[(size_t)(p - 2) * nxy + th.off1] = c2 - div + P.mob * lap;
        }
    }
}

template <bool WALL>
__global__ void __launch_bounds__(NTA, 3) ac_split_kernel(Grid G, Phys P, const float *__restrict__ phi_in,
                                                          const float *__restrict__ u_in, float *__restrict__ phi_out,
                                                          int ncols, int zlen, int units)
{
    __shared__ AcShared sh;
    AcThread th;
    const int tid = threadIdx.x;
    const int nx = G.nx, ny = G.ny, nz = G.nz, nxy = G.nxy;
    const int ncx = (nx + TX - 1) / TX;

    th.own = tid < N1;
    th.ry1 = tid / R1X;
    th.rx1 = tid - th.ry1 * R1X;
    th.core = th.own && th.ry1 >= 1 && th.ry1 <= TY && th.rx1 >= 1 && th.rx1 <= TX;
#pragma unroll
    for (int j = 0; j < 4; ++j) th.px[j] = th.py[j] = th.sd[j] = th.c[j] = th.q[j] = th.t[j] = 0.0f;

    for (int unit = blockIdx.x; unit < units; unit += gridDim.x) {
        const int col = unit % ncols;
        const int z0 = (unit / ncols) * zlen;
        const int zend = min(nz, z0 + zlen);
        const int x0 = (col % ncx) * TX, y0 = (col / ncx) * TY;
#pragma unroll
        for (int k = 0; k < KA2; ++k) {
            const int t = tid + k * NTA;
            const int ry = t / R2X, rx = t - ry * R2X;
            th.off2[k] = wrapc(y0 - 2 + ry, ny) * nx + wrapc(x0 - 2 + rx, nx);
        }
        th.off1 = wrapc(y0 - 1 + th.ry1, ny) * nx + wrapc(x0 - 1 + th.rx1, nx);
        th.store = th.core && x0 - 1 + th.rx1 < nx && y0 - 1 + th.ry1 < ny;
        {
            const int pl = zmap<WALL>(z0 - 2, nz) * nxy;
#pragma unroll
            for (int k = 0; k < KA2; ++k) th.nphi[k] = (tid + k * NTA < N2) ? __ldg(phi_in + pl + th.off2[k]) : 0.0f;
            th.nub[0] = th.nub[1] = th.nub[2] = 0.0f;
        }
        const int nsteps = (zend - z0) + 4;
        for (int s = 0; s < nsteps; s += 4) {
            ac_iteration<WALL, 0>(sh, th, G, P, phi_in, u_in, phi_out, z0, s, nsteps);
            if (s + 1 < nsteps) ac_iteration<WALL, 1>(sh, th, G, P, phi_in, u_in, phi_out, z0, s + 1, nsteps);
            if (s + 2 < nsteps) ac_iteration<WALL, 2>(sh, th, G, P, phi_in, u_in, phi_out, z0, s + 2, nsteps);
            if (s + 3 < nsteps) ac_iteration<WALL, 3>(sh, th, G, P, phi_in, u_in, phi_out, z0, s + 3, nsteps);
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
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L.blocks_per_sm, ac_split_kernel<WALL>, NTA, 0);
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
        ac_split_kernel<true><<<ctas, NTA, 0, s>>>(G, P, phi_in, u_in, phi_out, ncols, zlen, units);
    else
        ac_split_kernel<false><<<ctas, NTA, 0, s>>>(G, P, phi_in, u_in, phi_out, ncols, zlen, units);
    return cudaGetLastError();
}

cudaError_t launch_step_split(const Grid &G, const Phys &P, const StepArgs &a, int zchunks, cudaStream_t s)
{
    cudaError_t e = launch_ac_split(G, P, a.phi_in, a.u_in, a.phi_out, zchunks, s);
    if (e != cudaSuccess) return e;
    if (a.storage != 0)
        return launch_lbm16(G, P, a.storage, a.g_in, a.p_in, a.phi_out, a.u_in, a.g_out, a.p_out, a.u_out, s);
    return launch_lbm(G, P, 0, a.g_in, nullptr, a.phi_out, a.u_in, a.g_out, nullptr, a.u_out, s);
}

}  // namespace tslb

// Two-kernel step: a z-marching Allen–Cahn kernel writes phi^{n+1}; the one-thread-per-node
// lattice Boltzmann kernel (step_unfused.cu, or step_lbm16.cu for 16-bit populations) then
// streams the populations and also writes the Allen–Cahn flux of the new state.
//
// The flux W = ubar phi + kappa_AC max(phi (1 - phi), 0) n, n = grad phi / max(|grad phi|, eps),
// needs the gradient of phi and the velocity at the node: the lattice Boltzmann kernel of step n
// has both (grad phi^{n+1} for the surface-tension force, u^{n+1} from the collision), so it
// stores W^{n+1} next to ubar^{n+1}.  The Allen–Cahn update of step n+1,
//   phi^{n+2} = phi^{n+1} - div W^{n+1} + D lap phi^{n+1},
// is then a linear stencil of (phi, W): the same 20 bytes per node as reading phi and ubar, no
// normal or square root, and one barrier per plane.
//
// The 27-point stencils factorise over the D3Q27 weights (w = w1 w1 w1, w1(0) = 2/3,
// w1(+-1) = 1/6) into 3x3 partials of one z plane combined over three planes:
//   Q  = Px[W_x] + Py[W_y],  Px[V] = 2/3 (V(x+1,y) - V(x-1,y)) + 1/6 sum_{dy=+-1} (V(x+1,y+dy) - V(x-1,y+dy))
//   T  = sum_{dx,dy} w1(dx) w1(dy) W_z(x+dx, y+dy)
//   Sd = sum_{dx,dy} w1(dx) w1(dy) (phi(x+dx, y+dy) - phi(x, y)),  c = phi(x, y)
//   div W   = 1/2 [2/3 Q(z) + 1/6 (Q(z-1) + Q(z+1))] + 1/2 [T(z+1) - T(z-1)]
//   lap phi = 6 [2/3 Sd(z) + 1/6 (Sd(z-1) + Sd(z+1)) + 1/6 ((c(z-1) - c(z)) + (c(z+1) - c(z)))]
// (the paper's isotropic gradient and, reading R2, Laplacian).  A CTA of 256 threads owns a 32 x 8
// column tile, one column per thread, and marches a z chunk: per plane it stages (phi, W) of the
// 34 x 10 halo-1 plane as float4 in shared memory (double-buffered, so one barrier per plane),
// computes the partials of its column and keeps them in 3-slot register rings (march unrolled by
// 3).  The next plane is loaded into registers one iteration ahead.  At a wall the ghost plane is
// the mirror image with W_z negated (R13), so the wall flux vanishes.
#include "tslb_internal.h"

namespace tslb {
namespace {

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int NT = TX * TY;                     // 256 threads
constexpr int HX = TX + 2, HY = TY + 2, NH = HX * HY;   // halo-1 plane: 340 points
constexpr int KH = (NH + NT - 1) / NT;          // staged points per thread (2)

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

struct DivThread {
    int off[KH];              // in-plane offsets of the staged points
    int own;                  // in-plane offset of the own column
    bool store;               // own column inside the box
    float4 next[KH];          // (phi, W) of the next plane, loaded one iteration ahead
    float q[3], t[3], sd[3], c[3];   // rings, slot = plane index mod 3
};

// One plane of the march: iteration s (phase J = s mod 3) stages plane p = z0 - 1 + s and, from
// s = 2 on, writes phi^{n+1} of plane p - 1.
template <bool WALL, int J>
__device__ __forceinline__ void div_iteration(float4 (&sh)[2][NH], DivThread &th, const Grid &G, const Phys &P,
                                              const float *__restrict__ phi, const float *__restrict__ w,
                                              float *__restrict__ phi_out, int z0, int s, int nsteps)
{
    constexpr int S0 = J, S1 = (J + 2) % 3, S2 = (J + 1) % 3;   // slots of planes p, p-1, p-2
    const int tid = threadIdx.x;
    const size_t N = (size_t)G.N;
    const int p = z0 - 1 + s;
    float4 *buf = sh[s & 1];

#pragma unroll
    for (int k = 0; k < KH; ++k)
        if (tid + k * NT < NH) buf[tid + k * NT] = th.next[k];
    if (s + 1 < nsteps) {
        const int pl = zmap<WALL>(p + 1, G.nz) * G.nxy;
        const float sg = zsign<WALL>(p + 1, G.nz);
#pragma unroll
        for (int k = 0; k < KH; ++k)
            if (tid + k * NT < NH) {
                const int at = pl + th.off[k];
                th.next[k] = make_float4(__ldg(phi + at), __ldg(w + at), __ldg(w + N + at), sg * __ldg(w + 2 * N + at));
            }
    }
    __syncthreads();

    const int ty = tid / TX, tx = tid - ty * TX;
    const int ci = (ty + 1) * HX + tx + 1;
    const float4 m0 = buf[ci - HX - 1], m1 = buf[ci - HX], m2 = buf[ci - HX + 1];
    const float4 l0 = buf[ci - 1], cc = buf[ci], l2 = buf[ci + 1];
    const float4 q0 = buf[ci + HX - 1], q1 = buf[ci + HX], q2 = buf[ci + HX + 1];
    const float c = cc.x;
    th.c[S0] = c;
    th.sd[S0] = fmaf(WE, ((m1.x - c) + (q1.x - c)) + ((l0.x - c) + (l2.x - c)),
                     WC * (((m0.x - c) + (m2.x - c)) + ((q0.x - c) + (q2.x - c))));
    th.q[S0] = fmaf(W0, l2.y - l0.y, W1 * ((m2.y - m0.y) + (q2.y - q0.y)))
             + fmaf(W0, q1.z - m1.z, W1 * ((q0.z - m0.z) + (q2.z - m2.z)));
    th.t[S0] = fmaf(W0 * W0, cc.w, fmaf(WE, (l0.w + l2.w) + (m1.w + q1.w), WC * ((m0.w + m2.w) + (q0.w + q2.w))));

    if (s >= 2 && th.store) {
        const float c1 = th.c[S1];
        const float div = 0.5f * fmaf(W0, th.q[S1], W1 * (th.q[S2] + th.q[S0])) + 0.5f * (th.t[S0] - th.t[S2]);
        const float lap = 6.0f * fmaf(W0, th.sd[S1], W1 * ((th.sd[S2] + th.sd[S0]) + ((th.c[S2] - c1) + (th.c[S0] - c1))));
        phi_out[(size_t)(p - 1) * G.nxy + th.own] = c1 - div + P.mob * lap;
    }
}

template <bool WALL>
__global__ void __launch_bounds__(NT) ac_div_kernel(Grid G, Phys P, const float *__restrict__ phi,
                                                    const float *__restrict__ w, float *__restrict__ phi_out,
                                                    int ncols, int zlen, int units)
{
    __shared__ float4 sh[2][NH];
    DivThread th;
    const int tid = threadIdx.x;
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const int ncx = (nx + TX - 1) / TX;
    const size_t N = (size_t)G.N;
    const int ty = tid / TX, tx = tid - ty * TX;

    for (int unit = blockIdx.x; unit < units; unit += gridDim.x) {
        const int col = unit % ncols;
        const int z0 = (unit / ncols) * zlen;
        const int zend = min(nz, z0 + zlen);
        const int x0 = (col % ncx) * TX, y0 = (col / ncx) * TY;
#pragma unroll
        for (int k = 0; k < KH; ++k) {
            const int t = tid + k * NT;
            const int ry = t / HX, rx = t - ry * HX;
            th.off[k] = wrapc(y0 - 1 + ry, ny) * nx + wrapc(x0 - 1 + rx, nx);
        }
        th.own = min(y0 + ty, ny - 1) * nx + min(x0 + tx, nx - 1);
        th.store = x0 + tx < nx && y0 + ty < ny;
        {
            const int pl = zmap<WALL>(z0 - 1, nz) * G.nxy;
            const float sg = zsign<WALL>(z0 - 1, nz);
#pragma unroll
            for (int k = 0; k < KH; ++k) {
                th.next[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (tid + k * NT < NH) {
                    const int at = pl + th.off[k];
                    th.next[k] = make_float4(__ldg(phi + at), __ldg(w + at), __ldg(w + N + at),
                                             sg * __ldg(w + 2 * N + at));
                }
            }
        }
        const int nsteps = (zend - z0) + 2;
        for (int s = 0; s < nsteps; s += 3) {
            div_iteration<WALL, 0>(sh, th, G, P, phi, w, phi_out, z0, s, nsteps);
            if (s + 1 < nsteps) div_iteration<WALL, 1>(sh, th, G, P, phi, w, phi_out, z0, s + 1, nsteps);
            if (s + 2 < nsteps) div_iteration<WALL, 2>(sh, th, G, P, phi, w, phi_out, z0, s + 2, nsteps);
        }
        __syncthreads();   // the next unit restages both buffers
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
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L.blocks_per_sm, ac_div_kernel<WALL>, NT, 0);
}

}  // namespace

cudaError_t launch_ac_div(const Grid &G, const Phys &P, const float *phi_in, const float *w, float *phi_out,
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
    // default: one unit per resident CTA, chunks of at least 8 planes (2 halo planes per chunk)
    int m = zchunks;
    if (m <= 0) {
        m = slots / ncols;
        if (m > G.nz / 8) m = G.nz / 8;
        if (m < 1) m = 1;
    }
    if (m > G.nz) m = G.nz;
    const int zlen = (G.nz + m - 1) / m;
    m = (G.nz + zlen - 1) / zlen;
    const int units = ncols * m;
    const int rounds = (units + slots - 1) / slots;
    const int ctas = (units + rounds - 1) / rounds;
    if (G.wall)
        ac_div_kernel<true><<<ctas, NT, 0, s>>>(G, P, phi_in, w, phi_out, ncols, zlen, units);
    else
        ac_div_kernel<false><<<ctas, NT, 0, s>>>(G, P, phi_in, w, phi_out, ncols, zlen, units);
    return cudaGetLastError();
}

cudaError_t launch_step_split(const Grid &G, const Phys &P, const StepArgs &a, int zchunks, cudaStream_t s)
{
    cudaError_t e = launch_ac_div(G, P, a.phi_in, a.flux, a.phi_out, zchunks, s);
    if (e != cudaSuccess) return e;
    if (a.storage != 0)
        return launch_lbm16(G, P, a.storage, a.g_in, a.p_in, a.phi_out, a.u_in, a.g_out, a.p_out, a.u_out, a.flux, s);
    return launch_lbm(G, P, 0, a.g_in, nullptr, a.phi_out, a.u_in, a.g_out, nullptr, a.u_out, a.flux, s);
}

}  // namespace tslb

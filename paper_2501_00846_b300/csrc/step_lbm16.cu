// Lattice Boltzmann update with 16-bit population storage (BF16 / FP16 deviations h from the
// equilibrium; see the storage formats in tslb_device.cuh): the second kernel of the two-kernel
// step when the populations are 16-bit.
//
// Rebuilding a pulled population, g_i(x - c_i) = w_i (P + f^eq_i(0, ubar) / w_i + h_i), needs P
// and ubar of all 27 source nodes, and the force needs phi^{n+1} of the same 27 nodes.  Read from
// global memory one node per thread, those 135 scattered loads per node leave the kernel
// latency-bound.  Here a CTA owns a 32 x 4 x 2 tile of nodes (one per thread) and stages, for the
// tile plus a one-node halo (34 x 6 x 4 nodes), A = P - 1.5 |ubar|^2 and ubar as one float4,
// B = 3 - 4.5 |ubar|^2 and phi^{n+1} in shared memory with coalesced loads, so that
// P + f^eq_i(0, ubar) / w_i = A + 4.5 cu^2 + cu (4.5 cu^2 + B), cu = c_i . ubar, costs a few FMAs per
// direction.  The only per-direction global loads left are the 16-bit h_i, issued before the
// staging barrier so that their latency overlaps it.
//
// Halo nodes follow the same boundary rules as the one-node-per-thread kernel: periodic wrap in x
// and y; in z periodic or, with walls, the mirror image about the wall (phi ghosts).  At a wall
// the populations that would come from outside are bounced back from the node itself, so no
// (P, ubar) ghost value is ever used.
#include "tslb_internal.h"

namespace tslb {
namespace {

constexpr int TX = 32, TY = 4, TZ = 2;
constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
constexpr int HXY = HX * HY;
constexpr int HN = HXY * HZ;        // 816 staged nodes
constexpr int NT = TX * TY * TZ;    // 256 threads

// periodic image of a staged coordinate v in [-1, 2n); larger v (possible along x in boxes
// narrower than a tile) only feed threads outside the box and are clamped
__device__ __forceinline__ int wrap(int v, int n)
{
    v = v < 0 ? v + n : (v >= n ? v - n : v);
    return min(v, n - 1);
}

// global z of a staged plane: periodic wrap, or with walls the mirror image about the wall
// (planes beyond the mirror only feed threads outside the box)
__device__ __forceinline__ int staged_z(int z, const Grid &G)
{
    if (!G.wall) return wrap(z, G.nz);
    return z < 0 ? 0 : (z >= G.nz ? G.nz - 1 : z);
}

// The 27 pulled deviations h_i(x - c_i), and at a wall node (WN) h_{26-i}(x) for the directions
// that would come from outside.  Interior nodes take the branch-free form.
template <class S, bool WN>
__device__ __forceinline__ void pull_h(const typename S::T *__restrict__ hin, const Nbr &n, int k, size_t N,
                                       bool wlo, bool whi, float (&hv)[27])
{
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        bool bounce = false;
        if (WN && cz(i) == 1) bounce = wlo;
        if (WN && cz(i) == -1) bounce = whi;
        const int src = bounce ? k : n.zo[1 - cz(i)] + n.yo[1 - cy(i)] + n.xo[1 - cx(i)];
        hv[i] = S::to_f(hin[(size_t)(bounce ? 26 - i : i) * N + src]);
    }
}

// f_i = w_i (P + f^eq_i(0, ubar) / w_i + h_i) of the source node from the staged A, ubar, B
template <bool WN>
__device__ __forceinline__ void rebuild(const float4 *sq, const float *sb, int c0, bool wlo, bool whi,
                                        const float (&hv)[27], float (&f)[27])
{
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        bool bounce = false;
        if (WN && cz(i) == 1) bounce = wlo;
        if (WN && cz(i) == -1) bounce = whi;
        const int hs = bounce ? c0 : c0 - cz(i) * HXY - cy(i) * HX - cx(i);
        const float4 q = sq[hs];
        const float cu = cdot(i, q.y, q.z, q.w);
        f[i] = wgt(i) * (eq_from_ab(bounce ? -cu : cu, q.x, sb[hs]) + hv[i]);
    }
}

template <class S>
__global__ void __launch_bounds__(NT) lbm16_kernel(Grid G, Phys P, const typename S::T *__restrict__ hin,
                                                   const float *__restrict__ pin, const float *__restrict__ phi_new,
                                                   const float *__restrict__ ubar, typename S::T *__restrict__ hout,
                                                   float *__restrict__ pout, float *__restrict__ uout,
                                                   float *__restrict__ wout)
{
    __shared__ float4 sq[HN];    // (A = P - 1.5 |ubar|^2, ubar_x, ubar_y, ubar_z)
    __shared__ float sb[HN];     // B = 3 - 4.5 |ubar|^2
    __shared__ float sphi[HN];   // phi^{n+1}

    pdl_trigger();
    pdl_wait();
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = (tid / TX) % TY, tz = tid / (TX * TY);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
    const bool active = x < G.nx && y < G.ny && z < G.nz;
    const size_t N = (size_t)G.N;

    // own node (threads outside the box work on a clamped copy and store nothing)
    const int xc = min(x, G.nx - 1), yc = min(y, G.ny - 1), zc = min(z, G.nz - 1);
    const Nbr n = make_nbr(xc, yc, zc, G);
    const int k = n.zo[1] + n.yo[1] + xc;
    const bool wlo = G.wall && zc == 0;
    const bool whi = G.wall && zc == G.nz - 1;

    // the pulled deviations (a warp shares y and z, so the branch is uniform)
    const bool wall_node = wlo || whi;
    float hv[27];
    if (wall_node)
        pull_h<S, true>(hin, n, k, N, wlo, whi, hv);
    else
        pull_h<S, false>(hin, n, k, N, wlo, whi, hv);

    // stage (P, ubar) and phi^{n+1} of the tile and its halo
    for (int s = tid; s < HN; s += NT) {
        const int hx = s % HX, hy = (s / HX) % HY, hz = s / HXY;
        const int gk = (staged_z(z0 - 1 + hz, G) * G.ny + wrap(y0 - 1 + hy, G.ny)) * G.nx + wrap(x0 - 1 + hx, G.nx);
        const float vx = __ldg(ubar + gk), vy = __ldg(ubar + N + gk), vz = __ldg(ubar + 2 * N + gk);
        const float v2 = vx * vx + vy * vy + vz * vz;
        sq[s] = make_float4(__ldg(pin + gk) - 1.5f * v2, vx, vy, vz);
        sb[s] = 3.0f - 4.5f * v2;
        sphi[s] = __ldg(phi_new + gk);
    }
    __syncthreads();
    if (!active) return;

    const int c0 = ((tz + 1) * HY + (ty + 1)) * HX + (tx + 1);
    float f[27];
    if (wall_node)
        rebuild<true>(sq, sb, c0, wlo, whi, hv, f);
    else
        rebuild<false>(sq, sb, c0, wlo, whi, hv, f);

    float ps[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) ps[i] = sphi[c0 + cz(i) * HXY + cy(i) * HX + cx(i)];
    float gx, gy, gz, lap;
    grad_lap27(ps, gx, gy, gz, lap);

    const float4 own = sq[c0];
    float g[27], ux, uy, uz, pstar;
    collide_node<true>(f, ps[13], gx, gy, gz, lap, own.y, own.z, own.w, P, g, ux, uy, uz, &pstar);
    float sum = 0.0f;
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const typename S::T h = S::from_f(g[i]);
        hout[i * N + k] = h;
        sum = fmaf(wgt(i), S::to_f(h), sum);
    }
    pout[k] = pstar - sum;
    uout[k] = ux;
    uout[N + k] = uy;
    uout[2 * N + k] = uz;
    if (wout) {   // Allen–Cahn flux of the new state for the next step
        float wx, wy, wz;
        ac_flux(ps[13], gx, gy, gz, ux, uy, uz, P, wx, wy, wz);
        const unsigned long long pol = l2_keep_policy();
        st_keep(wout + k, wx, pol);
        st_keep(wout + N + k, wy, pol);
        st_keep(wout + 2 * N + k, wz, pol);
    }
}

}  // namespace

cudaError_t launch_lbm16(const Grid &G, const Phys &P, int storage, const void *h_in, const float *p_in,
                         const float *phi_new, const float *u_in, void *h_out, float *p_out, float *u_out,
                         float *w_out, cudaStream_t s)
{
    const dim3 grid((G.nx + TX - 1) / TX, (G.ny + TY - 1) / TY, (G.nz + TZ - 1) / TZ);
    if (storage == 1)
        return launch_pdl(lbm16_kernel<StoreB16>, grid, dim3(NT), 0, s, G, P, (const __nv_bfloat16 *)h_in, p_in, phi_new,
                          u_in, (__nv_bfloat16 *)h_out, p_out, u_out, w_out);
    if (storage == 2)
        return launch_pdl(lbm16_kernel<StoreF16>, grid, dim3(NT), 0, s, G, P, (const __half *)h_in, p_in, phi_new, u_in,
                          (__half *)h_out, p_out, u_out, w_out);
    return cudaErrorInvalidValue;
}

}  // namespace tslb

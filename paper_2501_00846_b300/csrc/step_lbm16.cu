// Lattice Boltzmann update with 16-bit population storage (BF16 / FP16 deviations h from the
// equilibrium; see the storage formats in tslb_device.cuh): the second kernel of the two-kernel
// step when the populations are 16-bit.
//
// Rebuilding a pulled population, g_i(x - c_i) = w_i (P + f^eq_i(0, ubar) / w_i + h_i), needs P
// and ubar of all 27 source nodes, and the force needs phi^{n+1} of the same 27 nodes.  A CTA of
// 256 threads owns a 32 x 8 column tile (one node per thread) and marches up a chunk of z planes.
// Every plane of (P, ubar) and of phi^{n+1}, with its one-node halo (34 x 10 nodes), is staged in
// shared memory exactly once, by cp.async, two planes ahead of the plane being completed; each
// thread converts the nodes it copied itself to A = P - 1.5 |ubar|^2, ubar and B = 3 - 4.5 |ubar|^2,
// so that P + f^eq_i(0, ubar) / w_i = A + 4.5 cu^2 + cu (4.5 cu^2 + B), cu = c_i . ubar, costs a
// few FMAs per direction, and one barrier per plane suffices.  The 27 16-bit h_i of the completed
// node are loaded from global memory at the start of its plane.  The moments of the streamed
// populations are summed per unit weight with the weights as FMA coefficients, the gradient and
// Laplacian of phi^{n+1} come from per-plane partial sums carried in registers, and the collision
// forms the new deviations directly.
//
// Boundaries as in the one-node-per-thread kernel: periodic wrap in x and y; in z periodic or,
// with walls, the populations that would come from outside are bounced back from the node itself
// (so no (P, ubar) ghost value is used), and phi^{n+1} beyond a wall is the mirror image of the
// wall plane.
#include "mom_tile.cuh"
#include "tslb_internal.h"

namespace tslb {
namespace {

using momt::MX;
using momt::MY;
using momt::PS;
using momt::SX;
using momt::SY;

constexpr int kThreads = MX * MY;   // 256: one thread per node of the column tile
constexpr int kQSlots = 4;          // converted (A, ubar), B of planes z-1 .. z+2
constexpr int kRawSlots = 2;        // raw (P, ubar) of the plane in flight and the one before
constexpr int kPhiSlots = 5;        // phi^{n+1} of planes z-1 .. z+3
constexpr size_t kSmem = (size_t)kQSlots * PS * (sizeof(float4) + sizeof(float)) + (size_t)kRawSlots * PS * sizeof(float4) +
                         (size_t)kPhiSlots * PS * sizeof(float);
constexpr int kStaged = (PS + kThreads - 1) / kThreads;   // staged nodes per thread (2)

__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <bool WALL, class S>
__global__ void __launch_bounds__(kThreads, 2)
    lbm16_kernel(Grid G, Phys P, const typename S::T *__restrict__ hin, const float *__restrict__ pin,
                 const float *__restrict__ phi_new, const float *__restrict__ ubar, typename S::T *__restrict__ hout,
                 float *__restrict__ pout, float *__restrict__ uout, float *__restrict__ wout, int tiles_x, int tiles_y,
                 int zlen)
{
    extern __shared__ float4 smem4[];
    float4 *sq = smem4;                                            // [kQSlots][PS] (A, ubar)
    float4 *raw = sq + kQSlots * PS;                               // [kRawSlots][PS] (P, ubar)
    float *sb = reinterpret_cast<float *>(raw + kRawSlots * PS);  // [kQSlots][PS] B
    float *sphi = sb + kQSlots * PS;                               // [kPhiSlots][PS] phi^{n+1}

    pdl_trigger();
    pdl_wait();
    int t = blockIdx.x;
    const int tx = t % tiles_x;
    t /= tiles_x;
    const int ty = t % tiles_y;
    const int z0 = (t / tiles_y) * zlen, z1 = min(G.nz, z0 + zlen);
    const int x0 = tx * MX, y0 = ty * MY;
    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    const size_t N = (size_t)G.N;
    const int nxy = G.nxy;

    // this thread's node (wrapped into the box on ragged tiles, where it is staged but not completed)
    const int x = (x0 + lane) % G.nx, y = (y0 + row) % G.ny;
    const bool active = x0 + lane < G.nx && y0 + row < G.ny;
    const int own = (row + 1) * SX + lane + 1;
    // in-plane offsets of the x and y neighbours (periodic)
    const int xo[3] = {x == 0 ? G.nx - 1 : x - 1, x, x == G.nx - 1 ? 0 : x + 1};
    const int yo[3] = {(y == 0 ? G.ny - 1 : y - 1) * G.nx, y * G.nx, (y == G.ny - 1 ? 0 : y + 1) * G.nx};

    // the staged nodes of this thread: position in the staged plane and offset in a box plane
    int spos[kStaged], sxy[kStaged];
#pragma unroll
    for (int j = 0; j < kStaged; ++j) {
        const int s = threadIdx.x + j * kThreads;
        spos[j] = s < PS ? s : -1;
        const int hy = s / SX, hx = s - (s / SX) * SX;
        sxy[j] = ((y0 - 1 + hy + G.ny) % G.ny) * G.nx + (x0 - 1 + hx + G.nx) % G.nx;
    }
    // a plane of the box for staged plane zs: (P, ubar) periodic, or clamped at walls (planes beyond a
    // wall are never read: those populations bounce back); phi^{n+1} mirrored at walls
    auto zwrap = [&](int zs) { return WALL ? min(max(zs, 0), G.nz - 1) : (zs + G.nz) % G.nz; };
    auto qslot = [&](int zs) { return (zs - z0 + 1) & (kQSlots - 1); };
    auto pslot = [&](int zs) { return (zs - z0 + 1) % kPhiSlots; };
    // cp.async of plane zs: raw (P, ubar) into raw slot zs & 1, phi^{n+1} into its ring slot
    auto stage = [&](int zs) {
        const int base = zwrap(zs) * nxy;
        float4 *r = raw + (zs & 1) * PS;
        float *ph = sphi + pslot(zs) * PS;
#pragma unroll
        for (int j = 0; j < kStaged; ++j) {
            if (spos[j] < 0) continue;
            const int k = base + sxy[j];
            float *d = reinterpret_cast<float *>(r + spos[j]);
            cp_async4(d, pin + k);
            cp_async4(d + 1, ubar + k);
            cp_async4(d + 2, ubar + N + k);
            cp_async4(d + 3, ubar + 2 * N + k);
            cp_async4(ph + spos[j], phi_new + k);
        }
    };
    // the nodes this thread staged for plane zs, converted to (A, ubar) and B
    auto convert = [&](int zs) {
        const float4 *r = raw + (zs & 1) * PS;
        float4 *q = sq + qslot(zs) * PS;
        float *b = sb + qslot(zs) * PS;
#pragma unroll
        for (int j = 0; j < kStaged; ++j) {
            if (spos[j] < 0) continue;
            const float4 v = r[spos[j]];
            const float v2 = v.y * v.y + v.z * v.z + v.w * v.w;
            q[spos[j]] = make_float4(v.x - 1.5f * v2, v.y, v.z, v.w);
            b[spos[j]] = 3.0f - 4.5f * v2;
        }
    };

    // prologue: planes z0-1, z0, z0+1 converted and their phi staged; plane z0+2 in flight
    stage(z0 - 1);
    stage(z0);
    cp_async_commit();
    cp_async_wait<0>();
    convert(z0 - 1);
    convert(z0);
    stage(z0 + 1);
    cp_async_commit();
    cp_async_wait<0>();
    convert(z0 + 1);
    stage(z0 + 2);
    cp_async_commit();
    __syncthreads();
    momt::PhiPartials pm = momt::phi_partials(sphi + pslot(z0 - 1) * PS, own);
    momt::PhiPartials p0 = momt::phi_partials(sphi + pslot(z0) * PS, own);

    for (int z = z0; z < z1; ++z) {
        const bool wlo = WALL && z == 0, whi = WALL && z == G.nz - 1;   // uniform across the CTA
        // the 27 deviations pulled into this node (bounced back from the node itself at a wall)
        float hv[27];
        if (active) {
            const int zo[3] = {zwrap(z - 1) * nxy, z * nxy, zwrap(z + 1) * nxy};
            const int k = zo[1] + yo[1] + x;
#pragma unroll
            for (int i = 0; i < 27; ++i) {
                const bool bounce = (cz(i) == 1 && wlo) || (cz(i) == -1 && whi);
                const int src = bounce ? k : zo[1 - cz(i)] + yo[1 - cy(i)] + xo[1 - cx(i)];
                hv[i] = S::to_f(hin[(size_t)(bounce ? 26 - i : i) * N + src]);
            }
        }
        // staging: plane z+3 in flight, plane z+2 (landed: this thread's own copies) converted
        if (z + 3 <= z1) stage(z + 3);
        cp_async_commit();
        cp_async_wait<1>();
        convert(z + 2);

        const momt::PhiPartials pp = momt::phi_partials(sphi + pslot(z + 1) * PS, own);
        if (active) {
            // rebuilt populations per unit weight, f_i / w_i = A + 4.5 cu^2 + cu (4.5 cu^2 + B) + h_i
            float gh[27];
            const float4 *qm = sq + qslot(z - 1) * PS, *q0 = sq + qslot(z) * PS, *qp = sq + qslot(z + 1) * PS;
            const float *bm = sb + qslot(z - 1) * PS, *b0 = sb + qslot(z) * PS, *bp = sb + qslot(z + 1) * PS;
#pragma unroll
            for (int i = 0; i < 27; ++i) {
                const bool bounce = (cz(i) == 1 && wlo) || (cz(i) == -1 && whi);
                const float4 *ql = bounce ? q0 : cz(i) == 1 ? qm : cz(i) == 0 ? q0 : qp;
                const float *bl = bounce ? b0 : cz(i) == 1 ? bm : cz(i) == 0 ? b0 : bp;
                const int pos = bounce ? own : own - cy(i) * SX - cx(i);
                const float4 q = ql[pos];
                const float cu = cdot(i, q.y, q.z, q.w);
                gh[i] = eq_from_ab(bounce ? -cu : cu, q.x, bl[pos]) + hv[i];
            }
            const float phi0 = sphi[pslot(z) * PS + own];
            float gx, gy, gz, lap;
            momt::phi_stencils(pm, p0, pp, phi0, gx, gy, gz, lap);
            const float4 ub = q0[own];
            const Collided c = collide_from_moments(raw_moments_hat(gh), phi0, gx, gy, gz, lap, ub.y, ub.z, ub.w, P);
            float h[27];
            populations_from<true>(c, h);
            const int k = z * nxy + y * G.nx + x;
            float sum = 0.0f;
#pragma unroll
            for (int i = 0; i < 27; ++i) {
                const typename S::T hq = S::from_f(h[i]);
                hout[(size_t)i * N + k] = hq;
                sum = fmaf(wgt(i), S::to_f(hq), sum);
            }
            pout[k] = c.ps - sum;
            uout[k] = c.ux;
            uout[N + k] = c.uy;
            uout[2 * N + k] = c.uz;
            if (wout) {   // Allen–Cahn flux of the new state for the next step
                float wx, wy, wz;
                ac_flux(phi0, gx, gy, gz, c.ux, c.uy, c.uz, P, wx, wy, wz);
                const unsigned long long pol = l2_keep_policy();
                st_keep(wout + k, wx, pol);
                st_keep(wout + N + k, wy, pol);
                st_keep(wout + 2 * N + k, wz, pol);
            }
        }
        pm = p0, p0 = pp;
        __syncthreads();   // plane z+2 converted and phi of z+2 landed for all; slots of z-1 free
    }
    cp_async_wait<0>();   // no copy of this block is still in flight when it returns
}

struct Launch16 {
    int sms = 0, blocks_per_sm = 0;
};

template <bool WALL, class S>
cudaError_t prepare16(Launch16 &L)
{
    int dev = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&L.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(lbm16_kernel<WALL, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem)) !=
        cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L.blocks_per_sm, lbm16_kernel<WALL, S>, kThreads, kSmem);
}

template <class S>
cudaError_t launch16_t(const Grid &G, const Phys &P, const void *h_in, const float *p_in, const float *phi_new,
                       const float *u_in, void *h_out, float *p_out, float *u_out, float *w_out, int zchunks,
                       cudaStream_t s)
{
    static Launch16 lw[2];
    Launch16 &L = lw[G.wall ? 1 : 0];
    if (L.sms == 0) {
        cudaError_t e = G.wall ? prepare16<true, S>(L) : prepare16<false, S>(L);
        if (e != cudaSuccess || L.blocks_per_sm < 1) {
            L.sms = 0;
            return e != cudaSuccess ? e : cudaErrorInvalidConfiguration;
        }
    }
    const int tiles_x = (G.nx + MX - 1) / MX, tiles_y = (G.ny + MY - 1) / MY;
    const long long ncols = (long long)tiles_x * tiles_y;
    int m = zchunks;
    if (m <= 0) {   // fewest waves x (planes per chunk + the two halo planes staged per chunk)
        const long long slots = (long long)L.sms * L.blocks_per_sm;
        double best = 0.0;
        m = 1;
        for (int c = 1; c <= G.nz; ++c) {
            const int zl = (G.nz + c - 1) / c;
            const int cc = (G.nz + zl - 1) / zl;
            const double waves = (double)((ncols * cc + slots - 1) / slots);
            const double cost = waves * (zl + 0.5);
            if (c == 1 || cost < best - 1e-9) best = cost, m = cc;
        }
    }
    if (m > G.nz) m = G.nz;
    const int zlen = (G.nz + m - 1) / m;
    m = (G.nz + zlen - 1) / zlen;
    const long long blocks = ncols * m;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    using T = typename S::T;
    return launch_pdl(G.wall ? lbm16_kernel<true, S> : lbm16_kernel<false, S>, dim3((unsigned)blocks), dim3(kThreads),
                      kSmem, s, G, P, (const T *)h_in, p_in, phi_new, u_in, (T *)h_out, p_out, u_out, w_out, tiles_x,
                      tiles_y, zlen);
}

}  // namespace

cudaError_t launch_lbm16(const Grid &G, const Phys &P, int storage, const void *h_in, const float *p_in,
                         const float *phi_new, const float *u_in, void *h_out, float *p_out, float *u_out,
                         float *w_out, int zchunks, cudaStream_t s)
{
    if (storage == 1)
        return launch16_t<StoreB16>(G, P, h_in, p_in, phi_new, u_in, h_out, p_out, u_out, w_out, zchunks, s);
    if (storage == 2)
        return launch16_t<StoreF16>(G, P, h_in, p_in, phi_new, u_in, h_out, p_out, u_out, w_out, zchunks, s);
    return cudaErrorInvalidValue;
}

}  // namespace tslb

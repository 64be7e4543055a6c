// Lattice Boltzmann update with moment-only storage (LBM_MOM): each node keeps the 13 numbers
// (p*, u, a, B) that fix its post-collision populations, and a puller rebuilds g_i(x - c_i) from
// the moments of x - c_i (mom_device.cuh).
//
// lbm_mom_kernel (the step's kernel): a CTA owns a 32 x 8 column tile and marches up a chunk of
// z planes.  For each plane it stages, ahead of the plane it completes, the populations leaving
// every node of the tile and its one-node halo: each thread loads its node's 13 moments
// (coalesced along x), evaluates the 27 populations once, and writes them per unit weight into
// shared memory, sorted by c_z into plane slots (c_z = +1 kept for three planes, 0 and -1 for two).
// Halo nodes evaluate only the 9 populations that point into the tile: warp 0 the row below
// (c_y = +1), warp 1 the row above (c_y = -1), warp 2 the left column (c_x = +1) and, from
// x-mirrored moments, the right column (c_x = -1).  The planes just below and above a z chunk
// keep only their c_z = +1 / -1 populations.  phi^{n+1} of the staged planes goes to a three-plane
// ring for the 27-point stencils.  Completing a plane reads the 27 streamed populations from
// the slots (halfway bounce-back at z walls: the node's own reversed population), runs the
// collision and stores the node's new moments, velocity and Allen–Cahn flux.
//
// lbm_mom_plain_kernel (path 1, the cross-check): one thread per node, each streamed population
// rebuilt from the source node's moments read from global memory.  The rebuilt populations are
// bit-identical to the tiled kernel's (explicitly rounded arithmetic); the collision may differ
// in the last bit where the compiler contracts products differently.
#include "mom_device.cuh"
#include "tslb_internal.h"

namespace tslb {
namespace {

constexpr int MX = 32, MY = 8;           // completed columns of a tile: one warp per row of 32
constexpr int SX = MX + 2, SY = MY + 2;  // staged plane including the one-node halo
constexpr int PS = SX * SY;              // floats of one staged plane (340)
constexpr int SLOT = 9 * PS;             // one plane's populations of one c_z, rows i % 9
constexpr int kMomThreads = MX * MY;
constexpr int kSlots = 7;
constexpr size_t kMomSmem = (size_t)(kSlots * SLOT + 3 * PS) * sizeof(float);

// Which populations a staged node keeps.  ZK: 0 all, +1 / -1 only those with c_z = ZK (the
// planes below / above a z chunk).  AX, SG: a halo node keeps only c_AX = SG (AX 0 = x, 1 = y,
// -1: no restriction).
__host__ __device__ constexpr bool mom_keep(int i, int AX, int SG, int ZK)
{
    return (ZK == 0 || cz(i) == ZK) && (AX < 0 || (AX == 0 ? cx(i) : cy(i)) == SG);
}

__device__ __forceinline__ float *slot_of(int i, float *rm, float *r0, float *rp)
{
    return cz(i) < 0 ? rm : cz(i) == 0 ? r0 : rp;
}

// Write the kept populations of one staged node, g_i / w_i, at row i % 9 of slot c_z(i); pos is
// the node's offset within a plane (the mirrored right column passes pos - 2 PS, which moves
// direction (+1, cy, cz) of the mirrored moments to the row of (-1, cy, cz)).
template <int AX, int SG, int ZK>
__device__ __forceinline__ void mom_emit(const Mom &m, float *rm, float *r0, float *rp, int pos)
{
    const MomPoly q = mom_poly(m);
#pragma unroll
    for (int i = 0; i < 13; ++i) {
        const bool ki = mom_keep(i, AX, SG, ZK), kj = mom_keep(26 - i, AX, SG, ZK);
        if (!ki && !kj) continue;
        float gp, gm;
        mom_pair(i, m, q, gp, gm);
        if (ki) slot_of(i, rm, r0, rp)[(i % 9) * PS + pos] = gp;
        if (kj) slot_of(26 - i, rm, r0, rp)[((26 - i) % 9) * PS + pos] = gm;
    }
    if (mom_keep(13, AX, SG, ZK)) r0[4 * PS + pos] = q.K0;
}

// Halo node of a thread (warps 0..2; see the file comment).
struct MomHalo {
    int xy;       // offset of the node within a z plane of the box
    int pos;      // staged position (plus -2 PS for the mirrored right column)
    int phi_pos;  // staged position
    bool on;
    bool mirror;
};

// Stage one plane: the thread's own node from its moments mo (loaded ahead), its halo node's
// from global memory (see mom_emit for ZK).
template <int ZK>
__device__ __forceinline__ void mom_stage_plane(const float *__restrict__ m_in, const float *__restrict__ u_in,
                                                size_t N, int plane, const Mom &mo, int own, int row, const MomHalo &h,
                                                float *rm, float *r0, float *rp)
{
    Mom mh;
    if (h.on) mh = mom_load(m_in, u_in, N, plane + h.xy);
    mom_emit<-1, 0, ZK>(mo, rm, r0, rp, own);
    if (h.on) {
        if (row == 0)
            mom_emit<1, 1, ZK>(mh, rm, r0, rp, h.pos);
        else if (row == 1)
            mom_emit<1, -1, ZK>(mh, rm, r0, rp, h.pos);
        else
            mom_emit<0, 1, ZK>(h.mirror ? mom_mirror_x(mh) : mh, rm, r0, rp, h.pos);
    }
}

__device__ __forceinline__ void mom_stage_phi(float own_phi, const float *__restrict__ phi, int plane,
                                              const MomHalo &h, int own, float *ring)
{
    ring[own] = own_phi;
    if (h.on) ring[h.phi_pos] = __ldg(phi + plane + h.xy);
}

template <bool WALL>
__global__ void __launch_bounds__(kMomThreads, 2)
    lbm_mom_kernel(Grid G, Phys P, const float *__restrict__ m_in, const float *__restrict__ u_in,
                   const float *__restrict__ phi_new, float *__restrict__ m_out, float *__restrict__ u_out,
                   float *__restrict__ w_out, int tiles_x, int tiles_y, int zlen)
{
    extern __shared__ float sm[];
    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    int b = blockIdx.x;
    const int tx = b % tiles_x;
    b /= tiles_x;
    const int ty = b % tiles_y;
    const int z0 = (b / tiles_y) * zlen;
    const int z1 = min(z0 + zlen, G.nz);
    const int x0 = tx * MX, y0 = ty * MY;
    const size_t N = (size_t)G.N;
    const int nxy = G.nxy;

    // this thread's node (wrapped into the box on ragged tiles, where it is staged but not completed)
    const int x = (x0 + lane) % G.nx, y = (y0 + row) % G.ny;
    const bool active = x0 + lane < G.nx && y0 + row < G.ny;
    const int own_xy = y * G.nx + x;
    const int own = (row + 1) * SX + lane + 1;

    MomHalo h{0, 0, 0, false, false};
    if (row < 2) {
        const int hy = row == 0 ? (y0 - 1 + G.ny) % G.ny : (y0 + MY) % G.ny;
        h.xy = hy * G.nx + x;
        h.pos = h.phi_pos = (row == 0 ? 0 : SY - 1) * SX + lane + 1;
        h.on = true;
    } else if (row == 2 && lane < 2 * SY) {
        h.mirror = lane >= SY;
        const int sy = h.mirror ? lane - SY : lane;
        const int hx = h.mirror ? (x0 + MX) % G.nx : (x0 - 1 + G.nx) % G.nx;
        h.xy = ((y0 - 1 + sy + G.ny) % G.ny) * G.nx + hx;
        h.phi_pos = sy * SX + (h.mirror ? SX - 1 : 0);
        h.pos = h.mirror ? h.phi_pos - 2 * PS : h.phi_pos;
        h.on = true;
    }

    float *rp_prev = sm, *rp_cur = sm + SLOT, *rp_next = sm + 2 * SLOT;
    float *r0_cur = sm + 3 * SLOT, *r0_next = sm + 4 * SLOT;
    float *rm_cur = sm + 5 * SLOT, *rm_next = sm + 6 * SLOT;
    float *ph_prev = sm + kSlots * SLOT, *ph_cur = ph_prev + PS, *ph_next = ph_cur + PS;

    // planes staged around the chunk (-1: none, beyond a wall); phi^{n+1} beyond a wall is the
    // mirror image of the wall plane
    auto moment_plane = [&](int zs) { return zs < 0 ? (WALL ? -1 : G.nz - 1) : zs >= G.nz ? (WALL ? -1 : 0) : zs; };
    auto phi_plane = [&](int zs) { return zs < 0 ? (WALL ? 0 : G.nz - 1) : zs >= G.nz ? (WALL ? G.nz - 1 : 0) : zs; };

    // prologue: the c_z = +1 populations of the plane below the chunk, the chunk's first plane,
    // phi^{n+1} of planes z0-1 and z0; the own moments and phi of plane z0+1 are loaded ahead
    Mom mo;
    const int zb = moment_plane(z0 - 1);
    if (zb >= 0) {
        mo = mom_load(m_in, u_in, N, zb * nxy + own_xy);
        mom_stage_plane<1>(m_in, u_in, N, zb * nxy, mo, own, row, h, rm_next, r0_next, rp_prev);
    }
    mo = mom_load(m_in, u_in, N, z0 * nxy + own_xy);
    mom_stage_plane<0>(m_in, u_in, N, z0 * nxy, mo, own, row, h, rm_cur, r0_cur, rp_cur);
    float ubx = mo.ux, uby = mo.uy, ubz = mo.uz;
    mom_stage_phi(__ldg(phi_new + phi_plane(z0 - 1) * nxy + own_xy), phi_new, phi_plane(z0 - 1) * nxy, h, own,
                  ph_prev);
    mom_stage_phi(__ldg(phi_new + z0 * nxy + own_xy), phi_new, z0 * nxy, h, own, ph_cur);
    int zn = moment_plane(z0 + 1);
    if (zn >= 0) mo = mom_load(m_in, u_in, N, zn * nxy + own_xy);
    float phn = __ldg(phi_new + phi_plane(z0 + 1) * nxy + own_xy);

    for (int z = z0; z < z1; ++z) {
        // stage plane z+1 (all of it inside the chunk, its c_z = -1 populations above the
        // chunk, nothing beyond a wall) and its phi^{n+1}
        const float nbx = mo.ux, nby = mo.uy, nbz = mo.uz;
        if (z + 1 < z1)
            mom_stage_plane<0>(m_in, u_in, N, zn * nxy, mo, own, row, h, rm_next, r0_next, rp_next);
        else if (zn >= 0)
            mom_stage_plane<-1>(m_in, u_in, N, zn * nxy, mo, own, row, h, rm_next, r0_next, rp_next);
        mom_stage_phi(phn, phi_new, phi_plane(z + 1) * nxy, h, own, ph_next);
        __syncthreads();

        // own moments and phi of plane z+2, in flight during the collision
        if (z + 1 < z1) {
            zn = moment_plane(z + 2);
            if (zn >= 0) mo = mom_load(m_in, u_in, N, zn * nxy + own_xy);
            phn = __ldg(phi_new + phi_plane(z + 2) * nxy + own_xy);
        }

        if (active) {
            const bool wlo = WALL && z == 0, whi = WALL && z == G.nz - 1;
            float f[27];
#pragma unroll
            for (int i = 0; i < 27; ++i) {
                const int nb = own - cy(i) * SX - cx(i);
                const float *src;
                if (cz(i) == 1)
                    src = wlo ? rm_cur + ((26 - i) % 9) * PS + own : rp_prev + (i % 9) * PS + nb;
                else if (cz(i) == 0)
                    src = r0_cur + (i % 9) * PS + nb;
                else
                    src = whi ? rp_cur + ((26 - i) % 9) * PS + own : rm_next + (i % 9) * PS + nb;
                f[i] = __fmul_rn(wgt(i), *src);   // not fused into the moment sums: same bits as the plain kernel
            }
            float psi[27];
#pragma unroll
            for (int i = 0; i < 27; ++i) {
                const float *pr = cz(i) < 0 ? ph_prev : cz(i) == 0 ? ph_cur : ph_next;
                psi[i] = pr[own + cy(i) * SX + cx(i)];
            }
            mom_collide_store(f, psi, ubx, uby, ubz, P, m_out, u_out, w_out, N, z * nxy + own_xy);
        }
        __syncthreads();

        float *t = rp_prev;
        rp_prev = rp_cur, rp_cur = rp_next, rp_next = t;
        t = r0_cur, r0_cur = r0_next, r0_next = t;
        t = rm_cur, rm_cur = rm_next, rm_next = t;
        t = ph_prev, ph_prev = ph_cur, ph_cur = ph_next, ph_next = t;
        ubx = nbx, uby = nby, ubz = nbz;
    }
}

template <bool WALL>
__global__ void __launch_bounds__(128)
    lbm_mom_plain_kernel(Grid G, Phys P, const float *__restrict__ m_in, const float *__restrict__ u_in,
                         const float *__restrict__ phi_new, float *__restrict__ m_out, float *__restrict__ u_out,
                         float *__restrict__ w_out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= G.nx) return;
    const Nbr n = make_nbr(x, y, z, G);
    const int k = n.zo[1] + n.yo[1] + x;
    const size_t N = (size_t)G.N;
    const bool wlo = WALL && z == 0, whi = WALL && z == G.nz - 1;
    float f[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const bool bounce = (cz(i) == 1 && wlo) || (cz(i) == -1 && whi);
        const int src = bounce ? k : n.zo[1 - cz(i)] + n.yo[1 - cy(i)] + n.xo[1 - cx(i)];
        const Mom m = mom_load(m_in, u_in, N, src);
        const MomPoly q = mom_poly(m);
        const float gi = bounce ? mom_one(26 - i, m, q) : mom_one(i, m, q);
        f[i] = __fmul_rn(wgt(i), gi);
    }
    float psi[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) psi[i] = __ldg(phi_new + nidx(n, i));
    mom_collide_store(f, psi, __ldg(u_in + k), __ldg(u_in + N + k), __ldg(u_in + 2 * N + k), P, m_out, u_out, w_out,
                      N, k);
}

// Equilibrium start: p* = pstar (or 0), a = 0, B = 0 (u is already in place).
__global__ void mom_init_kernel(Grid G, const float *__restrict__ pstar, float *__restrict__ m)
{
    const size_t N = (size_t)G.N;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) {
        m[k] = pstar ? pstar[k] : 0.0f;
#pragma unroll
        for (int q = 1; q < kMomArrays; ++q) m[q * N + k] = 0.0f;
    }
}

// g[(i - i0) N + node] = w_i (g_i / w_i)(moments of the node) for i in [i0, i0 + ni)
__global__ void mom_expand_kernel(Grid G, const float *__restrict__ m, const float *__restrict__ u, int i0, int ni,
                                  float *__restrict__ g)
{
    const size_t N = (size_t)G.N;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) {
        const Mom mm = mom_load(m, u, N, (int)k);
        const MomPoly q = mom_poly(mm);
#pragma unroll
        for (int i = 0; i < 27; ++i)
            if (i >= i0 && i < i0 + ni) g[(i - i0) * N + k] = wgt(i) * mom_one(i, mm, q);
    }
}

// acc += (sum g, sum g c (3), sum g c c (xx yy zz xy xz yz)) over directions [i0, i0 + ni) of
// g[(i - i0) N + node]; the sums of one launch are formed in FP64.
__global__ void mom_project_kernel(Grid G, const float *__restrict__ g, int i0, int ni, float *__restrict__ acc)
{
    const size_t N = (size_t)G.N;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) {
        double s[kMomArrays] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            if (i < i0 || i >= i0 + ni) continue;
            const double v = g[(i - i0) * N + k];
            s[0] += v;
            s[1] += cx(i) * v, s[2] += cy(i) * v, s[3] += cz(i) * v;
            s[4] += cx(i) * cx(i) * v, s[5] += cy(i) * cy(i) * v, s[6] += cz(i) * cz(i) * v;
            s[7] += cx(i) * cy(i) * v, s[8] += cx(i) * cz(i) * v, s[9] += cy(i) * cz(i) * v;
        }
#pragma unroll
        for (int q = 0; q < kMomArrays; ++q) acc[q * N + k] += (float)s[q];
    }
}

// Moment set from the population moments (in place): p* = sum g, a = 2 (sum g c - u),
// B = T - 4.5 u u - 4.5 sym(u a) with T = 4.5 (sum g c c - p* I / 3).
__global__ void mom_finish_kernel(Grid G, const float *__restrict__ u, float *__restrict__ m)
{
    const size_t N = (size_t)G.N;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) {
        const double ps = m[k];
        const double ux = u[k], uy = u[N + k], uz = u[2 * N + k];
        const double ax = 2.0 * (m[N + k] - ux), ay = 2.0 * (m[2 * N + k] - uy), az = 2.0 * (m[3 * N + k] - uz);
        const double p3 = ps / 3.0;
        m[N + k] = (float)ax;
        m[2 * N + k] = (float)ay;
        m[3 * N + k] = (float)az;
        m[4 * N + k] = (float)(4.5 * (m[4 * N + k] - p3) - 4.5 * ux * ux - 4.5 * ux * ax);
        m[5 * N + k] = (float)(4.5 * (m[5 * N + k] - p3) - 4.5 * uy * uy - 4.5 * uy * ay);
        m[6 * N + k] = (float)(4.5 * (m[6 * N + k] - p3) - 4.5 * uz * uz - 4.5 * uz * az);
        m[7 * N + k] = (float)(4.5 * m[7 * N + k] - 4.5 * ux * uy - 2.25 * (ux * ay + uy * ax));
        m[8 * N + k] = (float)(4.5 * m[8 * N + k] - 4.5 * ux * uz - 2.25 * (ux * az + uz * ax));
        m[9 * N + k] = (float)(4.5 * m[9 * N + k] - 4.5 * uy * uz - 2.25 * (uy * az + uz * ay));
    }
}

struct LaunchMom {
    int sms = 0;
    int blocks_per_sm = 0;
};

template <bool WALL>
cudaError_t prepare_mom(LaunchMom &L)
{
    int dev = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&L.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(lbm_mom_kernel<WALL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMomSmem)) !=
        cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L.blocks_per_sm, lbm_mom_kernel<WALL>, kMomThreads,
                                                         kMomSmem);
}

int grid_stride_blocks(const Grid &G)
{
    const long long b = ((long long)G.N + 255) / 256;
    return (int)(b < 148 * 16 ? b : 148 * 16);
}

}  // namespace

cudaError_t launch_mom(const Grid &G, const Phys &P, const float *m_in, const float *u_in, const float *phi_new,
                       float *m_out, float *u_out, float *w_out, int zchunks, cudaStream_t s)
{
    static LaunchMom lw[2];
    LaunchMom &L = lw[G.wall ? 1 : 0];
    if (L.sms == 0) {
        cudaError_t e = G.wall ? prepare_mom<true>(L) : prepare_mom<false>(L);
        if (e != cudaSuccess) {
            L.sms = 0;
            return e;
        }
        if (L.blocks_per_sm < 1) {
            L.sms = 0;
            return cudaErrorInvalidConfiguration;
        }
    }
    const int tiles_x = (G.nx + MX - 1) / MX, tiles_y = (G.ny + MY - 1) / MY;
    const long long ncols = (long long)tiles_x * tiles_y;
    int m = zchunks;
    if (m <= 0) {   // fewest waves x (planes per chunk + the two partial halo planes)
        const long long slots = (long long)L.sms * L.blocks_per_sm;
        double best = 0.0;
        m = 1;
        for (int c = 1; c <= G.nz; ++c) {
            const int zl = (G.nz + c - 1) / c;
            const int cc = (G.nz + zl - 1) / zl;
            const double waves = (double)((ncols * cc + slots - 1) / slots);
            const double cost = waves * (zl + 0.7);
            if (c == 1 || cost < best - 1e-9) best = cost, m = cc;
        }
    }
    if (m > G.nz) m = G.nz;
    const int zlen = (G.nz + m - 1) / m;
    m = (G.nz + zlen - 1) / zlen;
    const long long blocks = ncols * m;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (G.wall)
        lbm_mom_kernel<true><<<(unsigned)blocks, kMomThreads, kMomSmem, s>>>(G, P, m_in, u_in, phi_new, m_out, u_out,
                                                                             w_out, tiles_x, tiles_y, zlen);
    else
        lbm_mom_kernel<false><<<(unsigned)blocks, kMomThreads, kMomSmem, s>>>(G, P, m_in, u_in, phi_new, m_out, u_out,
                                                                              w_out, tiles_x, tiles_y, zlen);
    return cudaGetLastError();
}

cudaError_t launch_mom_plain(const Grid &G, const Phys &P, const float *m_in, const float *u_in, const float *phi_new,
                             float *m_out, float *u_out, float *w_out, cudaStream_t s)
{
    const dim3 grid((G.nx + 127) / 128, G.ny, G.nz);
    if (G.wall)
        lbm_mom_plain_kernel<true><<<grid, 128, 0, s>>>(G, P, m_in, u_in, phi_new, m_out, u_out, w_out);
    else
        lbm_mom_plain_kernel<false><<<grid, 128, 0, s>>>(G, P, m_in, u_in, phi_new, m_out, u_out, w_out);
    return cudaGetLastError();
}

cudaError_t launch_mom_init(const Grid &G, const float *pstar, float *m, cudaStream_t s)
{
    mom_init_kernel<<<grid_stride_blocks(G), 256, 0, s>>>(G, pstar, m);
    return cudaGetLastError();
}

cudaError_t launch_mom_expand(const Grid &G, const float *m, const float *u, int i0, int ni, float *g, cudaStream_t s)
{
    if (i0 < 0 || ni < 1 || i0 + ni > 27) return cudaErrorInvalidValue;
    mom_expand_kernel<<<grid_stride_blocks(G), 256, 0, s>>>(G, m, u, i0, ni, g);
    return cudaGetLastError();
}

cudaError_t launch_mom_project(const Grid &G, const float *g, int i0, int ni, float *acc, cudaStream_t s)
{
    if (i0 < 0 || ni < 1 || i0 + ni > 27) return cudaErrorInvalidValue;
    mom_project_kernel<<<grid_stride_blocks(G), 256, 0, s>>>(G, g, i0, ni, acc);
    return cudaGetLastError();
}

cudaError_t launch_mom_finish(const Grid &G, const float *u, float *m, cudaStream_t s)
{
    mom_finish_kernel<<<grid_stride_blocks(G), 256, 0, s>>>(G, u, m);
    return cudaGetLastError();
}

}  // namespace tslb

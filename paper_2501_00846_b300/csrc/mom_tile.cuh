// The tiled moment-storage lattice Boltzmann update of one column tile of one box, shared by the
// one-box kernel (step_mom.cu) and the batched ensemble (ensemble.cu).
//
// A CTA owns a 32 x 8 column tile and marches up a chunk of z planes.  For each plane it stages,
// ahead of the plane it completes, the populations leaving every node of the tile and its
// one-node halo: each thread evaluates its node's 27 populations once from the node's 13 moments
// and writes them per unit weight into shared memory, sorted by c_z into plane slots (c_z = +1
// kept for three planes, 0 and -1 for two).  Halo nodes evaluate only the 9 populations that
// point into the tile, spread over all 8 warps by c_z (rows below / above keep c_y = +1 / -1, the
// columns c_x = +1 / -1, the right column from x-mirrored moments); the planes just below and above
// a z chunk keep only their c_z = +1 / -1 populations.  Completing a plane reads the 27 streamed
// populations from the slots (halfway bounce-back at z walls: the node's own reversed
// population), sums the moments with the weights as FMA coefficients, takes the gradient and
// Laplacian of phi^{n+1} from per-plane partial sums carried in registers, runs the collision and
// stores the node's new moments, velocity and Allen–Cahn flux.  While a plane collides, the own
// node's moments and phi for the plane after next are loaded into registers and the halo's are
// copied into shared memory with cp.async.
#pragma once

#include <stdint.h>

#include "mom_device.cuh"

namespace tslb {
namespace momt {


constexpr int MX = 32, MY = 8;           // completed columns of a tile: one warp per row of 32
constexpr int SX = MX + 2, SY = MY + 2;  // staged plane including the one-node halo
constexpr int PS = SX * SY;              // floats of one staged plane (340)
constexpr int SLOT = 9 * PS;             // one plane's populations of one c_z, rows i % 9
constexpr int kMomThreads = MX * MY;
constexpr int kSlots = 7;
constexpr int kHalo = 2 * MX + 2 * SY;   // halo nodes of a staged plane (84)
constexpr int kPhiRing = 4;              // phi^{n+1} planes z-1, z, z+1 and the one in flight
constexpr size_t kMomSmem = (size_t)(kSlots * SLOT + 13 * kHalo + kPhiRing * PS) * sizeof(float);

// Which populations a staged node keeps.  ZF: 2 all, -1 / 0 / +1 only those with c_z = ZF.
// AX, SG: a halo node keeps only c_AX = SG (AX 0 = x, 1 = y; -1: no restriction).
__host__ __device__ constexpr bool mom_keep(int i, int AX, int SG, int ZF)
{
    return (ZF == 2 || cz(i) == ZF) && (AX < 0 || (AX == 0 ? cx(i) : cy(i)) == SG);
}

__device__ __forceinline__ float *slot_of(int i, float *rm, float *r0, float *rp)
{
    return cz(i) < 0 ? rm : cz(i) == 0 ? r0 : rp;
}

// Write the kept populations of one staged node, g_i / w_i, at row i % 9 of slot c_z(i); pos is
// the node's offset within a plane (the mirrored right column passes pos - 2 PS, which moves
// direction (+1, cy, cz) of the mirrored moments to the row of (-1, cy, cz)).
template <int AX, int SG, int ZF>
__device__ __forceinline__ void mom_emit(const Mom &m, float *rm, float *r0, float *rp, int pos)
{
    const MomPoly q = mom_poly(m);
#pragma unroll
    for (int i = 0; i < 13; ++i) {
        const bool ki = mom_keep(i, AX, SG, ZF), kj = mom_keep(26 - i, AX, SG, ZF);
        if (!ki && !kj) continue;
        float gp, gm;
        mom_pair(i, m, q, gp, gm);
        if (ki) slot_of(i, rm, r0, rp)[(i % 9) * PS + pos] = gp;
        if (kj) slot_of(26 - i, rm, r0, rp)[((26 - i) % 9) * PS + pos] = gm;
    }
    if (mom_keep(13, AX, SG, ZF)) r0[4 * PS + pos] = q.K0;
}

__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// The 84 halo nodes of a staged plane, numbered hn: 0..31 the row below the tile (keeps c_y = +1),
// 32..63 the row above (c_y = -1), 64..73 the left column over staged rows 0..9 (c_x = +1),
// 74..83 the right column (c_x = -1, evaluated from x-mirrored moments).  Thread hn fetches
// halo node hn's moments (into hb[q * kHalo + hn], q as in mom_lds) and phi^{n+1}.
struct HaloFetch {
    int xy;       // offset of the node within a z plane of the box
    int phi_pos;  // staged position
    bool on;
};

// Copies of one halo node's moments into hb[q * kHalo + hn]: q = 0 p*, 1..9 the deviation moments
// (FP32 storage: one value each; 16-bit storage: the node's 5 packed words in q = 1..5),
// 10..12 u.
template <class S>
__device__ __forceinline__ void halo_fetch(const float *__restrict__ m_in, const float *__restrict__ u_in, size_t N,
                                           int plane, const HaloFetch &h, float *hb)
{
    if (!h.on) return;
    const int k = plane + h.xy;
    cp_async4(hb + threadIdx.x, m_in + k);
    const float *d = m_in + N;
    if constexpr (sizeof(typename S::T) == 4) {
#pragma unroll
        for (int q = 0; q < 9; ++q) cp_async4(hb + (1 + q) * kHalo + threadIdx.x, d + q * N + k);
    } else {
#pragma unroll
        for (int j = 0; j < kMomWords; ++j)
            cp_async4(hb + (1 + j) * kHalo + threadIdx.x, d + (size_t)kMomWords * k + j);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) cp_async4(hb + (kMomArrays + a) * kHalo + threadIdx.x, u_in + a * N + k);
}

__device__ __forceinline__ void halo_fetch_phi(const float *__restrict__ phi, int plane, const HaloFetch &h,
                                               float *ring)
{
    if (h.on) cp_async4(ring + h.phi_pos, phi + plane + h.xy);
}

template <class S>
__device__ __forceinline__ Mom halo_lds(const float *hb, int hn)
{
    Mom r;
    r.ps = hb[hn];
    if constexpr (sizeof(typename S::T) == 4) {
        r.ax = hb[kHalo + hn];
        r.ay = hb[2 * kHalo + hn];
        r.az = hb[3 * kHalo + hn];
        r.bxx = hb[4 * kHalo + hn];
        r.byy = hb[5 * kHalo + hn];
        r.bzz = hb[6 * kHalo + hn];
        r.bxy = hb[7 * kHalo + hn];
        r.bxz = hb[8 * kHalo + hn];
        r.byz = hb[9 * kHalo + hn];
    } else {
        uint32_t w[kMomWords];
#pragma unroll
        for (int j = 0; j < kMomWords; ++j) w[j] = __float_as_uint(hb[(1 + j) * kHalo + hn]);
        mom_unpack<S>(w, r);
    }
    r.ux = hb[10 * kHalo + hn];
    r.uy = hb[11 * kHalo + hn];
    r.uz = hb[12 * kHalo + hn];
    return r;
}

// Halo populations of one staged plane, spread over the 8 warps by c_z: warps 0..2 the row below
// (c_z = -1, 0, +1), warps 3..5 the row above, warp 6 the columns' c_z = -1 and +1, warp 7 their
// c_z = 0 (3 populations per halo node and item).  PZ: the plane's filter (2 all, +-1 the planes
// below / above a z chunk).
template <int AX, int SG, int CZ, int PZ>
__device__ __forceinline__ void halo_item(const Mom &m, float *rm, float *r0, float *rp, int pos)
{
    if (PZ == 2 || PZ == CZ) mom_emit<AX, SG, CZ>(m, rm, r0, rp, pos);
}

template <class S, int PZ>
__device__ __forceinline__ void mom_stage_halo(const float *hb, int row, int lane, float *rm, float *r0, float *rp)
{
    if (row < 3) {
        if (PZ != 2 && PZ != row - 1) return;
        const Mom m = halo_lds<S>(hb, lane);
        const int pos = lane + 1;
        if (row == 0) halo_item<1, 1, -1, PZ>(m, rm, r0, rp, pos);
        else if (row == 1) halo_item<1, 1, 0, PZ>(m, rm, r0, rp, pos);
        else halo_item<1, 1, 1, PZ>(m, rm, r0, rp, pos);
    } else if (row < 6) {
        if (PZ != 2 && PZ != row - 4) return;
        const Mom m = halo_lds<S>(hb, MX + lane);
        const int pos = (SY - 1) * SX + lane + 1;
        if (row == 3) halo_item<1, -1, -1, PZ>(m, rm, r0, rp, pos);
        else if (row == 4) halo_item<1, -1, 0, PZ>(m, rm, r0, rp, pos);
        else halo_item<1, -1, 1, PZ>(m, rm, r0, rp, pos);
    } else if (lane < 2 * SY) {
        if (row == 6 && PZ == 0) return;
        if (row == 7 && PZ != 2 && PZ != 0) return;
        const bool mirror = lane >= SY;
        Mom m = halo_lds<S>(hb, 2 * MX + lane);
        if (mirror) m = mom_mirror_x(m);
        const int pos = (mirror ? lane - SY : lane) * SX + (mirror ? SX - 1 - 2 * PS : 0);
        if (row == 6) {
            halo_item<0, 1, -1, PZ>(m, rm, r0, rp, pos);
            halo_item<0, 1, 1, PZ>(m, rm, r0, rp, pos);
        } else {
            halo_item<0, 1, 0, PZ>(m, rm, r0, rp, pos);
        }
    }
}

// In-plane partial sums of the 27-point stencils at staged position pos of a phi^{n+1} plane pl:
//   A = S_x S_y phi,   X = S_y (phi(x+1) - phi(x-1)),   Y = S_x (phi(y+1) - phi(y-1)),
// with S f = f(-1) / 6 + 2 f(0) / 3 + f(+1) / 6 along one axis (the D3Q27 weights factor as
// w(c) = w1(cx) w1(cy) w1(cz), w1(0) = 2/3, w1(+-1) = 1/6).
struct PhiPartials {
    float A, X, Y;
};

__device__ __forceinline__ float smooth3(float m, float c, float p)
{
    return fmaf(1.0f / 6.0f, m + p, (2.0f / 3.0f) * c);
}

__device__ __forceinline__ PhiPartials phi_partials(const float *pl, int pos)
{
    const float a0 = pl[pos - SX - 1], a1 = pl[pos - SX], a2 = pl[pos - SX + 1];
    const float b0 = pl[pos - 1], b1 = pl[pos], b2 = pl[pos + 1];
    const float c0 = pl[pos + SX - 1], c1 = pl[pos + SX], c2 = pl[pos + SX + 1];
    const float s0 = smooth3(a0, b0, c0), s1 = smooth3(a1, b1, c1), s2 = smooth3(a2, b2, c2);
    PhiPartials r;
    r.A = smooth3(s0, s1, s2);
    r.X = s2 - s0;
    r.Y = smooth3(c0 - a0, c1 - a1, c2 - a2);
    return r;
}

// Gradient and Laplacian of phi^{n+1} at a node from the partial sums of planes z-1, z, z+1
// (the 27-point formulas of the paper's finite differences, evaluated separably):
//   grad_x = 3 sum w c_x phi = S_z X / 2,  grad_y = S_z Y / 2,  grad_z = (A(z+1) - A(z-1)) / 2,
//   lap = 6 (sum w phi - phi0) = (A(z-1) - phi0) + (A(z+1) - phi0) + 4 (A(z) - phi0).
__device__ __forceinline__ void phi_stencils(const PhiPartials &m, const PhiPartials &c, const PhiPartials &p,
                                             float phi0, float &gx, float &gy, float &gz, float &lap)
{
    gx = fmaf(1.0f / 12.0f, m.X + p.X, (1.0f / 3.0f) * c.X);
    gy = fmaf(1.0f / 12.0f, m.Y + p.Y, (1.0f / 3.0f) * c.Y);
    gz = 0.5f * (p.A - m.A);
    lap = fmaf(4.0f, c.A - phi0, (m.A - phi0) + (p.A - phi0));
}

// The tiled lattice Boltzmann update of the column tile with corner (x0, y0), planes [z0, z1), of
// one box (the body of lbm_mom_kernel and of the ensemble's moment kernel; one CTA of kMomThreads
// threads with kMomSmem bytes of dynamic shared memory).
template <bool WALL, class S>
__device__ __forceinline__ void mom_tile_task(const Grid &G, const Phys &P, const float *__restrict__ m_in,
                                              const float *__restrict__ u_in, const float *__restrict__ phi_new,
                                              float *__restrict__ m_out, float *__restrict__ u_out,
                                              float *__restrict__ w_out, int x0, int y0, int z0, int z1)
{
    extern __shared__ float sm[];
    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    const size_t N = (size_t)G.N;
    const int nxy = G.nxy;

    // this thread's node (wrapped into the box on ragged tiles, where it is staged but not completed)
    const int x = (x0 + lane) % G.nx, y = (y0 + row) % G.ny;
    const bool active = x0 + lane < G.nx && y0 + row < G.ny;
    const int own_xy = y * G.nx + x;
    const int own = (row + 1) * SX + lane + 1;

    HaloFetch h{0, 0, threadIdx.x < kHalo};
    if (threadIdx.x < MX) {
        h.xy = ((y0 - 1 + G.ny) % G.ny) * G.nx + (x0 + threadIdx.x) % G.nx;
        h.phi_pos = threadIdx.x + 1;
    } else if (threadIdx.x < 2 * MX) {
        const int c = threadIdx.x - MX;
        h.xy = ((y0 + MY) % G.ny) * G.nx + (x0 + c) % G.nx;
        h.phi_pos = (SY - 1) * SX + c + 1;
    } else if (threadIdx.x < kHalo) {
        const int c = threadIdx.x - 2 * MX;
        const bool right = c >= SY;
        const int sy = right ? c - SY : c;
        const int hx = right ? (x0 + MX) % G.nx : (x0 - 1 + G.nx) % G.nx;
        h.xy = ((y0 - 1 + sy + G.ny) % G.ny) * G.nx + hx;
        h.phi_pos = sy * SX + (right ? SX - 1 : 0);
    }

    float *rp_prev = sm, *rp_cur = sm + SLOT, *rp_next = sm + 2 * SLOT;
    float *r0_cur = sm + 3 * SLOT, *r0_next = sm + 4 * SLOT;
    float *rm_cur = sm + 5 * SLOT, *rm_next = sm + 6 * SLOT;
    float *const hb = sm + kSlots * SLOT;
    float *const ring = hb + 13 * kHalo;
    auto ring_of = [&](int zs) { return ring + ((zs - z0 + 1) & 3) * PS; };   // phi^{n+1} of plane zs

    // planes staged around the chunk (-1: none, beyond a wall); phi^{n+1} beyond a wall is the
    // mirror image of the wall plane
    auto moment_plane = [&](int zs) { return zs < 0 ? (WALL ? -1 : G.nz - 1) : zs >= G.nz ? (WALL ? -1 : 0) : zs; };
    auto phi_plane = [&](int zs) { return zs < 0 ? (WALL ? 0 : G.nz - 1) : zs >= G.nz ? (WALL ? G.nz - 1 : 0) : zs; };

    // prologue: the c_z = +1 populations of the plane below the chunk, then the chunk's first
    // plane with phi^{n+1} of planes z0-1 and z0; the own node's moments and phi of plane z0+1
    // are loaded into registers, its halo's into shared memory
    Mom mo;
    const int zb = moment_plane(z0 - 1);
    if (zb >= 0) {
        mo = mom_load<S>(m_in, u_in, N, zb * nxy + own_xy);
        halo_fetch<S>(m_in, u_in, N, zb * nxy, h, hb);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        mom_emit<-1, 0, 1>(mo, rm_next, r0_next, rp_prev, own);
        mom_stage_halo<S, 1>(hb, row, lane, rm_next, r0_next, rp_prev);
        __syncthreads();
    }
    mo = mom_load<S>(m_in, u_in, N, z0 * nxy + own_xy);
    halo_fetch<S>(m_in, u_in, N, z0 * nxy, h, hb);
    ring_of(z0 - 1)[own] = __ldg(phi_new + phi_plane(z0 - 1) * nxy + own_xy);
    halo_fetch_phi(phi_new, phi_plane(z0 - 1) * nxy, h, ring_of(z0 - 1));
    ring_of(z0)[own] = __ldg(phi_new + z0 * nxy + own_xy);
    halo_fetch_phi(phi_new, z0 * nxy, h, ring_of(z0));
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    PhiPartials pm = phi_partials(ring_of(z0 - 1), own), p0 = phi_partials(ring_of(z0), own);
    mom_emit<-1, 0, 2>(mo, rm_cur, r0_cur, rp_cur, own);
    mom_stage_halo<S, 2>(hb, row, lane, rm_cur, r0_cur, rp_cur);
    float ubx = mo.ux, uby = mo.uy, ubz = mo.uz;
    __syncthreads();
    int zn = moment_plane(z0 + 1);
    if (zn >= 0) {
        mo = mom_load<S>(m_in, u_in, N, zn * nxy + own_xy);
        halo_fetch<S>(m_in, u_in, N, zn * nxy, h, hb);
    }
    float phn = __ldg(phi_new + phi_plane(z0 + 1) * nxy + own_xy);
    halo_fetch_phi(phi_new, phi_plane(z0 + 1) * nxy, h, ring_of(z0 + 1));
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();

    for (int z = z0; z < z1; ++z) {
        // stage plane z+1 (all of it inside the chunk, its c_z = -1 populations above the
        // chunk, nothing beyond a wall) and its phi^{n+1}
        const float nbx = mo.ux, nby = mo.uy, nbz = mo.uz;
        if (z + 1 < z1) {
            mom_emit<-1, 0, 2>(mo, rm_next, r0_next, rp_next, own);
            mom_stage_halo<S, 2>(hb, row, lane, rm_next, r0_next, rp_next);
        } else if (zn >= 0) {
            mom_emit<-1, 0, -1>(mo, rm_next, r0_next, rp_next, own);
            mom_stage_halo<S, -1>(hb, row, lane, rm_next, r0_next, rp_next);
        }
        ring_of(z + 1)[own] = phn;
        __syncthreads();

        // plane z+2 in flight during the collision: own moments and phi into registers, the
        // halo's into shared memory
        if (z + 1 < z1) {
            zn = moment_plane(z + 2);
            if (zn >= 0) {
                mo = mom_load<S>(m_in, u_in, N, zn * nxy + own_xy);
                halo_fetch<S>(m_in, u_in, N, zn * nxy, h, hb);
            }
            phn = __ldg(phi_new + phi_plane(z + 2) * nxy + own_xy);
            halo_fetch_phi(phi_new, phi_plane(z + 2) * nxy, h, ring_of(z + 2));
        }
        cp_async_commit();

        const PhiPartials pp = phi_partials(ring_of(z + 1), own);
        if (active) {
            float gh[27];
            if (WALL && (z == 0 || z == G.nz - 1)) {   // a wall plane (uniform across the CTA)
                const bool wlo = z == 0, whi = z == G.nz - 1;
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
                    gh[i] = *src;
                }
            } else {
#pragma unroll
                for (int i = 0; i < 27; ++i) {
                    const float *sl = cz(i) == 1 ? rp_prev : cz(i) == 0 ? r0_cur : rm_next;
                    gh[i] = sl[(i % 9) * PS + own - cy(i) * SX - cx(i)];
                }
            }
            const float phi0 = ring_of(z)[own];
            float gx, gy, gz, lap;
            phi_stencils(pm, p0, pp, phi0, gx, gy, gz, lap);
            mom_finish<S>(raw_moments_hat(gh), phi0, gx, gy, gz, lap, ubx, uby, ubz, P, m_out, u_out, w_out, N,
                          z * nxy + own_xy);
        }
        pm = p0, p0 = pp;
        cp_async_wait_all();
        __syncthreads();

        float *t = rp_prev;
        rp_prev = rp_cur, rp_cur = rp_next, rp_next = t;
        t = r0_cur, r0_cur = r0_next, r0_next = t;
        t = rm_cur, rm_cur = rm_next, rm_next = t;
        ubx = nbx, uby = nby, ubz = nbz;
    }
}


}  // namespace momt
}  // namespace tslb

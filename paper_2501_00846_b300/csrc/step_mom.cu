// Lattice Boltzmann update with moment-only storage (LBM_MOM, LBM_MOM_BF16, LBM_MOM_FP16): each node
// keeps the 13 numbers (p*, u, a, B) that fix its post-collision populations, and a puller
// rebuilds g_i(x - c_i) from the moments of x - c_i (mom_device.cuh).
//
// lbm_mom_kernel (the step's kernel): one CTA per (32 x 8 column tile, z chunk), running
// mom_tile_task (mom_tile.cuh).
//
// lbm_mom_plain_kernel (path 1, the cross-check): one thread per node, each streamed population
// rebuilt from the source node's moments read from global memory.  The rebuilt populations are
// bit-identical to the tiled kernel's (explicitly rounded arithmetic); the collision may differ
// in the last bit where the compiler contracts products differently.
#include "mom_device.cuh"
#include "mom_tile.cuh"
#include "tslb_internal.h"

namespace tslb {
namespace {

using namespace momt;

template <bool WALL, class S>
__global__ void __launch_bounds__(momt::kMomThreads, 2)
    lbm_mom_kernel(Grid G, Phys P, const float *__restrict__ m_in, const float *__restrict__ u_in,
                   const float *__restrict__ phi_new, float *__restrict__ m_out, float *__restrict__ u_out,
                   float *__restrict__ w_out, int tiles_x, int tiles_y, int zlen)
{
    pdl_trigger();
    pdl_wait();
    int b = blockIdx.x;
    const int tx = b % tiles_x;
    b /= tiles_x;
    const int ty = b % tiles_y;
    const int z0 = (b / tiles_y) * zlen;
    momt::mom_tile_task<WALL, S>(G, P, m_in, u_in, phi_new, m_out, u_out, w_out, tx * momt::MX, ty * momt::MY, z0,
                                 min(z0 + zlen, G.nz));
}

template <bool WALL, class S>
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
    float gh[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const bool bounce = (cz(i) == 1 && wlo) || (cz(i) == -1 && whi);
        const int src = bounce ? k : n.zo[1 - cz(i)] + n.yo[1 - cy(i)] + n.xo[1 - cx(i)];
        const Mom m = mom_load<S>(m_in, u_in, N, src);
        const MomPoly q = mom_poly(m);
        gh[i] = bounce ? mom_one(26 - i, m, q) : mom_one(i, m, q);
    }
    float psi[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) psi[i] = __ldg(phi_new + nidx(n, i));
    float gx, gy, gz, lap;
    grad_lap27(psi, gx, gy, gz, lap);
    mom_finish<S>(raw_moments_hat(gh), psi[13], gx, gy, gz, lap, __ldg(u_in + k), __ldg(u_in + N + k),
                  __ldg(u_in + 2 * N + k), P, m_out, u_out, w_out, N, k);
}

// Equilibrium start: p* = pstar (or 0), a = 0, B = 0 (u is already in place).
template <class S>
__global__ void mom_init_kernel(Grid G, const float *__restrict__ pstar, float *__restrict__ m)
{
    const size_t N = (size_t)G.N;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) {
        Mom r;
        r.ps = pstar ? pstar[k] : 0.0f;
        r.ax = r.ay = r.az = r.bxx = r.byy = r.bzz = r.bxy = r.bxz = r.byz = 0.0f;
        mom_store_dev<S>(r, m, N, (int)k);
    }
}

// g[(i - i0) N + node] = w_i (g_i / w_i)(moments of the node) for i in [i0, i0 + ni)
template <class S>
__global__ void mom_expand_kernel(Grid G, const float *__restrict__ m, const float *__restrict__ u, int i0, int ni,
                                  float *__restrict__ g)
{
    const size_t N = (size_t)G.N;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) {
        const Mom mm = mom_load<S>(m, u, N, (int)k);
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

// Moment set from the population moments acc (FP32, 10 arrays: sum g, sum g c, sum g c c):
// p* = sum g, a = 2 (sum g c - u), B = T - 4.5 u u - 4.5 sym(u a) with T = 4.5 (sum g c c - p* I / 3),
// written to m in the storage S (m may be acc itself for FP32 storage).
template <class S>
__global__ void mom_finish_kernel(Grid G, const float *__restrict__ u, const float *acc, float *m)
{
    const size_t N = (size_t)G.N;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) {
        const double ps = acc[k];
        const double ux = u[k], uy = u[N + k], uz = u[2 * N + k];
        const double ax = 2.0 * (acc[N + k] - ux), ay = 2.0 * (acc[2 * N + k] - uy), az = 2.0 * (acc[3 * N + k] - uz);
        const double p3 = ps / 3.0;
        const double pxx = acc[4 * N + k], pyy = acc[5 * N + k], pzz = acc[6 * N + k];
        const double pxy = acc[7 * N + k], pxz = acc[8 * N + k], pyz = acc[9 * N + k];
        Mom r;
        r.ps = (float)ps;
        r.ux = (float)ux, r.uy = (float)uy, r.uz = (float)uz;
        r.ax = (float)ax, r.ay = (float)ay, r.az = (float)az;
        r.bxx = (float)(4.5 * (pxx - p3) - 4.5 * ux * ux - 4.5 * ux * ax);
        r.byy = (float)(4.5 * (pyy - p3) - 4.5 * uy * uy - 4.5 * uy * ay);
        r.bzz = (float)(4.5 * (pzz - p3) - 4.5 * uz * uz - 4.5 * uz * az);
        r.bxy = (float)(4.5 * pxy - 4.5 * ux * uy - 2.25 * (ux * ay + uy * ax));
        r.bxz = (float)(4.5 * pxz - 4.5 * ux * uz - 2.25 * (ux * az + uz * ax));
        r.byz = (float)(4.5 * pyz - 4.5 * uy * uz - 2.25 * (uy * az + uz * ay));
        mom_store_dev<S>(r, m, N, (int)k);
    }
}

struct LaunchMom {
    int sms = 0;
    int blocks_per_sm = 0;
};

template <bool WALL, class S>
cudaError_t prepare_mom(LaunchMom &L)
{
    int dev = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&L.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(lbm_mom_kernel<WALL, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kMomSmem)) != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L.blocks_per_sm, lbm_mom_kernel<WALL, S>, kMomThreads,
                                                         kMomSmem);
}

int grid_stride_blocks(const Grid &G)
{
    const long long b = ((long long)G.N + 255) / 256;
    return (int)(b < 148 * 16 ? b : 148 * 16);
}

template <class S>
cudaError_t launch_mom_t(const Grid &G, const Phys &P, const float *m_in, const float *u_in, const float *phi_new,
                         float *m_out, float *u_out, float *w_out, int zchunks, cudaStream_t s)
{
    static LaunchMom lw[2];
    LaunchMom &L = lw[G.wall ? 1 : 0];
    if (L.sms == 0) {
        cudaError_t e = G.wall ? prepare_mom<true, S>(L) : prepare_mom<false, S>(L);
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
    return launch_pdl(G.wall ? lbm_mom_kernel<true, S> : lbm_mom_kernel<false, S>, dim3((unsigned)blocks),
                      dim3(kMomThreads), kMomSmem, s, G, P, m_in, u_in, phi_new, m_out, u_out, w_out, tiles_x, tiles_y,
                      zlen);
}

template <class S>
cudaError_t launch_mom_plain_t(const Grid &G, const Phys &P, const float *m_in, const float *u_in,
                               const float *phi_new, float *m_out, float *u_out, float *w_out, cudaStream_t s)
{
    const dim3 grid((G.nx + 127) / 128, G.ny, G.nz);
    if (G.wall)
        lbm_mom_plain_kernel<true, S><<<grid, 128, 0, s>>>(G, P, m_in, u_in, phi_new, m_out, u_out, w_out);
    else
        lbm_mom_plain_kernel<false, S><<<grid, 128, 0, s>>>(G, P, m_in, u_in, phi_new, m_out, u_out, w_out);
    return cudaGetLastError();
}

}  // namespace

// storage: LBM_MOM (FP32 deviations), LBM_MOM_BF16, LBM_MOM_FP16
#define TSLB_MOM_DISPATCH(storage, ...)                                                            \
    switch (storage) {                                                                             \
    case LBM_MOM: { using S = StoreF32; __VA_ARGS__; }                                                  \
    case LBM_MOM_BF16: { using S = StoreB16; __VA_ARGS__; }                                             \
    case LBM_MOM_FP16: { using S = StoreF16; __VA_ARGS__; }                                             \
    default: return cudaErrorInvalidValue;                                                         \
    }

size_t mom_state_bytes(int storage, size_t N)
{
    // p* in FP32, then 9 FP32 arrays or 5 packed 32-bit words per node
    return N * sizeof(float) + (storage == LBM_MOM ? 9 : kMomWords) * N * sizeof(uint32_t);
}

cudaError_t launch_mom(const Grid &G, const Phys &P, int storage, const float *m_in, const float *u_in,
                       const float *phi_new, float *m_out, float *u_out, float *w_out, int zchunks, cudaStream_t s)
{
    TSLB_MOM_DISPATCH(storage, return launch_mom_t<S>(G, P, m_in, u_in, phi_new, m_out, u_out, w_out, zchunks, s))
}

cudaError_t launch_mom_plain(const Grid &G, const Phys &P, int storage, const float *m_in, const float *u_in,
                             const float *phi_new, float *m_out, float *u_out, float *w_out, cudaStream_t s)
{
    TSLB_MOM_DISPATCH(storage, return launch_mom_plain_t<S>(G, P, m_in, u_in, phi_new, m_out, u_out, w_out, s))
}

cudaError_t launch_mom_init(const Grid &G, int storage, const float *pstar, float *m, cudaStream_t s)
{
    TSLB_MOM_DISPATCH(storage, mom_init_kernel<S><<<grid_stride_blocks(G), 256, 0, s>>>(G, pstar, m);
                      return cudaGetLastError())
}

cudaError_t launch_mom_expand(const Grid &G, int storage, const float *m, const float *u, int i0, int ni, float *g,
                              cudaStream_t s)
{
    if (i0 < 0 || ni < 1 || i0 + ni > 27) return cudaErrorInvalidValue;
    TSLB_MOM_DISPATCH(storage, mom_expand_kernel<S><<<grid_stride_blocks(G), 256, 0, s>>>(G, m, u, i0, ni, g);
                      return cudaGetLastError())
}

cudaError_t launch_mom_project(const Grid &G, const float *g, int i0, int ni, float *acc, cudaStream_t s)
{
    if (i0 < 0 || ni < 1 || i0 + ni > 27) return cudaErrorInvalidValue;
    mom_project_kernel<<<grid_stride_blocks(G), 256, 0, s>>>(G, g, i0, ni, acc);
    return cudaGetLastError();
}

cudaError_t launch_mom_finish(const Grid &G, int storage, const float *u, const float *acc, float *m, cudaStream_t s)
{
    TSLB_MOM_DISPATCH(storage, mom_finish_kernel<S><<<grid_stride_blocks(G), 256, 0, s>>>(G, u, acc, m);
                      return cudaGetLastError())
}

}  // namespace tslb

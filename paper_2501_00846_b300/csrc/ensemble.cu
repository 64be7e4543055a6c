// Batched ensemble of independent boxes (lbm_ens_* in include/lbm.h).
//
// Small boxes (32^3 ... 96^3) cannot fill 148 SMs one at a time, and a launch per box and kernel
// costs more than the box's work.  Here the boxes' states are packed one after the other into
// shared arrays (box b: g[27][N_b], phi[N_b], ubar[3][N_b], W[3][N_b] at node offset off_b), and a
// step is two launches for the whole ensemble:
//   1. the Allen–Cahn kernel over a task list that concatenates every box's (column tile, z chunk)
//      tasks; a warp finds its box by binary search over the boxes' first task and runs
//      ac_div_task (ac_div.cuh) on it;
//   2. the lattice Boltzmann kernel over a block list that concatenates every box's node blocks;
//      a block finds its box the same way and each thread runs lbm_node (lbm_node.cuh) on its node.
//      With moment storage (LBM_MOM, LBM_MOM_BF16, LBM_MOM_FP16) the list concatenates every box's
//      (32 x 8 column tile, z chunk) tasks instead and a CTA runs mom_tile_task (mom_tile.cuh).
// The device functions are the ones the one-box kernels use, so every box evolves bit-identically
// to lbm_step on its own context.  Steps are replayed from a CUDA graph captured once per tuning
// (graph_steps steps, an even number so the ping-pong buffers return to their start).
//
// Tuning (lbm_ens_autotune): threads per lattice Boltzmann block, output rows per Allen–Cahn warp
// and planes per Allen–Cahn task, timed with CUDA events on launches that do not advance the
// state (the kernels read the current buffers and write the idle ones; the flux W that the
// lattice Boltzmann kernel overwrites is recomputed from the current state afterwards, with the
// same arithmetic).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <type_traits>
#include <vector>

#include <cuda_runtime.h>

#include "ac_div.cuh"
#include "lbm.h"
#include "lbm_node.cuh"
#include "mom_tile.cuh"
#include "tslb_internal.h"

namespace tslb {
namespace {

struct EnsBox {
    Grid G;
    Phys P;
    long long off;   // first node of the box in the packed arrays
    int blk0;        // first block of the box in the lattice Boltzmann grid
    int task0;       // first task of the box in the Allen–Cahn task list
    int ncols;       // Allen–Cahn column tiles of the box
    int zlen;        // planes per Allen–Cahn task of the box
    int mtask0;      // first task of the box in the moment-storage lattice Boltzmann task list
    int mzlen;       // planes per moment-storage task of the box
    float rnxy, rnx; // 1 / (nx ny) and 1 / nx, rounded: node coordinates without integer division
};

// q = n / d (integer division) for 0 <= n < 2^24 and d >= 1, with rd = 1/d rounded to FP32.  n is
// exact in FP32 and the product is within one unit of n / d (relative error below 2^-23 on a
// quotient below 2^23, or exact for d = 1), so its truncation is off by at most one either way,
// which the integer remainder corrects.
__device__ __forceinline__ int div_u24(int n, int d, float rd)
{
    int q = __float2int_rz(__fmul_rn(__int2float_rn(n), rd));
    const int r = n - q * d;
    if (r < 0)
        --q;
    else if (r >= d)
        ++q;
    return q;
}

// Coordinates of node `node` (flat index x + nx (y + ny z)) of box B.
__device__ __forceinline__ void box_coords(const EnsBox &B, int node, int &x, int &y, int &z)
{
    if (B.G.N < (1 << 24)) {   // uniform across a block: every thread of a block is in one box
        z = div_u24(node, B.G.nxy, B.rnxy);
        const int rem = node - z * B.G.nxy;
        y = div_u24(rem, B.G.nx, B.rnx);
        x = rem - y * B.G.nx;
    } else {
        z = node / B.G.nxy;
        const int rem = node - z * B.G.nxy;
        y = rem / B.G.nx;
        x = rem - y * B.G.nx;
    }
}

// Planes per moment-storage task (2 partial halo planes each): the longest of whole boxes, 128, 64
// and 32 planes that still gives every resident CTA kEnsMomTasksPerCta tasks (fewer, longer tasks
// re-stage fewer halo planes; measured on the 256-droplet ensemble with BF16 moments: whole boxes
// 4.06 ms per step, 32-plane tasks 4.17 ms, 16-plane tasks 4.40 ms).
constexpr int kEnsMomZlens[4] = {1 << 30, 128, 64, 32};
constexpr int kEnsMomTasksPerCta = 2;
constexpr int kEnsMomCtasPerSm = 2;   // the tiled kernel's 95 KB of shared memory

constexpr int AC_WPB = 4;   // warps per Allen–Cahn CTA

// The last box whose first Allen–Cahn task (FIELD 1) or first moment-storage task (FIELD 2) is
// <= v; box 0 starts at 0.  (The lattice Boltzmann node blocks find their box in a table.)
template <int FIELD>
__device__ __forceinline__ int find_box(const EnsBox *__restrict__ boxes, int nb, int v)
{
    static_assert(FIELD == 1 || FIELD == 2, "FIELD selects the task list");
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int start = FIELD == 1 ? boxes[mid].task0 : boxes[mid].mtask0;
        if (start <= v)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// blk_box[k]: the box of lattice Boltzmann block k (one table read instead of a search)
__global__ void __launch_bounds__(256, 3) ens_lbm_kernel(const EnsBox *__restrict__ boxes, const int *__restrict__ blk_box,
                                                      const float *__restrict__ g_in, const float *__restrict__ phi_new,
                                                      const float *__restrict__ u_in, float *__restrict__ g_out,
                                                      float *__restrict__ u_out, float *__restrict__ w_out)
{
    const int b = blk_box[blockIdx.x];
    const Grid G = boxes[b].G;
    const int node = (blockIdx.x - boxes[b].blk0) * blockDim.x + threadIdx.x;
    if (node >= G.N) return;
    const Phys P = boxes[b].P;
    const size_t o = (size_t)boxes[b].off;
    int x, y, z;
    box_coords(boxes[b], node, x, y, z);
    lbm_node<StoreF32>(G, P, g_in + 27 * o, nullptr, phi_new + o, u_in + 3 * o, g_out + 27 * o, nullptr,
                       u_out + 3 * o, w_out + 3 * o, x, y, z);
}

// Moment storage: one CTA per (box, column tile, z chunk) task; fpn = floats per node of a box's
// moment state (box b's state starts at float fpn * off_b).
template <class S>
__global__ void __launch_bounds__(momt::kMomThreads, 2)
    ens_mom_kernel(const EnsBox *__restrict__ boxes, int nb, int fpn, const float *__restrict__ m_in,
                   const float *__restrict__ phi_new, const float *__restrict__ u_in, float *__restrict__ m_out,
                   float *__restrict__ u_out, float *__restrict__ w_out)
{
    const int b = find_box<2>(boxes, nb, blockIdx.x);
    const Grid G = boxes[b].G;
    const Phys P = boxes[b].P;
    const size_t o = (size_t)boxes[b].off;
    const int tiles_x = (G.nx + momt::MX - 1) / momt::MX, tiles_y = (G.ny + momt::MY - 1) / momt::MY;
    int t = blockIdx.x - boxes[b].mtask0;
    const int tx = t % tiles_x;
    t /= tiles_x;
    const int ty = t % tiles_y;
    const int z0 = (t / tiles_y) * boxes[b].mzlen;
    const int z1 = min(z0 + boxes[b].mzlen, G.nz);
    const float *mi = m_in + (size_t)fpn * o;
    float *mo = m_out + (size_t)fpn * o;
    if (G.wall)   // uniform across the CTA
        momt::mom_tile_task<true, S>(G, P, mi, u_in + 3 * o, phi_new + o, mo, u_out + 3 * o, w_out + 3 * o,
                                     tx * momt::MX, ty * momt::MY, z0, z1);
    else
        momt::mom_tile_task<false, S>(G, P, mi, u_in + 3 * o, phi_new + o, mo, u_out + 3 * o, w_out + 3 * o,
                                      tx * momt::MX, ty * momt::MY, z0, z1);
}

template <int RY>
__global__ void __launch_bounds__(AC_WPB * 32) ens_ac_kernel(const EnsBox *__restrict__ boxes, int nb, int ntasks,
                                                             const float *__restrict__ phi,
                                                             const float *__restrict__ w, float *__restrict__ phi_out)
{
    const int nwarps = gridDim.x * AC_WPB;
    for (int task = blockIdx.x * AC_WPB + (threadIdx.x >> 5); task < ntasks; task += nwarps) {
        const int b = find_box<1>(boxes, nb, task);
        const Grid G = boxes[b].G;
        const Phys P = boxes[b].P;
        const size_t o = (size_t)boxes[b].off;
        const int local = task - boxes[b].task0;
        const int ncols = boxes[b].ncols, zlen = boxes[b].zlen;
        const int col = local % ncols;
        const int z0 = (local / ncols) * zlen;
        const int zend = min(G.nz, z0 + zlen);
        if (G.wall)   // uniform across the warp
            ac_div_task<true, RY>(G, P, phi + o, w + 3 * o, phi_out + o, col, z0, zend);
        else
            ac_div_task<false, RY>(G, P, phi + o, w + 3 * o, phi_out + o, col, z0, zend);
    }
}

// ---- one persistent launch per step ------------------------------------------------------------
//
// The persistent form runs a whole step in one cooperative launch of as many 256-thread CTAs as
// fit on the GPU at once: every warp takes Allen–Cahn tasks from the concatenated task list, the
// CTAs meet at a grid barrier, then every CTA takes lattice Boltzmann work (node blocks of
// lbm_block threads, or the moment storages' column-tile tasks).  The barrier is a counter and a
// generation word in global memory; a CTA's wait for the generation to move on is bounded by
// EnsSync::limit_ns of the GPU's global timer.  On expiry the CTA records the failure and returns
// without its lattice Boltzmann work; every later launch sees the record and returns at once, so
// the state of the last completed step is kept (apart from the flux W, which the host recomputes).

struct EnsSync {
    unsigned count;                 // CTAs arrived at the current barrier
    unsigned gen;                   // barrier generation: moves on when the last CTA arrives
    int err;                        // a wait expired; later launches do nothing
    unsigned done;                  // CTAs that completed a step (a step adds gridDim.x)
    unsigned long long limit_ns;    // bound of one barrier wait
    int stall;                      // test hook: CTA 0 does not arrive at the barrier
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long gtimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier of a cooperative launch: false if this CTA gave up after sync->limit_ns.
__device__ __forceinline__ bool ens_grid_barrier(EnsSync *sync, bool arrive)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = ld_acquire_u32(&sync->gen);
        if (arrive) {
            __threadfence();   // this CTA's writes before its arrival
            if (atomicAdd(&sync->count, 1u) == gridDim.x - 1) {
                atomicExch(&sync->count, 0u);
                __threadfence();
                atomicAdd(&sync->gen, 1u);
            }
        }
        const unsigned long long t0 = gtimer_ns(), limit = sync->limit_ns;
        while (ld_acquire_u32(&sync->gen) == g) {
            if (gtimer_ns() - t0 > limit) {
                ok = 0;
                break;
            }
            __nanosleep(200);
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// STORE: LBM_FP32 or one of the moment storages (LBM_MOM, LBM_MOM_BF16, LBM_MOM_FP16)
template <int RY, int STORE>
__global__ void __launch_bounds__(256, 2)
    ens_persistent_kernel(const EnsBox *__restrict__ boxes, const int *__restrict__ blk_box, int nb, int ac_tasks,
                          int lbm_work, int lbm_block,
                          int fpn, const float *__restrict__ phi, const float *__restrict__ w,
                          float *__restrict__ phi_new, const float *__restrict__ g_in, const float *__restrict__ u_in,
                          float *__restrict__ g_out, float *__restrict__ u_out, float *__restrict__ w_out,
                          EnsSync *sync)
{
    __shared__ int failed;
    if (threadIdx.x == 0) failed = *(volatile int *)&sync->err;
    __syncthreads();
    if (failed) return;   // an earlier step failed: keep its state
    // phase 1: Allen–Cahn tasks, one warp each
    const int nwarps = gridDim.x * 8;
    for (int task = blockIdx.x * 8 + (threadIdx.x >> 5); task < ac_tasks; task += nwarps) {
        const int b = find_box<1>(boxes, nb, task);
        const Grid G = boxes[b].G;
        const Phys P = boxes[b].P;
        const size_t o = (size_t)boxes[b].off;
        const int local = task - boxes[b].task0;
        const int ncols = boxes[b].ncols, zlen = boxes[b].zlen;
        const int col = local % ncols;
        const int z0 = (local / ncols) * zlen;
        const int zend = min(G.nz, z0 + zlen);
        if (G.wall)
            ac_div_task<true, RY>(G, P, phi + o, w + 3 * o, phi_new + o, col, z0, zend);
        else
            ac_div_task<false, RY>(G, P, phi + o, w + 3 * o, phi_new + o, col, z0, zend);
    }
    if (!ens_grid_barrier(sync, !(sync->stall && blockIdx.x == 0))) {
        if (threadIdx.x == 0) atomicExch(&sync->err, 1);
        return;
    }
    // phase 2: lattice Boltzmann work
    if constexpr (STORE == LBM_FP32) {
        // lbm_block is 64, 128 or 256: virtual block and lane by shift and mask
        const int lg = __ffs(lbm_block) - 1;
        const long long total = (long long)lbm_work << lg;
        for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < total;
             v += (long long)gridDim.x * blockDim.x) {
            const int vblk = (int)(v >> lg);
            const int b = blk_box[vblk];
            const Grid G = boxes[b].G;
            const int node = ((vblk - boxes[b].blk0) << lg) + (int)(v & (lbm_block - 1));
            if (node >= G.N) continue;
            const Phys P = boxes[b].P;
            const size_t o = (size_t)boxes[b].off;
            int x, y, z;
            box_coords(boxes[b], node, x, y, z);
            lbm_node<StoreF32>(G, P, g_in + 27 * o, nullptr, phi_new + o, u_in + 3 * o, g_out + 27 * o, nullptr,
                               u_out + 3 * o, w_out + 3 * o, x, y, z);
        }
    } else {
        using S = typename std::conditional<STORE == LBM_MOM, StoreF32,
                                            typename std::conditional<STORE == LBM_MOM_BF16, StoreB16,
                                                                      StoreF16>::type>::type;
        for (int task = blockIdx.x; task < lbm_work; task += gridDim.x) {
            const int b = find_box<2>(boxes, nb, task);
            const Grid G = boxes[b].G;
            const Phys P = boxes[b].P;
            const size_t o = (size_t)boxes[b].off;
            const int tiles_x = (G.nx + momt::MX - 1) / momt::MX, tiles_y = (G.ny + momt::MY - 1) / momt::MY;
            int t = task - boxes[b].mtask0;
            const int tx = t % tiles_x;
            t /= tiles_x;
            const int ty = t % tiles_y;
            const int z0 = (t / tiles_y) * boxes[b].mzlen;
            const int z1 = min(z0 + boxes[b].mzlen, G.nz);
            const float *mi = g_in + (size_t)fpn * o;
            float *mo = g_out + (size_t)fpn * o;
            __syncthreads();   // the previous task's shared memory is free
            if (G.wall)
                momt::mom_tile_task<true, S>(G, P, mi, u_in + 3 * o, phi_new + o, mo, u_out + 3 * o, w_out + 3 * o,
                                             tx * momt::MX, ty * momt::MY, z0, z1);
            else
                momt::mom_tile_task<false, S>(G, P, mi, u_in + 3 * o, phi_new + o, mo, u_out + 3 * o,
                                              w_out + 3 * o, tx * momt::MX, ty * momt::MY, z0, z1);
        }
    }
    if (threadIdx.x == 0) atomicAdd(&sync->done, 1u);
}

// 2x restriction of one box's state into a coarse state of half the size in every direction: the
// populations, phi and ubar of the coarse cell are the means over its 8 fine nodes (the means of
// the populations carry the fine non-equilibrium part over to the coarse grid).
__global__ void restrict_state_kernel(Grid F, const float *__restrict__ g, const float *__restrict__ phi,
                                      const float *__restrict__ u, Grid C, float *__restrict__ gc,
                                      float *__restrict__ phic, float *__restrict__ uc)
{
    const int kc = blockIdx.x * blockDim.x + threadIdx.x;
    if (kc >= C.N) return;
    const int z = kc / C.nxy, rem = kc - z * C.nxy, y = rem / C.nx, x = rem - y * C.nx;
    size_t f[8];
#pragma unroll
    for (int c = 0; c < 8; ++c)
        f[c] = ((size_t)(2 * z + (c >> 2)) * F.ny + (2 * y + ((c >> 1) & 1))) * F.nx + 2 * x + (c & 1);
    const size_t NF = (size_t)F.N, NC = (size_t)C.N;
    for (int i = 0; i < 27; ++i) {
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < 8; ++c) s += g[i * NF + f[c]];
        gc[i * NC + kc] = 0.125f * s;
    }
    float sp = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) sp += phi[f[c]];
    phic[kc] = 0.125f * sp;
    for (int a = 0; a < 3; ++a) {
        float su = 0.0f;
#pragma unroll
        for (int c = 0; c < 8; ++c) su += u[a * NF + f[c]];
        uc[a * NC + kc] = 0.125f * su;
    }
}

lbm_status ens_fail(lbm_status s, const char *fmt, ...)
{
    char msg[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    set_last_error(msg);
    return s;
}

}  // namespace
}  // namespace tslb

using tslb::ens_fail;
using tslb::EnsBox;

#define ENS_TRY(call)                                                                              \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return ens_fail(LBM_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                            __FILE__, __LINE__);                                                   \
    } while (0)

struct lbm_ens {
    int nb = 0;
    std::vector<lbm_params> prm;
    std::vector<EnsBox> box;          // host copy of the box table
    EnsBox *box_d = nullptr;          // device copy
    int *blk_box = nullptr;           // box of every lattice Boltzmann block (FP32 populations)
    long long blk_box_cap = 0;        // entries allocated: the block count at the smallest lbm_block
    long long ntot = 0;
    float *g[2] = {nullptr, nullptr};  // FP32 populations, or the boxes' moment states
    int storage = LBM_FP32;
    int fpn = 27;                     // floats per node of g (27, or 10 / 6 for the moment storages)
    int mom_tasks = 0;                // moment-storage lattice Boltzmann tasks of all boxes
    float *phi[2] = {nullptr, nullptr};
    float *u[2] = {nullptr, nullptr};
    float *w = nullptr;               // Allen–Cahn flux of the current state, all boxes
    double *partials = nullptr;       // observables scratch (largest box)
    double *result = nullptr;
    double *h_result = nullptr;
    std::vector<char> ready;          // box initialised
    int cur = 0;
    long long step = 0;
    cudaStream_t stream = nullptr;    // the caller's stream (NULL: legacy default)
    cudaStream_t cap = nullptr;       // private stream used only to capture the step graph
    lbm_tuning tun{};
    int sms = 0;
    int ac_bps[2] = {0, 0};           // resident Allen–Cahn CTAs per SM, ac_rows 2 and 4
    int lbm_blocks = 0, ac_tasks = 0, ac_ctas = 0;
    cudaGraphExec_t exec = nullptr;   // graph_steps steps from cur = 0
    cudaGraphExec_t pexec = nullptr;  // graph_steps persistent launches from cur = 0
    int persistent = 0;               // 1: one cooperative launch per step (ens_persistent_kernel)
    int pers_ctas[2] = {0, 0};        // co-resident CTAs of the persistent kernel, ac_rows 2 and 4
    tslb::EnsSync *sync = nullptr;    // barrier state of the persistent kernel
    unsigned done_seen = 0;           // sync->done after the last completed persistent step
};

namespace {

void free_ens(lbm_ens *e)
{
    if (!e) return;
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->pexec) cudaGraphExecDestroy(e->pexec);
    for (int b = 0; b < 2; ++b) {
        cudaFree(e->g[b]);
        cudaFree(e->phi[b]);
        cudaFree(e->u[b]);
    }
    cudaFree(e->w);
    cudaFree(e->sync);
    cudaFree(e->box_d);
    cudaFree(e->blk_box);
    cudaFree(e->partials);
    cudaFree(e->result);
    if (e->h_result) cudaFreeHost(e->h_result);
    if (e->cap) cudaStreamDestroy(e->cap);
    delete e;
}

bool tuning_valid(const lbm_tuning &t)
{
    return (t.lbm_block == 64 || t.lbm_block == 128 || t.lbm_block == 256) && (t.ac_rows == 2 || t.ac_rows == 4) &&
           t.ac_zlen >= 1 && (t.graph_steps == 0 || (t.graph_steps >= 2 && t.graph_steps % 2 == 0));
}

// Box table for the current tuning: block and task ranges of every box, uploaded to the device.
lbm_status build_tables(lbm_ens *e)
{
    long long blk = 0, task = 0, mtask = 0;
    const int ry = e->tun.ac_rows;
    int mzlen = tslb::kEnsMomZlens[3];
    for (int zl : tslb::kEnsMomZlens) {
        long long t = 0;
        for (int b = 0; b < e->nb; ++b) {
            const tslb::Grid &G = e->box[b].G;
            const int z = zl < G.nz ? zl : G.nz;
            t += (long long)((G.nx + tslb::momt::MX - 1) / tslb::momt::MX) * ((G.ny + tslb::momt::MY - 1) / tslb::momt::MY) *
                 ((G.nz + z - 1) / z);
        }
        if (t >= (long long)tslb::kEnsMomTasksPerCta * tslb::kEnsMomCtasPerSm * e->sms) {
            mzlen = zl;
            break;
        }
    }
    for (int b = 0; b < e->nb; ++b) {
        EnsBox &B = e->box[b];
        const int zlen = e->tun.ac_zlen < B.G.nz ? e->tun.ac_zlen : B.G.nz;
        const int m = (B.G.nz + zlen - 1) / zlen;
        B.blk0 = (int)blk;
        B.task0 = (int)task;
        B.ncols = ((B.G.nx + tslb::AC_XO - 1) / tslb::AC_XO) * ((B.G.ny + ry - 1) / ry);
        B.zlen = zlen;
        blk += (B.G.N + e->tun.lbm_block - 1) / e->tun.lbm_block;
        task += (long long)B.ncols * m;
        B.mtask0 = (int)mtask;
        B.mzlen = mzlen < B.G.nz ? mzlen : B.G.nz;
        mtask += (long long)((B.G.nx + tslb::momt::MX - 1) / tslb::momt::MX) *
                 ((B.G.ny + tslb::momt::MY - 1) / tslb::momt::MY) * ((B.G.nz + B.mzlen - 1) / B.mzlen);
    }
    if (blk >= (1LL << 31) || task >= (1LL << 31) || mtask >= (1LL << 31))
        return ens_fail(LBM_ERR_ARG, "ensemble too large for one launch (%lld blocks, %lld tasks)", blk, task);
    e->lbm_blocks = (int)blk;
    e->mom_tasks = (int)mtask;
    e->ac_tasks = (int)task;
    const long long warp_slots = (long long)e->sms * e->ac_bps[ry == 2 ? 0 : 1] * tslb::AC_WPB;
    const long long warps = task < warp_slots ? task : warp_slots;
    e->ac_ctas = (int)((warps + tslb::AC_WPB - 1) / tslb::AC_WPB);
    if (blk > e->blk_box_cap) return ens_fail(LBM_ERR_ARG, "block table too small (%lld > %lld)", blk, e->blk_box_cap);
    std::vector<int> bb((size_t)blk);
    for (int b = 0; b < e->nb; ++b) {
        const int end = b + 1 < e->nb ? e->box[b + 1].blk0 : (int)blk;
        for (int k = e->box[b].blk0; k < end; ++k) bb[k] = b;
    }
    ENS_TRY(cudaMemcpyAsync(e->box_d, e->box.data(), e->nb * sizeof(EnsBox), cudaMemcpyHostToDevice, e->stream));
    ENS_TRY(cudaMemcpyAsync(e->blk_box, bb.data(), bb.size() * sizeof(int), cudaMemcpyHostToDevice, e->stream));
    ENS_TRY(cudaStreamSynchronize(e->stream));
    if (e->exec) {
        cudaGraphExecDestroy(e->exec);
        e->exec = nullptr;
    }
    if (e->pexec) {
        cudaGraphExecDestroy(e->pexec);
        e->pexec = nullptr;
    }
    return LBM_OK;
}

cudaError_t ens_launch_ac(lbm_ens *e, int a, cudaStream_t s)
{
    if (e->tun.ac_rows == 2)
        tslb::ens_ac_kernel<2><<<e->ac_ctas, tslb::AC_WPB * 32, 0, s>>>(e->box_d, e->nb, e->ac_tasks, e->phi[a], e->w,
                                                                         e->phi[1 - a]);
    else
        tslb::ens_ac_kernel<4><<<e->ac_ctas, tslb::AC_WPB * 32, 0, s>>>(e->box_d, e->nb, e->ac_tasks, e->phi[a], e->w,
                                                                         e->phi[1 - a]);
    return cudaGetLastError();
}

template <class S>
cudaError_t ens_launch_mom(lbm_ens *e, int a, cudaStream_t s)
{
    tslb::ens_mom_kernel<S><<<e->mom_tasks, tslb::momt::kMomThreads, tslb::momt::kMomSmem, s>>>(
        e->box_d, e->nb, e->fpn, e->g[a], e->phi[1 - a], e->u[a], e->g[1 - a], e->u[1 - a], e->w);
    return cudaGetLastError();
}

cudaError_t ens_launch_lbm(lbm_ens *e, int a, cudaStream_t s)
{
    switch (e->storage) {
    case LBM_MOM: return ens_launch_mom<tslb::StoreF32>(e, a, s);
    case LBM_MOM_BF16: return ens_launch_mom<tslb::StoreB16>(e, a, s);
    case LBM_MOM_FP16: return ens_launch_mom<tslb::StoreF16>(e, a, s);
    default: break;
    }
    tslb::ens_lbm_kernel<<<e->lbm_blocks, e->tun.lbm_block, 0, s>>>(e->box_d, e->blk_box, e->g[a], e->phi[1 - a], e->u[a],
                                                                      e->g[1 - a], e->u[1 - a], e->w);
    return cudaGetLastError();
}

template <class S>
cudaError_t ens_prepare_mom()
{
    return cudaFuncSetAttribute(tslb::ens_mom_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tslb::momt::kMomSmem);
}

// One step from buffers a to 1 - a.
cudaError_t ens_launch_step(lbm_ens *e, int a, cudaStream_t s)
{
    cudaError_t err = ens_launch_ac(e, a, s);
    if (err != cudaSuccess) return err;
    return ens_launch_lbm(e, a, s);
}

lbm_status recompute_flux(lbm_ens *e);

template <int RY, int STORE>
cudaError_t ens_persistent_launch(lbm_ens *e, int a, cudaStream_t s)
{
    int ac_tasks = e->ac_tasks, lbm_work = STORE == LBM_FP32 ? e->lbm_blocks : e->mom_tasks, lbm_block = e->tun.lbm_block,
        fpn = e->fpn, nb = e->nb;
    const EnsBox *boxes = e->box_d;
    const int *blk_box = e->blk_box;
    const float *phi = e->phi[a], *w = e->w, *g_in = e->g[a], *u_in = e->u[a];
    float *phi_new = e->phi[1 - a], *g_out = e->g[1 - a], *u_out = e->u[1 - a], *w_out = e->w;
    tslb::EnsSync *sync = e->sync;
    void *args[] = {&boxes, &blk_box, &nb, &ac_tasks, &lbm_work, &lbm_block, &fpn, &phi, &w, &phi_new,
                    &g_in, &u_in, &g_out, &u_out, &w_out, &sync};
    const size_t smem = STORE == LBM_FP32 ? 0 : tslb::momt::kMomSmem;
    return cudaLaunchCooperativeKernel((const void *)tslb::ens_persistent_kernel<RY, STORE>,
                                       dim3(e->pers_ctas[RY == 2 ? 0 : 1]), dim3(256), args, smem, s);
}

template <int RY>
cudaError_t ens_persistent_step(lbm_ens *e, int a, cudaStream_t s)
{
    switch (e->storage) {
    case LBM_MOM: return ens_persistent_launch<RY, LBM_MOM>(e, a, s);
    case LBM_MOM_BF16: return ens_persistent_launch<RY, LBM_MOM_BF16>(e, a, s);
    case LBM_MOM_FP16: return ens_persistent_launch<RY, LBM_MOM_FP16>(e, a, s);
    default: return ens_persistent_launch<RY, LBM_FP32>(e, a, s);
    }
}

// Co-resident CTAs of the persistent kernel (ac_rows 2 and 4) for the ensemble's storage.
template <int STORE>
cudaError_t ens_persistent_setup(lbm_ens *e)
{
    const size_t smem = STORE == LBM_FP32 ? 0 : tslb::momt::kMomSmem;
    int bps[2] = {0, 0};
    cudaError_t err = cudaFuncSetAttribute(tslb::ens_persistent_kernel<2, STORE>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(tslb::ens_persistent_kernel<4, STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem);
    if (err == cudaSuccess)
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps[0], tslb::ens_persistent_kernel<2, STORE>, 256, smem);
    if (err == cudaSuccess)
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps[1], tslb::ens_persistent_kernel<4, STORE>, 256, smem);
    e->pers_ctas[0] = bps[0] * e->sms;
    e->pers_ctas[1] = bps[1] * e->sms;
    return err;
}

// Persistent steps: one cooperative launch each, then the barrier record is read.  Returns the
// steps completed; *timed_out when a barrier wait expired (the state is that of the last
// completed step, its flux W recomputed, and the record reset).
lbm_status build_persistent_graph(lbm_ens *e);

lbm_status ens_persistent_run(lbm_ens *e, int nsteps)
{
    const int K = e->tun.graph_steps;
    for (int k = 0; k < nsteps;) {
        const int a = e->cur ^ (k & 1);
        if (K >= 2 && a == 0 && nsteps - k >= K) {   // K launches from buffers 0, replayed from a graph
            if (!e->pexec) {
                lbm_status st = build_persistent_graph(e);
                if (st != LBM_OK) return st;
            }
            ENS_TRY(cudaGraphLaunch(e->pexec, e->stream));
            k += K;
        } else {
            ENS_TRY(e->tun.ac_rows == 2 ? ens_persistent_step<2>(e, a, e->stream)
                                        : ens_persistent_step<4>(e, a, e->stream));
            ++k;
        }
    }
    tslb::EnsSync h;
    ENS_TRY(cudaMemcpyAsync(&h, e->sync, sizeof h, cudaMemcpyDeviceToHost, e->stream));
    ENS_TRY(cudaStreamSynchronize(e->stream));
    const unsigned grid = (unsigned)e->pers_ctas[e->tun.ac_rows == 2 ? 0 : 1];
    const unsigned completed = (h.done - e->done_seen) / grid;
    e->done_seen += completed * grid;
    e->cur ^= (int)(completed & 1u);
    e->step += completed;
    if (!h.err) return LBM_OK;
    // a wait expired: reset the record (the counter of a barrier that never completed, the done
    // count of CTAs of an incomplete step) and recompute the flux of the kept state
    h.count = 0;
    h.err = 0;
    h.done = e->done_seen;
    ENS_TRY(cudaMemcpyAsync(e->sync, &h, sizeof h, cudaMemcpyHostToDevice, e->stream));
    lbm_status st = recompute_flux(e);
    if (st != LBM_OK) return st;
    ENS_TRY(cudaStreamSynchronize(e->stream));
    return ens_fail(LBM_ERR_TIMEOUT, "a grid barrier wait of the persistent step expired after %u of %d steps",
                    completed, nsteps);
}

// Capture graph_steps steps starting from buffers 0 on the private stream.
lbm_status build_graph(lbm_ens *e)
{
    cudaGraph_t graph = nullptr;
    ENS_TRY(cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < e->tun.graph_steps && err == cudaSuccess; ++k) err = ens_launch_step(e, k & 1, e->cap);
    cudaError_t end = cudaStreamEndCapture(e->cap, &graph);
    if (err != cudaSuccess || end != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return ens_fail(LBM_ERR_CUDA, "graph capture failed: %s",
                        cudaGetErrorString(err != cudaSuccess ? err : end));
    }
    err = cudaGraphInstantiate(&e->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) {
        e->exec = nullptr;
        return ens_fail(LBM_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(err));
    }
    return LBM_OK;
}

// Capture graph_steps persistent launches (one per step) starting from buffers 0 on the private
// stream.  A launch that finds the barrier record set returns at once, so a replay after an
// expired wait keeps the state of the last completed step, as direct launches do.
lbm_status build_persistent_graph(lbm_ens *e)
{
    cudaGraph_t graph = nullptr;
    ENS_TRY(cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < e->tun.graph_steps && err == cudaSuccess; ++k)
        err = e->tun.ac_rows == 2 ? ens_persistent_step<2>(e, k & 1, e->cap) : ens_persistent_step<4>(e, k & 1, e->cap);
    cudaError_t end = cudaStreamEndCapture(e->cap, &graph);
    if (err != cudaSuccess || end != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return ens_fail(LBM_ERR_CUDA, "persistent graph capture failed: %s",
                        cudaGetErrorString(err != cudaSuccess ? err : end));
    }
    err = cudaGraphInstantiate(&e->pexec, graph, 0);
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) {
        e->pexec = nullptr;
        return ens_fail(LBM_ERR_CUDA, "persistent graph instantiation failed: %s", cudaGetErrorString(err));
    }
    return LBM_OK;
}

// W of the current state of every box (after a launch that overwrote it)
lbm_status recompute_flux(lbm_ens *e)
{
    const int c = e->cur;
    for (int b = 0; b < e->nb; ++b) {
        const EnsBox &B = e->box[b];
        const size_t o = (size_t)B.off;
        ENS_TRY(tslb::launch_flux(B.G, B.P, e->phi[c] + o, e->u[c] + 3 * o, e->w + 3 * o, e->stream));
    }
    return LBM_OK;
}

bool all_ready(const lbm_ens *e)
{
    for (char r : e->ready)
        if (!r) return false;
    return true;
}

}  // namespace

extern "C" {

lbm_status lbm_ens_create(const lbm_params *params, int nboxes, void *stream, lbm_ens **out)
{
    if (!out) return ens_fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!params) return ens_fail(LBM_ERR_ARG, "params is NULL");
    if (nboxes < 1) return ens_fail(LBM_ERR_ARG, "nboxes must be >= 1");
    for (int b = 0; b < nboxes; ++b) {
        lbm_status st = tslb::check_params(&params[b]);
        if (st != LBM_OK) {
            char msg[512];
            snprintf(msg, sizeof msg, "box %d: %s", b, lbm_last_error());
            tslb::set_last_error(msg);
            return st;
        }
        if (params[b].storage != params[0].storage)
            return ens_fail(LBM_ERR_ARG, "box %d: every box of an ensemble has the same storage", b);
        if (params[b].storage != LBM_FP32 && params[b].storage < LBM_MOM)
            return ens_fail(LBM_ERR_ARG, "box %d: ensembles use LBM_FP32 or a moment storage", b);
    }
    lbm_ens *e = new (std::nothrow) lbm_ens;
    if (!e) return ens_fail(LBM_ERR_OOM, "host allocation failed");
    e->nb = nboxes;
    e->stream = (cudaStream_t)stream;
    e->storage = params[0].storage;
    e->fpn = e->storage == LBM_FP32 ? 27 : (int)(tslb::mom_state_bytes(e->storage, 1) / sizeof(float));
    e->prm.assign(params, params + nboxes);
    e->box.resize(nboxes);
    e->ready.assign(nboxes, 0);
    int max_obs = 1;
    for (int b = 0; b < nboxes; ++b) {
        EnsBox &B = e->box[b];
        memset(&B, 0, sizeof B);
        tslb::params_to_consts(params[b], B.G, B.P);
        B.rnxy = 1.0f / (float)B.G.nxy;
        B.rnx = 1.0f / (float)B.G.nx;
        B.off = e->ntot;
        e->ntot += B.G.N;
        e->blk_box_cap += (B.G.N + 63) / 64;
        const int ob = tslb::observables_blocks(B.G);
        if (ob > max_obs) max_obs = ob;
    }
    e->tun.lbm_block = 128;
    e->tun.ac_rows = 4;
    e->tun.ac_zlen = 32;
    e->tun.graph_steps = 16;
    const size_t N = (size_t)e->ntot;
    struct {
        void **p;
        size_t bytes;
    } allocs[] = {
        {(void **)&e->g[0], e->fpn * N * sizeof(float)}, {(void **)&e->g[1], e->fpn * N * sizeof(float)},
        {(void **)&e->phi[0], N * sizeof(float)},    {(void **)&e->phi[1], N * sizeof(float)},
        {(void **)&e->u[0], 3 * N * sizeof(float)},  {(void **)&e->u[1], 3 * N * sizeof(float)},
        {(void **)&e->w, 3 * N * sizeof(float)},     {(void **)&e->box_d, nboxes * sizeof(EnsBox)},
        {(void **)&e->blk_box, (size_t)e->blk_box_cap * sizeof(int)},
        {(void **)&e->sync, sizeof(tslb::EnsSync)},
        {(void **)&e->partials, (size_t)max_obs * tslb::kObsFields * sizeof(double)},
        {(void **)&e->result, tslb::kObsFields * sizeof(double)},
    };
    for (auto &a : allocs) {
        cudaError_t err = cudaMalloc(a.p, a.bytes);
        if (err != cudaSuccess) {
            cudaGetLastError();
            free_ens(e);
            return ens_fail(err == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "cudaMalloc(%zu) failed: %s",
                            a.bytes, cudaGetErrorString(err));
        }
    }
    cudaError_t err = cudaMallocHost(&e->h_result, tslb::kObsFields * sizeof(double));
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking);
    int dev = 0;
    if (err == cudaSuccess) err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, dev);
    if (err == cudaSuccess)
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&e->ac_bps[0], tslb::ens_ac_kernel<2>, tslb::AC_WPB * 32, 0);
    if (err == cudaSuccess)
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&e->ac_bps[1], tslb::ens_ac_kernel<4>, tslb::AC_WPB * 32, 0);
    if (err == cudaSuccess) {   // barrier record: no arrivals, 100 ms per wait
        tslb::EnsSync h{};
        h.limit_ns = 100000000ull;
        err = cudaMemcpy(e->sync, &h, sizeof h, cudaMemcpyHostToDevice);
    }
    if (err == cudaSuccess) {
        switch (e->storage) {
        case LBM_MOM: err = ens_persistent_setup<LBM_MOM>(e); break;
        case LBM_MOM_BF16: err = ens_persistent_setup<LBM_MOM_BF16>(e); break;
        case LBM_MOM_FP16: err = ens_persistent_setup<LBM_MOM_FP16>(e); break;
        default: err = ens_persistent_setup<LBM_FP32>(e); break;
        }
    }
    if (err == cudaSuccess && e->storage == LBM_MOM) err = ens_prepare_mom<tslb::StoreF32>();
    if (err == cudaSuccess && e->storage == LBM_MOM_BF16) err = ens_prepare_mom<tslb::StoreB16>();
    if (err == cudaSuccess && e->storage == LBM_MOM_FP16) err = ens_prepare_mom<tslb::StoreF16>();
    if (err != cudaSuccess) {
        cudaGetLastError();
        free_ens(e);
        return ens_fail(LBM_ERR_CUDA, "ensemble setup failed: %s", cudaGetErrorString(err));
    }
    if (e->ac_bps[0] < 1 || e->ac_bps[1] < 1) {
        free_ens(e);
        return ens_fail(LBM_ERR_CUDA, "Allen-Cahn ensemble kernel does not fit an SM");
    }
    lbm_status st = build_tables(e);
    if (st != LBM_OK) {
        free_ens(e);
        return st;
    }
    *out = e;
    return LBM_OK;
}

void lbm_ens_destroy(lbm_ens *ens)
{
    if (!ens) return;
    cudaStreamSynchronize(ens->stream);
    free_ens(ens);
}

int lbm_ens_num_boxes(const lbm_ens *ens) { return ens ? ens->nb : 0; }
long long lbm_ens_num_nodes(const lbm_ens *ens) { return ens ? ens->ntot : 0; }
long long lbm_ens_box_nodes(const lbm_ens *ens, int box)
{
    return (ens && box >= 0 && box < ens->nb) ? (long long)ens->box[box].G.N : 0;
}
long long lbm_ens_step_count(const lbm_ens *ens) { return ens ? ens->step : 0; }

lbm_status lbm_ens_init_fields(lbm_ens *ens, int box, const float *phi, const float *u, const float *pstar,
                               int on_device)
{
    if (!ens) return ens_fail(LBM_ERR_ARG, "ensemble is NULL");
    if (box < 0 || box >= ens->nb) return ens_fail(LBM_ERR_ARG, "box %d out of range [0, %d)", box, ens->nb);
    if (!phi || !u) return ens_fail(LBM_ERR_ARG, "phi and u are required");
    const EnsBox &B = ens->box[box];
    const size_t n = (size_t)B.G.N, o = (size_t)B.off;
    const int c = ens->cur;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    ENS_TRY(cudaMemcpyAsync(ens->phi[c] + o, phi, n * sizeof(float), k, ens->stream));
    ENS_TRY(cudaMemcpyAsync(ens->u[c] + 3 * o, u, 3 * n * sizeof(float), k, ens->stream));
    const float *ps = nullptr;
    const size_t go = (size_t)ens->fpn * o;   // the box's slice of the population / moment state
    if (pstar) {   // stage p*0 in the box's idle state slice
        ENS_TRY(cudaMemcpyAsync(ens->g[1 - c] + go, pstar, n * sizeof(float), k, ens->stream));
        ps = ens->g[1 - c] + go;
    }
    if (ens->storage == LBM_FP32)
        ENS_TRY(tslb::launch_init(B.G, ps, ens->u[c] + 3 * o, ens->g[c] + go, ens->stream));
    else
        ENS_TRY(tslb::launch_mom_init(B.G, ens->storage, ps, ens->g[c] + go, ens->stream));
    ENS_TRY(tslb::launch_flux(B.G, B.P, ens->phi[c] + o, ens->u[c] + 3 * o, ens->w + 3 * o, ens->stream));
    if (!on_device) ENS_TRY(cudaStreamSynchronize(ens->stream));
    ens->ready[box] = 1;
    return LBM_OK;
}

lbm_status lbm_ens_step(lbm_ens *ens, int nsteps)
{
    if (!ens) return ens_fail(LBM_ERR_ARG, "ensemble is NULL");
    if (nsteps < 0) return ens_fail(LBM_ERR_ARG, "nsteps must be >= 0");
    if (!all_ready(ens)) return ens_fail(LBM_ERR_STATE, "lbm_ens_step before every box was initialised");
    if (ens->persistent) return ens_persistent_run(ens, nsteps);
    const int K = ens->tun.graph_steps;
    while (nsteps > 0) {
        if (K >= 2 && ens->cur == 0 && nsteps >= K) {
            if (!ens->exec) {
                lbm_status st = build_graph(ens);
                if (st != LBM_OK) return st;
            }
            ENS_TRY(cudaGraphLaunch(ens->exec, ens->stream));
            nsteps -= K;
            ens->step += K;
        } else {
            ENS_TRY(ens_launch_step(ens, ens->cur, ens->stream));
            ens->cur ^= 1;
            --nsteps;
            ++ens->step;
        }
    }
    return LBM_OK;
}

lbm_status lbm_ens_observables(lbm_ens *ens, int box, lbm_obs *out)
{
    if (!ens) return ens_fail(LBM_ERR_ARG, "ensemble is NULL");
    if (box < 0 || box >= ens->nb) return ens_fail(LBM_ERR_ARG, "box %d out of range [0, %d)", box, ens->nb);
    if (!out) return ens_fail(LBM_ERR_ARG, "out is NULL");
    if (!ens->ready[box]) return ens_fail(LBM_ERR_STATE, "box %d is not initialised", box);
    const EnsBox &B = ens->box[box];
    const lbm_params &p = ens->prm[box];
    const size_t o = (size_t)B.off;
    const int c = ens->cur;
    ENS_TRY(tslb::launch_observables(B.G, p.rho_l, p.rho_g, ens->g[c] + (size_t)ens->fpn * o, ens->phi[c] + o,
                                     ens->u[c] + 3 * o, ens->partials, tslb::observables_blocks(B.G), ens->result,
                                     ens->stream, ens->storage));
    ENS_TRY(cudaMemcpyAsync(ens->h_result, ens->result, tslb::kObsFields * sizeof(double), cudaMemcpyDeviceToHost,
                            ens->stream));
    ENS_TRY(cudaStreamSynchronize(ens->stream));
    const double *r = ens->h_result;
    memset(out, 0, sizeof *out);
    out->step = (double)ens->step;
    out->sum_phi = r[0];
    out->mass = r[1];
    out->sum_pstar = r[2];
    for (int a = 0; a < 3; ++a) {
        out->momentum[a] = r[3 + a];
        out->centroid_liq[a] = r[6 + a] / r[0];
        out->centroid_gas[a] = r[9 + a] / r[26];
        out->vel_liq[a] = r[12 + a] / r[0];
        out->vel_gas[a] = r[15 + a] / r[26];
    }
    out->n_liq = r[19];
    out->n_gas = r[21];
    out->p_liq = r[19] > 0 ? r[18] / r[19] : NAN;
    out->p_gas = r[21] > 0 ? r[20] / r[21] : NAN;
    out->umax = r[22];
    out->phi_min = r[23];
    out->phi_max = r[24];
    out->n_nonfinite = r[25];
    if (out->n_nonfinite > 0) return ens_fail(LBM_ERR_NONFINITE, "box %d: %.0f non-finite nodes", box, out->n_nonfinite);
    return LBM_OK;
}

lbm_status lbm_ens_read_fields(lbm_ens *ens, int box, float *phi, float *u, float *p, int on_device)
{
    if (!ens) return ens_fail(LBM_ERR_ARG, "ensemble is NULL");
    if (box < 0 || box >= ens->nb) return ens_fail(LBM_ERR_ARG, "box %d out of range [0, %d)", box, ens->nb);
    if (!ens->ready[box]) return ens_fail(LBM_ERR_STATE, "box %d is not initialised", box);
    const EnsBox &B = ens->box[box];
    const size_t n = (size_t)B.G.N, o = (size_t)B.off;
    const int c = ens->cur;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (phi) ENS_TRY(cudaMemcpyAsync(phi, ens->phi[c] + o, n * sizeof(float), k, ens->stream));
    if (u) ENS_TRY(cudaMemcpyAsync(u, ens->u[c] + 3 * o, 3 * n * sizeof(float), k, ens->stream));
    if (p) {   // p into the box's idle state slice, then copy
        const size_t go = (size_t)ens->fpn * o;
        float *tmp = ens->g[1 - c] + go;
        ENS_TRY(tslb::launch_pressure(B.G, B.P, ens->storage, ens->g[c] + go, nullptr, ens->phi[c] + o, tmp,
                                      ens->stream));
        ENS_TRY(cudaMemcpyAsync(p, tmp, n * sizeof(float), k, ens->stream));
    }
    ENS_TRY(cudaStreamSynchronize(ens->stream));
    return LBM_OK;
}

lbm_status lbm_ens_get_tuning(const lbm_ens *ens, lbm_tuning *out)
{
    if (!ens || !out) return ens_fail(LBM_ERR_ARG, "ensemble and out are required");
    *out = ens->tun;
    return LBM_OK;
}

lbm_status lbm_ens_set_tuning(lbm_ens *ens, const lbm_tuning *t)
{
    if (!ens || !t) return ens_fail(LBM_ERR_ARG, "ensemble and tuning are required");
    if (!tuning_valid(*t))
        return ens_fail(LBM_ERR_ARG, "tuning out of range (lbm_block %d, ac_rows %d, ac_zlen %d, graph_steps %d)",
                        t->lbm_block, t->ac_rows, t->ac_zlen, t->graph_steps);
    ens->tun = *t;
    return build_tables(ens);
}

lbm_status lbm_ens_autotune(lbm_ens *ens, int reps, lbm_tuning *out)
{
    if (!ens) return ens_fail(LBM_ERR_ARG, "ensemble is NULL");
    if (reps < 1) return ens_fail(LBM_ERR_ARG, "reps must be >= 1");
    if (!all_ready(ens)) return ens_fail(LBM_ERR_STATE, "lbm_ens_autotune before every box was initialised");
    cudaEvent_t t0, t1;
    ENS_TRY(cudaEventCreate(&t0));
    cudaError_t err = cudaEventCreate(&t1);
    if (err != cudaSuccess) {
        cudaEventDestroy(t0);
        return ens_fail(LBM_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(err));
    }
    lbm_tuning best = ens->tun;
    lbm_status st = LBM_OK;
    const int a = ens->cur;
    // Allen–Cahn kernel: reads phi and W of the current state, writes the idle phi
    double best_ac = 1e30;
    const int rows[2] = {2, 4};
    const int zlens[4] = {8, 16, 32, 64};
    for (int ri = 0; ri < 2 && st == LBM_OK; ++ri)
        for (int zi = 0; zi < 4 && st == LBM_OK; ++zi) {
            ens->tun.ac_rows = rows[ri];
            ens->tun.ac_zlen = zlens[zi];
            if ((st = build_tables(ens)) != LBM_OK) break;
            err = ens_launch_ac(ens, a, ens->stream);
            if (err == cudaSuccess) err = cudaEventRecord(t0, ens->stream);
            for (int r = 0; r < reps && err == cudaSuccess; ++r) err = ens_launch_ac(ens, a, ens->stream);
            if (err == cudaSuccess) err = cudaEventRecord(t1, ens->stream);
            if (err == cudaSuccess) err = cudaEventSynchronize(t1);
            float ms = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, t0, t1);
            if (err != cudaSuccess) {
                st = ens_fail(LBM_ERR_CUDA, "autotune (Allen-Cahn): %s", cudaGetErrorString(err));
                break;
            }
            const double us = 1e3 * ms / reps;
            if (us < best_ac) {
                best_ac = us;
                best.ac_rows = rows[ri];
                best.ac_zlen = zlens[zi];
            }
        }
    // lattice Boltzmann kernel: reads g, ubar of the current state and the idle phi just written;
    // writes the idle g, ubar and W (W of the current state is recomputed below)
    // (moment storage: one tiled configuration; lbm_block does not apply and only the time is kept)
    double best_lbm = 1e30;
    const int blocks[3] = {64, 128, 256};
    const int nblock = ens->storage == LBM_FP32 ? 3 : 1;
    if (ens->storage != LBM_FP32) best.lbm_block = ens->tun.lbm_block;
    for (int bi = 0; bi < nblock && st == LBM_OK; ++bi) {
        if (ens->storage == LBM_FP32) ens->tun.lbm_block = blocks[bi];
        if ((st = build_tables(ens)) != LBM_OK) break;
        err = ens_launch_lbm(ens, a, ens->stream);
        if (err == cudaSuccess) err = cudaEventRecord(t0, ens->stream);
        for (int r = 0; r < reps && err == cudaSuccess; ++r) err = ens_launch_lbm(ens, a, ens->stream);
        if (err == cudaSuccess) err = cudaEventRecord(t1, ens->stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, t0, t1);
        if (err != cudaSuccess) {
            st = ens_fail(LBM_ERR_CUDA, "autotune (lattice Boltzmann): %s", cudaGetErrorString(err));
            break;
        }
        const double us = 1e3 * ms / reps;
        if (us < best_lbm) {
            best_lbm = us;
            if (ens->storage == LBM_FP32) best.lbm_block = blocks[bi];
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    best.lbm_us = best_lbm < 1e30 ? best_lbm : 0.0;
    best.ac_us = best_ac < 1e30 ? best_ac : 0.0;
    ens->tun = best;
    lbm_status st2 = build_tables(ens);
    lbm_status st3 = recompute_flux(ens);
    if (st == LBM_OK) st = st2 != LBM_OK ? st2 : st3;
    if (st == LBM_OK) {
        ENS_TRY(cudaStreamSynchronize(ens->stream));
        if (out) *out = ens->tun;
    }
    return st;
}

lbm_status lbm_ens_set_persistent(lbm_ens *ens, int on)
{
    if (!ens) return ens_fail(LBM_ERR_ARG, "ensemble is NULL");
    if (on != 0 && on != 1) return ens_fail(LBM_ERR_ARG, "on must be 0 or 1");
    if (on && (ens->pers_ctas[0] < 1 || ens->pers_ctas[1] < 1))
        return ens_fail(LBM_ERR_CUDA, "the persistent ensemble kernel does not fit an SM");
    ENS_TRY(cudaStreamSynchronize(ens->stream));
    ens->persistent = on;
    return LBM_OK;
}

lbm_status lbm_ens_test_stall_barrier(lbm_ens *ens, int on)
{
    if (!ens) return ens_fail(LBM_ERR_ARG, "ensemble is NULL");
    if (on != 0 && on != 1) return ens_fail(LBM_ERR_ARG, "on must be 0 or 1");
    tslb::EnsSync h;
    ENS_TRY(cudaMemcpyAsync(&h, ens->sync, sizeof h, cudaMemcpyDeviceToHost, ens->stream));
    ENS_TRY(cudaStreamSynchronize(ens->stream));
    h.stall = on;
    h.limit_ns = on ? 2000000ull : 100000000ull;
    ENS_TRY(cudaMemcpyAsync(ens->sync, &h, sizeof h, cudaMemcpyHostToDevice, ens->stream));
    ENS_TRY(cudaStreamSynchronize(ens->stream));
    return LBM_OK;
}

lbm_status lbm_ens_restrict_state(lbm_ens *ens, int box, lbm_ctx *coarse)
{
    if (!ens || !coarse) return ens_fail(LBM_ERR_ARG, "ensemble and coarse context are required");
    if (box < 0 || box >= ens->nb) return ens_fail(LBM_ERR_ARG, "box %d out of range [0, %d)", box, ens->nb);
    if (!ens->ready[box]) return ens_fail(LBM_ERR_STATE, "box %d is not initialised", box);
    tslb::CtxView v;
    lbm_status st = tslb::ctx_view(coarse, &v);
    if (st != LBM_OK) return st;
    const EnsBox &B = ens->box[box];
    if (ens->storage != LBM_FP32) return ens_fail(LBM_ERR_ARG, "restriction needs an ensemble with FP32 populations");
    if (v.storage != LBM_FP32 || B.G.nx != 2 * v.G.nx || B.G.ny != 2 * v.G.ny || B.G.nz != 2 * v.G.nz)
        return ens_fail(LBM_ERR_ARG, "coarse context must be FP32 with half the box size in every direction");
    const size_t o = (size_t)B.off;
    const int c = ens->cur;
    // order the coarse stream after the ensemble's work on this machine
    cudaEvent_t ev;
    ENS_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t err = cudaEventRecord(ev, ens->stream);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(v.stream, ev, 0);
    cudaEventDestroy(ev);
    if (err != cudaSuccess) return ens_fail(LBM_ERR_CUDA, "stream ordering failed: %s", cudaGetErrorString(err));
    tslb::restrict_state_kernel<<<(v.G.N + 255) / 256, 256, 0, v.stream>>>(
        B.G, ens->g[c] + 27 * o, ens->phi[c] + o, ens->u[c] + 3 * o, v.G, v.g, v.phi, v.u);
    ENS_TRY(cudaGetLastError());
    tslb::ctx_state_changed(coarse);
    return LBM_OK;
}

}  // extern "C"

// Learned closure: a 4-layer periodic 3x3x3 convolutional network (5 -> 32 -> 32 -> 32 -> 4
// channels, SiLU between layers) that corrects phi and ubar of a 2x-coarser grid after each step
// (lbm_cnn_* and lbm_closure_apply in include/lbm.h).  The paper has no learned component; this
// is the library's coarse-grid correction, measured against the fine-grid solver.
//
// Every convolution (forward, and the backward pass with respect to its input) is an implicit GEMM
// on the tensor cores: D[o][n] = sum_{k, i} W[o][i][k] a[n + off_k][i], BF16 operands, FP32
// accumulation, channel-last BF16 activations.  Three forms compute it with the same products in
// the same order (identical results): the default conv_umma_kernel (tcgen05.mma, accumulators in
// TMEM, operands staged in shared memory; described above it), and two mma.sync m16n8k16 forms
// (conv_tile_kernel from shared-memory tiles, conv_mma_kernel from global memory), where a warp
// computes 32 consecutive nodes of one x row for up to 32 output channels.  The weight gradient,
// a reduction over all nodes, runs on mma.sync from channel-last tiles with per-block partials
// added in a fixed order; master weights, gradients and Adam moments are FP32, and no reduction
// uses atomics, so training is reproducible run to run.
#include <limits.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "lbm.h"
#include "tslb_internal.h"

namespace tslb {
namespace {

constexpr int NLAYER = 4;
constexpr int CIN[NLAYER] = {5, 32, 32, 32};
constexpr int COUT[NLAYER] = {32, 32, 32, 4};
constexpr int CINP[NLAYER] = {16, 32, 32, 32};    // padded to multiples of 16
constexpr int COUTP[NLAYER] = {32, 32, 32, 16};

constexpr int wcount(int l) { return COUT[l] * CIN[l] * 27; }
constexpr int kCorrBlocks = 296;   // blocks of the correction's sums
constexpr int pcount(int l) { return wcount(l) + COUT[l]; }

// ---- tensor-core implicit-GEMM convolution -------------------------------------------------

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint4 &a, uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int cwrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// z[n][o] = bias[o] + sum_{k, i} W[o][i][k] in[n + off_k][i] for the MT*16 (padded) output
// channels, over a periodic nx x ny x nz grid with nx % 32 == 0.  in: channel-last BF16 with
// CB*16 channels; wfrag: fragment-ordered BF16 weights [27*CB][MT][32 lanes] (uint4 each);
// z: channel-last FP32 with MT*16 channels.  A warp owns 32 consecutive nodes of one x row.
template <int MT, int CB>
__global__ void __launch_bounds__(128) conv_mma_kernel(int nx, int ny, int nz, const uint4 *__restrict__ wfrag,
                                                       const __nv_bfloat16 *__restrict__ in,
                                                       const float *__restrict__ bias, float *__restrict__ z,
                                                       int ntiles)
{
    extern __shared__ uint4 sw[];
    constexpr int NW = 27 * CB * MT * 32;
    for (int i = threadIdx.x; i < NW; i += blockDim.x) sw[i] = wfrag[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int nxy = nx * ny;
    constexpr int CI = CB * 16, CO = MT * 16;
    for (int tile = blockIdx.x * 4 + warp; tile < ntiles; tile += gridDim.x * 4) {
        const int node0 = tile * 32;
        const int zc = node0 / nxy;
        const int rem = node0 - zc * nxy;
        const int yc = rem / nx;
        const int x0 = rem - yc * nx;
        float acc[MT][4][4];
#pragma unroll
        for (int m = 0; m < MT; ++m)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[m][j][0] = acc[m][j][1] = acc[m][j][2] = acc[m][j][3] = 0.0f;
#pragma unroll 1
        for (int k = 0; k < 27; ++k) {
            const int dz = k / 9 - 1, dy = (k / 3) % 3 - 1, dx = k % 3 - 1;
            const int row = (cwrap(zc + dz, nz) * ny + cwrap(yc + dy, ny)) * nx;
            int nb[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) nb[j] = row + cwrap(x0 + 8 * j + g + dx, nx);
#pragma unroll
            for (int cb = 0; cb < CB; ++cb) {
                uint32_t b[4][2];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t *p = reinterpret_cast<const uint32_t *>(in + (size_t)nb[j] * CI + cb * 16);
                    b[j][0] = __ldg(p + t);       // channels 2t, 2t+1 of the chunk
                    b[j][1] = __ldg(p + t + 4);   // channels 2t+8, 2t+9
                }
#pragma unroll
                for (int m = 0; m < MT; ++m) {
                    const uint4 a = sw[((k * CB + cb) * MT + m) * 32 + lane];
#pragma unroll
                    for (int j = 0; j < 4; ++j) mma_bf16(acc[m][j], a, b[j][0], b[j][1]);
                }
            }
        }
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            const int o = m * 16 + g;
            const float b0 = bias ? bias[o] : 0.0f, b1 = bias ? bias[o + 8] : 0.0f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const size_t n = (size_t)node0 + 8 * j + 2 * t;
                z[n * CO + o] = acc[m][j][0] + b0;
                z[(n + 1) * CO + o] = acc[m][j][1] + b0;
                z[n * CO + o + 8] = acc[m][j][2] + b1;
                z[(n + 1) * CO + o + 8] = acc[m][j][3] + b1;
            }
        }
    }
}

// ---- the same convolution with the input tile staged in shared memory ----------------------
//
// A block owns a 32 x 8 column tile of nodes (one x row of 32 nodes per warp) and marches a z
// chunk.  The tile's halo-1 plane (34 x 10 nodes, all input channels, channel stride padded by 8
// so that the eight 16-byte rows an ldmatrix reads fall in distinct banks) lives in a 4-slot ring
// of shared-memory planes filled by cp.async two planes ahead; each B fragment pair is one
// ldmatrix.x4 (8 nodes x 16 channels of two n8 tiles).  The MMAs and their order are those of
// conv_mma_kernel, so both kernels give the same result bit for bit.

constexpr int CT_TY = 8;                 // y rows per block, one per warp
constexpr int CT_HX = 34, CT_HY = CT_TY + 2;
constexpr int CT_SLOTS = 4;

template <int CB>
struct CtGeom {
    static constexpr int CI = CB * 16;
    static constexpr int CS = CI + 8;                 // staged channel stride (bf16)
    static constexpr int PLANE = CT_HY * CT_HX * CS;  // bf16 per staged plane
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// every cp.async group of this thread but the most recent one is complete
__device__ __forceinline__ void cp_async_wait_but_last() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const uint32_t l = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t h = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return l | (h << 16);
}

// silu(z) = z / (1 + e^-z) with the fast division (every kernel evaluates it through this function)
__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

// wait until at most N of this thread's most recent cp.async groups are still pending
template <int N>
__device__ __forceinline__ void cp_async_wait_group()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void *smem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(sa));
}

__device__ __forceinline__ int mwrap(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// stage plane p (any integer z; wrapped) of the halo-1 tile at (x0, y0) into a slot
template <int CB>
__device__ __forceinline__ void ct_load_plane(__nv_bfloat16 *slot, const __nv_bfloat16 *__restrict__ in, int nx,
                                              int ny, int nz, int x0, int y0, int p)
{
    using Gm = CtGeom<CB>;
    constexpr int CHUNKS = Gm::CI / 8;   // 16-byte chunks per node
    const size_t plane = (size_t)mwrap(p, nz) * nx * ny;
    for (int e = threadIdx.x; e < CT_HY * CT_HX * CHUNKS; e += blockDim.x) {
        const int chunk = e % CHUNKS, node = e / CHUNKS;
        const int hy = node / CT_HX, hx = node - hy * CT_HX;
        const size_t src = plane + (size_t)mwrap(y0 - 1 + hy, ny) * nx + mwrap(x0 - 1 + hx, nx);
        cp_async16(slot + (size_t)(hy * CT_HX + hx) * Gm::CS + chunk * 8, in + src * Gm::CI + chunk * 8);
    }
}

template <int MT, int CB>
__global__ void __launch_bounds__(256) conv_tile_kernel(int nx, int ny, int nz, const uint4 *__restrict__ wfrag,
                                                        const __nv_bfloat16 *__restrict__ in,
                                                        const float *__restrict__ bias, float *__restrict__ z,
                                                        int zlen)
{
    using Gm = CtGeom<CB>;
    extern __shared__ uint4 smem[];
    constexpr int NW = 27 * CB * MT * 32;
    constexpr int CO = MT * 16;
    uint4 *sw = smem;
    __nv_bfloat16 *win = reinterpret_cast<__nv_bfloat16 *>(smem + NW);
    const int ntx = nx / 32;
    const int x0 = (blockIdx.x % ntx) * 32, y0 = (blockIdx.x / ntx) * CT_TY;
    const int z0 = blockIdx.y * zlen, z1 = min(nz, z0 + zlen);
    if (z0 >= nz) return;   // whole block
    for (int i = threadIdx.x; i < NW; i += blockDim.x) sw[i] = wfrag[i];
    auto slot = [&](int p) { return win + (size_t)((p - (z0 - 1)) & (CT_SLOTS - 1)) * Gm::PLANE; };
#pragma unroll 1
    for (int j = 0; j < 3; ++j) ct_load_plane<CB>(slot(z0 - 1 + j), in, nx, ny, nz, x0, y0, z0 - 1 + j);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3, q = lane >> 3, r = lane & 7;
    const int yout = y0 + warp;
#pragma unroll 1
    for (int zc = z0; zc < z1; ++zc) {
        if (zc + 2 <= z1) ct_load_plane<CB>(slot(zc + 2), in, nx, ny, nz, x0, y0, zc + 2);
        cp_async_commit();
        float acc[MT][4][4];
#pragma unroll
        for (int m = 0; m < MT; ++m)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[m][j][0] = acc[m][j][1] = acc[m][j][2] = acc[m][j][3] = 0.0f;
#pragma unroll 1
        for (int k = 0; k < 27; ++k) {
            const int dz = k / 9 - 1, dy = (k / 3) % 3 - 1, dx = k % 3 - 1;
            const __nv_bfloat16 *pl = slot(zc + dz) + (size_t)(warp + 1 + dy) * CT_HX * Gm::CS;
#pragma unroll
            for (int cb = 0; cb < CB; ++cb) {
                uint32_t b[4][2];
#pragma unroll
                for (int jj = 0; jj < 2; ++jj) {
                    const int hx = 8 * (2 * jj + (q >> 1)) + r + 1 + dx;
                    uint32_t rr[4];
                    ldmatrix_x4(rr, pl + (size_t)hx * Gm::CS + cb * 16 + 8 * (q & 1));
                    b[2 * jj][0] = rr[0];
                    b[2 * jj][1] = rr[1];
                    b[2 * jj + 1][0] = rr[2];
                    b[2 * jj + 1][1] = rr[3];
                }
#pragma unroll
                for (int m = 0; m < MT; ++m) {
                    const uint4 a = sw[((k * CB + cb) * MT + m) * 32 + lane];
#pragma unroll
                    for (int j = 0; j < 4; ++j) mma_bf16(acc[m][j], a, b[j][0], b[j][1]);
                }
            }
        }
        if (yout < ny) {
            const size_t node0 = ((size_t)zc * ny + yout) * nx + x0;
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                const int o = m * 16 + g;
                const float b0 = bias ? bias[o] : 0.0f, b1 = bias ? bias[o + 8] : 0.0f;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const size_t n = node0 + 8 * j + 2 * t;
                    z[n * CO + o] = acc[m][j][0] + b0;
                    z[(n + 1) * CO + o] = acc[m][j][1] + b0;
                    z[n * CO + o + 8] = acc[m][j][2] + b1;
                    z[(n + 1) * CO + o + 8] = acc[m][j][3] + b1;
                }
            }
        }
        cp_async_wait_all();
        __syncthreads();
    }
}

// ---- the same convolution on the 5th-generation tensor cores (tcgen05, TMEM) ---------------
//
// GEMM orientation: one tcgen05.mma (kind::f16: BF16 operands, FP32 accumulation in TMEM) computes
//   D[n][(jb, o)] += sum_i a_zi[n + (dx, dy)][i] W[o][i][dx, dy, dz = 1 - jb]
// with M = 128 nodes n (an 8 x 16 x-by-y patch of input plane zi), K = 16 input channels at one
// in-plane offset (dx, dy), and N = 3 CO: the three z offsets of the stencil side by side.  Column
// block jb of the result is input plane zi's contribution to output plane zi - 1 + jb, so each
// staged input plane is read by the tensor core once, for all 27 taps, and the weights are three
// times wider per instruction than with one z offset at a time.  That matters because both
// operands come from shared memory: with N = CO = 32 an MMA reads 5 KB for 64 Ki MACs, more bytes
// per cycle than shared memory delivers; with N = 96 it reads 7 KB for 192 Ki MACs.
//   A: the block's halo tile, staged channel-group-major ([channel group of 8][hy][hx][8]), so the
//      8 x-consecutive nodes of a patch row are one 8 x 16-byte core matrix; patch rows are SBO =
//      HX * 16 bytes apart, the two channel groups of a K step LBO = HY * HX * 16 bytes apart, and an
//      in-plane offset (dx, dy) only moves the start address (K-major, unswizzled descriptors);
//   B: the weights, [(dx, dy)][channel chunk][group of 8 channels][(jb, o)][8] (LBO = 3 CO * 16,
//      SBO = 128); a sub-range of the z blocks is a sub-range of rows.
//   D: per patch, a ring of UM_ACC output planes of CO columns each; the three column blocks of an
//      MMA are three consecutive planes of the ring (an MMA that would wrap is split in two).
//      Block 2 is always the first write of output plane zi + 1: the first MMA of each input plane
//      issues it separately with accumulation off, so no accumulator is ever cleared.
// A block owns a 16 x 16 column tile (two patches) and marches a z chunk z0 .. z1 - 1 over input
// planes z0 - 1 .. z1 (at the chunk's ends only the blocks that land inside it are issued), with
// warps in two roles that hand work to each other through mbarriers:
//   warps 8, 9 (the MMA warps, one per patch): one thread of each issues input plane zi's MMAs
//     (9 offsets x CB channel chunks, fully unrolled; descriptors are precomputed words plus
//     compile-time offsets) as soon as the plane is staged and, when the MMAs open a new output
//     plane, that plane's accumulator slot has been read back; then commits them to the "empty"
//     barrier of the plane's staging slot and to the "done" barrier of output plane zi - 1;
//   warps 0..7 (load and epilogue): read back output plane p when its barrier completes
//     (tcgen05.ld; warp w owns TMEM lanes 32 (w % 4) .. + 31 = patch rows 4 (w % 4) .. + 3 and half
//     w / 4 of the output channels), report the slot drained, add the bias and store z (when
//     kept) and, for the forward pass, the next layer's input silu(z) in BF16; then stage the input
//     planes whose slots the consumed planes freed (cp.async; the copies are waited for, fenced for
//     the async proxy and reported "full" one iteration later, after that iteration's stores).
// The MMAs of later planes run while the epilogue drains and the staging is in flight, and no
// barrier of the whole block sits on the per-plane path.  The weights are staged with cp.async as
// well.  Every mbarrier wait is bounded in time: on expiry the kernel records an error, every role
// stops at its next wait, the MMA threads wait once more for the MMAs they committed, the copies in
// flight are waited for and the TMEM is released.

constexpr int UM_TX = 16, UM_TY = 16;              // column tile: two 8 x 16 patches
constexpr int UM_HX = UM_TX + 2, UM_HY = UM_TY + 2;
constexpr int UM_SLOTS = 6;                        // ring of staged input planes
// planes are reported staged one epilogue iteration after their copies are issued, and output
// plane z0 + 1 needs input plane z0 + 2 before the first such report: the prologue's planes
// z0 - 1 .. z0 + 2 must fit the ring
static_assert(UM_SLOTS >= 4, "staging ring too short: the pipeline would wait on itself");
// ring of output-plane accumulators per patch (TMEM): 8 planes, or 4 where the block's shared
// memory lets two blocks share an SM (CB = 1), so that two blocks' allocations fit the 512 columns
template <int CB>
__host__ __device__ constexpr int um_acc() { return CB == 1 ? 4 : 8; }
// Bounds of the mbarrier waits, in nanoseconds of %globaltimer: a plane's MMAs take about a
// microsecond, so a wait still open after 20 ms has failed; the test hook's wait gives up after
// 20 us.  Time bounds, unlike poll counts, do not depend on how long each poll suspends.
constexpr unsigned long long UM_WAIT_NS = 20000000ull;
constexpr unsigned long long UM_TEST_WAIT_NS = 20000ull;

template <int CB>
struct UmGeom {
    static constexpr int CG = CB * 2;                              // groups of 8 input channels
    static constexpr int PLANE_BYTES = CG * UM_HY * UM_HX * 16;    // one staged plane
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major, unswizzled shared-memory matrix descriptor (sm_100 layout: start >> 4, LBO >> 4,
// SBO >> 4, descriptor version 1)
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits until the phase of parity `parity` of the mbarrier has completed; false once limit_ns
// nanoseconds have passed without that, or (abort not null) once *abort is set.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, unsigned long long limit_ns = UM_WAIT_NS,
                                          const volatile int *abort = nullptr)
{
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((abort && *abort) || globaltimer_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_addr(bar))
                 : "memory");
}

template <int CB>
__device__ __forceinline__ void um_load_plane(uint8_t *slot, const __nv_bfloat16 *__restrict__ in, int nx, int ny,
                                              int nz, int x0, int y0, int p)
{
    constexpr int CG = UmGeom<CB>::CG;
    const size_t plane = (size_t)mwrap(p, nz) * nx * ny;
    for (int e = threadIdx.x; e < CG * UM_HY * UM_HX; e += blockDim.x) {
        const int node = e % (UM_HY * UM_HX), cg = e / (UM_HY * UM_HX);
        const int hy = node / UM_HX, hx = node - hy * UM_HX;
        const size_t src = plane + (size_t)mwrap(y0 - 1 + hy, ny) * nx + mwrap(x0 - 1 + hx, nx);
        cp_async16(slot + (size_t)e * 16, in + src * (CB * 16) + cg * 8);
    }
}

// z[n][o] = bias[o] + sum_{k, i} W[o][i][k] in[n + off_k][i], CO = MT * 16 output channels (padded),
// CB * 16 input channels (padded); wpack: [9][CB][2][3 CO][8] BF16 (pack_weights_umma_kernel).
// z is written when keep_z != 0 or act is null; act (not null): the next layer's input silu(z);
// ycf (not null, the last layer): also its first 4 channels channel-first, ycf[c][n].
constexpr int UM_EPI_WARPS = 8;                          // load and epilogue warps
constexpr int UM_MMA_WARPS = 2;                          // MMA warps: one per patch
constexpr int UM_THREADS = 32 * (UM_EPI_WARPS + UM_MMA_WARPS);
constexpr int UM_EPI_THREADS = 32 * UM_EPI_WARPS;

template <int MT, int CB, bool XF>
__global__ void __launch_bounds__(UM_THREADS, 1) conv_umma_kernel(int nx, int ny, int nz, const __nv_bfloat16 *__restrict__ wpack,
                                                           const __nv_bfloat16 *__restrict__ in,
                                                           const float *__restrict__ bias, float *__restrict__ z,
                                                           __nv_bfloat16 *__restrict__ act, float *__restrict__ ycf,
                                                           int zlen, int *__restrict__ err, int stall, int keep_z)
{
    constexpr int CO = MT * 16;
    constexpr int ROWS = 3 * CO;                       // B rows (jb, o)
    // in-plane taps per plane: 9 (dx, dy), or 3 (dy) when the input carries its x neighbours in
    // its channels (XF: the first layer's folded input, pack_input_kernel)
    constexpr int JT = XF ? 3 : 9;
    static_assert(!XF || CB == 1, "the folded input has one 16-channel chunk");
    constexpr int WBYTES = JT * CB * 2 * ROWS * 16;
    constexpr int PB = UmGeom<CB>::PLANE_BYTES;
    constexpr int CG = UmGeom<CB>::CG;
    constexpr int UM_ACC = um_acc<CB>();
    constexpr uint32_t TCOLS = 2 * UM_ACC * CO;        // 2 patches x UM_ACC planes x CO columns
    static_assert(TCOLS == 256 || TCOLS == 512, "TMEM allocation is a power of two");
    extern __shared__ __align__(1024) uint8_t usm[];
    __shared__ __align__(8) uint64_t bar_full[UM_SLOTS];     // an input plane is staged in the slot
    __shared__ __align__(8) uint64_t bar_empty[UM_SLOTS];    // the MMAs reading the slot are done
    __shared__ __align__(8) uint64_t bar_acc[UM_ACC];        // the accumulator slot holds a finished plane
    __shared__ __align__(8) uint64_t bar_drained[UM_ACC];    // the accumulator slot has been read back
    __shared__ __align__(8) uint64_t bar_fin;                // every MMA this block committed is done
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ float sbias[CO];
    uint8_t *sw = usm;
    uint8_t *ring = usm + ((WBYTES + 1023) / 1024) * 1024;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntx = nx / UM_TX;
    const int x0 = (blockIdx.x % ntx) * UM_TX, y0 = (blockIdx.x / ntx) * UM_TY;
    const int z0 = blockIdx.y * zlen, z1 = min(nz, z0 + zlen);
    pdl_trigger();          // the next kernel may be scheduled; it waits for this one before its loads
    if (z0 >= nz) return;   // whole block
    volatile int *abort_v = &abort_flag;

    // input planes z0 - 1 .. z1 take the staging slots in turn: slot and fill number of plane p
    auto slot_of = [&](int p) { return (p - (z0 - 1)) % UM_SLOTS; };
    auto fill_of = [&](int p) { return (p - (z0 - 1)) / UM_SLOTS; };
    auto slot = [&](int p) { return ring + (size_t)slot_of(p) * PB; };
    // output planes z0 .. z1 - 1 take the accumulator slots in turn: slot and use number of plane q
    auto aslot = [&](int q) { return (q - z0) % UM_ACC; };
    auto ause = [&](int q) { return (q - z0) / UM_ACC; };
    // the 16-byte chunks this epilogue thread stages in every plane: element offsets within a plane
    // of the input (wrapped once here; -1 past the end) and byte offsets within the slot.  Chunk
    // e = node * CG + cg, the channel group fastest, so that a warp copies the 8 x 64 contiguous
    // bytes of 8 x-consecutive nodes (4 lines per instruction, not 32) and writes the 8 nodes x 4
    // groups to every shared-memory bank exactly 4 times (the groups are HY * HX * 16 bytes apart,
    // 16 banks mod 32)
    constexpr int NCHUNK = CG * UM_HY * UM_HX;
    constexpr int PER = (NCHUNK + UM_EPI_THREADS - 1) / UM_EPI_THREADS;
    int soff[PER], doff[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int e = tid + j * UM_EPI_THREADS;
        const int node = e / CG, cg = e - node * CG;
        const int hy = node / UM_HX, hx = node - hy * UM_HX;
        const bool mine = e < NCHUNK && tid < UM_EPI_THREADS;
        soff[j] = mine ? (mwrap(y0 - 1 + hy, ny) * nx + mwrap(x0 - 1 + hx, nx)) * (CB * 16) + cg * 8 : -1;
        doff[j] = (cg * UM_HY * UM_HX + node) * 16;
    }
    auto stage = [&](int p) {   // cp.async copies of plane p by the epilogue threads (one group)
        const __nv_bfloat16 *src = in + (size_t)mwrap(p, nz) * nx * ny * (CB * 16);
        uint8_t *dst = slot(p);
#pragma unroll
        for (int j = 0; j < PER; ++j)
            if (soff[j] >= 0) cp_async16(dst + doff[j], src + soff[j]);
        cp_async_commit();
    };

    if (tid == 0) {
        abort_flag = 0;
        for (int q = 0; q < UM_SLOTS; ++q) {
            mbar_init(&bar_full[q], UM_EPI_THREADS);
            mbar_init(&bar_empty[q], UM_MMA_WARPS);
        }
        for (int q = 0; q < UM_ACC; ++q) {
            mbar_init(&bar_acc[q], UM_MMA_WARPS);
            mbar_init(&bar_drained[q], UM_EPI_WARPS);
        }
        mbar_init(&bar_fin, UM_MMA_WARPS);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_base)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();   // barriers initialised and the TMEM address visible before any other step
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;

    // prologue (epilogue threads): the weights and bias (written before the previous kernel of the
    // stream, so they are read before waiting for it), then the first UM_SLOTS input planes (that
    // kernel's output).  Group 0 holds the weights and plane z0 - 1, group j plane z0 - 1 + j; a
    // plane is reported full as soon as its group has landed, with the next one already in flight,
    // so the MMAs start after the first group rather than after the whole prologue.
    const int npro = min(UM_SLOTS, z1 - z0 + 2);
    if (tid < UM_EPI_THREADS) {
        for (int i = tid; i < WBYTES / 16; i += UM_EPI_THREADS) cp_async16(sw + (size_t)i * 16, wpack + (size_t)i * 8);
        if (tid < CO) sbias[tid] = bias ? bias[tid] : 0.0f;
        pdl_wait();
        stage(z0 - 1);
        for (int j = 1; j <= npro; ++j) {
            if (j < npro) {
                stage(z0 - 1 + j);
                cp_async_wait_but_last();
            } else {
                cp_async_wait_all();
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            mbar_arrive(&bar_full[slot_of(z0 - 2 + j)]);
        }
        asm volatile("bar.sync 1, %0;\n" ::"n"(UM_EPI_THREADS) : "memory");   // sbias visible to the epilogue
    }

    if (warp >= UM_EPI_WARPS) {
        // ---- MMA warps: warp UM_EPI_WARPS + pt issues the MMAs of patch pt ---------------------
        const int pt = warp - UM_EPI_WARPS;
        // instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M = 128, N = nb CO
        const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 4) << 24);
        auto idesc = [&](int nb) { return idesc0 | ((uint32_t)((nb * CO) >> 3) << 17); };
        const uint32_t lbo_a = UM_HY * UM_HX * 16, sbo_a = UM_HX * 16;
        const uint32_t lbo_b = ROWS * 16, sbo_b = 128;
        const uint64_t bdesc = umma_desc(smem_addr(sw), lbo_b, sbo_b);
        const uint32_t a_hi = (uint32_t)(umma_desc(0, lbo_a, sbo_a) >> 32);
        const uint32_t b_lo = (uint32_t)bdesc, b_hi = (uint32_t)(bdesc >> 32);
        const uint32_t tpatch = tmem + (uint32_t)(pt * UM_ACC * CO);   // this patch's accumulator ring
        bool ok = true;
        if (stall) {   // test hook: wait (briefly) on a barrier nothing is committed to, before any MMA
            ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(&bar_fin), 0u, UM_TEST_WAIT_NS));
            if (!ok && lane == 0) abort_flag = 1;
            ok = false;
        }
        for (int zi = z0 - 1; zi <= z1 && ok; ++zi) {
            // column blocks lo..hi of this input plane land in output planes zi - 1 + jb of the chunk
            const int lo = max(0, z0 - zi + 1), hi = min(2, z1 - zi);
            bool good = mbar_wait(smem_addr(&bar_full[slot_of(zi)]), (uint32_t)(fill_of(zi) & 1), UM_WAIT_NS, abort_v);
            // block 2 opens output plane zi + 1: the plane before it in that slot must be read back
            if (good && hi == 2 && zi + 1 - z0 >= UM_ACC)
                good = mbar_wait(smem_addr(&bar_drained[aslot(zi + 1)]), (uint32_t)((ause(zi + 1) - 1) & 1),
                                 UM_WAIT_NS, abort_v);
            good = __all_sync(0xffffffffu, good);
            if (!good) {
                if (lane == 0) abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            if (lane == 0) {
                const uint32_t a_lo = (uint32_t)umma_desc(smem_addr(slot(zi)), lbo_a, sbo_a);
                // blocks lo..hi split where the ring of accumulator slots wraps: segments [b0, b1]
                // starting at accumulator slot sa
                const int s_lo = aslot(zi - 1 + lo);
                const int n1 = min(hi - lo + 1, UM_ACC - s_lo);
                const int seg_b0[2] = {lo, lo + n1}, seg_b1[2] = {lo + n1 - 1, hi}, seg_sa[2] = {s_lo, 0};
                const int nseg = lo + n1 <= hi ? 2 : 1;
#pragma unroll
                for (int j = 0; j < JT * CB; ++j) {   // j = (in-plane offset) * CB + channel chunk
                    const int j9 = j / CB, cb = j % CB;
                    const int dy = XF ? j9 - 1 : j9 / 3 - 1, dx = XF ? 0 : j9 % 3 - 1;
                    const uint32_t aoff = (uint32_t)((1 + dy) * UM_HX + pt * 8 + 1 + dx) +
                                          (uint32_t)(2 * cb) * (lbo_a >> 4);   // 16-byte units
                    const uint64_t da = ((uint64_t)a_hi << 32) | (a_lo + aoff);
                    const uint32_t bj = b_lo + (uint32_t)(j * 2 * ROWS);          // 16-byte units
                    for (int sg = 0; sg < nseg; ++sg) {
                        const int b0 = seg_b0[sg], b1 = seg_b1[sg];
                        const uint32_t dcol = tpatch + (uint32_t)(seg_sa[sg] * CO);
                        if (j == 0 && b1 == 2) {   // plane zi + 1's first write: accumulation off for block 2
                            if (b0 < 2)
                                umma_bf16(dcol, da, ((uint64_t)b_hi << 32) | (bj + (uint32_t)(b0 * CO)), idesc(2 - b0), 1u);
                            umma_bf16(dcol + (uint32_t)((2 - b0) * CO), da, ((uint64_t)b_hi << 32) | (bj + 2u * CO),
                                      idesc(1), 0u);
                        } else {
                            umma_bf16(dcol, da, ((uint64_t)b_hi << 32) | (bj + (uint32_t)(b0 * CO)), idesc(b1 - b0 + 1),
                                      1u);
                        }
                    }
                }
                umma_commit(&bar_empty[slot_of(zi)]);                 // no later MMA reads input plane zi
                if (zi - 1 >= z0) umma_commit(&bar_acc[aslot(zi - 1)]);   // output plane zi - 1 is complete
            }
            __syncwarp();
        }
        // every committed MMA done before the TMEM and the ring are released
        if (lane == 0) umma_commit(&bar_fin);
        __syncwarp();
        const bool fin = __all_sync(0xffffffffu, mbar_wait(smem_addr(&bar_fin), 0u, UM_WAIT_NS));
        if (!fin && lane == 0) abort_flag = 1;
    } else {
        // ---- load and epilogue warps ----------------------------------------------------------
        constexpr int CH = CO / 2;
        const int q = warp & 3, h = warp >> 2;
        const int mrow = 32 * q + lane;                // patch row index: node (mrow % 8, mrow / 8)
        const int yy = y0 + mrow / 8;
        float bv[CH];                                  // this warp's half of the bias, in registers
#pragma unroll
        for (int o = 0; o < CH; ++o) bv[o] = sbias[h * CH + o];
        int staged = z0 - 1 + npro;                    // next input plane to stage
        int reported = staged;                         // planes reported .. staged - 1 are in flight
        bool aborted = false;                          // this warp gave up at a wait
        for (int p = z0; p < z1; ++p) {
            const int sa = aslot(p);
            aborted = !__all_sync(0xffffffffu, mbar_wait(smem_addr(&bar_acc[sa]), (uint32_t)(ause(p) & 1),
                                                         UM_WAIT_NS, abort_v));
            if (aborted) {
                if (lane == 0) abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            uint32_t r[2][CH];
#pragma unroll
            for (int pt = 0; pt < 2; ++pt) {
                const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((pt * UM_ACC + sa) * CO + h * CH);
                uint32_t(&rr)[CH] = r[pt];
                if constexpr (CH == 16) {
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                        "[%16];\n"
                        : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]),
                          "=r"(rr[7]), "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]),
                          "=r"(rr[13]), "=r"(rr[14]), "=r"(rr[15])
                        : "r"(taddr));
                } else {
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                                 : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]),
                                   "=r"(rr[6]), "=r"(rr[7])
                                 : "r"(taddr));
                }
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_drained[sa]);   // the MMA warps may reuse the slot
            if (yy < ny) {
#pragma unroll
                for (int pt = 0; pt < 2; ++pt) {
                    const size_t node = ((size_t)p * ny + yy) * nx + x0 + pt * 8 + (mrow % 8);
                    float v[CH];
#pragma unroll
                    for (int o = 0; o < CH; ++o) v[o] = __uint_as_float(r[pt][o]) + bv[o];
                    if (ycf && h == 0) {   // the network's output, channel-first: y[c][node], c < 4
                        const size_t nn = (size_t)nx * ny * nz;
#pragma unroll
                        for (int o = 0; o < 4; ++o) ycf[(size_t)o * nn + node] = v[o];
                    }
                    if (keep_z || !act) {
                        float4 *dst = reinterpret_cast<float4 *>(z + node * CO + h * CH);
#pragma unroll
                        for (int o = 0; o < CH; o += 4) dst[o / 4] = make_float4(v[o], v[o + 1], v[o + 2], v[o + 3]);
                    }
                    if (act) {   // the next layer's input, silu(z) in BF16
                        uint4 *ad = reinterpret_cast<uint4 *>(act + node * CO + h * CH);
#pragma unroll
                        for (int o = 0; o < CH; o += 8)
                            ad[o / 8] = make_uint4(pack_bf16(silu(v[o]), silu(v[o + 1])),
                                                   pack_bf16(silu(v[o + 2]), silu(v[o + 3])),
                                                   pack_bf16(silu(v[o + 4]), silu(v[o + 5])),
                                                   pack_bf16(silu(v[o + 6]), silu(v[o + 7])));
                    }
                }
            }
            // staging: report the planes staged last iteration (their copies had this iteration's
            // stores to land), then, output plane p being done, input planes up to p + 1 have been
            // consumed and their slots take input planes up to p + 1 + UM_SLOTS
            if (reported < staged) {
                cp_async_wait_all();
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                for (; reported < staged; ++reported) mbar_arrive(&bar_full[slot_of(reported)]);
            }
            while (staged <= z1 && staged <= p + 1 + UM_SLOTS) {
                aborted = !__all_sync(0xffffffffu, mbar_wait(smem_addr(&bar_empty[slot_of(staged)]),
                                                             (uint32_t)((fill_of(staged) - 1) & 1), UM_WAIT_NS, abort_v));
                if (aborted) break;
                stage(staged);
                ++staged;
            }
            if (aborted) {
                if (lane == 0) abort_flag = 1;
                break;
            }
        }
        if (reported < staged && !aborted) {
            cp_async_wait_all();
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            for (; reported < staged; ++reported) mbar_arrive(&bar_full[slot_of(reported)]);
        }
        cp_async_wait_all();   // no copy of this block is still in flight when it returns
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (abort_flag && tid == 0) atomicExch(err, 1);
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS));
}

// Weights for conv_umma_kernel: [9 in-plane offsets][CB][2][rows (jb, o): 3 CO][8] BF16.  Row
// (jb, o) of in-plane offset j9 = 3 (dy + 1) + (dx + 1) holds the tap of z offset dz = 1 - jb,
// k = 9 (2 - jb) + j9: value(o, i, k) = W[o][i][k], or for the input gradient (transpose)
// W[i][o][26 - k]; zero for padded rows or channels.  xfold (the first layer, forward): 3 in-plane
// offsets j9 = dy + 1, channel i = 5 dx' + c of the folded input holding tap k = 9 (2 - jb) + 3 j9
// + dx' of channel c (dx' = dx + 1), channel 15 zero.
__global__ void pack_weights_umma_kernel(const float *__restrict__ W, int cout, int cin, int co_pad, int cb_count,
                                         bool transpose, bool xfold, __nv_bfloat16 *__restrict__ out)
{
    const int rows3 = 3 * co_pad;
    const int total = (xfold ? 3 : 9) * cb_count * 2 * rows3 * 8;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int e = idx % 8, r = (idx / 8) % rows3, cg = (idx / (8 * rows3)) % 2;
    const int jc = idx / (16 * rows3);
    const int cb = jc % cb_count, j9 = jc / cb_count;
    const int jb = r / co_pad, o = r % co_pad;
    const int i = cb * 16 + cg * 8 + e;
    float v = 0.0f;
    if (xfold) {
        if (o < cout && i < 15) v = W[((size_t)o * cin + i % 5) * 27 + 9 * (2 - jb) + 3 * j9 + i / 5];
    } else {
        const int k = 9 * (2 - jb) + j9;
        const int rows = transpose ? cin : cout, cols = transpose ? cout : cin;
        if (o < rows && i < cols)
            v = transpose ? W[((size_t)i * cin + o) * 27 + (26 - k)] : W[((size_t)o * cin + i) * 27 + k];
    }
    out[idx] = __float2bfloat16_rn(v);
}


// Fragment-ordered BF16 weights of one layer from the FP32 master W[o][i][k] (cout x cin x 27).
// TRANSPOSE builds the weights of the backward pass with respect to the input,
// Wt[i][o][k] = W[o][i][26 - k], so that the same convolution kernel computes
// da[n][i] = sum_{k, o} W[o][i][k] dz[n - off_k][o].
__global__ void pack_weights_kernel(const float *__restrict__ W, int cout, int cin, int mt_count, int cb_count,
                                    bool transpose, bool xfold, uint4 *__restrict__ frag)
{
    const int total = 27 * cb_count * mt_count * 32;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int lane = idx & 31;
    const int m = (idx >> 5) % mt_count;
    const int kc = (idx >> 5) / mt_count;
    const int k = kc / cb_count, cb = kc % cb_count;
    const int g = lane >> 2, t = lane & 3;
    // the GEMM's (row, col) = (output channel, input channel) of this layer or of its transpose
    const int rows = transpose ? cin : cout, cols = transpose ? cout : cin;
    auto w = [&](int r, int c) -> float {
        if (xfold) {   // folded first-layer input: only the dx = 0 taps, carrying all three x taps
            if (r >= cout || c >= 15 || k % 3 != 1) return 0.0f;
            return W[((size_t)r * cin + c % 5) * 27 + (k - 1 + c / 5)];
        }
        if (r >= rows || c >= cols) return 0.0f;
        return transpose ? W[((size_t)c * cin + r) * 27 + (26 - k)] : W[((size_t)r * cin + c) * 27 + k];
    };
    const int r0 = m * 16 + g, c0 = cb * 16 + 2 * t;
    uint4 f;
    f.x = pack_bf16(w(r0, c0), w(r0, c0 + 1));
    f.y = pack_bf16(w(r0 + 8, c0), w(r0 + 8, c0 + 1));
    f.z = pack_bf16(w(r0, c0 + 8), w(r0, c0 + 9));
    f.w = pack_bf16(w(r0 + 8, c0 + 8), w(r0 + 8, c0 + 9));
    frag[idx] = f;
}

// ---- elementwise stages -------------------------------------------------------------------

__device__ __forceinline__ float silu_grad(float z)
{
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// x [5][N] (channel-first FP32) -> a0 [N][16] channel-last BF16 with the node's x neighbours
// folded into the channels: a0[n][5 dx + c] = x[c][n + (dx - 1) e_x] (periodic in x) for dx = 0..2,
// channel 15 zero.  The first layer then takes its three x taps of one (dy, dz) offset in one
// 16-channel step (3 tensor-core steps per plane rather than 9 steps of 5 real channels in 16).
__global__ void pack_input_kernel(const float *__restrict__ x, int nx, int N, __nv_bfloat16 *__restrict__ a0)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int xx = n % nx, row = n - xx;
    float f[16];
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
        const size_t src = (size_t)row + mwrap(xx + dx - 1, nx);
#pragma unroll
        for (int c = 0; c < 5; ++c) f[5 * dx + c] = x[(size_t)c * N + src];
    }
    f[15] = 0.0f;
    uint32_t v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = pack_bf16(f[2 * c], f[2 * c + 1]);
    uint4 *d = reinterpret_cast<uint4 *>(a0 + (size_t)n * 16);
    d[0] = make_uint4(v[0], v[1], v[2], v[3]);
    d[1] = make_uint4(v[4], v[5], v[6], v[7]);
}

// bpad[o] = bias[o] for o < cout, 0 up to 32 (one block of 32 threads)
__global__ void pad_bias_kernel(const float *__restrict__ bias, int cout, float *__restrict__ bpad)
{
    bpad[threadIdx.x] = (int)threadIdx.x < cout ? bias[threadIdx.x] : 0.0f;
}

// a = silu(z), z and a channel-last with C channels (count = N * C)
__global__ void silu_kernel(const float *__restrict__ z, size_t count, __nv_bfloat16 *__restrict__ a)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) a[i] = __float2bfloat16_rn(silu(z[i]));
}

// dz = da * silu'(z) (FP32 and its BF16 copy), count = N * C
// dz = da silu'(z) on [N][32] channel-last (FP32, and BF16 for the weight gradient), in float4
// groups q = 8 n + g (channels 4 g .. 4 g + 3 of node n), grid-stride with a stride that is a
// multiple of 8, so each thread keeps one channel group; and the bias gradient's per-block partial
// sums part[block][32] of the new dz: each thread adds its groups in order, then thread c adds the
// block's 32 per-thread sums of channel c in order (deterministic, no second pass over dz).
constexpr int kBackBlocks = 4 * 148;
__global__ void __launch_bounds__(256) silu_back_kernel(const float4 *__restrict__ da, const float4 *__restrict__ z,
                                                        size_t nq, float4 *__restrict__ dz, uint2 *__restrict__ dzb,
                                                        float *__restrict__ part)
{
    __shared__ float red[32][33];
    float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (size_t q = (size_t)blockIdx.x * 256 + threadIdx.x; q < nq; q += (size_t)gridDim.x * 256) {
        const float4 a = da[q], zz = z[q];
        const float4 v = make_float4(a.x * silu_grad(zz.x), a.y * silu_grad(zz.y), a.z * silu_grad(zz.z),
                                     a.w * silu_grad(zz.w));
        dz[q] = v;
        dzb[q] = make_uint2(pack_bf16(v.x, v.y), pack_bf16(v.z, v.w));
        s[0] += v.x;
        s[1] += v.y;
        s[2] += v.z;
        s[3] += v.w;
    }
    const int g = threadIdx.x & 7, m = threadIdx.x >> 3;   // channel group, and rank within it
#pragma unroll
    for (int c = 0; c < 4; ++c) red[m][4 * g + c] = s[c];
    __syncthreads();
    if (threadIdx.x < 32) {
        float tot = 0.0f;
        for (int r = 0; r < 32; ++r) tot += red[r][threadIdx.x];
        part[(size_t)blockIdx.x * 32 + threadIdx.x] = tot;
    }
}

// y [4][N] channel-first from the last layer's z [N][16]
__global__ void unpack_output_kernel(const float *__restrict__ z4, int N, float *__restrict__ y)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
#pragma unroll
    for (int c = 0; c < 4; ++c) y[(size_t)c * N + n] = z4[(size_t)n * 16 + c];
}

// Mean-squared loss over the 4 outputs and N nodes against t [4][N]; dz4 = 2 (y - t) / (4 N)
// (channels 4..15 zero, FP32 and BF16); per-block FP64 partial sums of (y - t)^2.
// Mean-squared-error loss over the 4 outputs: per-block FP64 partial sums of r^2 (partial), and
// dz = 2 r / (4 N) for channels 0..3 of z4 [N][16] (zero for the padded 4..15, FP32 and BF16),
// whose per-block sums part[block][0..3] are the last layer's bias gradient partials (in order:
// thread c < 4 adds the block's nodes in order; channels 4..31 of the record are zero).
__global__ void __launch_bounds__(256) loss_kernel(const float *__restrict__ z4, const float *__restrict__ t, int N,
                                                   float *__restrict__ dz, __nv_bfloat16 *__restrict__ dzb,
                                                   double *__restrict__ partial, float *__restrict__ part)
{
    __shared__ double red[256];
    __shared__ float gsh[256][5];
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    float g[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (n < N) {
        const float scale = 2.0f / (4.0f * (float)N);
        const float4 zz = reinterpret_cast<const float4 *>(z4)[(size_t)n * 4];
        const float zc[4] = {zz.x, zz.y, zz.z, zz.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float r = zc[c] - t[(size_t)c * N + n];
            s += (double)r * r;
            g[c] = scale * r;
        }
        float4 *d = reinterpret_cast<float4 *>(dz + (size_t)n * 16);
        d[0] = make_float4(g[0], g[1], g[2], g[3]);
        d[1] = d[2] = d[3] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        uint4 *db = reinterpret_cast<uint4 *>(dzb + (size_t)n * 16);
        db[0] = make_uint4(pack_bf16(g[0], g[1]), pack_bf16(g[2], g[3]), 0u, 0u);
        db[1] = make_uint4(0u, 0u, 0u, 0u);
    }
    red[threadIdx.x] = s;
#pragma unroll
    for (int c = 0; c < 4; ++c) gsh[threadIdx.x][c] = g[c];
    __syncthreads();
    if (threadIdx.x < 32) {
        float tot = 0.0f;
        if (threadIdx.x < 4)
            for (int r = 0; r < 256; ++r) tot += gsh[r][threadIdx.x];
        part[(size_t)blockIdx.x * 32 + threadIdx.x] = tot;
    }
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// ---- the weight gradient on the tensor cores -------------------------------------------------
//
// dW[o][i][k] = sum_n dz[n][o] a[n + off_k][i] as mma.sync m16n8k16 products with M = output
// channels o, N = input channels i and K = 16 nodes of one x row: the A operand dz^T and the B
// operand (the activations shifted by off_k) are both read from channel-last shared-memory tiles
// with transposing ldmatrix.  A block owns a 32 x 8 column tile, a z chunk and one z offset
// (blockIdx.y = dz + 1): per plane it stages dz of the plane (BF16, no halo) and the activation
// plane zc + dz with its one-node halo (the forward kernel's staging, ct_load_plane), double
// buffered with cp.async, and warp (m, n) accumulates the 9 offsets (dy, dx) of its 16 x 8
// output tile in registers and stores them as the block's partial sums; dw_reduce_kernel adds the
// partials of all blocks in a fixed order (the gradient is reproducible bit for bit).

__device__ __forceinline__ void ldmatrix_x4_trans(uint32_t (&r)[4], const void *smem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(sa));
}

__device__ __forceinline__ void ldmatrix_x2_trans(uint32_t (&r)[2], const void *smem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(sa));
}

// dz tile of one plane: 8 rows x 32 nodes, cop channels at stride cop + 8 (conflict-free ldmatrix
// rows); rows past ny are zero
template <int MT>
__device__ __forceinline__ void dw_load_dz(__nv_bfloat16 *dst, const __nv_bfloat16 *__restrict__ dzb, int nx, int ny,
                                           int x0, int y0, int zc)
{
    constexpr int COP = MT * 16, DS = COP + 8, CH = COP / 8;   // 16-byte chunks per node
    for (int e = threadIdx.x; e < CT_TY * 32 * CH; e += blockDim.x) {
        const int chunk = e % CH, node = e / CH;
        const int yr = node / 32, xr = node - yr * 32;
        __nv_bfloat16 *d = dst + (size_t)node * DS + chunk * 8;
        if (y0 + yr < ny)
            cp_async16(d, dzb + ((((size_t)zc * ny + y0 + yr) * nx + x0 + xr) * COP + chunk * 8));
        else
            *reinterpret_cast<uint4 *>(d) = make_uint4(0u, 0u, 0u, 0u);
    }
}

// partial sums of block (bx, bz) of z offset group gz: part[((gz * nblk + blk) * 9 + q) * 1024 + o * 32 + i]
// with blk = bz * gridDim.x + bx and q = 3 (dy + 1) + (dx + 1)
template <int MT, int CB>
__global__ void __launch_bounds__(256) dweight_mma_kernel(int nx, int ny, int nz, const __nv_bfloat16 *__restrict__ dzb,
                                                          const __nv_bfloat16 *__restrict__ a, int zlen,
                                                          float *__restrict__ part)
{
    using Gm = CtGeom<CB>;
    constexpr int COP = MT * 16, DS = COP + 8, NT = Gm::CI / 8;
    constexpr int DZB = CT_TY * 32 * DS;   // bf16 of one dz tile
    extern __shared__ uint4 dsm[];
    __nv_bfloat16 *act = reinterpret_cast<__nv_bfloat16 *>(dsm);   // 2 staged activation planes
    __nv_bfloat16 *dzs = act + 2 * Gm::PLANE;                       // 2 dz tiles
    const int ntx = nx / 32;
    const int x0 = (blockIdx.x % ntx) * 32, y0 = (blockIdx.x / ntx) * CT_TY;
    const int z0 = blockIdx.z * zlen, z1 = min(nz, z0 + zlen);
    const int dz = (int)blockIdx.y - 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool on = warp < MT * NT;
    const int m = warp / NT, n = warp % NT;
    float acc[9][4];
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.0f;

    ct_load_plane<CB>(act, a, nx, ny, nz, x0, y0, z0 + dz);
    dw_load_dz<MT>(dzs, dzb, nx, ny, x0, y0, z0);
    cp_async_commit();
#pragma unroll 1
    for (int zc = z0; zc < z1; ++zc) {
        const int b = (zc - z0) & 1;
        if (zc + 1 < z1) {   // the next plane into the other buffers
            ct_load_plane<CB>(act + (1 - b) * Gm::PLANE, a, nx, ny, nz, x0, y0, zc + 1 + dz);
            dw_load_dz<MT>(dzs + (1 - b) * DZB, dzb, nx, ny, x0, y0, zc + 1);
        }
        cp_async_commit();
        cp_async_wait_group<1>();
        __syncthreads();
        if (on) {
            const __nv_bfloat16 *pa = act + b * Gm::PLANE, *pd = dzs + b * DZB;
#pragma unroll 1
            for (int yr = 0; yr < CT_TY; ++yr) {
                if (y0 + yr >= ny) break;   // uniform
#pragma unroll
                for (int xs = 0; xs < 32; xs += 16) {
                    // A = dz^T of 16 nodes: matrices (o 0-7 | 8-15) x (nodes 0-7 | 8-15)
                    uint32_t ar[4];
                    ldmatrix_x4_trans(ar, pd + (size_t)(yr * 32 + xs + (lane & 7) + ((lane >> 4) & 1) * 8) * DS +
                                              m * 16 + ((lane >> 3) & 1) * 8);
                    const uint4 af = make_uint4(ar[0], ar[1], ar[2], ar[3]);
#pragma unroll
                    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx) {
                            // B = the activations of the same 16 nodes shifted by (kx - 1, ky - 1)
                            uint32_t br[2];
                            const int hx = xs + kx + (lane & 7) + ((lane >> 3) & 1) * 8;
                            ldmatrix_x2_trans(br, pa + (size_t)((yr + ky) * CT_HX + hx) * Gm::CS + n * 8);
                            mma_bf16(acc[ky * 3 + kx], af, br[0], br[1]);
                        }
                }
            }
        }
        __syncthreads();   // buffer b is refilled by the next iteration
    }
    if (!on) return;
    const int g = lane >> 2, t = lane & 3;
    const size_t nblk = (size_t)gridDim.x * gridDim.z, blk = (size_t)blockIdx.z * gridDim.x + blockIdx.x;
    float *pp = part + ((size_t)blockIdx.y * nblk + blk) * 9 * 1024;
#pragma unroll
    for (int q = 0; q < 9; ++q)
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int o = m * 16 + g + (h >> 1) * 8, i = n * 8 + 2 * t + (h & 1);
            pp[q * 1024 + o * 32 + i] = acc[q][h];
        }
}

// dW[o][i][k] += sum over the nblk blocks of k's z offset group.  A block of 256 threads takes 32
// consecutive partial columns (gz, q, o, is) -- consecutive in memory, so every load is coalesced
// -- and splits the blocks into 8 consecutive segments, one warp each; the 8 segment sums are then
// added in segment order.  The order is fixed, so the gradient is reproducible bit for bit, and no
// sum is longer than nblk terms.  A column maps back to its weight: k = 9 gz + q and i = is, or for
// the first layer (xfold) the folded layout's ks = k - k % 3 + 1, is = 5 (k % 3) + i.
constexpr int kDwSegs = 8;

__global__ void __launch_bounds__(256) dw_reduce_kernel(const float *__restrict__ part, int nblk, int cout, int cin,
                                                        bool xfold, float *__restrict__ dW)
{
    __shared__ float seg_sum[kDwSegs][32];
    const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
    const int col_all = blockIdx.x * 32 + lane;           // (gz, q) * 1024 + o * 32 + is, < 27 * 1024
    const int gq = col_all >> 10, col = col_all & 1023;
    const int gz = gq / 9, q = gq - 9 * gz;
    const float *pp = part + ((size_t)gz * nblk * 9 + q) * 1024 + col;
    const int b0 = (int)((long long)nblk * seg / kDwSegs), b1 = (int)((long long)nblk * (seg + 1) / kDwSegs);
    float s = 0.0f;
    for (int b = b0; b < b1; ++b) s += pp[(size_t)b * 9 * 1024];
    seg_sum[seg][lane] = s;
    __syncthreads();
    if (seg != 0) return;
    float tot = seg_sum[0][lane];
#pragma unroll
    for (int g = 1; g < kDwSegs; ++g) tot += seg_sum[g][lane];
    const int o = col >> 5, is = col & 31, ks = 9 * gz + q;
    if (o >= cout) return;
    int k, i;
    if (xfold) {
        if (ks % 3 != 1 || is >= 15) return;
        const int r = is / 5;
        i = is - 5 * r;
        k = ks - 1 + r;
    } else {
        k = ks;
        i = is;
    }
    if (i >= cin) return;
    dW[(o * cin + i) * 27 + k] += tot;
}

// db[o] += the sum of the per-block partials part[b][o] (written by the producers of dz: the loss
// kernel and silu_back_kernel).  One block of 256 threads: row r = threadIdx.x / 32 adds blocks
// r, r + 8, ... of channel threadIdx.x % 32 in order, then row 0 adds the 8 rows in order (a fixed
// order: deterministic).
__global__ void __launch_bounds__(256) dbias_reduce_kernel(const float *__restrict__ part, int nchunk, int cout,
                                                           float *__restrict__ db)
{
    __shared__ float red[8][33];
    const int c = threadIdx.x & 31, row = threadIdx.x >> 5;
    float s = 0.0f;
    for (int b = row; b < nchunk; b += 8) s += part[(size_t)b * 32 + c];
    red[row][c] = s;
    __syncthreads();
    if (row == 0 && c < cout) {
        float tot = 0.0f;
        for (int r = 0; r < 8; ++r) tot += red[r][c];
        db[c] += tot;
    }
}

// Adam (beta1 = 0.9, beta2 = 0.999, eps = 1e-8) on the flat FP32 parameters; step t >= 1
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int count, float lr, float gscale, float bc1, float bc2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i] * gscale;
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
}


// ---- closure inputs, targets, correction and restriction --------------------------------

// x = ((phi, ubar, p) - shift) / scale at every node of a one-box state (p = p* rho cs^2)
__global__ void features_kernel(Grid G, Phys P, const float *__restrict__ g, const float *__restrict__ phi,
                                const float *__restrict__ u, lbm_closure_norm nrm, float *__restrict__ x)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G.N) return;
    const size_t N = (size_t)G.N;
    float ps = 0.0f;
#pragma unroll
    for (int i = 0; i < 27; ++i) ps += g[i * N + k];
    const float ph = phi[k];
    const float p = ps * fmaf(ph, P.drho, P.rho_g) * (1.0f / 3.0f);
    const float v[5] = {ph, u[k], u[N + k], u[2 * N + k], p};
#pragma unroll
    for (int c = 0; c < 5; ++c) x[c * N + k] = (v[c] - nrm.in_shift[c]) / nrm.in_scale[c];
}

// t = ((phi, u) of the reference - (phi, ubar) of the state) / out_scale; ref: [>= 4][N]
__global__ void target_kernel(int N, const float *__restrict__ phi, const float *__restrict__ u,
                              const float *__restrict__ ref, lbm_closure_norm nrm, float *__restrict__ t)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    t[k] = (ref[k] - phi[k]) / nrm.out_scale[0];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        t[(size_t)(a + 1) * N + k] = (ref[(size_t)(a + 1) * N + k] - u[(size_t)a * N + k]) / nrm.out_scale[a + 1];
}

// The phi correction before the conservation step: s_0 y_0 limited so that phi stays in [0, 1]
// (a correction may not push a node out of the range the phase field has; phi already outside
// it is not pushed further)
__device__ __forceinline__ float bounded_dphi(float raw, float ph)
{
    return fminf(fmaxf(raw, -fmaxf(ph, 0.0f)), fmaxf(1.0f - ph, 0.0f));
}

// Sums for the conservative corrections (FP64): out[0] += sum of the bounded phi corrections,
// out[1] += sum of the interface weight w = max(4 phi (1 - phi), 0), out[2..4] += sum of rho du
// (the momentum the velocity correction would add), out[5] += sum of rho
__global__ void __launch_bounds__(256) corr_sums_kernel(const float *__restrict__ y, const float *__restrict__ phi,
                                                        lbm_closure_norm nrm, float rho_g, float drho, int N,
                                                        double *__restrict__ part)
{
    __shared__ double red[6][256];
    double s[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const size_t NN = (size_t)N;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        const float p = phi[k];
        const double rho = (double)fmaf(p, drho, rho_g);
        s[0] += bounded_dphi(nrm.out_scale[0] * y[k], p);
        s[1] += fmaxf(4.0f * p * (1.0f - p), 0.0f);
#pragma unroll
        for (int a = 0; a < 3; ++a) s[2 + a] += rho * (double)(nrm.out_scale[a + 1] * y[(a + 1) * NN + k]);
        s[5] += rho;
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) red[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < 6; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 6) part[(size_t)blockIdx.x * 6 + threadIdx.x] = red[threadIdx.x][0];
}

// the six sums of corr_sums_kernel from its blocks' records, in a fixed order (deterministic):
// warp q takes sum q, lane l adds records l, l + 32, ... in order, then a fixed shuffle tree
__global__ void __launch_bounds__(192) corr_final_kernel(const double *__restrict__ part, int nblocks,
                                                         double *__restrict__ out)
{
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += part[(size_t)b * 6 + q];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) out[q] = s;
}

// Apply the network's correction y [4][N] to a one-box FP32 state.  phi: dphi = d - w c with d
// the bounded correction s_0 y_0 (phi kept in [0, 1]), w = max(4 phi (1 - phi), 0) and
// c = sum(d) / sum(w), so the sum of phi is unchanged and the compensation sits in the interfaces
// (a uniform shift, or an unbounded correction, pushes the bulk phases out of [0, 1], and with a
// density ratio of 100 rho(phi) turns negative at phi = -0.0101); with no interface (sum w = 0)
// the plain mean is removed.  ubar: du = s_a y_a - sum(rho s_a y_a) / sum(rho), so the correction
// adds no momentum to the box (as the step itself, on a periodic box).  Populations:
// g_i += f^eq_i(p*, ubar + du) - f^eq_i(p*, ubar) (Eq. eqts; p* = sum g unchanged), so they carry
// the new velocity.
__global__ void correct_kernel(Grid G, const float *__restrict__ y, lbm_closure_norm nrm,
                               const double *__restrict__ sums, float *__restrict__ g, float *__restrict__ phi,
                               float *__restrict__ u)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G.N) return;
    const size_t N = (size_t)G.N;
    const double total = sums[0];
    const float ph = phi[k];
    const float w = fmaxf(4.0f * ph * (1.0f - ph), 0.0f);
    const float comp = sums[1] > 0.0 ? (float)(total / sums[1]) * w : (float)(total / (double)G.N);
    const float dphi = bounded_dphi(nrm.out_scale[0] * y[k], ph) - comp;
    const float du[3] = {nrm.out_scale[1] * y[N + k] - (float)(sums[2] / sums[5]),
                         nrm.out_scale[2] * y[2 * N + k] - (float)(sums[3] / sums[5]),
                         nrm.out_scale[3] * y[3 * N + k] - (float)(sums[4] / sums[5])};
    float ps = 0.0f;
    float gi[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        gi[i] = g[i * N + k];
        ps += gi[i];
    }
    const float ux = u[k], uy = u[N + k], uz = u[2 * N + k];
    float e0[27], e1[27];
    equilibrium(ps, ux, uy, uz, e0);
    equilibrium(ps, ux + du[0], uy + du[1], uz + du[2], e1);
    // __fsub_rn / __fadd_rn are never contracted into an FMA with the products inside e0, e1, so
    // a zero correction leaves g bit for bit
#pragma unroll
    for (int i = 0; i < 27; ++i) g[i * N + k] = __fadd_rn(gi[i], __fsub_rn(e1[i], e0[i]));
    phi[k] = ph + dphi;
    u[k] = ux + du[0];
    u[N + k] = uy + du[1];
    u[2 * N + k] = uz + du[2];
}

// 2x restriction of a fine state (phi, u, p on an nx x ny x nz grid, channel-first) to the coarse
// grid: phi and p averaged over the 8 fine nodes of a coarse cell, u averaged with rho(phi) as
// weight (momentum / mass), and p* = 3 p / rho(phi_coarse).  out: [6][N/8] = (phi, u, p, p*).
__global__ void restrict2_kernel(int nx, int ny, int nz, const float *__restrict__ phi, const float *__restrict__ u,
                                 const float *__restrict__ p, float rho_g, float drho, float *__restrict__ out)
{
    const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    const int Nc = cx * cy * cz;
    const int kc = blockIdx.x * blockDim.x + threadIdx.x;
    if (kc >= Nc) return;
    const int z = kc / (cx * cy), rem = kc - z * cx * cy, y = rem / cx, x = rem - y * cx;
    const size_t N = (size_t)nx * ny * nz;
    float sphi = 0.f, sp = 0.f, sm = 0.f, sj[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const size_t f = ((size_t)(2 * z + (c >> 2)) * ny + (2 * y + ((c >> 1) & 1))) * nx + 2 * x + (c & 1);
        const float ph = phi[f];
        const float rho = fmaf(ph, drho, rho_g);
        sphi += ph;
        sp += p[f];
        sm += rho;
#pragma unroll
        for (int a = 0; a < 3; ++a) sj[a] += rho * u[a * N + f];
    }
    const float phc = 0.125f * sphi, pc = 0.125f * sp;
    out[kc] = phc;
#pragma unroll
    for (int a = 0; a < 3; ++a) out[(size_t)(a + 1) * Nc + kc] = sj[a] / sm;
    out[(size_t)4 * Nc + kc] = pc;
    out[(size_t)5 * Nc + kc] = 3.0f * pc / fmaf(phc, drho, rho_g);
}

// Cell-centred 2x prolongation of a coarse state to the fine grid (the fallback from the corrected
// coarse run to the fine solver).  Fine index X of coarse cell i = X / 2 lies a quarter of a coarse
// cell from that cell's centre, towards the neighbour i - 1 (X even) or i + 1 (X odd), so along each
// axis it takes 3/4 of cell i and 1/4 of that neighbour; the 8 products of the three axes' weights
// (27/64, 9/64, 3/64, 1/64) are exact in FP32 and added in a fixed order.  Periodic axes wrap; at a
// z wall the neighbour beyond the wall is the wall cell itself (the mirror image of cell-centred
// values).  The sum over the fine nodes is 8 times the sum over the coarse cells for every field,
// and every field is interpolated the same way: the 27 populations (so p* and their first moment
// keep their sums too), phi and ubar.
__device__ __forceinline__ int prolong_nbr(int X, int n, bool clamp)
{
    const int i = X >> 1, j = (X & 1) ? i + 1 : i - 1;
    if (j < 0) return clamp ? 0 : n - 1;
    if (j >= n) return clamp ? n - 1 : 0;
    return j;
}

__global__ void prolong2_kernel(Grid C, const float *__restrict__ gc, const float *__restrict__ phic,
                                const float *__restrict__ uc, Grid F, float *__restrict__ gf,
                                float *__restrict__ phif, float *__restrict__ uf)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= F.N) return;
    const int Z = k / F.nxy, rem = k - Z * F.nxy, Y = rem / F.nx, X = rem - Y * F.nx;
    const int ix[2] = {X >> 1, prolong_nbr(X, C.nx, false)};
    const int iy[2] = {Y >> 1, prolong_nbr(Y, C.ny, false)};
    const int iz[2] = {Z >> 1, prolong_nbr(Z, C.nz, C.wall != 0)};
    int off[8];
    float wt[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int a = c & 1, b = (c >> 1) & 1, d = c >> 2;
        off[c] = (iz[d] * C.ny + iy[b]) * C.nx + ix[a];
        wt[c] = (a ? 0.25f : 0.75f) * (b ? 0.25f : 0.75f) * (d ? 0.25f : 0.75f);
    }
    const size_t NC = (size_t)C.N, NF = (size_t)F.N;
    auto interp = [&](const float *src) {
        float v = 0.0f;
#pragma unroll
        for (int c = 0; c < 8; ++c) v = fmaf(wt[c], src[off[c]], v);
        return v;
    };
    for (int i = 0; i < 27; ++i) gf[i * NF + k] = interp(gc + i * NC);
    phif[k] = interp(phic);
#pragma unroll
    for (int a = 0; a < 3; ++a) uf[a * NF + k] = interp(uc + a * NC);
}

}  // namespace
}  // namespace tslb

using tslb::CINP;
using tslb::COUTP;

struct lbm_cnn {
    int nx = 0, ny = 0, nz = 0, N = 0;
    cudaStream_t stream = nullptr;
    int pofs[tslb::NLAYER + 1] = {};     // parameter offsets: layer l's W at pofs[l], b after it
    int nparams = 0;
    float *p = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;   // FP32 master state
    uint4 *wf[tslb::NLAYER] = {};        // forward fragments
    uint4 *wt[tslb::NLAYER] = {};        // transposed fragments (layers 2..4)
    __nv_bfloat16 *wu[tslb::NLAYER] = {};   // tcgen05 operand layout of the weights
    __nv_bfloat16 *wut[tslb::NLAYER] = {};  // ... and of the transposed weights (layers 2..4)
    float *bpad = nullptr;               // biases zero-padded to 32 channels per layer (repack)
    float *dwpart = nullptr;             // per-block partial sums of the weight gradient
    float *dbpart = nullptr;             // per-chunk partial sums of the bias gradient [chunks][32]
    int test_expire = 0;                 // test hook: tensor-core waits expire (lbm_cnn_test_expire_wait)
    int *derr = nullptr;                 // set by a tensor-core kernel whose mbarrier wait expired
    __nv_bfloat16 *a[tslb::NLAYER] = {}; // layer inputs, channel-last BF16: a[0] [N][16], a[1..3] [N][32]
    float *z[tslb::NLAYER] = {};         // pre-activations, channel-last FP32 ([N][32], last [N][16])
    float *dz[tslb::NLAYER] = {};        // gradient of the loss w.r.t. z_l, channel-last FP32 [N][COUTP[l]]
    float *da = nullptr;                 // [N][32] FP32
    __nv_bfloat16 *dzb = nullptr;        // [N][32] BF16
    float *xbuf = nullptr, *ybuf = nullptr;   // [5][N], [4][N] scratch of lbm_closure_apply
    double *dsum = nullptr;              // loss partials / correction mean
    double *h_sum = nullptr;             // pinned
    int loss_blocks = 0;
    long long adam_t = 0;
    int conv_blocks = 0;
    int sms = 0;
    int conv_kernel = 0;                 // 0: tcgen05 / TMEM (default, fastest measured; SiLU fused into
                                         // its epilogue); 1: mma.sync from shared-memory tiles; 2: mma.sync
                                         // from global memory
};

namespace {

lbm_status cnn_fail(lbm_status s, const char *fmt, ...)
{
    char msg[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    tslb::set_last_error(msg);
    return s;
}

#define CNN_TRY(call)                                                                              \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return cnn_fail(LBM_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                            __FILE__, __LINE__);                                                   \
    } while (0)

void free_cnn(lbm_cnn *c)
{
    if (!c) return;
    cudaFree(c->p);
    cudaFree(c->grad);
    cudaFree(c->m);
    cudaFree(c->v);
    for (int l = 0; l < tslb::NLAYER; ++l) {
        cudaFree(c->wf[l]);
        cudaFree(c->wt[l]);
        cudaFree(c->wu[l]);
        cudaFree(c->wut[l]);
        cudaFree(c->a[l]);
        cudaFree(c->z[l]);
    }
    for (int l = 0; l < tslb::NLAYER; ++l) cudaFree(c->dz[l]);
    cudaFree(c->da);
    cudaFree(c->dzb);
    cudaFree(c->xbuf);
    cudaFree(c->ybuf);
    cudaFree(c->dsum);
    cudaFree(c->derr);
    cudaFree(c->bpad);
    cudaFree(c->dwpart);
    cudaFree(c->dbpart);
    if (c->h_sum) cudaFreeHost(c->h_sum);
    delete c;
}

int frag_count(int mt, int cb) { return 27 * cb * mt * 32; }

// forward fragments of every layer and transposed fragments of layers 2..4 from the master weights,
// and the biases zero-padded to 32 channels per layer
cudaError_t repack(lbm_cnn *c)
{
    for (int l = 0; l < tslb::NLAYER; ++l)
        tslb::pad_bias_kernel<<<1, 32, 0, c->stream>>>(c->p + c->pofs[l] + tslb::wcount(l), tslb::COUT[l],
                                                      c->bpad + 32 * l);
    for (int l = 0; l < tslb::NLAYER; ++l) {
        const int mt = COUTP[l] / 16, cb = CINP[l] / 16;
        const int n = frag_count(mt, cb);
        const bool xfold = l == 0;   // the first layer's input carries its x neighbours (pack_input_kernel)
        tslb::pack_weights_kernel<<<(n + 255) / 256, 256, 0, c->stream>>>(c->p + c->pofs[l], tslb::COUT[l],
                                                                           tslb::CIN[l], mt, cb, false, xfold, c->wf[l]);
        const int nu = (xfold ? 3 : 9) * cb * 2 * 3 * COUTP[l] * 8;
        tslb::pack_weights_umma_kernel<<<(nu + 255) / 256, 256, 0, c->stream>>>(c->p + c->pofs[l], tslb::COUT[l],
                                                                                 tslb::CIN[l], COUTP[l], cb, false,
                                                                                 xfold, c->wu[l]);
        if (l > 0) {
            const int mtt = CINP[l] / 16, cbt = COUTP[l] / 16;
            const int nt = frag_count(mtt, cbt);
            tslb::pack_weights_kernel<<<(nt + 255) / 256, 256, 0, c->stream>>>(c->p + c->pofs[l], tslb::COUT[l],
                                                                                tslb::CIN[l], mtt, cbt, true, false,
                                                                                c->wt[l]);
            const int nut = 27 * cbt * 2 * CINP[l] * 8;
            tslb::pack_weights_umma_kernel<<<(nut + 255) / 256, 256, 0, c->stream>>>(c->p + c->pofs[l], tslb::COUT[l],
                                                                                      tslb::CIN[l], CINP[l], cbt, true,
                                                                                      false, c->wut[l]);
        }
    }
    return cudaGetLastError();
}

// the two mma.sync forms of the convolution (kernels 1 and 2)
template <int MT, int CB>
cudaError_t launch_conv_mma(lbm_cnn *c, const uint4 *wfrag, const __nv_bfloat16 *in, const float *bias, float *out)
{
    if (c->conv_kernel <= 1) {   // mma.sync from shared-memory tiles
        const size_t smem = (size_t)frag_count(MT, CB) * sizeof(uint4) +
                            (size_t)tslb::CT_SLOTS * tslb::CtGeom<CB>::PLANE * sizeof(__nv_bfloat16);
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(tslb::conv_tile_kernel<MT, CB>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        const int tiles = (c->nx / 32) * ((c->ny + tslb::CT_TY - 1) / tslb::CT_TY);
        int nzc = c->sms / tiles;                   // about one block per SM
        if (nzc < 1) nzc = 1;
        if (nzc > c->nz) nzc = c->nz;
        const int zlen = (c->nz + nzc - 1) / nzc;
        nzc = (c->nz + zlen - 1) / zlen;
        tslb::conv_tile_kernel<MT, CB><<<dim3(tiles, nzc), 256, smem, c->stream>>>(c->nx, c->ny, c->nz, wfrag, in,
                                                                                    bias, out, zlen);
        return cudaGetLastError();
    }
    const size_t smem = (size_t)frag_count(MT, CB) * sizeof(uint4);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tslb::conv_mma_kernel<MT, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int ntiles = c->N / 32;
    int blocks = (ntiles + 3) / 4;
    if (blocks > c->conv_blocks) blocks = c->conv_blocks;
    tslb::conv_mma_kernel<MT, CB><<<blocks, 128, smem, c->stream>>>(c->nx, c->ny, c->nz, wfrag, in, bias, out, ntiles);
    return cudaGetLastError();
}

// out = conv(in) + bias (FP32, channel-last); with act non-null also act = silu(out) in BF16 (the
// next layer's input; fused into the tcgen05 kernel's epilogue, a separate pass for the others).
template <int MT, int CB, bool XF = false>
cudaError_t launch_conv(lbm_cnn *c, int layer, bool transpose, const __nv_bfloat16 *in, const float *bias, float *out,
                        __nv_bfloat16 *act = nullptr, bool keep_z = true, float *ycf = nullptr)
{
    const uint4 *wfrag = transpose ? c->wt[layer] : c->wf[layer];
    const __nv_bfloat16 *wpack = transpose ? c->wut[layer] : c->wu[layer];
    if (c->conv_kernel == 0 && c->nx % tslb::UM_TX == 0) {   // tcgen05 / TMEM
        constexpr int WB = (XF ? 3 : 9) * CB * 2 * 3 * MT * 16 * 16;
        const size_t smem = (size_t)((WB + 1023) / 1024) * 1024 + (size_t)tslb::UM_SLOTS * tslb::UmGeom<CB>::PLANE_BYTES;
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(tslb::conv_umma_kernel<MT, CB, XF>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        const int tiles = (c->nx / tslb::UM_TX) * ((c->ny + tslb::UM_TY - 1) / tslb::UM_TY);
        int nzc = c->sms / tiles;
        if (nzc < 1) nzc = 1;
        if (nzc > c->nz) nzc = c->nz;
        const int zlen = (c->nz + nzc - 1) / nzc;
        nzc = (c->nz + zlen - 1) / zlen;
        // programmatic dependent launch: the kernel sets up and loads its weights and bias while the
        // previous kernel drains, and waits for it before reading its input.  So no kernel that
        // writes packed weights or biases may directly precede a convolution on the stream (repack
        // is always followed by pack_input_kernel or another ordinary launch).
        return tslb::launch_pdl(tslb::conv_umma_kernel<MT, CB, XF>, dim3(tiles, nzc), dim3(tslb::UM_THREADS), smem, c->stream,
                                c->nx, c->ny, c->nz, wpack, in, bias, out, act, ycf, zlen, c->derr,
                                c->test_expire, keep_z ? 1 : 0);
    }
    cudaError_t e = launch_conv_mma<MT, CB>(c, wfrag, in, bias, out);
    if (e == cudaSuccess && act) {
        const size_t cnt = (size_t)c->N * MT * 16;
        tslb::silu_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, c->stream>>>(out, cnt, act);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && ycf) {
        tslb::unpack_output_kernel<<<(c->N + 255) / 256, 256, 0, c->stream>>>(out, c->N, ycf);
        e = cudaGetLastError();
    }
    return e;
}

// train: keep every layer's pre-activation z (the backward pass needs it); otherwise only the last
// layer's, the output (the tensor-core kernel then skips the other z stores).  y (not null): the
// output also channel-first, y[c][n] (written by the last layer's epilogue).
cudaError_t forward(lbm_cnn *c, const float *x, bool train, float *y = nullptr)
{
    const int N = c->N;
    cudaError_t e;
    tslb::pack_input_kernel<<<(N + 255) / 256, 256, 0, c->stream>>>(x, c->nx, N, c->a[0]);
    // z_l = conv_l(a_l) + b_l and a_{l+1} = silu(z_l); biases zero-padded to the padded channels
    if ((e = launch_conv<2, 1, true>(c, 0, false, c->a[0], c->bpad, c->z[0], c->a[1], train)) != cudaSuccess) return e;
    for (int l = 1; l < tslb::NLAYER; ++l) {
        const float *bias = c->bpad + 32 * l;
        e = l < 3 ? launch_conv<2, 2>(c, l, false, c->a[l], bias, c->z[l], c->a[l + 1], train)
                  : launch_conv<1, 2>(c, l, false, c->a[l], bias, c->z[l], nullptr, true, y);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// block grid of the weight-gradient kernel: column tiles, and z chunks so that the 3 z offset groups
// give about 4 blocks per SM
int dw_tiles(const lbm_cnn *c) { return (c->nx / 32) * ((c->ny + tslb::CT_TY - 1) / tslb::CT_TY); }
int dw_chunks(const lbm_cnn *c)
{
    int nzc = (4 * c->sms) / (3 * dw_tiles(c));
    if (nzc < 1) nzc = 1;
    if (nzc > c->nz) nzc = c->nz;
    const int zlen = (c->nz + nzc - 1) / nzc;
    return (c->nz + zlen - 1) / zlen;
}

// dW_l += sum_n dz_l[n][o] a_l[n + off_k][i] on the tensor cores (dweight_mma_kernel, then the
// ordered reduction of the blocks' partial sums), MT = COUTP/16, CB = CINP/16
template <int MT, int CB>
cudaError_t launch_dweight(lbm_cnn *c, int layer, float *dW)
{
    using Gm = tslb::CtGeom<CB>;
    const size_t smem = (size_t)(2 * Gm::PLANE + 2 * tslb::CT_TY * 32 * (MT * 16 + 8)) * sizeof(__nv_bfloat16);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tslb::dweight_mma_kernel<MT, CB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int tiles = dw_tiles(c), nzc = dw_chunks(c), zlen = (c->nz + nzc - 1) / nzc;
    tslb::dweight_mma_kernel<MT, CB><<<dim3(tiles, 3, nzc), 256, smem, c->stream>>>(c->nx, c->ny, c->nz, c->dzb,
                                                                                   c->a[layer], zlen, c->dwpart);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    tslb::dw_reduce_kernel<<<27 * 1024 / 32, 256, 0, c->stream>>>(c->dwpart, tiles * nzc, tslb::COUT[layer],
                                                                 tslb::CIN[layer], layer == 0, dW);
    return cudaGetLastError();
}

cudaError_t backward(lbm_cnn *c)
{
    const int N = c->N;
    cudaError_t e;
    // dz of the last layer is in dz / dzb with 16 channels (written by the loss kernel)
    for (int l = tslb::NLAYER - 1; l >= 0; --l) {
        float *dW = c->grad + c->pofs[l];
        float *db = dW + tslb::wcount(l);
        e = l == 0   ? launch_dweight<2, 1>(c, l, dW)
            : l == 3 ? launch_dweight<1, 2>(c, l, dW)
                     : launch_dweight<2, 2>(c, l, dW);
        if (e != cudaSuccess) return e;
        // the bias gradient from the per-block partials of dz_l, written by its producer (the loss
        // kernel for the last layer, silu_back_kernel for the others)
        tslb::dbias_reduce_kernel<<<1, 256, 0, c->stream>>>(c->dbpart, l == tslb::NLAYER - 1 ? c->loss_blocks
                                                                                             : tslb::kBackBlocks,
                                                           tslb::COUT[l], db);
        if (l == 0) break;
        // da_{l-1}[n][i] = sum_{k,o} W_l[o][i][k] dz_l[n - off_k][o]
        e = l == 3 ? launch_conv<2, 1>(c, l, true, c->dzb, nullptr, c->da)
                   : launch_conv<2, 2>(c, l, true, c->dzb, nullptr, c->da);
        if (e != cudaSuccess) return e;
        tslb::silu_back_kernel<<<tslb::kBackBlocks, 256, 0, c->stream>>>(
            reinterpret_cast<const float4 *>(c->da), reinterpret_cast<const float4 *>(c->z[l - 1]), (size_t)N * 8,
            reinterpret_cast<float4 *>(c->dz[l - 1]), reinterpret_cast<uint2 *>(c->dzb), c->dbpart);
    }
    return cudaGetLastError();
}

// seeded Glorot-uniform weights (splitmix64 stream), zero biases
void init_params(lbm_cnn *c, unsigned long long seed, float *h)
{
    unsigned long long s = seed + 0x9E3779B97F4A7C15ULL;
    auto next = [&]() {
        unsigned long long z = (s += 0x9E3779B97F4A7C15ULL);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    for (int l = 0; l < tslb::NLAYER; ++l) {
        const double bound = sqrt(6.0 / (27.0 * (tslb::CIN[l] + tslb::COUT[l])));
        float *w = h + c->pofs[l];
        for (int i = 0; i < tslb::wcount(l); ++i) w[i] = (float)((2.0 * next() - 1.0) * bound);
        for (int o = 0; o < tslb::COUT[l]; ++o) w[tslb::wcount(l) + o] = 0.0f;
    }
}

}  // namespace

extern "C" {

int lbm_cnn_num_params(void)
{
    int n = 0;
    for (int l = 0; l < tslb::NLAYER; ++l) n += tslb::pcount(l);
    return n;
}

lbm_status lbm_cnn_create(int nx, int ny, int nz, unsigned long long seed, void *stream, lbm_cnn **out)
{
    if (!out) return cnn_fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 32 || nx % 32 != 0 || ny < 1 || nz < 1)
        return cnn_fail(LBM_ERR_ARG, "network grid needs nx a positive multiple of 32 and ny, nz >= 1");
    const long long n = (long long)nx * ny * nz;
    if (n * 32 >= (1LL << 31)) return cnn_fail(LBM_ERR_ARG, "network grid too large");
    lbm_cnn *c = new (std::nothrow) lbm_cnn;
    if (!c) return cnn_fail(LBM_ERR_OOM, "host allocation failed");
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->N = (int)n;
    c->stream = (cudaStream_t)stream;
    int ofs = 0;
    for (int l = 0; l < tslb::NLAYER; ++l) {
        c->pofs[l] = ofs;
        ofs += tslb::pcount(l);
    }
    c->pofs[tslb::NLAYER] = ofs;
    c->nparams = ofs;
    const size_t N = (size_t)n;
    c->loss_blocks = (int)((N + 255) / 256);
    struct {
        void **p;
        size_t bytes;
    } allocs[] = {
        {(void **)&c->p, ofs * sizeof(float)},         {(void **)&c->grad, ofs * sizeof(float)},
        {(void **)&c->m, ofs * sizeof(float)},         {(void **)&c->v, ofs * sizeof(float)},
        {(void **)&c->da, N * 32 * sizeof(float)},
        {(void **)&c->dzb, N * 32 * 2},                {(void **)&c->xbuf, 5 * N * sizeof(float)},
        {(void **)&c->ybuf, 4 * N * sizeof(float)},
        // loss partials, or the correction's 6 sums then its blocks' records at offset 8
        {(void **)&c->dsum, (size_t)(std::max(c->loss_blocks, tslb::kCorrBlocks * 6) + 8) * sizeof(double)},
        {(void **)&c->dbpart, (size_t)std::max(c->loss_blocks, tslb::kBackBlocks) * 32 * sizeof(float)},
        {(void **)&c->bpad, (size_t)tslb::NLAYER * 32 * sizeof(float)},
    };
    cudaError_t err = cudaSuccess;
    for (auto &a : allocs)
        if (err == cudaSuccess) err = cudaMalloc(a.p, a.bytes);
    for (int l = 0; l < tslb::NLAYER && err == cudaSuccess; ++l) {
        err = cudaMalloc(&c->wf[l], frag_count(COUTP[l] / 16, CINP[l] / 16) * sizeof(uint4));
        if (err == cudaSuccess && l > 0) err = cudaMalloc(&c->wt[l], frag_count(CINP[l] / 16, COUTP[l] / 16) * sizeof(uint4));
        if (err == cudaSuccess) err = cudaMalloc(&c->wu[l], (size_t)27 * CINP[l] * COUTP[l] * 2);
        if (err == cudaSuccess && l > 0) err = cudaMalloc(&c->wut[l], (size_t)27 * CINP[l] * COUTP[l] * 2);
        if (err == cudaSuccess) err = cudaMalloc(&c->a[l], N * CINP[l] * 2);
        if (err == cudaSuccess) err = cudaMalloc(&c->z[l], N * COUTP[l] * sizeof(float));
        if (err == cudaSuccess) err = cudaMalloc(&c->dz[l], N * COUTP[l] * sizeof(float));
    }
    if (err == cudaSuccess) err = cudaMallocHost(&c->h_sum, sizeof(double) * 2);
    if (err == cudaSuccess) err = cudaMalloc(&c->derr, sizeof(int));
    if (err == cudaSuccess) err = cudaMemset(c->derr, 0, sizeof(int));
    int dev = 0, sms = 0;
    if (err == cudaSuccess) err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) {
        cudaGetLastError();
        free_cnn(c);
        return cnn_fail(err == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "network setup failed: %s",
                        cudaGetErrorString(err));
    }
    c->conv_blocks = sms * 4;
    c->sms = sms;
    // weight-gradient partials: 3 z offset groups x blocks x 9 offsets x 32 x 32
    err = cudaMalloc(&c->dwpart, (size_t)3 * dw_tiles(c) * dw_chunks(c) * 9 * 1024 * sizeof(float));
    if (err != cudaSuccess) {
        cudaGetLastError();
        free_cnn(c);
        return cnn_fail(err == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "network setup failed: %s",
                        cudaGetErrorString(err));
    }
    float *h = new (std::nothrow) float[ofs];
    if (!h) {
        free_cnn(c);
        return cnn_fail(LBM_ERR_OOM, "host allocation failed");
    }
    init_params(c, seed, h);
    err = cudaMemcpyAsync(c->p, h, ofs * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    if (err == cudaSuccess) err = cudaMemsetAsync(c->grad, 0, ofs * sizeof(float), c->stream);
    if (err == cudaSuccess) err = cudaMemsetAsync(c->m, 0, ofs * sizeof(float), c->stream);
    if (err == cudaSuccess) err = cudaMemsetAsync(c->v, 0, ofs * sizeof(float), c->stream);
    if (err == cudaSuccess) err = repack(c);
    if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
    delete[] h;
    if (err != cudaSuccess) {
        free_cnn(c);
        return cnn_fail(LBM_ERR_CUDA, "network initialisation failed: %s", cudaGetErrorString(err));
    }
    *out = c;
    return LBM_OK;
}

void lbm_cnn_destroy(lbm_cnn *cnn)
{
    if (!cnn) return;
    cudaStreamSynchronize(cnn->stream);
    free_cnn(cnn);
}

lbm_status lbm_cnn_get_params(lbm_cnn *cnn, float *params)
{
    if (!cnn || !params) return cnn_fail(LBM_ERR_ARG, "network and params are required");
    CNN_TRY(cudaMemcpyAsync(params, cnn->p, cnn->nparams * sizeof(float), cudaMemcpyDeviceToHost, cnn->stream));
    CNN_TRY(cudaStreamSynchronize(cnn->stream));
    return LBM_OK;
}

lbm_status lbm_cnn_set_params(lbm_cnn *cnn, const float *params)
{
    if (!cnn || !params) return cnn_fail(LBM_ERR_ARG, "network and params are required");
    CNN_TRY(cudaMemcpyAsync(cnn->p, params, cnn->nparams * sizeof(float), cudaMemcpyHostToDevice, cnn->stream));
    CNN_TRY(repack(cnn));
    CNN_TRY(cudaStreamSynchronize(cnn->stream));
    return LBM_OK;
}

lbm_status lbm_cnn_get_grads(lbm_cnn *cnn, float *grads)
{
    if (!cnn || !grads) return cnn_fail(LBM_ERR_ARG, "network and grads are required");
    CNN_TRY(cudaMemcpyAsync(grads, cnn->grad, cnn->nparams * sizeof(float), cudaMemcpyDeviceToHost, cnn->stream));
    CNN_TRY(cudaStreamSynchronize(cnn->stream));
    return LBM_OK;
}

lbm_status lbm_cnn_set_conv_kernel(lbm_cnn *cnn, int kernel)
{
    if (!cnn) return cnn_fail(LBM_ERR_ARG, "network is NULL");
    if (kernel < 0 || kernel > 2) return cnn_fail(LBM_ERR_ARG, "kernel must be 0, 1 or 2");
    cnn->conv_kernel = kernel;
    return LBM_OK;
}

// LBM_ERR_TIMEOUT once a tensor-core kernel reported an expired mbarrier wait (synchronises)
lbm_status check_timeout(lbm_cnn *cnn)
{
    int h = 0;
    CNN_TRY(cudaMemcpyAsync(&h, cnn->derr, sizeof(int), cudaMemcpyDeviceToHost, cnn->stream));
    CNN_TRY(cudaStreamSynchronize(cnn->stream));
    if (h) {   // report once; the flag is cleared so that the network stays usable
        CNN_TRY(cudaMemsetAsync(cnn->derr, 0, sizeof(int), cnn->stream));
        CNN_TRY(cudaStreamSynchronize(cnn->stream));
        return cnn_fail(LBM_ERR_TIMEOUT, "a tensor-core convolution gave up waiting for its MMAs");
    }
    return LBM_OK;
}

lbm_status lbm_cnn_test_expire_wait(lbm_cnn *cnn, int on)
{
    if (!cnn) return cnn_fail(LBM_ERR_ARG, "network is NULL");
    if (on != 0 && on != 1) return cnn_fail(LBM_ERR_ARG, "on must be 0 or 1");
    cnn->test_expire = on;
    return LBM_OK;
}

lbm_status lbm_cnn_forward(lbm_cnn *cnn, const float *x, float *y)
{
    if (!cnn || !x || !y) return cnn_fail(LBM_ERR_ARG, "network, x and y are required");
    CNN_TRY(forward(cnn, x, false, y));
    CNN_TRY(cudaGetLastError());
    return check_timeout(cnn);
}

lbm_status lbm_cnn_grad(lbm_cnn *cnn, const float *x, const float *t, int accumulate, double *loss)
{
    if (!cnn || !x || !t) return cnn_fail(LBM_ERR_ARG, "network, x and t are required");
    if (!accumulate) CNN_TRY(cudaMemsetAsync(cnn->grad, 0, cnn->nparams * sizeof(float), cnn->stream));
    CNN_TRY(forward(cnn, x, true));
    tslb::loss_kernel<<<cnn->loss_blocks, 256, 0, cnn->stream>>>(cnn->z[3], t, cnn->N, cnn->dz[3], cnn->dzb,
                                                                  cnn->dsum, cnn->dbpart);
    CNN_TRY(cudaGetLastError());
    CNN_TRY(backward(cnn));
    // loss: sum of the per-block partials
    double *hp = new (std::nothrow) double[cnn->loss_blocks];
    if (!hp) return cnn_fail(LBM_ERR_OOM, "host allocation failed");
    cudaError_t err = cudaMemcpyAsync(hp, cnn->dsum, cnn->loss_blocks * sizeof(double), cudaMemcpyDeviceToHost,
                                      cnn->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(cnn->stream);
    if (err != cudaSuccess) {
        delete[] hp;
        return cnn_fail(LBM_ERR_CUDA, "loss read-back failed: %s", cudaGetErrorString(err));
    }
    double s = 0.0;
    for (int b = 0; b < cnn->loss_blocks; ++b) s += hp[b];
    delete[] hp;
    if (loss) *loss = s / (4.0 * cnn->N);
    return check_timeout(cnn);
}

lbm_status lbm_cnn_get_layer(lbm_cnn *cnn, int layer, float *a_in, float *z, float *dz)
{
    if (!cnn) return cnn_fail(LBM_ERR_ARG, "network is NULL");
    if (layer < 0 || layer >= tslb::NLAYER) return cnn_fail(LBM_ERR_ARG, "layer must be 0..3");
    const size_t N = (size_t)cnn->N;
    const int cin = tslb::CIN[layer], cinp = CINP[layer], cout = tslb::COUT[layer], coutp = COUTP[layer];
    // copy the channel-last device buffer to the host, then reorder to channel-first there
    if (a_in) {
        uint16_t *h = new (std::nothrow) uint16_t[N * cinp];
        if (!h) return cnn_fail(LBM_ERR_OOM, "host allocation failed");
        cudaError_t e = cudaMemcpyAsync(h, cnn->a[layer], N * cinp * 2, cudaMemcpyDeviceToHost, cnn->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cnn->stream);
        if (e == cudaSuccess)
            for (size_t n = 0; n < N; ++n)
                for (int i = 0; i < cin; ++i) {
                    // the first layer's input holds the node's own channels at 5 .. 9 (pack_input_kernel)
                    const int is = layer == 0 ? 5 + i : i;
                    const uint32_t bits = (uint32_t)h[n * cinp + is] << 16;   // BF16 is the top half of FP32
                    memcpy(&a_in[(size_t)i * N + n], &bits, 4);
                }
        delete[] h;
        if (e != cudaSuccess) return cnn_fail(LBM_ERR_CUDA, "layer input read-back: %s", cudaGetErrorString(e));
    }
    const float *src[2] = {cnn->z[layer], cnn->dz[layer]};
    float *dst[2] = {z, dz};
    for (int q = 0; q < 2; ++q) {
        if (!dst[q]) continue;
        float *h = new (std::nothrow) float[N * coutp];
        if (!h) return cnn_fail(LBM_ERR_OOM, "host allocation failed");
        cudaError_t e = cudaMemcpyAsync(h, src[q], N * coutp * sizeof(float), cudaMemcpyDeviceToHost, cnn->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cnn->stream);
        if (e == cudaSuccess)
            for (size_t n = 0; n < N; ++n)
                for (int o = 0; o < cout; ++o) dst[q][(size_t)o * N + n] = h[n * coutp + o];
        delete[] h;
        if (e != cudaSuccess) return cnn_fail(LBM_ERR_CUDA, "layer read-back: %s", cudaGetErrorString(e));
    }
    return LBM_OK;
}

lbm_status lbm_cnn_adam_step(lbm_cnn *cnn, float lr, float grad_scale)
{
    if (!cnn) return cnn_fail(LBM_ERR_ARG, "network is NULL");
    if (!(lr > 0.0f) || !isfinite(grad_scale)) return cnn_fail(LBM_ERR_ARG, "lr must be > 0, grad_scale finite");
    ++cnn->adam_t;
    const float bc1 = (float)(1.0 - pow(0.9, (double)cnn->adam_t));
    const float bc2 = (float)(1.0 - pow(0.999, (double)cnn->adam_t));
    tslb::adam_kernel<<<(cnn->nparams + 255) / 256, 256, 0, cnn->stream>>>(cnn->p, cnn->grad, cnn->m, cnn->v,
                                                                            cnn->nparams, lr, grad_scale, bc1, bc2);
    CNN_TRY(cudaGetLastError());
    CNN_TRY(repack(cnn));
    return LBM_OK;
}

lbm_status lbm_closure_features(lbm_ctx *ctx, const lbm_closure_norm *norm, float *x)
{
    if (!norm || !x) return cnn_fail(LBM_ERR_ARG, "norm and x are required");
    tslb::CtxView v;
    lbm_status st = tslb::ctx_view(ctx, &v);
    if (st != LBM_OK) return st;
    if (v.storage != LBM_FP32) return cnn_fail(LBM_ERR_ARG, "the closure needs FP32 population storage");
    tslb::features_kernel<<<(v.G.N + 255) / 256, 256, 0, v.stream>>>(v.G, v.P, v.g, v.phi, v.u, *norm, x);
    CNN_TRY(cudaGetLastError());
    return LBM_OK;
}

lbm_status lbm_closure_target(lbm_ctx *ctx, const float *ref, const lbm_closure_norm *norm, float *t)
{
    if (!norm || !ref || !t) return cnn_fail(LBM_ERR_ARG, "ref, norm and t are required");
    tslb::CtxView v;
    lbm_status st = tslb::ctx_view(ctx, &v);
    if (st != LBM_OK) return st;
    tslb::target_kernel<<<(v.G.N + 255) / 256, 256, 0, v.stream>>>(v.G.N, v.phi, v.u, ref, *norm, t);
    CNN_TRY(cudaGetLastError());
    return LBM_OK;
}

lbm_status lbm_closure_apply(lbm_ctx *ctx, lbm_cnn *cnn, const lbm_closure_norm *norm)
{
    if (!cnn || !norm) return cnn_fail(LBM_ERR_ARG, "network and norm are required");
    tslb::CtxView v;
    lbm_status st = tslb::ctx_view(ctx, &v);
    if (st != LBM_OK) return st;
    if (v.storage != LBM_FP32) return cnn_fail(LBM_ERR_ARG, "the closure needs FP32 population storage");
    if (v.G.wall) return cnn_fail(LBM_ERR_ARG, "the closure is for periodic boxes");
    if (v.G.nx != cnn->nx || v.G.ny != cnn->ny || v.G.nz != cnn->nz)
        return cnn_fail(LBM_ERR_ARG, "network grid %dx%dx%d differs from the box %dx%dx%d", cnn->nx, cnn->ny, cnn->nz,
                        v.G.nx, v.G.ny, v.G.nz);
    if (v.stream != cnn->stream) return cnn_fail(LBM_ERR_ARG, "network and context must share a stream");
    const int N = v.G.N;
    tslb::features_kernel<<<(N + 255) / 256, 256, 0, v.stream>>>(v.G, v.P, v.g, v.phi, v.u, *norm, cnn->xbuf);
    CNN_TRY(cudaGetLastError());
    CNN_TRY(forward(cnn, cnn->xbuf, false, cnn->ybuf));
    tslb::corr_sums_kernel<<<tslb::kCorrBlocks, 256, 0, v.stream>>>(cnn->ybuf, v.phi, *norm, v.P.rho_g, v.P.drho, N,
                                                                     cnn->dsum + 8);
    tslb::corr_final_kernel<<<1, 192, 0, v.stream>>>(cnn->dsum + 8, tslb::kCorrBlocks, cnn->dsum);
    tslb::correct_kernel<<<(N + 255) / 256, 256, 0, v.stream>>>(v.G, cnn->ybuf, *norm, cnn->dsum, v.g, v.phi, v.u);
    CNN_TRY(cudaGetLastError());
    tslb::ctx_state_changed(ctx);
    return LBM_OK;
}

lbm_status lbm_prolong2_state(lbm_ctx *coarse, lbm_ctx *fine)
{
    if (!coarse || !fine || coarse == fine) return cnn_fail(LBM_ERR_ARG, "two distinct contexts are required");
    tslb::CtxView c, f;
    lbm_status st = tslb::ctx_view(coarse, &c);
    if (st != LBM_OK) return st;
    if ((st = tslb::ctx_view(fine, &f)) != LBM_OK) return st;
    if (c.storage != LBM_FP32 || f.storage != LBM_FP32) return cnn_fail(LBM_ERR_ARG, "both contexts need FP32 populations");
    if (f.G.nx != 2 * c.G.nx || f.G.ny != 2 * c.G.ny || f.G.nz != 2 * c.G.nz || f.G.wall != c.G.wall)
        return cnn_fail(LBM_ERR_ARG, "fine box %dx%dx%d must be twice the coarse box %dx%dx%d with the same walls",
                        f.G.nx, f.G.ny, f.G.nz, c.G.nx, c.G.ny, c.G.nz);
    // the fine stream waits for the coarse context's pending work
    cudaEvent_t ev;
    CNN_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t err = cudaEventRecord(ev, c.stream);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(f.stream, ev, 0);
    cudaEventDestroy(ev);
    if (err != cudaSuccess) return cnn_fail(LBM_ERR_CUDA, "stream ordering failed: %s", cudaGetErrorString(err));
    tslb::prolong2_kernel<<<(f.G.N + 255) / 256, 256, 0, f.stream>>>(c.G, c.g, c.phi, c.u, f.G, f.g, f.phi, f.u);
    CNN_TRY(cudaGetLastError());
    tslb::ctx_state_changed(fine);
    return LBM_OK;
}

lbm_status lbm_restrict2(const float *phi, const float *u, const float *p, int nx, int ny, int nz, double rho_l,
                         double rho_g, float *out, void *stream)
{
    if (!phi || !u || !p || !out) return cnn_fail(LBM_ERR_ARG, "phi, u, p and out are required");
    if (nx < 2 || ny < 2 || nz < 2 || nx % 2 || ny % 2 || nz % 2) return cnn_fail(LBM_ERR_ARG, "sizes must be even");
    if ((long long)nx * ny * nz >= (1LL << 31)) return cnn_fail(LBM_ERR_ARG, "grid too large");
    const int Nc = (nx / 2) * (ny / 2) * (nz / 2);
    tslb::restrict2_kernel<<<(Nc + 255) / 256, 256, 0, (cudaStream_t)stream>>>(nx, ny, nz, phi, u, p, (float)rho_g,
                                                                                (float)(rho_l - rho_g), out);
    CNN_TRY(cudaGetLastError());
    return LBM_OK;
}

}  // extern "C"

// FP64 conservation and interface diagnostics of the state (phi, ubar, p* = sum g).
// Pass 1: a grid-stride loop; each thread adds its nodes' terms exactly in FP32 pairs (TwoSum /
// TwoProduct), moves them into FP64 accumulators every 16 nodes, and counts in 64-bit integers;
// the per-thread FP64 records are reduced in each block with warp shuffles and a shared-memory
// stage, and each block writes one record of kObsFields doubles.
// Pass 2: one warp per field sums the block records in a fixed order (deterministic result).
#include <float.h>

#include "tslb_internal.h"

namespace tslb {
namespace {

// record layout
enum : int {
    F_SUM_PHI = 0, F_MASS = 1, F_SUM_PS = 2, F_MOM = 3,      // 3..5
    F_XPHI = 6,                                             // 6..8   sum phi x
    F_XGAS = 9,                                             // 9..11  sum (1-phi) x
    F_UPHI = 12,                                            // 12..14 sum phi u
    F_UGAS = 15,                                            // 15..17 sum (1-phi) u
    F_PLIQ = 18, F_NLIQ = 19, F_PGAS = 20, F_NGAS = 21,
    F_UMAX = 22, F_PHIMIN = 23, F_PHIMAX = 24, F_NONFIN = 25, F_SUM_GAS = 26,
    F_USED = 27
};
static_assert(F_USED <= kObsFields, "record too small");

__device__ __forceinline__ double combine(int f, double a, double b)
{
    if (f == F_UMAX || f == F_PHIMAX) return fmax(a, b);
    if (f == F_PHIMIN) return fmin(a, b);
    return a + b;
}

constexpr int kThreads = 256;
constexpr int kFlush = 16;   // nodes per thread between flushes of the FP32 pair sums into FP64

// Error-free FP32 accumulation: hi + lo carries a running sum whose every addition to hi is
// exact as hi + (rounding error), the error collected in lo (Knuth's TwoSum).  Over kFlush terms
// the sum is within about kFlush * 2^-48 of sum |terms| (Neumaier's bound), then it is added to an
// FP64 accumulator; the FP64 pipe, about 1/60 of the FP32 rate on this GPU, then does a few
// operations per 16 nodes instead of some forty per node.
struct Pair {
    float hi, lo;
};

__device__ __forceinline__ void pair_add(Pair &a, float x)
{
    const float s = __fadd_rn(a.hi, x);
    const float bp = __fsub_rn(s, a.hi);
    a.lo = __fadd_rn(a.lo, __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(x, bp)));
    a.hi = s;
}

// adds the exact product x y = p + e (TwoProduct: e = fma(x, y, -p) is exact)
__device__ __forceinline__ void pair_add_prod(Pair &a, float x, float y)
{
    const float p = __fmul_rn(x, y);
    const float e = __fmaf_rn(x, y, -p);
    pair_add(a, p);
    a.lo = __fadd_rn(a.lo, e);
}

// adds x c exactly for an integer coordinate c: c is exact in FP32 below 2^24, larger values are
// split into a multiple of 4096 and the remainder, each exact
__device__ __forceinline__ void pair_add_coord(Pair &a, float x, int c, bool big)
{
    if (big) {
        pair_add_prod(a, x, (float)(c & ~4095));
        pair_add_prod(a, x, (float)(c & 4095));
    } else {
        pair_add_prod(a, x, (float)c);
    }
}

__device__ __forceinline__ double pair_value(const Pair &a) { return (double)a.hi + (double)a.lo; }

__global__ void __launch_bounds__(kThreads) obs_partial_kernel(Grid G, double rho_g, double drho,
                                                               const void *__restrict__ gv, int storage,
                                                               const float *__restrict__ pst,
                                                               const float *__restrict__ phi,
                                                               const float *__restrict__ u,
                                                               double *__restrict__ partials)
{
    double r[F_USED];
#pragma unroll
    for (int f = 0; f < F_USED; ++f) r[f] = 0.0;
    const size_t N = (size_t)G.N;
    const bool big = G.nx > (1 << 24) || G.ny > (1 << 24) || G.nz > (1 << 24);
    const float rho_g32 = (float)rho_g, drho32 = (float)drho;

    // FP32 pair sums since the last flush: sum phi, p*, phi x (3), phi u (3), u (3), p in the
    // liquid and in the gas; integer counts and coordinate sums are exact in 64-bit integers
    Pair sphi{}, sps{}, sxphi[3]{}, suphi[3]{}, su[3]{}, spl{}, spg{};
    long long cnt = 0, nvalid = 0, nliq = 0, ngas = 0, nbad = 0, sx[3] = {0, 0, 0};
    float umax = 0.0f, phimin = FLT_MAX, phimax = -FLT_MAX;
    auto flush = [&]() {
        const double vphi = pair_value(sphi);
        r[F_SUM_PHI] += vphi;
        r[F_MASS] += fma(drho, vphi, rho_g * (double)cnt);   // sum (rho_g + phi drho) of the flushed nodes
        r[F_SUM_PS] += pair_value(sps);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double vu = pair_value(su[a]), vuphi = pair_value(suphi[a]);
            r[F_MOM + a] += fma(drho, vuphi, rho_g * vu);    // sum (rho_g + phi drho) u
            r[F_XPHI + a] += pair_value(sxphi[a]);
            r[F_UPHI + a] += vuphi;
            r[F_UGAS + a] += vu;
            sxphi[a] = Pair{}, suphi[a] = Pair{}, su[a] = Pair{};
        }
        r[F_PLIQ] += pair_value(spl);
        r[F_PGAS] += pair_value(spg);
        sphi = Pair{}, sps = Pair{}, spl = Pair{}, spg = Pair{};
        cnt = 0;
    };

    // 64-bit node index: with N close to 2^31 an int index would wrap past INT_MAX on its last
    // stride.  Inside the loop k < N < 2^31, so the coordinates come from 32-bit divisions.
    for (size_t k = (size_t)blockIdx.x * kThreads + threadIdx.x; k < N; k += (size_t)gridDim.x * kThreads) {
        const int kk = (int)k;
        const int z = kk / G.nxy;
        const int rem = kk - z * G.nxy;
        const int y = rem / G.nx;
        const int x = rem - y * G.nx;
        float ps_hi = 0.0f, ps_lo = 0.0f;
        if (storage >= LBM_MOM) {   // moment storages: p* is the first moment array
            ps_hi = ((const float *)gv)[k];
        } else if (pst) {   // 16-bit formats: p* = P + sum_i w_i h_i
            float s = pst[k];
#pragma unroll
            for (int i = 0; i < 27; ++i) s = fmaf(wgt(i), load_h16(gv, storage, i * N + k), s);
            ps_hi = s;
        } else {   // FP32 populations: an error-free FP32 sum (TwoSum; hi + lo carries p* to ~2^-46)
            const float *g = (const float *)gv;
            Pair a{};
#pragma unroll
            for (int i = 0; i < 27; ++i) pair_add(a, g[i * N + k]);
            ps_hi = a.hi, ps_lo = a.lo;
        }
        const float ph = phi[k];
        const float ux = u[k], uy = u[N + k], uz = u[2 * N + k];
        if (!(isfinite(ph) && isfinite(ux) && isfinite(uy) && isfinite(uz) && isfinite(ps_hi) && isfinite(ps_lo))) {
            ++nbad;
            continue;
        }
        // the (1 - phi)-weighted sums are formed at the end as (count, sum x, sum u) minus the
        // phi-weighted ones (obs_final_kernel); here F_SUM_GAS, F_XGAS, F_UGAS hold the former
        pair_add(sphi, ph);
        pair_add(sps, ps_hi);
        sps.lo = __fadd_rn(sps.lo, ps_lo);
        pair_add_coord(sxphi[0], ph, x, big);
        pair_add_coord(sxphi[1], ph, y, big);
        pair_add_coord(sxphi[2], ph, z, big);
        sx[0] += x, sx[1] += y, sx[2] += z;
        pair_add_prod(suphi[0], ph, ux);
        pair_add_prod(suphi[1], ph, uy);
        pair_add_prod(suphi[2], ph, uz);
        pair_add(su[0], ux);
        pair_add(su[1], uy);
        pair_add(su[2], uz);
        // pressure p = p* rho cs^2 for the phase means (an FP32 product: a diagnostic of the bulk).
        // The phases are phi > 0.999 and phi < 0.001: 0.999f is the least float above 0.999 and
        // 0.001f the least float above 0.001, so these FP32 tests select the same nodes.
        const bool liq = ph >= 0.999f, gas = ph < 0.001f;
        if (liq || gas) {
            const float p = __fadd_rn(ps_hi, ps_lo) * fmaf(ph, drho32, rho_g32) * (1.0f / 3.0f);
            if (liq) pair_add(spl, p), ++nliq;
            else pair_add(spg, p), ++ngas;
        }
        umax = fmaxf(umax, sqrtf(fmaf(ux, ux, fmaf(uy, uy, uz * uz))));
        phimin = fminf(phimin, ph);
        phimax = fmaxf(phimax, ph);
        ++nvalid;
        if (++cnt == kFlush) flush();
    }
    flush();
    r[F_SUM_GAS] = (double)nvalid;
    r[F_XGAS + 0] = (double)sx[0];
    r[F_XGAS + 1] = (double)sx[1];
    r[F_XGAS + 2] = (double)sx[2];
    r[F_NLIQ] = (double)nliq;
    r[F_NGAS] = (double)ngas;
    r[F_NONFIN] = (double)nbad;
    r[F_UMAX] = umax;
    r[F_PHIMIN] = nvalid ? (double)phimin : DBL_MAX;
    r[F_PHIMAX] = nvalid ? (double)phimax : -DBL_MAX;

    // warp stage
#pragma unroll
    for (int f = 0; f < F_USED; ++f)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) r[f] = combine(f, r[f], __shfl_down_sync(0xffffffffu, r[f], off));

    __shared__ double s[kThreads / 32][F_USED];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int f = 0; f < F_USED; ++f) s[warp][f] = r[f];
    __syncthreads();
    if (threadIdx.x < F_USED) {
        const int f = threadIdx.x;
        double acc = s[0][f];
        for (int w = 1; w < kThreads / 32; ++w) acc = combine(f, acc, s[w][f]);
        partials[(size_t)blockIdx.x * kObsFields + f] = acc;
    }
}

// Pass 2: one warp per record field.  Lane l combines the records of blocks l, l + 32, l + 64, ...
// in that order, then the 32 lane values meet in a fixed shuffle tree: the same order, and so the
// same bits, for a given block count.
__global__ void __launch_bounds__(F_USED * 32) obs_final_kernel(const double *__restrict__ partials, int nblocks,
                                                               double *__restrict__ out)
{
    __shared__ double tot[F_USED];
    const int f = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double acc = f == F_PHIMIN ? DBL_MAX : (f == F_UMAX || f == F_PHIMAX) ? -DBL_MAX : 0.0;
    for (int b = lane; b < nblocks; b += 32) acc = combine(f, acc, partials[(size_t)b * kObsFields + f]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc = combine(f, acc, __shfl_down_sync(0xffffffffu, acc, off));
    if (lane == 0) tot[f] = acc;
    __syncthreads();
    if (threadIdx.x >= F_USED) return;
    const int g = threadIdx.x;
    double v = tot[g];   // (1 - phi)-weighted sums: (count, sum x, sum u) minus the phi-weighted ones
    if (g == F_SUM_GAS) v -= tot[F_SUM_PHI];
    if (g >= F_XGAS && g < F_XGAS + 3) v -= tot[F_XPHI + g - F_XGAS];
    if (g >= F_UGAS && g < F_UGAS + 3) v -= tot[F_UPHI + g - F_UGAS];
    out[g] = v;
}

}  // namespace

int observables_blocks(const Grid &G)
{
    const long long need = ((long long)G.N + kThreads - 1) / kThreads;
    return (int)(need < kObsMaxBlocks ? need : kObsMaxBlocks);
}

cudaError_t launch_observables(const Grid &G, double rho_l, double rho_g, const void *g, const float *phi,
                               const float *u, double *partials, int nblocks, double *result, cudaStream_t s,
                               int storage, const float *pst)
{
    obs_partial_kernel<<<nblocks, kThreads, 0, s>>>(G, rho_g, rho_l - rho_g, g, storage, pst, phi, u, partials);
    obs_final_kernel<<<1, F_USED * 32, 0, s>>>(partials, nblocks, result);
    return cudaGetLastError();
}

}  // namespace tslb

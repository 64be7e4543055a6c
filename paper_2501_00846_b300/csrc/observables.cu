// FP64 conservation and interface diagnostics of the state (phi, ubar, p* = sum g).
// Pass 1: a grid-stride loop accumulates per-thread FP64 records, reduced in each block with
// warp shuffles and a shared-memory stage; each block writes one record of kObsFields doubles.
// Pass 2: one warp sums the block records in a fixed order (deterministic result).
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
    r[F_PHIMIN] = DBL_MAX;
    r[F_PHIMAX] = -DBL_MAX;
    const size_t N = (size_t)G.N;

    // 64-bit node index: with N close to 2^31 an int index would wrap past INT_MAX on its last
    // stride.  Inside the loop k < N < 2^31, so the coordinates come from 32-bit divisions.
    for (size_t k = (size_t)blockIdx.x * kThreads + threadIdx.x; k < N; k += (size_t)gridDim.x * kThreads) {
        const int kk = (int)k;
        const int z = kk / G.nxy;
        const int rem = kk - z * G.nxy;
        const int y = rem / G.nx;
        const int x = rem - y * G.nx;
        double ps = 0.0;
        if (storage >= LBM_MOM) {   // moment storages: p* is the first moment array
            ps = ((const float *)gv)[k];
        } else if (pst) {   // 16-bit formats: p* = P + sum_i w_i h_i
            float s = pst[k];
#pragma unroll
            for (int i = 0; i < 27; ++i) s = fmaf(wgt(i), load_h16(gv, storage, i * N + k), s);
            ps = s;
        } else {   // FP32 populations: an error-free FP32 sum (TwoSum; hi + lo carries p* to ~2^-46), then FP64
            const float *g = (const float *)gv;
            float hi = 0.0f, lo = 0.0f;
#pragma unroll
            for (int i = 0; i < 27; ++i) {
                const float a = g[i * N + k];
                const float sum = __fadd_rn(hi, a);
                const float bp = __fsub_rn(sum, hi);
                lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bp)), __fsub_rn(a, bp)));
                hi = sum;
            }
            ps = (double)hi + (double)lo;
        }
        const double ph = phi[k];
        const double ux = u[k], uy = u[N + k], uz = u[2 * N + k];
        if (!(isfinite(ph) && isfinite(ux) && isfinite(uy) && isfinite(uz) && isfinite(ps))) {
            r[F_NONFIN] += 1.0;
            continue;
        }
        const double rho = rho_g + ph * drho;
        // the (1 - phi)-weighted sums are formed at the end as (count, sum x, sum u) minus the
        // phi-weighted ones (obs_final_kernel); here F_SUM_GAS, F_XGAS, F_UGAS hold the former
        r[F_SUM_PHI] += ph;
        r[F_SUM_GAS] += 1.0;
        r[F_MASS] += rho;
        r[F_SUM_PS] += ps;
        r[F_MOM + 0] += rho * ux;
        r[F_MOM + 1] += rho * uy;
        r[F_MOM + 2] += rho * uz;
        r[F_XPHI + 0] += ph * x;
        r[F_XPHI + 1] += ph * y;
        r[F_XPHI + 2] += ph * z;
        r[F_XGAS + 0] += (double)x;
        r[F_XGAS + 1] += (double)y;
        r[F_XGAS + 2] += (double)z;
        r[F_UPHI + 0] += ph * ux;
        r[F_UPHI + 1] += ph * uy;
        r[F_UPHI + 2] += ph * uz;
        r[F_UGAS + 0] += ux;
        r[F_UGAS + 1] += uy;
        r[F_UGAS + 2] += uz;
        const double p = ps * rho * (1.0 / 3.0);
        if (ph > 0.999) { r[F_PLIQ] += p; r[F_NLIQ] += 1.0; }
        if (ph < 0.001) { r[F_PGAS] += p; r[F_NGAS] += 1.0; }
        r[F_UMAX] = fmax(r[F_UMAX], sqrt(ux * ux + uy * uy + uz * uz));
        r[F_PHIMIN] = fmin(r[F_PHIMIN], ph);
        r[F_PHIMAX] = fmax(r[F_PHIMAX], ph);
    }

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

__global__ void obs_final_kernel(const double *__restrict__ partials, int nblocks, double *__restrict__ out)
{
    __shared__ double tot[F_USED];
    const int f = threadIdx.x;
    if (f < F_USED) {
        double acc = partials[f];
        for (int b = 1; b < nblocks; ++b) acc = combine(f, acc, partials[(size_t)b * kObsFields + f]);
        tot[f] = acc;
    }
    __syncwarp();
    if (f >= F_USED) return;
    double v = tot[f];   // (1 - phi)-weighted sums: (count, sum x, sum u) minus the phi-weighted ones
    if (f == F_SUM_GAS) v -= tot[F_SUM_PHI];
    if (f >= F_XGAS && f < F_XGAS + 3) v -= tot[F_XPHI + f - F_XGAS];
    if (f >= F_UGAS && f < F_UGAS + 3) v -= tot[F_UPHI + f - F_UGAS];
    out[f] = v;
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
    obs_final_kernel<<<1, 32, 0, s>>>(partials, nblocks, result);
    return cudaGetLastError();
}

}  // namespace tslb

// Diagnostics of a caller-owned state with no device allocation (lbm_observables_noalloc).
//
// Some callers cannot allocate device memory: code that runs inside a host application whose
// device memory is managed entirely by someone else (a fixed arena handed out at start-up, a
// framework whose caching allocator must see every allocation), or code that runs where a
// cudaMalloc would synchronise the device and stall work the caller has queued.  This entry
// point gives them the FP64 diagnostics of a state they own, using a scratch buffer that lives
// in the library image itself instead of a per-call or per-context allocation.
//
// Scratch: one file-scope __device__ array of kMaxBlocks + 1 records of kObsFields doubles
// (1185 x 32 x 8 B = 303,360 B).  Every GPU that loads the library holds it until the process
// exits.  The reduction never uses more than kMaxBlocks blocks (it strides over the grid), so
// every box with fewer than 2^31 nodes fits; larger boxes are rejected with LBM_ERR_ARG.
// Every record the final pass reads is written earlier in the same call, so nothing has to be
// cleared between calls.  All calls share the one array: two calls whose kernels overlap on
// the GPU (for example on two streams) race on it and both results are undefined.
#include <math.h>
#include <mutex>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cuda_runtime.h>

#include "lbm.h"
#include "tslb_internal.h"

namespace {

constexpr int kMaxBlocks = tslb::kObsMaxBlocks;   // the most blocks the reduction's first pass launches
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_obs_scratch[(kMaxBlocks + 1) * tslb::kObsFields];
static_assert(sizeof(g_obs_scratch) == 303360, "the scratch size is stated in lbm.h: update it there too");

// Device address of the scratch array, looked up once per device with that device current.
// In host code the name g_obs_scratch is only a host-side stand-in for the symbol, not a device
// address: handing it to a kernel would fault (or, where the GPU can reach host memory, silently
// use the wrong memory).  Kernels get the address returned by cudaGetSymbolAddress.
std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices] = {};

lbm_status noalloc_fail(lbm_status s, const char *fmt, ...)
{
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    tslb::set_last_error(msg);
    return s;
}

lbm_status scratch_for_current_device(double **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(LBM_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(LBM_ERR_ARG, "device index %d not supported", dev);
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_obs_scratch);
        if (e != cudaSuccess || !p)
            return noalloc_fail(LBM_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_observables_noalloc(const float *g, const float *phi, const float *u, int nx, int ny,
                                              int nz, double rho_l, double rho_g, void *stream, lbm_obs *out)
{
    if (!g || !phi || !u || !out) return noalloc_fail(LBM_ERR_ARG, "g, phi, u and out are required");
    if (nx < 1 || ny < 1 || nz < 1) return noalloc_fail(LBM_ERR_ARG, "nx, ny, nz must be >= 1");
    const long long n = (long long)nx * ny * nz;
    if (n >= (1LL << 31))
        return noalloc_fail(LBM_ERR_ARG, "box of %lld nodes exceeds the maximum of 2^31 - 1 nodes", n);
    if (!(rho_l > 0) || !(rho_g > 0)) return noalloc_fail(LBM_ERR_ARG, "densities must be > 0");

    double *scratch = nullptr;
    lbm_status st = scratch_for_current_device(&scratch);
    if (st != LBM_OK) return st;

    tslb::Grid G;
    G.nx = nx;
    G.ny = ny;
    G.nz = nz;
    G.nxy = nx * ny;
    G.N = (int)n;
    G.wall = 0;
    const int nblocks = tslb::observables_blocks(G);
    if (nblocks > kMaxBlocks) return noalloc_fail(LBM_ERR_ARG, "reduction needs %d blocks > %d", nblocks, kMaxBlocks);
    double *partials = scratch;
    double *result = scratch + (size_t)kMaxBlocks * tslb::kObsFields;
    cudaStream_t s = (cudaStream_t)stream;

    cudaError_t e = tslb::launch_observables(G, rho_l, rho_g, g, phi, u, partials, nblocks, result, s);
    if (e != cudaSuccess) return noalloc_fail(LBM_ERR_CUDA, "reduction launch: %s", cudaGetErrorString(e));
    double r[tslb::kObsFields];
    e = cudaMemcpyAsync(r, result, sizeof r, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return noalloc_fail(LBM_ERR_CUDA, "result copy: %s", cudaGetErrorString(e));

    memset(out, 0, sizeof *out);
    out->step = 0.0;
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
    if (out->n_nonfinite > 0) return noalloc_fail(LBM_ERR_NONFINITE, "%.0f non-finite nodes", out->n_nonfinite);
    return LBM_OK;
}

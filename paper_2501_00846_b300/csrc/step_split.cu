// Two-kernel step: the Allen–Cahn kernel (ac_div.cuh: a linear stencil of phi^n and the flux
// W^n) writes phi^{n+1}; the one-thread-per-node lattice Boltzmann kernel (step_unfused.cu, or
// step_lbm16.cu for 16-bit populations) then streams the populations and writes W^{n+1}.
#include <cstdint>
#include <mutex>

#include "ac_div.cuh"
#include "tslb_internal.h"

namespace tslb {
namespace {

constexpr int RY = 4;               // output rows per warp
constexpr int WPB = 4;              // warps per CTA

template <bool WALL>
__global__ void __launch_bounds__(WPB * 32) ac_div_kernel(Grid G, Phys P, const float *__restrict__ phi,
                                                          const float *__restrict__ w, float *__restrict__ phi_out,
                                                          int ncols, int zlen, int tasks)
{
    pdl_trigger();
    pdl_wait();
    const int nwarps = gridDim.x * WPB;
    for (int task = blockIdx.x * WPB + (threadIdx.x >> 5); task < tasks; task += nwarps) {
        const int col = task % ncols;
        const int z0 = (task / ncols) * zlen;
        ac_div_task<WALL, RY>(G, P, phi, w, phi_out, col, z0, min(G.nz, z0 + zlen));
    }
}

constexpr int RYV = 2;              // output rows per warp, vector form
constexpr bool PREF = true;         // vector form: load the next plane while computing this one

template <bool WALL, bool XWRAP>
__global__ void __launch_bounds__(WPB * 32) ac_div4_kernel(Grid G, Phys P, const float *__restrict__ phi,
                                                           const float *__restrict__ w, float *__restrict__ phi_out,
                                                           int ncols, int zlen, int tasks)
{
    pdl_trigger();
    pdl_wait();
    const int nwarps = gridDim.x * WPB;
    for (int task = blockIdx.x * WPB + (threadIdx.x >> 5); task < tasks; task += nwarps) {
        const int col = task % ncols;
        const int z0 = (task / ncols) * zlen;
        ac_div_task4<WALL, RYV, XWRAP, PREF>(G, P, phi, w, phi_out, col, z0, min(G.nz, z0 + zlen));
    }
}

using AcKernel = void (*)(Grid, Phys, const float *, const float *, float *, int, int, int);

// The kernel for a box: the vector form when the x extent is a multiple of 128 and the arrays
// are 16-byte aligned, else the scalar form; rows is its number of output rows per warp.
AcKernel pick_ac(const Grid &G, const float *phi_in, const float *w, const float *phi_out, int &rows, int &xcols)
{
    const bool aligned = ((reinterpret_cast<uintptr_t>(phi_in) | reinterpret_cast<uintptr_t>(w) |
                           reinterpret_cast<uintptr_t>(phi_out)) & 15) == 0;
    if (G.nx % AC_XV == 0 && aligned) {
        rows = RYV;
        xcols = AC_XV;
        if (G.nx == AC_XV) return G.wall ? ac_div4_kernel<true, true> : ac_div4_kernel<false, true>;
        return G.wall ? ac_div4_kernel<true, false> : ac_div4_kernel<false, false>;
    }
    rows = RY;
    xcols = AC_XO;
    return G.wall ? ac_div_kernel<true> : ac_div_kernel<false>;
}

// Resident warps of an Allen–Cahn kernel on the current device, computed once per (device,
// kernel) and then read from a small table.
cudaError_t ac_warp_slots(AcKernel k, int &slots)
{
    struct Entry {
        int dev;
        AcKernel k;
        int slots;
    };
    constexpr int kEntries = 32;
    static Entry table[kEntries];
    static int used = 0;
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < used; ++i)
        if (table[i].dev == dev && table[i].k == k) {
            slots = table[i].slots;
            return cudaSuccess;
        }
    int sms = 0, per_sm = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, WPB * 32, 0)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    slots = sms * per_sm * WPB;
    if (used < kEntries) table[used++] = Entry{dev, k, slots};
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_ac_div(const Grid &G, const Phys &P, const float *phi_in, const float *w, float *phi_out,
                          int zchunks, cudaStream_t s)
{
    int rows = 0, xcols = 0, warp_slots = 0;
    const AcKernel k = pick_ac(G, phi_in, w, phi_out, rows, xcols);
    const cudaError_t e = ac_warp_slots(k, warp_slots);
    if (e != cudaSuccess) return e;
    const int ncols = ((G.nx + xcols - 1) / xcols) * ((G.ny + rows - 1) / rows);
    // default: as many z chunks as keep every task in one wave of resident warps, chunks of at
    // least 2 planes.  A warp's planes form a chain of dependent loads, so on boxes with few
    // column tiles the step time follows the chunk length, not the 2 halo planes each chunk adds
    // (measured: 64^3 takes 6.0 us in 2-plane chunks against 11.4 us in 16-plane ones)
    int m = zchunks;
    if (m <= 0) {
        m = warp_slots / ncols;
        if (m > G.nz / 2) m = G.nz / 2;
        if (m < 1) m = 1;
    }
    if (m > G.nz) m = G.nz;
    const int zlen = (G.nz + m - 1) / m;
    m = (G.nz + zlen - 1) / zlen;
    const int tasks = ncols * m;
    const int warps = tasks < warp_slots ? tasks : warp_slots;
    const int ctas = (warps + WPB - 1) / WPB;
    return launch_pdl(k, dim3(ctas), dim3(WPB * 32), 0, s, G, P, phi_in, w, phi_out, ncols, zlen, tasks);
}

cudaError_t launch_step_split(const Grid &G, const Phys &P, const StepArgs &a, int zchunks, cudaStream_t s)
{
    cudaError_t e = launch_ac_div(G, P, a.phi_in, a.flux, a.phi_out, zchunks, s);
    if (e != cudaSuccess) return e;
    if (a.storage >= LBM_MOM)
        return launch_mom(G, P, a.storage, a.g_in, a.u_in, a.phi_out, a.g_out, a.u_out, a.flux, zchunks, s);
    if (a.storage != 0)
        return launch_lbm16(G, P, a.storage, a.g_in, a.p_in, a.phi_out, a.u_in, a.g_out, a.p_out, a.u_out, a.flux,
                            zchunks, s);
    return launch_lbm(G, P, 0, a.g_in, nullptr, a.phi_out, a.u_in, a.g_out, nullptr, a.u_out, a.flux, s);
}

}  // namespace tslb

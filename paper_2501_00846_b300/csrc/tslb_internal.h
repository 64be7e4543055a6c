// Internal launch interface shared by the translation units of the library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include "lbm.h"
#include "mom_device.cuh"
#include "tslb_device.cuh"

namespace tslb {

// Launches kernel k with programmatic stream serialisation, so that it is scheduled while the
// previous kernel on the stream drains; k must call pdl_wait() before touching global memory.
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

struct StepArgs {
    const float *g_in;       // populations (FP32 g, 16-bit h for storage 1 / 2, moments for 3)
    float *g_out;
    const float *phi_in;
    float *phi_out;
    const float *u_in;
    float *u_out;
    float *flux;           // 3N Allen–Cahn flux W: read (W^n) and rewritten (W^{n+1}) by the two-kernel
                           // step; scratch of the unfused path; unused by the fused path
    int storage = 0;       // 0 FP32, 1 BF16, 2 FP16, 3..5 moments (paths 0 and 1 only for 1..5)
    const float *p_in = nullptr;   // stored p* of the 16-bit formats
    float *p_out = nullptr;
    int advect = 0;                // 1: literal advection u . grad(phi) (unfused path only)
};

// One step S^n -> S^{n+1}.  zchunks = z chunks per column tile of the marching kernels (<= 0:
// the default for the grid and GPU).
cudaError_t launch_step_split(const Grid &G, const Phys &P, const StepArgs &a, int zchunks, cudaStream_t s);
cudaError_t launch_step_unfused(const Grid &G, const Phys &P, const StepArgs &a, cudaStream_t s);
cudaError_t launch_step_fused2(const Grid &G, const Phys &P, const StepArgs &a, int zchunks, cudaStream_t s);

// The two kernels of the two-kernel step: phi^{n+1} = phi^n - div W^n + D lap phi^n from
// (phi^n, W^n), then the lattice Boltzmann update of every node from g^n, phi^{n+1} and ubar^n,
// which also writes W^{n+1} = W(phi^{n+1}, u^{n+1}) into w_out when w_out is not null.
cudaError_t launch_ac_div(const Grid &G, const Phys &P, const float *phi_in, const float *w, float *phi_out,
                          int zchunks, cudaStream_t s);
// storage: 0 FP32 g; 1 BF16, 2 FP16 h (see the storage formats) with P in p_in / p_out; 3 the
// moment arrays (one thread per node, lbm_mom_plain_kernel).
cudaError_t launch_lbm(const Grid &G, const Phys &P, int storage, const void *g_in, const float *p_in,
                       const float *phi_new, const float *u_in, void *g_out, float *p_out, float *u_out,
                       float *w_out, cudaStream_t s);
// W = W(phi, ubar) at every node (the flux the lattice Boltzmann kernels write), for a state set
// from outside the step (initialisation, restore, after a path that does not keep W).
cudaError_t launch_flux(const Grid &G, const Phys &P, const float *phi, const float *u, float *w, cudaStream_t s);

// z-marching lattice Boltzmann kernel for the 16-bit formats (storage 1 BF16, 2 FP16), with (P,
// ubar) and phi^{n+1} staged in shared memory once per plane; arguments as launch_lbm, zchunks as
// for the other marching kernels (<= 0: the default for the grid and GPU).
cudaError_t launch_lbm16(const Grid &G, const Phys &P, int storage, const void *h_in, const float *p_in,
                         const float *phi_new, const float *u_in, void *h_out, float *p_out, float *u_out,
                         float *w_out, int zchunks, cudaStream_t s);

// 16-bit population formats (h and P; see the storage formats in tslb_device.cuh):
// initialise from equilibrium (h = 0, P = p*0 or 0), expand to FP32 g (directions [i0, i0+ni)
// at g[(i-i0)*N + node]), compress FP32 g back (mode 0: P += sum g; mode 1: h and the
// rounding correction corr += sum w h), and apply the correction P -= corr.
cudaError_t launch_init16(const Grid &G, int storage, const float *pstar, void *h, float *pst, cudaStream_t s);
cudaError_t launch_expand16(const Grid &G, int storage, const void *h, const float *pst, const float *u, int i0,
                            int ni, float *g, cudaStream_t s);
cudaError_t launch_compress16(const Grid &G, int storage, const float *g, const float *u, int i0, int ni, int mode,
                              void *h, float *pst, float *corr, cudaStream_t s);
cudaError_t launch_finish16(const Grid &G, const float *corr, float *pst, cudaStream_t s);

// Moment storage (mom_device.cuh; storage LBM_MOM, LBM_MOM_BF16 or LBM_MOM_FP16): bytes of one
// state copy, the tiled step kernel (zchunks as for the marching kernels), the
// one-thread-per-node kernel, the equilibrium start (p* = pstar or 0, a = B = 0), the expansion to
// FP32 g (directions [i0, i0+ni) at g[(i-i0)*N + node]), and the import of FP32 g: acc (10 FP32
// arrays) += population moments of directions [i0, i0+ni), then (p*, a, B) from acc and u into m
// (m may be acc for LBM_MOM).
size_t mom_state_bytes(int storage, size_t N);
cudaError_t launch_mom(const Grid &G, const Phys &P, int storage, const float *m_in, const float *u_in,
                       const float *phi_new, float *m_out, float *u_out, float *w_out, int zchunks, cudaStream_t s);
cudaError_t launch_mom_plain(const Grid &G, const Phys &P, int storage, const float *m_in, const float *u_in,
                             const float *phi_new, float *m_out, float *u_out, float *w_out, cudaStream_t s);
cudaError_t launch_mom_init(const Grid &G, int storage, const float *pstar, float *m, cudaStream_t s);
cudaError_t launch_mom_expand(const Grid &G, int storage, const float *m, const float *u, int i0, int ni, float *g,
                              cudaStream_t s);
cudaError_t launch_mom_project(const Grid &G, const float *g, int i0, int ni, float *acc, cudaStream_t s);
cudaError_t launch_mom_finish(const Grid &G, int storage, const float *u, const float *acc, float *m, cudaStream_t s);

// g = f^eq(p*, u); pstar may be nullptr (p* = 0).
cudaError_t launch_init(const Grid &G, const float *pstar, const float *u, float *g, cudaStream_t s);

// p = p* rho cs^2 with p* = sum_i g_i (FP32, pst null), P + sum_i w_i h_i (16-bit formats) or the
// stored p* (moment storages: g holds the moment state, p* first).
cudaError_t launch_pressure(const Grid &G, const Phys &P, int storage, const void *g, const float *pst,
                            const float *phi, float *p, cudaStream_t s);

// FP64 reductions: number of doubles in one partial record, and the two-pass reduction.
constexpr int kObsFields = 32;
// Most blocks the first pass launches (it strides over the grid beyond that): 8 per SM of a B300.
constexpr int kObsMaxBlocks = 148 * 8;
int observables_blocks(const Grid &G);   // min(ceil(N / 256), kObsMaxBlocks)
// rho_l, rho_g in FP64 so the mass sum uses the exact parameter values.
// p* is summed from the 27 FP32 population arrays g, or (storage 1 / 2, pst not null) is
// P + sum_i w_i h_i of a 16-bit format whose h arrays g points to, or (storage 3..5) is the
// first array of the moment state g points to.
cudaError_t launch_observables(const Grid &G, double rho_l, double rho_g, const void *g, const float *phi,
                               const float *u, double *partials, int nblocks, double *result, cudaStream_t s,
                               int storage = 0, const float *pst = nullptr);

// Message returned by lbm_last_error() for the calling thread.
void set_last_error(const char *msg);

// Parameter validation of lbm_create (sets the thread's last error) and the kernel constants of
// a parameter set; shared by the one-box context and the ensemble.
lbm_status check_params(const lbm_params *p);
void params_to_consts(const lbm_params &p, Grid &G, Phys &P);

// The one-box context's current state, for the closure (closure.cu).
struct CtxView {
    Grid G;
    Phys P;
    float *g, *phi, *u;
    int storage;
    cudaStream_t stream;
};
lbm_status ctx_view(lbm_ctx *ctx, CtxView *v);
// Mark the context's carried Allen–Cahn flux stale after its state was changed in place.
void ctx_state_changed(lbm_ctx *ctx);

}  // namespace tslb

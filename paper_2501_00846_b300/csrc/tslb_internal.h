// Internal launch interface shared by the translation units of the library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include "tslb_device.cuh"

namespace tslb {

struct StepArgs {
    const float *g_in;
    float *g_out;
    const float *phi_in;
    float *phi_out;
    const float *u_in;
    float *u_out;
    float *flux;           // 3N scratch of the unfused path (Allen–Cahn flux); unused by the fused path
};

// One step S^n -> S^{n+1}.  zchunks = z chunks per column tile of the marching kernels (<= 0:
// the default for the grid and GPU).
cudaError_t launch_step_split(const Grid &G, const Phys &P, const StepArgs &a, int zchunks, cudaStream_t s);
cudaError_t launch_step_unfused(const Grid &G, const Phys &P, const StepArgs &a, cudaStream_t s);
cudaError_t launch_step_fused2(const Grid &G, const Phys &P, const StepArgs &a, int zchunks, cudaStream_t s);

// The two kernels of the two-kernel step: phi^{n+1} from (phi^n, ubar^n), then the lattice
// Boltzmann update of every node from g^n, phi^{n+1} and ubar^n.
cudaError_t launch_ac_split(const Grid &G, const Phys &P, const float *phi_in, const float *u_in, float *phi_out,
                            int zchunks, cudaStream_t s);
cudaError_t launch_lbm(const Grid &G, const Phys &P, const float *g_in, const float *phi_new, const float *u_in,
                       float *g_out, float *u_out, cudaStream_t s);

// g = f^eq(p*, u); pstar may be nullptr (p* = 0).
cudaError_t launch_init(const Grid &G, const float *pstar, const float *u, float *g, cudaStream_t s);

// p = (sum_i g_i) rho cs^2.
cudaError_t launch_pressure(const Grid &G, const Phys &P, const float *g, const float *phi, float *p,
                            cudaStream_t s);

// FP64 reductions: number of doubles in one partial record, and the two-pass reduction.
constexpr int kObsFields = 32;
int observables_blocks(const Grid &G);
// rho_l, rho_g in FP64 so the mass sum uses the exact parameter values.
cudaError_t launch_observables(const Grid &G, double rho_l, double rho_g, const float *g, const float *phi,
                               const float *u, double *partials, int nblocks, double *result, cudaStream_t s);

// Message returned by lbm_last_error() for the calling thread.
void set_last_error(const char *msg);

}  // namespace tslb

// The lattice Boltzmann update of one node: pull streaming with halfway bounce-back at z walls,
// the 27-point phi^{n+1} stencil, the regularised collision (collide_node), and the stores of the
// node's populations, velocity and Allen–Cahn flux.
#pragma once

#include "tslb_device.cuh"

namespace tslb {

// Lattice Boltzmann update of node (x, y, z) (pull, forces from phi^{n+1}, regularised
// collision), shared by the one-box kernels and the batched ensemble kernel.  S selects the
// population format: FP32 g, or a 16-bit deviation from equilibrium h_i with P in FP32 (pin / pout; see the storage formats in tslb_device.cuh).  A 16-bit puller
// rebuilds g_i(x - c_i) = w_i (P + f^eq_i(0, ubar) / w_i + h_i) from the source node's P, ubar
// and h; the collision forms h_i = (g_i - f^eq_i(p*, u)) / w_i directly and stores it with
// P = p* - sum w_i h_i(rounded).
template <class S>
__device__ __forceinline__ void lbm_node(const Grid &G, const Phys &P, const typename S::T *__restrict__ gin,
                                         const float *__restrict__ pin, const float *__restrict__ phi_new,
                                         const float *__restrict__ ubar, typename S::T *__restrict__ gout,
                                         float *__restrict__ pout, float *__restrict__ uout, float *__restrict__ wout,
                                         int x, int y, int z)
{
    const Nbr n = make_nbr(x, y, z, G);
    const int k = n.zo[1] + n.yo[1] + x;
    const size_t N = (size_t)G.N;
    const bool wlo = G.wall && z == 0;
    const bool whi = G.wall && z == G.nz - 1;

    // pull f_i(x) = g_i(x - c_i); at a wall the population returns reversed: g_{26-i}(x)
    float f[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const int j = n.zo[1 - cz(i)] + n.yo[1 - cy(i)] + n.xo[1 - cx(i)];
        bool bounce = false;
        if (cz(i) == 1) bounce = wlo;
        if (cz(i) == -1) bounce = whi;
        const int src = bounce ? k : j;
        const size_t at = (size_t)(bounce ? 26 - i : i) * N + src;
        if (S::kShifted) {
            const float vx = __ldg(ubar + src), vy = __ldg(ubar + N + src), vz = __ldg(ubar + 2 * N + src);
            const float v2 = vx * vx + vy * vy + vz * vz;
            const float cu = cdot(i, vx, vy, vz);
            const float e = eq_shifted(bounce ? -cu : cu, v2);
            f[i] = wgt(i) * (__ldg(pin + src) + e + S::to_f(gin[at]));
        } else {
            f[i] = S::to_f(gin[at]);
        }
    }

    float ps[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) ps[i] = __ldg(phi_new + nidx(n, i));
    float gx, gy, gz, lap;
    grad_lap27(ps, gx, gy, gz, lap);

    float g[27], ux, uy, uz, pstar;
    collide_node<S::kShifted>(f, ps[13], gx, gy, gz, lap, ubar[k], ubar[N + k], ubar[2 * N + k], P, g, ux, uy, uz,
                              &pstar);
    if (S::kShifted) {
        float sum = 0.0f;
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            const typename S::T h = S::from_f(g[i]);
            gout[i * N + k] = h;
            sum = fmaf(wgt(i), S::to_f(h), sum);
        }
        pout[k] = pstar - sum;
    } else {
#pragma unroll
        for (int i = 0; i < 27; ++i) gout[i * N + k] = S::from_f(g[i]);
    }
    uout[k] = ux;
    uout[N + k] = uy;
    uout[2 * N + k] = uz;
    if (wout) {   // Allen–Cahn flux of the new state for the next step
        float wx, wy, wz;
        ac_flux(ps[13], gx, gy, gz, ux, uy, uz, P, wx, wy, wz);
        const unsigned long long pol = l2_keep_policy();
        st_keep(wout + k, wx, pol);
        st_keep(wout + N + k, wy, pol);
        st_keep(wout + 2 * N + k, wz, pol);
    }
}

}  // namespace tslb

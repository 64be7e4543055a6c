// Device building blocks of the coupled TSLB + conservative Allen–Cahn step (arXiv 2501.00846).
//
// D3Q27, cs^2 = 1/3, dx = dt = 1.  Velocity index i = 9 (cz+1) + 3 (cy+1) + (cx+1); opposite
// 26 - i; rest 13.  Every loop over i is unrolled at compile time, so each c_i component is a
// literal {-1, 0, 1} and the products with it fold into adds.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tslb {

__host__ __device__ constexpr int cx(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int cy(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int cz(int i) { return i / 9 - 1; }
__host__ __device__ constexpr int cnorm2(int i) { return cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i); }
// weights: 8/27 rest, 2/27 faces, 1/54 edges, 1/216 corners
__host__ __device__ constexpr float wgt(int i)
{
    return cnorm2(i) == 0 ? 8.0f / 27.0f : cnorm2(i) == 1 ? 2.0f / 27.0f : cnorm2(i) == 2 ? 1.0f / 54.0f : 1.0f / 216.0f;
}

// Physical constants of one launch (FP32).
struct Phys {
    float rho_g, drho;     // rho = rho_g + phi * drho
    float mu_g, dmu;       // mu  = mu_g  + phi * dmu
    float beta4, kappa;    // mu_phi = beta4 phi (phi-1)(phi-1/2) - kappa lap(phi); beta4 = 48 sigma/W
    float mob, kac;        // Allen–Cahn diffusivity D and sharpening 4 D / W
    float grav[3];         // gravity vector
    float rho_ref;         // buoyancy reference density
    float body[3];         // uniform body-force density
};

struct Grid {
    int nx, ny, nz;
    int nxy;
    int N;                 // nx*ny*nz < 2^31
    int wall;              // 1: z walls
};

// Minimum |grad phi| of the interface normal n = grad(phi) / max(|grad(phi)|, eps) in FP32.
// The sharpening flux kappa_AC max(phi (1 - phi), 0) n weights the normal by zero wherever phi
// has left [0, 1] (an overshoot extremum, where n is undefined).
constexpr float kNormalEps = 1e-9f;

// Isotropic gradient and Laplacian of a scalar on the 27-point stencil (paper Section "Model
// extension", finite-difference formulas; Laplacian read as (2/cs^2) sum_{i!=0} w_i (psi_i - psi_0)).
// psi[i] holds psi(x + c_i).  Evaluated over opposite pairs (c, -c) from differences:
//   grad = 3 sum_pairs w c (psi_c - psi_-c),   lap = 6 sum_pairs w ((psi_c - psi_0) + (psi_-c - psi_0))
// The differences psi_c - psi_0 are exact in FP32 for neighbouring values of a smooth field, so the
// Laplacian carries no cancellation error of the size of psi itself.
__device__ __forceinline__ void grad27(const float (&psi)[27], float &gx, float &gy, float &gz)
{
    gx = gy = gz = 0.0f;
#pragma unroll
    for (int i = 0; i < 13; ++i) {
        const float a = psi[i] - psi[26 - i];
        const float w3 = 3.0f * wgt(i);
        if (cx(i)) gx = fmaf(cx(i) * w3, a, gx);
        if (cy(i)) gy = fmaf(cy(i) * w3, a, gy);
        if (cz(i)) gz = fmaf(cz(i) * w3, a, gz);
    }
}

__device__ __forceinline__ float lap27(const float (&psi)[27])
{
    const float p0 = psi[13];
    float l = 0.0f;
#pragma unroll
    for (int i = 0; i < 13; ++i) l = fmaf(6.0f * wgt(i), (psi[i] - p0) + (psi[26 - i] - p0), l);
    return l;
}

__device__ __forceinline__ void grad_lap27(const float (&psi)[27], float &gx, float &gy, float &gz, float &lap)
{
    grad27(psi, gx, gy, gz);
    lap = lap27(psi);
}

// Macroscopic update and third-order regularised collision of one node.
//   f        streamed populations f_i(x) = g_i(x - c_i)
//   phi      phase field phi^{n+1}(x); (gpx, gpy, gpz), lap: its gradient and Laplacian
//   ub*      lagged velocity ubar^n(x) (used by the viscous correction)
// Writes the post-collision populations g and the velocity u (Eq. moments1).
//
// Arithmetic (paper Eqs. moments0, moments1, eqts, noneqts, hermite_neq2, guoforce, press_corr,
// visc_corr; the forcing enters through the acceleration a = F/rho):
//   p* = sum f, j = sum f c, Pi = sum f c c
//   F = mu_phi grad(phi) - p* cs^2 grad(rho) - (1 - omega/2) [Pi - cs^2 p* I - ubar ubar] grad(rho)
//       + (rho - rho_ref) g + G_body                    (nu omega / cs^2 = 1 - omega/2)
//   u = j + a/2,  A = Pi - cs^2 p* I - u u + (u a + a u)/2
//   g_i = f^eq_i(p*, u) + (1 - omega) f^neq_i(A, u) + S_i(u, a)/2
// The collision is evaluated in even/odd form over opposite pairs (c, -c):
//   g_{+-c} = w (E +- O),
//   E = K0 + 4.5 cu (cu + ca) + k2 cAc,                       K0 = p* - 1.5 u^2 - 1.5 u.a - 1.5 (1-omega) trA
//   O = cu (K1 + 4.5 cu^2 + 3 k2 cAc) + c.v,                  K1 = 3 - 4.5 u^2 - k2 trA
//   k2 = 4.5 (1 - omega),  v = 1.5 a - 2 k2 A u
// which is the full contraction of the Hermite terms (H3_aaa vanishes on D3Q27).
__device__ __forceinline__ void collide_node(const float (&f)[27], float phi, float gpx, float gpy, float gpz,
                                             float lap, float ubx, float uby, float ubz, const Phys &P,
                                             float (&g)[27], float &ux, float &uy, float &uz)
{
    // moments over opposite pairs
    float ps = f[13];
    float jx = 0.f, jy = 0.f, jz = 0.f;
    float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
    for (int i = 0; i < 13; ++i) {
        const float s = f[i] + f[26 - i];
        const float d = f[i] - f[26 - i];
        ps += s;
        if (cx(i)) { jx += cx(i) * d; pxx += s; }
        if (cy(i)) { jy += cy(i) * d; pyy += s; }
        if (cz(i)) { jz += cz(i) * d; pzz += s; }
        if (cx(i) * cy(i)) pxy += (cx(i) * cy(i)) * s;
        if (cx(i) * cz(i)) pxz += (cx(i) * cz(i)) * s;
        if (cy(i) * cz(i)) pyz += (cy(i) * cz(i)) * s;
    }

    // local properties
    const float rho = fmaf(phi, P.drho, P.rho_g);
    const float irho = 1.0f / rho;
    const float mu = fmaf(phi, P.dmu, P.mu_g);
    const float nu = mu * irho;
    const float omega = 1.0f / fmaf(3.0f, nu, 0.5f);

    // forces
    const float third = 1.0f / 3.0f;
    const float pc = ps * third;
    const float mu_phi = P.beta4 * phi * (phi - 1.0f) * (phi - 0.5f) - P.kappa * lap;
    const float grx = P.drho * gpx, gry = P.drho * gpy, grz = P.drho * gpz;
    const float mxx = pxx - pc - ubx * ubx, myy = pyy - pc - uby * uby, mzz = pzz - pc - ubz * ubz;
    const float mxy = pxy - ubx * uby, mxz = pxz - ubx * ubz, myz = pyz - uby * ubz;
    const float cvis = -(1.0f - 0.5f * omega);
    const float bf = rho - P.rho_ref;
    const float Fx = mu_phi * gpx - pc * grx + cvis * (mxx * grx + mxy * gry + mxz * grz) + bf * P.grav[0] + P.body[0];
    const float Fy = mu_phi * gpy - pc * gry + cvis * (mxy * grx + myy * gry + myz * grz) + bf * P.grav[1] + P.body[1];
    const float Fz = mu_phi * gpz - pc * grz + cvis * (mxz * grx + myz * gry + mzz * grz) + bf * P.grav[2] + P.body[2];
    const float ax = Fx * irho, ay = Fy * irho, az = Fz * irho;

    // velocity (Eq. moments1) and pre-regularisation (closed form of Eq. hermite_neq2)
    ux = fmaf(0.5f, ax, jx);
    uy = fmaf(0.5f, ay, jy);
    uz = fmaf(0.5f, az, jz);
    const float Axx = pxx - pc - ux * ux + ux * ax;
    const float Ayy = pyy - pc - uy * uy + uy * ay;
    const float Azz = pzz - pc - uz * uz + uz * az;
    const float Axy = pxy - ux * uy + 0.5f * (ux * ay + ax * uy);
    const float Axz = pxz - ux * uz + 0.5f * (ux * az + ax * uz);
    const float Ayz = pyz - uy * uz + 0.5f * (uy * az + ay * uz);

    // collision constants
    const float om1 = 1.0f - omega;
    const float k2 = 4.5f * om1;
    const float k3 = 3.0f * k2;
    const float trA = Axx + Ayy + Azz;
    const float u2 = ux * ux + uy * uy + uz * uz;
    const float ua = ux * ax + uy * ay + uz * az;
    const float K0 = ps - 1.5f * u2 - 1.5f * ua - 1.5f * om1 * trA;
    const float K1 = 3.0f - 4.5f * u2 - k2 * trA;
    const float twok2 = 2.0f * k2;
    const float vx = 1.5f * ax - twok2 * (Axx * ux + Axy * uy + Axz * uz);
    const float vy = 1.5f * ay - twok2 * (Axy * ux + Ayy * uy + Ayz * uz);
    const float vz = 1.5f * az - twok2 * (Axz * ux + Ayz * uy + Azz * uz);
    const float A2xy = 2.0f * Axy, A2xz = 2.0f * Axz, A2yz = 2.0f * Ayz;

    g[13] = wgt(13) * K0;
#pragma unroll
    for (int i = 0; i < 13; ++i) {
        float cu = 0.f, ca = 0.f, cv = 0.f, cac = 0.f;
        if (cx(i)) { cu += cx(i) * ux; ca += cx(i) * ax; cv += cx(i) * vx; cac += Axx; }
        if (cy(i)) { cu += cy(i) * uy; ca += cy(i) * ay; cv += cy(i) * vy; cac += Ayy; }
        if (cz(i)) { cu += cz(i) * uz; ca += cz(i) * az; cv += cz(i) * vz; cac += Azz; }
        if (cx(i) * cy(i)) cac += (cx(i) * cy(i)) * A2xy;
        if (cx(i) * cz(i)) cac += (cx(i) * cz(i)) * A2xz;
        if (cy(i) * cz(i)) cac += (cy(i) * cz(i)) * A2yz;
        const float hcu = 4.5f * cu;
        const float E = fmaf(k2, cac, fmaf(hcu, cu + ca, K0));
        const float O = fmaf(cu, fmaf(k3, cac, fmaf(hcu, cu, K1)), cv);
        g[i] = wgt(i) * (E + O);
        g[26 - i] = wgt(i) * (E - O);
    }
}

// Equilibrium populations f^eq_i(p*, u) (Eq. eqts), even/odd form, for initialisation.
__device__ __forceinline__ void equilibrium(float ps, float ux, float uy, float uz, float (&g)[27])
{
    const float u2 = ux * ux + uy * uy + uz * uz;
    const float K0 = ps - 1.5f * u2;
    const float K1 = 3.0f - 4.5f * u2;
    g[13] = wgt(13) * K0;
#pragma unroll
    for (int i = 0; i < 13; ++i) {
        float cu = 0.f;
        if (cx(i)) cu += cx(i) * ux;
        if (cy(i)) cu += cy(i) * uy;
        if (cz(i)) cu += cz(i) * uz;
        const float E = fmaf(4.5f * cu, cu, K0);
        const float O = cu * fmaf(4.5f * cu, cu, K1);
        g[i] = wgt(i) * (E + O);
        g[26 - i] = wgt(i) * (E - O);
    }
}

}  // namespace tslb

// The Allen–Cahn update as a linear stencil of (phi, W), one warp per column tile; shared by the
// one-box kernel (step_split.cu) and the batched ensemble kernel.
//
// The flux W = ubar phi + kappa_AC max(phi (1 - phi), 0) n, n = grad phi / max(|grad phi|, eps),
// needs the gradient of phi and the velocity at the node: the lattice Boltzmann kernel of step n
// has both (grad phi^{n+1} for the surface-tension force, u^{n+1} from the collision), so it
// stores W^{n+1} next to ubar^{n+1}.  The Allen–Cahn update of step n+1,
//   phi^{n+2} = phi^{n+1} - div W^{n+1} + D lap phi^{n+1},
// is then a linear stencil of (phi, W): the same 20 bytes per node as reading phi and ubar, no
// normal or square root, and no barrier.
//
// The 27-point stencils factorise over the D3Q27 weights (w = w1 w1 w1, w1(0) = 2/3,
// w1(+-1) = 1/6) into 3x3 partials of one z plane combined over three planes:
//   Q  = Px[W_x] + Py[W_y],  Px[V] = 2/3 (V(x+1,y) - V(x-1,y)) + 1/6 sum_{dy=+-1} (V(x+1,y+dy) - V(x-1,y+dy))
//   T  = sum_{dx,dy} w1(dx) w1(dy) W_z(x+dx, y+dy)
//   Sd = sum_{dx,dy} w1(dx) w1(dy) (phi(x+dx, y+dy) - phi(x, y)),  c = phi(x, y)
//   div W   = 1/2 [2/3 Q(z) + 1/6 (Q(z-1) + Q(z+1))] + 1/2 [T(z+1) - T(z-1)]
//   lap phi = 6 [2/3 Sd(z) + 1/6 (Sd(z-1) + Sd(z+1)) + 1/6 ((c(z-1) - c(z)) + (c(z+1) - c(z)))]
// (the paper's isotropic gradient and, reading R2, Laplacian).  Both in-plane sums factorise once
// more, over y then x: with the y-sums of one column
//   Yp = 2/3 phi(y) + 1/6 (phi(y-1) + phi(y+1)),  Yx, Yz likewise for W_x, W_z,
//   Dy = W_y(y+1) - W_y(y-1),
// the partials are  Sd = 2/3 Yd(x) + 1/6 (Yd(x-1) + Yd(x+1)) + 1/6 ((c(x-1) - c) + (c(x+1) - c)),
// with Yd = 1/6 ((phi(y-1) - phi(y)) + (phi(y+1) - phi(y))) (difference form, as FP32 needs),
// Q = (Yx(x+1) - Yx(x-1)) + 2/3 Dy(x) + 1/6 (Dy(x-1) + Dy(x+1)),  T = 2/3 Yz(x) + 1/6 (Yz(x-1) + Yz(x+1)).
//
// One warp owns a column tile of 30 x RY nodes and marches a z chunk with no shared memory and no
// barrier: lane l holds column x0 - 1 + l (lanes 0 and 31 are the x halo), loads rows y0 - 1 ..
// y0 + RY of the plane (phi, W) with coalesced loads one plane ahead, forms the y-sums in
// registers and takes the x-neighbours' sums by warp shuffles.  Plane p (c_p = phi there)
// contributes to the targets p - 1, p, p + 1 (D is the mobility):
//   p - 1:  D (Sd + (c_p - c_{p-1})) - Q/12 - T/2      p:  D (4 Sd + (c_{p-1} - c_p)) - Q/3      p + 1:  D Sd - Q/12 + T/2
// accumulated in two registers per row; target p - 1 is complete after plane p and is stored as
// c_{p-1} + its sum (the z differences of c in the Laplacian are taken plane to plane, and the
// large c itself is added last, so Sum phi stays conserved to FP32 round-off).
// At a wall the ghost plane is the mirror image with W_z negated (R13), so the wall flux
// vanishes.
#pragma once

#include "tslb_device.cuh"

namespace tslb {

constexpr float AC_W0 = 2.0f / 3.0f, AC_W1 = 1.0f / 6.0f;

__device__ __forceinline__ int ac_wrapc(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

template <bool WALL>
__device__ __forceinline__ int ac_zmap(int p, int nz)
{
    if (WALL) return p < 0 ? -1 - p : (p >= nz ? 2 * nz - 1 - p : p);
    return p < 0 ? p + nz : (p >= nz ? p - nz : p);
}

template <bool WALL>
__device__ __forceinline__ float ac_zsign(int p, int nz)
{
    return (WALL && (p < 0 || p >= nz)) ? -1.0f : 1.0f;
}



constexpr int AC_XO = 30;           // output columns per warp (lanes 1..30)
constexpr unsigned AC_FULL = 0xffffffffu;

template <int NROW>
struct PlaneRows {
    float phi[NROW], wx[NROW], wy[NROW], wz[NROW];
};

template <int NROW>
__device__ __forceinline__ void load_rows(PlaneRows<NROW> &v, const float *__restrict__ phi,
                                          const float *__restrict__ w, size_t N, int plane_off,
                                          const int (&roff)[NROW], int xg)
{
#pragma unroll
    for (int r = 0; r < NROW; ++r) {
        const int at = plane_off + roff[r] + xg;
        v.phi[r] = __ldg(phi + at);
        v.wx[r] = __ldg(w + at);
        v.wy[r] = __ldg(w + N + at);
        v.wz[r] = __ldg(w + 2 * N + at);
    }
}

// One task of the Allen–Cahn update: the warp's column tile col (30 x RY output columns; tiles
// ordered x fastest) over the planes [z0, zend), for a box with grid G.
template <bool WALL, int RY>
__device__ __forceinline__ void ac_div_task(const Grid &G, const Phys &P, const float *__restrict__ phi,
                                            const float *__restrict__ w, float *__restrict__ phi_out, int col,
                                            int z0, int zend)
{
    constexpr int NROW = RY + 2;
    const int lane = threadIdx.x & 31;
    const int nx = G.nx, ny = G.ny, nz = G.nz, nxy = G.nxy;
    const int ncx = (nx + AC_XO - 1) / AC_XO;
    const size_t N = (size_t)G.N;
    const float D = P.mob;
    {
        const int x0 = (col % ncx) * AC_XO, y0 = (col / ncx) * RY;
        const int x = x0 - 1 + lane;                       // this lane's column (before wrapping)
        const int xg = ac_wrapc(x, nx);
        const bool xout = lane >= 1 && lane <= AC_XO && x < nx;
        int roff[NROW];
#pragma unroll
        for (int r = 0; r < NROW; ++r) roff[r] = ac_wrapc(y0 - 1 + r, ny) * nx;

        float acc1[RY], acc2[RY], cprev[RY];
#pragma unroll
        for (int r = 0; r < RY; ++r) acc1[r] = acc2[r] = cprev[r] = 0.0f;
        PlaneRows<NROW> cur, nxt;
        load_rows(cur, phi, w, N, ac_zmap<WALL>(z0 - 1, nz) * nxy, roff, xg);
        for (int p = z0 - 1; p <= zend; ++p) {
            if (p + 1 <= zend) load_rows(nxt, phi, w, N, ac_zmap<WALL>(p + 1, nz) * nxy, roff, xg);
            const float sg = ac_zsign<WALL>(p, nz);
            const bool store = p - 1 >= z0;
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                // y-sums of this column (phi in difference form against the row's own value)
                const float c = cur.phi[r + 1];
                const float yd = AC_W1 * ((cur.phi[r] - c) + (cur.phi[r + 2] - c));
                const float yx = fmaf(AC_W0, cur.wx[r + 1], AC_W1 * (cur.wx[r] + cur.wx[r + 2]));
                const float dy = cur.wy[r + 2] - cur.wy[r];
                const float yz = fmaf(AC_W0, cur.wz[r + 1], AC_W1 * (cur.wz[r] + cur.wz[r + 2]));
                // the x-neighbours' sums
                const float cl = __shfl_up_sync(AC_FULL, c, 1), cr = __shfl_down_sync(AC_FULL, c, 1);
                const float ydl = __shfl_up_sync(AC_FULL, yd, 1), ydr = __shfl_down_sync(AC_FULL, yd, 1);
                const float yxl = __shfl_up_sync(AC_FULL, yx, 1), yxr = __shfl_down_sync(AC_FULL, yx, 1);
                const float dyl = __shfl_up_sync(AC_FULL, dy, 1), dyr = __shfl_down_sync(AC_FULL, dy, 1);
                const float yzl = __shfl_up_sync(AC_FULL, yz, 1), yzr = __shfl_down_sync(AC_FULL, yz, 1);
                // plane partials: Sd (difference form), Q, T
                const float sd = fmaf(AC_W0, yd, AC_W1 * ((ydl + ydr) + ((cl - c) + (cr - c))));
                const float q = (yxr - yxl) + fmaf(AC_W0, dy, AC_W1 * (dyl + dyr));
                const float t = sg * fmaf(AC_W0, yz, AC_W1 * (yzl + yzr));
                // contributions of plane p to the targets p - 1, p, p + 1; the z differences of c
                // are taken between neighbouring planes (cp = c of plane p - 1), and each target's
                // own c is added last
                const float cp = cprev[r];
                const float qs = q * (-1.0f / 12.0f);
                const float lo = fmaf(D, sd + (c - cp), fmaf(-0.5f, t, qs));
                const float mid = fmaf(D, fmaf(4.0f, sd, cp - c), q * (-1.0f / 3.0f));
                const float hi = fmaf(D, sd, fmaf(0.5f, t, qs));
                const float done = cp + (acc1[r] + lo);                  // phi^{n+1} of plane p - 1
                if (store && xout && y0 + r < ny) phi_out[(size_t)(p - 1) * nxy + (y0 + r) * nx + x] = done;
                acc1[r] = acc2[r] + mid;
                acc2[r] = hi;
                cprev[r] = c;
            }
            cur = nxt;
        }
    }
}

}  // namespace tslb

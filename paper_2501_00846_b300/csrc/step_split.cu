// Two-kernel step: a z-marching Allen–Cahn kernel writes phi^{n+1}; the one-thread-per-node
// lattice Boltzmann kernel (step_unfused.cu, or step_lbm16.cu for 16-bit populations) then
// streams the populations and also writes the Allen–Cahn flux of the new state.
//
// The flux W = ubar phi + kappa_AC max(phi (1 - phi), 0) n, n = grad phi / max(|grad phi|, eps),
// needs the gradient of phi and the velocity at the node: the lattice Boltzmann kernel of step n
// has both (grad phi^{n+1} for the surface-tension force, u^{n+1} from the collision), so it
// stores W^{n+1} next to ubar^{n+1}.  The Allen–Cahn update of step n+1,
//   phi^{n+2} = phi^{n+1} - div W^{n+1} + D lap phi^{n+1},
// is then a linear stencil of (phi, W): the same 20 bytes per node as reading phi and ubar, no
// normal or square root, and one barrier per plane.
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
#include "tslb_internal.h"

namespace tslb {
namespace {

constexpr float W0 = 2.0f / 3.0f, W1 = 1.0f / 6.0f;

__device__ __forceinline__ int wrapc(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

template <bool WALL>
__device__ __forceinline__ int zmap(int p, int nz)
{
    if (WALL) return p < 0 ? -1 - p : (p >= nz ? 2 * nz - 1 - p : p);
    return p < 0 ? p + nz : (p >= nz ? p - nz : p);
}

template <bool WALL>
__device__ __forceinline__ float zsign(int p, int nz)
{
    return (WALL && (p < 0 || p >= nz)) ? -1.0f : 1.0f;
}

constexpr int XO = 30;              // output columns per warp (lanes 1..30)
constexpr int RY = 4;               // output rows per warp
constexpr int NROW = RY + 2;        // rows loaded per plane
constexpr int WPB = 4;              // warps per CTA
constexpr unsigned FULL = 0xffffffffu;

struct PlaneRows {
    float phi[NROW], wx[NROW], wy[NROW], wz[NROW];
};

__device__ __forceinline__ void load_rows(PlaneRows &v, const float *__restrict__ phi, const float *__restrict__ w,
                                          size_t N, int plane_off, const int (&roff)[NROW], int xg)
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

template <bool WALL>
__global__ void __launch_bounds__(WPB * 32) ac_div_kernel(Grid G, Phys P, const float *__restrict__ phi,
                                                          const float *__restrict__ w, float *__restrict__ phi_out,
                                                          int ncols, int zlen, int tasks)
{
    const int lane = threadIdx.x & 31;
    const int nx = G.nx, ny = G.ny, nz = G.nz, nxy = G.nxy;
    const int ncx = (nx + XO - 1) / XO;
    const size_t N = (size_t)G.N;
    const float D = P.mob;
    const int nwarps = gridDim.x * WPB;

    for (int task = blockIdx.x * WPB + (threadIdx.x >> 5); task < tasks; task += nwarps) {
        const int col = task % ncols;
        const int z0 = (task / ncols) * zlen;
        const int zend = min(nz, z0 + zlen);
        const int x0 = (col % ncx) * XO, y0 = (col / ncx) * RY;
        const int x = x0 - 1 + lane;                       // this lane's column (before wrapping)
        const int xg = wrapc(x, nx);
        const bool xout = lane >= 1 && lane <= XO && x < nx;
        int roff[NROW];
#pragma unroll
        for (int r = 0; r < NROW; ++r) roff[r] = wrapc(y0 - 1 + r, ny) * nx;

        float acc1[RY], acc2[RY], cprev[RY];
#pragma unroll
        for (int r = 0; r < RY; ++r) acc1[r] = acc2[r] = cprev[r] = 0.0f;
        PlaneRows cur, nxt;
        load_rows(cur, phi, w, N, zmap<WALL>(z0 - 1, nz) * nxy, roff, xg);
        for (int p = z0 - 1; p <= zend; ++p) {
            if (p + 1 <= zend) load_rows(nxt, phi, w, N, zmap<WALL>(p + 1, nz) * nxy, roff, xg);
            const float sg = zsign<WALL>(p, nz);
            const bool store = p - 1 >= z0;
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                // y-sums of this column (phi in difference form against the row's own value)
                const float c = cur.phi[r + 1];
                const float yd = W1 * ((cur.phi[r] - c) + (cur.phi[r + 2] - c));
                const float yx = fmaf(W0, cur.wx[r + 1], W1 * (cur.wx[r] + cur.wx[r + 2]));
                const float dy = cur.wy[r + 2] - cur.wy[r];
                const float yz = fmaf(W0, cur.wz[r + 1], W1 * (cur.wz[r] + cur.wz[r + 2]));
                // the x-neighbours' sums
                const float cl = __shfl_up_sync(FULL, c, 1), cr = __shfl_down_sync(FULL, c, 1);
                const float ydl = __shfl_up_sync(FULL, yd, 1), ydr = __shfl_down_sync(FULL, yd, 1);
                const float yxl = __shfl_up_sync(FULL, yx, 1), yxr = __shfl_down_sync(FULL, yx, 1);
                const float dyl = __shfl_up_sync(FULL, dy, 1), dyr = __shfl_down_sync(FULL, dy, 1);
                const float yzl = __shfl_up_sync(FULL, yz, 1), yzr = __shfl_down_sync(FULL, yz, 1);
                // plane partials: Sd (difference form), Q, T
                const float sd = fmaf(W0, yd, W1 * ((ydl + ydr) + ((cl - c) + (cr - c))));
                const float q = (yxr - yxl) + fmaf(W0, dy, W1 * (dyl + dyr));
                const float t = sg * fmaf(W0, yz, W1 * (yzl + yzr));
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

struct LaunchAC {
    int blocks_per_sm = 0;
    int sms = 0;
};

template <bool WALL>
cudaError_t prepare_ac(LaunchAC &L)
{
    int dev = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&L.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L.blocks_per_sm, ac_div_kernel<WALL>, WPB * 32, 0);
}

}  // namespace

cudaError_t launch_ac_div(const Grid &G, const Phys &P, const float *phi_in, const float *w, float *phi_out,
                          int zchunks, cudaStream_t s)
{
    static LaunchAC lw[2];
    LaunchAC &L = lw[G.wall ? 1 : 0];
    if (L.sms == 0) {
        cudaError_t e = G.wall ? prepare_ac<true>(L) : prepare_ac<false>(L);
        if (e != cudaSuccess) return e;
        if (L.blocks_per_sm < 1) return cudaErrorInvalidConfiguration;
    }
    const int warp_slots = L.sms * L.blocks_per_sm * WPB;
    const int ncols = ((G.nx + XO - 1) / XO) * ((G.ny + RY - 1) / RY);
    // default: about one task per resident warp, chunks of at least 16 planes (2 halo planes each)
    int m = zchunks;
    if (m <= 0) {
        m = warp_slots / ncols;
        if (m > G.nz / 16) m = G.nz / 16;
        if (m < 1) m = 1;
    }
    if (m > G.nz) m = G.nz;
    const int zlen = (G.nz + m - 1) / m;
    m = (G.nz + zlen - 1) / zlen;
    const int tasks = ncols * m;
    const int warps = tasks < warp_slots ? tasks : warp_slots;
    const int ctas = (warps + WPB - 1) / WPB;
    if (G.wall)
        ac_div_kernel<true><<<ctas, WPB * 32, 0, s>>>(G, P, phi_in, w, phi_out, ncols, zlen, tasks);
    else
        ac_div_kernel<false><<<ctas, WPB * 32, 0, s>>>(G, P, phi_in, w, phi_out, ncols, zlen, tasks);
    return cudaGetLastError();
}

cudaError_t launch_step_split(const Grid &G, const Phys &P, const StepArgs &a, int zchunks, cudaStream_t s)
{
    cudaError_t e = launch_ac_div(G, P, a.phi_in, a.flux, a.phi_out, zchunks, s);
    if (e != cudaSuccess) return e;
    if (a.storage != 0)
        return launch_lbm16(G, P, a.storage, a.g_in, a.p_in, a.phi_out, a.u_in, a.g_out, a.p_out, a.u_out, a.flux, s);
    return launch_lbm(G, P, 0, a.g_in, nullptr, a.phi_out, a.u_in, a.g_out, nullptr, a.u_out, a.flux, s);
}

}  // namespace tslb

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

// The y-sums of one column (c = phi at the row, Yd in difference form, Yx, Dy, Yz) from rows
// y - 1, y, y + 1 of (phi, W_x, W_y, W_z).  Rounded operations throughout, so that the scalar and
// the vector forms below give the same bits whatever the compiler contracts.
struct AcY {
    float c, yd, yx, dy, yz;
};

__device__ __forceinline__ AcY ac_ysum(float p0, float p1, float p2, float x0, float x1, float x2, float y0,
                                       float y2, float z0, float z1, float z2)
{
    AcY s;
    s.c = p1;
    s.yd = __fmul_rn(AC_W1, __fadd_rn(__fsub_rn(p0, p1), __fsub_rn(p2, p1)));
    s.yx = __fmaf_rn(AC_W0, x1, __fmul_rn(AC_W1, __fadd_rn(x0, x2)));
    s.dy = __fsub_rn(y2, y0);
    s.yz = __fmaf_rn(AC_W0, z1, __fmul_rn(AC_W1, __fadd_rn(z0, z2)));
    return s;
}

// One node, plane p: the plane partials Sd, Q, T from the y-sums of the node's column (m) and of
// its x-neighbours (l, r), their contributions to the targets p - 1, p, p + 1 (the z differences
// of c taken between neighbouring planes, cprev = c of plane p - 1), and phi^{n+1} of plane
// p - 1, complete now, with its own c added last.  sg = -1 on a wall's ghost plane.
__device__ __forceinline__ float ac_node(const AcY &l, const AcY &m, const AcY &r, float sg, float D, float &acc1,
                                         float &acc2, float &cprev)
{
    const float c = m.c;
    const float sd = __fmaf_rn(AC_W0, m.yd, __fmul_rn(AC_W1, __fadd_rn(__fadd_rn(l.yd, r.yd),
                                                                       __fadd_rn(__fsub_rn(l.c, c), __fsub_rn(r.c, c)))));
    const float q = __fadd_rn(__fsub_rn(r.yx, l.yx), __fmaf_rn(AC_W0, m.dy, __fmul_rn(AC_W1, __fadd_rn(l.dy, r.dy))));
    const float t = __fmul_rn(sg, __fmaf_rn(AC_W0, m.yz, __fmul_rn(AC_W1, __fadd_rn(l.yz, r.yz))));
    const float cp = cprev;
    const float qs = __fmul_rn(q, -1.0f / 12.0f);
    const float lo = __fmaf_rn(D, __fadd_rn(sd, __fsub_rn(c, cp)), __fmaf_rn(-0.5f, t, qs));
    const float mid = __fmaf_rn(D, __fmaf_rn(4.0f, sd, __fsub_rn(cp, c)), __fmul_rn(q, -1.0f / 3.0f));
    const float hi = __fmaf_rn(D, sd, __fmaf_rn(0.5f, t, qs));
    const float done = __fadd_rn(cp, __fadd_rn(acc1, lo));
    acc1 = __fadd_rn(acc2, mid);
    acc2 = hi;
    cprev = c;
    return done;
}

__device__ __forceinline__ AcY ac_shfl(const AcY &s, int src)
{
    return AcY{__shfl_sync(AC_FULL, s.c, src), __shfl_sync(AC_FULL, s.yd, src), __shfl_sync(AC_FULL, s.yx, src),
               __shfl_sync(AC_FULL, s.dy, src), __shfl_sync(AC_FULL, s.yz, src)};
}

__device__ __forceinline__ AcY ac_shfl_up(const AcY &s)
{
    return AcY{__shfl_up_sync(AC_FULL, s.c, 1), __shfl_up_sync(AC_FULL, s.yd, 1), __shfl_up_sync(AC_FULL, s.yx, 1),
               __shfl_up_sync(AC_FULL, s.dy, 1), __shfl_up_sync(AC_FULL, s.yz, 1)};
}

__device__ __forceinline__ AcY ac_shfl_down(const AcY &s)
{
    return AcY{__shfl_down_sync(AC_FULL, s.c, 1), __shfl_down_sync(AC_FULL, s.yd, 1),
               __shfl_down_sync(AC_FULL, s.yx, 1), __shfl_down_sync(AC_FULL, s.dy, 1),
               __shfl_down_sync(AC_FULL, s.yz, 1)};
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
    const int x0 = (col % ncx) * AC_XO, y0 = (col / ncx) * RY;
    const int x = x0 - 1 + lane;                           // this lane's column (before wrapping)
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
            const AcY m = ac_ysum(cur.phi[r], cur.phi[r + 1], cur.phi[r + 2], cur.wx[r], cur.wx[r + 1], cur.wx[r + 2],
                                  cur.wy[r], cur.wy[r + 2], cur.wz[r], cur.wz[r + 1], cur.wz[r + 2]);
            const AcY l = ac_shfl_up(m), rr = ac_shfl_down(m);   // the x-neighbours' sums
            const float done = ac_node(l, m, rr, sg, D, acc1[r], acc2[r], cprev[r]);
            if (store && xout && y0 + r < ny) phi_out[(size_t)(p - 1) * nxy + (y0 + r) * nx + x] = done;
        }
        cur = nxt;
    }
}

// The vector form, for boxes whose x extent is a multiple of AC_XV = 128 (every benchmark box):
// a warp owns 128 consecutive columns, 4 per lane, loaded and stored as float4.  A lane's two
// inner columns find both x-neighbours in its own registers, the outer two take one shuffle
// each, and no lane is spent on a halo column: when the warp spans the whole periodic row
// (XWRAP, nx = 128) the halo is the shuffle's wrap-around, otherwise lane 0 loads column x0 - 1
// and lane 31 column x0 + 128.  Every node takes ac_ysum and ac_node in the same order as the
// scalar form, so the two forms give the same bits.  phi^{n+1} is stored with the L2 evict-last
// hint: the lattice Boltzmann kernel reads it next, and the Allen–Cahn kernel of the next step.
constexpr int AC_XV = 128;

template <int NROW>
struct PlaneRows4 {
    float4 phi[NROW], wx[NROW], wy[NROW], wz[NROW];
};

template <int NROW>
__device__ __forceinline__ void load_rows4(PlaneRows4<NROW> &v, const float *__restrict__ phi,
                                           const float *__restrict__ w, size_t N, int plane_off,
                                           const int (&roff)[NROW], int xl)
{
#pragma unroll
    for (int r = 0; r < NROW; ++r) {
        const int at = plane_off + roff[r] + xl;
        v.phi[r] = __ldg(reinterpret_cast<const float4 *>(phi + at));
        v.wx[r] = __ldg(reinterpret_cast<const float4 *>(w + at));
        v.wy[r] = __ldg(reinterpret_cast<const float4 *>(w + N + at));
        v.wz[r] = __ldg(reinterpret_cast<const float4 *>(w + 2 * N + at));
    }
}

template <int K>
__device__ __forceinline__ float ac_f4(const float4 &v)
{
    return K == 0 ? v.x : (K == 1 ? v.y : (K == 2 ? v.z : v.w));
}

template <int K, int NROW>
__device__ __forceinline__ AcY ac_ysum4(const PlaneRows4<NROW> &v, int r)
{
    return ac_ysum(ac_f4<K>(v.phi[r]), ac_f4<K>(v.phi[r + 1]), ac_f4<K>(v.phi[r + 2]), ac_f4<K>(v.wx[r]),
                   ac_f4<K>(v.wx[r + 1]), ac_f4<K>(v.wx[r + 2]), ac_f4<K>(v.wy[r]), ac_f4<K>(v.wy[r + 2]),
                   ac_f4<K>(v.wz[r]), ac_f4<K>(v.wz[r + 1]), ac_f4<K>(v.wz[r + 2]));
}

// One task of the vector form: column tile col (128 x RY output columns; tiles ordered x
// fastest) over the planes [z0, zend).  Requires nx % 128 == 0 and 16-byte aligned arrays.
// PREF loads plane p + 1 while plane p is computed (twice the registers for the rows);
// otherwise the loads of plane p + 1 follow its computation and other warps hide their latency.
template <bool WALL, int RY, bool XWRAP, bool PREF>
__device__ __forceinline__ void ac_div_task4(const Grid &G, const Phys &P, const float *__restrict__ phi,
                                             const float *__restrict__ w, float *__restrict__ phi_out, int col,
                                             int z0, int zend)
{
    constexpr int NROW = RY + 2;
    const int lane = threadIdx.x & 31;
    const int nx = G.nx, ny = G.ny, nz = G.nz, nxy = G.nxy;
    const int ncx = nx / AC_XV;
    const size_t N = (size_t)G.N;
    const float D = P.mob;
    const int x0 = (col % ncx) * AC_XV, y0 = (col / ncx) * RY;
    const int xl = x0 + 4 * lane;                          // this lane's first column
    const int hx = ac_wrapc(lane == 0 ? x0 - 1 : x0 + AC_XV, nx);
    int roff[NROW];
#pragma unroll
    for (int r = 0; r < NROW; ++r) roff[r] = ac_wrapc(y0 - 1 + r, ny) * nx;

    float acc1[RY][4], acc2[RY][4], cprev[RY][4];
#pragma unroll
    for (int r = 0; r < RY; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc1[r][k] = acc2[r][k] = cprev[r][k] = 0.0f;
    PlaneRows4<NROW> cur, nxt;
    PlaneRows<NROW> hcur, hnxt;
    load_rows4(cur, phi, w, N, ac_zmap<WALL>(z0 - 1, nz) * nxy, roff, xl);
    if (!XWRAP) load_rows(hcur, phi, w, N, ac_zmap<WALL>(z0 - 1, nz) * nxy, roff, hx);
    for (int p = z0 - 1; p <= zend; ++p) {
        if (PREF && p + 1 <= zend) {
            load_rows4(nxt, phi, w, N, ac_zmap<WALL>(p + 1, nz) * nxy, roff, xl);
            if (!XWRAP) load_rows(hnxt, phi, w, N, ac_zmap<WALL>(p + 1, nz) * nxy, roff, hx);
        }
        const float sg = ac_zsign<WALL>(p, nz);
        const bool store = p - 1 >= z0;
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            const AcY m0 = ac_ysum4<0>(cur, r), m1 = ac_ysum4<1>(cur, r), m2 = ac_ysum4<2>(cur, r),
                      m3 = ac_ysum4<3>(cur, r);
            AcY l, rr;
            if (XWRAP) {
                l = ac_shfl(m3, (lane + 31) & 31);
                rr = ac_shfl(m0, (lane + 1) & 31);
            } else {
                const AcY h = ac_ysum(hcur.phi[r], hcur.phi[r + 1], hcur.phi[r + 2], hcur.wx[r], hcur.wx[r + 1],
                                      hcur.wx[r + 2], hcur.wy[r], hcur.wy[r + 2], hcur.wz[r], hcur.wz[r + 1],
                                      hcur.wz[r + 2]);
                l = ac_shfl_up(m3);
                rr = ac_shfl_down(m0);
                if (lane == 0) l = h;
                if (lane == 31) rr = h;
            }
            float4 o;
            o.x = ac_node(l, m0, m1, sg, D, acc1[r][0], acc2[r][0], cprev[r][0]);
            o.y = ac_node(m0, m1, m2, sg, D, acc1[r][1], acc2[r][1], cprev[r][1]);
            o.z = ac_node(m1, m2, m3, sg, D, acc1[r][2], acc2[r][2], cprev[r][2]);
            o.w = ac_node(m2, m3, rr, sg, D, acc1[r][3], acc2[r][3], cprev[r][3]);
            if (store && y0 + r < ny)
                st_keep4(phi_out + (size_t)(p - 1) * nxy + (y0 + r) * nx + xl, o, l2_keep_policy());
        }
        if (PREF) {
            cur = nxt;
            if (!XWRAP) hcur = hnxt;
        } else if (p + 1 <= zend) {
            load_rows4(cur, phi, w, N, ac_zmap<WALL>(p + 1, nz) * nxy, roff, xl);
            if (!XWRAP) load_rows(hcur, phi, w, N, ac_zmap<WALL>(p + 1, nz) * nxy, roff, hx);
        }
    }
}

}  // namespace tslb

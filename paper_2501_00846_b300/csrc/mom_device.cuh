// Moment-only ("thread-safe") storage of the lattice Boltzmann state.
//
// The paper's collision rebuilds each post-collision population from macroscopic fields alone
// (Section "Thread-safe lattice Boltzmann", Eq. LBexp with the equilibrium Eq. eqts, the
// regularised non-equilibrium Eq. noneqts and the forcing): the populations leaving a node are a
// fixed polynomial in c_i of that node's
//     p*,  u,  a = F / rho,  B = k2 A,   k2 = (1 - omega) / (2 cs^4) = 4.5 (1 - omega),
// 13 numbers (A symmetric).  Storing those instead of the 27 populations, and letting the node
// that pulls g_i(x - c_i) rebuild it from the moments of x - c_i, moves 52 bytes per node and
// step each way instead of 108.
//
// Per unit weight, with cu = c.u, ca = c.a, cBc = c^T B c (the same even/odd contraction as
// collide_node):
//     g_{+-c} / w = E +- O,
//     E = K0 + 4.5 cu (cu + ca) + cBc,              K0 = p* - 1.5 u^2 - 1.5 u.a - tr(B) / 3
//     O = cu (K1 + 4.5 cu^2 + 3 cBc) + c.v,         K1 = 3 - 4.5 u^2 - tr(B),   v = 1.5 a - 2 B u.
// The moments of these populations give the set back (used to import a population state):
//     sum g = p*,   sum g c = u + a / 2,   sum g c c = p* I / 3 + (2/9) T,
//     T = B + 4.5 u u + 4.5 sym(u a),   sym(u a)_{ab} = (u_a a_b + u_b a_a) / 2
// (fourth-order isotropy of D3Q27: sum w c_a c_b c_c c_d = (d_ab d_cd + d_ac d_bd + d_ad d_bc) / 9).
//
// Array layout of a moment state: p*[node] in FP32, then the 9 deviation moments a (3) and
// B (xx yy zz xy xz yz; 6).  FP32 storage: arrays d[q * N + node] (so m[q * N + node] for q = 0 p*,
// 1..3 a, 4..9 B).  BF16 / FP16 storage (FP16 holding 2^12 times the value; a and B vanish at
// equilibrium, so 16 bits round only the deviation, as for 16-bit populations): the 9 values of a
// node packed in five 32-bit words, d16[10 node + q] with the tenth half zero, so a node's
// moments move in five aligned 4-byte accesses.  u lives in the context's velocity arrays.
#pragma once

#include <string.h>

#include "tslb_device.cuh"

namespace tslb {

constexpr int kMomArrays = 10;

struct Mom {
    float ps, ux, uy, uz, ax, ay, az, bxx, byy, bzz, bxy, bxz, byz;
};

// Node constants of the population polynomial.
struct MomPoly {
    float K0, K1, vx, vy, vz, b2xy, b2xz, b2yz;
};

// the deviation part of a moment state m (after the N FP32 values of p*)
template <class S>
__device__ __forceinline__ const typename S::T *mom_dev(const float *m, size_t N)
{
    return reinterpret_cast<const typename S::T *>(m + N);
}
template <class S>
__device__ __forceinline__ typename S::T *mom_dev(float *m, size_t N)
{
    return reinterpret_cast<typename S::T *>(m + N);
}

constexpr int kMomWords = 5;   // 32-bit words of a node's packed 16-bit deviation moments

// a 16-bit storage value from / to its bits
template <class S>
__device__ __forceinline__ float mom_h2f(unsigned short b)
{
    typename S::T t;
    memcpy(&t, &b, 2);
    return S::to_f(t);
}
template <class S>
__device__ __forceinline__ uint32_t mom_f2h(float v)
{
    const typename S::T t = S::from_f(v);
    unsigned short b;
    memcpy(&b, &t, 2);
    return b;
}

// the 9 deviation moments of a node from its packed words (16-bit storage)
template <class S>
__device__ __forceinline__ void mom_unpack(const uint32_t (&w)[kMomWords], Mom &r)
{
    r.ax = mom_h2f<S>(w[0] & 0xFFFF), r.ay = mom_h2f<S>(w[0] >> 16);
    r.az = mom_h2f<S>(w[1] & 0xFFFF), r.bxx = mom_h2f<S>(w[1] >> 16);
    r.byy = mom_h2f<S>(w[2] & 0xFFFF), r.bzz = mom_h2f<S>(w[2] >> 16);
    r.bxy = mom_h2f<S>(w[3] & 0xFFFF), r.bxz = mom_h2f<S>(w[3] >> 16);
    r.byz = mom_h2f<S>(w[4] & 0xFFFF);
}

template <class S = StoreF32>
__device__ __forceinline__ Mom mom_load(const float *__restrict__ m, const float *__restrict__ u, size_t N, int k)
{
    Mom r;
    r.ps = __ldg(m + k);
    if constexpr (sizeof(typename S::T) == 4) {
        const float *d = m + N;
        r.ax = __ldg(d + k);
        r.ay = __ldg(d + N + k);
        r.az = __ldg(d + 2 * N + k);
        r.bxx = __ldg(d + 3 * N + k);
        r.byy = __ldg(d + 4 * N + k);
        r.bzz = __ldg(d + 5 * N + k);
        r.bxy = __ldg(d + 6 * N + k);
        r.bxz = __ldg(d + 7 * N + k);
        r.byz = __ldg(d + 8 * N + k);
    } else {
        const uint32_t *wp = reinterpret_cast<const uint32_t *>(m + N) + (size_t)kMomWords * k;
        uint32_t w[kMomWords];
#pragma unroll
        for (int j = 0; j < kMomWords; ++j) w[j] = __ldg(wp + j);
        mom_unpack<S>(w, r);
    }
    r.ux = __ldg(u + k);
    r.uy = __ldg(u + N + k);
    r.uz = __ldg(u + 2 * N + k);
    return r;
}

// The moment set left by a collision: B = 4.5 (1 - omega) A.
__device__ __forceinline__ Mom mom_from_collided(const Collided &c)
{
    const float k2 = 4.5f * (1.0f - c.omega);
    Mom m;
    m.ps = c.ps;
    m.ux = c.ux, m.uy = c.uy, m.uz = c.uz;
    m.ax = c.ax, m.ay = c.ay, m.az = c.az;
    m.bxx = k2 * c.Axx, m.byy = k2 * c.Ayy, m.bzz = k2 * c.Azz;
    m.bxy = k2 * c.Axy, m.bxz = k2 * c.Axz, m.byz = k2 * c.Ayz;
    return m;
}

// p* and the deviation moments of a node (not u)
template <class S = StoreF32>
__device__ __forceinline__ void mom_store_dev(const Mom &r, float *__restrict__ m, size_t N, int k)
{
    m[k] = r.ps;
    if constexpr (sizeof(typename S::T) == 4) {
        float *d = m + N;
        d[k] = r.ax;
        d[N + k] = r.ay;
        d[2 * N + k] = r.az;
        d[3 * N + k] = r.bxx;
        d[4 * N + k] = r.byy;
        d[5 * N + k] = r.bzz;
        d[6 * N + k] = r.bxy;
        d[7 * N + k] = r.bxz;
        d[8 * N + k] = r.byz;
    } else {
        uint32_t *wp = reinterpret_cast<uint32_t *>(m + N) + (size_t)kMomWords * k;
        wp[0] = mom_f2h<S>(r.ax) | (mom_f2h<S>(r.ay) << 16);
        wp[1] = mom_f2h<S>(r.az) | (mom_f2h<S>(r.bxx) << 16);
        wp[2] = mom_f2h<S>(r.byy) | (mom_f2h<S>(r.bzz) << 16);
        wp[3] = mom_f2h<S>(r.bxy) | (mom_f2h<S>(r.bxz) << 16);
        wp[4] = mom_f2h<S>(r.byz);
    }
}

template <class S = StoreF32>
__device__ __forceinline__ void mom_store(const Mom &r, float *__restrict__ m, float *__restrict__ u, size_t N, int k)
{
    mom_store_dev<S>(r, m, N, k);
    u[k] = r.ux;
    u[N + k] = r.uy;
    u[2 * N + k] = r.uz;
}

// The polynomial is evaluated with explicit round-to-nearest intrinsics (no contraction or
// reordering left to the compiler), so every kernel and every staging variant that evaluates a
// population gets the same bits, and a mirrored moment set gives exactly the negated odd terms.
__device__ __forceinline__ MomPoly mom_poly(const Mom &m)
{
    MomPoly q;
    const float u2 = __fmaf_rn(m.uz, m.uz, __fmaf_rn(m.uy, m.uy, __fmul_rn(m.ux, m.ux)));
    const float ua = __fmaf_rn(m.uz, m.az, __fmaf_rn(m.uy, m.ay, __fmul_rn(m.ux, m.ax)));
    const float trb = __fadd_rn(__fadd_rn(m.bxx, m.byy), m.bzz);
    q.K0 = __fmaf_rn(-1.0f / 3.0f, trb, __fmaf_rn(-1.5f, ua, __fmaf_rn(-1.5f, u2, m.ps)));
    q.K1 = __fmaf_rn(-4.5f, u2, __fsub_rn(3.0f, trb));
    const float bux = __fmaf_rn(m.bxz, m.uz, __fmaf_rn(m.bxy, m.uy, __fmul_rn(m.bxx, m.ux)));
    const float buy = __fmaf_rn(m.byz, m.uz, __fmaf_rn(m.byy, m.uy, __fmul_rn(m.bxy, m.ux)));
    const float buz = __fmaf_rn(m.bzz, m.uz, __fmaf_rn(m.byz, m.uy, __fmul_rn(m.bxz, m.ux)));
    q.vx = __fmaf_rn(-2.0f, bux, __fmul_rn(1.5f, m.ax));
    q.vy = __fmaf_rn(-2.0f, buy, __fmul_rn(1.5f, m.ay));
    q.vz = __fmaf_rn(-2.0f, buz, __fmul_rn(1.5f, m.az));
    q.b2xy = __fmul_rn(2.0f, m.bxy);
    q.b2xz = __fmul_rn(2.0f, m.bxz);
    q.b2yz = __fmul_rn(2.0f, m.byz);
    return q;
}

// s + c v for a lattice component c in {-1, 0, 1} (c a compile-time constant after unrolling)
__device__ __forceinline__ float mom_acc(float s, int c, float v)
{
    return c > 0 ? __fadd_rn(s, v) : c < 0 ? __fsub_rn(s, v) : s;
}

// c_x a + c_y b + c_z c for lattice components in {-1, 0, 1} (compile-time constants after
// unrolling), summed in the order x, y, z; the first nonzero term is taken as it is (a negation is
// exact), so no addition to zero is executed.
__device__ __forceinline__ float mom_dot(int X, int Y, int Z, float a, float b, float c)
{
    if (X) return mom_acc(mom_acc(X > 0 ? a : -a, Y, b), Z, c);
    if (Y) return mom_acc(Y > 0 ? b : -b, Z, c);
    return Z > 0 ? c : Z < 0 ? -c : 0.0f;
}

// g_i / w_i and g_{26-i} / w_i of the pair i < 13 (i a compile-time constant after unrolling).
__device__ __forceinline__ void mom_pair(int i, const Mom &m, const MomPoly &q, float &gp, float &gm)
{
    const int X = cx(i), Y = cy(i), Z = cz(i);
    const float cu = mom_dot(X, Y, Z, m.ux, m.uy, m.uz);
    const float ca = mom_dot(X, Y, Z, m.ax, m.ay, m.az);
    const float cv = mom_dot(X, Y, Z, q.vx, q.vy, q.vz);
    float cbc = mom_dot(X * X, Y * Y, Z * Z, m.bxx, m.byy, m.bzz);
    cbc = mom_acc(mom_acc(mom_acc(cbc, X * Y, q.b2xy), X * Z, q.b2xz), Y * Z, q.b2yz);
    const float hcu = __fmul_rn(4.5f, cu);
    const float E = __fadd_rn(__fmaf_rn(hcu, __fadd_rn(cu, ca), q.K0), cbc);
    const float O = __fmaf_rn(cu, __fmaf_rn(3.0f, cbc, __fmaf_rn(hcu, cu, q.K1)), cv);
    gp = __fadd_rn(E, O);
    gm = __fsub_rn(E, O);
}

// g_i / w_i of one direction (i a compile-time constant after unrolling)
__device__ __forceinline__ float mom_one(int i, const Mom &m, const MomPoly &q)
{
    if (i == 13) return q.K0;
    float gp, gm;
    mom_pair(i < 13 ? i : 26 - i, m, q, gp, gm);
    return i < 13 ? gp : gm;
}

// Mirror image x -> -x of a moment set (the components odd in x change sign): the population
// of direction (cx, cy, cz) of the mirrored set is that of (-cx, cy, cz) of the original.
__device__ __forceinline__ Mom mom_mirror_x(const Mom &m)
{
    Mom r = m;
    r.ux = -m.ux;
    r.ax = -m.ax;
    r.bxy = -m.bxy;
    r.bxz = -m.bxz;
    return r;
}

// Raw moments of streamed populations given per unit weight, f_i = w_i gh_i (the weights folded
// into the sums instead of multiplying each population).
__device__ __forceinline__ RawMoments raw_moments_hat(const float (&gh)[27])
{
    RawMoments r;
    float ps = wgt(13) * gh[13];
    float jx = 0.f, jy = 0.f, jz = 0.f;
    float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
    for (int i = 0; i < 13; ++i) {
        const float w = wgt(i);
        const float s = gh[i] + gh[26 - i];
        const float d = gh[i] - gh[26 - i];
        ps = fmaf(w, s, ps);
        if (cx(i)) { jx = fmaf(cx(i) * w, d, jx); pxx = fmaf(w, s, pxx); }
        if (cy(i)) { jy = fmaf(cy(i) * w, d, jy); pyy = fmaf(w, s, pyy); }
        if (cz(i)) { jz = fmaf(cz(i) * w, d, jz); pzz = fmaf(w, s, pzz); }
        if (cx(i) * cy(i)) pxy = fmaf((cx(i) * cy(i)) * w, s, pxy);
        if (cx(i) * cz(i)) pxz = fmaf((cx(i) * cz(i)) * w, s, pxz);
        if (cy(i) * cz(i)) pyz = fmaf((cy(i) * cz(i)) * w, s, pyz);
    }
    r.ps = ps;
    r.jx = jx, r.jy = jy, r.jz = jz;
    r.pxx = pxx, r.pyy = pyy, r.pzz = pzz, r.pxy = pxy, r.pxz = pxz, r.pyz = pyz;
    return r;
}

// The lattice Boltzmann update of one node once the raw moments of its streamed populations and
// the gradient and Laplacian of phi^{n+1} are known: the collision, the new moment set, and the
// Allen–Cahn flux of the new state (as lbm_node).
template <class S = StoreF32>
__device__ __forceinline__ void mom_finish(const RawMoments &r, float phi, float gx, float gy, float gz, float lap,
                                           float ubx, float uby, float ubz, const Phys &P, float *__restrict__ m_out,
                                           float *__restrict__ u_out, float *__restrict__ w_out, size_t N, int k)
{
    const Collided c = collide_from_moments(r, phi, gx, gy, gz, lap, ubx, uby, ubz, P);
    mom_store<S>(mom_from_collided(c), m_out, u_out, N, k);
    if (w_out) {
        float wx, wy, wz;
        ac_flux(phi, gx, gy, gz, c.ux, c.uy, c.uz, P, wx, wy, wz);
        const unsigned long long pol = l2_keep_policy();
        st_keep(w_out + k, wx, pol);
        st_keep(w_out + N + k, wy, pol);
        st_keep(w_out + 2 * N + k, wz, pol);
    }
}

}  // namespace tslb

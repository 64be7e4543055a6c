/*
 * FP64 CPU oracle of the coupled thread-safe lattice Boltzmann (TSLB) + conservative
 * Allen–Cahn step of arXiv 2501.00846 ("Thread-safe multiphase lattice Boltzmann model for
 * droplet and bubble dynamics at high density and viscosity contrasts").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, literal reference that the CUDA path is
 * checked against.  Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header, table or constant with the CUDA library: every lattice
 * table below is generated here from the definition of the D3Q27 velocity set.
 *
 * Style: every sum over populations is an explicit loop over the 27 velocities; every Hermite
 * contraction is an explicit loop over tensor indices (alpha, beta, gamma).  Nothing is fused
 * or reordered beyond what the paper's formulas state.
 *
 * Notation (paper Section "Method"):
 *   c_i, w_i   D3Q27 velocities and weights, cs^2 = 1/3, dx = dt = 1
 *   f_i        populations after streaming (pre-collision)
 *   p*         non-dimensional pressure, p* = sum_i f_i                  (Eq. moments0)
 *   u          velocity, u = sum_i f_i c_i + a/2                          (Eq. moments1, reading R1)
 *   A          a^2_neq = sum_i H2_i (f_i - fbar^eq_i)                     (Eq. hermite_neq2)
 *   phi        phase field, phi = 1 liquid (rho_L), phi = 0 gas (rho_G)
 *
 * State convention.  The stored state after step n is (g^n, phi^n, ubar^n): g^n_i(x) is the
 * post-collision population at its origin node x, phi^n the phase field used by that
 * collision and ubar^n the velocity it produced.  Streaming is written as a pull,
 * f_i(x) = g_i(x - c_i), which is the left-hand side of Eq. lbe read from the receiving node.
 * One call of oracle_step performs, in this order:
 *   1. the interface-tracking update of the previous iteration (Section "Implementation of the
 *      hybrid LB-finite difference implementation", last item): phi^{n+1} from phi^n, ubar^n;
 *   2. streaming (pull, halfway bounce-back at z walls);
 *   3. moments and forces (first item of the same list): p*, F^s, F^p, F^nu, body force;
 *   4. velocity (Eq. moments1);
 *   5. pre-regularisation (Eq. hermite_neq2);
 *   6. regularised collision (Eqs. LBexp, eqts, noneqts, guoforce).
 * This is the paper's cycle with its last item moved to the front of the next iteration.
 *
 * Readings of garbled or unstated points (each one is applied identically on the GPU side):
 *   R1  S_i uses the acceleration a = F/rho; u = sum f c + a/2.
 *   R2  Laplacian  L[psi] = (2/cs^2) sum_{i!=0} w_i (psi(x+c_i) - psi(x)).
 *   R3  collision  g = fbar^eq + (1-omega) f^neq + S  with fbar^eq = f^eq - S/2.
 *   R4  advection in flux form div(ubar phi) (advect = 0, the default); advect = 1 takes the
 *       literal form ubar . G[phi] of the paper's update, which does not conserve sum phi.
 *   R5  n = grad(phi) / max(|grad(phi)|, 1e-12).
 *   R6  F^nu uses f^eq(p*, ubar^n) (lagged velocity); contraction [..]_{ab} d_b rho.
 *   R7  f^neq_i = w_i [H2_i:A/(2cs^4) + H3_i:a3/(6cs^6)],  a3 = sym(u (x) A).
 *   R10 mu(phi) = mu_G + phi (mu_L - mu_G) (dynamic), nu = mu/rho, tau = nu/cs^2 + 1/2.
 *   R11 body force (rho - rho_ref) g + G_body.
 *   R13 z walls: halfway bounce-back for populations; scalar fields mirrored about the wall;
 *       vector fields mirrored with their z component negated.
 *   R15 the sharpening weight phi (1 - phi) is taken as max(phi (1 - phi), 0): the paper's phi
 *       lives in [0, 1]; outside it the weight would turn the sharpening flux around exactly
 *       where phi has an extremum and the normal is undefined.  literal_weight = 1 takes the
 *       printed phi (1 - phi) everywhere, to measure how far the reading moves the results.
 *
 * Not from the paper: storage16 = 1 / 2 emulates the library's 16-bit population storage (its
 * precision form, BF16 / FP16 deviations from equilibrium; store16 below), and storage16 = 3 / 4
 * its 16-bit moment storage (BF16 / FP16 deviation moments a and B; store_mom16 below), so that
 * the tests know each case's 16-bit effect from the oracle alone.  storage16 = 0 (the default) is
 * the method.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 27
#define CS2 (1.0 / 3.0)

typedef struct {
    int nx, ny, nz;
    int wall_z;            /* 0: periodic in z; 1: no-slip walls at z = -1/2 and z = nz - 1/2 */
    double rho_l, rho_g;   /* liquid / gas density */
    double mu_l, mu_g;     /* liquid / gas dynamic viscosity */
    double sigma;          /* surface tension */
    double width;          /* interface width delta (W) */
    double mobility;       /* Allen–Cahn diffusivity D */
    double gravity[3];     /* gravitational acceleration vector */
    double rho_ref;        /* reference density of the buoyancy force */
    double body[3];        /* uniform body-force density */
    int advect;            /* 0: flux form div(ubar phi); 1: literal form ubar . grad(phi) */
    int literal_weight;    /* 0: sharpening weight max(phi (1 - phi), 0) (R15); 1: phi (1 - phi) as printed */
    int storage16;         /* 0: FP64 populations; 1 / 2: the library's BF16 / FP16 deviation storage (store16);
                              3 / 4: its BF16 / FP16 deviation moments (store_mom16) */
} oracle_params;

/* ------------------------------------------------------------------------------------------ */
/* D3Q27 lattice (generated from its definition: c in {-1,0,1}^3, weights by |c|^2).          */
/* Index i = 9 (cz+1) + 3 (cy+1) + (cx+1); the opposite of i is 26 - i; the rest vector is 13. */
/* ------------------------------------------------------------------------------------------ */
static int C[Q][3];
static double Wt[Q];
static double H2[Q][3][3];        /* H2_ab = c_a c_b - cs^2 delta_ab */
static double H3[Q][3][3][3];     /* H3_abg = c_a c_b c_g - cs^2 (c_a d_bg + c_b d_ag + c_g d_ab) */
static int lattice_ready = 0;

static void build_lattice(void)
{
    if (lattice_ready) return;
    for (int cz = -1; cz <= 1; ++cz)
        for (int cy = -1; cy <= 1; ++cy)
            for (int cx = -1; cx <= 1; ++cx) {
                int i = 9 * (cz + 1) + 3 * (cy + 1) + (cx + 1);
                C[i][0] = cx; C[i][1] = cy; C[i][2] = cz;
                int n2 = cx * cx + cy * cy + cz * cz;
                Wt[i] = (n2 == 0) ? 8.0 / 27.0 : (n2 == 1) ? 2.0 / 27.0 : (n2 == 2) ? 1.0 / 54.0 : 1.0 / 216.0;
            }
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                H2[i][a][b] = C[i][a] * C[i][b] - CS2 * (a == b);
                for (int g = 0; g < 3; ++g)
                    H3[i][a][b][g] = C[i][a] * C[i][b] * C[i][g]
                                   - CS2 * (C[i][a] * (b == g) + C[i][b] * (a == g) + C[i][g] * (a == b));
            }
    lattice_ready = 1;
}

void oracle_lattice(int *c_out, double *w_out)
{
    build_lattice();
    for (int i = 0; i < Q; ++i) {
        for (int a = 0; a < 3; ++a) c_out[3 * i + a] = C[i][a];
        w_out[i] = Wt[i];
    }
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------------ */
/* Grid access with the boundary treatment of reading R13.                                     */
/* ------------------------------------------------------------------------------------------ */
static inline long node(const oracle_params *P, int x, int y, int z)
{
    return ((long)z * P->ny + y) * P->nx + x;
}

static inline int wrap(int v, int n) { v %= n; return v < 0 ? v + n : v; }

/* Map a possibly out-of-range coordinate to a stored node.  *zsign is -1 when the z coordinate
 * was mirrored at a wall (used to negate the z component of vector fields), else +1. */
static inline long ext_node(const oracle_params *P, int x, int y, int z, int *zsign)
{
    x = wrap(x, P->nx);
    y = wrap(y, P->ny);
    *zsign = 1;
    if (P->wall_z) {
        if (z < 0) { z = -1 - z; *zsign = -1; }
        else if (z >= P->nz) { z = 2 * P->nz - 1 - z; *zsign = -1; }
    } else {
        z = wrap(z, P->nz);
    }
    return node(P, x, y, z);
}

static inline double ext_scalar(const oracle_params *P, const double *psi, int x, int y, int z)
{
    int s;
    return psi[ext_node(P, x, y, z, &s)];
}

/* component a of a vector field stored as v[a*N + node] */
static inline double ext_vector(const oracle_params *P, const double *v, int a, int x, int y, int z)
{
    int s;
    long N = (long)P->nx * P->ny * P->nz;
    long k = ext_node(P, x, y, z, &s);
    double val = v[a * N + k];
    return (a == 2) ? s * val : val;
}

/* ------------------------------------------------------------------------------------------ */
/* Isotropic finite differences (Section "Model extension", gradient and Laplacian formulas).  */
/* ------------------------------------------------------------------------------------------ */

/* d_a psi = (1/cs^2) sum_i w_i c_ia psi(x + c_i) */
static void grad_at(const oracle_params *P, const double *psi, int x, int y, int z, double out[3])
{
    out[0] = out[1] = out[2] = 0.0;
    for (int i = 0; i < Q; ++i) {
        double v = ext_scalar(P, psi, x + C[i][0], y + C[i][1], z + C[i][2]);
        for (int a = 0; a < 3; ++a) out[a] += Wt[i] * C[i][a] * v / CS2;
    }
}

/* Reading R2: L[psi] = (2/cs^2) sum_{i != 0} w_i (psi(x + c_i) - psi(x)) */
static double lap_at(const oracle_params *P, const double *psi, int x, int y, int z)
{
    double c0 = ext_scalar(P, psi, x, y, z);
    double s = 0.0;
    for (int i = 0; i < Q; ++i) {
        if (C[i][0] == 0 && C[i][1] == 0 && C[i][2] == 0) continue;
        s += Wt[i] * (ext_scalar(P, psi, x + C[i][0], y + C[i][1], z + C[i][2]) - c0);
    }
    return 2.0 * s / CS2;
}

/* divergence of a vector field with the same gradient stencil: sum_a d_a V_a */
static double div_at(const oracle_params *P, const double *V, int x, int y, int z)
{
    double s = 0.0;
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < 3; ++a)
            s += Wt[i] * C[i][a] * ext_vector(P, V, a, x + C[i][0], y + C[i][1], z + C[i][2]) / CS2;
    return s;
}

void oracle_grad(const oracle_params *P, const double *psi, double *out)
{
    build_lattice();
    long N = (long)P->nx * P->ny * P->nz;
    #pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                double g[3];
                grad_at(P, psi, x, y, z, g);
                long k = node(P, x, y, z);
                for (int a = 0; a < 3; ++a) out[a * N + k] = g[a];
            }
}

void oracle_lap(const oracle_params *P, const double *psi, double *out)
{
    build_lattice();
    #pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x)
                out[node(P, x, y, z)] = lap_at(P, psi, x, y, z);
}

void oracle_div(const oracle_params *P, const double *V, double *out)
{
    build_lattice();
    #pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x)
                out[node(P, x, y, z)] = div_at(P, V, x, y, z);
}

/* ------------------------------------------------------------------------------------------ */
/* Per-node kinetic building blocks.                                                           */
/* ------------------------------------------------------------------------------------------ */

/* Eq. eqts: third-order Hermite equilibrium in pressure form. */
void oracle_equilibrium(double pstar, const double u[3], double feq[Q])
{
    build_lattice();
    for (int i = 0; i < Q; ++i) {
        double h1 = 0.0, h2 = 0.0, h3 = 0.0;
        for (int a = 0; a < 3; ++a) {
            h1 += C[i][a] * u[a];
            for (int b = 0; b < 3; ++b) {
                h2 += H2[i][a][b] * u[a] * u[b];
                for (int g = 0; g < 3; ++g) h3 += H3[i][a][b][g] * u[a] * u[b] * u[g];
            }
        }
        feq[i] = Wt[i] * (pstar + h1 / CS2 + h2 / (2.0 * CS2 * CS2) + h3 / (6.0 * CS2 * CS2 * CS2));
    }
}

/* Eq. guoforce with F replaced by the acceleration a (reading R1):
 * S_i = w_i [ (c_i - u)/cs^2 + (c_i . u) c_i / cs^4 ] . a */
void oracle_guo_source(const double u[3], const double acc[3], double S[Q])
{
    build_lattice();
    for (int i = 0; i < Q; ++i) {
        double cu = 0.0;
        for (int a = 0; a < 3; ++a) cu += C[i][a] * u[a];
        double s = 0.0;
        for (int a = 0; a < 3; ++a) s += ((C[i][a] - u[a]) / CS2 + cu * C[i][a] / (CS2 * CS2)) * acc[a];
        S[i] = Wt[i] * s;
    }
}

/* Eq. noneqts with weights and Hermite H2 (reading R7):
 * f^neq_i = w_i [ H2_i:A/(2cs^4) + H3_i:a3/(6cs^6) ],  a3_abg = u_a A_bg + u_b A_ag + u_g A_ab.
 * A is given as a full symmetric 3x3 matrix (row-major). */
void oracle_nonequilibrium(const double A[9], const double u[3], double fneq[Q])
{
    build_lattice();
    double a3[3][3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int g = 0; g < 3; ++g)
                a3[a][b][g] = u[a] * A[3 * b + g] + u[b] * A[3 * a + g] + u[g] * A[3 * a + b];
    for (int i = 0; i < Q; ++i) {
        double s2 = 0.0, s3 = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                s2 += H2[i][a][b] * A[3 * a + b];
                for (int g = 0; g < 3; ++g) s3 += H3[i][a][b][g] * a3[a][b][g];
            }
        fneq[i] = Wt[i] * (s2 / (2.0 * CS2 * CS2) + s3 / (6.0 * CS2 * CS2 * CS2));
    }
}

/* Moments of the streamed populations: p* (Eq. moments0), j = sum f c, Pi = sum f c c. */
static void raw_moments(const double f[Q], double *pstar, double j[3], double Pi[9])
{
    *pstar = 0.0;
    for (int a = 0; a < 3; ++a) j[a] = 0.0;
    for (int k = 0; k < 9; ++k) Pi[k] = 0.0;
    for (int i = 0; i < Q; ++i) {
        *pstar += f[i];
        for (int a = 0; a < 3; ++a) {
            j[a] += f[i] * C[i][a];
            for (int b = 0; b < 3; ++b) Pi[3 * a + b] += f[i] * C[i][a] * C[i][b];
        }
    }
}

/* Velocity, pre-regularisation and regularised collision of one node, given the streamed
 * populations f and the acceleration acc = F/rho (Eqs. moments0, moments1, hermite_neq2,
 * noneqts, LBexp; readings R1, R3, R7).
 * Outputs: g (post-collision), u (Eq. moments1), A (full 3x3, Eq. hermite_neq2). */
void oracle_collide_node(const double f[Q], const double acc[3], double omega,
                         double g[Q], double u[3], double A[9])
{
    build_lattice();
    double pstar, j[3], Pi[9];
    raw_moments(f, &pstar, j, Pi);
    for (int a = 0; a < 3; ++a) u[a] = j[a] + 0.5 * acc[a];

    double feq[Q], S[Q], fbar[Q], fneq[Q];
    oracle_equilibrium(pstar, u, feq);
    oracle_guo_source(u, acc, S);
    for (int i = 0; i < Q; ++i) fbar[i] = feq[i] - 0.5 * S[i];

    /* Eq. hermite_neq2, literal sum over populations */
    for (int k = 0; k < 9; ++k) A[k] = 0.0;
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                A[3 * a + b] += H2[i][a][b] * (f[i] - fbar[i]);

    oracle_nonequilibrium(A, u, fneq);
    for (int i = 0; i < Q; ++i) g[i] = fbar[i] + (1.0 - omega) * fneq[i] + S[i];
}

/* Local fluid properties from phi (density interpolation of the paper, reading R10). */
static void properties(const oracle_params *P, double phi, double *rho, double *nu, double *omega)
{
    *rho = P->rho_l * phi + (1.0 - phi) * P->rho_g;
    double mu = P->mu_l * phi + (1.0 - phi) * P->mu_g;
    *nu = mu / *rho;
    double tau = *nu / CS2 + 0.5;
    *omega = 1.0 / tau;
}

/* Total force density at one node (Section "Model extension"):
 *   F = F^s + F^p + F^nu + F^b
 *   F^s  = mu_phi grad(phi), mu_phi = 4 beta (phi-phi_l)(phi-phi_g)(phi-phi_0) - kappa lap(phi)
 *          with phi_l = 1, phi_g = 0, phi_0 = 1/2, beta = 12 sigma/delta, kappa = 3 sigma delta/2
 *   F^p  = -p* cs^2 grad(rho)                                                (Eq. press_corr)
 *   F^nu = -(nu omega / cs^2) [sum_i (f_i - f^eq_i(p*, ubar)) c_ia c_ib] d_b rho (Eq. visc_corr)
 *   F^b  = (rho - rho_ref) g + G_body                                        (reading R11)   */
void oracle_force_node(const oracle_params *P, const double f[Q], double phi, const double gphi[3],
                       double lphi, const double ubar[3], double F[3])
{
    build_lattice();
    double rho, nu, omega;
    properties(P, phi, &rho, &nu, &omega);
    double beta = 12.0 * P->sigma / P->width;
    double kappa = 1.5 * P->sigma * P->width;
    double mu_phi = 4.0 * beta * (phi - 1.0) * (phi - 0.0) * (phi - 0.5) - kappa * lphi;

    double grho[3];
    for (int a = 0; a < 3; ++a) grho[a] = (P->rho_l - P->rho_g) * gphi[a];

    double pstar = 0.0;
    for (int i = 0; i < Q; ++i) pstar += f[i];

    double feq[Q];
    oracle_equilibrium(pstar, ubar, feq);
    double M[9] = {0};
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) M[3 * a + b] += (f[i] - feq[i]) * C[i][a] * C[i][b];

    for (int a = 0; a < 3; ++a) {
        double Fs = mu_phi * gphi[a];
        double Fp = -pstar * CS2 * grho[a];
        double Fv = 0.0;
        for (int b = 0; b < 3; ++b) Fv += M[3 * a + b] * grho[b];
        Fv *= -(nu * omega / CS2);
        double Fb = (rho - P->rho_ref) * P->gravity[a] + P->body[a];
        F[a] = Fs + Fp + Fv + Fb;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Allen–Cahn FTCS update (interface-tracking item of the step list, readings R4, R5, R13):     */
/*   phi^{n+1} = phi^n - div(ubar phi^n) + D lap(phi^n) - kappa_AC div(phi^n (1-phi^n) n^n)   */
/*   kappa_AC = 4 D / delta,  n = grad(phi) / max(|grad(phi)|, 1e-12),  phi(1-phi) >= 0 (R15).  */
/* ------------------------------------------------------------------------------------------ */
void oracle_ac_update(const oracle_params *P, const double *phi, const double *ubar, double *phi_new)
{
    build_lattice();
    long N = (long)P->nx * P->ny * P->nz;
    double kac = 4.0 * P->mobility / P->width;
    double *V = (double *)malloc(sizeof(double) * 3 * N);   /* flux ubar phi + kac phi(1-phi) n */

    #pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long k = node(P, x, y, z);
                double g[3];
                grad_at(P, phi, x, y, z, g);
                double mag = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
                double den = mag > 1e-12 ? mag : 1e-12;
                double p = phi[k];
                double wgt = P->literal_weight ? p * (1.0 - p) : fmax(p * (1.0 - p), 0.0);
                for (int a = 0; a < 3; ++a)
                    V[a * N + k] = (P->advect ? 0.0 : ubar[a * N + k] * p) + kac * wgt * g[a] / den;
            }

    #pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long k = node(P, x, y, z);
                double adv = 0.0;   /* the literal advection term ubar . G[phi] */
                if (P->advect) {
                    double g[3];
                    grad_at(P, phi, x, y, z, g);
                    for (int a = 0; a < 3; ++a) adv += ubar[a * N + k] * g[a];
                }
                phi_new[k] = phi[k] - adv - div_at(P, V, x, y, z) + P->mobility * lap_at(P, phi, x, y, z);
            }
    free(V);
}

/* ------------------------------------------------------------------------------------------ */
/* Streaming: pull f_i(x) = g_i(x - c_i); at a z wall the population leaving x towards the wall */
/* comes back reversed to x (halfway bounce-back, reading R13): f_i(x) = g_{opp(i)}(x).        */
/* ------------------------------------------------------------------------------------------ */
static void pull(const oracle_params *P, const double *g, int x, int y, int z, double f[Q])
{
    long N = (long)P->nx * P->ny * P->nz;
    for (int i = 0; i < Q; ++i) {
        int sz = z - C[i][2];
        if (P->wall_z && (sz < 0 || sz >= P->nz)) {
            f[i] = g[(long)(Q - 1 - i) * N + node(P, x, y, z)];
        } else {
            int sx = wrap(x - C[i][0], P->nx);
            int sy = wrap(y - C[i][1], P->ny);
            sz = wrap(sz, P->nz);
            f[i] = g[(long)i * N + node(P, sx, sy, sz)];
        }
    }
}

/* One full step S^n = (g, phi, ubar) -> S^{n+1} = (g_new, phi_new, u_new). */
/* ------------------------------------------------------------------------------------------ */
/* The library's 16-bit population storage, emulated (not in the paper: the precision form of   */
/* the storage, its own design).  A node keeps h_i = g_i / w_i - p* - e_i(u), with              */
/* e_i(u) = f^eq_i(0, u) / w_i, rounded to BF16, or to FP16 after scaling by 2^12, from its FP32 */
/* value (the precision in which the library takes the rounding), plus P = p* - sum_i w_i hr_i.  */
/* The populations it represents are w_i (P + e_i(u) + hr_i): their sum is p*, because          */
/* sum_i w_i e_i(u) = 0.  Rounding is to nearest, ties to even.                                  */
/* ------------------------------------------------------------------------------------------ */
static float round_bf16(float v)
{
    uint32_t b;
    memcpy(&b, &v, 4);
    if ((b & 0x7fffffffu) > 0x7f800000u) return v;        /* NaN */
    b += 0x7fffu + ((b >> 16) & 1u);                      /* half an ulp of BF16, ties to even */
    b &= 0xffff0000u;
    float r;
    memcpy(&r, &b, 4);
    return r;
}

static double round16(int fmt, double h)
{
    const float h32 = (float)h;
    if (fmt == 1) return (double)round_bf16(h32);
    return (double)(float)(_Float16)(h32 * 4096.0f) / 4096.0;   /* IEEE binary16 conversion, scaled */
}

/* One node: the stored pair (P, hr) of populations g with velocity u, and the populations it
   represents (gout; may alias g). */
void oracle_store16_node(int fmt, const double g[Q], const double u[3], double *P_out, double hr[Q], double gout[Q])
{
    build_lattice();
    double ps = 0.0;
    for (int i = 0; i < Q; ++i) ps += g[i];
    double feq0[Q], sum = 0.0;
    oracle_equilibrium(0.0, u, feq0);
    for (int i = 0; i < Q; ++i) {
        hr[i] = round16(fmt, g[i] / Wt[i] - ps - feq0[i] / Wt[i]);
        sum += Wt[i] * hr[i];
    }
    const double Pv = ps - sum;
    for (int i = 0; i < Q; ++i) gout[i] = Wt[i] * (Pv + feq0[i] / Wt[i] + hr[i]);
    *P_out = Pv;
}

static void store16(int fmt, double g[Q], const double u[3])
{
    double Pv, hr[Q];
    oracle_store16_node(fmt, g, u, &Pv, hr, g);
}

/* ------------------------------------------------------------------------------------------ */
/* The library's 16-bit moment storage, emulated (not in the paper: its moment-only storage with */
/* a and B in BF16 / FP16).  After a collision a node's populations are a polynomial in c of its  */
/* p*, u, the acceleration a they carry and the non-equilibrium second moment B; the storage      */
/* keeps p* and u and rounds a and B.  The moments of the populations give the set back:          */
/*   sum g = p*,   sum g c = u + a / 2,                                                           */
/*   sum g c c = p* I / 3 + (2/9) (B + 4.5 u u + 4.5 sym(u a)),  sym(u a)_ab = (u_a a_b + u_b a_a)/2 */
/* and the polynomial, per unit weight, with cu = c.u, ca = c.a, cBc = c B c, is                  */
/*   g_i / w_i = K0 + 4.5 cu (cu + ca) + cBc + cu (K1 + 4.5 cu^2 + 3 cBc) + c.v,                  */
/*   K0 = p* - 1.5 u^2 - 1.5 u.a - tr B / 3,  K1 = 3 - 4.5 u^2 - tr B,  v = 1.5 a - 2 B u,         */
/* the third-order equilibrium of (p*, u), plus the Guo source for a, plus the regularised        */
/* non-equilibrium of B (its Hermite-2 and Hermite-3 parts).  The tests pin both directions       */
/* against the collision (mom_rebuild of mom_extract returns the collided populations).           */
/* ------------------------------------------------------------------------------------------ */
void oracle_mom_extract(const double g[Q], const double u[3], double *ps_out, double a[3], double B[9])
{
    build_lattice();
    double ps = 0.0, j[3] = {0, 0, 0}, Pi[3][3] = {{0}};
    for (int i = 0; i < Q; ++i) {
        ps += g[i];
        for (int x = 0; x < 3; ++x) {
            j[x] += g[i] * C[i][x];
            for (int y = 0; y < 3; ++y) Pi[x][y] += g[i] * C[i][x] * C[i][y];
        }
    }
    for (int x = 0; x < 3; ++x) a[x] = 2.0 * (j[x] - u[x]);
    for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y) {
            const double T = 4.5 * (Pi[x][y] - (x == y ? ps * CS2 : 0.0));
            B[3 * x + y] = T - 4.5 * u[x] * u[y] - 2.25 * (u[x] * a[y] + u[y] * a[x]);
        }
    *ps_out = ps;
}

void oracle_mom_rebuild(double ps, const double u[3], const double a[3], const double B[9], double g[Q])
{
    build_lattice();
    double u2 = 0.0, ua = 0.0, trB = 0.0, v[3];
    for (int x = 0; x < 3; ++x) {
        u2 += u[x] * u[x];
        ua += u[x] * a[x];
        trB += B[3 * x + x];
    }
    for (int x = 0; x < 3; ++x) {
        double Bu = 0.0;
        for (int y = 0; y < 3; ++y) Bu += B[3 * x + y] * u[y];
        v[x] = 1.5 * a[x] - 2.0 * Bu;
    }
    const double K0 = ps - 1.5 * u2 - 1.5 * ua - trB / 3.0;
    const double K1 = 3.0 - 4.5 * u2 - trB;
    for (int i = 0; i < Q; ++i) {
        double cu = 0.0, ca = 0.0, cv = 0.0, cBc = 0.0;
        for (int x = 0; x < 3; ++x) {
            cu += C[i][x] * u[x];
            ca += C[i][x] * a[x];
            cv += C[i][x] * v[x];
            for (int y = 0; y < 3; ++y) cBc += C[i][x] * B[3 * x + y] * C[i][y];
        }
        const double E = K0 + 4.5 * cu * (cu + ca) + cBc;
        const double O = cu * (K1 + 4.5 * cu * cu + 3.0 * cBc) + cv;
        g[i] = Wt[i] * (E + O);
    }
}

/* One node: the rounded deviation moments ab_out = (a_x, a_y, a_z, B_xx, B_yy, B_zz, B_xy, B_xz,
   B_yz) that the 16-bit moment storage (fmt 1 BF16, 2 FP16) keeps for populations g with
   velocity u, and the populations they represent (gout; may alias g). */
void oracle_store_mom16_node(int fmt, const double g[Q], const double u[3], double ab_out[9], double gout[Q])
{
    double ps, a[3], B[9];
    oracle_mom_extract(g, u, &ps, a, B);
    for (int x = 0; x < 3; ++x) a[x] = round16(fmt, a[x]);
    static const int pair[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    for (int m = 0; m < 6; ++m) {
        const double r = round16(fmt, B[3 * pair[m][0] + pair[m][1]]);
        B[3 * pair[m][0] + pair[m][1]] = B[3 * pair[m][1] + pair[m][0]] = r;
    }
    for (int x = 0; x < 3; ++x) ab_out[x] = a[x];
    for (int m = 0; m < 6; ++m) ab_out[3 + m] = B[3 * pair[m][0] + pair[m][1]];
    oracle_mom_rebuild(ps, u, a, B, gout);
}

void oracle_step(const oracle_params *P, const double *g, const double *phi, const double *ubar,
                 double *g_new, double *phi_new, double *u_new)
{
    build_lattice();
    long N = (long)P->nx * P->ny * P->nz;

    /* 1. interface tracking */
    oracle_ac_update(P, phi, ubar, phi_new);

    /* 2-6. streaming, moments, forces, velocity, pre-regularisation, collision */
    #pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long k = node(P, x, y, z);
                double f[Q];
                pull(P, g, x, y, z, f);

                double ph = phi_new[k];
                double rho, nu, omega;
                properties(P, ph, &rho, &nu, &omega);
                double gphi[3];
                grad_at(P, phi_new, x, y, z, gphi);
                double lphi = lap_at(P, phi_new, x, y, z);
                double ub[3] = {ubar[k], ubar[N + k], ubar[2 * N + k]};

                double F[3], acc[3];
                oracle_force_node(P, f, ph, gphi, lphi, ub, F);
                for (int a = 0; a < 3; ++a) acc[a] = F[a] / rho;

                double gout[Q], u[3], A[9];
                oracle_collide_node(f, acc, omega, gout, u, A);
                if (P->storage16 == 1 || P->storage16 == 2) store16(P->storage16, gout, u);
                if (P->storage16 == 3 || P->storage16 == 4) {
                    double ab[9];
                    oracle_store_mom16_node(P->storage16 - 2, gout, u, ab, gout);
                }
                for (int i = 0; i < Q; ++i) g_new[(long)i * N + k] = gout[i];
                for (int a = 0; a < 3; ++a) u_new[a * N + k] = u[a];
            }
}

/* Initial state: g = f^eq(p*0, u0), phi = phi0, ubar = u0 (treated as a post-collision state). */
void oracle_init(const oracle_params *P, const double *phi0, const double *u0, const double *pstar0,
                 double *g, double *phi, double *ubar)
{
    build_lattice();
    long N = (long)P->nx * P->ny * P->nz;
    for (long k = 0; k < N; ++k) {
        double u[3] = {u0[k], u0[N + k], u0[2 * N + k]};
        double feq[Q];
        oracle_equilibrium(pstar0 ? pstar0[k] : 0.0, u, feq);
        for (int i = 0; i < Q; ++i) g[(long)i * N + k] = feq[i];
        phi[k] = phi0[k];
        for (int a = 0; a < 3; ++a) ubar[a * N + k] = u[a];
    }
}

/* nsteps steps in place (ping-pong buffers allocated here). */
void oracle_run(const oracle_params *P, int nsteps, double *g, double *phi, double *ubar)
{
    long N = (long)P->nx * P->ny * P->nz;
    double *g2 = (double *)malloc(sizeof(double) * Q * N);
    double *p2 = (double *)malloc(sizeof(double) * N);
    double *u2 = (double *)malloc(sizeof(double) * 3 * N);
    double *ga = g, *pa = phi, *ua = ubar, *gb = g2, *pb = p2, *ub = u2;
    for (int s = 0; s < nsteps; ++s) {
        oracle_step(P, ga, pa, ua, gb, pb, ub);
        double *t;
        t = ga; ga = gb; gb = t;
        t = pa; pa = pb; pb = t;
        t = ua; ua = ub; ub = t;
    }
    if (ga != g) {
        memcpy(g, ga, sizeof(double) * Q * N);
        memcpy(phi, pa, sizeof(double) * N);
        memcpy(ubar, ua, sizeof(double) * 3 * N);
    }
    free(g2); free(p2); free(u2);
}

/* Macroscopic pressure p = p* rho cs^2 with p* = sum_i g_i (the collision conserves p*). */
void oracle_pressure(const oracle_params *P, const double *g, const double *phi, double *p)
{
    build_lattice();
    long N = (long)P->nx * P->ny * P->nz;
    for (long k = 0; k < N; ++k) {
        double ps = 0.0;
        for (int i = 0; i < Q; ++i) ps += g[(long)i * N + k];
        double rho = P->rho_l * phi[k] + (1.0 - phi[k]) * P->rho_g;
        p[k] = ps * rho * CS2;
    }
}

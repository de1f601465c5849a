/*
 * lbm_oracle.c -- plain FP64 CPU reference of the D3Q27 cumulant lattice
 * Boltzmann time step used to generate the channel-flow data set
 * (Sec. 3.1 "Generated dataset", Sec. 3.2 "waLBerla framework and solver
 * setup" of the paper; collision operator of Geier et al. 2015, which the
 * paper cites in Sec. 3.2).
 *
 * TEST INFRASTRUCTURE.  This file is the checker, not the product: only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg load it.
 * It shares no code, table or header with the CUDA library; the two meet only
 * through seeded inputs (obstacle masks, initial states).
 *
 * Deliberately different from the GPU path, so that agreement means something:
 *   - two arrays (pre-/post-collision) with pull streaming instead of the
 *     in-place AA pattern,
 *   - full populations f_i (not the shifted f_i - w_i) in FP64,
 *   - central moments by direct summation over the 27 velocities instead of
 *     the chimera transform,
 *   - pdfs recovered from post-collision central moments by Gaussian
 *     elimination on the 27x27 moment matrix instead of the inverse chimera.
 *
 * Lattice: c_i in {-1,0,1}^3, i = (cx+1) + 3(cy+1) + 9(cz+1), so that the
 * opposite direction of i is 26 - i.  Cells are stored x fastest:
 * cell = x + nx*(y + ny*z); pdf arrays are direction-major, f[i*N + cell].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 27
#define MI(a, b, c) ((a) + 3 * (b) + 9 * (c)) /* moment index, x order fastest */

/* ---- lattice --------------------------------------------------------- */

static void velocity(int i, int *cx, int *cy, int *cz)
{
    *cx = i % 3 - 1;
    *cy = (i / 3) % 3 - 1;
    *cz = i / 9 - 1;
}

/* D3Q27 weights by speed class: rest 8/27, face 2/27, edge 1/54, corner 1/216. */
static double weight(int i)
{
    int cx, cy, cz;
    velocity(i, &cx, &cy, &cz);
    int n = abs(cx) + abs(cy) + abs(cz);
    switch (n) {
    case 0: return 8.0 / 27.0;
    case 1: return 2.0 / 27.0;
    case 2: return 1.0 / 54.0;
    default: return 1.0 / 216.0;
    }
}

void oracle_weights(double *w)
{
    for (int i = 0; i < Q; ++i) w[i] = weight(i);
}

/* ---- parameters ------------------------------------------------------ */

/* Face kinds.  x high: FACE_OUTLET is the pressure outlet (anti-bounce-back
 * at rho_out), FACE_OUTFLOW the convective extrapolation outflow. */
enum { FACE_WALL = 0, FACE_PERIODIC = 1, FACE_INLET = 2, FACE_OUTLET = 3, FACE_OUTFLOW = 4 };

typedef struct {
    int32_t nx, ny, nz;
    int32_t face_x_lo, face_x_hi; /* inlet / outlet / wall / periodic   */
    int32_t face_y, face_z;       /* wall or periodic (both sides)     */
    double omega1;                /* shear rate                         */
    double omega2;                /* bulk rate                          */
    double omega3;                /* one rate for cumulants of order 3..6 */
    int32_t galilean;             /* 1: Galilean-corrected diagonal relaxation */
    int32_t pad0;
    double u_in;                  /* inlet velocity, along +x           */
    double rho_in;                /* wall density in the moving-wall term */
    double rho_out;               /* outlet density                     */
    int64_t mean_start, mean_end, mean_every; /* averaging window (steps) */
    int32_t param4;               /* 1: fourth-order parametrisation with limiter
                                   * (Geier et al. 2017) instead of omega3      */
    int32_t pad1;
    double limiter;               /* lambda of that limiter                    */
} oracle_params;

/* Shear rate from the Reynolds number at fixed inlet velocity (Sec. 3.1:
 * Re is set through the lattice viscosity): nu = U L / Re, tau = 3 nu + 1/2. */
double oracle_omega_from_re(double re, double u, double l_ref)
{
    double nu = u * l_ref / re;
    return 1.0 / (3.0 * nu + 0.5);
}

/* ---- equilibrium ------------------------------------------------------ */

/* Product-form equilibrium of the cumulant method: f_eq = rho Phi(ux)Phi(uy)Phi(uz)
 * with Phi_0(u) = 2/3 - u^2 and Phi_{+-1}(u) = (1/3 + u^2 +- u)/2.  Its cumulants
 * of order >= 3 vanish and its diagonal second-order cumulants equal 1/3. */
static double phi(int c, double u)
{
    if (c == 0) return 2.0 / 3.0 - u * u;
    return 0.5 * (1.0 / 3.0 + u * u + c * u);
}

void oracle_equilibrium(double rho, double ux, double uy, double uz, double *feq)
{
    for (int i = 0; i < Q; ++i) {
        int cx, cy, cz;
        velocity(i, &cx, &cy, &cz);
        feq[i] = rho * phi(cx, ux) * phi(cy, uy) * phi(cz, uz);
    }
}

/* ---- moments ------------------------------------------------------------ */

static double ipow(double v, int n)
{
    double r = 1.0;
    for (int k = 0; k < n; ++k) r *= v;
    return r;
}

void oracle_macros(const double *f, double *rho, double *u)
{
    double r = 0, jx = 0, jy = 0, jz = 0;
    for (int i = 0; i < Q; ++i) {
        int cx, cy, cz;
        velocity(i, &cx, &cy, &cz);
        r += f[i];
        jx += cx * f[i];
        jy += cy * f[i];
        jz += cz * f[i];
    }
    *rho = r;
    u[0] = jx / r;
    u[1] = jy / r;
    u[2] = jz / r;
}

/* Powers (c - u_d)^a for c in {-1,0,1}, a in {0,1,2}, per axis d. */
static void shifted_powers(const double *u, double pw[3][3][3])
{
    for (int d = 0; d < 3; ++d)
        for (int c = -1; c <= 1; ++c)
            for (int a = 0; a < 3; ++a) pw[d][c + 1][a] = ipow(c - u[d], a);
}

/* Normalised central moments k_abc = sum_i f_i (cx-ux)^a (cy-uy)^b (cz-uz)^c / rho,
 * a,b,c in {0,1,2}, by direct summation. */
void oracle_central_moments(const double *f, double *k, double *rho_out, double *u_out)
{
    double rho, u[3], pw[3][3][3];
    oracle_macros(f, &rho, u);
    shifted_powers(u, pw);
    for (int c = 0; c < 3; ++c)
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) {
                double s = 0.0;
                for (int i = 0; i < Q; ++i) {
                    int cx, cy, cz;
                    velocity(i, &cx, &cy, &cz);
                    s += f[i] * pw[0][cx + 1][a] * pw[1][cy + 1][b] * pw[2][cz + 1][c];
                }
                k[MI(a, b, c)] = s / rho;
            }
    if (rho_out) *rho_out = rho;
    if (u_out) { u_out[0] = u[0]; u_out[1] = u[1]; u_out[2] = u[2]; }
}

/* ---- cumulants (normalised, zero-mean frame) ------------------------- */
/* Orders 2 and 3 coincide with the central moments; orders 4..6 subtract the
 * products of lower-order moments over the set partitions of the index
 * multiset whose blocks all have at least two elements (the first central
 * moments vanish).  C_000 and the first-order entries are set to zero. */

#define K(a, b, c) k[MI(a, b, c)]

static double sum42(const double *k)
{
    return K(2,0,0) * K(0,2,2) + K(0,2,0) * K(2,0,2) + K(0,0,2) * K(2,2,0)
         + 4.0 * (K(0,1,1) * K(2,1,1) + K(1,0,1) * K(1,2,1) + K(1,1,0) * K(1,1,2));
}

static double sum33(const double *k)
{
    return 4.0 * K(1,1,1) * K(1,1,1)
         + 2.0 * (K(1,2,0) * K(1,0,2) + K(2,1,0) * K(0,1,2) + K(2,0,1) * K(0,2,1));
}

static double sum222(const double *k)
{
    return 8.0 * K(1,1,0) * K(1,0,1) * K(0,1,1)
         + 2.0 * (K(1,0,1) * K(1,0,1) * K(0,2,0) + K(0,1,1) * K(0,1,1) * K(2,0,0)
                + K(1,1,0) * K(1,1,0) * K(0,0,2))
         + K(2,0,0) * K(0,2,0) * K(0,0,2);
}

/* fourth-order product terms for C_211-type and C_220-type entries */
static double p211(const double *k) { return K(2,0,0) * K(0,1,1) + 2.0 * K(1,1,0) * K(1,0,1); }
static double p121(const double *k) { return K(0,2,0) * K(1,0,1) + 2.0 * K(1,1,0) * K(0,1,1); }
static double p112(const double *k) { return K(0,0,2) * K(1,1,0) + 2.0 * K(1,0,1) * K(0,1,1); }
static double p220(const double *k) { return K(2,0,0) * K(0,2,0) + 2.0 * K(1,1,0) * K(1,1,0); }
static double p202(const double *k) { return K(2,0,0) * K(0,0,2) + 2.0 * K(1,0,1) * K(1,0,1); }
static double p022(const double *k) { return K(0,2,0) * K(0,0,2) + 2.0 * K(0,1,1) * K(0,1,1); }
/* fifth order: pairs (2 elements) times the remaining triple */
static double p122(const double *k)
{
    return K(0,0,2) * K(1,2,0) + K(0,2,0) * K(1,0,2) + 4.0 * K(0,1,1) * K(1,1,1)
         + 2.0 * (K(1,0,1) * K(0,2,1) + K(1,1,0) * K(0,1,2));
}
static double p212(const double *k)
{
    return K(2,0,0) * K(0,1,2) + K(0,0,2) * K(2,1,0) + 4.0 * K(1,0,1) * K(1,1,1)
         + 2.0 * (K(1,1,0) * K(1,0,2) + K(0,1,1) * K(2,0,1));
}
static double p221(const double *k)
{
    return K(2,0,0) * K(0,2,1) + K(0,2,0) * K(2,0,1) + 4.0 * K(1,1,0) * K(1,1,1)
         + 2.0 * (K(1,0,1) * K(1,2,0) + K(0,1,1) * K(2,1,0));
}

void oracle_cumulants_from_moments(const double *k, double *C)
{
    for (int m = 0; m < Q; ++m) C[m] = k[m];     /* orders 2, 3 (and 4..6 overwritten) */
    C[MI(0,0,0)] = 0.0;
    C[MI(1,0,0)] = C[MI(0,1,0)] = C[MI(0,0,1)] = 0.0;
    C[MI(2,1,1)] = K(2,1,1) - p211(k);
    C[MI(1,2,1)] = K(1,2,1) - p121(k);
    C[MI(1,1,2)] = K(1,1,2) - p112(k);
    C[MI(2,2,0)] = K(2,2,0) - p220(k);
    C[MI(2,0,2)] = K(2,0,2) - p202(k);
    C[MI(0,2,2)] = K(0,2,2) - p022(k);
    C[MI(1,2,2)] = K(1,2,2) - p122(k);
    C[MI(2,1,2)] = K(2,1,2) - p212(k);
    C[MI(2,2,1)] = K(2,2,1) - p221(k);
    C[MI(2,2,2)] = K(2,2,2) - sum42(k) - sum33(k) + 2.0 * sum222(k);
}

/* Inverse of the above: rebuild central moments order by order, each order
 * using the already rebuilt lower orders. */
void oracle_moments_from_cumulants(const double *C, double *k)
{
    for (int m = 0; m < Q; ++m) k[m] = C[m];
    k[MI(0,0,0)] = 1.0;
    k[MI(1,0,0)] = k[MI(0,1,0)] = k[MI(0,0,1)] = 0.0;
    /* order 4 from orders 2 */
    k[MI(2,1,1)] = C[MI(2,1,1)] + p211(k);
    k[MI(1,2,1)] = C[MI(1,2,1)] + p121(k);
    k[MI(1,1,2)] = C[MI(1,1,2)] + p112(k);
    k[MI(2,2,0)] = C[MI(2,2,0)] + p220(k);
    k[MI(2,0,2)] = C[MI(2,0,2)] + p202(k);
    k[MI(0,2,2)] = C[MI(0,2,2)] + p022(k);
    /* order 5 from orders 2, 3 */
    k[MI(1,2,2)] = C[MI(1,2,2)] + p122(k);
    k[MI(2,1,2)] = C[MI(2,1,2)] + p212(k);
    k[MI(2,2,1)] = C[MI(2,2,1)] + p221(k);
    /* order 6 from orders 2, 3, 4 */
    k[MI(2,2,2)] = C[MI(2,2,2)] + sum42(k) + sum33(k) - 2.0 * sum222(k);
}
#undef K

/* ---- relaxation --------------------------------------------------------- */
/* Rates of the fourth-order parametrisation (Geier, Pasquali & Schoenherr
 * 2017), functions of the shear rate w1 and the bulk rate w2 chosen so that
 * the leading error of the diffusion term cancels: omega3 (sums of third-
 * order cumulant pairs), omega4 (their differences), omega5 (C_111), and the
 * coefficients A, B of the fourth-order cumulants' equilibria.  Undefined at
 * w1 = w2 (A and B have the factor w1 - w2 in their denominators). */
void oracle_param4_rates(double w1, double w2, double *out5)
{
    out5[0] = 8.0 * (w1 - 2.0) * (w2 * (3.0 * w1 - 1.0) - 5.0 * w1)
            / (8.0 * (5.0 - 2.0 * w1) * w1 + w2 * (8.0 + w1 * (9.0 * w1 - 26.0)));
    out5[1] = 8.0 * (w1 - 2.0) * (w1 + w2 * (3.0 * w1 - 7.0))
            / (w2 * (56.0 - 42.0 * w1 + 9.0 * w1 * w1) - 8.0 * w1);
    out5[2] = 24.0 * (w1 - 2.0) * (4.0 * w1 * w1 + w1 * w2 * (18.0 - 13.0 * w1) + w2 * w2 * (2.0 + w1 * (6.0 * w1 - 11.0)))
            / (16.0 * w1 * w1 * (w1 - 6.0) - 2.0 * w1 * w2 * (216.0 + 5.0 * w1 * (9.0 * w1 - 46.0))
               + w2 * w2 * (w1 * (3.0 * w1 - 10.0) * (15.0 * w1 - 28.0) - 48.0));
    const double den = (w1 - w2) * (w2 * (2.0 + 3.0 * w1) - 8.0 * w1);
    out5[3] = (4.0 * w1 * w1 + 2.0 * w1 * w2 * (w1 - 6.0) + w2 * w2 * (w1 * (10.0 - 3.0 * w1) - 4.0)) / den;
    out5[4] = (4.0 * w1 * w2 * (9.0 * w1 - 16.0) - 4.0 * w1 * w1 - 2.0 * w2 * w2 * (2.0 + 9.0 * w1 * (w1 - 2.0)))
            / (3.0 * den);
}

/* Relaxation rate w raised towards 1 where the cumulant X is large against
 * the limiter lambda: w + (1 - w) |X| / (|X| + lambda). */
static double limited(double w, double X, double lambda)
{
    return w + (1.0 - w) * fabs(X) / (fabs(X) + lambda);
}

/* Orders 3..6 of the parametrised operator (normalised cumulants):
 *   third order in the combinations C_210 +- C_012, C_201 +- C_021,
 *   C_120 +- C_102 (sums with omega3, differences with omega4) and C_111
 *   (omega5), each rate limited by the size of its own combination;
 *   fourth order set to the equilibria that carry the velocity gradients
 *   (rates 1): C*_220 = -(2/3) A (1/w1 - 1/2)(dxu + dyv) and its two
 *   permutations, C*_211 = -(1/3) B (1/w1 - 1/2) D_yz with D_yz = -3 w1 C_011
 *   the shear-rate estimate, and its two permutations;
 *   fifth and sixth orders to 0. */
static void parametrised_higher_orders(const oracle_params *p, const double *C, double dxu, double dyv, double dzw,
                                       double *Cs)
{
    const double w1 = p->omega1, lam = p->limiter;
    double r[5];
    oracle_param4_rates(w1, p->omega2, r);
    const double w3 = r[0], w4 = r[1], w5 = r[2], A = r[3], B = r[4];
    /* third order: (first, second) of each pair, sum and difference */
    static const int pairs[3][2][3] = {{{2, 1, 0}, {0, 1, 2}}, {{2, 0, 1}, {0, 2, 1}}, {{1, 2, 0}, {1, 0, 2}}};
    for (int k = 0; k < 3; ++k) {
        const int a = MI(pairs[k][0][0], pairs[k][0][1], pairs[k][0][2]);
        const int b = MI(pairs[k][1][0], pairs[k][1][1], pairs[k][1][2]);
        const double sp = C[a] + C[b], sm = C[a] - C[b];
        const double sps = (1.0 - limited(w3, sp, lam)) * sp;
        const double sms = (1.0 - limited(w4, sm, lam)) * sm;
        Cs[a] = 0.5 * (sps + sms);
        Cs[b] = 0.5 * (sps - sms);
    }
    Cs[MI(1,1,1)] = (1.0 - limited(w5, C[MI(1,1,1)], lam)) * C[MI(1,1,1)];
    /* fourth order */
    const double visc = 1.0 / w1 - 0.5;
    Cs[MI(2,2,0)] = -(2.0 / 3.0) * A * visc * (dxu + dyv);
    Cs[MI(2,0,2)] = -(2.0 / 3.0) * A * visc * (dxu + dzw);
    Cs[MI(0,2,2)] = -(2.0 / 3.0) * A * visc * (dyv + dzw);
    Cs[MI(2,1,1)] = -(1.0 / 3.0) * B * visc * (-3.0 * w1 * C[MI(0,1,1)]);
    Cs[MI(1,2,1)] = -(1.0 / 3.0) * B * visc * (-3.0 * w1 * C[MI(1,0,1)]);
    Cs[MI(1,1,2)] = -(1.0 / 3.0) * B * visc * (-3.0 * w1 * C[MI(1,1,0)]);
    /* fifth and sixth */
    Cs[MI(1,2,2)] = Cs[MI(2,1,2)] = Cs[MI(2,2,1)] = 0.0;
    Cs[MI(2,2,2)] = 0.0;
}

/* Cumulant relaxation (Geier et al. 2015, the operator of Sec. 3.2):
 *   - off-diagonal second order relaxes with the shear rate omega1,
 *   - the two deviatoric differences of the diagonal with omega1 and the trace
 *     with the bulk rate omega2, towards 0 and 1 (normalised), each carrying the
 *     Galilean correction built from the velocity-derivative estimates
 *     dxu, dyv, dzw that the non-equilibrium diagonal moments imply,
 *   - every cumulant of order 3..6 relaxes with omega3 towards 0, or, with
 *     param4, as the fourth-order parametrisation prescribes (see
 *     parametrised_higher_orders). */
void oracle_relax(const oracle_params *p, const double *u, const double *C, double *Cs)
{
    const double w1 = p->omega1, w2 = p->omega2, w3 = p->omega3;
    for (int m = 0; m < Q; ++m) Cs[m] = (1.0 - w3) * C[m];
    Cs[MI(0,0,0)] = 0.0;
    Cs[MI(1,0,0)] = Cs[MI(0,1,0)] = Cs[MI(0,0,1)] = 0.0;

    Cs[MI(1,1,0)] = (1.0 - w1) * C[MI(1,1,0)];
    Cs[MI(1,0,1)] = (1.0 - w1) * C[MI(1,0,1)];
    Cs[MI(0,1,1)] = (1.0 - w1) * C[MI(0,1,1)];

    const double cxx = C[MI(2,0,0)], cyy = C[MI(0,2,0)], czz = C[MI(0,0,2)];
    const double dxy = cxx - cyy, dxz = cxx - czz, tr = cxx + cyy + czz;
    const double dxu = -0.5 * w1 * (2.0 * cxx - cyy - czz) - 0.5 * w2 * (tr - 1.0);
    const double dyv = dxu + 1.5 * w1 * dxy;
    const double dzw = dxu + 1.5 * w1 * dxz;
    const double g = p->galilean ? 1.0 : 0.0;
    const double ux2 = u[0] * u[0], uy2 = u[1] * u[1], uz2 = u[2] * u[2];

    const double dxy_s = (1.0 - w1) * dxy - g * 3.0 * (1.0 - 0.5 * w1) * (ux2 * dxu - uy2 * dyv);
    const double dxz_s = (1.0 - w1) * dxz - g * 3.0 * (1.0 - 0.5 * w1) * (ux2 * dxu - uz2 * dzw);
    const double tr_s = w2 * 1.0 + (1.0 - w2) * tr
                      - g * 3.0 * (1.0 - 0.5 * w2) * (ux2 * dxu + uy2 * dyv + uz2 * dzw);

    Cs[MI(2,0,0)] = (dxy_s + dxz_s + tr_s) / 3.0;
    Cs[MI(0,2,0)] = Cs[MI(2,0,0)] - dxy_s;
    Cs[MI(0,0,2)] = Cs[MI(2,0,0)] - dxz_s;

    if (p->param4) parametrised_higher_orders(p, C, dxu, dyv, dzw, Cs);
}

/* ---- back to populations -------------------------------------------- */
/* Solve sum_i M[m][i] f_i = rho k_m with M[abc][i] = (cx-ux)^a (cy-uy)^b (cz-uz)^c
 * by Gaussian elimination with partial pivoting. */
void oracle_pdfs_from_moments(const double *k, double rho, const double *u, double *f)
{
    double A[Q][Q + 1], pw[3][3][3];
    shifted_powers(u, pw);
    for (int c = 0; c < 3; ++c)
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) {
                int m = MI(a, b, c);
                for (int i = 0; i < Q; ++i) {
                    int cx, cy, cz;
                    velocity(i, &cx, &cy, &cz);
                    A[m][i] = pw[0][cx + 1][a] * pw[1][cy + 1][b] * pw[2][cz + 1][c];
                }
                A[m][Q] = rho * k[m];
            }
    for (int col = 0; col < Q; ++col) {
        int piv = col;
        for (int r = col + 1; r < Q; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (piv != col)
            for (int j = 0; j <= Q; ++j) { double t = A[col][j]; A[col][j] = A[piv][j]; A[piv][j] = t; }
        for (int r = col + 1; r < Q; ++r) {
            double fct = A[r][col] / A[col][col];
            if (fct == 0.0) continue;
            for (int j = col; j <= Q; ++j) A[r][j] -= fct * A[col][j];
        }
    }
    for (int r = Q - 1; r >= 0; --r) {
        double s = A[r][Q];
        for (int j = r + 1; j < Q; ++j) s -= A[r][j] * f[j];
        f[r] = s / A[r][r];
    }
}

/* One collision: f -> f*.  Also returns the pre-collision rho and u. */
void oracle_collide(const oracle_params *p, const double *f, double *fout, double *rho_out, double *u_out)
{
    double k[Q], C[Q], Cs[Q], ks[Q], rho, u[3];
    oracle_central_moments(f, k, &rho, u);
    oracle_cumulants_from_moments(k, C);
    oracle_relax(p, u, C, Cs);
    oracle_moments_from_cumulants(Cs, ks);
    oracle_pdfs_from_moments(ks, rho, u, fout);
    if (rho_out) *rho_out = rho;
    if (u_out) { u_out[0] = u[0]; u_out[1] = u[1]; u_out[2] = u[2]; }
}

/* ---- lattice state ---------------------------------------------------- */

typedef struct {
    oracle_params p;
    int64_t n;           /* cells */
    uint8_t *solid;      /* 1 = obstacle cell */
    double *f;           /* f[i*n + cell], pre-collision at time t */
    double *post;        /* post-collision */
    double *rho, *u;     /* pre-collision macros of the last step (u[3*cell + d]) */
    double *msum;        /* 4*n mean sums: rho-1, ux, uy, uz */
    double *qsum;        /* 6*n sums of velocity products: uxux, uyuy, uzuz, uxuy, uxuz, uyuz */
    int64_t msamples;
    double *q;           /* wall distances q[j*n + cell] of links x -> x + c_j into
                            obstacle cells (fraction of the link in the fluid), or
                            NULL for halfway bounce-back everywhere */
    double *force;       /* 3 per step */
    int64_t force_cap;
    int64_t t;
} oracle_lbm;

static int64_t cell_of(const oracle_lbm *o, int x, int y, int z)
{
    return (int64_t)x + (int64_t)o->p.nx * ((int64_t)y + (int64_t)o->p.ny * z);
}

oracle_lbm *oracle_lbm_create(const oracle_params *p, const uint8_t *solid)
{
    oracle_lbm *o = (oracle_lbm *)calloc(1, sizeof(oracle_lbm));
    o->p = *p;
    o->n = (int64_t)p->nx * p->ny * p->nz;
    o->solid = (uint8_t *)malloc(o->n);
    for (int64_t c = 0; c < o->n; ++c) o->solid[c] = solid ? (solid[c] != 0) : 0;
    o->f = (double *)malloc(sizeof(double) * Q * o->n);
    o->post = (double *)malloc(sizeof(double) * Q * o->n);
    o->rho = (double *)calloc(o->n, sizeof(double));
    o->u = (double *)calloc(3 * o->n, sizeof(double));
    o->msum = (double *)calloc(4 * o->n, sizeof(double));
    o->qsum = (double *)calloc(6 * o->n, sizeof(double));
    for (int i = 0; i < Q; ++i) {
        double w = weight(i);
        for (int64_t c = 0; c < o->n; ++c) { o->f[i * o->n + c] = w; o->post[i * o->n + c] = w; }
    }
    o->force_cap = 1024;
    o->force = (double *)calloc(3 * o->force_cap, sizeof(double));
    return o;
}

void oracle_lbm_destroy(oracle_lbm *o)
{
    if (!o) return;
    free(o->solid); free(o->f); free(o->post); free(o->rho); free(o->u);
    free(o->msum); free(o->qsum); free(o->q); free(o->force); free(o);
}

void oracle_lbm_set_f(oracle_lbm *o, const double *f) { memcpy(o->f, f, sizeof(double) * Q * o->n); }

/* Wall distances for the interpolated bounce-back on obstacle links (Sec.
 * 3.2): q[j*n + cell] in (0, 1] for each link from a fluid cell into an
 * obstacle cell along c_j; other entries are ignored.  NULL restores
 * halfway bounce-back (q = 1/2 on every link). */
void oracle_lbm_set_q(oracle_lbm *o, const double *q)
{
    free(o->q);
    o->q = NULL;
    if (!q) return;
    o->q = (double *)malloc(sizeof(double) * Q * o->n);
    memcpy(o->q, q, sizeof(double) * Q * o->n);
}

/* A fluid cell at (x, y, z), reached through periodic faces if needed (a
 * wall, inlet or outlet face ends the interpolation stencil). */
static int inner_fluid(const oracle_lbm *o, int x, int y, int z, int64_t *cell)
{
    const oracle_params *p = &o->p;
    if (x < 0 || x >= p->nx) {
        if (p->face_x_lo != FACE_PERIODIC) return 0;
        x = ((x % p->nx) + p->nx) % p->nx;
    }
    if (y < 0 || y >= p->ny) {
        if (p->face_y != FACE_PERIODIC) return 0;
        y = ((y % p->ny) + p->ny) % p->ny;
    }
    if (z < 0 || z >= p->nz) {
        if (p->face_z != FACE_PERIODIC) return 0;
        z = ((z % p->nz) + p->nz) % p->nz;
    }
    *cell = cell_of(o, x, y, z);
    return !o->solid[*cell];
}

/* Population returned into pull direction i of fluid cell c = (x, y, z) whose
 * link to x - c_i ends in an obstacle at fraction q of the link (Bouzidi,
 * Firdaouss & Lallemand 2001): j = 26 - i heads into the wall; x1 = x + c_i
 * and x2 = x + 2 c_i are the cells behind.  Quadratic interpolation when x1
 * and x2 are fluid cells (inside, or across periodic faces), linear when only
 * x1 is, halfway bounce-back otherwise (for q = 1/2 all three coincide):
 *   q <  1/2: q(1+2q) f*_j(x) + (1-4q^2) f*_j(x1) - q(1-2q) f*_j(x2)
 *             [linear: 2q f*_j(x) + (1-2q) f*_j(x1)]
 *   q >= 1/2: f*_j(x)/(q(2q+1)) + (2q-1)/q f*_i(x) - (2q-1)/(2q+1) f*_i(x1)
 *             [linear: f*_j(x)/(2q) + (2q-1)/(2q) f*_i(x)]                   */
static double interpolated_bounce_back(const oracle_lbm *o, int64_t c, int x, int y, int z, int i)
{
    const int64_t n = o->n;
    const int j = Q - 1 - i;
    int cx, cy, cz;
    velocity(i, &cx, &cy, &cz);
    const double a0 = o->post[j * n + c];
    const double q = o->q[j * n + c];
    int64_t x1 = -1, x2 = -1;
    const int v1 = inner_fluid(o, x + cx, y + cy, z + cz, &x1);
    const int v2 = v1 && inner_fluid(o, x + 2 * cx, y + 2 * cy, z + 2 * cz, &x2);
    if (!v1) return a0;
    if (q < 0.5) {
        if (v2)
            return q * (1.0 + 2.0 * q) * a0 + (1.0 - 4.0 * q * q) * o->post[j * n + x1]
                 - q * (1.0 - 2.0 * q) * o->post[j * n + x2];
        return 2.0 * q * a0 + (1.0 - 2.0 * q) * o->post[j * n + x1];
    }
    if (v2)
        return a0 / (q * (2.0 * q + 1.0)) + (2.0 * q - 1.0) / q * o->post[i * n + c]
             - (2.0 * q - 1.0) / (2.0 * q + 1.0) * o->post[i * n + x1];
    return a0 / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * o->post[i * n + c];
}
void oracle_lbm_get_f(const oracle_lbm *o, double *f) { memcpy(f, o->f, sizeof(double) * Q * o->n); }
int64_t oracle_lbm_time(const oracle_lbm *o) { return o->t; }
void oracle_lbm_set_time(oracle_lbm *o, int64_t t) { o->t = t; }

/* Macros of the current (pre-collision) state; solid cells report rho=1, u=0. */
void oracle_lbm_macros(const oracle_lbm *o, double *rho, double *u)
{
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < o->n; ++c) {
        double fc[Q], r, v[3];
        if (o->solid[c]) { rho[c] = 1.0; u[3 * c] = u[3 * c + 1] = u[3 * c + 2] = 0.0; continue; }
        for (int i = 0; i < Q; ++i) fc[i] = o->f[i * o->n + c];
        oracle_macros(fc, &r, v);
        rho[c] = r; u[3 * c] = v[0]; u[3 * c + 1] = v[1]; u[3 * c + 2] = v[2];
    }
}

/* Mean fields: (ux, uy, uz, p) per cell, p = (rho - 1)/3; solid cells 0. */
/* Velocity covariances over the same samples as the means (Reynolds
 * stresses, the turbulence statistics of Sec. 3.3): per cell
 * <ux ux> - <ux><ux>, <uy uy> - ..., <uz uz> - ..., <ux uy> - <ux><uy>,
 * <ux uz> - ..., <uy uz> - ... .  Returns the sample count. */
int64_t oracle_lbm_stats(const oracle_lbm *o, double *out)
{
    const double s = o->msamples > 0 ? 1.0 / (double)o->msamples : 0.0;
    for (int64_t c = 0; c < o->n; ++c) {
        const double mx = o->msum[4 * c + 1] * s, my = o->msum[4 * c + 2] * s, mz = o->msum[4 * c + 3] * s;
        out[6 * c + 0] = o->qsum[6 * c + 0] * s - mx * mx;
        out[6 * c + 1] = o->qsum[6 * c + 1] * s - my * my;
        out[6 * c + 2] = o->qsum[6 * c + 2] * s - mz * mz;
        out[6 * c + 3] = o->qsum[6 * c + 3] * s - mx * my;
        out[6 * c + 4] = o->qsum[6 * c + 4] * s - mx * mz;
        out[6 * c + 5] = o->qsum[6 * c + 5] * s - my * mz;
    }
    return o->msamples;
}

int64_t oracle_lbm_means(const oracle_lbm *o, double *out)
{
    for (int64_t c = 0; c < o->n; ++c) {
        double s = o->msamples > 0 ? 1.0 / (double)o->msamples : 0.0;
        out[4 * c + 0] = o->msum[4 * c + 1] * s;
        out[4 * c + 1] = o->msum[4 * c + 2] * s;
        out[4 * c + 2] = o->msum[4 * c + 3] * s;
        out[4 * c + 3] = o->msum[4 * c + 0] * s / 3.0;
    }
    return o->msamples;
}

void oracle_lbm_forces(const oracle_lbm *o, double *out) { memcpy(out, o->force, sizeof(double) * 3 * o->t); }

static int in_sample_window(const oracle_params *p, int64_t t)
{
    if (p->mean_every <= 0) return 0;
    if (t < p->mean_start || t >= p->mean_end) return 0;
    return (t - p->mean_start) % p->mean_every == 0;
}

/* Classification of the cell a link comes from / goes to (Sec. 3.1: velocity
 * inlet, outflow, no-slip lateral walls; obstacle bounce-back Sec. 3.2). */
enum { SRC_FLUID = 0, SRC_WALL = 1, SRC_INLET = 2, SRC_OUTLET = 3, SRC_OUTFLOW = 4 };

static int classify(const oracle_lbm *o, int x, int y, int z, int64_t *cell)
{
    const oracle_params *p = &o->p;
    /* lateral walls first: a link that leaves through y or z is a wall link */
    if (y < 0 || y >= p->ny) {
        if (p->face_y != FACE_PERIODIC) return SRC_WALL;
        y = (y + p->ny) % p->ny;
    }
    if (z < 0 || z >= p->nz) {
        if (p->face_z != FACE_PERIODIC) return SRC_WALL;
        z = (z + p->nz) % p->nz;
    }
    if (x < 0) {
        if (p->face_x_lo == FACE_INLET) return SRC_INLET;
        if (p->face_x_lo == FACE_WALL) return SRC_WALL;
        x += p->nx;
    } else if (x >= p->nx) {
        if (p->face_x_hi == FACE_OUTLET) return SRC_OUTLET;
        if (p->face_x_hi == FACE_OUTFLOW) return SRC_OUTFLOW;
        if (p->face_x_hi == FACE_WALL) return SRC_WALL;
        x -= p->nx;
    }
    *cell = cell_of(o, x, y, z);
    return o->solid[*cell] ? SRC_WALL : SRC_FLUID;
}

void oracle_lbm_step(oracle_lbm *o, int nsteps)
{
    const oracle_params *p = &o->p;
    const int64_t n = o->n;
    for (int s = 0; s < nsteps; ++s) {
        const int sample = in_sample_window(p, o->t);
        /* 1. collide every fluid cell (pre-collision macros kept for the
         *    outlet condition and the time average) */
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t c = 0; c < n; ++c) {
            if (o->solid[c]) continue;
            double fc[Q], fs[Q], r, v[3];
            for (int i = 0; i < Q; ++i) fc[i] = o->f[i * n + c];
            oracle_collide(p, fc, fs, &r, v);
            for (int i = 0; i < Q; ++i) o->post[i * n + c] = fs[i];
            o->rho[c] = r;
            o->u[3 * c] = v[0]; o->u[3 * c + 1] = v[1]; o->u[3 * c + 2] = v[2];
            if (sample) {
                o->msum[4 * c + 0] += r - 1.0;
                o->msum[4 * c + 1] += v[0];
                o->msum[4 * c + 2] += v[1];
                o->msum[4 * c + 3] += v[2];
                o->qsum[6 * c + 0] += v[0] * v[0];
                o->qsum[6 * c + 1] += v[1] * v[1];
                o->qsum[6 * c + 2] += v[2] * v[2];
                o->qsum[6 * c + 3] += v[0] * v[1];
                o->qsum[6 * c + 4] += v[0] * v[2];
                o->qsum[6 * c + 5] += v[1] * v[2];
            }
        }
        if (sample) o->msamples++;

        /* 2. momentum exchange on obstacle links: every post-collision
         *    population f*_i that heads into an obstacle cell and the
         *    population returned into the opposite direction hand
         *    c_i (f*_i + f_returned) to the body, 2 c_i f*_i for halfway
         *    bounce-back (walls are not part of the body) */
        if (o->t >= o->force_cap) {
            int64_t cap = o->force_cap * 2;
            while (cap <= o->t) cap *= 2;
            o->force = (double *)realloc(o->force, sizeof(double) * 3 * cap);
            memset(o->force + 3 * o->force_cap, 0, sizeof(double) * 3 * (cap - o->force_cap));
            o->force_cap = cap;
        }
        double fx = 0, fy = 0, fz = 0;
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x) {
                    int64_t c = cell_of(o, x, y, z);
                    if (o->solid[c]) continue;
                    for (int i = 0; i < Q; ++i) {
                        int cx, cy, cz;
                        velocity(i, &cx, &cy, &cz);
                        int xx = x + cx, yy = y + cy, zz = z + cz;
                        if (yy < 0 || yy >= p->ny) { if (p->face_y != FACE_PERIODIC) continue; yy = (yy + p->ny) % p->ny; }
                        if (zz < 0 || zz >= p->nz) { if (p->face_z != FACE_PERIODIC) continue; zz = (zz + p->nz) % p->nz; }
                        if (xx < 0 || xx >= p->nx) {
                            if ((xx < 0 ? p->face_x_lo : p->face_x_hi) != FACE_PERIODIC) continue;
                            xx = (xx + p->nx) % p->nx;
                        }
                        if (!o->solid[cell_of(o, xx, yy, zz)]) continue;
                        double fs = o->post[i * n + c];
                        double back = o->q ? interpolated_bounce_back(o, c, x, y, z, Q - 1 - i) : fs;
                        fx += cx * (fs + back); fy += cy * (fs + back); fz += cz * (fs + back);
                    }
                }
        o->force[3 * o->t + 0] = fx;
        o->force[3 * o->t + 1] = fy;
        o->force[3 * o->t + 2] = fz;

        /* 3a. the outflow condition needs the pre-collision populations of
         *     the outlet plane and of the plane next to it; streaming
         *     overwrites f, so keep copies of both planes */
        const int64_t P = (int64_t)p->ny * p->nz;
        double *fo = NULL, *fi = NULL;
        if (p->face_x_hi == FACE_OUTFLOW) {
            fo = (double *)malloc(sizeof(double) * Q * P);
            fi = (double *)malloc(sizeof(double) * Q * P);
            for (int64_t yz = 0; yz < P; ++yz) {
                const int64_t co = (int64_t)(p->nx - 1) + (int64_t)p->nx * yz;
                /* an obstacle cell (or no cell) next to the outlet: the
                 * outlet cell extrapolates from itself */
                const int64_t ci = (p->nx >= 2 && !o->solid[co - 1]) ? co - 1 : co;
                for (int i = 0; i < Q; ++i) {
                    fo[i * P + yz] = o->f[i * n + co];
                    fi[i * P + yz] = o->f[i * n + ci];
                }
            }
        }

        /* 3. pull streaming with boundary rules: for fluid cell x and
         *    direction i the incoming value comes from x - c_i */
#pragma omp parallel for schedule(static)
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x) {
                    int64_t c = cell_of(o, x, y, z);
                    if (o->solid[c]) continue;
                    for (int i = 0; i < Q; ++i) {
                        int cx, cy, cz;
                        velocity(i, &cx, &cy, &cz);
                        int inv = Q - 1 - i;
                        int64_t src = -1;
                        int kind = classify(o, x - cx, y - cy, z - cz, &src);
                        double v;
                        if (kind == SRC_FLUID) {
                            v = o->post[i * n + src];
                        } else if (kind == SRC_WALL) {
                            /* halfway bounce-back: the population that left
                             * towards the wall comes back reversed; on
                             * obstacle links with wall distances, the
                             * interpolated bounce-back */
                            if (o->q && src >= 0 && o->solid[src])
                                v = interpolated_bounce_back(o, c, x, y, z, i);
                            else
                                v = o->post[inv * n + c];
                        } else if (kind == SRC_INLET) {
                            /* bounce-back from a wall moving with the inlet
                             * velocity (u_in, 0, 0) */
                            v = o->post[inv * n + c] + 6.0 * weight(i) * p->rho_in * (cx * p->u_in);
                        } else if (kind == SRC_OUTFLOW) {
                            /* convective outflow (Geier et al. 2015, App. F):
                             * the missing population is carried out of the
                             * domain at the speed of sound, first-order
                             * upwind in time and space from the pre-collision
                             * values of this cell and of its inner neighbour:
                             * f_i(x_b, t+1) = c_s f_i(x_b - e_x, t)
                             *                 + (1 - c_s) f_i(x_b, t) */
                            const int64_t yz = (int64_t)y + (int64_t)p->ny * z;
                            const double cs = sqrt(1.0 / 3.0);
                            v = cs * fi[i * P + yz] + (1.0 - cs) * fo[i * P + yz];
                        } else {
                            /* pressure outlet: anti-bounce-back against the
                             * even part of the equilibrium at rho_out and the
                             * cell's own velocity (zero-gradient extrapolation) */
                            const double *ub = &o->u[3 * c];
                            double cu = cx * ub[0] + cy * ub[1] + cz * ub[2];
                            double uu = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
                            v = -o->post[inv * n + c]
                              + 2.0 * weight(i) * p->rho_out * (1.0 + 4.5 * cu * cu - 1.5 * uu);
                        }
                        o->f[i * n + c] = v;
                    }
                }
        free(fo);
        free(fi);
        o->t++;
    }
}

/* Totals over fluid cells of the current state: mass and momentum. */
void oracle_lbm_totals(const oracle_lbm *o, double *out4)
{
    double m = 0, jx = 0, jy = 0, jz = 0;
    for (int64_t c = 0; c < o->n; ++c) {
        if (o->solid[c]) continue;
        for (int i = 0; i < Q; ++i) {
            int cx, cy, cz;
            velocity(i, &cx, &cy, &cz);
            double v = o->f[i * o->n + c];
            m += v; jx += cx * v; jy += cy * v; jz += cz * v;
        }
    }
    out4[0] = m; out4[1] = jx; out4[2] = jy; out4[3] = jz;
}

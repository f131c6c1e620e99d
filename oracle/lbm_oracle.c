/*
 * Oracle for the two-component Shan-Chen D3Q19 lattice Boltzmann update of
 * Otomo et al., "Multi-component lattice Boltzmann models for accurate
 * simulation of flows with wide viscosity variation" (arXiv:1711.03254).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, FP64 CPU statement
 * of what the CUDA library computes.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code, header
 * or table with the CUDA path; the GPU library never links it.
 *
 * Every step is written out in the paper's order and notation:
 *   S1 streaming (Eq. 1 / Eq. 9, pull form) with halfway bounce-back as the
 *      voxel-aligned special case of the volumetric no-slip wall (Sec. 2);
 *   S2 moments rho_alpha, rho, j (Eq. 4);
 *   S3 pseudo-potential psi_beta = rho_beta in fluid, rho^s_beta in solid
 *      (Eq. 7, Eq. 11, wall potential definition of Sec. 2);
 *   S4 Shan-Chen force (Eq. 7) + wall force (Eq. 11) + body force;
 *   S5 velocity u_F (Eq. 8), mixture viscosity (Eq. 6, density weighted) and
 *      tau_mix (Eq. 5);
 *   S6 equilibrium (Eq. 3), non-equilibrium momentum flux and its 2nd-order
 *      Hermite regularisation (Eq. 10), forcing term;
 *   S7 collision f* = feq + (1 - 1/tau) f' + F_i (Eq. 9).
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes of the repository):
 *   - D3Q19 weights 1/3, 1/18, 1/36 (the paper only names "isotropic weights").
 *   - The interaction-force stencil of Eq. 7 / Eq. 11 uses 2 w_i (see
 *     force_weight below for why).
 *   - eq_order 0 ("stokes3") is Eq. 3 as printed (no quadratic terms);
 *     eq_order 1 ("full3") adds (c.u)^2/(2T0^2) - u^2/(2T0) (the full form the
 *     paper keeps beside Eq. 3).
 *   - p in Eq. 6 is rho_1/rho (density-weighted viscosity, Sec. 3.2), held in
 *     [0, 1] as Eq. 6 requires (a slightly negative minority density would
 *     otherwise push tau_mix below 1/2 at viscosity ratio 1000).
 *   - Forcing F_i (the paper defers to Li, Luo & Li 2012, a second-order
 *     forcing scheme): Guo-type forcing restated for a regularised collision.
 *     First order: F_i = w_i c_i.F / (2 T0), so that with u_F = u + F/(2 rho)
 *     the momentum gained per step is exactly F.  Second order, in both
 *     equilibrium modes: (1 - 1/(2 tau)) w_i/(2T0^2) (c_i c_i - T0 I):(u_F F + F u_F).
 *     Without it, flow along an interface carries a spurious shear stress
 *     proportional to u . grad(rho) and the layered Poiseuille profiles of
 *     Sec. 3.2 are missed by tens of percent.
 *   - Regularisation: f'_i = w_i/(2 T0^2) (c_i c_i - T0 I) : Pi^neq with
 *     Pi^neq = sum_i c_i c_i (f_i - feq_i) (reg_order 2, the default).
 *     reg_order 3 adds the third-order Hermite terms of the regularised
 *     collision the paper cites (Chen/Zhang 2006): the third-order
 *     non-equilibrium moments follow from Pi^neq and u_F as
 *     a3_abg = u_a Pi_bg + u_b Pi_ag + u_g Pi_ab, and f' is the function in
 *     the span of w_i H_k(c_i) (second- and third-order Hermite polynomials)
 *     whose Hermite moments equal Pi^neq and a3 (see oracle_regularize3).
 *   - rho'_beta of a solid neighbour (Eq. 11).  Wall model 2 (recommended):
 *     rho_beta of the cell itself plus rho^s_beta, so the transition into the
 *     wall is smooth and a uniform fluid next to a wall feels no interaction
 *     force (local momentum conserved).  Wall model 1 ("B", plain):
 *     psi_beta(solid) = rho^s_beta.  Wall model 0 ("A", balanced): B, then the
 *     wall part of the force is projected so that F_w^1 + F_w^2 = 0 in every
 *     cell (forces along walls balanced between components).  Wall model 3
 *     (both statements of the paper): the neutral part of model 2 (the solid
 *     neighbour carries the cell's own rho_beta), and the wall potential's part
 *     G rho_alpha sum_solid ws_i c_i rho^s_beta projected as in model A, so that
 *     the wall's forces on the two components cancel in every cell.
 *   - Surface scattering (the paper defers to another work): a wall returns
 *     the fraction 1 - slip of the particles by bounce-back and reflects the
 *     fraction slip specularly about the voxel wall's plane (specular_source);
 *     slip = 0 (the default) is the no-slip bounce-back.
 *   - rho^s_1 = -rho^s * Theta(-rho^s), rho^s_2 = rho^s * Theta(rho^s).
 *   - INLET cells hold feq(rho_in, u_in) after every step; an OUTLET cell
 *     takes the streamed distributions of its upstream (-x) neighbour.
 *
 * Precision: FP64 throughout, no fused multiply-add contraction (built with
 * -ffp-contract=off).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#define Q 19
#define T0 (1.0 / 3.0)

enum { CELL_FLUID = 0, CELL_SOLID = 1, CELL_INLET = 2, CELL_OUTLET = 3 };

/* D3Q19 velocities: rest, 6 faces, 12 edges. */
static const int C[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double weight_def(int i)
{
    int s = abs(C[i][0]) + abs(C[i][1]) + abs(C[i][2]);
    if (s == 0) return 1.0 / 3.0;
    if (s == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

static int opposite_def(int i)
{
    for (int k = 0; k < Q; ++k)
        if (C[k][0] == -C[i][0] && C[k][1] == -C[i][1] && C[k][2] == -C[i][2]) return k;
    return -1;
}

static double W[Q];
static int OPP[Q];
static int tables_ready = 0;

static void init_tables(void)
{
    if (tables_ready) return;
    for (int i = 0; i < Q; ++i) {
        W[i] = weight_def(i);
        OPP[i] = opposite_def(i);
    }
    tables_ready = 1;
}

static double weight(int i) { return W[i]; }
static int opposite(int i) { return OPP[i]; }

static int direction_of(int cx, int cy, int cz)
{
    for (int k = 0; k < Q; ++k)
        if (C[k][0] == cx && C[k][1] == cy && C[k][2] == cz) return k;
    return -1;
}

/* Weights of the interaction-force stencil (Eq. 7, Eq. 11): twice the D3Q19
 * weights, sum_i ws_i c_i c_i = 2 T0 I (1/9 on faces, 1/18 on edges).  With
 * the bare lattice weights the mixture at total density 1 cannot separate for
 * |G| < 2, yet Sec. 3.1 reports droplets at G = -1.72; the factor 2 reproduces
 * both surface tensions Sec. 3.1 reports (0.071 at G = -1.72, 0.11 at
 * G = -2.2). */
static double force_weight(int i) { return 2.0 * W[i]; }

typedef struct {
    int nx, ny, nz, batch;
    int eq_order;   /* 0 = Eq. 3 as printed, 1 = with quadratic terms */
    int wall_model; /* 0 = balanced (A), 1 = plain (B), 2 = own density + rho^s,
                       3 = own density, wall potential's part balanced */
    int reg_order;  /* 0 or 2 = second-order regularisation, 3 = with third-order terms */
} oracle_config;

typedef struct {
    double tau[2];
    double G;
    double rho_s;
    double g[3];
    double rho_in[2];
    double u_in[3];
    double slip;    /* fraction of the particles a wall reflects specularly (0 = no-slip) */
} oracle_params;

typedef struct oracle_ctx {
    oracle_config cfg;
    oracle_params *par; /* [batch] */
    size_t n;           /* cells per instance */
    uint8_t *type;      /* [batch][n] */
    double *f;          /* [batch][2][Q][n] post-collision distributions */
    double *fs;         /* [2][Q][n] streamed distributions (one instance) */
    double *psi;        /* [2][n] pseudo-potential */
    double *force;      /* [batch][2][n][3] total force per component, last update */
    double *rho;        /* [batch][2][n] macroscopic densities of the last update */
    double *u;          /* [batch][n][3] velocity u_F of the last update */
    double *u_snap;     /* [batch][n][3] velocity at the previous reduction */
    long steps_since_snap;
    long step;
} oracle_ctx;

/* ------------------------------------------------------------------------- */
/* Lattice and per-cell pieces                                               */
/* ------------------------------------------------------------------------- */

void oracle_lattice(int *c, double *w, int *opp)
{
    init_tables();
    for (int i = 0; i < Q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = C[i][a];
        w[i] = weight(i);
        opp[i] = opposite(i);
    }
}

/* Eq. 3: equilibrium of one component with velocity u (u_F after Eq. 8). */
void oracle_feq(double rho_a, const double *u, int eq_order, double *feq)
{
    init_tables();
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; ++i) {
        double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
        double e = 1.0 + cu / T0 + (cu * cu * cu) / (6.0 * T0 * T0 * T0)
                 - cu * uu / (2.0 * T0 * T0);
        if (eq_order == 1) e += (cu * cu) / (2.0 * T0 * T0) - uu / (2.0 * T0);
        feq[i] = rho_a * weight(i) * e;
    }
}

/* Non-equilibrium momentum flux Pi^neq = sum_i c_i c_i (f_i - feq_i), as a
 * full 3x3 matrix (row-major), Eq. 10. */
void oracle_pi_neq(const double *f, const double *feq, double *pi)
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int i = 0; i < Q; ++i) s += C[i][a] * C[i][b] * (f[i] - feq[i]);
            pi[3 * a + b] = s;
        }
}

/* Eq. 10: f'_i = Phi : Pi, 2nd-order Hermite projection
 * f'_i = w_i / (2 T0^2) (c_i c_i - T0 I) : Pi. */
void oracle_regularize(const double *pi, double *fprime)
{
    init_tables();
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double h = C[i][a] * C[i][b] - (a == b ? T0 : 0.0);
                s += h * pi[3 * a + b];
            }
        fprime[i] = weight(i) / (2.0 * T0 * T0) * s;
    }
}

/* Hermite polynomials at velocity i: H2_ab = c_a c_b - T0 d_ab and
 * H3_abg = c_a c_b c_g - T0 (c_a d_bg + c_b d_ag + c_g d_ab). */
static double hermite2(int i, int a, int b)
{
    return C[i][a] * C[i][b] - (a == b ? T0 : 0.0);
}

static double hermite3(int i, int a, int b, int g)
{
    return C[i][a] * C[i][b] * C[i][g]
         - T0 * (C[i][a] * (b == g) + C[i][b] * (a == g) + C[i][g] * (a == b));
}

/* Solve M x = r (n x n, row-major, overwritten) by Gaussian elimination with
 * partial pivoting.  Returns 0, or -1 for a singular matrix. */
static int solve_dense(int n, double *M, double *r, double *x)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (fabs(M[i * n + k]) > fabs(M[p * n + k])) p = i;
        if (M[p * n + k] == 0.0) return -1;
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                double t = M[k * n + j]; M[k * n + j] = M[p * n + j]; M[p * n + j] = t;
            }
            double t = r[k]; r[k] = r[p]; r[p] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            double l = M[i * n + k] / M[k * n + k];
            for (int j = k; j < n; ++j) M[i * n + j] -= l * M[k * n + j];
            r[i] -= l * r[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = r[k];
        for (int j = k + 1; j < n; ++j) s -= M[k * n + j] * x[j];
        x[k] = s / M[k * n + k];
    }
    return 0;
}

/* Eq. 10 with third-order terms.  The target Hermite moments of f' are
 * a2 = Pi^neq and the recursive third-order moments
 * a3_abg = u_a Pi_bg + u_b Pi_ag + u_g Pi_ab.  Of the ten third-order
 * polynomials, H_xxx, H_yyy, H_zzz (c^3 = c on the lattice) and H_xyz (no
 * D3Q19 velocity has three non-zero components) vanish at every velocity;
 * the other six (xxy, yzz, xzz, xyy, yyz, xxz) and the six second-order ones
 * span the basis.  f'_i = w_i sum_k b_k H_k(c_i) with the coefficients b that
 * make sum_i H_m(c_i) f'_i equal the target of every basis polynomial m:
 * M b = a with M_mk = sum_i w_i H_m(c_i) H_k(c_i). */
void oracle_regularize3(const double *pi, const double *u, double *fprime)
{
    enum { NB = 12 };
    static const int I2[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    static const int I3[6][3] = {{0, 0, 1}, {1, 2, 2}, {0, 2, 2}, {0, 1, 1}, {1, 1, 2}, {0, 0, 2}};
    init_tables();
    double H[NB][Q], a[NB], M[NB * NB], b[NB];
    for (int i = 0; i < Q; ++i) {
        for (int k = 0; k < 6; ++k) H[k][i] = hermite2(i, I2[k][0], I2[k][1]);
        for (int k = 0; k < 6; ++k) H[6 + k][i] = hermite3(i, I3[k][0], I3[k][1], I3[k][2]);
    }
    for (int k = 0; k < 6; ++k) a[k] = pi[3 * I2[k][0] + I2[k][1]];
    for (int k = 0; k < 6; ++k) {
        int x = I3[k][0], y = I3[k][1], z = I3[k][2];
        a[6 + k] = u[x] * pi[3 * y + z] + u[y] * pi[3 * x + z] + u[z] * pi[3 * x + y];
    }
    for (int m = 0; m < NB; ++m)
        for (int k = 0; k < NB; ++k) {
            double s = 0.0;
            for (int i = 0; i < Q; ++i) s += weight(i) * H[m][i] * H[k][i];
            M[m * NB + k] = s;
        }
    if (solve_dense(NB, M, a, b) != 0) {
        for (int i = 0; i < Q; ++i) fprime[i] = NAN;
        return;
    }
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int k = 0; k < NB; ++k) s += b[k] * H[k][i];
        fprime[i] = weight(i) * s;
    }
}

/* Forcing term of Eq. 1 / Eq. 9 for one component with force F and
 * velocity u (= u_F), see the reading in the file header. */
void oracle_forcing(const double *F, const double *u, double tau, int eq_order, double *Fi)
{
    (void)eq_order; /* the same forcing serves both equilibria */
    init_tables();
    for (int i = 0; i < Q; ++i) {
        double cF = C[i][0] * F[0] + C[i][1] * F[1] + C[i][2] * F[2];
        double v = weight(i) * cF / (2.0 * T0);
        {
            double s = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double h = C[i][a] * C[i][b] - (a == b ? T0 : 0.0);
                    s += h * (u[a] * F[b] + F[a] * u[b]);
                }
            v += (1.0 - 1.0 / (2.0 * tau)) * weight(i) / (2.0 * T0 * T0) * s;
        }
        Fi[i] = v;
    }
}

/* S5: mixture viscosity (Eq. 6 with p = rho_1/rho) and tau_mix (Eq. 5). */
double oracle_tau_mix(double rho1, double rho2, const double *tau)
{
    double nu1 = T0 * (tau[0] - 0.5);
    double nu2 = T0 * (tau[1] - 0.5);
    double p = rho1 / (rho1 + rho2);
    if (p < 0.0) p = 0.0; /* p ranges over [0, 1] (Eq. 6) */
    if (p > 1.0) p = 1.0;
    double nu_mix = p * nu1 + (1.0 - p) * nu2;
    return nu_mix / T0 + 0.5;
}

/* S2, S5-S7 for one cell.  f: [2][Q] streamed distributions, F: [2][3] total
 * force on each component.  Writes the post-collision distributions fout
 * [2][Q], the velocity u_F [3], the densities rho_out [2] and tau_mix. */
void oracle_collide_cell(const double *f, const double *F, const double *tau, int eq_order, int reg_order,
                         double *fout, double *uF, double *rho_out, double *tau_out)
{
    double rho_a[2], j[3] = {0.0, 0.0, 0.0};
    for (int al = 0; al < 2; ++al) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) s += f[al * Q + i];
        rho_a[al] = s;
        for (int a = 0; a < 3; ++a) {
            double m = 0.0;
            for (int i = 0; i < Q; ++i) m += C[i][a] * f[al * Q + i];
            j[a] += m;
        }
    }
    double rho = rho_a[0] + rho_a[1];
    /* Eq. 8: u_F = u + g/2, g = sum_alpha g_alpha rho_alpha / rho = F_tot / rho */
    for (int a = 0; a < 3; ++a) {
        double u = j[a] / rho;
        double g = (F[a] + F[3 + a]) / rho;
        uF[a] = u + 0.5 * g;
    }
    double tau_mix = oracle_tau_mix(rho_a[0], rho_a[1], tau);
    for (int al = 0; al < 2; ++al) {
        double feq[Q], pi[9], fp[Q], Fi[Q];
        oracle_feq(rho_a[al], uF, eq_order, feq);
        oracle_pi_neq(f + al * Q, feq, pi);
        if (reg_order == 3)
            oracle_regularize3(pi, uF, fp);
        else
            oracle_regularize(pi, fp);
        oracle_forcing(F + 3 * al, uF, tau_mix, eq_order, Fi);
        for (int i = 0; i < Q; ++i)
            fout[al * Q + i] = feq[i] + (1.0 - 1.0 / tau_mix) * fp[i] + Fi[i];
    }
    rho_out[0] = rho_a[0];
    rho_out[1] = rho_a[1];
    *tau_out = tau_mix;
}

/* Wall potential of the two components from the single parameter rho^s
 * (definition kept beside Eq. 11; rho_0 = 1). */
void oracle_wall_potential(double rho_s, double *rs)
{
    rs[0] = rho_s < 0.0 ? -rho_s : 0.0;
    rs[1] = rho_s > 0.0 ? rho_s : 0.0;
}

/* ------------------------------------------------------------------------- */
/* Domain                                                                    */
/* ------------------------------------------------------------------------- */

static size_t cell_index(const oracle_config *cfg, int x, int y, int z)
{
    return (size_t)x + (size_t)cfg->nx * ((size_t)y + (size_t)cfg->ny * (size_t)z);
}

static int wrap(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

int oracle_create(const oracle_config *cfg, const oracle_params *par, oracle_ctx **out)
{
    init_tables();
    if (!cfg || !par || !out) return 1;
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1 || cfg->batch < 1) return 1;
    for (int b = 0; b < cfg->batch; ++b)
        if (!(par[b].tau[0] > 0.5) || !(par[b].tau[1] > 0.5) || !(par[b].slip >= 0.0 && par[b].slip <= 1.0))
            return 1;
    oracle_ctx *ctx = (oracle_ctx *)calloc(1, sizeof(oracle_ctx));
    ctx->cfg = *cfg;
    ctx->n = (size_t)cfg->nx * cfg->ny * cfg->nz;
    size_t B = (size_t)cfg->batch, n = ctx->n;
    ctx->par = (oracle_params *)malloc(B * sizeof(oracle_params));
    memcpy(ctx->par, par, B * sizeof(oracle_params));
    ctx->type = (uint8_t *)calloc(B * n, 1);
    ctx->f = (double *)calloc(B * 2 * Q * n, sizeof(double));
    ctx->fs = (double *)calloc(2 * Q * n, sizeof(double));
    ctx->psi = (double *)calloc(2 * n, sizeof(double));
    ctx->force = (double *)calloc(B * 2 * n * 3, sizeof(double));
    ctx->rho = (double *)calloc(B * 2 * n, sizeof(double));
    ctx->u = (double *)calloc(B * n * 3, sizeof(double));
    ctx->u_snap = (double *)calloc(B * n * 3, sizeof(double));
    *out = ctx;
    return 0;
}

void oracle_destroy(oracle_ctx *ctx)
{
    if (!ctx) return;
    free(ctx->par); free(ctx->type); free(ctx->f); free(ctx->fs); free(ctx->psi);
    free(ctx->force); free(ctx->rho); free(ctx->u); free(ctx->u_snap);
    free(ctx);
}

int oracle_set_geometry(oracle_ctx *ctx, const uint8_t *type)
{
    size_t tot = (size_t)ctx->cfg.batch * ctx->n;
    for (size_t k = 0; k < tot; ++k)
        if (type[k] > CELL_OUTLET) return 1;
    memcpy(ctx->type, type, tot);
    return 0;
}

/* Initialisation: f = feq(rho_alpha, u) in every non-solid cell (no force
 * correction at t = 0); INLET cells take feq(rho_in, u_in). */
int oracle_set_fields(oracle_ctx *ctx, const double *rho1, const double *rho2, const double *u)
{
    size_t n = ctx->n;
    for (int b = 0; b < ctx->cfg.batch; ++b) {
        const oracle_params *p = &ctx->par[b];
        for (size_t k = 0; k < n; ++k) {
            size_t gk = (size_t)b * n + k;
            uint8_t t = ctx->type[gk];
            double r[2] = {rho1[gk], rho2[gk]};
            double v[3] = {u[3 * gk], u[3 * gk + 1], u[3 * gk + 2]};
            if (t == CELL_SOLID) {
                r[0] = r[1] = 0.0;
                v[0] = v[1] = v[2] = 0.0;
            } else if (t == CELL_INLET) {
                r[0] = p->rho_in[0]; r[1] = p->rho_in[1];
                v[0] = p->u_in[0]; v[1] = p->u_in[1]; v[2] = p->u_in[2];
            }
            for (int al = 0; al < 2; ++al) {
                double feq[Q];
                oracle_feq(r[al], v, ctx->cfg.eq_order, feq);
                for (int i = 0; i < Q; ++i)
                    ctx->f[(((size_t)b * 2 + al) * Q + i) * n + k] = t == CELL_SOLID ? 0.0 : feq[i];
                ctx->rho[((size_t)b * 2 + al) * n + k] = r[al];
            }
            for (int a = 0; a < 3; ++a) {
                ctx->u[3 * gk + a] = v[a];
                ctx->u_snap[3 * gk + a] = v[a];
            }
        }
    }
    ctx->steps_since_snap = 0;
    return 0;
}

/* Specular reflection at a voxel wall (the partial-slip reading of the
 * surface scattering model, Sec. 2).  The value arriving at (x, y, z) in
 * direction i comes from the SOLID cell x - c_i.  For an edge direction with
 * non-zero components along axes a and b: if the face neighbour x - c_ia e_a
 * is not SOLID and x - c_ib e_b is, the wall's normal is e_b and the particle
 * came from x - c_ia e_a moving with c_i's b-component reversed (and the same
 * with a and b exchanged).  Writes that cell and direction and returns 1.
 * Face directions (normal incidence) and corners (both face neighbours SOLID,
 * or neither) return 0: they bounce back.  The pairing is mutual: the cell
 * found here reflects the value of direction opp(i) of (x, y, z) the same way,
 * so a blend of bounce-back and reflection conserves mass. */
static int specular_source(const oracle_config *cfg, const uint8_t *type, int x, int y, int z, int i,
                           size_t *s, int *j)
{
    int ax[2], na = 0;
    for (int a = 0; a < 3; ++a)
        if (C[i][a] != 0) ax[na++] = a;
    if (na != 2) return 0;
    int pos[3] = {x, y, z}, dim[3] = {cfg->nx, cfg->ny, cfg->nz};
    int solid[2];
    size_t face[2];
    for (int m = 0; m < 2; ++m) {
        int q[3] = {pos[0], pos[1], pos[2]};
        q[ax[m]] = wrap(q[ax[m]] - C[i][ax[m]], dim[ax[m]]);
        face[m] = cell_index(cfg, q[0], q[1], q[2]);
        solid[m] = type[face[m]] == CELL_SOLID;
    }
    if (solid[0] == solid[1]) return 0;
    int keep = solid[0] ? 1 : 0; /* the open face: the particle moved along its axis */
    int flip = 1 - keep;         /* the wall's normal axis */
    int c[3] = {C[i][0], C[i][1], C[i][2]};
    c[ax[flip]] = -c[ax[flip]];
    *s = face[keep];
    *j = direction_of(c[0], c[1], c[2]);
    return 1;
}

/* One update of instance b. */
static void step_instance(oracle_ctx *ctx, int b)
{
    const oracle_config *cfg = &ctx->cfg;
    const oracle_params *p = &ctx->par[b];
    const int nx = cfg->nx, ny = cfg->ny, nz = cfg->nz;
    const size_t n = ctx->n;
    const uint8_t *type = ctx->type + (size_t)b * n;
    const double *f = ctx->f + (size_t)b * 2 * Q * n;
    double *force = ctx->force + (size_t)b * 2 * n * 3;
    double rs[2];
    oracle_wall_potential(p->rho_s, rs);

    /* S1: pull streaming; a link from a solid cell is bounced back, or, for
     * the fraction p->slip, reflected specularly (see specular_source). */
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t k = cell_index(cfg, x, y, z);
                if (type[k] == CELL_SOLID) continue;
                for (int al = 0; al < 2; ++al)
                    for (int i = 0; i < Q; ++i) {
                        size_t src = cell_index(cfg, wrap(x - C[i][0], nx), wrap(y - C[i][1], ny),
                                                wrap(z - C[i][2], nz));
                        double v;
                        if (type[src] == CELL_SOLID) {
                            v = f[((size_t)al * Q + opposite(i)) * n + k];
                            size_t s;
                            int j;
                            if (p->slip != 0.0 && specular_source(cfg, type, x, y, z, i, &s, &j))
                                v = (1.0 - p->slip) * v + p->slip * f[((size_t)al * Q + j) * n + s];
                        } else {
                            v = f[((size_t)al * Q + i) * n + src];
                        }
                        ctx->fs[((size_t)al * Q + i) * n + k] = v;
                    }
            }
    /* OUTLET: zero-gradient copy of the upstream neighbour's streamed values. */
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t k = cell_index(cfg, x, y, z);
                if (type[k] != CELL_OUTLET) continue;
                size_t up = cell_index(cfg, wrap(x - 1, nx), y, z);
                if (type[up] == CELL_SOLID || type[up] == CELL_OUTLET) continue;
                for (int al = 0; al < 2; ++al)
                    for (int i = 0; i < Q; ++i)
                        ctx->fs[((size_t)al * Q + i) * n + k] = ctx->fs[((size_t)al * Q + i) * n + up];
            }

    /* S2/S3: densities and pseudo-potential. */
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t k = cell_index(cfg, x, y, z);
                for (int al = 0; al < 2; ++al) {
                    double v;
                    if (type[k] == CELL_SOLID) {
                        v = rs[al];
                    } else if (type[k] == CELL_INLET) {
                        v = p->rho_in[al];
                    } else {
                        v = 0.0;
                        for (int i = 0; i < Q; ++i) v += ctx->fs[((size_t)al * Q + i) * n + k];
                    }
                    ctx->psi[(size_t)al * n + k] = v;
                }
            }

    /* S4: Shan-Chen force (Eq. 7), wall force (Eq. 11), body force. */
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t k = cell_index(cfg, x, y, z);
                if (type[k] == CELL_SOLID || type[k] == CELL_INLET) continue;
                double rho_a[2] = {ctx->psi[k], ctx->psi[n + k]};
                double rho = rho_a[0] + rho_a[1];
                double Fb[2][3], Fw[2][3], Fs[2][3];
                for (int al = 0; al < 2; ++al) {
                    int be = 1 - al;
                    double sb[3] = {0.0, 0.0, 0.0}, sw[3] = {0.0, 0.0, 0.0}, ss[3] = {0.0, 0.0, 0.0};
                    for (int i = 1; i < Q; ++i) {
                        size_t nb = cell_index(cfg, wrap(x + C[i][0], nx), wrap(y + C[i][1], ny),
                                               wrap(z + C[i][2], nz));
                        double ps = ctx->psi[(size_t)be * n + nb];
                        /* wall model 2: the solid neighbour carries the fluid
                         * density of this cell plus the wall potential; wall
                         * model 3: the fluid density here, the wall potential
                         * in the separate sum ss */
                        if (type[nb] == CELL_SOLID && cfg->wall_model == 2) ps = rho_a[be] + rs[be];
                        if (type[nb] == CELL_SOLID && cfg->wall_model == 3) ps = rho_a[be];
                        for (int a = 0; a < 3; ++a) {
                            if (type[nb] == CELL_SOLID) {
                                sw[a] += force_weight(i) * C[i][a] * ps;
                                ss[a] += force_weight(i) * C[i][a] * rs[be];
                            } else {
                                sb[a] += force_weight(i) * C[i][a] * ps;
                            }
                        }
                    }
                    for (int a = 0; a < 3; ++a) {
                        Fb[al][a] = p->G * rho_a[al] * sb[a];
                        Fw[al][a] = p->G * rho_a[al] * sw[a];
                        Fs[al][a] = p->G * rho_a[al] * ss[a];
                    }
                }
                if (cfg->wall_model == 0) {
                    for (int a = 0; a < 3; ++a) {
                        double net = Fw[0][a] + Fw[1][a];
                        Fw[0][a] -= rho_a[0] / rho * net;
                        Fw[1][a] -= rho_a[1] / rho * net;
                    }
                }
                if (cfg->wall_model == 3) {
                    /* the wall potential's part, balanced between components */
                    for (int a = 0; a < 3; ++a) {
                        double net = Fs[0][a] + Fs[1][a];
                        Fw[0][a] += Fs[0][a] - rho_a[0] / rho * net;
                        Fw[1][a] += Fs[1][a] - rho_a[1] / rho * net;
                    }
                }
                for (int al = 0; al < 2; ++al)
                    for (int a = 0; a < 3; ++a)
                        force[((size_t)al * n + k) * 3 + a] =
                            Fb[al][a] + Fw[al][a] + rho_a[al] * p->g[a];
            }

    /* S5-S7: collision into the post-collision state. */
    double *fo = ctx->f + (size_t)b * 2 * Q * n;
    double *rho_o = ctx->rho + (size_t)b * 2 * n;
    double *u_o = ctx->u + (size_t)b * n * 3;
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t k = cell_index(cfg, x, y, z);
                if (type[k] == CELL_SOLID) {
                    rho_o[k] = rho_o[n + k] = 0.0;
                    u_o[3 * k] = u_o[3 * k + 1] = u_o[3 * k + 2] = 0.0;
                    continue;
                }
                if (type[k] == CELL_INLET) {
                    for (int al = 0; al < 2; ++al) {
                        double feq[Q];
                        oracle_feq(p->rho_in[al], p->u_in, cfg->eq_order, feq);
                        for (int i = 0; i < Q; ++i) fo[((size_t)al * Q + i) * n + k] = feq[i];
                        rho_o[(size_t)al * n + k] = p->rho_in[al];
                    }
                    for (int a = 0; a < 3; ++a) u_o[3 * k + a] = p->u_in[a];
                    continue;
                }
                double fl[2 * Q], F[6], out[2 * Q], uF[3], r[2], tm;
                for (int al = 0; al < 2; ++al) {
                    for (int i = 0; i < Q; ++i) fl[al * Q + i] = ctx->fs[((size_t)al * Q + i) * n + k];
                    for (int a = 0; a < 3; ++a) F[3 * al + a] = force[((size_t)al * n + k) * 3 + a];
                }
                oracle_collide_cell(fl, F, p->tau, cfg->eq_order, cfg->reg_order, out, uF, r, &tm);
                for (int al = 0; al < 2; ++al) {
                    for (int i = 0; i < Q; ++i) fo[((size_t)al * Q + i) * n + k] = out[al * Q + i];
                    rho_o[(size_t)al * n + k] = r[al];
                }
                for (int a = 0; a < 3; ++a) u_o[3 * k + a] = uF[a];
            }
}

int oracle_step(oracle_ctx *ctx, int nsteps)
{
    if (nsteps < 0) return 1;
    for (int s = 0; s < nsteps; ++s) {
        for (int b = 0; b < ctx->cfg.batch; ++b) step_instance(ctx, b);
        ctx->step++;
        ctx->steps_since_snap++;
    }
    return 0;
}

int oracle_get_fields(const oracle_ctx *ctx, double *rho1, double *rho2, double *u)
{
    size_t n = ctx->n;
    for (int b = 0; b < ctx->cfg.batch; ++b)
        for (size_t k = 0; k < n; ++k) {
            size_t gk = (size_t)b * n + k;
            if (rho1) rho1[gk] = ctx->rho[((size_t)b * 2) * n + k];
            if (rho2) rho2[gk] = ctx->rho[((size_t)b * 2 + 1) * n + k];
            if (u)
                for (int a = 0; a < 3; ++a) u[3 * gk + a] = ctx->u[3 * gk + a];
        }
    return 0;
}

/* Post-collision distributions of instance b, component al, direction i. */
int oracle_get_f(const oracle_ctx *ctx, double *out)
{
    memcpy(out, ctx->f, (size_t)ctx->cfg.batch * 2 * Q * ctx->n * sizeof(double));
    return 0;
}

int oracle_set_f(oracle_ctx *ctx, const double *in)
{
    memcpy(ctx->f, in, (size_t)ctx->cfg.batch * 2 * Q * ctx->n * sizeof(double));
    return 0;
}

/* Per instance: M1, M2, Px, Py, Pz (momentum rho u_F), residual, max |u_F|.
 * Sums over non-solid cells in cell order.  residual =
 * |u - u_snap|_2 / (k |u|_2 + 1e-30) with k the updates since the previous
 * reduction (0 when k = 0); the snapshot is then replaced by u. */
int oracle_reduce(oracle_ctx *ctx, double *out)
{
    size_t n = ctx->n;
    long k = ctx->steps_since_snap;
    for (int b = 0; b < ctx->cfg.batch; ++b) {
        double m1 = 0, m2 = 0, px = 0, py = 0, pz = 0, d2 = 0, u2 = 0, umax = 0;
        for (size_t c = 0; c < n; ++c) {
            size_t gk = (size_t)b * n + c;
            if (ctx->type[gk] == CELL_SOLID) continue;
            double r1 = ctx->rho[((size_t)b * 2) * n + c];
            double r2 = ctx->rho[((size_t)b * 2 + 1) * n + c];
            const double *u = ctx->u + 3 * gk;
            const double *us = ctx->u_snap + 3 * gk;
            m1 += r1;
            m2 += r2;
            px += (r1 + r2) * u[0];
            py += (r1 + r2) * u[1];
            pz += (r1 + r2) * u[2];
            double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            u2 += uu;
            for (int a = 0; a < 3; ++a) d2 += (u[a] - us[a]) * (u[a] - us[a]);
            double um = sqrt(uu);
            if (um > umax || um != um) umax = um;
        }
        double *o = out + 7 * b;
        o[0] = m1; o[1] = m2; o[2] = px; o[3] = py; o[4] = pz;
        o[5] = k > 0 ? sqrt(d2) / ((double)k * sqrt(u2) + 1e-30) : 0.0;
        o[6] = umax;
    }
    memcpy(ctx->u_snap, ctx->u, (size_t)ctx->cfg.batch * n * 3 * sizeof(double));
    ctx->steps_since_snap = 0;
    return 0;
}

/* Total force F^alpha [batch][2][n][3] of the last update (zero in SOLID and
 * INLET cells). */
int oracle_get_force(const oracle_ctx *ctx, double *out)
{
    memcpy(out, ctx->force, (size_t)ctx->cfg.batch * 2 * ctx->n * 3 * sizeof(double));
    return 0;
}

long oracle_step_count(const oracle_ctx *ctx) { return ctx->step; }

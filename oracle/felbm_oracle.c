/*
 * felbm_oracle.c -- plain FP64 CPU oracle of the finite-element lattice
 * Boltzmann method for binary fluids (Lee-Lin free-energy model, D2Q9, P1
 * triangles).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or constant with the CUDA library; it is written to be
 * checked against the paper by eye, not to be fast: element loops, plain
 * arrays, one thread, no blocking or fusion.
 *
 * Sections and equations followed (Matin, Misztal, Hernandez-Garcia,
 * Mathiesen, "Evaluation of the Finite Element Lattice Boltzmann Method for
 * Binary Fluid Flows"):
 *   Sec. 2.1  Eqs. lbmf/lbmg (trapezoidal LBE), Eq. omega (BGK), Eq. F,
 *             Eq. G, Eqs. f_eq/g_eq, the beta/kappa relations, the bulk
 *             chemical potential and the harmonic relaxation-time mixing.
 *   Sec. 2.2  pre-streaming collision, streaming, post-streaming collision,
 *             exact-difference body force, moment Eqs. velocity/pressure.
 *   Sec. 2.2.1 Taylor expansion (Eq. local_formulation), P1 Bubnov-Galerkin
 *             form (Eqs. discrete_field, galerkin_lbm, fem_matrices) with the
 *             lumped mass matrix.
 *   Sec. 2.3  element gradients and volume-weighted nodal recovery.
 *
 * Readings where the paper is silent or 3-D specific (restated in 2-D):
 *   - D2Q9 replaces D3Q19; P1 triangles replace tetrahedra.
 *   - f of the paper is called h here (zeroth moment rho).
 *   - The Laplacian of rho is the recovery operator applied to the recovered
 *     gradient (divergence of the P1 interpolant of the nodal gradient,
 *     averaged like a gradient); the alternative lumped weak Laplacian is
 *     selectable (laplacian = 1).
 *   - The stress term d_i(d_k rho d_k rho) - d_j(d_i rho d_j rho) is formed
 *     from nodal products of the recovered gradient, whose gradients are
 *     recovered by the same operator.
 *   - C is clamped to [0, 1] inside the relaxation-time formula only.
 *   - Exact-difference body force: prefactor 1/2 and du = g dt (the printed
 *     dt/2 at dt = 1), so that its first moment is the dt/2 rho g term of the
 *     velocity moment for any dt.
 *   - Walls: a node tagged k in 1..8 has inward normal e_k; after streaming
 *     every population with e_a . e_k > 0 is replaced by its opposite.
 *   - Weak-form boundary terms are dropped (exact on periodic meshes).
 *   - Initial state: the post-collision distribution is the equilibrium of
 *     (rho0, u0, p0); the stored pre-collided value is eq + source.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- D2Q9 lattice (Sec. 2.1, restated for two dimensions) -------------- */
#define Q 9
static const double ORC_EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const double ORC_EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double ORC_W[Q] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                                1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const int ORC_OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double CS2 = 1.0 / 3.0; /* c_s = 1/sqrt(3) */

/* ---- problem description passed from Python ---------------------------- */
typedef struct {
    int64_t n_nodes, n_tri;
    const int32_t *tri;   /* 3T, CCW */
    const double *area;   /* T      : |T| */
    const double *dNdx;   /* 3T     : d N_a / dx on T for its vertex a */
    const double *dNdy;   /* 3T */
    const double *mass;   /* N      : lumped mass m_i = sum_{T∋i} |T|/3 */
    const uint8_t *tag;   /* N or NULL : 0 fluid, k=1..8 wall, inward normal e_k */
    double rho_l, rho_v, sigma, xi, tau_l, tau_v, dt, grav_x, grav_y;
    int32_t laplacian;    /* 0: recovery of the recovered gradient, 1: lumped weak form */
    int32_t pad;
} orc_problem;

static double orc_wrap(double d, double L) {
    if (L > 0.0) d -= L * nearbyint(d / L);
    return d;
}

/* Per-triangle area and shape-function gradients, lumped mass (Sec. 2.2.1,
 * Eq. discrete_field; "lumped-mass approximation" of M).  Coordinates of the
 * second and third vertex are taken relative to the first with the minimum
 * image of the periodic box.  Returns the index+1 of the first triangle with
 * non-positive area, 0 on success. */
int64_t orc_geometry(int64_t n_nodes, int64_t n_tri, const double *xy, const int32_t *tri,
                     const double *box, double *area, double *dNdx, double *dNdy,
                     double *mass) {
    for (int64_t i = 0; i < n_nodes; ++i) mass[i] = 0.0;
    for (int64_t t = 0; t < n_tri; ++t) {
        int32_t a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
        double xb = orc_wrap(xy[2 * b] - xy[2 * a], box[0]);
        double yb = orc_wrap(xy[2 * b + 1] - xy[2 * a + 1], box[1]);
        double xc = orc_wrap(xy[2 * c] - xy[2 * a], box[0]);
        double yc = orc_wrap(xy[2 * c + 1] - xy[2 * a + 1], box[1]);
        double xa = 0.0, ya = 0.0;
        double twoA = (xb - xa) * (yc - ya) - (xc - xa) * (yb - ya);
        if (!(twoA > 0.0)) return t + 1;
        /* N_a = ((x_b y_c - x_c y_b) + (y_b - y_c) x + (x_c - x_b) y) / 2|T|, cyclic */
        dNdx[3 * t + 0] = (yb - yc) / twoA;
        dNdy[3 * t + 0] = (xc - xb) / twoA;
        dNdx[3 * t + 1] = (yc - ya) / twoA;
        dNdy[3 * t + 1] = (xa - xc) / twoA;
        dNdx[3 * t + 2] = (ya - yb) / twoA;
        dNdy[3 * t + 2] = (xb - xa) / twoA;
        area[t] = 0.5 * twoA;
        mass[a] += area[t] / 3.0;
        mass[b] += area[t] / 3.0;
        mass[c] += area[t] / 3.0;
    }
    return 0;
}

/* FE streaming of one population with velocity e = (ex, ey) (Eq.
 * galerkin_lbm with the lumped M):
 *   psi_out = psi_in - M_L^{-1} (dt C_e + dt^2 D_e) psi_in,
 *   (C_e psi)_i = sum_{T∋i} |T|/3 * e.grad(psi)_T           (int N_i e.grad N^T)
 *   (D_e psi)_i = 1/2 sum_{T∋i} |T| (e.grad N_i)(e.grad psi)_T  (Eq. fem_matrices) */
void orc_stream(const orc_problem *P, double ex, double ey, const double *in, double *out) {
    int64_t N = P->n_nodes;
    double *Cpsi = (double *)calloc((size_t)N, sizeof(double));
    double *Dpsi = (double *)calloc((size_t)N, sizeof(double));
    for (int64_t t = 0; t < P->n_tri; ++t) {
        double egrad = 0.0; /* e . grad psi on T */
        for (int b = 0; b < 3; ++b) {
            int32_t vb = P->tri[3 * t + b];
            egrad += (ex * P->dNdx[3 * t + b] + ey * P->dNdy[3 * t + b]) * in[vb];
        }
        for (int a = 0; a < 3; ++a) {
            int32_t va = P->tri[3 * t + a];
            double egNa = ex * P->dNdx[3 * t + a] + ey * P->dNdy[3 * t + a];
            Cpsi[va] += P->area[t] / 3.0 * egrad;
            Dpsi[va] += 0.5 * P->area[t] * egNa * egrad;
        }
    }
    double dt = P->dt;
    for (int64_t i = 0; i < N; ++i)
        out[i] = in[i] + (-dt * Cpsi[i] - dt * dt * Dpsi[i]) / P->mass[i];
    free(Cpsi);
    free(Dpsi);
}

/* Element gradient of the P1 interpolant and volume(area)-weighted nodal
 * average (Sec. 2.3). */
void orc_recover(const orc_problem *P, const double *f, double *gx, double *gy) {
    int64_t N = P->n_nodes;
    double *vol = (double *)calloc((size_t)N, sizeof(double));
    for (int64_t i = 0; i < N; ++i) gx[i] = gy[i] = 0.0;
    for (int64_t t = 0; t < P->n_tri; ++t) {
        double tx = 0.0, ty = 0.0;
        for (int b = 0; b < 3; ++b) {
            int32_t vb = P->tri[3 * t + b];
            tx += P->dNdx[3 * t + b] * f[vb];
            ty += P->dNdy[3 * t + b] * f[vb];
        }
        for (int a = 0; a < 3; ++a) {
            int32_t va = P->tri[3 * t + a];
            gx[va] += P->area[t] * tx;
            gy[va] += P->area[t] * ty;
            vol[va] += P->area[t];
        }
    }
    for (int64_t i = 0; i < N; ++i) {
        gx[i] /= vol[i];
        gy[i] /= vol[i];
    }
    free(vol);
}

/* Alternative Laplacian reading: lumped weak form
 *   L_i = -(1/m_i) sum_{T∋i} |T| grad N_i . grad rho_T. */
static void orc_weak_laplacian(const orc_problem *P, const double *f, double *L) {
    int64_t N = P->n_nodes;
    for (int64_t i = 0; i < N; ++i) L[i] = 0.0;
    for (int64_t t = 0; t < P->n_tri; ++t) {
        double tx = 0.0, ty = 0.0;
        for (int b = 0; b < 3; ++b) {
            int32_t vb = P->tri[3 * t + b];
            tx += P->dNdx[3 * t + b] * f[vb];
            ty += P->dNdy[3 * t + b] * f[vb];
        }
        for (int a = 0; a < 3; ++a) {
            int32_t va = P->tri[3 * t + a];
            L[va] -= P->area[t] * (P->dNdx[3 * t + a] * tx + P->dNdy[3 * t + a] * ty);
        }
    }
    for (int64_t i = 0; i < N; ++i) L[i] /= P->mass[i];
}

/* beta and kappa from sigma and xi (Sec. 2.1), with the density jump
 * rho_l - rho_v. */
static double orc_beta(const orc_problem *P) {
    double d = P->rho_l - P->rho_v;
    return 12.0 * P->sigma / (P->xi * d * d * d * d);
}
static double orc_kappa(const orc_problem *P) {
    double d = P->rho_l - P->rho_v;
    return 1.5 * P->xi * P->sigma / (d * d);
}

/* Bulk chemical potential mu_phi (Sec. 2.1). */
static double orc_mu_bulk(const orc_problem *P, double rho) {
    return 4.0 * orc_beta(P) * (rho - P->rho_v) * (rho - P->rho_l) *
           (rho - 0.5 * (P->rho_v + P->rho_l));
}

/* Gamma_a(u) = f_eq / rho (Eq. f_eq). */
static double orc_gamma(int a, double ux, double uy) {
    double eu = ORC_EX[a] * ux + ORC_EY[a] * uy;
    double uu = ux * ux + uy * uy;
    return ORC_W[a] * (1.0 + eu / CS2 + (eu * eu - CS2 * uu) / (2.0 * CS2 * CS2));
}

/* g_eq (Eq. g_eq). */
static double orc_geq(int a, double rho, double p, double ux, double uy) {
    return ORC_W[a] * p / CS2 + rho * (orc_gamma(a, ux, uy) - ORC_W[a]);
}

/* Local collision terms of one node: equilibria and the sources
 * F (Eq. F), G (Eq. G) and the exact-difference body force B.
 *   in: rho, p, u, grad rho, grad mu (mu = mu_phi - kappa lap rho),
 *       K = kappa [d_i(d_k rho d_k rho) - d_j(d_i rho d_j rho)]. */
void orc_local_terms(const orc_problem *P, double rho, double p, double ux, double uy,
                     double drx, double dry, double dmx, double dmy, double Kx, double Ky,
                     double *heq, double *geq, double *F, double *G, double *B) {
    double dt = P->dt;
    for (int a = 0; a < Q; ++a) {
        double ga = orc_gamma(a, ux, uy);
        double emx = ORC_EX[a] - ux, emy = ORC_EY[a] - uy;
        heq[a] = rho * ga;
        geq[a] = orc_geq(a, rho, p, ux, uy);
        /* F = dt/2 (e-u).[c_s^2 grad rho - rho grad mu] / c_s^2 Gamma(u) */
        F[a] = 0.5 * dt * (emx * (drx * CS2 - rho * dmx) + emy * (dry * CS2 - rho * dmy)) / CS2 * ga;
        /* G = dt/2 (e-u).grad rho c_s^2 / c_s^2 [Gamma(u) - Gamma(0)]
         *   + dt/2 (e-u).K / c_s^2 Gamma(u) */
        G[a] = 0.5 * dt * (emx * drx * CS2 + emy * dry * CS2) / CS2 * (ga - orc_gamma(a, 0.0, 0.0)) +
               0.5 * dt * (emx * Kx + emy * Ky) / CS2 * ga;
        /* exact-difference body force, du = g dt */
        B[a] = 0.5 * (orc_geq(a, rho, p, ux + P->grav_x * dt, uy + P->grav_y * dt) -
                      orc_geq(a, rho, p, ux, uy));
    }
}

/* Non-local fields of one time level, all from rho (Secs. 2.1, 2.3). */
typedef struct {
    double *drx, *dry;     /* recovered grad rho */
    double *lap;           /* Laplacian of rho */
    double *Kx, *Ky;       /* kappa [d_i(|grad rho|^2) - d_j(d_i rho d_j rho)] */
    double *mu;            /* mu_phi - kappa lap rho */
    double *dmx, *dmy;     /* recovered grad mu */
} orc_fields;

static void orc_fields_alloc(orc_fields *S, int64_t N) {
    double **p[] = {&S->drx, &S->dry, &S->lap, &S->Kx, &S->Ky, &S->mu, &S->dmx, &S->dmy};
    for (size_t k = 0; k < sizeof(p) / sizeof(p[0]); ++k)
        *p[k] = (double *)calloc((size_t)N, sizeof(double));
}
static void orc_fields_free(orc_fields *S) {
    free(S->drx); free(S->dry); free(S->lap); free(S->Kx); free(S->Ky);
    free(S->mu); free(S->dmx); free(S->dmy);
}

static void orc_compute_fields(const orc_problem *P, const double *rho, orc_fields *S) {
    int64_t N = P->n_nodes;
    double kappa = orc_kappa(P);
    orc_recover(P, rho, S->drx, S->dry);
    double *t1x = (double *)malloc((size_t)N * sizeof(double));
    double *t1y = (double *)malloc((size_t)N * sizeof(double));
    double *t2x = (double *)malloc((size_t)N * sizeof(double));
    double *t2y = (double *)malloc((size_t)N * sizeof(double));
    double *prod = (double *)malloc((size_t)N * sizeof(double));
    /* Laplacian */
    if (P->laplacian == 0) {
        orc_recover(P, S->drx, t1x, t1y);
        orc_recover(P, S->dry, t2x, t2y);
        for (int64_t i = 0; i < N; ++i) S->lap[i] = t1x[i] + t2y[i];
    } else {
        orc_weak_laplacian(P, rho, S->lap);
    }
    /* stress term: products of the nodal gradient, then their recovered derivatives */
    for (int64_t i = 0; i < N; ++i) S->Kx[i] = S->Ky[i] = 0.0;
    /* d_i (d_k rho d_k rho) */
    for (int64_t i = 0; i < N; ++i) prod[i] = S->drx[i] * S->drx[i] + S->dry[i] * S->dry[i];
    orc_recover(P, prod, t1x, t1y);
    for (int64_t i = 0; i < N; ++i) { S->Kx[i] += t1x[i]; S->Ky[i] += t1y[i]; }
    /* - d_j (d_x rho d_j rho): j = x uses (d_x rho)^2, j = y uses d_x rho d_y rho */
    for (int64_t i = 0; i < N; ++i) prod[i] = S->drx[i] * S->drx[i];
    orc_recover(P, prod, t1x, t1y);
    for (int64_t i = 0; i < N; ++i) S->Kx[i] -= t1x[i];
    for (int64_t i = 0; i < N; ++i) prod[i] = S->drx[i] * S->dry[i];
    orc_recover(P, prod, t1x, t1y);
    for (int64_t i = 0; i < N; ++i) { S->Kx[i] -= t1y[i]; S->Ky[i] -= t1x[i]; }
    /* - d_j (d_y rho d_j rho), j = y */
    for (int64_t i = 0; i < N; ++i) prod[i] = S->dry[i] * S->dry[i];
    orc_recover(P, prod, t1x, t1y);
    for (int64_t i = 0; i < N; ++i) S->Ky[i] -= t1y[i];
    for (int64_t i = 0; i < N; ++i) { S->Kx[i] *= kappa; S->Ky[i] *= kappa; }
    /* chemical potential and its gradient */
    for (int64_t i = 0; i < N; ++i) S->mu[i] = orc_mu_bulk(P, rho[i]) - kappa * S->lap[i];
    orc_recover(P, S->mu, S->dmx, S->dmy);
    free(t1x); free(t1y); free(t2x); free(t2y); free(prod);
}

/* 1/tau = C/tau_l + (1-C)/tau_v, C = (rho - rho_v)/(rho_l - rho_v) clamped. */
static double orc_tau(const orc_problem *P, double rho) {
    double C = (rho - P->rho_v) / (P->rho_l - P->rho_v);
    if (C < 0.0) C = 0.0;
    if (C > 1.0) C = 1.0;
    return 1.0 / (C / P->tau_l + (1.0 - C) / P->tau_v);
}

/* Initial pre-collided state: psi = psi_eq(rho0, u0, p0), psibar = psi + (-Omega + S)
 * with Omega(psi_eq) = 0. */
void orc_init(const orc_problem *P, const double *rho0, const double *ux0, const double *uy0,
              const double *p0, double *hbar, double *gbar) {
    int64_t N = P->n_nodes;
    orc_fields S;
    orc_fields_alloc(&S, N);
    orc_compute_fields(P, rho0, &S);
    double heq[Q], geq[Q], F[Q], G[Q], B[Q];
    for (int64_t i = 0; i < N; ++i) {
        orc_local_terms(P, rho0[i], p0[i], ux0[i], uy0[i], S.drx[i], S.dry[i], S.dmx[i],
                        S.dmy[i], S.Kx[i], S.Ky[i], heq, geq, F, G, B);
        for (int a = 0; a < Q; ++a) {
            hbar[a * N + i] = heq[a] + F[a];
            gbar[a * N + i] = geq[a] + G[a] + B[a];
        }
    }
    orc_fields_free(&S);
}

/* n_steps full time steps on the stored pre-collided distributions
 * (hbar, gbar: SoA, population-major, 9N each), in place.  The moments
 * rho, u, p of the last step (computed from the streamed distributions,
 * Eqs. velocity/pressure) are written to rho, ux, uy, p when non-NULL. */
void orc_step(const orc_problem *P, double *hbar, double *gbar, int64_t n_steps, double *rho_out,
              double *ux_out, double *uy_out, double *p_out) {
    int64_t N = P->n_nodes;
    double dt = P->dt;
    double *hs = (double *)malloc((size_t)(Q * N) * sizeof(double));
    double *gs = (double *)malloc((size_t)(Q * N) * sizeof(double));
    double *rho = (double *)malloc((size_t)N * sizeof(double));
    orc_fields S;
    orc_fields_alloc(&S, N);
    for (int64_t step = 0; step < n_steps; ++step) {
        /* streaming: psibar(x + e dt, t + dt) = psibar(x, t), Taylor-Galerkin form */
        for (int a = 0; a < Q; ++a) {
            orc_stream(P, ORC_EX[a], ORC_EY[a], hbar + a * N, hs + a * N);
            orc_stream(P, ORC_EX[a], ORC_EY[a], gbar + a * N, gs + a * N);
        }
        /* no-slip walls: bounce-back of the populations entering the fluid */
        if (P->tag) {
            for (int64_t i = 0; i < N; ++i) {
                int k = P->tag[i];
                if (k == 0) continue;
                for (int a = 1; a < Q; ++a) {
                    if (ORC_EX[a] * ORC_EX[k] + ORC_EY[a] * ORC_EY[k] > 0.0) {
                        hs[a * N + i] = hs[ORC_OPP[a] * N + i];
                        gs[a * N + i] = gs[ORC_OPP[a] * N + i];
                    }
                }
            }
        }
        /* rho = sum_a h_a of the streamed distribution */
        for (int64_t i = 0; i < N; ++i) {
            double r = 0.0;
            for (int a = 0; a < Q; ++a) r += hs[a * N + i];
            rho[i] = r;
        }
        orc_compute_fields(P, rho, &S);
        double heq[Q], geq[Q], F[Q], G[Q], B[Q];
        for (int64_t i = 0; i < N; ++i) {
            /* rho u = sum e g + dt/2 K + dt/2 rho g  (Eq. velocity) */
            double mx = 0.0, my = 0.0, sg = 0.0;
            for (int a = 0; a < Q; ++a) {
                mx += ORC_EX[a] * gs[a * N + i];
                my += ORC_EY[a] * gs[a * N + i];
                sg += gs[a * N + i];
            }
            double r = rho[i];
            double ux = (mx + 0.5 * dt * S.Kx[i] + 0.5 * dt * r * P->grav_x) / r;
            double uy = (my + 0.5 * dt * S.Ky[i] + 0.5 * dt * r * P->grav_y) / r;
            /* p = c_s^2 sum g + dt/2 u.grad rho c_s^2  (Eq. pressure) */
            double p = CS2 * sg + 0.5 * dt * (ux * S.drx[i] + uy * S.dry[i]) * CS2;
            double tau = orc_tau(P, r);
            orc_local_terms(P, r, p, ux, uy, S.drx[i], S.dry[i], S.dmx[i], S.dmy[i], S.Kx[i],
                            S.Ky[i], heq, geq, F, G, B);
            double post = 2.0 * tau / (2.0 * tau + 1.0);
            for (int a = 0; a < Q; ++a) {
                /* post-streaming collision (Eqs. lbmf_post, lbmg_post), Omega on the
                 * streamed value */
                double h = hs[a * N + i] + post * (-(hs[a * N + i] - heq[a]) / (2.0 * tau) + F[a]);
                double g = gs[a * N + i] +
                           post * (-(gs[a * N + i] - geq[a]) / (2.0 * tau) + G[a] + B[a]);
                /* pre-streaming collision of the next step (Eqs. lbmf_pre, lbmg_pre) */
                hbar[a * N + i] = h + (-(h - heq[a]) / (2.0 * tau) + F[a]);
                gbar[a * N + i] = g + (-(g - geq[a]) / (2.0 * tau) + G[a] + B[a]);
            }
            if (step == n_steps - 1) {
                if (rho_out) rho_out[i] = r;
                if (ux_out) ux_out[i] = ux;
                if (uy_out) uy_out[i] = uy;
                if (p_out) p_out[i] = p;
            }
        }
    }
    orc_fields_free(&S);
    free(hs);
    free(gs);
    free(rho);
}

/* Non-local fields of a given density field, exported for tests. */
void orc_fields_of(const orc_problem *P, const double *rho, double *drx, double *dry,
                   double *lap, double *Kx, double *Ky, double *mu, double *dmx, double *dmy) {
    int64_t N = P->n_nodes;
    orc_fields S;
    orc_fields_alloc(&S, N);
    orc_compute_fields(P, rho, &S);
    memcpy(drx, S.drx, (size_t)N * sizeof(double));
    memcpy(dry, S.dry, (size_t)N * sizeof(double));
    memcpy(lap, S.lap, (size_t)N * sizeof(double));
    memcpy(Kx, S.Kx, (size_t)N * sizeof(double));
    memcpy(Ky, S.Ky, (size_t)N * sizeof(double));
    memcpy(mu, S.mu, (size_t)N * sizeof(double));
    memcpy(dmx, S.dmx, (size_t)N * sizeof(double));
    memcpy(dmy, S.dmy, (size_t)N * sizeof(double));
    orc_fields_free(&S);
}

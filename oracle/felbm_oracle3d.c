/*
 * felbm_oracle3d.c -- plain FP64 CPU oracle of the finite-element lattice
 * Boltzmann method for binary fluids in three dimensions (Lee-Lin
 * free-energy model, D3Q19, P1 tetrahedra): the paper's own setting.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or constant with the CUDA library; it is written to be
 * checked against the paper by eye: element loops, plain arrays, one thread.
 *
 * Sections and equations followed (Matin, Misztal, Hernandez-Garcia,
 * Mathiesen, "Evaluation of the Finite Element Lattice Boltzmann Method for
 * Binary Fluid Flows"):
 *   Sec. 2.1  trapezoidal LBE for f and g (D3Q19 velocities and weights),
 *             BGK collision, forcing terms F and G, equilibria, beta and
 *             kappa from sigma and xi, the bulk chemical potential and the
 *             harmonic relaxation-time mixing.
 *   Sec. 2.2  pre-streaming collision, streaming, post-streaming collision,
 *             exact-difference body force, the velocity and pressure moments.
 *   Sec. 2.2.1 Taylor expansion and the P1 Bubnov-Galerkin form on linear
 *             tetrahedra (Eqs. discrete_field, galerkin_lbm, fem_matrices)
 *             with the lumped mass matrix.
 *   Sec. 2.3  element gradients and volume-weighted nodal recovery.
 *
 * Readings where the paper is silent (the same as the two-dimensional
 * oracle, felbm_oracle.c):
 *   - f of the paper is called h here (zeroth moment rho).
 *   - The Laplacian of rho is the recovery operator applied to the recovered
 *     gradient; the stress term d_i(d_k rho d_k rho) - d_j(d_i rho d_j rho)
 *     is formed from nodal products of the recovered gradient, whose
 *     gradients are recovered by the same operator.
 *   - C is clamped to [0, 1] inside the relaxation-time formula only.
 *   - Exact-difference body force with du = g dt.
 *   - Walls: a node tagged k in 1..18 has inward normal e_k; after streaming
 *     every population with e_a . e_k > 0 is replaced by its opposite.
 *   - Weak-form boundary terms are dropped (exact on periodic meshes).
 *   - Initial state: the stored pre-collided value is eq + source.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- D3Q19 lattice (Sec. 2.1): rest, 6 axis and 12 edge directions,
 * ordered so that direction 2k-1 and 2k are opposite ----------------------- */
#define Q3 19
static const double E3X[Q3] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const double E3Y[Q3] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const double E3Z[Q3] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const double W3[Q3] = {1.0 / 3,  1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const double CS2 = 1.0 / 3.0;

static int opp3(int a) { return a == 0 ? 0 : (a % 2 ? a + 1 : a - 1); }

/* ---- problem description passed from Python ---------------------------- */
typedef struct {
    int64_t n_nodes, n_tet;
    const int32_t *tet;   /* 4T, positive orientation */
    const double *vol;    /* T      : |T| */
    const double *dN;     /* 12T    : d N_a / d(x, y, z) of vertex a on T, [t][a][3] */
    const double *mass;   /* N      : lumped mass m_i = sum_{T∋i} |T|/4 */
    const uint8_t *tag;   /* N or NULL : 0 fluid, k = 1..18 wall, inward normal e_k */
    double rho_l, rho_v, sigma, xi, tau_l, tau_v, dt, grav[3];
} orc3_problem;

static double wrap3(double d, double L) {
    if (L > 0.0) d -= L * nearbyint(d / L);
    return d;
}

/* Per-tetrahedron volume and shape-function gradients, lumped mass (Sec.
 * 2.2.1).  Vertices b, c, d are taken relative to a with the minimum image
 * of the periodic box.  grad N of the four vertices from the inverse of the
 * edge matrix J = [b - a; c - a; d - a]: grad N_b, grad N_c, grad N_d are the
 * columns of J^{-1}, grad N_a = -(their sum).  Returns index+1 of the first
 * tetrahedron with non-positive volume, 0 on success. */
int64_t orc3_geometry(int64_t n_nodes, int64_t n_tet, const double *xyz, const int32_t *tet,
                      const double *box, double *vol, double *dN, double *mass) {
    for (int64_t i = 0; i < n_nodes; ++i) mass[i] = 0.0;
    for (int64_t t = 0; t < n_tet; ++t) {
        const int32_t *v = tet + 4 * t;
        double J[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                J[r][c] = wrap3(xyz[3 * v[r + 1] + c] - xyz[3 * v[0] + c], box[c]);
        double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        if (!(det > 0.0)) return t + 1;
        /* inverse by cofactors: Jinv[c][r] = cof(J)[r][c] / det */
        double inv[3][3];
        inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
        inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
        inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
        inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
        /* N_{b+1}(x) = row b of J^{-T} (x - x_a): grad N_{b+1} = column b of J^{-1},
         * i.e. (inv[0][b], inv[1][b], inv[2][b]) */
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int b = 0; b < 3; ++b) {
                dN[12 * t + 3 * (b + 1) + c] = inv[c][b];
                s += inv[c][b];
            }
            dN[12 * t + c] = -s;
        }
        vol[t] = det / 6.0;
        for (int a = 0; a < 4; ++a) mass[v[a]] += vol[t] / 4.0;
    }
    return 0;
}

/* FE streaming of one population with velocity e (Eq. galerkin_lbm with the
 * lumped M, Eq. fem_matrices):
 *   (C_e psi)_i = sum_{T∋i} |T|/4 * e.grad(psi)_T
 *   (D_e psi)_i = 1/2 sum_{T∋i} |T| (e.grad N_i)(e.grad psi)_T
 *   psi_out = psi_in - (dt C_e psi + dt^2 D_e psi) / m_i */
void orc3_stream(const orc3_problem *P, double ex, double ey, double ez, const double *in,
                 double *out) {
    int64_t N = P->n_nodes;
    double *Cpsi = (double *)calloc((size_t)N, sizeof(double));
    double *Dpsi = (double *)calloc((size_t)N, sizeof(double));
    for (int64_t t = 0; t < P->n_tet; ++t) {
        const double *g = P->dN + 12 * t;
        double egrad = 0.0;
        for (int b = 0; b < 4; ++b)
            egrad += (ex * g[3 * b] + ey * g[3 * b + 1] + ez * g[3 * b + 2]) * in[P->tet[4 * t + b]];
        for (int a = 0; a < 4; ++a) {
            int32_t va = P->tet[4 * t + a];
            double egNa = ex * g[3 * a] + ey * g[3 * a + 1] + ez * g[3 * a + 2];
            Cpsi[va] += P->vol[t] / 4.0 * egrad;
            Dpsi[va] += 0.5 * P->vol[t] * egNa * egrad;
        }
    }
    double dt = P->dt;
    for (int64_t i = 0; i < N; ++i) out[i] = in[i] + (-dt * Cpsi[i] - dt * dt * Dpsi[i]) / P->mass[i];
    free(Cpsi);
    free(Dpsi);
}

/* Element gradient of the P1 interpolant, volume-weighted nodal average
 * (Sec. 2.3).  g: 3N, [i][3]. */
void orc3_recover(const orc3_problem *P, const double *f, double *g) {
    int64_t N = P->n_nodes;
    double *vsum = (double *)calloc((size_t)N, sizeof(double));
    for (int64_t i = 0; i < 3 * N; ++i) g[i] = 0.0;
    for (int64_t t = 0; t < P->n_tet; ++t) {
        const double *d = P->dN + 12 * t;
        double tg[3] = {0.0, 0.0, 0.0};
        for (int b = 0; b < 4; ++b)
            for (int c = 0; c < 3; ++c) tg[c] += d[3 * b + c] * f[P->tet[4 * t + b]];
        for (int a = 0; a < 4; ++a) {
            int32_t va = P->tet[4 * t + a];
            for (int c = 0; c < 3; ++c) g[3 * va + c] += P->vol[t] * tg[c];
            vsum[va] += P->vol[t];
        }
    }
    for (int64_t i = 0; i < N; ++i)
        for (int c = 0; c < 3; ++c) g[3 * i + c] /= vsum[i];
    free(vsum);
}

static double beta3(const orc3_problem *P) {
    double d = P->rho_l - P->rho_v;
    return 12.0 * P->sigma / (P->xi * d * d * d * d);
}
static double kappa3(const orc3_problem *P) {
    double d = P->rho_l - P->rho_v;
    return 1.5 * P->xi * P->sigma / (d * d);
}
static double mu_bulk3(const orc3_problem *P, double rho) {
    return 4.0 * beta3(P) * (rho - P->rho_v) * (rho - P->rho_l) * (rho - 0.5 * (P->rho_v + P->rho_l));
}

/* Gamma_a(u) = f_eq / rho (Eq. f_eq). */
static double gamma3(int a, const double *u) {
    double eu = E3X[a] * u[0] + E3Y[a] * u[1] + E3Z[a] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return W3[a] * (1.0 + eu / CS2 + (eu * eu - CS2 * uu) / (2.0 * CS2 * CS2));
}

/* g_eq (Eq. g_eq). */
static double geq3(int a, double rho, double p, const double *u) {
    return W3[a] * p / CS2 + rho * (gamma3(a, u) - W3[a]);
}

/* Local collision terms of one node: equilibria, F (Eq. F), G (Eq. G) and the
 * exact-difference body force B; dr = grad rho, dm = grad mu, K = stress
 * force (3 components each). */
void orc3_local_terms(const orc3_problem *P, double rho, double p, const double *u, const double *dr,
                      const double *dm, const double *K, double *heq, double *geq, double *F,
                      double *G, double *B) {
    double dt = P->dt;
    double zero[3] = {0.0, 0.0, 0.0};
    double uplus[3] = {u[0] + P->grav[0] * dt, u[1] + P->grav[1] * dt, u[2] + P->grav[2] * dt};
    for (int a = 0; a < Q3; ++a) {
        double e[3] = {E3X[a], E3Y[a], E3Z[a]};
        double ga = gamma3(a, u);
        double X = 0.0, D = 0.0, KK = 0.0;
        for (int c = 0; c < 3; ++c) {
            double em = e[c] - u[c];
            X += em * (dr[c] * CS2 - rho * dm[c]);
            D += em * dr[c] * CS2;
            KK += em * K[c];
        }
        heq[a] = rho * ga;
        geq[a] = geq3(a, rho, p, u);
        F[a] = 0.5 * dt * X / CS2 * ga;
        G[a] = 0.5 * dt * D / CS2 * (ga - gamma3(a, zero)) + 0.5 * dt * KK / CS2 * ga;
        B[a] = 0.5 * (geq3(a, rho, p, uplus) - geq3(a, rho, p, u));
    }
}

/* Non-local fields of one time level, all from rho (Secs. 2.1, 2.3);
 * vectors are [i][3]. */
typedef struct {
    double *dr;   /* recovered grad rho */
    double *lap;  /* Laplacian of rho */
    double *K;    /* kappa [d_i(|grad rho|^2) - d_j(d_i rho d_j rho)] */
    double *mu;   /* mu_phi - kappa lap rho */
    double *dm;   /* recovered grad mu */
} orc3_fields;

static void fields3_alloc(orc3_fields *S, int64_t N) {
    S->dr = (double *)calloc((size_t)(3 * N), sizeof(double));
    S->lap = (double *)calloc((size_t)N, sizeof(double));
    S->K = (double *)calloc((size_t)(3 * N), sizeof(double));
    S->mu = (double *)calloc((size_t)N, sizeof(double));
    S->dm = (double *)calloc((size_t)(3 * N), sizeof(double));
}
static void fields3_free(orc3_fields *S) {
    free(S->dr); free(S->lap); free(S->K); free(S->mu); free(S->dm);
}

static void compute_fields3(const orc3_problem *P, const double *rho, orc3_fields *S) {
    int64_t N = P->n_nodes;
    double kappa = kappa3(P);
    orc3_recover(P, rho, S->dr);
    double *comp = (double *)malloc((size_t)N * sizeof(double));
    double *g = (double *)malloc((size_t)(3 * N) * sizeof(double));
    /* Laplacian: sum over c of d_c of the recovered d_c rho */
    for (int64_t i = 0; i < N; ++i) S->lap[i] = 0.0;
    for (int c = 0; c < 3; ++c) {
        for (int64_t i = 0; i < N; ++i) comp[i] = S->dr[3 * i + c];
        orc3_recover(P, comp, g);
        for (int64_t i = 0; i < N; ++i) S->lap[i] += g[3 * i + c];
    }
    /* stress term: + d_i |grad rho|^2 */
    for (int64_t i = 0; i < 3 * N; ++i) S->K[i] = 0.0;
    for (int64_t i = 0; i < N; ++i)
        comp[i] = S->dr[3 * i] * S->dr[3 * i] + S->dr[3 * i + 1] * S->dr[3 * i + 1] +
                  S->dr[3 * i + 2] * S->dr[3 * i + 2];
    orc3_recover(P, comp, g);
    for (int64_t i = 0; i < 3 * N; ++i) S->K[i] += g[i];
    /* - d_j (d_i rho d_j rho) for every component i, summed over j */
    for (int ci = 0; ci < 3; ++ci)
        for (int cj = 0; cj < 3; ++cj) {
            for (int64_t i = 0; i < N; ++i) comp[i] = S->dr[3 * i + ci] * S->dr[3 * i + cj];
            orc3_recover(P, comp, g);
            for (int64_t i = 0; i < N; ++i) S->K[3 * i + ci] -= g[3 * i + cj];
        }
    for (int64_t i = 0; i < 3 * N; ++i) S->K[i] *= kappa;
    for (int64_t i = 0; i < N; ++i) S->mu[i] = mu_bulk3(P, rho[i]) - kappa * S->lap[i];
    orc3_recover(P, S->mu, S->dm);
    free(comp);
    free(g);
}

static double tau3(const orc3_problem *P, double rho) {
    double C = (rho - P->rho_v) / (P->rho_l - P->rho_v);
    if (C < 0.0) C = 0.0;
    if (C > 1.0) C = 1.0;
    return 1.0 / (C / P->tau_l + (1.0 - C) / P->tau_v);
}

/* Initial pre-collided state (eq + source of rho0, u0, p0); u0: [i][3]. */
void orc3_init(const orc3_problem *P, const double *rho0, const double *u0, const double *p0,
               double *hbar, double *gbar) {
    int64_t N = P->n_nodes;
    orc3_fields S;
    fields3_alloc(&S, N);
    compute_fields3(P, rho0, &S);
    double heq[Q3], geq[Q3], F[Q3], G[Q3], B[Q3];
    for (int64_t i = 0; i < N; ++i) {
        orc3_local_terms(P, rho0[i], p0[i], u0 + 3 * i, S.dr + 3 * i, S.dm + 3 * i, S.K + 3 * i,
                         heq, geq, F, G, B);
        for (int a = 0; a < Q3; ++a) {
            hbar[a * N + i] = heq[a] + F[a];
            gbar[a * N + i] = geq[a] + G[a] + B[a];
        }
    }
    fields3_free(&S);
}

/* n_steps time steps on the pre-collided distributions (19N each,
 * population-major), in place; the last step's moments to rho, u ([i][3]),
 * p when non-NULL. */
void orc3_step(const orc3_problem *P, double *hbar, double *gbar, int64_t n_steps, double *rho_out,
               double *u_out, double *p_out) {
    int64_t N = P->n_nodes;
    double dt = P->dt;
    double *hs = (double *)malloc((size_t)(Q3 * N) * sizeof(double));
    double *gs = (double *)malloc((size_t)(Q3 * N) * sizeof(double));
    double *rho = (double *)malloc((size_t)N * sizeof(double));
    orc3_fields S;
    fields3_alloc(&S, N);
    for (int64_t step = 0; step < n_steps; ++step) {
        for (int a = 0; a < Q3; ++a) {
            orc3_stream(P, E3X[a], E3Y[a], E3Z[a], hbar + a * N, hs + a * N);
            orc3_stream(P, E3X[a], E3Y[a], E3Z[a], gbar + a * N, gs + a * N);
        }
        if (P->tag) {
            for (int64_t i = 0; i < N; ++i) {
                int k = P->tag[i];
                if (k == 0) continue;
                for (int a = 1; a < Q3; ++a)
                    if (E3X[a] * E3X[k] + E3Y[a] * E3Y[k] + E3Z[a] * E3Z[k] > 0.0) {
                        hs[a * N + i] = hs[opp3(a) * N + i];
                        gs[a * N + i] = gs[opp3(a) * N + i];
                    }
            }
        }
        for (int64_t i = 0; i < N; ++i) {
            double r = 0.0;
            for (int a = 0; a < Q3; ++a) r += hs[a * N + i];
            rho[i] = r;
        }
        compute_fields3(P, rho, &S);
        double heq[Q3], geq[Q3], F[Q3], G[Q3], B[Q3];
        for (int64_t i = 0; i < N; ++i) {
            /* rho u = sum e g + dt/2 K + dt/2 rho g  (Eq. velocity) */
            double m[3] = {0.0, 0.0, 0.0}, sg = 0.0;
            for (int a = 0; a < Q3; ++a) {
                m[0] += E3X[a] * gs[a * N + i];
                m[1] += E3Y[a] * gs[a * N + i];
                m[2] += E3Z[a] * gs[a * N + i];
                sg += gs[a * N + i];
            }
            double r = rho[i], u[3], ud = 0.0;
            for (int c = 0; c < 3; ++c) {
                u[c] = (m[c] + 0.5 * dt * S.K[3 * i + c] + 0.5 * dt * r * P->grav[c]) / r;
                ud += u[c] * S.dr[3 * i + c];
            }
            /* p = c_s^2 sum g + dt/2 u.grad rho c_s^2  (Eq. pressure) */
            double p = CS2 * sg + 0.5 * dt * ud * CS2;
            double tau = tau3(P, r);
            orc3_local_terms(P, r, p, u, S.dr + 3 * i, S.dm + 3 * i, S.K + 3 * i, heq, geq, F, G, B);
            double post = 2.0 * tau / (2.0 * tau + 1.0);
            for (int a = 0; a < Q3; ++a) {
                double h = hs[a * N + i] + post * (-(hs[a * N + i] - heq[a]) / (2.0 * tau) + F[a]);
                double g = gs[a * N + i] + post * (-(gs[a * N + i] - geq[a]) / (2.0 * tau) + G[a] + B[a]);
                hbar[a * N + i] = h + (-(h - heq[a]) / (2.0 * tau) + F[a]);
                gbar[a * N + i] = g + (-(g - geq[a]) / (2.0 * tau) + G[a] + B[a]);
            }
            if (step == n_steps - 1) {
                if (rho_out) rho_out[i] = r;
                if (u_out)
                    for (int c = 0; c < 3; ++c) u_out[3 * i + c] = u[c];
                if (p_out) p_out[i] = p;
            }
        }
    }
    fields3_free(&S);
    free(hs);
    free(gs);
    free(rho);
}

/* Non-local fields of a given density, exported for tests; vectors [i][3]. */
void orc3_fields_of(const orc3_problem *P, const double *rho, double *dr, double *lap, double *K,
                    double *mu, double *dm) {
    int64_t N = P->n_nodes;
    orc3_fields S;
    fields3_alloc(&S, N);
    compute_fields3(P, rho, &S);
    memcpy(dr, S.dr, (size_t)(3 * N) * sizeof(double));
    memcpy(lap, S.lap, (size_t)N * sizeof(double));
    memcpy(K, S.K, (size_t)(3 * N) * sizeof(double));
    memcpy(mu, S.mu, (size_t)N * sizeof(double));
    memcpy(dm, S.dm, (size_t)(3 * N) * sizeof(double));
    fields3_free(&S);
}

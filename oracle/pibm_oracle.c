/*
 * pibm_oracle.c -- plain FP64 single-threaded CPU oracle of the thermal
 * LBM-PIBM-DEM lattice step (Zhang et al., arXiv 1502.01159).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline leg of the benchmark, never by the product path.  It shares no
 * code with the CUDA library.  Every step is written out in the order the
 * paper applies it, with plain loops and no blocking, fusion or reordering:
 *
 *   state at time t : f_a(r,t), g_a(r,t) before collision (after streaming),
 *                     particles X, U, omega, T_p at t, and the coupling of
 *                     time t (F_B, Q_B on the lattice; F, torque, H per particle)
 *   one step        : 1. collide f and g with the forcing of time t and stream
 *                        (Eqs lbm2, lbm2.5, lbm3, lbm3.5, lbm9, lbm12.5)
 *                     2. DEM: n_sub substeps of the particle equations of
 *                        motion with the hydrodynamic force of time t frozen
 *                        (Eq demgov, Hertz / Mindlin-Deresiewicz contact law)
 *                     3. thermosensitive particles: C_p dT_p/dt = -H_p
 *                     4. PIBM coupling of time t+1 from the new state
 *                        (Eqs lbm5-lbm13, lbm11, lbm12, lbm12.6)
 *
 * Readings of passages the paper leaves silent, ambiguous or garbled:
 *   - thermal lattice D2Q5 / D3Q7 with the linear equilibrium
 *     g_eq = w T (1 + e.u / cs_T^2), tau_g = alpha / cs_T^2 + 1/2;
 *   - macroscopic temperature T = sum g + Q_B / 2 (zeroth moment);
 *   - buoyancy force (U_c^2 / L_c)(T - T_ref) along -gravity, added to F_B;
 *   - Eq lbm8 read as the change of each population, which with Eq lbm7
 *     gives F_f = 2 (rho_l U_l - j_l); Eq lbm7.5 likewise gives
 *     Q_l = 2 kappa_T (T_p - T_l);
 *   - a resolved particle (d >> h) is the set of nodes it covers, each a PIBM
 *     point of area eps = clamp(R + 1/2 - |r - X|, 0, 1), a node belonging to
 *     the particle with the largest eps (ties: lower index);
 *   - off-node static markers (the concentric cylinder of the cavity case)
 *     use 4-point Lagrange interpolation (Eq lbm6 with i_max = 4) and the
 *     4-point cosine kernel (Eqs lbm11, lbm12);
 *   - particle equation of motion m dU/dt = m (1 - rho_f/rho_p) g + F_fpi
 *     + sum F_c, integrated with velocity Verlet in n_sub substeps;
 *   - tangential contact: incremental spring with k_t = 8 G* r_a (theta_k = 1,
 *     Mindlin-Deresiewicz loading branch), Coulomb cap mu |F_n|;
 *   - walls: halfway bounce-back for f, anti-bounce-back for g at isothermal
 *     walls, bounce-back for g at adiabatic walls.
 *
 * Compile with -ffp-contract=off so that the cell and contact decisions are
 * taken with the exact IEEE operation sequence written here.
 */
#include "pibm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- tables */
static const int E2[9][3] = {{0, 0, 0},  {1, 0, 0},  {0, 1, 0},  {-1, 0, 0}, {0, -1, 0},
                             {1, 1, 0},  {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
static const double W2Q9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                               1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const double W2Q5[5] = {1.0 / 3, 1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6};
static const int E3[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                              {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                              {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                              {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double W3Q19[19] = {1.0 / 3,  1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
                                 1.0 / 18, 1.0 / 18, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                                 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                                 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const double W3Q7[7] = {1.0 / 4, 1.0 / 8, 1.0 / 8, 1.0 / 8, 1.0 / 8, 1.0 / 8, 1.0 / 8};
/* D3Q15 (Section 2.1): rest, six axis links, eight cube diagonals; c_s^2 = 1/3 */
static const int E15[15][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
                               {0, 0, 1},  {0, 0, -1},  {1, 1, 1},   {-1, -1, -1}, {1, 1, -1},
                               {-1, -1, 1}, {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1},  {1, -1, -1}};
static const double W3Q15[15] = {2.0 / 9,  1.0 / 9,  1.0 / 9,  1.0 / 9,  1.0 / 9,
                                 1.0 / 9,  1.0 / 9,  1.0 / 72, 1.0 / 72, 1.0 / 72,
                                 1.0 / 72, 1.0 / 72, 1.0 / 72, 1.0 / 72, 1.0 / 72};

static const double PI = 3.14159265358979323846;

/* ---------------------------------------------------------------- state */
/* Mindlin-Deresiewicz loading history of one contact (law ORC_HERTZ_MD_HIST):
 * e the contact's reference tangential direction (set at its first tangential
 * displacement, carried in the tangent plane), k the branch (0 loading,
 * 1 unloading, 2 reloading), Ts / Tss the tangential force along e at the
 * last unloading / reloading turning point, Fn_prev the normal force of the
 * previous update. */
typedef struct {
    double e[3];
    double Ts, Tss, Fn_prev;
    int k;
} md_state;

typedef struct {
    int i, j;
    double ft[3];
    md_state md;
} contact;

struct orc_sim {
    orc_params P;
    int D, Q, QG;
    const int (*e)[3];
    const double* w;
    const double* wg;
    double csT2;
    int n[3];
    long N;
    double nu, alpha, tau_f, tau_g, buoy;
    int wall[6], therm[6];
    double Tw[6];
    double *f, *g, *fpost, *gpost;
    double *FB, *QB;
    /* particles */
    int np;
    double *X, *U, *W, *R, *rho, *Tp, *Cp, *m, *I;
    unsigned char* fixed;
    double *Fh, *Th, *Hh, *Fc, *Tc;
    double *Fp, *Tq, *Hp; /* coupling of the previous time (force, torque, heat) */
    int have_prev;
    double *J, *U0, *W0;  /* optional hydrodynamic Jacobian [np][18] and the velocities at the step start */
    int point;            /* particle model: 1 = one PIBM point per particle, d_p <= h (the paper's own regime) */
    double* wall_ft; /* [np][6][3] */
    md_state* wall_md; /* [np][6] loading history of the wall contacts */
    contact* cont;
    int ncont;
    /* static off-node markers */
    int nm;
    double *MX, *MA, *MT;
    double nu_sum;
    /* contact law */
    int law;
    double E, pois, mu, kn, kt, gn, gt;
    long t;
};

static long nidx(const orc_sim* s, int x, int y, int z) { return ((long)z * s->n[1] + y) * s->n[0] + x; }

static int opposite(const orc_sim* s, int i, int q) {
    for (int k = 0; k < q; k++)
        if (s->e[k][0] == -s->e[i][0] && s->e[k][1] == -s->e[i][1] && s->e[k][2] == -s->e[i][2]) return k;
    return -1;
}

static int axis_periodic(const orc_sim* s, int a) { return s->wall[2 * a] == ORC_PERIODIC; }

/* ------------------------------------------------------- relaxation times */
/* Eq lbm2.6: tau_f = sqrt(Pr) L_c u_c / (sqrt(Ra) cs^2 dt) + 1/2, i.e. nu = U_c L_c sqrt(Pr/Ra).
 * Eq lbm2.7 with Pr = nu/alpha: alpha = nu / Pr, and tau_g = alpha / cs_T^2 + 1/2 on D2Q5/D3Q7. */
static void relaxation(orc_sim* s) {
    s->nu = s->P.U_c * s->P.L_c * sqrt(s->P.Pr / s->P.Ra);
    s->alpha = s->nu / s->P.Pr;
    s->tau_f = 3.0 * s->nu + 0.5;
    s->tau_g = s->alpha / s->csT2 + 0.5;
    /* u_c = sqrt(g beta L_c dT) (text after Eq lbm2.7): g beta dT = U_c^2 / L_c per unit temperature */
    s->buoy = s->P.U_c * s->P.U_c / s->P.L_c;
}

/* ------------------------------------------------------------- equilibria */
/* Eq lbm3 */
static double feq(const orc_sim* s, int i, double rho, const double u[3]) {
    double eu = s->e[i][0] * u[0] + s->e[i][1] * u[1] + s->e[i][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return s->w[i] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
}

/* Eq lbm3.5, linear form on D2Q5/D3Q7 */
static double geq(const orc_sim* s, int k, double T, const double u[3]) {
    double eu = s->e[k][0] * u[0] + s->e[k][1] * u[1] + s->e[k][2] * u[2];
    return s->wg[k] * T * (1.0 + eu / s->csT2);
}

/* Eq lbm12: cosine regularised delta function */
double orc_delta_h(double a) {
    if (fabs(a) <= 2.0) return 0.25 * (1.0 + cos(PI * a / 2.0));
    return 0.0;
}

/* Eq lbm6: 1-D Lagrange weights on the npts nodes floor(x)-npts/2+1 ... */
int orc_lagrange_weights(double x, int npts, double* w) {
    int base = (int)floor(x) - npts / 2 + 1;
    for (int k = 0; k < npts; k++) {
        double xk = base + k, L = 1.0;
        for (int m = 0; m < npts; m++) {
            if (m == k) continue;
            double xm = base + m;
            L *= (x - xm) / (xk - xm);
        }
        w[k] = L;
    }
    return base;
}

/* --------------------------------------------------------------- moments */
static void moments(const orc_sim* s, long r, double* rho, double j[3], double* T0) {
    *rho = 0.0;
    j[0] = j[1] = j[2] = 0.0;
    for (int i = 0; i < s->Q; i++) {
        double fi = s->f[(long)i * s->N + r];
        *rho += fi;
        j[0] += s->e[i][0] * fi;
        j[1] += s->e[i][1] * fi;
        j[2] += s->e[i][2] * fi;
    }
    *T0 = 0.0;
    for (int k = 0; k < s->QG; k++) *T0 += s->g[(long)k * s->N + r];
}

/* total force and macroscopic u, T at a node (text after Eq lbm3.5, readings above) */
static void macro(const orc_sim* s, long r, double* rho, double u[3], double* T, double F[3]) {
    double j[3], T0;
    moments(s, r, rho, j, &T0);
    *T = T0 + 0.5 * s->QB[r];
    for (int a = 0; a < 3; a++) F[a] = s->FB[3 * r + a] + s->P.body_force[a];
    if (s->P.buoyancy) F[s->P.gravity_axis] += s->buoy * (*T - s->P.T_ref);
    for (int a = 0; a < 3; a++) u[a] = (j[a] + 0.5 * F[a]) / *rho;
}

/* ------------------------------------------------------ collide + stream */
static void lattice_step(orc_sim* s) {
    const double tf = s->tau_f, tg = s->tau_g;
    for (long r = 0; r < s->N; r++) {
        double rho, u[3], T, F[3];
        macro(s, r, &rho, u, &T, F);
        for (int i = 0; i < s->Q; i++) {
            double fi = s->f[(long)i * s->N + r];
            double eu = s->e[i][0] * u[0] + s->e[i][1] * u[1] + s->e[i][2] * u[2];
            /* Eq lbm9: (1 - 1/2tau) w [3 (e - u) + 9 (e.u) e] . F */
            double Fi = 0.0;
            for (int a = 0; a < 3; a++) Fi += (3.0 * (s->e[i][a] - u[a]) + 9.0 * eu * s->e[i][a]) * F[a];
            Fi *= (1.0 - 0.5 / tf) * s->w[i];
            /* Eq lbm2 */
            s->fpost[(long)i * s->N + r] = fi - (fi - feq(s, i, rho, u)) / tf + Fi;
        }
        for (int k = 0; k < s->QG; k++) {
            double gk = s->g[(long)k * s->N + r];
            double Gk = (1.0 - 0.5 / tg) * s->wg[k] * s->QB[r]; /* Eq lbm12.5 */
            s->gpost[(long)k * s->N + r] = gk - (gk - geq(s, k, T, u)) / tg + Gk; /* Eq lbm2.5 */
        }
    }
    /* streaming f(r + e dt, t + dt) = f*(r, t); halfway bounce-back at walls */
    for (int z = 0; z < s->n[2]; z++)
        for (int y = 0; y < s->n[1]; y++)
            for (int x = 0; x < s->n[0]; x++) {
                long r = nidx(s, x, y, z);
                int c[3] = {x, y, z};
                for (int i = 0; i < s->Q; i++) {
                    int tgt[3], out = 0, face = -1;
                    for (int a = 0; a < 3; a++) {
                        tgt[a] = c[a] + s->e[i][a];
                        if (tgt[a] < 0 || tgt[a] >= s->n[a]) {
                            if (axis_periodic(s, a))
                                tgt[a] = (tgt[a] + s->n[a]) % s->n[a];
                            else {
                                out = 1;
                                face = 2 * a + (tgt[a] >= s->n[a]);
                            }
                        }
                    }
                    double v = s->fpost[(long)i * s->N + r];
                    if (out) {
                        s->f[(long)opposite(s, i, s->Q) * s->N + r] = v;
                    } else {
                        s->f[(long)i * s->N + nidx(s, tgt[0], tgt[1], tgt[2])] = v;
                    }
                    (void)face;
                }
                for (int k = 0; k < s->QG; k++) {
                    int tgt[3], out = 0, face = -1;
                    for (int a = 0; a < 3; a++) {
                        tgt[a] = c[a] + s->e[k][a];
                        if (tgt[a] < 0 || tgt[a] >= s->n[a]) {
                            if (axis_periodic(s, a))
                                tgt[a] = (tgt[a] + s->n[a]) % s->n[a];
                            else {
                                out = 1;
                                face = 2 * a + (tgt[a] >= s->n[a]);
                            }
                        }
                    }
                    double v = s->gpost[(long)k * s->N + r];
                    if (out) {
                        int kb = opposite(s, k, s->QG);
                        if (s->therm[face] == ORC_ISOTHERMAL)
                            s->g[(long)kb * s->N + r] = -v + 2.0 * s->wg[k] * s->Tw[face];
                        else
                            s->g[(long)kb * s->N + r] = v;
                    } else {
                        s->g[(long)k * s->N + nidx(s, tgt[0], tgt[1], tgt[2])] = v;
                    }
                }
            }
}

/* ------------------------------------------------------------ PIBM coupling */
static void cross(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* add W * (MF, MQ) to F_B, Q_B at node c + d if that node lies in the fluid (Eqs lbm10, lbm12.6) */
static void spread_to(orc_sim* s, const int c[3], double W, const double MF[3], double MQ) {
    int t[3];
    for (int a = 0; a < 3; a++) {
        t[a] = c[a];
        if (t[a] < 0 || t[a] >= s->n[a]) {
            if (!axis_periodic(s, a)) return; /* outside a wall: dropped */
            t[a] = ((t[a] % s->n[a]) + s->n[a]) % s->n[a];
        }
    }
    long r = nidx(s, t[0], t[1], t[2]);
    for (int a = 0; a < 3; a++) s->FB[3 * r + a] += W * MF[a];
    s->QB[r] += W * MQ;
}

static void coupling(orc_sim* s) {
    memset(s->FB, 0, sizeof(double) * 3 * s->N);
    memset(s->QB, 0, sizeof(double) * s->N);
    for (int p = 0; p < s->np; p++)
        for (int a = 0; a < 3; a++) s->Fh[3 * p + a] = s->Th[3 * p + a] = 0.0;
    for (int p = 0; p < s->np; p++) s->Hh[p] = 0.0;
    s->nu_sum = 0.0;
    if (!s->P.pibm) return;

    /* sub-grid particles (d_p <= h): one PIBM point each at the particle centre,
     * moving with it (Eqs lbm5-lbm8 at the point, Eqs lbm10-lbm12 for the spreading) */
    if (s->np > 0 && s->point) {
        for (int p = 0; p < s->np; p++) {
            const double* Xl = &s->X[3 * p];
            double L[3][4];
            int base[3] = {0, 0, 0};
            for (int a = 0; a < 3; a++) {
                if (a < s->D) {
                    /* Eq lbm6, four points per axis; at a wall the stencil is shifted inside */
                    int b = (int)floor(Xl[a]) - 1;
                    if (b > s->n[a] - 4) b = s->n[a] - 4;
                    if (b < 0) b = 0;
                    base[a] = b;
                    for (int k = 0; k < 4; k++) {
                        double Lk = 1.0;
                        for (int m = 0; m < 4; m++)
                            if (m != k) Lk *= (Xl[a] - (b + m)) / (double)(k - m);
                        L[a][k] = Lk;
                    }
                } else {
                    L[a][0] = 1.0;
                }
            }
            int nz4 = (s->D == 3) ? 4 : 1;
            double fl[19], gl[7];
            for (int i = 0; i < s->Q; i++) fl[i] = 0.0;
            for (int k = 0; k < s->QG; k++) gl[k] = 0.0;
            for (int kz = 0; kz < nz4; kz++)
                for (int ky = 0; ky < 4; ky++)
                    for (int kx = 0; kx < 4; kx++) {
                        long r = nidx(s, base[0] + kx, base[1] + ky, (s->D == 3) ? base[2] + kz : 0);
                        double Lw = L[0][kx] * L[1][ky] * (s->D == 3 ? L[2][kz] : 1.0);
                        for (int i = 0; i < s->Q; i++) fl[i] += Lw * s->f[(long)i * s->N + r];
                        for (int k = 0; k < s->QG; k++) gl[k] += Lw * s->g[(long)k * s->N + r];
                    }
            double rho = 0, j[3] = {0, 0, 0}, Tl = 0;
            for (int i = 0; i < s->Q; i++) {
                rho += fl[i];
                for (int a = 0; a < 3; a++) j[a] += s->e[i][a] * fl[i];
            }
            for (int k = 0; k < s->QG; k++) Tl += gl[k];
            /* Eqs lbm7 + lbm8 with A_p = pi d_p^2 / 4; Eq lbm7.5 */
            const double A = PI * s->R[p] * s->R[p];
            double MF[3], MQ;
            for (int a = 0; a < 3; a++) MF[a] = A * 2.0 * (rho * s->U[3 * p + a] - j[a]);
            if (s->D == 2) MF[2] = 0.0;
            MQ = A * 2.0 * s->P.kappa_T * (s->Tp[p] - Tl);
            for (int a = 0; a < 3; a++) s->Fh[3 * p + a] = -MF[a]; /* Eq lbm13 */
            s->Hh[p] = MQ;
            int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
            for (int a = 0; a < s->D; a++) {
                lo[a] = (int)ceil(Xl[a] - 2.0);
                hi[a] = (int)floor(Xl[a] + 2.0);
            }
            for (int z = lo[2]; z <= hi[2]; z++)
                for (int y = lo[1]; y <= hi[1]; y++)
                    for (int x = lo[0]; x <= hi[0]; x++) {
                        double Wk = orc_delta_h(x - Xl[0]) * orc_delta_h(y - Xl[1]);
                        if (s->D == 3) Wk *= orc_delta_h(z - Xl[2]);
                        int c[3] = {x, y, z};
                        spread_to(s, c, Wk, MF, MQ);
                    }
        }
    }

    /* resolved particles: covered nodes are the PIBM points */
    if (s->np > 0 && !s->point) {
        int* owner = (int*)malloc(sizeof(int) * s->N);
        double* best = (double*)calloc(s->N, sizeof(double));
        for (long r = 0; r < s->N; r++) owner[r] = -1;
        for (int p = 0; p < s->np; p++) {
            int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
            for (int a = 0; a < s->D; a++) {
                lo[a] = (int)ceil(s->X[3 * p + a] - s->R[p] - 0.5);
                hi[a] = (int)floor(s->X[3 * p + a] + s->R[p] + 0.5);
                if (lo[a] < 0) lo[a] = 0;
                if (hi[a] > s->n[a] - 1) hi[a] = s->n[a] - 1;
            }
            for (int z = lo[2]; z <= hi[2]; z++)
                for (int y = lo[1]; y <= hi[1]; y++)
                    for (int x = lo[0]; x <= hi[0]; x++) {
                        double dx = x - s->X[3 * p], dy = y - s->X[3 * p + 1], dz = z - s->X[3 * p + 2];
                        double eps = s->R[p] + 0.5 - sqrt(dx * dx + dy * dy + dz * dz);
                        if (eps > 1.0) eps = 1.0;
                        long r = nidx(s, x, y, z);
                        if (eps > 0.0 && eps > best[r]) { /* strict: the lower index keeps a tie */
                            best[r] = eps;
                            owner[r] = p;
                        }
                    }
        }
        for (int z = 0; z < s->n[2]; z++)
            for (int y = 0; y < s->n[1]; y++)
                for (int x = 0; x < s->n[0]; x++) {
                    long r = nidx(s, x, y, z);
                    int p = owner[r];
                    if (p < 0) continue;
                    double rho, j[3], T0;
                    moments(s, r, &rho, j, &T0); /* Eqs lbm5, lbm5.5 at a node: L is the identity */
                    double arm[3] = {x - s->X[3 * p], y - s->X[3 * p + 1], z - s->X[3 * p + 2]};
                    double wxr[3], Ul[3], MF[3], MQ;
                    cross(&s->W[3 * p], arm, wxr);
                    for (int a = 0; a < 3; a++) Ul[a] = s->U[3 * p + a] + wxr[a];
                    /* Eqs lbm7 + lbm8: F_f = 2 (rho U_l - j); Eq lbm7.5: Q = 2 kappa (T_p - T) */
                    for (int a = 0; a < 3; a++) MF[a] = best[r] * 2.0 * (rho * Ul[a] - j[a]);
                    MQ = best[r] * 2.0 * s->P.kappa_T * (s->Tp[p] - T0);
                    /* Eq lbm13: F_fpi = -F_f A_p; torque about the particle centre */
                    double tq[3];
                    cross(arm, MF, tq);
                    for (int a = 0; a < 3; a++) {
                        s->Fh[3 * p + a] -= MF[a];
                        s->Th[3 * p + a] -= tq[a];
                    }
                    s->Hh[p] += MQ;
                    /* Eqs lbm10, lbm11, lbm12: node-located point, delta_h weights 1/2, 1/4, 1/4 */
                    for (int dz = (s->D == 3 ? -1 : 0); dz <= (s->D == 3 ? 1 : 0); dz++)
                        for (int dy = -1; dy <= 1; dy++)
                            for (int dx = -1; dx <= 1; dx++) {
                                double Wk = orc_delta_h(dx) * orc_delta_h(dy);
                                if (s->D == 3) Wk *= orc_delta_h(dz);
                                int c[3] = {x + dx, y + dy, z + dz};
                                spread_to(s, c, Wk, MF, MQ);
                            }
                }
        free(owner);
        free(best);
    }

    /* static off-node markers (cylinder built from small particles) */
    for (int l = 0; l < s->nm; l++) {
        const double* Xl = &s->MX[3 * l];
        double L[3][4];
        int base[3] = {0, 0, 0};
        for (int a = 0; a < 3; a++) {
            if (a < s->D)
                base[a] = orc_lagrange_weights(Xl[a], 4, L[a]);
            else {
                L[a][0] = 1.0;
            }
        }
        int nz4 = (s->D == 3) ? 4 : 1;
        double fl[19], gl[7];
        for (int i = 0; i < s->Q; i++) fl[i] = 0.0;
        for (int k = 0; k < s->QG; k++) gl[k] = 0.0;
        /* Eqs lbm5, lbm5.5 */
        for (int kz = 0; kz < nz4; kz++)
            for (int ky = 0; ky < 4; ky++)
                for (int kx = 0; kx < 4; kx++) {
                    int c[3] = {base[0] + kx, base[1] + ky, (s->D == 3) ? base[2] + kz : 0};
                    for (int a = 0; a < s->D; a++) c[a] = ((c[a] % s->n[a]) + s->n[a]) % s->n[a];
                    long r = nidx(s, c[0], c[1], c[2]);
                    double Lw = L[0][kx] * L[1][ky] * (s->D == 3 ? L[2][kz] : 1.0);
                    for (int i = 0; i < s->Q; i++) fl[i] += Lw * s->f[(long)i * s->N + r];
                    for (int k = 0; k < s->QG; k++) gl[k] += Lw * s->g[(long)k * s->N + r];
                }
        double rho = 0, j[3] = {0, 0, 0}, Tl = 0;
        for (int i = 0; i < s->Q; i++) {
            rho += fl[i];
            for (int a = 0; a < 3; a++) j[a] += s->e[i][a] * fl[i];
        }
        for (int k = 0; k < s->QG; k++) Tl += gl[k];
        double MF[3], MQ;
        for (int a = 0; a < 3; a++) MF[a] = s->MA[l] * 2.0 * (rho * 0.0 - j[a]); /* static: U_l = 0 */
        MQ = s->MA[l] * 2.0 * s->P.kappa_T * (s->MT[l] - Tl);
        s->nu_sum += s->MA[l] * (s->MT[l] - Tl);
        int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int a = 0; a < s->D; a++) {
            lo[a] = (int)ceil(Xl[a] - 2.0);
            hi[a] = (int)floor(Xl[a] + 2.0);
        }
        for (int z = lo[2]; z <= hi[2]; z++)
            for (int y = lo[1]; y <= hi[1]; y++)
                for (int x = lo[0]; x <= hi[0]; x++) {
                    double Wk = orc_delta_h(x - Xl[0]) * orc_delta_h(y - Xl[1]);
                    if (s->D == 3) Wk *= orc_delta_h(z - Xl[2]);
                    int c[3] = {x, y, z};
                    spread_to(s, c, Wk, MF, MQ);
                }
    }
}

/* -------------------------------------------------------------------- DEM */
static void cell_grid(const orc_sim* s, int nc[3], double inv[3]) {
    double rmax = 0.0;
    for (int p = 0; p < s->np; p++)
        if (s->R[p] > rmax) rmax = s->R[p];
    double cmin = s->P.cell_size > 0.0 ? s->P.cell_size : 2.0 * rmax + 1.5;
    for (int a = 0; a < 3; a++) {
        nc[a] = 1;
        inv[a] = 1.0 / (double)s->n[a];
        if (a < s->D) {
            nc[a] = (int)floor((double)s->n[a] / cmin);
            if (nc[a] < 1) nc[a] = 1;
            inv[a] = (double)nc[a] / (double)s->n[a];
        }
    }
}

static int cell_coord(double x, double inv, int nc) {
    int c = (int)floor((x + 0.5) * inv);
    if (c < 0) c = 0;
    if (c > nc - 1) c = nc - 1;
    return c;
}

int orc_cells(orc_sim* s, int* cell, int* ncell) {
    int nc[3];
    double inv[3];
    cell_grid(s, nc, inv);
    for (int p = 0; p < s->np; p++) {
        int c[3];
        for (int a = 0; a < 3; a++) c[a] = cell_coord(s->X[3 * p + a], inv[a], nc[a]);
        cell[p] = (c[2] * nc[1] + c[1]) * nc[0] + c[0];
    }
    if (ncell)
        for (int a = 0; a < 3; a++) ncell[a] = nc[a];
    return s->np;
}

static int in_contact(const orc_sim* s, int i, int j) {
    double dx = s->X[3 * j] - s->X[3 * i];
    double dy = s->X[3 * j + 1] - s->X[3 * i + 1];
    double dz = s->X[3 * j + 2] - s->X[3 * i + 2];
    double d2 = dx * dx + dy * dy + dz * dz;
    double sr = s->R[i] + s->R[j];
    return d2 < sr * sr;
}

static int cmp_contact(const void* a, const void* b) {
    const contact* x = (const contact*)a;
    const contact* y = (const contact*)b;
    if (x->i != y->i) return x->i < y->i ? -1 : 1;
    if (x->j != y->j) return x->j < y->j ? -1 : 1;
    return 0;
}

/* cell-list contact search: pairs (i < j) with |X_i - X_j| < R_i + R_j, sorted by (i, j) */
static contact* find_contacts(const orc_sim* s, int* count) {
    int nc[3];
    double inv[3];
    cell_grid(s, nc, inv);
    int ncells = nc[0] * nc[1] * nc[2];
    int* head = (int*)malloc(sizeof(int) * ncells);
    int* next = (int*)malloc(sizeof(int) * (s->np + 1));
    int* cc = (int*)malloc(sizeof(int) * 3 * (s->np + 1));
    for (int c = 0; c < ncells; c++) head[c] = -1;
    for (int p = s->np - 1; p >= 0; p--) {
        for (int a = 0; a < 3; a++) cc[3 * p + a] = cell_coord(s->X[3 * p + a], inv[a], nc[a]);
        int c = (cc[3 * p + 2] * nc[1] + cc[3 * p + 1]) * nc[0] + cc[3 * p];
        next[p] = head[c];
        head[c] = p;
    }
    int cap = 64, n = 0;
    contact* out = (contact*)malloc(sizeof(contact) * cap);
    for (int i = 0; i < s->np; i++) {
        for (int z = cc[3 * i + 2] - 1; z <= cc[3 * i + 2] + 1; z++)
            for (int y = cc[3 * i + 1] - 1; y <= cc[3 * i + 1] + 1; y++)
                for (int x = cc[3 * i] - 1; x <= cc[3 * i] + 1; x++) {
                    if (x < 0 || y < 0 || z < 0 || x >= nc[0] || y >= nc[1] || z >= nc[2]) continue;
                    for (int j = head[(z * nc[1] + y) * nc[0] + x]; j >= 0; j = next[j]) {
                        if (j <= i || !in_contact(s, i, j)) continue;
                        if (n == cap) {
                            cap *= 2;
                            out = (contact*)realloc(out, sizeof(contact) * cap);
                        }
                        out[n].i = i;
                        out[n].j = j;
                        out[n].ft[0] = out[n].ft[1] = out[n].ft[2] = 0.0;
                        memset(&out[n].md, 0, sizeof(md_state));
                        n++;
                    }
                }
    }
    qsort(out, n, sizeof(contact), cmp_contact);
    free(head);
    free(next);
    free(cc);
    *count = n;
    return out;
}

int orc_contacts(orc_sim* s, int* pairs, int cap) {
    int n;
    contact* c = find_contacts(s, &n);
    for (int k = 0; k < n && k < cap; k++) {
        pairs[2 * k] = c[k].i;
        pairs[2 * k + 1] = c[k].j;
    }
    free(c);
    return n;
}

int orc_contacts_bruteforce(orc_sim* s, int* pairs, int cap) {
    int n = 0;
    for (int i = 0; i < s->np; i++)
        for (int j = i + 1; j < s->np; j++)
            if (in_contact(s, i, j)) {
                if (n < cap) {
                    pairs[2 * n] = i;
                    pairs[2 * n + 1] = j;
                }
                n++;
            }
    return n;
}

/* contact pairs and cells of a bare point set (same definitions, no lattice):
 * brute force over all pairs i < j with |X_i - X_j|^2 < (R_i + R_j)^2 */
int orc_point_contacts(int np, const double* X, const double* R, int* pairs, int cap) {
    int n = 0;
    for (int i = 0; i < np; i++)
        for (int j = i + 1; j < np; j++) {
            double dx = X[3 * j] - X[3 * i], dy = X[3 * j + 1] - X[3 * i + 1], dz = X[3 * j + 2] - X[3 * i + 2];
            double d2 = dx * dx + dy * dy + dz * dz;
            double sr = R[i] + R[j];
            if (d2 < sr * sr) {
                if (n < cap) {
                    pairs[2 * n] = i;
                    pairs[2 * n + 1] = j;
                }
                n++;
            }
        }
    return n;
}

int orc_point_cells(int dim, const int* nlat, double cell_size, int np, const double* X, const double* R, int* cell,
                    int* ncell) {
    double rmax = 0.0;
    for (int p = 0; p < np; p++)
        if (R[p] > rmax) rmax = R[p];
    double cmin = cell_size > 0.0 ? cell_size : 2.0 * rmax + 1.5;
    int nc[3];
    double inv[3];
    for (int a = 0; a < 3; a++) {
        nc[a] = 1;
        inv[a] = 1.0 / (double)nlat[a];
        if (a < dim) {
            nc[a] = (int)floor((double)nlat[a] / cmin);
            if (nc[a] < 1) nc[a] = 1;
            inv[a] = (double)nc[a] / (double)nlat[a];
        }
    }
    for (int p = 0; p < np; p++) {
        int c[3];
        for (int a = 0; a < 3; a++) c[a] = cell_coord(X[3 * p + a], inv[a], nc[a]);
        cell[p] = (c[2] * nc[1] + c[1]) * nc[0] + c[0];
    }
    for (int a = 0; a < 3; a++) ncell[a] = nc[a];
    return np;
}

/* Hertz normal force (text after Eq demgov) and Mindlin-Deresiewicz loading stiffness
 * k_t = 8 G* r_a, or the linear spring-dashpot law; returns F_n and sets kt_eff */
static double normal_law(const orc_sim* s, double delta, double vn, double Rstar, double* kt_eff) {
    if (s->law == ORC_HERTZ_MD || s->law == ORC_HERTZ_MD_HIST) {
        double Estar = s->E / (2.0 * (1.0 - s->pois * s->pois));
        double G = s->E / (2.0 * (1.0 + s->pois));
        double Gstar = G / (2.0 * (1.0 - s->pois * s->pois));
        double ra = sqrt(delta * Rstar);
        *kt_eff = 8.0 * Gstar * ra;
        return 4.0 / 3.0 * Estar * sqrt(Rstar) * delta * sqrt(delta) + s->gn * vn;
    }
    *kt_eff = s->kt;
    return s->kn * delta + s->gn * vn;
}

/* tangential force: rotate the history into the tangent plane, add -k_t v_t dt, Coulomb cap */
static void tangential(const orc_sim* s, double ft[3], const double n[3], const double vt[3], double kt_eff,
                       double Fn, double dt, double Ft_total[3]) {
    double fn = ft[0] * n[0] + ft[1] * n[1] + ft[2] * n[2];
    for (int a = 0; a < 3; a++) ft[a] = ft[a] - fn * n[a] - kt_eff * vt[a] * dt;
    double mag = sqrt(ft[0] * ft[0] + ft[1] * ft[1] + ft[2] * ft[2]);
    double cap = s->mu * fabs(Fn);
    if (mag > cap) {
        double sc = (mag > 0.0) ? cap / mag : 0.0;
        for (int a = 0; a < 3; a++) ft[a] *= sc;
    }
    for (int a = 0; a < 3; a++) Ft_total[a] = ft[a] - s->gt * vt[a];
}

/* Tangential force with the Mindlin-Deresiewicz loading history (text after
 * Eq demgov: increment 8 G* r_a theta_k dd_t + (-1)^k mu dF_n (1 - theta_k)),
 * theta_k by the closure of Thornton and Yin (1991) for loading (k = 0),
 * unloading (k = 1) and reloading (k = 2):
 *   theta_0^3 = 1 - (T + mu dF_n) / (mu F_n)
 *   theta_1^3 = 1 - (T* - T + 2 mu dF_n) / (2 mu F_n)
 *   theta_2^3 = 1 - (T - T** + 2 mu dF_n) / (2 mu F_n)
 * with T the tangential force along the contact's reference direction e and
 * T*, T** its values at the last turning points.  The branch changes when the
 * tangential displacement increment along e changes sign (loading -> unloading
 * at T*, unloading -> reloading at T**, reloading -> loading once T climbs back
 * to T*).  The force increment acts along the displacement increment (vector
 * form, e carried in the tangent plane); Coulomb cap mu |F_n| on the total.
 * kt8a = 8 G* r_a. */
static void tangential_md(const orc_sim* s, double ft[3], md_state* md, const double n[3], const double vt[3],
                          double kt8a, double Fn, double dt, double Ft_total[3]) {
    double fn = ft[0] * n[0] + ft[1] * n[1] + ft[2] * n[2];
    double en = md->e[0] * n[0] + md->e[1] * n[1] + md->e[2] * n[2];
    for (int a = 0; a < 3; a++) {
        ft[a] -= fn * n[a];
        md->e[a] -= en * n[a];
    }
    double el = sqrt(md->e[0] * md->e[0] + md->e[1] * md->e[1] + md->e[2] * md->e[2]);
    double ds[3] = {vt[0] * dt, vt[1] * dt, vt[2] * dt};
    double dsl = sqrt(ds[0] * ds[0] + ds[1] * ds[1] + ds[2] * ds[2]);
    if (el > 0.0) {
        for (int a = 0; a < 3; a++) md->e[a] /= el;
    } else if (dsl > 0.0) { /* first tangential displacement: T grows along e */
        for (int a = 0; a < 3; a++) md->e[a] = -ds[a] / dsl;
    }
    const double mu = s->mu, N = fabs(Fn);
    /* a contact's first update carries no loading history: its normal force
     * jump from zero is not an increment of the slip annulus */
    const double dFn = md->Fn_prev > 0.0 ? N - md->Fn_prev : 0.0;
    const double T = ft[0] * md->e[0] + ft[1] * md->e[1] + ft[2] * md->e[2];
    const double sgn = -(ds[0] * md->e[0] + ds[1] * md->e[1] + ds[2] * md->e[2]); /* > 0: T increases */
    if (md->k == 0 && sgn < 0.0) {
        md->k = 1;
        md->Ts = T;
    } else if (md->k == 1 && sgn > 0.0) {
        md->k = 2;
        md->Tss = T;
    } else if (md->k == 2) {
        if (sgn < 0.0) {
            md->k = 1;
            md->Ts = T;
        } else if (T >= md->Ts) {
            md->k = 0;
        }
    }
    double th3 = 0.0;
    if (mu * N > 0.0) {
        if (md->k == 0) th3 = 1.0 - (T + mu * dFn) / (mu * N);
        else if (md->k == 1) th3 = 1.0 - (md->Ts - T + 2.0 * mu * dFn) / (2.0 * mu * N);
        else th3 = 1.0 - (T - md->Tss + 2.0 * mu * dFn) / (2.0 * mu * N);
    }
    if (th3 < 0.0) th3 = 0.0;
    if (th3 > 1.0) th3 = 1.0;
    const double th = cbrt(th3);
    const double sk = (md->k == 1) ? -1.0 : 1.0; /* (-1)^k */
    for (int a = 0; a < 3; a++) ft[a] += -kt8a * th * ds[a] + sk * mu * dFn * (1.0 - th) * md->e[a];
    double mag = sqrt(ft[0] * ft[0] + ft[1] * ft[1] + ft[2] * ft[2]);
    double cap = mu * N;
    if (mag > cap) {
        double sc = (mag > 0.0) ? cap / mag : 0.0;
        for (int a = 0; a < 3; a++) ft[a] *= sc;
    }
    md->Fn_prev = N;
    for (int a = 0; a < 3; a++) Ft_total[a] = ft[a] - s->gt * vt[a];
}

static void contact_forces(orc_sim* s, double dt) {
    /* new contact list; carry the tangential history of pairs that stay in contact */
    int n;
    contact* nc = find_contacts(s, &n);
    for (int k = 0; k < n; k++) {
        contact* old = (contact*)bsearch(&nc[k], s->cont, s->ncont, sizeof(contact), cmp_contact);
        if (old) {
            for (int a = 0; a < 3; a++) nc[k].ft[a] = old->ft[a];
            nc[k].md = old->md;
        }
    }
    free(s->cont);
    s->cont = nc;
    s->ncont = n;

    for (int p = 0; p < 3 * s->np; p++) s->Fc[p] = s->Tc[p] = 0.0;
    for (int k = 0; k < n; k++) {
        int i = nc[k].i, j = nc[k].j;
        double d[3], dist = 0.0;
        for (int a = 0; a < 3; a++) {
            d[a] = s->X[3 * j + a] - s->X[3 * i + a];
            dist += d[a] * d[a];
        }
        dist = sqrt(dist);
        double nrm[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
        double delta = s->R[i] + s->R[j] - dist;
        double ai = s->R[i] - 0.5 * delta, aj = s->R[j] - 0.5 * delta;
        double ri[3], rj[3], wi[3], wj[3], vrel[3];
        for (int a = 0; a < 3; a++) {
            ri[a] = ai * nrm[a];
            rj[a] = -aj * nrm[a];
        }
        cross(&s->W[3 * i], ri, wi);
        cross(&s->W[3 * j], rj, wj);
        for (int a = 0; a < 3; a++) vrel[a] = (s->U[3 * i + a] + wi[a]) - (s->U[3 * j + a] + wj[a]);
        double vn = vrel[0] * nrm[0] + vrel[1] * nrm[1] + vrel[2] * nrm[2];
        double vt[3];
        for (int a = 0; a < 3; a++) vt[a] = vrel[a] - vn * nrm[a];
        double Rstar = s->R[i] * s->R[j] / (s->R[i] + s->R[j]), kt_eff;
        double Fn = normal_law(s, delta, vn, Rstar, &kt_eff);
        double Ft[3], Fi[3], Ti[3], Tj[3];
        if (s->law == ORC_HERTZ_MD_HIST) tangential_md(s, nc[k].ft, &nc[k].md, nrm, vt, kt_eff, Fn, dt, Ft);
        else tangential(s, nc[k].ft, nrm, vt, kt_eff, Fn, dt, Ft);
        for (int a = 0; a < 3; a++) Fi[a] = -Fn * nrm[a] + Ft[a];
        cross(ri, Ft, Ti);
        double rjn[3] = {aj * nrm[0], aj * nrm[1], aj * nrm[2]};
        cross(rjn, Ft, Tj);
        for (int a = 0; a < 3; a++) {
            s->Fc[3 * i + a] += Fi[a];
            s->Fc[3 * j + a] -= Fi[a];
            s->Tc[3 * i + a] += Ti[a];
            s->Tc[3 * j + a] += Tj[a];
        }
    }
    /* particle-wall contacts: the same law with R_wall = infinity, wall at rest */
    for (int i = 0; i < s->np; i++)
        for (int face = 0; face < 2 * s->D; face++) {
            int a = face / 2, hi = face % 2;
            double* ft = &s->wall_ft[(6 * (long)i + face) * 3];
            md_state* wmd = &s->wall_md[6 * (long)i + face];
            if (axis_periodic(s, a)) continue;
            double dist = hi ? (s->n[a] - 0.5) - s->X[3 * i + a] : s->X[3 * i + a] + 0.5;
            double delta = s->R[i] - dist;
            if (!(delta > 0.0)) {
                ft[0] = ft[1] = ft[2] = 0.0;
                memset(wmd, 0, sizeof(md_state));
                continue;
            }
            double nrm[3] = {0, 0, 0};
            nrm[a] = hi ? 1.0 : -1.0;
            double ai = s->R[i] - 0.5 * delta;
            double ri[3] = {ai * nrm[0], ai * nrm[1], ai * nrm[2]}, wi[3], vrel[3];
            cross(&s->W[3 * i], ri, wi);
            for (int b = 0; b < 3; b++) vrel[b] = s->U[3 * i + b] + wi[b];
            double vn = vrel[0] * nrm[0] + vrel[1] * nrm[1] + vrel[2] * nrm[2];
            double vt[3];
            for (int b = 0; b < 3; b++) vt[b] = vrel[b] - vn * nrm[b];
            double kt_eff;
            double Fn = normal_law(s, delta, vn, s->R[i], &kt_eff);
            double Ft[3], Ti[3];
            if (s->law == ORC_HERTZ_MD_HIST) tangential_md(s, ft, wmd, nrm, vt, kt_eff, Fn, dt, Ft);
            else tangential(s, ft, nrm, vt, kt_eff, Fn, dt, Ft);
            cross(ri, Ft, Ti);
            for (int b = 0; b < 3; b++) {
                s->Fc[3 * i + b] += -Fn * nrm[b] + Ft[b];
                s->Tc[3 * i + b] += Ti[b];
            }
        }
}

/* Hydrodynamic force, torque and heat felt by particle p over one lattice step:
 * the mean of the coupling of time t and of time t-1.  Under the half-force
 * velocity of the text after Eq lbm3.5 the fluid's physical momentum advances
 * by the mean of consecutive forcing terms, so the particle receives the same
 * mean; this removes the step-to-step sign flip that a bounce-back impulse
 * (Eqs lbm7, lbm8) applied on every covered node imprints on the reaction. */
static double hydro(const orc_sim* s, const double* cur, const double* prev, int k) {
    return s->have_prev ? 0.5 * (cur[k] + prev[k]) : cur[k];
}

/* Eq demgov: m dU/dt = m (1 - rho_f/rho_p) g + F_fpi + sum F_c ; I domega/dt = tau_p + sum T_c.
 * With a hydrodynamic Jacobian J set (19 values per particle: a learned
 * estimate of dF_fpi/dU, dtau_p/domega and dH_p/dT_p), the held hydrodynamic
 * load is corrected inside the step by J_FU (U - U_start) and J_TW (omega -
 * omega_start); the heat row acts in the thermosensitive update (orc_step). */
static void kick(orc_sim* s, double h) {
    for (int p = 0; p < s->np; p++) {
        if (s->fixed[p]) continue;
        double mg = s->m[p] * (1.0 - 1.0 / s->rho[p]);
        double dF[3] = {0, 0, 0}, dT[3] = {0, 0, 0};
        if (s->J) {
            const double* J = s->J + 19 * p;
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) {
                    dF[a] += J[3 * a + b] * (s->U[3 * p + b] - s->U0[3 * p + b]);
                    dT[a] += J[9 + 3 * a + b] * (s->W[3 * p + b] - s->W0[3 * p + b]);
                }
        }
        for (int a = 0; a < 3; a++) {
            double F = s->Fc[3 * p + a] + (hydro(s, s->Fh, s->Fp, 3 * p + a) + dF[a]) + mg * s->P.g_particle[a];
            s->U[3 * p + a] += h * F / s->m[p];
            s->W[3 * p + a] += h * (s->Tc[3 * p + a] + (hydro(s, s->Th, s->Tq, 3 * p + a) + dT[a])) / s->I[p];
        }
        if (s->D == 2) {
            s->U[3 * p + 2] = 0.0;
            s->W[3 * p] = s->W[3 * p + 1] = 0.0;
        }
    }
}

static void dem(orc_sim* s) {
    if (s->np == 0) return;
    int nsub = s->P.dem_substeps > 0 ? s->P.dem_substeps : 1;
    double dt = 1.0 / nsub;
    if (s->J) {
        memcpy(s->U0, s->U, sizeof(double) * 3 * s->np);
        memcpy(s->W0, s->W, sizeof(double) * 3 * s->np);
    }
    for (int sub = 0; sub < nsub; sub++) {
        kick(s, 0.5 * dt); /* velocity Verlet: half kick with the last contact force */
        for (int p = 0; p < s->np; p++) {
            if (s->fixed[p]) continue;
            for (int a = 0; a < 3; a++) s->X[3 * p + a] += dt * s->U[3 * p + a];
        }
        contact_forces(s, dt);
        kick(s, 0.5 * dt);
    }
}

/* ----------------------------------------------------------------- API */
orc_sim* orc_create(const orc_params* p) {
    if (!p || (p->dim != 2 && p->dim != 3) || p->nx < 1 || p->ny < 1 || p->nz < 1) return NULL;
    if (p->dim == 2 && p->nz != 1) return NULL;
    if (p->flow_q != 0 && !(p->dim == 3 && (p->flow_q == 15 || p->flow_q == 19)) && !(p->dim == 2 && p->flow_q == 9))
        return NULL;
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->P = *p;
    s->D = p->dim;
    if (s->D == 2) {
        s->Q = 9;
        s->QG = 5;
        s->e = E2;
        s->w = W2Q9;
        s->wg = W2Q5;
        s->csT2 = 1.0 / 3.0;
    } else if (p->flow_q == 15) {
        s->Q = 15;
        s->QG = 7;
        s->e = E15;
        s->w = W3Q15;
        s->wg = W3Q7;
        s->csT2 = 1.0 / 4.0;
    } else {
        s->Q = 19;
        s->QG = 7;
        s->e = E3;
        s->w = W3Q19;
        s->wg = W3Q7;
        s->csT2 = 1.0 / 4.0;
    }
    s->n[0] = p->nx;
    s->n[1] = p->ny;
    s->n[2] = p->nz;
    s->N = (long)p->nx * p->ny * p->nz;
    relaxation(s);
    for (int f = 0; f < 6; f++) s->wall[f] = ORC_PERIODIC;
    s->f = (double*)malloc(sizeof(double) * s->Q * s->N);
    s->fpost = (double*)malloc(sizeof(double) * s->Q * s->N);
    s->g = (double*)malloc(sizeof(double) * s->QG * s->N);
    s->gpost = (double*)malloc(sizeof(double) * s->QG * s->N);
    s->FB = (double*)calloc(3 * s->N, sizeof(double));
    s->QB = (double*)calloc(s->N, sizeof(double));
    double u0[3] = {0, 0, 0};
    for (long r = 0; r < s->N; r++) {
        for (int i = 0; i < s->Q; i++) s->f[(long)i * s->N + r] = feq(s, i, 1.0, u0);
        for (int k = 0; k < s->QG; k++) s->g[(long)k * s->N + r] = geq(s, k, p->T_init, u0);
    }
    s->law = ORC_SPRING_DASHPOT;
    coupling(s);
    return s;
}

static void free_particles(orc_sim* s) {
    double** arr[] = {&s->X, &s->U, &s->W, &s->R, &s->rho, &s->Tp, &s->Cp, &s->m, &s->I,
                      &s->Fh, &s->Th, &s->Hh, &s->Fc, &s->Tc, &s->Fp, &s->Tq, &s->Hp, &s->wall_ft,
                      &s->J, &s->U0, &s->W0};
    for (unsigned k = 0; k < sizeof(arr) / sizeof(arr[0]); k++) {
        free(*arr[k]);
        *arr[k] = NULL;
    }
    free(s->fixed);
    s->fixed = NULL;
    free(s->wall_md);
    s->wall_md = NULL;
    free(s->cont);
    s->cont = NULL;
    s->ncont = 0;
    s->np = 0;
}

void orc_destroy(orc_sim* s) {
    if (!s) return;
    free(s->f);
    free(s->fpost);
    free(s->g);
    free(s->gpost);
    free(s->FB);
    free(s->QB);
    free_particles(s);
    free(s->MX);
    free(s->MA);
    free(s->MT);
    free(s);
}

int orc_set_wall(orc_sim* s, int face, int kind, int thermal, double T_w) {
    if (face < 0 || face >= 2 * s->D) return -1;
    s->wall[face] = kind;
    s->therm[face] = thermal;
    s->Tw[face] = T_w;
    coupling(s);
    return 0;
}

int orc_set_contact_law(orc_sim* s, int law, double E, double poisson, double mu, double kn, double kt,
                        double gamma_n, double gamma_t) {
    /* entering the loading-history law: the other laws keep no such history, so
     * every contact's tangential force and history start afresh (its next update
     * is its first) */
    if (law == ORC_HERTZ_MD_HIST && s->law != ORC_HERTZ_MD_HIST) {
        for (int k = 0; k < s->ncont; k++) {
            memset(&s->cont[k].md, 0, sizeof(md_state));
            s->cont[k].ft[0] = s->cont[k].ft[1] = s->cont[k].ft[2] = 0.0;
        }
        if (s->wall_md) memset(s->wall_md, 0, sizeof(md_state) * 6 * (size_t)s->np);
        if (s->wall_ft) memset(s->wall_ft, 0, sizeof(double) * 18 * (size_t)s->np);
    }
    s->law = law;
    s->E = E;
    s->pois = poisson;
    s->mu = mu;
    s->kn = kn;
    s->kt = kt;
    s->gn = gamma_n;
    s->gt = gamma_t;
    return 0;
}

int orc_set_particles(orc_sim* s, int n, const double* X, const double* U, const double* W, const double* R,
                      const double* rho_p, const double* T_p, const double* heat_cap,
                      const unsigned char* fixed) {
    free_particles(s);
    if (n < 0) return -1;
    s->np = n;
    size_t v = sizeof(double) * 3 * (n + 1), sc = sizeof(double) * (n + 1);
    s->X = (double*)malloc(v);
    s->U = (double*)malloc(v);
    s->W = (double*)malloc(v);
    s->R = (double*)malloc(sc);
    s->rho = (double*)malloc(sc);
    s->Tp = (double*)malloc(sc);
    s->Cp = (double*)malloc(sc);
    s->m = (double*)malloc(sc);
    s->I = (double*)malloc(sc);
    s->Fh = (double*)calloc(3 * (n + 1), sizeof(double));
    s->Th = (double*)calloc(3 * (n + 1), sizeof(double));
    s->Hh = (double*)calloc(n + 1, sizeof(double));
    s->Fc = (double*)calloc(3 * (n + 1), sizeof(double));
    s->Tc = (double*)calloc(3 * (n + 1), sizeof(double));
    s->Fp = (double*)calloc(3 * (n + 1), sizeof(double));
    s->Tq = (double*)calloc(3 * (n + 1), sizeof(double));
    s->Hp = (double*)calloc(n + 1, sizeof(double));
    s->have_prev = 0;
    if (s->point)
        for (int p = 0; p < n; p++)
            if (R[p] > 0.5) return -1; /* a point particle has d_p <= h */
    s->wall_ft = (double*)calloc(18 * (n + 1), sizeof(double));
    s->wall_md = (md_state*)calloc(6 * (n + 1), sizeof(md_state));
    s->fixed = (unsigned char*)calloc(n + 1, 1);
    for (int p = 0; p < n; p++) {
        for (int a = 0; a < 3; a++) {
            s->X[3 * p + a] = X[3 * p + a];
            s->U[3 * p + a] = U ? U[3 * p + a] : 0.0;
            s->W[3 * p + a] = W ? W[3 * p + a] : 0.0;
        }
        if (s->D == 2) {
            s->X[3 * p + 2] = 0.0;
            s->U[3 * p + 2] = 0.0;
            s->W[3 * p] = s->W[3 * p + 1] = 0.0;
        }
        s->R[p] = R[p];
        s->rho[p] = rho_p[p];
        s->Tp[p] = T_p ? T_p[p] : 0.0;
        s->Cp[p] = heat_cap ? heat_cap[p] : 0.0;
        s->fixed[p] = fixed ? fixed[p] : 0;
        if (s->D == 2) {
            s->m[p] = s->rho[p] * PI * R[p] * R[p];
            s->I[p] = 0.5 * s->m[p] * R[p] * R[p];
        } else {
            s->m[p] = s->rho[p] * 4.0 / 3.0 * PI * R[p] * R[p] * R[p];
            s->I[p] = 0.4 * s->m[p] * R[p] * R[p];
        }
    }
    coupling(s);
    return 0;
}

int orc_set_markers(orc_sim* s, int n, const double* X, const double* A, const double* T_p) {
    free(s->MX);
    free(s->MA);
    free(s->MT);
    s->nm = n;
    s->MX = (double*)malloc(sizeof(double) * 3 * (n + 1));
    s->MA = (double*)malloc(sizeof(double) * (n + 1));
    s->MT = (double*)malloc(sizeof(double) * (n + 1));
    for (int l = 0; l < n; l++) {
        for (int a = 0; a < 3; a++) s->MX[3 * l + a] = (a < s->D) ? X[3 * l + a] : 0.0;
        s->MA[l] = A[l];
        s->MT[l] = T_p[l];
    }
    coupling(s);
    return 0;
}

int orc_set_populations(orc_sim* s, const double* f, const double* g) {
    if (f) memcpy(s->f, f, sizeof(double) * s->Q * s->N);
    if (g) memcpy(s->g, g, sizeof(double) * s->QG * s->N);
    coupling(s);
    return 0;
}

int orc_step(orc_sim* s, int nsteps) {
    for (int k = 0; k < nsteps; k++) {
        lattice_step(s);
        dem(s);
        /* thermosensitive particles: C_p dT_p = -H_p dt.  With a Jacobian set, the
         * held heat flux is corrected by J_HT (T_p,new - T_p) as well, solved for
         * T_p,new: C_p (T_new - T) = -(H + J_HT (T_new - T)); J_HT < 0 (a particle
         * that warms drawing more heat) is taken as 0. */
        for (int p = 0; p < s->np; p++)
            if (s->Cp[p] > 0.0) {
                double Jh = s->J ? s->J[19 * p + 18] : 0.0;
                if (!(Jh > 0.0)) Jh = 0.0;
                s->Tp[p] -= hydro(s, s->Hh, s->Hp, p) / (s->Cp[p] + Jh);
            }
        s->t++;
        if (s->np > 0) {
            memcpy(s->Fp, s->Fh, sizeof(double) * 3 * s->np);
            memcpy(s->Tq, s->Th, sizeof(double) * 3 * s->np);
            memcpy(s->Hp, s->Hh, sizeof(double) * s->np);
            s->have_prev = 1;
        }
        coupling(s);
    }
    return 0;
}

int orc_read_field(orc_sim* s, int field, double* dst) {
    for (long r = 0; r < s->N; r++) {
        double rho, u[3], T, F[3];
        macro(s, r, &rho, u, &T, F);
        switch (field) {
            case ORC_RHO: dst[r] = rho; break;
            case ORC_UX: dst[r] = u[0]; break;
            case ORC_UY: dst[r] = u[1]; break;
            case ORC_UZ: dst[r] = u[2]; break;
            case ORC_T: dst[r] = T; break;
            case ORC_FBX: dst[r] = s->FB[3 * r]; break;
            case ORC_FBY: dst[r] = s->FB[3 * r + 1]; break;
            case ORC_FBZ: dst[r] = s->FB[3 * r + 2]; break;
            case ORC_QB: dst[r] = s->QB[r]; break;
            default: return -1;
        }
    }
    return 0;
}

int orc_read_populations(orc_sim* s, double* f, double* g) {
    if (f) memcpy(f, s->f, sizeof(double) * s->Q * s->N);
    if (g) memcpy(g, s->g, sizeof(double) * s->QG * s->N);
    return 0;
}

int orc_read_particles(orc_sim* s, double* X, double* U, double* W, double* T_p) {
    if (X) memcpy(X, s->X, sizeof(double) * 3 * s->np);
    if (U) memcpy(U, s->U, sizeof(double) * 3 * s->np);
    if (W) memcpy(W, s->W, sizeof(double) * 3 * s->np);
    if (T_p) memcpy(T_p, s->Tp, sizeof(double) * s->np);
    return s->np;
}

int orc_read_particle_forces(orc_sim* s, double* F, double* T, double* H) {
    if (F) memcpy(F, s->Fh, sizeof(double) * 3 * s->np);
    if (T) memcpy(T, s->Th, sizeof(double) * 3 * s->np);
    if (H) memcpy(H, s->Hh, sizeof(double) * s->np);
    return s->np;
}

int orc_set_particle_model(orc_sim* s, int point) {
    if (point != 0 && point != 1) return -1;
    s->point = point;
    return 0;
}

int orc_set_hydro_jacobian(orc_sim* s, const double* J) {
    free(s->J);
    free(s->U0);
    free(s->W0);
    s->J = s->U0 = s->W0 = NULL;
    if (!J || s->np == 0) return 0;
    s->J = (double*)malloc(sizeof(double) * 19 * s->np);
    s->U0 = (double*)malloc(sizeof(double) * 3 * s->np);
    s->W0 = (double*)malloc(sizeof(double) * 3 * s->np);
    memcpy(s->J, J, sizeof(double) * 19 * s->np);
    return 0;
}

int orc_read_contact_forces(orc_sim* s, double* F, double* T) {
    if (F) memcpy(F, s->Fc, sizeof(double) * 3 * s->np);
    if (T) memcpy(T, s->Tc, sizeof(double) * 3 * s->np);
    return s->np;
}

/* average Nusselt number over the static markers (Nu formula of the cavity case, k = alpha) */
double orc_nusselt(orc_sim* s) { return s->nu_sum / (s->alpha * s->P.nu_dT); }

/* out: [sum rho, sum g, particle kinetic energy, min particle coordinate along gravity, max |u|, non-finite] */
int orc_diagnostics(orc_sim* s, double* out) {
    double mass = 0, heat = 0, umax = 0, bad = 0;
    for (long r = 0; r < s->N; r++) {
        double rho, u[3], T, F[3], j[3], T0;
        moments(s, r, &rho, j, &T0);
        mass += rho;
        heat += T0;
        macro(s, r, &rho, u, &T, F);
        double um = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        if (um > umax) umax = um;
        if (!isfinite(rho) || !isfinite(T0)) bad = 1;
    }
    double ke = 0, hmin = 1e300;
    for (int p = 0; p < s->np; p++) {
        double v2 = 0, w2 = 0;
        for (int a = 0; a < 3; a++) {
            v2 += s->U[3 * p + a] * s->U[3 * p + a];
            w2 += s->W[3 * p + a] * s->W[3 * p + a];
        }
        ke += 0.5 * s->m[p] * v2 + 0.5 * s->I[p] * w2;
        double h = s->X[3 * p + s->P.gravity_axis];
        if (h < hmin) hmin = h;
    }
    out[0] = mass;
    out[1] = heat;
    out[2] = ke;
    out[3] = s->np ? hmin : 0.0;
    out[4] = umax;
    out[5] = bad;
    return 0;
}

int orc_relaxation(orc_sim* s, double* out) {
    out[0] = s->nu;
    out[1] = s->alpha;
    out[2] = s->tau_f;
    out[3] = s->tau_g;
    out[4] = s->buoy;
    return 0;
}

long orc_time(orc_sim* s) { return s->t; }

/* Test entry: the tangential update of one contact with the Mindlin-Deresiewicz
 * history along a prescribed path.  Normal n, contact radius a (k_t base
 * 8 G* a with the law's G*), normal force Fn[k] and tangential displacement
 * increment ds[3k..3k+2] at update k; writes the tangential force after each
 * update to T_out[3k..].  Returns 0, or -1 if the law is not ORC_HERTZ_MD_HIST. */
int orc_md_path(const orc_sim* s, const double* n, double a, int nsteps, const double* Fn, const double* ds,
                double* T_out) {
    if (s->law != ORC_HERTZ_MD_HIST) return -1;
    double G = s->E / (2.0 * (1.0 + s->pois));
    double Gstar = G / (2.0 * (1.0 - s->pois * s->pois));
    double ft[3] = {0.0, 0.0, 0.0}, Ft[3];
    md_state md;
    memset(&md, 0, sizeof md);
    for (int k = 0; k < nsteps; k++) {
        tangential_md(s, ft, &md, n, ds + 3 * k, 8.0 * Gstar * a, Fn[k], 1.0, Ft);
        for (int c = 0; c < 3; c++) T_out[3 * k + c] = ft[c];
    }
    return 0;
}

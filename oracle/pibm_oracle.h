/*
 * pibm_oracle.h -- plain FP64, single-threaded CPU oracle of the thermal
 * LBM-PIBM-DEM lattice step of Zhang et al., "Particulate immersed boundary
 * method for complex fluid-particle interaction problems with heat transfer"
 * (arXiv 1502.01159).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header,
 * table or helper with the CUDA library under paper_1502_01159_gb300/.
 *
 * Units are lattice units throughout: h = dt = 1, reference density 1.
 * Node (x, y, z) has linear index (z*ny + y)*nx + x.  Halfway walls sit half
 * a node outside the first and last node of a walled axis, i.e. at -0.5 and
 * n-0.5.  Vectors are interleaved n*3 (z component 0 in 2-D).
 *
 * Velocity sets (direction order is part of the contract, both libraries use it):
 *   D2Q9 : 0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1) 5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1)
 *   D2Q5 : directions 0..4 of D2Q9
 *   D3Q19: 0 (0,0,0) 1 (1,0,0) 2 (-1,0,0) 3 (0,1,0) 4 (0,-1,0) 5 (0,0,1) 6 (0,0,-1)
 *          7 (1,1,0) 8 (-1,-1,0) 9 (1,-1,0) 10 (-1,1,0) 11 (1,0,1) 12 (-1,0,-1)
 *          13 (1,0,-1) 14 (-1,0,1) 15 (0,1,1) 16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1)
 *   D3Q7 : directions 0..6 of D3Q19
 */
#ifndef PIBM_ORACLE_H
#define PIBM_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_sim orc_sim;

typedef struct {
    int dim;                 /* 2 or 3 */
    int nx, ny, nz;          /* nz = 1 in 2-D */
    double Ra, Pr;           /* Rayleigh and Prandtl numbers (Eqs lbm2.6, lbm2.7) */
    double U_c, L_c;         /* characteristic velocity (lattice units) and length (nodes) */
    double T_ref;            /* Boussinesq reference temperature */
    double T_init;           /* initial fluid temperature */
    int buoyancy;            /* 1: add the thermal buoyancy force */
    int gravity_axis;        /* gravity points along -axis (0, 1 or 2) */
    double body_force[3];    /* constant body force added at every node */
    double g_particle[3];    /* gravitational acceleration felt by particles */
    int dem_substeps;        /* DEM substeps per lattice step */
    double kappa_T;          /* prefactor of the thermal PIBM correction */
    double cell_size;        /* minimum DEM cell side; <= 0: 2*R_max + 1.5 */
    double nu_dT;            /* T_hot - T_inf in the Nusselt number */
    int pibm;                /* 1: particles and fluid are coupled */
    int flow_q;              /* 3-D flow lattice: 0 or 19 D3Q19, 15 D3Q15 (Section 2.1's own); 2-D: D2Q9 */
} orc_params;

enum { ORC_PERIODIC = 0, ORC_WALL = 1 };
enum { ORC_ADIABATIC = 0, ORC_ISOTHERMAL = 1 };
/* ORC_HERTZ_MD: Hertz normal force, Mindlin no-slip tangential spring (theta_k = 1);
 * ORC_HERTZ_MD_HIST: the same with the Mindlin-Deresiewicz loading history (theta_k
 * of Thornton and Yin for loading, unloading and reloading) */
enum { ORC_SPRING_DASHPOT = 0, ORC_HERTZ_MD = 1, ORC_HERTZ_MD_HIST = 2 };
enum { ORC_RHO = 0, ORC_UX, ORC_UY, ORC_UZ, ORC_T, ORC_FBX, ORC_FBY, ORC_FBZ, ORC_QB };

orc_sim* orc_create(const orc_params* p);
void     orc_destroy(orc_sim* s);
int      orc_set_wall(orc_sim* s, int face, int kind, int thermal, double T_w);
int      orc_set_contact_law(orc_sim* s, int law, double E, double poisson, double mu,
                             double kn, double kt, double gamma_n, double gamma_t);
int      orc_set_particles(orc_sim* s, int n, const double* X, const double* U,
                           const double* W, const double* R, const double* rho_p,
                           const double* T_p, const double* heat_cap,
                           const unsigned char* fixed);
int      orc_set_markers(orc_sim* s, int n, const double* X, const double* A, const double* T_p);
int      orc_set_populations(orc_sim* s, const double* f, const double* g);
int      orc_step(orc_sim* s, int nsteps);
int      orc_read_field(orc_sim* s, int field, double* dst);
int      orc_read_populations(orc_sim* s, double* f, double* g);
int      orc_read_particles(orc_sim* s, double* X, double* U, double* W, double* T_p);
int      orc_read_particle_forces(orc_sim* s, double* F, double* T, double* H);
int      orc_read_contact_forces(orc_sim* s, double* F, double* T);
/* Optional hydrodynamic Jacobian, 19 doubles per particle: J_FU (3x3,
 * row-major, dF_a/dU_b), J_TW (dtau_a/domega_b), then J_HT (dH/dT_p); NULL
 * removes it.  Kept until replaced or until the particles are reset. */
int      orc_set_hydro_jacobian(orc_sim* s, const double* J);
/* Particle model for the next orc_set_particles: 0 resolved (the covered
 * nodes are the PIBM points), 1 one PIBM point per particle at its centre
 * (d_p <= h, the paper's own regime; radii above 1/2 are rejected). */
int      orc_set_particle_model(orc_sim* s, int point);
double   orc_nusselt(orc_sim* s);
int      orc_contacts(orc_sim* s, int* pairs, int cap);
int      orc_contacts_bruteforce(orc_sim* s, int* pairs, int cap);
int      orc_cells(orc_sim* s, int* cell, int* ncell);
int      orc_point_contacts(int np, const double* X, const double* R, int* pairs, int cap);
int      orc_point_cells(int dim, const int* nlat, double cell_size, int np, const double* X, const double* R,
                         int* cell, int* ncell);
int      orc_diagnostics(orc_sim* s, double* out);
int      orc_relaxation(orc_sim* s, double* out);
long     orc_time(orc_sim* s);
int      orc_lagrange_weights(double x, int npts, double* w);
double   orc_delta_h(double a);
int      orc_md_path(const orc_sim* s, const double* n, double a, int nsteps, const double* Fn, const double* ds,
                     double* T_out);

#ifdef __cplusplus
}
#endif
#endif

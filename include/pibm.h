/*
 * pibm.h -- C ABI of the GB300 (sm_103a) library for the thermal lattice
 * Boltzmann / particulate immersed boundary / discrete element step of
 * Zhang, Yuan, Trias, Yu, Tan, Oliva, "Particulate immersed boundary method
 * for complex fluid-particle interaction problems with heat transfer"
 * (arXiv 1502.01159).
 *
 * One lattice step t -> t+1 runs, on one GPU:
 *   1. BGK collision of the flow populations f (D2Q9 / D3Q19) and thermal
 *      populations g (D2Q5 / D3Q7) with the immersed-boundary force F_B, the
 *      heat source Q_B and Boussinesq buoyancy, then streaming, fused in one
 *      in-place kernel (Section 2.1, Eqs lbm2, lbm2.5, lbm3, lbm3.5, lbm9,
 *      lbm12.5);
 *   2. the particle equations of motion in n_sub DEM substeps with the
 *      hydrodynamic force of time t held fixed and Hertz / Mindlin-Deresiewicz
 *      or linear spring-dashpot contacts found with a cell list (Section 2.3,
 *      Eq demgov);
 *   3. the PIBM coupling of time t+1: no-slip velocity and particle
 *      temperature imposed on the lattice nodes each particle covers, spread
 *      back as F_B, Q_B, and reduced to per-particle force, torque and heat
 *      flux (Section 2.2, Eqs lbm5-lbm13).
 *
 * Units: lattice units (h = dt = 1, reference density 1).  Node (x, y, z) has
 * linear index (z*ny + y)*nx + x.  Walls sit half a node outside the first and
 * last node of a walled axis (at -0.5 and n-0.5).  Vectors are interleaved
 * n*3 (z component 0 in 2-D).  Direction order:
 *   D2Q9 : 0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1) 5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1)
 *   D2Q5 : directions 0..4 of D2Q9
 *   D3Q19: 0 (0,0,0) 1 (1,0,0) 2 (-1,0,0) 3 (0,1,0) 4 (0,-1,0) 5 (0,0,1) 6 (0,0,-1)
 *          7 (1,1,0) 8 (-1,-1,0) 9 (1,-1,0) 10 (-1,1,0) 11 (1,0,1) 12 (-1,0,-1)
 *          13 (1,0,-1) 14 (-1,0,1) 15 (0,1,1) 16 (0,-1,-1) 17 (0,1,-1) 18 (0,-1,1)
 *   D3Q7 : directions 0..6 of D3Q19
 *
 * Ownership: the caller owns every pointer it passes; the library copies
 * inputs during the call and never keeps a caller pointer.  The context owns
 * all device memory; it comes from the optional allocator (for instance the
 * PyTorch caching allocator) or from cudaMalloc, and pibm_destroy releases it.
 *
 * Errors: every call returns a status and never aborts, exits or traps.  On
 * failure the context keeps its previous state unless the status says
 * otherwise; pibm_last_error gives a one-line message.
 *
 * Streams: all device work is ordered on the stream given at creation (plus
 * one internal stream forked and joined inside each step).  Calls that return
 * data to host memory synchronise that stream.  A context is not thread-safe.
 */
#ifndef PIBM_H
#define PIBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pibm_ctx pibm_ctx;

typedef enum {
    PIBM_OK = 0,
    PIBM_ERR_ARG = 1,       /* invalid argument or description */
    PIBM_ERR_OOM = 2,       /* device allocation failed */
    PIBM_ERR_CUDA = 3,      /* a CUDA call failed; see pibm_last_error */
    PIBM_ERR_STATE = 4,     /* call not valid in the current state, or a device-side
                               consistency check failed (e.g. neighbour list overflow) */
    PIBM_ERR_UNSTABLE = 5,  /* non-finite values detected; state kept for inspection */
    PIBM_ERR_TIMEOUT = 6    /* a bounded device-side wait gave up */
} pibm_status;

enum { PIBM_PERIODIC = 0, PIBM_WALL = 1 };           /* wall kind per face */
enum { PIBM_ADIABATIC = 0, PIBM_ISOTHERMAL = 1 };    /* thermal condition per wall face */
enum { PIBM_SPRING_DASHPOT = 0, PIBM_HERTZ_MD = 1, PIBM_HERTZ_MD_HIST = 2 }; /* contact law */
/* population storage (deviation form f - w, g - w T_ref; arithmetic in FP32
 * for F32 / F16 / BF16, FP64 for F64; F16 stores the deviations scaled by 2^10
 * (flow) and 2^8 (thermal), BF16 unscaled) */
enum { PIBM_STORE_F32 = 0, PIBM_STORE_F64 = 1, PIBM_STORE_F16 = 2, PIBM_STORE_BF16 = 3 };
enum {                                                /* fields for pibm_read_field */
    PIBM_RHO = 0, PIBM_UX, PIBM_UY, PIBM_UZ, PIBM_T, PIBM_FBX, PIBM_FBY, PIBM_FBZ, PIBM_QB
};

/* Device allocator hook.  alloc returns a device pointer aligned to >= 256
 * bytes or NULL; free releases it.  user is passed back unchanged. */
typedef struct {
    void* (*alloc)(size_t bytes, void* user);
    void (*free)(void* ptr, void* user);
    void* user;
} pibm_allocator;

/* Problem description (Section 2.1; Eqs lbm2.6, lbm2.7 give the relaxation
 * times from Ra, Pr, U_c, L_c: nu = U_c L_c sqrt(Pr/Ra), alpha = nu/Pr,
 * tau_f = 3 nu + 1/2, tau_g = alpha / cs_T^2 + 1/2). */
typedef struct {
    int dim;                /* 2 or 3 */
    int nx, ny, nz;         /* lattice size; nz = 1 in 2-D */
    int storage;            /* PIBM_STORE_F32, _F64, _F16 or _BF16 */
    double Ra, Pr;          /* Rayleigh and Prandtl numbers */
    double U_c, L_c;        /* characteristic velocity (lattice units) and length (nodes) */
    double T_ref;           /* Boussinesq reference temperature */
    double T_init;          /* initial fluid temperature */
    int buoyancy;           /* 1: buoyancy (U_c^2/L_c)(T - T_ref) along -gravity */
    int gravity_axis;       /* gravity points along -axis */
    double body_force[3];   /* constant body force at every node */
    double g_particle[3];   /* gravitational acceleration of the particles */
    int dem_substeps;       /* DEM substeps per lattice step (>= 1) */
    double kappa_T;         /* prefactor of the thermal correction Q = 2 kappa_T (T_p - T) */
    double cell_size;       /* minimum DEM cell side; <= 0 selects 2 R_max + 1.5 */
    double nu_dT;           /* T_hot - T_inf in the Nusselt number */
    int pibm;               /* 1: couple fluid and particles */
    int flow_q;             /* 3-D flow lattice: 0 or 19 D3Q19, 15 D3Q15 (Section 2.1's own 3-D
                               lattice: rest 2/9, six axis links 1/9, eight cube diagonals 1/72);
                               2-D: 0 or 9 (D2Q9).  The thermal lattice is D2Q5 / D3Q7. */
} pibm_desc;

/* Create a context: allocates the lattice (f and g initialised to the rest
 * equilibrium at density 1 and temperature T_init, Eqs lbm3, lbm3.5) with all
 * faces periodic.  stream: a cudaStream_t, or NULL for the default stream.
 * alloc: NULL uses cudaMalloc / cudaFree.  Returns PIBM_ERR_ARG for an
 * invalid description, PIBM_ERR_OOM if the device memory cannot be obtained. */
pibm_status pibm_create(const pibm_desc* desc, void* stream, const pibm_allocator* alloc, pibm_ctx** out);

/* Release every device buffer of the context and the context itself. */
pibm_status pibm_destroy(pibm_ctx* ctx);

/* Boundary of face 0..2*dim-1 (x-lo, x-hi, y-lo, y-hi, z-lo, z-hi).  Both
 * faces of an axis must end up with the same kind.  A wall is a halfway
 * bounce-back no-slip wall for f; for g it is isothermal at T_w
 * (anti-bounce-back) or adiabatic (bounce-back).  Recomputes the coupling. */
pibm_status pibm_set_wall(pibm_ctx* ctx, int face, int kind, int thermal, double T_w);

/* Contact law (text after Eq demgov).  HERTZ_MD: F_n = 4/3 E* sqrt(R*) d^1.5 +
 * gamma_n v_n with 1/E* = (1-nu^2)/E + (1-nu^2)/E, tangential stiffness
 * 8 G* sqrt(d R*) (the loading branch, theta_k = 1).  HERTZ_MD_HIST: the same
 * normal force, tangential increment 8 G* r_a theta_k dd_t + (-1)^k mu dF_n
 * (1 - theta_k) with the Mindlin-Deresiewicz loading history: theta_k of
 * Thornton and Yin for loading (k = 0), unloading (1) and reloading (2) along
 * the contact's reference direction, T* / T** the turning points; its history
 * is evaluated and kept in FP64 (theta_k is a cube root that is not Lipschitz
 * at full slip).  Switching to HERTZ_MD_HIST with particles in place starts
 * every contact's tangential force and history afresh.  SPRING_DASHPOT: F_n = kn d + gamma_n v_n, stiffness kt.  All: tangential
 * force capped at mu |F_n|, tangential damping gamma_t. */
pibm_status pibm_set_contact_law(pibm_ctx* ctx, int law, double E, double poisson, double mu,
                                 double kn, double kt, double gamma_n, double gamma_t);

/* Particles (host arrays, copied).  X, U, W: n*3; R, rho_p, T_p: n;
 * heat_cap: n or NULL (isothermal); fixed: n bytes or NULL (all free).
 * Radii in (0, 600] nodes (PIBM_ERR_ARG otherwise).  At most 10 240 particles
 * (the DEM runs as one cluster of 16 CTAs of at most 640 particles each;
 * PIBM_ERR_ARG beyond).  Requires every axis to be walled when n > 0.  Resets the contact history, rebuilds the cell list and
 * recomputes the coupling of the current time. */
pibm_status pibm_set_particles(pibm_ctx* ctx, int n, const double* X, const double* U, const double* W,
                               const double* R, const double* rho_p, const double* T_p,
                               const double* heat_cap, const uint8_t* fixed);

/* Static off-node markers (the concentric cylinder of the cavity case):
 * positions n*3, areas A_p, temperatures T_p.  Each marker needs its 4-point
 * interpolation stencil inside the lattice.  Recomputes the coupling. */
pibm_status pibm_set_markers(pibm_ctx* ctx, int n, const double* X, const double* A, const double* T_p);

/* Overwrite the populations of the current time with host arrays in the
 * layout [q][z][y][x] (either pointer may be NULL).  Recomputes the coupling. */
pibm_status pibm_set_populations(pibm_ctx* ctx, const double* f, const double* g);

/* Advance nsteps lattice steps (replayed CUDA graphs).  Asynchronous: returns
 * once the work is enqueued.  PIBM_ERR_STATE / PIBM_ERR_UNSTABLE from an
 * earlier step are reported by the next synchronising call. */
pibm_status pibm_step(pibm_ctx* ctx, int nsteps);

/* Macroscopic field of the current time into host_dst (n = nx*ny*nz doubles):
 * rho, u = (j + F/2)/rho, T = sum g + Q_B/2, F_B, Q_B. */
pibm_status pibm_read_field(pibm_ctx* ctx, int field, double* host_dst, size_t n);

/* Populations of the current time (before collision) as doubles [q][z][y][x]. */
pibm_status pibm_read_populations(pibm_ctx* ctx, double* f, double* g);

/* Particle state: X, U, W (n*3) and T_p (n); NULL pointers are skipped. */
pibm_status pibm_read_particles(pibm_ctx* ctx, double* X, double* U, double* W, double* T_p);

/* Hydrodynamic force, torque (n*3) and heat release H (n) of the current
 * time (Eq lbm13 summed over each particle's nodes). */
pibm_status pibm_read_particle_forces(pibm_ctx* ctx, double* F, double* T, double* H);

/* Average Nusselt number over the static markers (sum A (T_p - T) / (alpha nu_dT)). */
pibm_status pibm_nusselt(pibm_ctx* ctx, double* nu);

/* Contacts at the current positions: pairs (i < j) with |X_i - X_j| < R_i + R_j,
 * sorted by (i, j), written as 2*min(cap, n) ints; *n_out = total count. */
pibm_status pibm_read_contacts(pibm_ctx* ctx, int32_t* pairs, int cap, int* n_out);

/* Cell of each particle at the current positions (cell side n_a / nc_a with
 * nc_a = floor(n_a / cell_min); index (cz*ncy + cy)*ncx + cx); ncell: 3 ints or NULL. */
pibm_status pibm_read_cells(pibm_ctx* ctx, int32_t* cell, int32_t* ncell);

/* out[6]: sum rho, sum of g, particle kinetic energy, minimum particle
 * coordinate along the gravity axis, max |u|, 1 if any value is non-finite. */
pibm_status pibm_diagnostics(pibm_ctx* ctx, double* out);

/* out[5]: nu, alpha, tau_f, tau_g, buoyancy coefficient U_c^2/L_c. */
pibm_status pibm_relaxation(pibm_ctx* ctx, double* out);

/* Current lattice time (number of steps taken). */
pibm_status pibm_time(pibm_ctx* ctx, int64_t* t);

/* Checkpoint: every device buffer that carries state between steps (f, g,
 * coupling fields, particles, contact histories, neighbour lists, markers)
 * and the time, written to a file.  pibm_load restores it into a context
 * created with the same description, walls and contact law, and with the
 * same number of particles or markers already set; stepping then continues
 * bit-exactly as the saved run would have.  Both synchronise the stream. */
pibm_status pibm_save(pibm_ctx* ctx, const char* path);
pibm_status pibm_load(pibm_ctx* ctx, const char* path);

/* One lattice step as a replay of the step graph with CUDA event-record nodes
 * around each kernel group, on the stream the group runs on (the same kernels,
 * streams and dependencies as pibm_step).  ms[0] collide-and-stream, ms[1] DEM,
 * ms[2] PIBM coupling, ms[3] the whole step.  Synchronises. */
pibm_status pibm_step_timed(pibm_ctx* ctx, double* ms);

/* Particle model, set before pibm_set_particles:
 *   PIBM_PARTICLES_RESOLVED (default): a particle is the set of lattice nodes
 *     it covers, each a PIBM point with covered fraction epsilon (for
 *     particles several nodes across);
 *   PIBM_PARTICLES_POINT: one PIBM point per particle at its centre (Section
 *     2.2's own regime, d_p <= h): Eq lbm6 with four points per axis (shifted
 *     inside at walls), Eqs lbm7, lbm8, lbm7.5 with A_p = pi d_p^2 / 4, Eq lbm13,
 *     delta_h spreading (Eqs lbm10-lbm12); no hydrodynamic torque.  Radii
 *     above 1/2 and lattices with fewer than 4 nodes on an axis are rejected
 *     by pibm_set_particles.  The spreading adds overlapping supports with
 *     atomics, so the last bits of F_B can differ between runs.
 * PIBM_ERR_STATE if particles are already set. */
enum { PIBM_PARTICLES_RESOLVED = 0, PIBM_PARTICLES_POINT = 1 };
pibm_status pibm_set_particle_model(pibm_ctx* ctx, int model);

/* Launch-shape tuning (used by autotuning sweeps; results do not depend on it,
 * except for PIBM_TUNE_TC_WAIT_POLLS below).
 * PIBM_TUNE_DEM_PARTICLES_PER_CTA: particles per CTA of the DEM cluster
 * (0 = default 32; at most 16 CTAs and 640 particles per CTA).
 * PIBM_TUNE_LATTICE_ROW_TILES: 1 = collide-and-stream blocks span the largest
 * multiple of 32 nodes (at most 256) that divides the row rounded up to 32, so
 * no block straddles a row end with idle warps; 0 (default) = blocks span
 * min(256, row rounded up to 32) nodes.  Identical results either way.
 * PIBM_TUNE_LATTICE_THREADS: threads per block of the collide-and-stream
 * kernel, 0 (default shape: 256 threads for rows of 256 or more nodes, 128
 * for shorter rows and for FP16 / BF16 storage) or a multiple of 32 in
 * [32, 512] (FP16 / BF16 storage: at most 384, larger values act as 384);
 * a block spans
 * min(threads, row width rounded up to 32) nodes of a row (or the row-dividing
 * width above) and as many rows as the remaining factor gives.
 * PIBM_TUNE_WIDE_INDEX: 1 = 64-bit slot offsets in the collide-and-stream
 * kernel even where 32-bit ones suffice (default 0: 32-bit offsets whenever
 * Q N < 2^31 elements, 64-bit beyond; the two give identical results).
 * PIBM_TUNE_TC_WAIT_POLLS: how many times a tensor-core kernel of the learned
 * surrogate polls its completion barrier before it gives up (default
 * 4194304).  It exists to exercise the timeout path: with 0 the next
 * inference (pibm_surrogate_infer, or the surrogate pipeline of a step) gives
 * up at once, waits with the default limit for its own work in flight, frees
 * its tensor memory and the call returns PIBM_ERR_TIMEOUT; the context stays
 * usable.  It is the one knob that changes results.
 * PIBM_TUNE_COUPLING_THREADS: threads per block of the PIBM footprint and
 * spread kernels (one block per particle), 0 (default: 256 in 3-D, sized to
 * the largest disk's box in 2-D) or a multiple of 32 in [64, 256]; the force
 * sums regroup (FP32 rounding of their partial sums).
 * PIBM_TUNE_COUPLING_ORDER: 1 (default) = the footprint and spread blocks
 * take the particles in the spatial order of the DEM's cell list; 0 = in
 * index order (identical results).
 * PIBM_TUNE_LATTICE_PAIRS: 1 (default) = the even (own-slot) step of FP16 /
 * BF16 storage updates two x-adjacent nodes per thread with 32-bit accesses
 * when the row length is even (blocks of PIBM_TUNE_LATTICE_THREADS threads
 * over the row's node pairs); 0 = one node per thread (identical results). */
enum { PIBM_TUNE_DEM_PARTICLES_PER_CTA = 0, PIBM_TUNE_LATTICE_ROW_TILES = 1, PIBM_TUNE_LATTICE_THREADS = 2,
       PIBM_TUNE_WIDE_INDEX = 3, PIBM_TUNE_TC_WAIT_POLLS = 4, PIBM_TUNE_COUPLING_THREADS = 5,
       PIBM_TUNE_COUPLING_ORDER = 6, PIBM_TUNE_LATTICE_PAIRS = 7 };
pibm_status pibm_set_tuning(pibm_ctx* ctx, int knob, int value);

/* Number of kernels one lattice step launches (for launch accounting). */
pibm_status pibm_kernels_per_step(pibm_ctx* ctx, int* n);

/* Contact search for callers that cannot allocate device memory.  The paper
 * has no counterpart of this entry point: it serves code that runs inside
 * another framework's memory pool or arena, plug-ins loaded into a host that
 * owns every device allocation, and processes whose device memory is
 * reserved up front -- they hold particles on the device but cannot create a
 * context (which allocates) or call cudaMalloc.  It computes the same contact
 * list as pibm_read_contacts (pairs i < j with |X_i - X_j| < R_i + R_j in the
 * library's FP64 operation order, sorted by (i, j)) on the caller's device
 * arrays and allocates nothing: its cell list and offsets live in one fixed
 * file-scope device array of 786 440 bytes that every GPU loading the library
 * holds until the process exits.
 *   d_X: n*3 doubles, d_R: n doubles (device); n <= 16384.
 *   dim, nlat[3]: lattice dimension and extents, walls at -0.5 and n - 0.5.
 *   cell_size: minimum cell side (> 0, at least the largest diameter; the
 *     library's default is 2 R_max + 1.5); at most 65536 cells.
 *   d_pairs: 2*cap ints (device); d_count: 2 ints (device): [0] number of
 *     pairs found, keeping at most 64 partners j > i per particle i (the
 *     first min(count, cap) are written, in order, with no gaps), [1] a bit
 *     set: 1 when a particle had more than 64 partners (its extra pairs are
 *     left out), 2 when a diameter exceeds the cell side (pairs may be
 *     missed).
 *   stream: cudaStream_t or NULL.  Asynchronous; the results are valid once
 *     the stream has reached this call.
 * Sizes beyond the limits return PIBM_ERR_ARG (pibm_last_error(NULL, ...)
 * says which).  The scratch array's device address belongs to the CUDA
 * context current at the call: every call made outside stream capture looks
 * it up again (after a device reset or with another context current, the next
 * uncaptured call picks up the new address); a call inside a stream capture
 * uses the address of the last uncaptured call on that device, so make one
 * call before capturing (PIBM_ERR_STATE otherwise).  Every call shares the
 * one array and clears what it needs, so calls that overlap on the GPU (on
 * different streams) race. */
pibm_status pibm_contacts_static(const double* d_X, const double* d_R, int n, int dim, const int32_t* nlat,
                                 double cell_size, int32_t* d_pairs, int cap, int32_t* d_count, void* stream);

/* ------------------------------------------------------------------------
 * Learned coupling surrogate (no counterpart in the paper).  Eq demgov holds
 * the PIBM hydrodynamic force and torque (Eq lbm13 and its torque analogue)
 * fixed over the DEM substeps of a lattice step, and the thermosensitive
 * update holds the heat flux; a small network predicts how they change with
 * the particle's own velocity, spin and temperature, and half its secant
 * Jacobian (the held load is the mean of the couplings of t and t-1, and a
 * change of the particle's state enters only the newer one) corrects them:
 *   F = F_held + J_FU (U - U_step_start),  tau = tau_held + J_TW (omega - omega_step_start)
 * inside the substeps, and C_p (T_new - T) = -(H_held + J_HT (T_new - T)) in
 * the thermosensitive update (a negative J_HT counts as 0).
 * Features (12 per particle, lattice units), over the nodes the particle owns
 * in the coupling (epsilon > 0, the larger epsilon, ties to the lower index)
 * and from the raw moments before the coupling's correction: the fluid
 * velocity fitted by a rigid motion V + Om x (r - X), least squares weighted
 * by epsilon rho (the coupling's weights); U - V (3), omega - Om (3), T_p -
 * the epsilon-weighted mean fluid temperature (1), the solid fraction
 * sum_{q != p, |X_q - X_p| < 4 R_p} (R_q / 4 R_p)^D (1) and the four smallest
 * surface gaps capped at 2 R_p (4).  With these weights the coupling's load at
 * a frozen fluid state is an exact linear function of the first seven.
 * Targets: the PIBM coupling's force (3), torque (3) and heat flux (1) of the
 * state.  Network: 12 -> 64 -> 64 -> 64 -> 7, tanh hidden layers, plus a
 * linear path from the inputs to the outputs: y = W4 a3 + b4 + Ws x.  FP32
 * parameters packed [W1 (64x12), b1, W2 (64x64), b2, W3, b3, W4 (7x64), b4,
 * Ws (7x12)], W[out][in] row-major (PIBM_SURROGATE_PARAMS floats);
 * standardisation norm = [mu_x (12), sd_x (12), mu_y (7), sd_y (7)].
 * Inference runs on the tensor cores in BF16 with FP32 accumulation; training
 * runs in FP32. */
enum { PIBM_SURROGATE_PARAMS = 9691, PIBM_SURROGATE_NORM = 38 };
/* The 12 features of every particle for the current state (n*12 doubles, host). */
pibm_status pibm_read_features(pibm_ctx* ctx, double* out);
/* Set / read the network (host arrays as above).  Scales must be positive. */
pibm_status pibm_surrogate_set_params(pibm_ctx* ctx, const float* params, const float* norm);
pibm_status pibm_surrogate_get_params(pibm_ctx* ctx, float* params, float* norm);
/* Tensor-core inference of rows standardised inputs (rows x 16 floats, the
 * last 4 columns ignored) into rows x 8 standardised outputs (column 7 is 0).
 * PIBM_ERR_TIMEOUT if a bounded device wait gave up. */
pibm_status pibm_surrogate_infer(pibm_ctx* ctx, const float* in, int rows, float* out);
/* FP32 gradient (PIBM_SURROGATE_PARAMS floats) and loss of the mean squared
 * standardised error on B rows (X: B x 12, Y: B x 7, standardised). */
pibm_status pibm_surrogate_gradient(pibm_ctx* ctx, const float* X, const float* Y, int B, float* grad, double* loss);
/* Train on n samples (feat: n x 12, targ: n x 7, raw units, host): the
 * standardisation comes from the data; the hidden layers start
 * Glorot-uniform from seed with zero output weights W4, the linear path Ws
 * and the output bias b4 start at the least-squares fit over all n samples
 * (ridge 1e-8 n on the normal equations); then epochs of shuffled
 * mini-batches of batch rows train every parameter with Adam (lr).
 * loss_per_epoch: NULL or epochs doubles (mean standardised loss). */
pibm_status pibm_surrogate_train(pibm_ctx* ctx, const double* feat, const double* targ, int64_t n, int epochs, int batch,
                                 double lr, uint64_t seed, double* loss_per_epoch);
/* Put the surrogate in the step: after each step's coupling the features,
 * inference, Jacobian and gate run on the device; the next step applies the
 * Jacobian only when sum_p |F_net,p - F_pibm,p| / sum_p |F_pibm,p| <= bound
 * for the current state, F_pibm the coupling's force (else the held PIBM load
 * alone, the plain method).  delta: secant step in standard deviations of
 * each velocity, spin and temperature feature (widened to two BF16 spacings
 * of a feature far out in the tails).  A particle's J_FU or J_TW block that
 * cannot be physical for an explicit substep (a positive diagonal entry, a
 * row not diagonally dominant, or |J_aa| h >= 2 m with h the substep and m
 * the mass or moment of inertia) is zeroed for that step.
 * on = 0 removes it.  A new particle set removes it. */
pibm_status pibm_surrogate_enable(pibm_ctx* ctx, int on, double bound, double delta);
/* [0] steps with the Jacobian applied, [1] steps that fell back, [2] the last relative force error. */
pibm_status pibm_surrogate_stats(pibm_ctx* ctx, double* out);
/* A caller-supplied Jacobian (19 doubles per particle: J_FU row-major, J_TW
 * row-major, J_HT), applied every step until replaced; NULL removes it. */
pibm_status pibm_set_hydro_jacobian(pibm_ctx* ctx, const double* J);
/* The Jacobian in use (n*19, host) and whether the next step applies it. */
pibm_status pibm_read_hydro_jacobian(pibm_ctx* ctx, double* J, int* on);

/* ------------------------------------------------------------------------
 * Batched ensemble (no counterpart in the paper, which runs one case at a
 * time): n_boxes independent lattices -- sizes, Rayleigh numbers, particle
 * sets and every other descriptor field may differ -- advanced together by
 * one CUDA graph launch per lattice step on the ensemble stream.  Each box is
 * an ordinary context, owned by the ensemble: set it up and read it back with
 * the per-context calls on the handle pibm_ensemble_box returns (never
 * pibm_destroy it).  Results of every box are identical to stepping it alone.
 *   descs: n_boxes descriptors (copied).  stream: the ensemble's
 *   cudaStream_t or NULL (one is created).  alloc: device memory hook shared
 *   by all boxes, or NULL.
 * Errors: as pibm_create for any box (the message names the box). */
typedef struct pibm_ensemble pibm_ensemble;
pibm_status pibm_ensemble_create(const pibm_desc* descs, int n_boxes, void* stream, const pibm_allocator* alloc,
                                 pibm_ensemble** out);
pibm_status pibm_ensemble_destroy(pibm_ensemble* e);
/* The context of box b (0 <= b < n_boxes), owned by the ensemble. */
pibm_status pibm_ensemble_box(pibm_ensemble* e, int b, pibm_ctx** out);
/* nsteps lattice steps of every box, one graph launch each.  All boxes must
 * be at the same time step (PIBM_ERR_STATE otherwise); a box whose set-up
 * changed since the last call is re-captured automatically.  Ordered after
 * work already queued on the boxes' streams; later per-box calls are ordered
 * after it.  Device-side errors of a box are reported by the next call. */
pibm_status pibm_ensemble_step(pibm_ensemble* e, int nsteps);
/* Kernels one ensemble step launches (sum over the boxes). */
pibm_status pibm_ensemble_kernels_per_step(pibm_ensemble* e, int* n);
/* Autotuner.  First each box's DEM shape alone: reps steps (pibm_step_timed)
 * of each of PIBM_TUNE_DEM_PARTICLES_PER_CTA in {default, 16, 48, 64, 96}
 * (shapes a box cannot take time the default), the fastest DEM kernel kept as
 * the box's pick.  Then 16 whole-ensemble configurations --
 * PIBM_TUNE_LATTICE_THREADS in {default, 128, 256, 512} x
 * PIBM_TUNE_LATTICE_ROW_TILES in {0, 1} x {default DEM shapes, the picks} --
 * each applied to every box and timed as ensemble steps (graph launches,
 * CUDA events; median of reps + 2 after two untimed steps).  The fastest is kept
 * if it beats the defaults by more than 1 %, else the defaults stay.  These are
 * real steps: every box advances by 5 reps + 16 (reps + 4) steps (launch shapes
 * change no result).  choice: NULL or 3*n_boxes ints receiving (lattice threads,
 * row tiles, DEM particles per CTA) per box, 0 meaning the default. */
pibm_status pibm_ensemble_autotune(pibm_ensemble* e, int reps, int32_t* choice);
/* Last error message of the ensemble (or of a failed create when e is NULL:
 * use pibm_last_error(NULL, ...)); returns its length. */
int pibm_ensemble_last_error(pibm_ensemble* e, char* buf, size_t n);

const char* pibm_status_string(pibm_status s);
/* Copies the last error message of the context (or of the last failed
 * pibm_create when ctx is NULL) into buf; returns its length. */
int pibm_last_error(pibm_ctx* ctx, char* buf, size_t n);

#ifdef __cplusplus
}
#endif
#endif

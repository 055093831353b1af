// Internal declarations of the GB300 LBM-PIBM-DEM library: device-side lattice
// tables, the A-A population addressing shared by every kernel that touches
// f and g, the context structure and the launch wrappers of each kernel file.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/pibm.h"

namespace pibm {

// ------------------------------------------------------------------ lattices
// D2Q9 / D2Q5 and D3Q19 / D3Q7 in the direction order of pibm.h.  Functions of
// a compile-time index fold to constants after unrolling.
template <int D> struct Lat;
template <> struct Lat<2> {
    static constexpr int Q = 9, QG = 5, dim = 2;
    __host__ __device__ static constexpr int ex(int i) { return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0); }
    __host__ __device__ static constexpr int ey(int i) { return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0); }
    __host__ __device__ static constexpr int ez(int) { return 0; }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5); }
    __host__ __device__ static constexpr double w(int i) { return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }
    __host__ __device__ static constexpr double wg(int k) { return k == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }
    static constexpr double inv_csT2 = 3.0;  // D2Q5: cs_T^2 = 1/3
};
template <> struct Lat<3> {
    static constexpr int Q = 19, QG = 7, dim = 3;
    __host__ __device__ static constexpr int ex(int i) {
        return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1 : ((i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ey(int i) {
        return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1 : ((i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ez(int i) {
        return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1 : ((i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0);
    }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
    __host__ __device__ static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
    __host__ __device__ static constexpr double wg(int k) { return k == 0 ? 0.25 : 0.125; }
    static constexpr double inv_csT2 = 4.0;  // D3Q7: cs_T^2 = 1/4
};

// D3Q15 (Section 2.1's own 3-D lattice) with the D3Q7 thermal lattice: rest,
// six axis links (1/9), eight cube diagonals (1/72); c_s^2 = 1/3.  Lattice id
// 4 in the kernels' first template argument (2: D2Q9, 3: D3Q19).
template <> struct Lat<4> {
    static constexpr int Q = 15, QG = 7, dim = 3;
    __host__ __device__ static constexpr int ex(int i) {
        return (i == 1 || i == 7 || i == 9 || i == 11 || i == 14) ? 1 : ((i == 2 || i == 8 || i == 10 || i == 12 || i == 13) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ey(int i) {
        return (i == 3 || i == 7 || i == 9 || i == 12 || i == 13) ? 1 : ((i == 4 || i == 8 || i == 10 || i == 11 || i == 14) ? -1 : 0);
    }
    __host__ __device__ static constexpr int ez(int i) {
        return (i == 5 || i == 7 || i == 10 || i == 11 || i == 13) ? 1 : ((i == 6 || i == 8 || i == 9 || i == 12 || i == 14) ? -1 : 0);
    }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
    __host__ __device__ static constexpr double w(int i) { return i == 0 ? 2.0 / 9.0 : (i <= 6 ? 1.0 / 9.0 : 1.0 / 72.0); }
    __host__ __device__ static constexpr double wg(int k) { return k == 0 ? 0.25 : 0.125; }
    static constexpr double inv_csT2 = 4.0;  // D3Q7: cs_T^2 = 1/4
};

template <typename S> struct Vec4;
template <> struct Vec4<float> { using T = float4; };
template <> struct Vec4<double> { using T = double4_32a; };

// Population storage: the type S kept in HBM, the arithmetic type R, the
// per-node force / heat-source field type V4, and the conversions.  FP32 and
// FP64 store the deviations as they are.  FP16 stores them scaled by a power
// of two (exact), so that deviations of order 1e-4 .. 1e-1 sit in the normal
// FP16 range (flow x 1024, thermal x 256); BF16 keeps FP32's exponent range
// and needs no scale.  All collision arithmetic is in R = FP32 for both.
// rawf / raws convert without the scale: the 16-bit lattice kernel collides in
// the storage's own units (deviations times 2^KF for f, 2^KG for g).
template <typename S> struct Store {
    using R = S;
    using V4 = typename Vec4<S>::T;
    static constexpr int KF = 0, KG = 0;
    static __host__ __device__ __forceinline__ R ldf(S v) { return v; }
    static __host__ __device__ __forceinline__ R ldg(S v) { return v; }
    static __host__ __device__ __forceinline__ S stf(R v) { return v; }
    static __host__ __device__ __forceinline__ S stg(R v) { return v; }
};
template <> struct Store<__half> {
    using R = float;
    using V4 = float4;
    static __device__ __forceinline__ float ldf(__half v) { return __half2float(v) * 0.0009765625f; }
    static __device__ __forceinline__ float ldg(__half v) { return __half2float(v) * 0.00390625f; }
    static __device__ __forceinline__ __half stf(float v) { return __float2half_rn(v * 1024.0f); }
    static __device__ __forceinline__ __half stg(float v) { return __float2half_rn(v * 256.0f); }
    static constexpr int KF = 10, KG = 8;
    static __device__ __forceinline__ float rawf(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half raws(float v) { return __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
    using R = float;
    using V4 = float4;
    static __device__ __forceinline__ float ldf(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ float ldg(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 stf(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ __nv_bfloat16 stg(float v) { return __float2bfloat16_rn(v); }
    static constexpr int KF = 0, KG = 0;
    static __device__ __forceinline__ float rawf(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 raws(float v) { return __float2bfloat16_rn(v); }
};

// Run FN<D, S>(args...) for the context's dimension and storage type.
#define PIBM_DISPATCH(c, FN, ...)                                                                       \
    do {                                                                                                \
        switch ((c)->desc.storage) {                                                                    \
            case PIBM_STORE_F64:                                                                        \
                return (c)->D == 2 ? FN<2, double>(__VA_ARGS__) : ((c)->lat == 4 ? FN<4, double>(__VA_ARGS__) : FN<3, double>(__VA_ARGS__));           \
            case PIBM_STORE_F16:                                                                        \
                return (c)->D == 2 ? FN<2, __half>(__VA_ARGS__) : ((c)->lat == 4 ? FN<4, __half>(__VA_ARGS__) : FN<3, __half>(__VA_ARGS__));           \
            case PIBM_STORE_BF16:                                                                       \
                return (c)->D == 2 ? FN<2, __nv_bfloat16>(__VA_ARGS__) : ((c)->lat == 4 ? FN<4, __nv_bfloat16>(__VA_ARGS__) : FN<3, __nv_bfloat16>(__VA_ARGS__)); \
            default:                                                                                    \
                return (c)->D == 2 ? FN<2, float>(__VA_ARGS__) : ((c)->lat == 4 ? FN<4, float>(__VA_ARGS__) : FN<3, float>(__VA_ARGS__));             \
        }                                                                                               \
    } while (0)

// ------------------------------------------------------------ lattice state
// Geometry and boundary data every lattice kernel needs (passed by value).
struct Geo {
    int nx, ny, nz;
    long long N;      // nodes = plane stride
    int ntx;          // 32-node tiles along x
    int per[3];       // 1 if the axis is periodic
    int iso;          // bit f set: face f is an isothermal wall
    double dTw[6];    // T_w - T_ref per face
};

// Anti-bounce-back offset 2 w (T_w - T_ref) of face f, or -1 if face f is not
// isothermal (constant indices only, so the struct stays in registers).
__host__ __device__ __forceinline__ bool face_iso(const Geo& G, int f) { return f >= 0 && ((G.iso >> f) & 1); }
__host__ __device__ __forceinline__ double face_dTw(const Geo& G, int f) {
    switch (f) {
        case 0: return G.dTw[0];
        case 1: return G.dTw[1];
        case 2: return G.dTw[2];
        case 3: return G.dTw[3];
        case 4: return G.dTw[4];
        default: return G.dTw[5];
    }
}

__host__ __device__ inline long long node_index(const Geo& G, int x, int y, int z) {
    return ((long long)z * G.ny + y) * G.nx + x;
}

// Location of the population of direction i (opposite io) that node (x,y,z)
// holds before collision at time parity p under the A-A pattern:
//   even t: plane i at the node itself;
//   odd t : plane io at node x - e_i, or -- when x - e_i lies beyond a wall --
//           plane i at the node itself (halfway bounce-back of the value the
//           node wrote in the previous step).
// Returns the face crossed (>= 0) or -1.  The population value is the stored
// value, except at a crossed isothermal face of the thermal lattice where it
// is 2 w (T_w - T_ref) minus the stored value (anti-bounce-back).
__device__ __forceinline__ int pop_slot(const Geo& G, int x, int y, int z, int exi, int eyi, int ezi, int i, int io,
                                        int parity, long long& idx) {
    long long n = node_index(G, x, y, z);
    if (parity == 0) {
        idx = (long long)i * G.N + n;
        return -1;
    }
    int sx = x - exi, sy = y - eyi, sz = z - ezi, face = -1;
    if (sx < 0) { if (G.per[0]) sx += G.nx; else face = 0; }
    else if (sx >= G.nx) { if (G.per[0]) sx -= G.nx; else face = 1; }
    if (sy < 0) { if (G.per[1]) sy += G.ny; else face = 2; }
    else if (sy >= G.ny) { if (G.per[1]) sy -= G.ny; else face = 3; }
    if (sz < 0) { if (G.per[2]) sz += G.nz; else face = 4; }
    else if (sz >= G.nz) { if (G.per[2]) sz -= G.nz; else face = 5; }
    if (face >= 0)
        idx = (long long)i * G.N + n;
    else
        idx = (long long)io * G.N + node_index(G, sx, sy, sz);
    return face;
}

// Destination of the post-collision population of direction i of node
// (x,y,z) at time parity p (the inverse of pop_slot one step later):
//   even t: plane io at the node;
//   odd t : plane i at node x + e_i, or plane io at the node when x + e_i lies
//           beyond a wall (bounce-back; anti-bounce-back at isothermal faces).
__device__ __forceinline__ int post_slot(const Geo& G, int x, int y, int z, int exi, int eyi, int ezi, int i, int io,
                                         int parity, long long& idx) {
    long long n = node_index(G, x, y, z);
    if (parity == 0) {
        idx = (long long)io * G.N + n;
        return -1;
    }
    int tx = x + exi, ty = y + eyi, tz = z + ezi, face = -1;
    if (tx < 0) { if (G.per[0]) tx += G.nx; else face = 0; }
    else if (tx >= G.nx) { if (G.per[0]) tx -= G.nx; else face = 1; }
    if (ty < 0) { if (G.per[1]) ty += G.ny; else face = 2; }
    else if (ty >= G.ny) { if (G.per[1]) ty -= G.ny; else face = 3; }
    if (tz < 0) { if (G.per[2]) tz += G.nz; else face = 4; }
    else if (tz >= G.nz) { if (G.per[2]) tz -= G.nz; else face = 5; }
    if (face >= 0)
        idx = (long long)io * G.N + n;
    else
        idx = (long long)i * G.N + node_index(G, tx, ty, tz);
    return face;
}

// Load the pre-collision deviations s_i = f_i - w_i and s_gk = g_k - w_k T_ref
// of one node at parity p (generic path: any node, any boundary).
template <int D, typename S, typename R>
__device__ __forceinline__ void load_node(const Geo& G, const S* __restrict__ f, const S* __restrict__ g, int x, int y,
                                          int z, int parity, R* s, R* sg) {
    using L = Lat<D>;
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        long long idx;
        pop_slot(G, x, y, z, L::ex(i), L::ey(i), L::ez(i), i, L::opp(i), parity, idx);
        s[i] = (R)Store<S>::ldf(f[idx]);
    }
#pragma unroll
    for (int k = 0; k < L::QG; k++) {
        long long idx;
        int face = pop_slot(G, x, y, z, L::ex(k), L::ey(k), L::ez(k), k, L::opp(k), parity, idx);
        R v = (R)Store<S>::ldg(g[idx]);
        if (face_iso(G, face)) v = (R)(2.0 * L::wg(k) * face_dTw(G, face)) - v;
        sg[k] = v;
    }
}

// ------------------------------------------------------------------ context
// FP64 record of one contact's Mindlin-Deresiewicz loading history: tangential
// force (3), loading direction e (3), previous normal force, T*, T**, branch k
constexpr int MD_REC = 10;
struct DemCfg {
    int n;            // particles
    int dim;
    int nsub;         // substeps per lattice step
    double dt;        // 1 / nsub
    int law;
    float E_star, G_star, mu, kn, kt, gn, gt;
    double mu_d;      // mu in FP64 (the loading-history law evaluates in FP64)
    double g[3];      // particle gravity
    double lo[3], hi[3];  // wall planes (-0.5, n - 0.5)
    float lof[3], hif[3]; // the same in FP32 (prefilters)
    int walled[3];
    int nc[3];        // cells per axis
    double inv[3];    // nc / n per axis
    int ncell;
    double skin;      // neighbour-list margin
    int cap;          // capacity of the canonical pair list
    int maxnb;        // candidates per particle
    int per;          // particles per CTA of the DEM cluster
    const float* J;   // learned hydrodynamic Jacobian [n][SG_NJ] or null
    const int* J_on;  // device gate: apply J this step when non-zero
};

// learned coupling surrogate (surrogate.cu)
constexpr int SG_NFEAT = 12, SG_NOUT = 7;
// 12 -> 64 -> 64 -> 64 -> 7 tanh layers plus the 7 x 12 linear path
constexpr int SG_NPARAMS = 64 * 12 + 64 + 2 * (64 * 64 + 64) + 7 * 64 + 7 + 7 * 12;
constexpr int SG_NFSUM = 18;  // feature sums per particle from the footprint pass
constexpr int SG_ROWS = 8;    // network rows per particle: the state and seven perturbations
constexpr int SG_NJ = 19;     // Jacobian values per particle: J_FU (9), J_TW (9), J_HT
constexpr int SG_TRAIN_BLOCKS = 152;
constexpr int SG_NB_SLICES = 16;  // neighbour-feature slices of the particle set
struct Surrogate {
    float *params, *m, *v, *norm;   // FP32 master parameters, Adam moments, standardisation (38)
    unsigned char* wimg;             // BF16 weight image of the inference kernel (mlp_image_bytes())
    float *partial, *lossp;          // training reduction scratch
    int adam_t;
    int trained;                     // parameters set or trained
    int enabled;                     // Jacobian pipeline in the step graph
    int fixed;                       // a caller-supplied Jacobian is in use
    double bound, delta;
    int cap;                         // particles the per-particle buffers hold
    double* feat;                    // [n][12]
    double* fsum;                    // [n][SG_NFSUM] feature sums of the footprint pass
    float4* xr;                      // [n] FP32 positions and radii (neighbour prefilter)
    double* nbpart;                  // [slices][n][5] neighbour-feature partials
    float *rows, *yrows, *J;         // [SG_ROWS n][16], [SG_ROWS n][8], [n][SG_NJ]
    double* part;                    // gate partial sums
    int *J_on, *err;                 // device gate flag, tensor-core wait status
    int wait_polls;                  // poll limit of a tensor-core completion wait
    double* stats;                   // [on steps, off steps, last relative error]
};

struct Ctx {
    pibm_desc desc;
    int D, Q, QG;
    Geo G;
    int walls_kind[6];
    int walls_therm[6];
    double walls_T[6];
    double nu, alpha, tau_f, tau_g, buoy;
    long long t;
    size_t es;  // bytes per stored population element
    size_t v4;  // bytes per node of the F_B / Q_B and marker fields

    cudaStream_t s0;  // caller's stream
    cudaStream_t s1;  // internal stream for the DEM branch
    cudaStream_t s2;  // internal stream for the clear of the previous coupling set
    cudaEvent_t ev_fork, ev_join, ev_join2, ev_k1;
    pibm_allocator alloc;
    int own_s0;  // 1 if the library created s0

    // lattice buffers
    void* f;
    void* g;
    // coupling fields, double-buffered by time parity: the coupling of time t
    // writes set t & 1, the lattice step of time t reads it, and the set of the
    // other parity is cleared concurrently with that step
    void* fb[2];      // F_B (xyz) and Q_B (w) per node, valid on flagged tiles
    void* mk[2];      // marker field of covered nodes (eps * F_f, eps * Q)
    uint8_t* flags[2];  // one byte per 32-node tile along x
    double* plane;    // one plane of doubles (reads / writes through the API)
    double* red;      // reduction scratch
    int* dstat;       // device status words [code, detail]

    // particles
    int np;
    double *X, *U, *W, *Xb, *R, *rho, *Tp, *Cp, *m, *I, *mg;
    double *im, *iI;                 // 1/m, 1/I (computed on the host: no FP64 division on the device)
    uint8_t* fixed;
    double *Fh, *Th, *Hh;
    float *Fc, *Tc;  // contact force / torque of the last DEM evaluation (FP32, as the substeps form them)
    double *Fh_prev, *Th_prev, *Hh_prev;  // coupling of the previous time
    int* have_prev;   // device int: 1 once a previous coupling exists
    int* adj_start_new;  // scratch for the adjacency offsets of a rebuild
    int* box[2];      // spread box per particle and parity (lo xyz, hi xyz); empty = hi < lo
    DemCfg dem;
    int *cell_of, *cell_cnt, *cell_start, *cell_ids, *cnt_hi, *cnt_lo;
    int* nb_start[2];
    int* nb_i[2];
    int* nb_j[2];
    float* nb_ft[2];
    double* nb_md[2];  // Mindlin-Deresiewicz history per pair (law PIBM_HERTZ_MD_HIST), MD_REC doubles per entry
    double* wall_md;   // [n][6][MD_REC] the same for the wall contacts
    int* nb_cur;      // device ints: current list, current history buffer
    int *adj_start, *adj_nb, *adj_k;
    float* wall_ft;
    int adj_cap;
    int dem_cs;           // CTAs in the DEM cluster
    int tune_dem_particles_per_cta;  // 0: default (32)
    int tune_lattice_row_tiles;      // 1: lattice blocks span a divisor of the row (no block straddles a row end)
    int tune_coupling_threads;       // 0: default; threads per footprint / spread block
    int tune_coupling_order;         // 1 (default): coupling blocks take the particles in cell-list order
    int tune_lattice_threads;        // 0: default block shape; else threads per lattice block
    int tune_wide_index;             // 1: 64-bit slot offsets in the lattice kernel even where 32-bit suffice
    int tune_lattice_pairs;          // 1 (default): two nodes per thread in the even step of 16-bit storage
    int dem_attr_ok;                 // bit per DEM kernel variant (dimension, law) whose launch attributes are set
    int spread_smem;                 // shared memory per CTA of the spread kernel (from the largest radius)
    double rmax;                     // largest particle radius
    Surrogate sg;
    int lat;                         // lattice id: 2 D2Q9, 3 D3Q19, 4 D3Q15 (all with D2Q5 / D3Q7 thermal)
    int point;                       // particle model: 1 = one PIBM point per particle (d_p <= h)
    unsigned gen;                    // bumped whenever the captured step graphs become stale
    int* contact_pairs;   // 2 * dem.cap ints
    int* contact_scratch; // 2 * np + 4 ints

    // static markers
    int nm;
    double *MX, *MA, *MT, *nu_part, *nu_val;
    void* Ml;         // per-marker (A F_f, A Q)
    int n_csr_nodes;
    long long* csr_node;
    int *csr_start, *csr_marker;
    double* csr_w;

    // CUDA graphs: one lattice step starting at even / odd time
    cudaGraphExec_t graph[2];
    int graph_ok[2];
    cudaGraphExec_t tgraph[2];  // the step graph with event-record nodes around each kernel group (pibm_step_timed)
    int tgraph_ok[2];
    cudaEvent_t tev[8];         // its timing events (created on first use)
    int tev_ok;
    int kernels_per_step;

    std::string err;
};

// ---------------------------------------------------------- launch wrappers
// lattice.cu
cudaError_t launch_init_equilibrium(Ctx* c);
cudaError_t launch_stream_collide(Ctx* c, cudaStream_t s, int parity);
cudaError_t launch_read_plane(Ctx* c, int which, int plane, int parity);    // which: 0 f, 1 g
cudaError_t launch_write_plane(Ctx* c, int which, int plane, int parity);
cudaError_t launch_macro(Ctx* c, int field, int parity);
cudaError_t launch_diagnostics(Ctx* c, int parity);
cudaError_t launch_features(Ctx* c, cudaStream_t s, int parity, double* out);  // n x 12 surrogate features
// coupling.cu
cudaError_t launch_coupling(Ctx* c, cudaStream_t s, int parity);
cudaError_t launch_coupling_clear(Ctx* c, cudaStream_t s, int parity);
int spread_smem_bytes(int dim, double rmax, size_t v4);
cudaError_t launch_footprint_sums(Ctx* c, cudaStream_t s, int parity);  // surrogate feature sums of the state
int coupling_kernel_count(Ctx* c);
// dem.cu
cudaError_t launch_dem(Ctx* c, cudaStream_t s, int nsub);
cudaError_t launch_contacts(Ctx* c, int* d_pairs, int cap, int* d_count);
cudaError_t launch_cells(Ctx* c, int* d_cell);
int dem_cluster_size(Ctx* c);
int dem_max_particles();
// api.cu: message returned by pibm_last_error(NULL, ...)
void set_global_error(const std::string& msg);
int dem_max_per_cta();
// api.cu: for the ensemble (ensemble.cu)
cudaError_t record_step(Ctx* c, int parity, int* kernels, const cudaEvent_t* tev = nullptr);
// surrogate.cu
cudaError_t launch_mlp(Ctx* c, cudaStream_t s, const float* in, int rows, float* out);
cudaError_t launch_surrogate(Ctx* c, cudaStream_t s, int parity, bool need_sums);
int surrogate_kernel_count(Ctx* c);
cudaError_t train_batch(Ctx* c, cudaStream_t s, const float* xb, const float* yb, int B, float lr, float* grad_out,
                        double* loss_out);
cudaError_t launch_gather(cudaStream_t s, int B, const int* idx, const float* X, const float* Y, float* xb, float* yb);
size_t lsq_scratch_doubles();
size_t mlp_image_bytes();
cudaError_t launch_mlp_image(Ctx* c, cudaStream_t s);
cudaError_t launch_lsq(Ctx* c, cudaStream_t s, const float* X, const float* Y, long long n, double ridge, double* part,
                       int* status);
Ctx* ctx_state(pibm_ctx* ctx);
pibm_status ctx_ready(pibm_ctx* ctx);

}  // namespace pibm

// Host side of the C ABI declared in include/pibm.h: argument checks, device
// memory through the caller's allocator, set-up of particles and static
// markers, CUDA-graph capture of one lattice step per time parity, and the
// read-back calls.  All arithmetic of the step runs in the kernels of
// lattice.cu, coupling.cu and dem.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <random>
#include <string>
#include <vector>

#include "pibm_internal.cuh"

using namespace pibm;

struct pibm_ctx {
    Ctx c;
    std::vector<std::pair<void*, int>> allocs;  // (pointer, group): 0 lattice, 1 particles, 2 markers, 3 scratch
    double* hstage = nullptr;                   // pinned host staging for the per-step read-backs
    size_t hstage_n = 0;                        // its size in doubles
};

// Pinned host buffer of at least n doubles (grown on demand; null if the host
// cannot pin memory, and the caller then copies directly).
static double* host_stage(pibm_ctx* ctx, size_t n) {
    if (ctx->hstage_n >= n) return ctx->hstage;
    if (ctx->hstage) cudaFreeHost(ctx->hstage);
    ctx->hstage = nullptr;
    ctx->hstage_n = 0;
    if (cudaMallocHost((void**)&ctx->hstage, sizeof(double) * n) != cudaSuccess) {
        cudaGetLastError();
        ctx->hstage = nullptr;
        return nullptr;
    }
    ctx->hstage_n = n;
    return ctx->hstage;
}

static std::string g_create_error;

void pibm::set_global_error(const std::string& msg) { g_create_error = msg; }

enum { GRP_LATTICE = 0, GRP_PARTICLES = 1, GRP_MARKERS = 2, GRP_SCRATCH = 3, GRP_SURROGATE = 4, GRP_SG_PART = 5 };

#define PCHECK(call)                                                                         \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            ctx->c.err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
            return e_ == cudaErrorMemoryAllocation ? PIBM_ERR_OOM : PIBM_ERR_CUDA;           \
        }                                                                                    \
    } while (0)

static pibm_status fail(pibm_ctx* ctx, pibm_status s, const std::string& msg) {
    if (ctx) ctx->c.err = msg;
    return s;
}

static void* dalloc(pibm_ctx* ctx, size_t bytes, int group) {
    Ctx& c = ctx->c;
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (c.alloc.alloc) {
        p = c.alloc.alloc(bytes, c.alloc.user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        p = nullptr;
    }
    if (!p) return nullptr;
    if (cudaMemsetAsync(p, 0, bytes, c.s0) != cudaSuccess) {  // give the block back: nothing leaks
        if (c.alloc.free) c.alloc.free(p, c.alloc.user);
        else cudaFree(p);
        return nullptr;
    }
    ctx->allocs.push_back({p, group});
    return p;
}

static void dfree_group(pibm_ctx* ctx, int group) {
    Ctx& c = ctx->c;
    cudaStreamSynchronize(c.s0);
    std::vector<std::pair<void*, int>> keep;
    for (auto& a : ctx->allocs) {
        if (group >= 0 && a.second != group) {
            keep.push_back(a);
            continue;
        }
        if (c.alloc.free) c.alloc.free(a.first, c.alloc.user);
        else cudaFree(a.first);
    }
    ctx->allocs.swap(keep);
}

static void drop_graphs(Ctx& c) {
    c.gen++;  // graphs that captured this context (its own and any ensemble's) are stale
    for (int p = 0; p < 2; p++) {
        if (c.graph_ok[p]) cudaGraphExecDestroy(c.graph[p]);
        c.graph_ok[p] = 0;
        if (c.tgraph_ok[p]) cudaGraphExecDestroy(c.tgraph[p]);
        c.tgraph_ok[p] = 0;
    }
}

// Device status words written by kernels (sticky until particles are reset).
static pibm_status status_word(pibm_ctx* ctx, const int* st);

static pibm_status device_status(pibm_ctx* ctx) {
    Ctx& c = ctx->c;
    cudaError_t e = cudaStreamSynchronize(c.s0);
    if (e != cudaSuccess) return fail(ctx, PIBM_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
    int st[2] = {0, 0};
    e = cudaMemcpy(st, c.dstat, sizeof(st), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(ctx, PIBM_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
    return status_word(ctx, st);
}

// the device status word (code, detail) as a status and message
static pibm_status status_word(pibm_ctx* ctx, const int* st) {
    if (st[0] != 0) {
        const char* what = st[1] == 1   ? "more than 64 neighbour candidates for one particle"
                           : st[1] == 2 ? "a particle moved more than half the neighbour skin in one lattice step"
                           : st[1] == 3 ? "neighbour list capacity exceeded"
                                        : "neighbour list inconsistent";
        return fail(ctx, (pibm_status)st[0], std::string("device check failed: ") + what);
    }
    return PIBM_OK;
}

static pibm_status check_config(pibm_ctx* ctx) {
    Ctx& c = ctx->c;
    for (int a = 0; a < c.D; a++)
        if ((c.walls_kind[2 * a] == PIBM_PERIODIC) != (c.walls_kind[2 * a + 1] == PIBM_PERIODIC))
            return fail(ctx, PIBM_ERR_STATE, "both faces of an axis must be periodic or both walls");
    if (c.np > 0)
        for (int a = 0; a < c.D; a++)
            if (c.walls_kind[2 * a] == PIBM_PERIODIC)
                return fail(ctx, PIBM_ERR_STATE, "particles require walls on every axis");
    return PIBM_OK;
}

static void update_geo(Ctx& c) {
    for (int a = 0; a < 3; a++) c.G.per[a] = (a >= c.D) ? 1 : (c.walls_kind[2 * a] == PIBM_PERIODIC);
    c.G.iso = 0;
    for (int f = 0; f < 6; f++) {
        if ((f < 2 * c.D) && c.walls_kind[f] == PIBM_WALL && c.walls_therm[f] == PIBM_ISOTHERMAL) c.G.iso |= 1 << f;
        c.G.dTw[f] = c.walls_T[f] - c.desc.T_ref;
    }
    for (int a = 0; a < 3; a++) {
        c.dem.walled[a] = a < c.D && c.walls_kind[2 * a] == PIBM_WALL;
        int n = a == 0 ? c.G.nx : (a == 1 ? c.G.ny : c.G.nz);
        c.dem.lo[a] = -0.5;
        c.dem.hi[a] = n - 0.5;
        c.dem.lof[a] = -0.5f;
        c.dem.hif[a] = (float)(n - 0.5);
    }
}

static int parity(const Ctx& c) { return (int)(c.t & 1); }

// Coupling of the current time (after any change of state outside a step).
static pibm_status prime(pibm_ctx* ctx) {
    Ctx& c = ctx->c;
    PCHECK(launch_coupling_clear(&c, c.s0, parity(c)));
    PCHECK(launch_coupling(&c, c.s0, parity(c)));
    PCHECK(cudaStreamSynchronize(c.s0));
    return PIBM_OK;
}

// The launches of one lattice step at parity par, ordered on s0 with the
// DEM branch forked onto s1 and the clear of the other coupling set onto s2,
// both joined back before the coupling (s0 may be capturing).  The three
// branches touch disjoint data, so the DEM's latency-bound substeps, the
// clear and the bandwidth-bound lattice kernel overlap; the step's critical
// path is max(DEM, lattice) + coupling.
cudaError_t pibm::record_step(Ctx* cp, int par, int* kernels_out, const cudaEvent_t* tev) {
    Ctx& c = *cp;
    cudaError_t e = cudaSuccess;
    int kernels = 1;
    auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    // tev (timing graph only): event-record nodes around each kernel group
    auto mark = [&](int k, cudaStream_t s) { if (tev) chk(cudaEventRecordWithFlags(tev[k], s, cudaEventRecordExternal)); };
    mark(0, c.s0);
    chk(cudaEventRecord(c.ev_fork, c.s0));
    chk(cudaStreamWaitEvent(c.s1, c.ev_fork, 0));
    mark(2, c.s1);
    // The clear of the other coupling set runs beside the lattice kernel when that kernel is the
    // longer branch (it then costs nothing), and after it when the DEM is the longer branch (the
    // lattice kernel then runs without the clear's CTAs in the way and the clear still ends
    // before the DEM): estimated from the lattice kernel's bytes at 6.5 TB/s against ~2 us per
    // DEM substep.
    const double lattice_us = (double)c.G.N * 2.0 * (c.Q + c.QG) * (double)c.es / 6.5e6;
    const bool clear_after = c.np > 0 && lattice_us < 2.0 * c.desc.dem_substeps;
    if (c.np > 0) {
        chk(launch_dem(&c, c.s1, c.desc.dem_substeps));  // particles t -> t+1, concurrent, launched first
        if (!clear_after) {
            chk(cudaStreamWaitEvent(c.s2, c.ev_fork, 0));
            chk(launch_coupling_clear(&c, c.s2, par ^ 1));  // free the other coupling set (read at t-1)
            chk(cudaEventRecord(c.ev_join2, c.s2));
        }
        kernels++;
    }
    mark(3, c.s1);
    mark(7, c.s0);
    chk(launch_stream_collide(&c, c.s0, par));        // collide + stream, t -> t+1
    mark(1, c.s0);
    if (clear_after) {
        chk(cudaEventRecord(c.ev_k1, c.s0));
        chk(cudaStreamWaitEvent(c.s2, c.ev_k1, 0));
        chk(launch_coupling_clear(&c, c.s2, par ^ 1));
        chk(cudaEventRecord(c.ev_join2, c.s2));
    }
    chk(cudaEventRecord(c.ev_join, c.s1));
    chk(cudaStreamWaitEvent(c.s0, c.ev_join, 0));
    if (c.np > 0) chk(cudaStreamWaitEvent(c.s0, c.ev_join2, 0));
    mark(4, c.s0);
    chk(launch_coupling(&c, c.s0, par ^ 1));         // coupling of time t+1
    mark(5, c.s0);
    kernels += coupling_kernel_count(&c);
    if (c.sg.enabled && c.np > 0) {                  // surrogate Jacobian for the next step's DEM, checked against t+1's coupling
        chk(launch_surrogate(&c, c.s0, par ^ 1, false));  // the coupling left the feature sums
        kernels += surrogate_kernel_count(&c);
    }
    mark(6, c.s0);
    if (kernels_out) *kernels_out = kernels;
    return e;
}

pibm::Ctx* pibm::ctx_state(pibm_ctx* ctx) { return &ctx->c; }

pibm_status pibm::ctx_ready(pibm_ctx* ctx) { return check_config(ctx); }

extern "C" {

const char* pibm_status_string(pibm_status s) {
    switch (s) {
        case PIBM_OK: return "ok";
        case PIBM_ERR_ARG: return "invalid argument";
        case PIBM_ERR_OOM: return "out of device memory";
        case PIBM_ERR_CUDA: return "CUDA error";
        case PIBM_ERR_STATE: return "invalid state";
        case PIBM_ERR_UNSTABLE: return "non-finite values";
        case PIBM_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

int pibm_last_error(pibm_ctx* ctx, char* buf, size_t n) {
    const std::string& s = ctx ? ctx->c.err : g_create_error;
    if (buf && n) {
        size_t k = std::min(n - 1, s.size());
        memcpy(buf, s.data(), k);
        buf[k] = 0;
    }
    return (int)s.size();
}

pibm_status pibm_create(const pibm_desc* d, void* stream, const pibm_allocator* alloc, pibm_ctx** out) {
    if (!d || !out) return g_create_error = "null argument", PIBM_ERR_ARG;
    *out = nullptr;
    if ((d->dim != 2 && d->dim != 3) || d->nx < 1 || d->ny < 1 || d->nz < 1 || (d->dim == 2 && d->nz != 1))
        return g_create_error = "invalid lattice size", PIBM_ERR_ARG;
    if (d->storage != PIBM_STORE_F32 && d->storage != PIBM_STORE_F64 && d->storage != PIBM_STORE_F16 &&
        d->storage != PIBM_STORE_BF16)
        return g_create_error = "invalid storage", PIBM_ERR_ARG;
    if (!(d->Ra > 0) || !(d->Pr > 0) || !(d->U_c > 0) || !(d->L_c > 0) || d->gravity_axis < 0 ||
        d->gravity_axis >= d->dim || d->dem_substeps < 1 || d->nu_dT == 0.0)
        return g_create_error = "invalid physical parameters", PIBM_ERR_ARG;
    if ((long long)d->nx * d->ny * d->nz > (1LL << 31) - 1) return g_create_error = "lattice too large", PIBM_ERR_ARG;
    if (d->flow_q != 0 && !(d->dim == 2 && d->flow_q == 9) && !(d->dim == 3 && (d->flow_q == 19 || d->flow_q == 15)))
        return g_create_error = "flow lattice: 9 in 2-D, 19 or 15 in 3-D (0 = default)", PIBM_ERR_ARG;

    pibm_ctx* ctx = new pibm_ctx();
    Ctx& c = ctx->c;
    memset((void*)&c.desc, 0, sizeof(c.desc));
    c.desc = *d;
    c.D = d->dim;
    c.lat = c.D == 2 ? 2 : (d->flow_q == 15 ? 4 : 3);
    c.sg.wait_polls = 1 << 22;
    c.tune_coupling_order = 1;
    c.tune_lattice_pairs = 1;
    c.Q = c.D == 2 ? 9 : (c.lat == 4 ? 15 : 19);
    c.QG = c.D == 2 ? 5 : 7;
    c.G.nx = d->nx, c.G.ny = d->ny, c.G.nz = d->nz;
    c.G.N = (long long)d->nx * d->ny * d->nz;
    c.G.ntx = (d->nx + 31) / 32;
    c.es = d->storage == PIBM_STORE_F64 ? 8 : (d->storage == PIBM_STORE_F32 ? 4 : 2);
    c.v4 = d->storage == PIBM_STORE_F64 ? 32 : 16;  // F_B / Q_B and marker fields: double4 or float4
    // Eq lbm2.6: nu = U_c L_c sqrt(Pr / Ra); Eq lbm2.7 with Pr = nu / alpha
    c.nu = d->U_c * d->L_c * sqrt(d->Pr / d->Ra);
    c.alpha = c.nu / d->Pr;
    c.tau_f = 3.0 * c.nu + 0.5;
    c.tau_g = c.alpha * (c.D == 2 ? 3.0 : 4.0) + 0.5;
    c.buoy = d->U_c * d->U_c / d->L_c;
    c.t = 0;
    c.alloc = alloc ? *alloc : pibm_allocator{nullptr, nullptr, nullptr};
    for (int f = 0; f < 6; f++) c.walls_kind[f] = PIBM_PERIODIC, c.walls_therm[f] = PIBM_ADIABATIC, c.walls_T[f] = 0.0;
    c.graph_ok[0] = c.graph_ok[1] = 0;
    c.np = 0;
    c.nm = 0;

    cudaError_t e;
    if (stream) {
        c.s0 = (cudaStream_t)stream;
    } else if ((e = cudaStreamCreateWithFlags(&c.s0, cudaStreamNonBlocking)) != cudaSuccess) {
        delete ctx;
        return g_create_error = cudaGetErrorString(e), PIBM_ERR_CUDA;
    }
    c.own_s0 = stream ? 0 : 1;
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    // the DEM branch is latency-bound on a few SMs: give it the highest priority
    if ((e = cudaStreamCreateWithPriority(&c.s1, cudaStreamNonBlocking, prio_hi)) != cudaSuccess ||
        (e = cudaStreamCreateWithPriority(&c.s2, cudaStreamNonBlocking, prio_hi)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c.ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c.ev_join, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c.ev_join2, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c.ev_k1, cudaEventDisableTiming)) != cudaSuccess) {
        delete ctx;
        return g_create_error = cudaGetErrorString(e), PIBM_ERR_CUDA;
    }
    long long N = c.G.N;
    c.f = dalloc(ctx, (size_t)c.Q * N * c.es, GRP_LATTICE);
    c.g = dalloc(ctx, (size_t)c.QG * N * c.es, GRP_LATTICE);
    for (int b = 0; b < 2; b++) {
        c.fb[b] = dalloc(ctx, (size_t)N * c.v4, GRP_LATTICE);
        c.mk[b] = dalloc(ctx, (size_t)N * c.v4, GRP_LATTICE);
        c.flags[b] = (uint8_t*)dalloc(ctx, (size_t)c.G.ntx * d->ny * d->nz, GRP_LATTICE);
    }
    c.red = (double*)dalloc(ctx, sizeof(double) * (4 * 512 + 16), GRP_LATTICE);
    c.dstat = (int*)dalloc(ctx, sizeof(int) * 4, GRP_LATTICE);
    c.nu_val = (double*)dalloc(ctx, sizeof(double) * 2, GRP_LATTICE);
    c.nb_cur = (int*)dalloc(ctx, sizeof(int) * 2, GRP_LATTICE);
    c.plane = nullptr;
    if (!c.f || !c.g || !c.fb[0] || !c.mk[0] || !c.flags[0] || !c.fb[1] || !c.mk[1] || !c.flags[1] || !c.red ||
        !c.dstat || !c.nu_val || !c.nb_cur) {
        g_create_error = "device allocation failed";
        pibm_destroy(ctx);
        return PIBM_ERR_OOM;
    }
    update_geo(c);
    c.dem.n = 0;
    c.dem.dim = c.D;
    c.dem.nsub = d->dem_substeps;
    c.dem.dt = 1.0 / d->dem_substeps;
    c.dem.law = PIBM_SPRING_DASHPOT;
    if ((e = launch_init_equilibrium(&c)) != cudaSuccess || (e = cudaStreamSynchronize(c.s0)) != cudaSuccess) {
        g_create_error = cudaGetErrorString(e);
        pibm_destroy(ctx);
        return PIBM_ERR_CUDA;
    }
    c.kernels_per_step = 1;
    *out = ctx;
    return PIBM_OK;
}

pibm_status pibm_destroy(pibm_ctx* ctx) {
    if (!ctx) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    if (c.s0) cudaStreamSynchronize(c.s0);
    if (c.s1) cudaStreamSynchronize(c.s1);
    if (c.s2) cudaStreamSynchronize(c.s2);
    drop_graphs(c);
    dfree_group(ctx, -1);
    if (ctx->hstage) cudaFreeHost(ctx->hstage);
    if (c.ev_fork) cudaEventDestroy(c.ev_fork);
    if (c.ev_join) cudaEventDestroy(c.ev_join);
    if (c.ev_join2) cudaEventDestroy(c.ev_join2);
    if (c.ev_k1) cudaEventDestroy(c.ev_k1);
    if (c.tev_ok)
        for (int k = 0; k < 8; k++) cudaEventDestroy(c.tev[k]);
    if (c.s1) cudaStreamDestroy(c.s1);
    if (c.s2) cudaStreamDestroy(c.s2);
    if (c.own_s0 && c.s0) cudaStreamDestroy(c.s0);
    delete ctx;
    return PIBM_OK;
}

pibm_status pibm_set_wall(pibm_ctx* ctx, int face, int kind, int thermal, double T_w) {
    if (!ctx) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    if (face < 0 || face >= 2 * c.D || (kind != PIBM_PERIODIC && kind != PIBM_WALL) ||
        (thermal != PIBM_ADIABATIC && thermal != PIBM_ISOTHERMAL) || !isfinite(T_w))
        return fail(ctx, PIBM_ERR_ARG, "invalid wall");
    c.walls_kind[face] = kind;
    c.walls_therm[face] = thermal;
    c.walls_T[face] = T_w;
    update_geo(c);
    drop_graphs(c);
    return prime(ctx);
}

pibm_status pibm_set_contact_law(pibm_ctx* ctx, int law, double E, double poisson, double mu, double kn, double kt,
                                 double gamma_n, double gamma_t) {
    if (!ctx) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    const bool hertz = law == PIBM_HERTZ_MD || law == PIBM_HERTZ_MD_HIST;
    if ((law != PIBM_SPRING_DASHPOT && !hertz) || mu < 0 || (hertz && !(E > 0)) ||
        (hertz && !(poisson > -1 && poisson < 1)) || (law == PIBM_SPRING_DASHPOT && !(kn >= 0)))
        return fail(ctx, PIBM_ERR_ARG, "invalid contact law");
    // entering the loading-history law with particles in place: its FP64 records
    // were not kept by the other laws, so every contact's history starts afresh
    // (a contact's next update is then its first)
    if (law == PIBM_HERTZ_MD_HIST && c.dem.law != PIBM_HERTZ_MD_HIST && c.np > 0) {
        for (int b = 0; b < 2; b++)
            PCHECK(cudaMemsetAsync(c.nb_md[b], 0, sizeof(double) * 2 * MD_REC * c.dem.cap, c.s0));
        PCHECK(cudaMemsetAsync(c.wall_md, 0, sizeof(double) * 6 * MD_REC * (c.np + 1), c.s0));
    }
    c.dem.law = law;
    // text after Eq demgov: 1/E* = (1 - nu^2)/E_1 + (1 - nu^2)/E_2, same for G*; equal materials
    double Estar = hertz ? E / (2.0 * (1.0 - poisson * poisson)) : 0.0;
    double G = hertz ? E / (2.0 * (1.0 + poisson)) : 0.0;
    double Gstar = hertz ? G / (2.0 * (1.0 - poisson * poisson)) : 0.0;
    c.dem.E_star = (float)Estar;
    c.dem.G_star = (float)Gstar;
    c.dem.mu = (float)mu;
    c.dem.mu_d = mu;
    c.dem.kn = (float)kn;
    c.dem.kt = (float)kt;
    c.dem.gn = (float)gamma_n;
    c.dem.gt = (float)gamma_t;
    drop_graphs(c);
    return PIBM_OK;
}

pibm_status pibm_set_particles(pibm_ctx* ctx, int n, const double* X, const double* U, const double* W, const double* R,
                               const double* rho_p, const double* T_p, const double* heat_cap, const uint8_t* fixed) {
    if (!ctx) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    if (n < 0 || (n > 0 && (!X || !R || !rho_p))) return fail(ctx, PIBM_ERR_ARG, "invalid particle arrays");
    if (n > 0 && c.nm > 0) return fail(ctx, PIBM_ERR_STATE, "static markers and particles cannot be combined");
    int nn[3] = {c.G.nx, c.G.ny, c.G.nz};
    double rmax = 0.0;
    for (int p = 0; p < n; p++) {
        if (!(R[p] > 0) || !(rho_p[p] > 0)) return fail(ctx, PIBM_ERR_ARG, "particle radius and density must be positive");
        if (R[p] > 600.0) return fail(ctx, PIBM_ERR_ARG, "particle radius above 600 nodes");
        for (int a = 0; a < c.D; a++)
            if (!(X[3 * p + a] > -0.5 && X[3 * p + a] < nn[a] - 0.5))
                return fail(ctx, PIBM_ERR_ARG, "particle centre outside the domain");
        rmax = std::max(rmax, R[p]);
    }
    if (n > 0)
        for (int a = 0; a < c.D; a++)
            if (c.walls_kind[2 * a] == PIBM_PERIODIC || c.walls_kind[2 * a + 1] == PIBM_PERIODIC)
                return fail(ctx, PIBM_ERR_STATE, "particles require walls on every axis");
    double cmin = c.desc.cell_size > 0 ? c.desc.cell_size : 2.0 * rmax + 1.5;
    if (n > 0 && cmin < 2.0 * rmax + 1.0)
        return fail(ctx, PIBM_ERR_ARG, "cell size must be at least the largest diameter plus one node");
    if (n > dem_max_particles()) return fail(ctx, PIBM_ERR_ARG, "too many particles for one DEM cluster");
    if (c.point)
        for (int p = 0; p < n; p++)
            if (R[p] > 0.5) return fail(ctx, PIBM_ERR_ARG, "point particles need a diameter of at most one node");
    if (c.point && n > 0)
        for (int a = 0; a < c.D; a++)
            if ((a == 0 ? c.G.nx : a == 1 ? c.G.ny : c.G.nz) < 4)
                return fail(ctx, PIBM_ERR_ARG, "point particles need at least 4 nodes per axis");

    drop_graphs(c);
    dfree_group(ctx, GRP_PARTICLES);
    c.np = 0;
    c.dem.n = 0;
    // a new particle set invalidates any hydrodynamic Jacobian (surrogate or fixed)
    c.sg.enabled = 0;
    c.sg.fixed = 0;
    c.dem.J = nullptr;
    c.dem.J_on = nullptr;
    for (int b = 0; b < 2; b++) {
        PCHECK(cudaMemsetAsync(c.mk[b], 0, (size_t)c.G.N * c.v4, c.s0));
        PCHECK(cudaMemsetAsync(c.fb[b], 0, (size_t)c.G.N * c.v4, c.s0));
        PCHECK(cudaMemsetAsync(c.flags[b], 0, (size_t)c.G.ntx * c.G.ny * c.G.nz, c.s0));
    }
    PCHECK(cudaMemsetAsync(c.dstat, 0, sizeof(int) * 4, c.s0));
    PCHECK(cudaMemsetAsync(c.nb_cur, 0, sizeof(int) * 2, c.s0));
    if (n == 0) return prime(ctx);

    // host-side derived quantities (FP64): mass, moment of inertia, buoyant weight factor
    const double PI = 3.14159265358979323846;
    std::vector<double> hX(3 * n), hU(3 * n, 0.0), hW(3 * n, 0.0), hR(n), hrho(n), hT(n, 0.0), hC(n, 0.0), hm(n), hI(n), hmg(n);
    std::vector<uint8_t> hfix(n, 0);
    std::vector<int> hbox(6 * n);
    for (int p = 0; p < n; p++) {
        for (int a = 0; a < 3; a++) {
            hX[3 * p + a] = X[3 * p + a];
            if (U) hU[3 * p + a] = U[3 * p + a];
            if (W) hW[3 * p + a] = W[3 * p + a];
        }
        if (c.D == 2) {
            hX[3 * p + 2] = 0.0;
            hU[3 * p + 2] = 0.0;
            hW[3 * p] = hW[3 * p + 1] = 0.0;
        }
        hR[p] = R[p];
        hrho[p] = rho_p[p];
        if (T_p) hT[p] = T_p[p];
        if (heat_cap) hC[p] = heat_cap[p];
        if (fixed) hfix[p] = fixed[p];
        if (c.D == 2) {
            hm[p] = hrho[p] * PI * R[p] * R[p];
            hI[p] = 0.5 * hm[p] * R[p] * R[p];
        } else {
            hm[p] = hrho[p] * 4.0 / 3.0 * PI * R[p] * R[p] * R[p];
            hI[p] = 0.4 * hm[p] * R[p] * R[p];
        }
        hmg[p] = hm[p] * (1.0 - 1.0 / hrho[p]);  // Eq demgov: m (1 - rho_f / rho_p), rho_f = 1
        for (int a = 0; a < 3; a++) hbox[6 * p + a] = 0, hbox[6 * p + 3 + a] = -1;
    }
    // cell grid: nc_a = floor(n_a / cell_min), side n_a / nc_a >= cell_min >= 2 R_max + skin
    DemCfg& C = c.dem;
    C.n = n;
    C.dim = c.D;
    C.nsub = c.desc.dem_substeps;
    C.dt = 1.0 / c.desc.dem_substeps;
    for (int a = 0; a < 3; a++) C.g[a] = c.desc.g_particle[a];
    C.ncell = 1;
    for (int a = 0; a < 3; a++) {
        C.nc[a] = 1;
        C.inv[a] = 1.0 / (double)nn[a];
        if (a < c.D) {
            C.nc[a] = std::max(1, (int)floor((double)nn[a] / cmin));
            C.inv[a] = (double)C.nc[a] / (double)nn[a];
        }
        C.ncell *= C.nc[a];
    }
    C.skin = cmin - 2.0 * rmax;
    c.spread_smem = spread_smem_bytes(c.D, rmax, c.v4);
    c.rmax = rmax;
    C.cap = std::max(64, 16 * n);
    C.maxnb = 64;
    c.adj_cap = 2 * C.cap;
    update_geo(c);

    size_t v3 = sizeof(double) * 3 * (n + 1), v1 = sizeof(double) * (n + 1), v3f = sizeof(float) * 3 * (n + 1);
    auto A = [&](size_t b) { return dalloc(ctx, b, GRP_PARTICLES); };
    c.X = (double*)A(v3), c.U = (double*)A(v3), c.W = (double*)A(v3), c.Xb = (double*)A(v3);
    c.R = (double*)A(v1), c.rho = (double*)A(v1), c.Tp = (double*)A(v1), c.Cp = (double*)A(v1);
    c.m = (double*)A(v1), c.I = (double*)A(v1), c.mg = (double*)A(v1);
    c.im = (double*)A(v1), c.iI = (double*)A(v1);
    c.fixed = (uint8_t*)A(n + 1);
    c.Fh = (double*)A(v3), c.Th = (double*)A(v3), c.Hh = (double*)A(v1), c.Fc = (float*)A(v3f), c.Tc = (float*)A(v3f);
    c.Fh_prev = (double*)A(v3), c.Th_prev = (double*)A(v3), c.Hh_prev = (double*)A(v1);
    c.have_prev = (int*)A(sizeof(int) * 2);
    c.adj_start_new = (int*)A(sizeof(int) * (n + 2));
    c.box[0] = (int*)A(sizeof(int) * 6 * (n + 1));
    c.box[1] = (int*)A(sizeof(int) * 6 * (n + 1));
    c.cell_of = (int*)A(sizeof(int) * (n + 1));
    c.cell_cnt = (int*)A(sizeof(int) * (C.ncell + 1));
    c.cell_start = (int*)A(sizeof(int) * (C.ncell + 2));
    c.cell_ids = (int*)A(sizeof(int) * (n + 1));
    c.cnt_hi = (int*)A(sizeof(int) * (n + 1));
    c.cnt_lo = (int*)A(sizeof(int) * (n + 1));
    for (int b = 0; b < 2; b++) {
        c.nb_start[b] = (int*)A(sizeof(int) * (n + 2));
        c.nb_i[b] = (int*)A(sizeof(int) * C.cap);
        c.nb_j[b] = (int*)A(sizeof(int) * C.cap);
        c.nb_ft[b] = (float*)A(sizeof(float4) * 2 * C.cap);  // two substep buffers of (history, stamp)
        c.nb_md[b] = (double*)A(sizeof(double) * 2 * MD_REC * C.cap);  // two substep buffers (loading history)
    }
    c.adj_start = (int*)A(sizeof(int) * (n + 2));
    c.adj_nb = (int*)A(sizeof(int) * c.adj_cap);
    c.adj_k = (int*)A(sizeof(int) * c.adj_cap);
    c.wall_ft = (float*)A(sizeof(float) * 18 * (n + 1));
    c.wall_md = (double*)A(sizeof(double) * 6 * MD_REC * (n + 1));
    c.contact_pairs = (int*)A(sizeof(int) * 2 * C.cap);
    c.contact_scratch = (int*)A(sizeof(int) * (2 * n + 8));
    void* need[] = {c.X, c.U, c.W, c.Xb, c.R, c.rho, c.Tp, c.Cp, c.m, c.I, c.mg, c.im, c.iI, c.fixed, c.Fh, c.Th, c.Hh, c.Fc,
                    c.Fh_prev, c.Th_prev, c.Hh_prev, c.have_prev, c.adj_start_new,
                    c.Tc, c.box[0], c.box[1], c.cell_of, c.cell_cnt, c.cell_start, c.cell_ids, c.cnt_hi, c.cnt_lo, c.nb_start[0],
                    c.nb_start[1], c.nb_i[0], c.nb_i[1], c.nb_j[0], c.nb_j[1], c.nb_ft[0], c.nb_ft[1], c.adj_start,
                    c.adj_nb, c.adj_k, c.wall_ft, c.contact_pairs, c.contact_scratch, c.nb_md[0], c.nb_md[1], c.wall_md};
    for (void* p : need)
        if (!p) {
            dfree_group(ctx, GRP_PARTICLES);
            return fail(ctx, PIBM_ERR_OOM, "particle buffers: device allocation failed");
        }
    auto up = [&](void* dst, const void* src, size_t b) { return cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, c.s0); };
    PCHECK(up(c.X, hX.data(), sizeof(double) * 3 * n));
    PCHECK(up(c.U, hU.data(), sizeof(double) * 3 * n));
    PCHECK(up(c.W, hW.data(), sizeof(double) * 3 * n));
    PCHECK(up(c.R, hR.data(), sizeof(double) * n));
    PCHECK(up(c.rho, hrho.data(), sizeof(double) * n));
    PCHECK(up(c.Tp, hT.data(), sizeof(double) * n));
    PCHECK(up(c.Cp, hC.data(), sizeof(double) * n));
    PCHECK(up(c.m, hm.data(), sizeof(double) * n));
    {
        std::vector<double> him(n), hiI(n);
        for (int p = 0; p < n; p++) him[p] = 1.0 / hm[p], hiI[p] = 1.0 / hI[p];
        PCHECK(up(c.im, him.data(), sizeof(double) * n));
        PCHECK(up(c.iI, hiI.data(), sizeof(double) * n));
    }
    PCHECK(up(c.I, hI.data(), sizeof(double) * n));
    PCHECK(up(c.mg, hmg.data(), sizeof(double) * n));
    PCHECK(up(c.fixed, hfix.data(), n));
    PCHECK(up(c.box[0], hbox.data(), sizeof(int) * 6 * n));
    PCHECK(up(c.box[1], hbox.data(), sizeof(int) * 6 * n));
    PCHECK(cudaStreamSynchronize(c.s0));  // host vectors go out of scope
    c.np = n;
    c.dem_cs = dem_cluster_size(&c);
    if ((n + c.dem_cs - 1) / c.dem_cs > dem_max_per_cta()) {
        c.np = 0;
        dfree_group(ctx, GRP_PARTICLES);
        return fail(ctx, PIBM_ERR_ARG, "too many particles for one DEM cluster on this device");
    }
    // neighbour list at the initial positions, then the coupling of the current time
    PCHECK(launch_dem(&c, c.s0, 0));
    pibm_status st = device_status(ctx);
    if (st != PIBM_OK) return st;
    return prime(ctx);
}

pibm_status pibm_set_markers(pibm_ctx* ctx, int n, const double* X, const double* A, const double* T_p) {
    if (!ctx) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    if (n < 0 || (n > 0 && (!X || !A || !T_p))) return fail(ctx, PIBM_ERR_ARG, "invalid marker arrays");
    if (n > 0 && c.np > 0) return fail(ctx, PIBM_ERR_STATE, "static markers and particles cannot be combined");
    int nn[3] = {c.G.nx, c.G.ny, c.G.nz};
    for (int l = 0; l < n; l++)
        for (int a = 0; a < c.D; a++) {
            double x = X[3 * l + a];
            if (!isfinite(x)) return fail(ctx, PIBM_ERR_ARG, "non-finite marker position");
            bool per = c.walls_kind[2 * a] == PIBM_PERIODIC;
            if (!per && (floor(x) - 1 < 0 || floor(x) + 2 > nn[a] - 1))
                return fail(ctx, PIBM_ERR_ARG, "marker interpolation stencil leaves the lattice");
        }
    drop_graphs(c);
    dfree_group(ctx, GRP_MARKERS);
    c.nm = 0;
    for (int b = 0; b < 2; b++) {
        PCHECK(cudaMemsetAsync(c.fb[b], 0, (size_t)c.G.N * c.v4, c.s0));
        PCHECK(cudaMemsetAsync(c.flags[b], 0, (size_t)c.G.ntx * c.G.ny * c.G.nz, c.s0));
    }
    if (n == 0) return prime(ctx);
    // node -> (marker, weight) lists for the spreading gather; delta_h of Eq lbm12
    const double PI = 3.14159265358979323846;
    auto dh = [&](double a) { return fabs(a) <= 2.0 ? 0.25 * (1.0 + cos(PI * a / 2.0)) : 0.0; };
    struct E3 { long long node; int l; double w; };
    std::vector<E3> ent;
    for (int l = 0; l < n; l++) {
        int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int a = 0; a < c.D; a++) lo[a] = (int)ceil(X[3 * l + a] - 2.0), hi[a] = (int)floor(X[3 * l + a] + 2.0);
        for (int z = lo[2]; z <= hi[2]; z++)
            for (int y = lo[1]; y <= hi[1]; y++)
                for (int x = lo[0]; x <= hi[0]; x++) {
                    int cc[3] = {x, y, z};
                    bool skip = false;
                    for (int a = 0; a < c.D; a++) {
                        if (cc[a] < 0 || cc[a] >= nn[a]) {
                            if (c.walls_kind[2 * a] != PIBM_PERIODIC) skip = true;
                            cc[a] = ((cc[a] % nn[a]) + nn[a]) % nn[a];
                        }
                    }
                    if (skip) continue;
                    double w = dh(x - X[3 * l]) * dh(y - X[3 * l + 1]);
                    if (c.D == 3) w *= dh(z - X[3 * l + 2]);
                    if (w == 0.0) continue;
                    ent.push_back({node_index(c.G, cc[0], cc[1], cc[2]), l, w});
                }
    }
    std::stable_sort(ent.begin(), ent.end(), [](const E3& a, const E3& b) { return a.node < b.node; });
    std::vector<long long> nodes;
    std::vector<int> start, mk;
    std::vector<double> wt;
    for (size_t k = 0; k < ent.size(); k++) {
        if (k == 0 || ent[k].node != ent[k - 1].node) {
            nodes.push_back(ent[k].node);
            start.push_back((int)k);
        }
        mk.push_back(ent[k].l);
        wt.push_back(ent[k].w);
    }
    start.push_back((int)ent.size());
    std::vector<uint8_t> hflags((size_t)c.G.ntx * c.G.ny * c.G.nz, 0);
    for (long long nd : nodes) {
        long long x = nd % c.G.nx, yz = nd / c.G.nx;
        hflags[yz * c.G.ntx + (x >> 5)] = 1;
    }
    std::vector<double> hX(3 * n);
    for (int l = 0; l < n; l++)
        for (int a = 0; a < 3; a++) hX[3 * l + a] = a < c.D ? X[3 * l + a] : 0.0;
    c.n_csr_nodes = (int)nodes.size();
    auto Al = [&](size_t b) { return dalloc(ctx, b, GRP_MARKERS); };
    c.MX = (double*)Al(sizeof(double) * 3 * n);
    c.MA = (double*)Al(sizeof(double) * n);
    c.MT = (double*)Al(sizeof(double) * n);
    c.nu_part = (double*)Al(sizeof(double) * n);
    c.Ml = Al((size_t)n * c.v4);
    c.csr_node = (long long*)Al(sizeof(long long) * nodes.size());
    c.csr_start = (int*)Al(sizeof(int) * start.size());
    c.csr_marker = (int*)Al(sizeof(int) * mk.size());
    c.csr_w = (double*)Al(sizeof(double) * wt.size());
    if (!c.MX || !c.MA || !c.MT || !c.nu_part || !c.Ml || !c.csr_node || !c.csr_start || !c.csr_marker || !c.csr_w) {
        dfree_group(ctx, GRP_MARKERS);
        return fail(ctx, PIBM_ERR_OOM, "marker buffers: device allocation failed");
    }
    PCHECK(cudaMemcpy(c.MX, hX.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice));
    PCHECK(cudaMemcpy(c.MA, A, sizeof(double) * n, cudaMemcpyHostToDevice));
    PCHECK(cudaMemcpy(c.MT, T_p, sizeof(double) * n, cudaMemcpyHostToDevice));
    PCHECK(cudaMemcpy(c.csr_node, nodes.data(), sizeof(long long) * nodes.size(), cudaMemcpyHostToDevice));
    PCHECK(cudaMemcpy(c.csr_start, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice));
    PCHECK(cudaMemcpy(c.csr_marker, mk.data(), sizeof(int) * mk.size(), cudaMemcpyHostToDevice));
    PCHECK(cudaMemcpy(c.csr_w, wt.data(), sizeof(double) * wt.size(), cudaMemcpyHostToDevice));
    PCHECK(cudaMemcpy(c.flags[0], hflags.data(), hflags.size(), cudaMemcpyHostToDevice));  // static: both parities
    PCHECK(cudaMemcpy(c.flags[1], hflags.data(), hflags.size(), cudaMemcpyHostToDevice));
    c.nm = n;
    return prime(ctx);
}

static pibm_status ensure_plane(pibm_ctx* ctx) {
    Ctx& c = ctx->c;
    if (!c.plane) c.plane = (double*)dalloc(ctx, sizeof(double) * c.G.N, GRP_SCRATCH);
    return c.plane ? PIBM_OK : fail(ctx, PIBM_ERR_OOM, "read buffer: device allocation failed");
}

pibm_status pibm_set_populations(pibm_ctx* ctx, const double* f, const double* g) {
    if (!ctx) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    pibm_status st = ensure_plane(ctx);
    if (st != PIBM_OK) return st;
    for (int which = 0; which < 2; which++) {
        const double* src = which == 0 ? f : g;
        if (!src) continue;
        int nq = which == 0 ? c.Q : c.QG;
        for (int q = 0; q < nq; q++) {
            PCHECK(cudaMemcpyAsync(c.plane, src + (size_t)q * c.G.N, sizeof(double) * c.G.N, cudaMemcpyHostToDevice, c.s0));
            PCHECK(launch_write_plane(&c, which, q, parity(c)));
        }
    }
    return prime(ctx);
}

static pibm_status capture(pibm_ctx* ctx, int par, bool timed = false) {
    Ctx& c = ctx->c;
    cudaGraph_t graph;
    PCHECK(cudaStreamBeginCapture(c.s0, cudaStreamCaptureModeThreadLocal));
    int kernels = 0;
    cudaError_t e = record_step(&c, par, &kernels, timed ? c.tev : nullptr);
    cudaError_t e2 = cudaStreamEndCapture(c.s0, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (e2 == cudaSuccess) cudaGraphDestroy(graph);
        return fail(ctx, PIBM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(timed ? &c.tgraph[par] : &c.graph[par], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(ctx, PIBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    if (timed) {
        c.tgraph_ok[par] = 1;
    } else {
        c.graph_ok[par] = 1;
        c.kernels_per_step = kernels;
    }
    return PIBM_OK;
}

pibm_status pibm_step(pibm_ctx* ctx, int nsteps) {
    if (!ctx) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    if (nsteps < 0) return fail(ctx, PIBM_ERR_ARG, "negative step count");
    pibm_status st = check_config(ctx);
    if (st != PIBM_OK) return st;
    for (int k = 0; k < nsteps; k++) {
        int par = parity(c);
        if (!c.graph_ok[par]) {
            st = capture(ctx, par);
            if (st != PIBM_OK) return st;
        }
        PCHECK(cudaGraphLaunch(c.graph[par], c.s0));
        c.t++;
    }
    return PIBM_OK;
}

pibm_status pibm_step_timed(pibm_ctx* ctx, double* ms) {
    if (!ctx || !ms) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    pibm_status st = check_config(ctx);
    if (st != PIBM_OK) return st;
    if (!c.tev_ok) {
        for (int k = 0; k < 8; k++) PCHECK(cudaEventCreate(&c.tev[k]));
        c.tev_ok = 1;
    }
    const int par = parity(c);
    if (!c.tgraph_ok[par]) {
        st = capture(ctx, par, true);
        if (st != PIBM_OK) return st;
    }
    PCHECK(cudaGraphLaunch(c.tgraph[par], c.s0));
    PCHECK(cudaEventSynchronize(c.tev[6]));
    float t[4] = {0, 0, 0, 0};
    PCHECK(cudaEventElapsedTime(&t[0], c.tev[7], c.tev[1]));  // collide-and-stream
    PCHECK(cudaEventElapsedTime(&t[1], c.tev[2], c.tev[3]));  // DEM
    PCHECK(cudaEventElapsedTime(&t[2], c.tev[4], c.tev[5]));  // coupling
    PCHECK(cudaEventElapsedTime(&t[3], c.tev[0], c.tev[6]));  // whole step
    for (int k = 0; k < 4; k++) ms[k] = t[k];
    c.t++;
    return device_status(ctx);
}

pibm_status pibm_read_field(pibm_ctx* ctx, int field, double* dst, size_t n) {
    if (!ctx || !dst) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    if (field < PIBM_RHO || field > PIBM_QB || n != (size_t)c.G.N) return fail(ctx, PIBM_ERR_ARG, "invalid field request");
    pibm_status st = ensure_plane(ctx);
    if (st != PIBM_OK) return st;
    PCHECK(launch_macro(&c, field, parity(c)));
    PCHECK(cudaMemcpyAsync(dst, c.plane, sizeof(double) * n, cudaMemcpyDeviceToHost, c.s0));
    return device_status(ctx);
}

pibm_status pibm_read_populations(pibm_ctx* ctx, double* f, double* g) {
    if (!ctx) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    pibm_status st = ensure_plane(ctx);
    if (st != PIBM_OK) return st;
    for (int which = 0; which < 2; which++) {
        double* dst = which == 0 ? f : g;
        if (!dst) continue;
        int nq = which == 0 ? c.Q : c.QG;
        for (int q = 0; q < nq; q++) {
            PCHECK(launch_read_plane(&c, which, q, parity(c)));
            PCHECK(cudaMemcpyAsync(dst + (size_t)q * c.G.N, c.plane, sizeof(double) * c.G.N, cudaMemcpyDeviceToHost, c.s0));
        }
    }
    return device_status(ctx);
}

pibm_status pibm_read_particles(pibm_ctx* ctx, double* X, double* U, double* W, double* T_p) {
    if (!ctx) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    int n = c.np;
    // per-step read-back path: the state and the device status word go into one
    // pinned buffer with asynchronous copies, one synchronisation, then host copies
    double* h = n > 0 ? host_stage(ctx, (size_t)10 * n + 1) : nullptr;
    if (h) {
        PCHECK(cudaMemcpyAsync(h, c.X, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c.s0));
        PCHECK(cudaMemcpyAsync(h + 3 * n, c.U, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c.s0));
        PCHECK(cudaMemcpyAsync(h + 6 * n, c.W, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c.s0));
        PCHECK(cudaMemcpyAsync(h + 9 * n, c.Tp, sizeof(double) * n, cudaMemcpyDeviceToHost, c.s0));
        PCHECK(cudaMemcpyAsync(h + 10 * n, c.dstat, sizeof(int) * 2, cudaMemcpyDeviceToHost, c.s0));
        cudaError_t e = cudaStreamSynchronize(c.s0);
        if (e != cudaSuccess) return fail(ctx, PIBM_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
        if (X) memcpy(X, h, sizeof(double) * 3 * n);
        if (U) memcpy(U, h + 3 * n, sizeof(double) * 3 * n);
        if (W) memcpy(W, h + 6 * n, sizeof(double) * 3 * n);
        if (T_p) memcpy(T_p, h + 9 * n, sizeof(double) * n);
        int st[2];
        memcpy(st, h + 10 * n, sizeof(st));
        return status_word(ctx, st);
    }
    if (n > 0) {
        if (X) PCHECK(cudaMemcpyAsync(X, c.X, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c.s0));
        if (U) PCHECK(cudaMemcpyAsync(U, c.U, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c.s0));
        if (W) PCHECK(cudaMemcpyAsync(W, c.W, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c.s0));
        if (T_p) PCHECK(cudaMemcpyAsync(T_p, c.Tp, sizeof(double) * n, cudaMemcpyDeviceToHost, c.s0));
    }
    return device_status(ctx);
}

pibm_status pibm_read_particle_forces(pibm_ctx* ctx, double* F, double* T, double* H) {
    if (!ctx) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    int n = c.np;
    if (n > 0) {
        if (F) PCHECK(cudaMemcpyAsync(F, c.Fh, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c.s0));
        if (T) PCHECK(cudaMemcpyAsync(T, c.Th, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c.s0));
        if (H) PCHECK(cudaMemcpyAsync(H, c.Hh, sizeof(double) * n, cudaMemcpyDeviceToHost, c.s0));
    }
    return device_status(ctx);
}

pibm_status pibm_nusselt(pibm_ctx* ctx, double* nu) {
    if (!ctx || !nu) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    *nu = 0.0;
    if (c.nm > 0) PCHECK(cudaMemcpyAsync(nu, c.nu_val, sizeof(double), cudaMemcpyDeviceToHost, c.s0));
    return device_status(ctx);
}

pibm_status pibm_read_contacts(pibm_ctx* ctx, int32_t* pairs, int cap, int* n_out) {
    if (!ctx || !n_out || cap < 0 || (cap > 0 && !pairs)) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    *n_out = 0;
    if (c.np == 0) return device_status(ctx);
    pibm_status st = device_status(ctx);
    if (st != PIBM_OK) return st;
    PCHECK(launch_contacts(&c, c.contact_pairs, c.dem.cap, c.contact_scratch));
    int total = 0;
    PCHECK(cudaMemcpyAsync(&total, c.contact_scratch, sizeof(int), cudaMemcpyDeviceToHost, c.s0));
    PCHECK(cudaStreamSynchronize(c.s0));
    *n_out = total;
    int k = std::min(cap, total);
    if (k > 0) PCHECK(cudaMemcpy(pairs, c.contact_pairs, sizeof(int) * 2 * k, cudaMemcpyDeviceToHost));
    return device_status(ctx);
}

pibm_status pibm_read_cells(pibm_ctx* ctx, int32_t* cell, int32_t* ncell) {
    if (!ctx) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    if (ncell)
        for (int a = 0; a < 3; a++) ncell[a] = c.np > 0 ? c.dem.nc[a] : 0;
    if (c.np > 0 && cell) {
        PCHECK(launch_cells(&c, c.cell_of));
        PCHECK(cudaMemcpyAsync(cell, c.cell_of, sizeof(int) * c.np, cudaMemcpyDeviceToHost, c.s0));
    }
    return device_status(ctx);
}

pibm_status pibm_diagnostics(pibm_ctx* ctx, double* out) {
    if (!ctx || !out) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    PCHECK(launch_diagnostics(&c, parity(c)));
    PCHECK(cudaMemcpyAsync(out, c.red + 4 * 512, sizeof(double) * 6, cudaMemcpyDeviceToHost, c.s0));
    pibm_status st = device_status(ctx);
    if (st != PIBM_OK) return st;
    if (out[5] != 0.0) return fail(ctx, PIBM_ERR_UNSTABLE, "non-finite values in the lattice or particle state");
    return PIBM_OK;
}

pibm_status pibm_relaxation(pibm_ctx* ctx, double* out) {
    if (!ctx || !out) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    out[0] = c.nu, out[1] = c.alpha, out[2] = c.tau_f, out[3] = c.tau_g, out[4] = c.buoy;
    return PIBM_OK;
}

pibm_status pibm_time(pibm_ctx* ctx, int64_t* t) {
    if (!ctx || !t) return PIBM_ERR_ARG;
    *t = ctx->c.t;
    return PIBM_OK;
}

pibm_status pibm_set_tuning(pibm_ctx* ctx, int knob, int value) {
    if (!ctx) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    if (knob == PIBM_TUNE_LATTICE_THREADS) {
        if (value != 0 && (value < 32 || value > 512 || value % 32 != 0))
            return fail(ctx, PIBM_ERR_ARG, "lattice threads per block: 0 or a multiple of 32 in [32, 512]");
        c.tune_lattice_threads = value;
        drop_graphs(c);
        return PIBM_OK;
    }
    if (knob == PIBM_TUNE_LATTICE_ROW_TILES) {
        if (value != 0 && value != 1) return fail(ctx, PIBM_ERR_ARG, "invalid tuning value");
        c.tune_lattice_row_tiles = value;
        drop_graphs(c);
        return PIBM_OK;
    }
    if (knob == PIBM_TUNE_COUPLING_THREADS) {
        if (value != 0 && (value < 64 || value > 256 || value % 32 != 0))
            return fail(ctx, PIBM_ERR_ARG, "coupling threads per block: 0 or a multiple of 32 in [64, 256]");
        c.tune_coupling_threads = value;
        drop_graphs(c);
        return PIBM_OK;
    }
    if (knob == PIBM_TUNE_LATTICE_PAIRS) {
        if (value != 0 && value != 1) return fail(ctx, PIBM_ERR_ARG, "invalid tuning value");
        c.tune_lattice_pairs = value;
        drop_graphs(c);
        return PIBM_OK;
    }
    if (knob == PIBM_TUNE_COUPLING_ORDER) {
        if (value != 0 && value != 1) return fail(ctx, PIBM_ERR_ARG, "invalid tuning value");
        c.tune_coupling_order = value;
        drop_graphs(c);
        return PIBM_OK;
    }
    if (knob == PIBM_TUNE_TC_WAIT_POLLS) {
        if (value < 0) return fail(ctx, PIBM_ERR_ARG, "poll limit: 0 or more");
        c.sg.wait_polls = value;
        drop_graphs(c);
        return PIBM_OK;
    }
    if (knob == PIBM_TUNE_WIDE_INDEX) {
        if (value != 0 && value != 1) return fail(ctx, PIBM_ERR_ARG, "invalid tuning value");
        c.tune_wide_index = value;
        drop_graphs(c);
        return PIBM_OK;
    }
    if (knob != PIBM_TUNE_DEM_PARTICLES_PER_CTA || value < 0 || value > dem_max_per_cta())
        return fail(ctx, PIBM_ERR_ARG, "invalid tuning knob or value");
    c.tune_dem_particles_per_cta = value;
    if (c.np > 0) {
        int cs = dem_cluster_size(&c);
        if ((c.np + cs - 1) / cs > dem_max_per_cta()) return fail(ctx, PIBM_ERR_ARG, "too many particles per CTA");
        c.dem_cs = cs;
    }
    drop_graphs(c);
    return PIBM_OK;
}

// ------------------------------------------------------------- checkpoints
// Every device buffer that carries state between steps, by name and size.
struct BufRef {
    const char* name;
    void* ptr;
    size_t bytes;
};

static std::vector<BufRef> state_buffers(Ctx& c) {
    std::vector<BufRef> v;
    long long N = c.G.N;
    v.push_back({"f", c.f, (size_t)c.Q * N * c.es});
    v.push_back({"g", c.g, (size_t)c.QG * N * c.es});
    const char* fbn[2] = {"fb0", "fb1"};
    const char* mkn[2] = {"mk0", "mk1"};
    const char* fln[2] = {"flags0", "flags1"};
    for (int b = 0; b < 2; b++) {
        v.push_back({fbn[b], c.fb[b], (size_t)N * c.v4});
        v.push_back({mkn[b], c.mk[b], (size_t)N * c.v4});
        v.push_back({fln[b], c.flags[b], (size_t)c.G.ntx * c.G.ny * c.G.nz});
    }
    v.push_back({"nu_val", c.nu_val, sizeof(double) * 2});
    v.push_back({"nb_cur", c.nb_cur, sizeof(int) * 2});
    int n = c.np;
    if (n > 0) {
        size_t v3 = sizeof(double) * 3 * n, v1 = sizeof(double) * n;
        BufRef pv[] = {{"X", c.X, v3}, {"U", c.U, v3}, {"W", c.W, v3}, {"Xb", c.Xb, v3}, {"R", c.R, v1},
                       {"rho", c.rho, v1}, {"Tp", c.Tp, v1}, {"Cp", c.Cp, v1}, {"m", c.m, v1}, {"I", c.I, v1}, {"im", c.im, v1}, {"iI", c.iI, v1},
                       {"mg", c.mg, v1}, {"fixed", c.fixed, (size_t)n}, {"Fh", c.Fh, v3}, {"Th", c.Th, v3},
                       {"Hh", c.Hh, v1}, {"Fc", c.Fc, sizeof(float) * 3 * n}, {"Tc", c.Tc, sizeof(float) * 3 * n}, {"Fh_prev", c.Fh_prev, v3},
                       {"Th_prev", c.Th_prev, v3}, {"Hh_prev", c.Hh_prev, v1}, {"have_prev", c.have_prev, sizeof(int)},
                       {"box0", c.box[0], sizeof(int) * 6 * n}, {"box1", c.box[1], sizeof(int) * 6 * n},
                       {"wall_ft", c.wall_ft, sizeof(float) * 18 * n}, {"wall_md", c.wall_md, sizeof(double) * 6 * MD_REC * n},
                       {"nb_start0", c.nb_start[0], sizeof(int) * (n + 1)}, {"nb_start1", c.nb_start[1], sizeof(int) * (n + 1)},
                       {"nb_i0", c.nb_i[0], sizeof(int) * c.dem.cap}, {"nb_i1", c.nb_i[1], sizeof(int) * c.dem.cap},
                       {"nb_j0", c.nb_j[0], sizeof(int) * c.dem.cap}, {"nb_j1", c.nb_j[1], sizeof(int) * c.dem.cap},
                       {"nb_ft0", c.nb_ft[0], sizeof(float4) * 2 * c.dem.cap}, {"nb_ft1", c.nb_ft[1], sizeof(float4) * 2 * c.dem.cap},
                       {"nb_md0", c.nb_md[0], sizeof(double) * 2 * MD_REC * c.dem.cap},
                       {"nb_md1", c.nb_md[1], sizeof(double) * 2 * MD_REC * c.dem.cap},
                       {"adj_start", c.adj_start, sizeof(int) * (n + 1)}, {"adj_nb", c.adj_nb, sizeof(int) * c.adj_cap},
                       {"adj_k", c.adj_k, sizeof(int) * c.adj_cap}};
        for (auto& b : pv) v.push_back(b);
    }
    if (c.nm > 0) {
        v.push_back({"Ml", c.Ml, (size_t)c.nm * c.v4});
        v.push_back({"nu_part", c.nu_part, sizeof(double) * c.nm});
    }
    return v;
}

struct CkptHeader {
    char magic[8];
    int version, dim, nx, ny, nz, storage, np, nm, nbuf;
    long long t;
};

pibm_status pibm_save(pibm_ctx* ctx, const char* path) {
    if (!ctx || !path) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    pibm_status st = device_status(ctx);
    if (st != PIBM_OK) return st;
    FILE* fp = fopen(path, "wb");
    if (!fp) return fail(ctx, PIBM_ERR_ARG, std::string("cannot open ") + path);
    std::vector<BufRef> bufs = state_buffers(c);
    CkptHeader h;
    memcpy(h.magic, "PIBMCKP", 8);
    h.version = 1, h.dim = c.D, h.nx = c.G.nx, h.ny = c.G.ny, h.nz = c.G.nz, h.storage = c.desc.storage;
    h.np = c.np, h.nm = c.nm, h.nbuf = (int)bufs.size(), h.t = c.t;
    bool ok = fwrite(&h, sizeof(h), 1, fp) == 1;
    std::vector<char> host;
    for (auto& b : bufs) {
        char name[16] = {0};
        strncpy(name, b.name, 15);
        unsigned long long bytes = b.bytes;
        host.resize(b.bytes);
        if (cudaMemcpy(host.data(), b.ptr, b.bytes, cudaMemcpyDeviceToHost) != cudaSuccess) ok = false;
        ok = ok && fwrite(name, 16, 1, fp) == 1 && fwrite(&bytes, sizeof(bytes), 1, fp) == 1 &&
             (b.bytes == 0 || fwrite(host.data(), b.bytes, 1, fp) == 1);
    }
    ok = (fclose(fp) == 0) && ok;
    return ok ? PIBM_OK : fail(ctx, PIBM_ERR_CUDA, std::string("checkpoint write failed: ") + path);
}

pibm_status pibm_load(pibm_ctx* ctx, const char* path) {
    if (!ctx || !path) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    FILE* fp = fopen(path, "rb");
    if (!fp) return fail(ctx, PIBM_ERR_ARG, std::string("cannot open ") + path);
    CkptHeader h;
    if (fread(&h, sizeof(h), 1, fp) != 1 || memcmp(h.magic, "PIBMCKP", 8) != 0 || h.version != 1) {
        fclose(fp);
        return fail(ctx, PIBM_ERR_ARG, "not a checkpoint of this library");
    }
    if (h.dim != c.D || h.nx != c.G.nx || h.ny != c.G.ny || h.nz != c.G.nz || h.storage != c.desc.storage ||
        h.np != c.np || h.nm != c.nm) {
        fclose(fp);
        return fail(ctx, PIBM_ERR_STATE, "checkpoint does not match this context (lattice, storage, particle or marker count)");
    }
    std::vector<BufRef> bufs = state_buffers(c);
    std::vector<char> host;
    pibm_status st = PIBM_OK;
    for (int k = 0; k < h.nbuf && st == PIBM_OK; k++) {
        char name[16];
        unsigned long long bytes = 0;
        if (fread(name, 16, 1, fp) != 1 || fread(&bytes, sizeof(bytes), 1, fp) != 1) {
            st = fail(ctx, PIBM_ERR_ARG, "truncated checkpoint");
            break;
        }
        name[15] = 0;
        BufRef* dst = nullptr;
        for (auto& b : bufs)
            if (strcmp(b.name, name) == 0) dst = &b;
        if (!dst || dst->bytes != bytes) {
            st = fail(ctx, PIBM_ERR_STATE, std::string("checkpoint buffer does not match: ") + name);
            break;
        }
        host.resize(bytes);
        if (bytes && fread(host.data(), bytes, 1, fp) != 1) {
            st = fail(ctx, PIBM_ERR_ARG, "truncated checkpoint");
            break;
        }
        if (bytes && cudaMemcpy(dst->ptr, host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess)
            st = fail(ctx, PIBM_ERR_CUDA, "checkpoint upload failed");
    }
    fclose(fp);
    if (st != PIBM_OK) return st;
    c.t = h.t;
    drop_graphs(c);
    return device_status(ctx);
}

// ------------------------------------------------------------ surrogate
static pibm_status sg_ensure(pibm_ctx* ctx) {
    Ctx& c = ctx->c;
    if (!c.sg.params) {
        c.sg.params = (float*)dalloc(ctx, sizeof(float) * SG_NPARAMS, GRP_SURROGATE);
        c.sg.m = (float*)dalloc(ctx, sizeof(float) * SG_NPARAMS, GRP_SURROGATE);
        c.sg.v = (float*)dalloc(ctx, sizeof(float) * SG_NPARAMS, GRP_SURROGATE);
        c.sg.norm = (float*)dalloc(ctx, sizeof(float) * (2 * SG_NFEAT + 2 * SG_NOUT), GRP_SURROGATE);
        c.sg.partial = (float*)dalloc(ctx, sizeof(float) * SG_NPARAMS * SG_TRAIN_BLOCKS, GRP_SURROGATE);
        c.sg.lossp = (float*)dalloc(ctx, sizeof(float) * SG_TRAIN_BLOCKS, GRP_SURROGATE);
        c.sg.J_on = (int*)dalloc(ctx, sizeof(int) * 2, GRP_SURROGATE);
        c.sg.err = (int*)dalloc(ctx, sizeof(int) * 2, GRP_SURROGATE);
        c.sg.stats = (double*)dalloc(ctx, sizeof(double) * 4, GRP_SURROGATE);
        c.sg.wimg = (unsigned char*)dalloc(ctx, mlp_image_bytes(), GRP_SURROGATE);
        if (!c.sg.params || !c.sg.m || !c.sg.v || !c.sg.norm || !c.sg.partial || !c.sg.lossp || !c.sg.J_on ||
            !c.sg.err || !c.sg.stats || !c.sg.wimg) {
            c.sg.params = nullptr;
            return fail(ctx, PIBM_ERR_OOM, "surrogate buffers");
        }
    }
    if (c.np > c.sg.cap) {
        dfree_group(ctx, GRP_SG_PART);
        const size_t n = (size_t)c.np;
        c.sg.feat = (double*)dalloc(ctx, sizeof(double) * 12 * n, GRP_SG_PART);
        c.sg.fsum = (double*)dalloc(ctx, sizeof(double) * SG_NFSUM * n, GRP_SG_PART);
        c.sg.xr = (float4*)dalloc(ctx, sizeof(float4) * n, GRP_SG_PART);
        c.sg.nbpart = (double*)dalloc(ctx, sizeof(double) * 5 * SG_NB_SLICES * n, GRP_SG_PART);
        c.sg.rows = (float*)dalloc(ctx, sizeof(float) * SG_ROWS * 16 * n, GRP_SG_PART);
        c.sg.yrows = (float*)dalloc(ctx, sizeof(float) * SG_ROWS * 8 * n, GRP_SG_PART);
        c.sg.J = (float*)dalloc(ctx, sizeof(float) * SG_NJ * n, GRP_SG_PART);
        c.sg.part = (double*)dalloc(ctx, sizeof(double) * 2 * (n / 256 + 2), GRP_SG_PART);
        if (!c.sg.feat || !c.sg.fsum || !c.sg.xr || !c.sg.nbpart || !c.sg.rows || !c.sg.yrows || !c.sg.J || !c.sg.part) {
            c.sg.cap = 0;
            return fail(ctx, PIBM_ERR_OOM, "surrogate particle buffers");
        }
        c.sg.cap = c.np;
    }
    return PIBM_OK;
}

pibm_status pibm_read_features(pibm_ctx* ctx, double* out) {
    if (!ctx || !out) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    if (c.np == 0) return PIBM_OK;
    pibm_status st = sg_ensure(ctx);
    if (st != PIBM_OK) return st;
    PCHECK(launch_footprint_sums(&c, c.s0, parity(c)));
    PCHECK(launch_features(&c, c.s0, parity(c), c.sg.feat));
    PCHECK(cudaMemcpyAsync(out, c.sg.feat, sizeof(double) * 12 * c.np, cudaMemcpyDeviceToHost, c.s0));
    PCHECK(cudaStreamSynchronize(c.s0));
    return PIBM_OK;
}

pibm_status pibm_surrogate_set_params(pibm_ctx* ctx, const float* params, const float* norm) {
    if (!ctx || !params || !norm) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    pibm_status st = sg_ensure(ctx);
    if (st != PIBM_OK) return st;
    for (int k = 0; k < SG_NFEAT; k++)
        if (!(norm[SG_NFEAT + k] > 0)) return fail(ctx, PIBM_ERR_ARG, "feature scales must be positive");
    for (int k = 0; k < SG_NOUT; k++)
        if (!(norm[2 * SG_NFEAT + SG_NOUT + k] > 0)) return fail(ctx, PIBM_ERR_ARG, "target scales must be positive");
    PCHECK(cudaMemcpyAsync(c.sg.params, params, sizeof(float) * SG_NPARAMS, cudaMemcpyHostToDevice, c.s0));
    PCHECK(cudaMemcpyAsync(c.sg.norm, norm, sizeof(float) * (2 * SG_NFEAT + 2 * SG_NOUT), cudaMemcpyHostToDevice, c.s0));
    PCHECK(cudaMemsetAsync(c.sg.m, 0, sizeof(float) * SG_NPARAMS, c.s0));
    PCHECK(cudaMemsetAsync(c.sg.v, 0, sizeof(float) * SG_NPARAMS, c.s0));
    PCHECK(launch_mlp_image(&c, c.s0));
    PCHECK(cudaStreamSynchronize(c.s0));
    c.sg.adam_t = 0;
    c.sg.trained = 1;
    return PIBM_OK;
}

pibm_status pibm_surrogate_get_params(pibm_ctx* ctx, float* params, float* norm) {
    if (!ctx) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    if (!c.sg.trained) return fail(ctx, PIBM_ERR_STATE, "surrogate has no parameters yet");
    if (params) PCHECK(cudaMemcpyAsync(params, c.sg.params, sizeof(float) * SG_NPARAMS, cudaMemcpyDeviceToHost, c.s0));
    if (norm)
        PCHECK(cudaMemcpyAsync(norm, c.sg.norm, sizeof(float) * (2 * SG_NFEAT + 2 * SG_NOUT), cudaMemcpyDeviceToHost, c.s0));
    PCHECK(cudaStreamSynchronize(c.s0));
    return PIBM_OK;
}

pibm_status pibm_surrogate_infer(pibm_ctx* ctx, const float* in, int rows, float* out) {
    if (!ctx || rows < 0 || (rows > 0 && (!in || !out))) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    if (!c.sg.trained) return fail(ctx, PIBM_ERR_STATE, "surrogate has no parameters yet");
    if (rows == 0) return PIBM_OK;
    float* din = (float*)dalloc(ctx, sizeof(float) * 16 * (size_t)rows, GRP_SCRATCH);
    float* dout = (float*)dalloc(ctx, sizeof(float) * 8 * (size_t)rows, GRP_SCRATCH);
    if (!din || !dout) {
        dfree_group(ctx, GRP_SCRATCH);
        return fail(ctx, PIBM_ERR_OOM, "inference buffers");
    }
    cudaError_t e = cudaMemcpyAsync(din, in, sizeof(float) * 16 * (size_t)rows, cudaMemcpyHostToDevice, c.s0);
    if (e == cudaSuccess) e = cudaMemsetAsync(c.sg.err, 0, sizeof(int), c.s0);
    if (e == cudaSuccess) e = launch_mlp(&c, c.s0, din, rows, dout);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, sizeof(float) * 8 * (size_t)rows, cudaMemcpyDeviceToHost, c.s0);
    int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, c.sg.err, sizeof(int), cudaMemcpyDeviceToHost, c.s0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.s0);
    dfree_group(ctx, GRP_SCRATCH);
    if (e != cudaSuccess) return fail(ctx, PIBM_ERR_CUDA, std::string("inference: ") + cudaGetErrorString(e));
    if (err) return fail(ctx, PIBM_ERR_TIMEOUT, "tensor-core wait gave up");
    return PIBM_OK;
}

pibm_status pibm_surrogate_gradient(pibm_ctx* ctx, const float* X, const float* Y, int B, float* grad, double* loss) {
    if (!ctx || !X || !Y || B < 1) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    if (!c.sg.trained) return fail(ctx, PIBM_ERR_STATE, "surrogate has no parameters yet");
    float* xb = (float*)dalloc(ctx, sizeof(float) * SG_NFEAT * (size_t)B, GRP_SCRATCH);
    float* yb = (float*)dalloc(ctx, sizeof(float) * SG_NOUT * (size_t)B, GRP_SCRATCH);
    float* g = (float*)dalloc(ctx, sizeof(float) * SG_NPARAMS, GRP_SCRATCH);
    double* l = (double*)dalloc(ctx, sizeof(double), GRP_SCRATCH);
    if (!xb || !yb || !g || !l) {
        dfree_group(ctx, GRP_SCRATCH);
        return fail(ctx, PIBM_ERR_OOM, "gradient buffers");
    }
    cudaError_t e = cudaMemcpyAsync(xb, X, sizeof(float) * SG_NFEAT * (size_t)B, cudaMemcpyHostToDevice, c.s0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(yb, Y, sizeof(float) * SG_NOUT * (size_t)B, cudaMemcpyHostToDevice, c.s0);
    if (e == cudaSuccess) e = train_batch(&c, c.s0, xb, yb, B, 0.f, g, l);
    if (e == cudaSuccess && grad) e = cudaMemcpyAsync(grad, g, sizeof(float) * SG_NPARAMS, cudaMemcpyDeviceToHost, c.s0);
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, l, sizeof(double), cudaMemcpyDeviceToHost, c.s0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.s0);
    dfree_group(ctx, GRP_SCRATCH);
    if (e != cudaSuccess) return fail(ctx, PIBM_ERR_CUDA, std::string("gradient: ") + cudaGetErrorString(e));
    return PIBM_OK;
}

pibm_status pibm_surrogate_train(pibm_ctx* ctx, const double* feat, const double* targ, int64_t n, int epochs, int batch,
                                 double lr, uint64_t seed, double* loss_per_epoch) {
    if (!ctx || !feat || !targ || n < 2 || epochs < 0 || batch < 1 || !(lr > 0)) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    pibm_status st = sg_ensure(ctx);
    if (st != PIBM_OK) return st;
    // standardisation from the data (FP64, population standard deviation; below 1e-12 counts as 1)
    std::vector<double> mu(SG_NFEAT + SG_NOUT, 0.0), sd(SG_NFEAT + SG_NOUT, 0.0);
    for (int64_t i = 0; i < n; i++) {
        for (int k = 0; k < SG_NFEAT; k++) mu[k] += feat[i * SG_NFEAT + k];
        for (int k = 0; k < SG_NOUT; k++) mu[SG_NFEAT + k] += targ[i * SG_NOUT + k];
    }
    for (auto& v : mu) v /= (double)n;
    for (int64_t i = 0; i < n; i++) {
        for (int k = 0; k < SG_NFEAT; k++) sd[k] += (feat[i * SG_NFEAT + k] - mu[k]) * (feat[i * SG_NFEAT + k] - mu[k]);
        for (int k = 0; k < SG_NOUT; k++)
            sd[SG_NFEAT + k] += (targ[i * SG_NOUT + k] - mu[SG_NFEAT + k]) * (targ[i * SG_NOUT + k] - mu[SG_NFEAT + k]);
    }
    for (auto& v : sd) {
        v = sqrt(v / (double)n);
        if (v < 1e-12) v = 1.0;
    }
    std::vector<float> norm(2 * SG_NFEAT + 2 * SG_NOUT);
    for (int k = 0; k < SG_NFEAT; k++) norm[k] = (float)mu[k], norm[SG_NFEAT + k] = (float)sd[k];
    for (int k = 0; k < SG_NOUT; k++)
        norm[2 * SG_NFEAT + k] = (float)mu[SG_NFEAT + k], norm[2 * SG_NFEAT + SG_NOUT + k] = (float)sd[SG_NFEAT + k];
    std::vector<float> Xn((size_t)n * SG_NFEAT), Yn((size_t)n * SG_NOUT);
    for (int64_t i = 0; i < n; i++) {
        for (int k = 0; k < SG_NFEAT; k++) Xn[i * SG_NFEAT + k] = (float)((feat[i * SG_NFEAT + k] - mu[k]) / sd[k]);
        for (int k = 0; k < SG_NOUT; k++)
            Yn[i * SG_NOUT + k] = (float)((targ[i * SG_NOUT + k] - mu[SG_NFEAT + k]) / sd[SG_NFEAT + k]);
    }
    // Glorot-uniform initial weights, zero biases (the linear path and W4 come
    // from the least-squares fit below)
    std::mt19937_64 rng(seed);
    std::vector<float> params(SG_NPARAMS, 0.f);
    const int sizes[4][2] = {{SG_NFEAT, 64}, {64, 64}, {64, 64}, {64, SG_NOUT}};
    for (int l = 0, off = 0; l < 4; l++) {
        const int fi = sizes[l][0], fo = sizes[l][1];
        std::uniform_real_distribution<double> U(-sqrt(6.0 / (fi + fo)), sqrt(6.0 / (fi + fo)));
        for (int k = 0; k < fi * fo; k++) params[off + k] = (float)U(rng);
        off += fi * fo + fo;
    }
    st = pibm_surrogate_set_params(ctx, params.data(), norm.data());
    if (st != PIBM_OK) return st;
    const int B = (int)std::min<int64_t>(batch, n);
    float* dX = (float*)dalloc(ctx, sizeof(float) * Xn.size(), GRP_SCRATCH);
    float* dY = (float*)dalloc(ctx, sizeof(float) * Yn.size(), GRP_SCRATCH);
    int* didx = (int*)dalloc(ctx, sizeof(int) * (size_t)n, GRP_SCRATCH);
    float* xb = (float*)dalloc(ctx, sizeof(float) * SG_NFEAT * (size_t)B, GRP_SCRATCH);
    float* yb = (float*)dalloc(ctx, sizeof(float) * SG_NOUT * (size_t)B, GRP_SCRATCH);
    double* dl = (double*)dalloc(ctx, sizeof(double) * 2, GRP_SCRATCH);
    double* lsq = (double*)dalloc(ctx, sizeof(double) * lsq_scratch_doubles(), GRP_SCRATCH);
    int* lsq_status = (int*)dalloc(ctx, sizeof(int), GRP_SCRATCH);
    if (!dX || !dY || !didx || !xb || !yb || !dl || !lsq || !lsq_status) {
        dfree_group(ctx, GRP_SCRATCH);
        return fail(ctx, PIBM_ERR_OOM, "training buffers");
    }
    cudaError_t e = cudaMemcpyAsync(dX, Xn.data(), sizeof(float) * Xn.size(), cudaMemcpyHostToDevice, c.s0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dY, Yn.data(), sizeof(float) * Yn.size(), cudaMemcpyHostToDevice, c.s0);
    // the linear path and the output bias by least squares over every sample, W4 = 0
    int lsq_bad = 0;
    if (e == cudaSuccess) e = launch_lsq(&c, c.s0, dX, dY, (long long)n, 1e-8, lsq, lsq_status);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&lsq_bad, lsq_status, sizeof(int), cudaMemcpyDeviceToHost, c.s0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.s0);
    if (e == cudaSuccess && lsq_bad) {
        dfree_group(ctx, GRP_SCRATCH);
        if (launch_mlp_image(&c, c.s0) != cudaSuccess || cudaStreamSynchronize(c.s0) != cudaSuccess)
            return fail(ctx, PIBM_ERR_CUDA, "inference weight image");
        return fail(ctx, PIBM_ERR_STATE, "least-squares fit of the linear path is singular");
    }
    std::vector<int> idx((size_t)n);
    for (int64_t i = 0; i < n; i++) idx[i] = (int)i;
    const int64_t nb = n / B;  // full batches per epoch
    for (int ep = 0; ep < epochs && e == cudaSuccess; ep++) {
        std::shuffle(idx.begin(), idx.end(), rng);
        e = cudaMemcpyAsync(didx, idx.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, c.s0);
        double loss_sum = 0.0;
        for (int64_t b = 0; b < nb && e == cudaSuccess; b++) {
            e = launch_gather(c.s0, B, didx + b * B, dX, dY, xb, yb);
            if (e == cudaSuccess) e = train_batch(&c, c.s0, xb, yb, B, (float)lr, nullptr, dl);
            if (e == cudaSuccess && loss_per_epoch) {
                double lv = 0.0;
                e = cudaMemcpyAsync(&lv, dl, sizeof(double), cudaMemcpyDeviceToHost, c.s0);
                if (e == cudaSuccess) e = cudaStreamSynchronize(c.s0);
                loss_sum += lv;
            }
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.s0);
        if (loss_per_epoch) loss_per_epoch[ep] = nb > 0 ? loss_sum / (double)nb : 0.0;
    }
    if (e == cudaSuccess) e = launch_mlp_image(&c, c.s0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.s0);
    dfree_group(ctx, GRP_SCRATCH);
    if (e != cudaSuccess) return fail(ctx, PIBM_ERR_CUDA, std::string("training: ") + cudaGetErrorString(e));
    drop_graphs(c);
    return PIBM_OK;
}

pibm_status pibm_surrogate_enable(pibm_ctx* ctx, int on, double bound, double delta) {
    if (!ctx) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    drop_graphs(c);
    if (!on) {
        c.sg.enabled = 0;
        if (!c.sg.fixed) c.dem.J = nullptr, c.dem.J_on = nullptr;
        return PIBM_OK;
    }
    if (!c.sg.trained) return fail(ctx, PIBM_ERR_STATE, "surrogate has no parameters yet");
    if (c.np == 0) return fail(ctx, PIBM_ERR_STATE, "no particles");
    if (c.point) return fail(ctx, PIBM_ERR_STATE, "the surrogate's features need resolved particles");
    if (!(bound >= 0) || !(delta > 0)) return fail(ctx, PIBM_ERR_ARG, "bound must be >= 0 and delta > 0");
    pibm_status st = sg_ensure(ctx);
    if (st != PIBM_OK) return st;
    c.sg.enabled = 1;
    c.sg.fixed = 0;
    c.sg.bound = bound;
    c.sg.delta = delta;
    c.dem.J = c.sg.J;
    c.dem.J_on = c.sg.J_on;
    PCHECK(cudaMemsetAsync(c.sg.stats, 0, sizeof(double) * 4, c.s0));
    PCHECK(cudaMemsetAsync(c.sg.err, 0, sizeof(int), c.s0));
    PCHECK(launch_surrogate(&c, c.s0, parity(c), true));  // Jacobian and gate of the current state for the next step
    PCHECK(cudaStreamSynchronize(c.s0));
    return PIBM_OK;
}

pibm_status pibm_surrogate_stats(pibm_ctx* ctx, double* out) {
    if (!ctx || !out) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    out[0] = out[1] = out[2] = 0.0;
    if (!c.sg.stats) return PIBM_OK;
    PCHECK(cudaMemcpyAsync(out, c.sg.stats, sizeof(double) * 3, cudaMemcpyDeviceToHost, c.s0));
    PCHECK(cudaStreamSynchronize(c.s0));
    return PIBM_OK;
}

pibm_status pibm_read_hydro_jacobian(pibm_ctx* ctx, double* J, int* on) {
    if (!ctx) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    if (!c.dem.J) return fail(ctx, PIBM_ERR_STATE, "no hydrodynamic Jacobian in use");
    std::vector<float> h((size_t)SG_NJ * c.np);
    int o = 0;
    PCHECK(cudaMemcpyAsync(h.data(), c.dem.J, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, c.s0));
    PCHECK(cudaMemcpyAsync(&o, c.dem.J_on, sizeof(int), cudaMemcpyDeviceToHost, c.s0));
    PCHECK(cudaStreamSynchronize(c.s0));
    if (J)
        for (size_t k = 0; k < h.size(); k++) J[k] = h[k];
    if (on) *on = o;
    return PIBM_OK;
}

pibm_status pibm_set_hydro_jacobian(pibm_ctx* ctx, const double* J) {
    if (!ctx) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    drop_graphs(c);
    if (!J) {
        c.sg.fixed = 0;
        if (!c.sg.enabled) c.dem.J = nullptr, c.dem.J_on = nullptr;
        return PIBM_OK;
    }
    if (c.np == 0) return fail(ctx, PIBM_ERR_STATE, "no particles");
    pibm_status st = sg_ensure(ctx);
    if (st != PIBM_OK) return st;
    std::vector<float> h((size_t)SG_NJ * c.np);
    for (size_t k = 0; k < h.size(); k++) h[k] = (float)J[k];
    const int one = 1;
    PCHECK(cudaMemcpyAsync(c.sg.J, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, c.s0));
    PCHECK(cudaMemcpyAsync(c.sg.J_on, &one, sizeof(int), cudaMemcpyHostToDevice, c.s0));
    PCHECK(cudaStreamSynchronize(c.s0));
    c.sg.enabled = 0;
    c.sg.fixed = 1;
    c.dem.J = c.sg.J;
    c.dem.J_on = c.sg.J_on;
    return PIBM_OK;
}

pibm_status pibm_set_particle_model(pibm_ctx* ctx, int model) {
    if (!ctx) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    if (model != PIBM_PARTICLES_RESOLVED && model != PIBM_PARTICLES_POINT)
        return fail(ctx, PIBM_ERR_ARG, "unknown particle model");
    if (c.np > 0) return fail(ctx, PIBM_ERR_STATE, "set the particle model before the particles");
    c.point = model == PIBM_PARTICLES_POINT;
    drop_graphs(c);
    return PIBM_OK;
}

pibm_status pibm_kernels_per_step(pibm_ctx* ctx, int* n) {
    if (!ctx || !n) return PIBM_ERR_ARG;
    Ctx& c = ctx->c;
    *n = 1 + (c.np > 0 ? 1 : 0) + coupling_kernel_count(&c);
    return PIBM_OK;
}

}  // extern "C"

// Batched ensemble: many independent lattices (boxes of different sizes,
// Rayleigh numbers and particle counts) advanced together, one CUDA graph
// launch per lattice step for all of them.
//
// Each box is an ordinary context with its own pair of streams.  The ensemble
// step graph forks from the ensemble stream into every box's streams and
// joins back, so the boxes' kernels (collide-and-stream, the DEM cluster, the
// coupling) are independent branches of one graph and run concurrently on
// the GPU; one launch replaces 5-6 launches per box.  Box set-up and
// read-back go through the usual per-context calls.
//
// The autotuner times candidate launch shapes with CUDA events on real steps
// (launch shapes change no result): each box's DEM shape alone, then whole
// configurations as ensemble steps, and keeps the fastest by a margin.
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pibm_internal.cuh"

using namespace pibm;

struct pibm_ensemble {
    std::vector<pibm_ctx*> box;
    cudaStream_t s = nullptr;
    int own_s = 0;
    cudaEvent_t ev_fork = nullptr, ev_done = nullptr;
    std::vector<cudaEvent_t> ev_join, ev_ready;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_ok[2] = {0, 0};
    std::vector<unsigned> gen[2];  // box graph generations the ensemble graphs were captured with
    int kernels = 0;
    std::string err;
};

static pibm_status efail(pibm_ensemble* e, pibm_status s, const std::string& msg) {
    e->err = msg;
    return s;
}

#define ECHECK(call)                                                                  \
    do {                                                                              \
        cudaError_t r_ = (call);                                                      \
        if (r_ != cudaSuccess) return efail(e, PIBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(r_)); \
    } while (0)

static void drop_ensemble_graphs(pibm_ensemble* e) {
    for (int p = 0; p < 2; p++) {
        if (e->graph_ok[p]) cudaGraphExecDestroy(e->graph[p]);
        e->graph_ok[p] = 0;
    }
}

static bool graphs_current(const pibm_ensemble* e, int par) {
    if (!e->graph_ok[par]) return false;
    for (size_t b = 0; b < e->box.size(); b++)
        if (e->gen[par][b] != ctx_state(e->box[b])->gen) return false;
    return true;
}

static pibm_status capture_ensemble(pibm_ensemble* e, int par) {
    if (e->graph_ok[par]) {
        cudaGraphExecDestroy(e->graph[par]);
        e->graph_ok[par] = 0;
    }
    ECHECK(cudaStreamBeginCapture(e->s, cudaStreamCaptureModeThreadLocal));
    cudaError_t r = cudaEventRecord(e->ev_fork, e->s);
    int kernels = 0;
    for (size_t b = 0; b < e->box.size() && r == cudaSuccess; b++) {
        Ctx* c = ctx_state(e->box[b]);
        int k = 0;
        if ((r = cudaStreamWaitEvent(c->s0, e->ev_fork, 0)) != cudaSuccess) break;
        if ((r = record_step(c, par, &k)) != cudaSuccess) break;
        if ((r = cudaEventRecord(e->ev_join[b], c->s0)) != cudaSuccess) break;
        r = cudaStreamWaitEvent(e->s, e->ev_join[b], 0);
        kernels += k;
    }
    cudaGraph_t graph;
    cudaError_t r2 = cudaStreamEndCapture(e->s, &graph);
    if (r != cudaSuccess || r2 != cudaSuccess) {
        if (r2 == cudaSuccess) cudaGraphDestroy(graph);
        return efail(e, PIBM_ERR_CUDA, std::string("ensemble graph capture: ") + cudaGetErrorString(r != cudaSuccess ? r : r2));
    }
    r = cudaGraphInstantiate(&e->graph[par], graph, 0);
    cudaGraphDestroy(graph);
    if (r != cudaSuccess) return efail(e, PIBM_ERR_CUDA, std::string("ensemble graph instantiate: ") + cudaGetErrorString(r));
    e->graph_ok[par] = 1;
    e->gen[par].resize(e->box.size());
    for (size_t b = 0; b < e->box.size(); b++) e->gen[par][b] = ctx_state(e->box[b])->gen;
    e->kernels = kernels;
    return PIBM_OK;
}

extern "C" {

pibm_status pibm_ensemble_create(const pibm_desc* descs, int n_boxes, void* stream, const pibm_allocator* alloc,
                                 pibm_ensemble** out) {
    if (!descs || !out || n_boxes < 1) {
        set_global_error("pibm_ensemble_create: null argument or no boxes");
        return PIBM_ERR_ARG;
    }
    *out = nullptr;
    pibm_ensemble* e = new pibm_ensemble();
    auto bail = [&](pibm_status st, const std::string& msg) {
        set_global_error(msg);
        pibm_ensemble_destroy(e);
        return st;
    };
    if (stream) {
        e->s = (cudaStream_t)stream;
    } else {
        cudaError_t r = cudaStreamCreateWithFlags(&e->s, cudaStreamNonBlocking);
        if (r != cudaSuccess) return bail(PIBM_ERR_CUDA, cudaGetErrorString(r));
        e->own_s = 1;
    }
    if (cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->ev_done, cudaEventDisableTiming) != cudaSuccess)
        return bail(PIBM_ERR_CUDA, "event creation failed");
    for (int b = 0; b < n_boxes; b++) {
        pibm_ctx* c = nullptr;
        pibm_status st = pibm_create(&descs[b], nullptr, alloc, &c);  // the box owns its streams
        if (st != PIBM_OK) {
            char buf[256];
            pibm_last_error(nullptr, buf, sizeof buf);
            return bail(st, "box " + std::to_string(b) + ": " + buf);
        }
        e->box.push_back(c);
        cudaEvent_t j, rd;
        if (cudaEventCreateWithFlags(&j, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&rd, cudaEventDisableTiming) != cudaSuccess)
            return bail(PIBM_ERR_CUDA, "event creation failed");
        e->ev_join.push_back(j);
        e->ev_ready.push_back(rd);
    }
    *out = e;
    return PIBM_OK;
}

pibm_status pibm_ensemble_destroy(pibm_ensemble* e) {
    if (!e) return PIBM_ERR_ARG;
    if (e->s) cudaStreamSynchronize(e->s);
    drop_ensemble_graphs(e);
    for (pibm_ctx* c : e->box) pibm_destroy(c);
    for (cudaEvent_t v : e->ev_join) cudaEventDestroy(v);
    for (cudaEvent_t v : e->ev_ready) cudaEventDestroy(v);
    if (e->ev_fork) cudaEventDestroy(e->ev_fork);
    if (e->ev_done) cudaEventDestroy(e->ev_done);
    if (e->own_s && e->s) cudaStreamDestroy(e->s);
    delete e;
    return PIBM_OK;
}

pibm_status pibm_ensemble_box(pibm_ensemble* e, int b, pibm_ctx** out) {
    if (!e || !out || b < 0 || b >= (int)e->box.size()) return PIBM_ERR_ARG;
    *out = e->box[b];
    return PIBM_OK;
}

pibm_status pibm_ensemble_step(pibm_ensemble* e, int nsteps) {
    if (!e) return PIBM_ERR_ARG;
    if (nsteps < 0) return efail(e, PIBM_ERR_ARG, "negative step count");
    if (nsteps == 0) return PIBM_OK;
    const int64_t t0 = ctx_state(e->box[0])->t;
    for (size_t b = 0; b < e->box.size(); b++) {
        pibm_status st = ctx_ready(e->box[b]);  // configuration and device status of the box
        if (st != PIBM_OK) {
            char buf[256];
            pibm_last_error(e->box[b], buf, sizeof buf);
            return efail(e, st, "box " + std::to_string(b) + ": " + buf);
        }
        if (ctx_state(e->box[b])->t != t0) return efail(e, PIBM_ERR_STATE, "boxes are at different time steps");
    }
    // order after any per-box work already queued on the boxes' streams
    for (size_t b = 0; b < e->box.size(); b++) {
        Ctx* c = ctx_state(e->box[b]);
        ECHECK(cudaEventRecord(e->ev_ready[b], c->s0));
        ECHECK(cudaStreamWaitEvent(e->s, e->ev_ready[b], 0));
    }
    for (int k = 0; k < nsteps; k++) {
        const int par = (int)((t0 + k) & 1);
        if (!graphs_current(e, par)) {
            pibm_status st = capture_ensemble(e, par);
            if (st != PIBM_OK) return st;
        }
        ECHECK(cudaGraphLaunch(e->graph[par], e->s));
    }
    for (size_t b = 0; b < e->box.size(); b++) ctx_state(e->box[b])->t += nsteps;
    // later per-box calls (read-back, set-up) are ordered after the ensemble's steps
    ECHECK(cudaEventRecord(e->ev_done, e->s));
    for (size_t b = 0; b < e->box.size(); b++) ECHECK(cudaStreamWaitEvent(ctx_state(e->box[b])->s0, e->ev_done, 0));
    return PIBM_OK;
}

pibm_status pibm_ensemble_kernels_per_step(pibm_ensemble* e, int* n) {
    if (!e || !n) return PIBM_ERR_ARG;
    if (!e->graph_ok[0] && !e->graph_ok[1]) {
        int total = 0;
        for (pibm_ctx* c : e->box) {
            int k = 0;
            pibm_kernels_per_step(c, &k);
            total += k;
        }
        *n = total;
    } else {
        *n = e->kernels;
    }
    return PIBM_OK;
}

// Median device time of one ensemble step (graph launch) over reps steps,
// CUDA events on the ensemble stream; two untimed steps first, so that the
// graphs of both step parities are captured outside the timed region.
static pibm_status time_ensemble(pibm_ensemble* e, int reps, double* median_ms) {
    pibm_status st = pibm_ensemble_step(e, 2);
    if (st != PIBM_OK) return st;
    cudaEvent_t a, b;
    ECHECK(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return efail(e, PIBM_ERR_CUDA, "autotune: event creation failed");
    }
    std::vector<double> ms;
    for (int r = 0; r < reps && st == PIBM_OK; r++) {
        cudaError_t x = cudaEventRecord(a, e->s);
        if (x == cudaSuccess && (st = pibm_ensemble_step(e, 1)) != PIBM_OK) break;
        if (x == cudaSuccess) x = cudaEventRecord(b, e->s);
        if (x == cudaSuccess) x = cudaEventSynchronize(b);
        float v = 0.f;
        if (x == cudaSuccess) x = cudaEventElapsedTime(&v, a, b);
        if (x != cudaSuccess) st = efail(e, PIBM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(x));
        ms.push_back(v);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != PIBM_OK) return st;
    std::sort(ms.begin(), ms.end());
    *median_ms = ms[ms.size() / 2];
    return PIBM_OK;
}

pibm_status pibm_ensemble_autotune(pibm_ensemble* e, int reps, int32_t* choice) {
    if (!e || reps < 1) return PIBM_ERR_ARG;
    const int nb = (int)e->box.size();
    // 1. each box's DEM shape, timed alone (the DEM kernel of each candidate;
    //    every box runs the same number of steps, so the boxes stay at one time)
    static const int dem_cand[] = {0, 16, 48, 64, 96};
    std::vector<int> pick_dem(nb, 0);
    for (int b = 0; b < nb; b++) {
        pibm_ctx* c = e->box[b];
        Ctx* cs = ctx_state(c);
        double best = 1e300;
        for (int k = 0; k < 5; k++) {
            const bool ok = cs->np > 0 && dem_cand[k] <= dem_max_per_cta() &&
                            (dem_cand[k] == 0 || (cs->np + dem_cand[k] - 1) / dem_cand[k] <= 16) &&
                            pibm_set_tuning(c, PIBM_TUNE_DEM_PARTICLES_PER_CTA, dem_cand[k]) == PIBM_OK;
            if (cs->np > 0 && !ok) pibm_set_tuning(c, PIBM_TUNE_DEM_PARTICLES_PER_CTA, 0);
            for (int r = 0; r < reps; r++) {
                double ms[4];
                pibm_status st = pibm_step_timed(c, ms);
                if (st != PIBM_OK) {
                    char buf[256];
                    pibm_last_error(c, buf, sizeof buf);
                    return efail(e, st, "autotune: box " + std::to_string(b) + ": " + buf);
                }
                if (ok && ms[1] < best) best = ms[1], pick_dem[b] = dem_cand[k];
            }
        }
        if (cs->np > 0) pibm_set_tuning(c, PIBM_TUNE_DEM_PARTICLES_PER_CTA, 0);
    }
    for (int b = 1; b < nb; b++)
        if (ctx_state(e->box[b])->t != ctx_state(e->box[0])->t) return efail(e, PIBM_ERR_STATE, "autotune: time mismatch");
    // 2. whole-ensemble configurations, timed as ensemble steps (the boxes share
    //    the GPU there, so a box's fastest shape alone need not be fastest in the
    //    ensemble): lattice threads per block x whole-row lattice blocks, each with
    //    the default DEM shapes and with the picks of step 1
    struct Cfg {
        int lat, rows, dem;
    };
    std::vector<Cfg> cand;
    static const int lat_cand[] = {0, 128, 256, 512};
    for (int dem = 0; dem < 2; dem++)
        for (int rows = 0; rows < 2; rows++)
            for (int l = 0; l < 4; l++) cand.push_back({lat_cand[l], rows, dem});
    auto apply = [&](const Cfg& g) -> pibm_status {
        for (int b = 0; b < nb; b++) {
            pibm_ctx* c = e->box[b];
            pibm_status st = pibm_set_tuning(c, PIBM_TUNE_LATTICE_THREADS, g.lat);
            if (st == PIBM_OK) st = pibm_set_tuning(c, PIBM_TUNE_LATTICE_ROW_TILES, g.rows);
            if (st == PIBM_OK && ctx_state(c)->np > 0)
                st = pibm_set_tuning(c, PIBM_TUNE_DEM_PARTICLES_PER_CTA, g.dem ? pick_dem[b] : 0);
            if (st != PIBM_OK) return efail(e, st, "autotune: launch shape rejected");
        }
        return PIBM_OK;
    };
    double best = 1e300, base = 1e300;
    size_t pick = 0;
    for (size_t k = 0; k < cand.size(); k++) {
        double ms = 0.0;
        pibm_status st = apply(cand[k]);
        if (st == PIBM_OK) st = time_ensemble(e, reps + 2, &ms);
        if (st != PIBM_OK) return st;
        if (k == 0) base = ms;
        if (ms < best) best = ms, pick = k;
    }
    // keep the defaults unless the best candidate is faster by more than 1 %
    if (!(best < 0.99 * base)) pick = 0;
    pibm_status st = apply(cand[pick]);
    if (st != PIBM_OK) return st;
    if (choice)
        for (int b = 0; b < nb; b++) {
            choice[3 * b] = cand[pick].lat;
            choice[3 * b + 1] = cand[pick].rows;
            choice[3 * b + 2] = cand[pick].dem ? pick_dem[b] : 0;
        }
    return PIBM_OK;
}

int pibm_ensemble_last_error(pibm_ensemble* e, char* buf, size_t n) {
    const std::string& s = e ? e->err : std::string();
    if (buf && n > 0) {
        size_t m = s.size() < n - 1 ? s.size() : n - 1;
        memcpy(buf, s.data(), m);
        buf[m] = 0;
    }
    return (int)s.size();
}

}  // extern "C"

// Contact search that allocates nothing (pibm_contacts_static in pibm.h).
//
// Some callers cannot allocate device memory: code that runs inside another
// framework's memory pool or arena, plug-ins loaded into a host that owns
// every allocation, or processes whose device memory is fully reserved up
// front.  They can still ask for the contact list of particles they already
// hold on the device.  This file computes it with the same definitions as the
// library's neighbour-list path (cell side n_a / floor(n_a / cell_min), cell
// id floor((X + 1/2) nc / n) in FP64, pairs i < j with |X_i - X_j|^2 <
// (R_i + R_j)^2 in the same operation order, sorted by (i, j)), keeping its
// working arrays (cell counts and starts, sorted particle ids, per-particle
// pair counts and offsets) in one file-scope device array of fixed size.
#include <string>

#include "pibm_internal.cuh"

namespace pibm {

constexpr int NA_MAX_PARTICLES = 16384;
constexpr int NA_MAX_CELLS = 65536;
constexpr int NA_THREADS = 1024;
// layout: cell_count[NA_MAX_CELLS] | cell_start[NA_MAX_CELLS + 1] | cell_ids[NA_MAX_PARTICLES] |
//         cell_of[NA_MAX_PARTICLES] | pair_count[NA_MAX_PARTICLES] | pair_offset[NA_MAX_PARTICLES + 1]
constexpr int NA_SCRATCH_INTS = NA_MAX_CELLS + (NA_MAX_CELLS + 1) + 3 * NA_MAX_PARTICLES + (NA_MAX_PARTICLES + 1);

// 2 * 65536 + 4 * 16384 + 2 ints = 786 440 bytes, held by every GPU that loads the library
static __device__ __align__(256) int g_contact_scratch[NA_SCRATCH_INTS];

struct NaGrid {
    int dim, nc[3];
    double inv[3], side[3];
    int ncell;
};

__device__ __forceinline__ double na_dist2(const double* X, int i, int j) {
    double dx = __dsub_rn(X[3 * j], X[3 * i]), dy = __dsub_rn(X[3 * j + 1], X[3 * i + 1]),
           dz = __dsub_rn(X[3 * j + 2], X[3 * i + 2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__device__ __forceinline__ void na_cell(const NaGrid& G, const double* X, int p, int* c) {
    for (int a = 0; a < 3; a++) {
        int v = 0;
        if (a < G.dim) {
            v = (int)floor(__dmul_rn(__dadd_rn(X[3 * p + a], 0.5), G.inv[a]));
            if (v < 0) v = 0;
            if (v > G.nc[a] - 1) v = G.nc[a] - 1;
        }
        c[a] = v;
    }
}

// one CTA: exclusive scan of in[0..M) into out[0..M]
__device__ void na_scan(const int* in, int* out, int M, int* sh) {
    const int T = blockDim.x, t = threadIdx.x;
    const int chunk = (M + T - 1) / T;
    const int b = min(M, t * chunk), e = min(M, b + chunk);
    int s = 0;
    for (int i = b; i < e; i++) s += in[i];
    sh[t] = s;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        int v = t >= off ? sh[t - off] : 0;
        __syncthreads();
        sh[t] += v;
        __syncthreads();
    }
    int base = t ? sh[t - 1] : 0;
    for (int i = b; i < e; i++) {
        int v = in[i];
        out[i] = base;
        base += v;
    }
    if (t == T - 1) out[M] = sh[T - 1];
    __syncthreads();
}

template <typename F>
__device__ __forceinline__ void na_visit(const NaGrid& G, const int* cell_start, const int* cell_ids, const int* c, F&& fn) {
    for (int z = c[2] - 1; z <= c[2] + 1; z++) {
        if (z < 0 || z >= G.nc[2]) continue;
        for (int y = c[1] - 1; y <= c[1] + 1; y++) {
            if (y < 0 || y >= G.nc[1]) continue;
            for (int x = c[0] - 1; x <= c[0] + 1; x++) {
                if (x < 0 || x >= G.nc[0]) continue;
                int cell = (z * G.nc[1] + y) * G.nc[0] + x;
                for (int k = cell_start[cell]; k < cell_start[cell + 1]; k++) fn(cell_ids[k]);
            }
        }
    }
}

// Single CTA: cell list (counting sort, stable by index), per-particle pair
// counts (at most 64 partners j > i kept per particle i), offsets, then the
// pairs in (i, j) order.  Every scratch region that must start at zero is
// cleared here, because the array keeps the previous call's contents.
// count[0]: number of pairs kept (no holes: every kept pair is written while
// it fits in cap); count[1]: a bit set -- 1 if a particle had more than 64
// partners (the extra pairs dropped), 2 if a diameter exceeds the cell side.
__global__ void __launch_bounds__(NA_THREADS) k_contacts_static(NaGrid G, int n, const double* __restrict__ X,
                                                               const double* __restrict__ R, int* pairs, int cap,
                                                               int* count, int* scratch) {
    __shared__ int sh[NA_THREADS];
    int* cell_count = scratch;
    int* cell_start = cell_count + NA_MAX_CELLS;
    int* cell_ids = cell_start + NA_MAX_CELLS + 1;
    int* cell_of = cell_ids + NA_MAX_PARTICLES;
    int* pair_count = cell_of + NA_MAX_PARTICLES;
    int* pair_offset = pair_count + NA_MAX_PARTICLES;
    const int t = threadIdx.x, T = blockDim.x;
    for (int c = t; c < G.ncell; c += T) cell_count[c] = 0;
    for (int p = t; p < n; p += T)  // a contact must lie within the 3^D neighbouring cells
        for (int a = 0; a < G.dim; a++)
            if (2.0 * R[p] > G.side[a]) atomicOr(count + 1, 2);
    __syncthreads();
    for (int p = t; p < n; p += T) {
        int c[3];
        na_cell(G, X, p, c);
        int id = (c[2] * G.nc[1] + c[1]) * G.nc[0] + c[0];
        cell_of[p] = id;
        atomicAdd(cell_count + id, 1);
    }
    __syncthreads();
    na_scan(cell_count, cell_start, G.ncell, sh);
    for (int c = t; c < G.ncell; c += T) cell_count[c] = 0;
    __syncthreads();
    for (int p = t; p < n; p += T) {
        int id = cell_of[p];
        cell_ids[cell_start[id] + atomicAdd(cell_count + id, 1)] = p;
    }
    __syncthreads();
    for (int c = t; c < G.ncell; c += T) {  // order within a cell: by particle index
        int b = cell_start[c], e = cell_start[c + 1];
        for (int a = b + 1; a < e; a++) {
            int v = cell_ids[a], q = a - 1;
            while (q >= b && cell_ids[q] > v) {
                cell_ids[q + 1] = cell_ids[q];
                q--;
            }
            cell_ids[q + 1] = v;
        }
    }
    __syncthreads();
    for (int i = t; i < n; i += T) {
        int c[3], k = 0;
        na_cell(G, X, i, c);
        na_visit(G, cell_start, cell_ids, c, [&](int j) {
            double s = R[i] + R[j];
            if (j > i && na_dist2(X, i, j) < s * s) k++;
        });
        pair_count[i] = k < 64 ? k : 64;  // the pairs kept (the rest are reported by the flag)
    }
    __syncthreads();
    na_scan(pair_count, pair_offset, n, sh);
    for (int i = t; i < n; i += T) {
        int c[3], cand[64], k = 0, extra = 0;
        na_cell(G, X, i, c);
        na_visit(G, cell_start, cell_ids, c, [&](int j) {
            double s = R[i] + R[j];
            if (j > i && na_dist2(X, i, j) < s * s) {
                if (k < 64) cand[k++] = j;
                else extra++;
            }
        });
        for (int a = 1; a < k; a++) {  // partners in increasing index
            int v = cand[a], q = a - 1;
            while (q >= 0 && cand[q] > v) {
                cand[q + 1] = cand[q];
                q--;
            }
            cand[q + 1] = v;
        }
        int o = pair_offset[i];
        for (int r = 0; r < k; r++, o++)
            if (o < cap) {
                pairs[2 * o] = i;
                pairs[2 * o + 1] = cand[r];
            }
        if (extra) atomicOr(count + 1, 1);  // more than 64 partners for one particle
    }
    if (t == 0) count[0] = pair_offset[n];
}

// Device address of the scratch array, per device.  Host code must not pass the
// symbol itself (on the host it is only a stand-in), and a symbol's device
// address belongs to the CUDA context that loaded the module: every call made
// outside stream capture looks it up again with the caller's context current
// (so a device reset or another context is picked up); a call inside a capture
// (where the lookup may not be issued) uses the address of the device's last
// uncaptured call.
static int* g_scratch_addr[64];

}  // namespace pibm

using namespace pibm;

extern "C" pibm_status pibm_contacts_static(const double* d_X, const double* d_R, int n, int dim, const int32_t* nlat,
                                            double cell_size, int32_t* d_pairs, int cap, int32_t* d_count,
                                            void* stream) {
    if (n < 0 || (dim != 2 && dim != 3) || !nlat || cap < 0 || !d_count || (n > 0 && (!d_X || !d_R)) ||
        (cap > 0 && !d_pairs) || !(cell_size > 0)) {
        set_global_error("pibm_contacts_static: invalid argument");
        return PIBM_ERR_ARG;
    }
    if (n > NA_MAX_PARTICLES) {
        set_global_error("pibm_contacts_static: more than 16384 particles (the fixed scratch limit)");
        return PIBM_ERR_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        set_global_error("pibm_contacts_static: no current CUDA device");
        return PIBM_ERR_CUDA;
    }
    cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cap_status) != cudaSuccess) {
        set_global_error("pibm_contacts_static: invalid stream");
        return PIBM_ERR_CUDA;
    }
    if (cap_status == cudaStreamCaptureStatusNone) {  // look up the array's device address in this context
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_contact_scratch);
        if (e != cudaSuccess || !ptr) {
            set_global_error(std::string("pibm_contacts_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return PIBM_ERR_CUDA;
        }
        g_scratch_addr[dev] = (int*)ptr;
    } else if (!g_scratch_addr[dev]) {
        set_global_error("pibm_contacts_static: the first call on a device must come before any stream capture");
        return PIBM_ERR_STATE;
    }
    NaGrid G;
    G.dim = dim;
    G.ncell = 1;
    for (int a = 0; a < 3; a++) {
        int na = a < dim ? nlat[a] : 1;
        if (na < 1) {
            set_global_error("pibm_contacts_static: invalid lattice size");
            return PIBM_ERR_ARG;
        }
        G.nc[a] = 1;
        G.inv[a] = 1.0 / (double)na;
        if (a < dim) {  // the library's cell grid: nc = floor(n / cell_min), side n / nc
            const double q = floor((double)na / cell_size);  // checked before it becomes an int
            if (q > (double)NA_MAX_CELLS) {
                set_global_error("pibm_contacts_static: more than 65536 cells (the fixed scratch limit)");
                return PIBM_ERR_ARG;
            }
            G.nc[a] = q < 1.0 ? 1 : (int)q;
            G.inv[a] = (double)G.nc[a] / (double)na;
        }
        G.side[a] = (double)na / (double)G.nc[a];
        if ((long long)G.ncell * G.nc[a] > NA_MAX_CELLS) {
            set_global_error("pibm_contacts_static: more than 65536 cells (the fixed scratch limit)");
            return PIBM_ERR_ARG;
        }
        G.ncell *= G.nc[a];
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_count, 0, 2 * sizeof(int32_t), s);
    if (e == cudaSuccess) {
        k_contacts_static<<<1, NA_THREADS, 0, s>>>(G, n, d_X, d_R, d_pairs, cap, d_count, g_scratch_addr[dev]);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_global_error(std::string("pibm_contacts_static: ") + cudaGetErrorString(e));
        return PIBM_ERR_CUDA;
    }
    return PIBM_OK;
}

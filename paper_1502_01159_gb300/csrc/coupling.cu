// PIBM coupling kernels (Section 2.2, Eqs lbm5-lbm13).
//
// Resolved particles: every lattice node a particle covers is a PIBM point of
// area eps = clamp(R + 1/2 - |r - X|, 0, 1); a node shared by two footprints
// belongs to the particle with the larger eps (ties: lower index).  At a node
// the interpolation of Eqs lbm5/lbm5.5 is the identity, and Eqs lbm7 + lbm8
// give the force density F_f = 2 (rho U_l - j); Eq lbm7.5 gives the heat
// source Q = 2 kappa_T (T_p - T).  Three kernels, one CTA per particle, no
// atomics:
//   clear     : zero the marker field, F_B / Q_B and tile flags on the boxes
//               recorded in the previous step;
//   footprint : ownership test against the particle's neighbours, marker
//               values eps (F_f, Q) for the nodes it owns, and the FP64 block
//               reduction to force, torque and heat release (Eq lbm13);
//   spread    : F_B(r) = sum_d W(d) M(r + d), W = product of delta_h weights
//               1/2, 1/4, 1/4 (Eqs lbm10-lbm12, lbm12.6) over the footprint
//               grown by one node; overlapping boxes write identical values.
// The footprint and spread blocks take the particles in the spatial order of
// the DEM's cell list (results do not depend on the order).
//
// Static off-node markers (the cavity cylinder): one thread per marker does
// the 4-point Lagrange interpolation (Eq lbm6) and forms A (F_f, Q); spreading
// is a gather over a precomputed node -> marker list in marker order.
#include "pibm_internal.cuh"

namespace pibm {

constexpr int CP_THREADS = 256;
constexpr int CP_MAXNB = 64;

__device__ __forceinline__ double eps_of(double x, double y, double z, const double* Xp, double Rp) {
    double dx = __dsub_rn(x, Xp[0]), dy = __dsub_rn(y, Xp[1]), dz = __dsub_rn(z, Xp[2]);
    double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    double e = __dsub_rn(__dadd_rn(Rp, 0.5), __dsqrt_rn(d2));
    return e > 1.0 ? 1.0 : e;
}

// One axis of the footprint box (ceil(X - R - 1/2), floor(X + R + 1/2),
// clamped to the lattice) and the base node floor(X), exactly as the FP64
// expressions give them.  FP64 issues slowly on this GPU, so the integers come
// from FP32 estimates (error below 2.5e-7 (|X| + R + 1)) whenever these lie
// more than 1e-6 (|X| + R + 1) from an integer, and from FP64 otherwise.
__device__ __forceinline__ void axis_box(double X, float xf, double R, float Rf, int n, int* lo, int* hi, int* base) {
    const float g = 1e-6f * (fabsf(xf) + Rf + 1.f);
    const float tl = xf - (Rf + 0.5f), th = xf + (Rf + 0.5f);
    float cl = ceilf(tl), fh = floorf(th), fb = floorf(xf);
    if (cl - tl < g || tl - (cl - 1.f) < g) cl = (float)ceil(X - R - 0.5);
    if (th - fh < g || (fh + 1.f) - th < g) fh = (float)floor(X + R + 0.5);
    if (xf - fb < g || (fb + 1.f) - xf < g) fb = (float)floor(X);
    *lo = max((int)cl, 0);
    *hi = min((int)fh, n - 1);
    *base = (int)fb;
}

template <typename V>
__device__ __forceinline__ V zero4();
template <> __device__ __forceinline__ float4 zero4<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ double4_32a zero4<double4_32a>() { return make_double4_32a(0., 0., 0., 0.); }

template <typename V>
__global__ void __launch_bounds__(CP_THREADS) k_clear(Geo G, const int* __restrict__ box, V* mk, V* fb, uint8_t* flags) {
    const int p = blockIdx.x;
    int lo[3] = {box[6 * p], box[6 * p + 1], box[6 * p + 2]}, hi[3] = {box[6 * p + 3], box[6 * p + 4], box[6 * p + 5]};
    if (hi[0] < lo[0]) return;
    int ex = hi[0] - lo[0] + 1, ey = hi[1] - lo[1] + 1, ez = hi[2] - lo[2] + 1;
    const int cnt = ex * ey * ez;  // boxes span at most 2 R + 6 nodes per axis (R <= 600): 32-bit
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int qy = q / ex, qz = qy / ey;
        const int x = lo[0] + (q - qy * ex), y = lo[1] + (qy - qz * ey), z = lo[2] + qz;
        long long n = node_index(G, x, y, z);
        mk[n] = zero4<V>();
        fb[n] = zero4<V>();
        flags[((long long)z * G.ny + y) * G.ntx + (x >> 5)] = 0;
    }
}

// Pre-collision deviations of a node whose neighbours are all inside the
// lattice (no wall or wrap): direct A-A addressing; other nodes take the
// generic path.
template <int D, typename S, typename R>
__device__ __forceinline__ void load_node_fast(const Geo& G, const S* __restrict__ f, const S* __restrict__ g, int x,
                                               int y, int z, int parity, R* s, R* sg) {
    using L = Lat<D>;
    const bool inner = x > 0 && x < G.nx - 1 && y > 0 && y < G.ny - 1 && (D == 2 || (z > 0 && z < G.nz - 1));
    if (!inner) {
        load_node<D, S, R>(G, f, g, x, y, z, parity, s, sg);
        return;
    }
    const long long n = node_index(G, x, y, z), sy = G.nx, sz = (long long)G.nx * G.ny;
    if (parity == 0) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) s[i] = (R)Store<S>::ldf(f[i * G.N + n]);
#pragma unroll
        for (int k = 0; k < L::QG; k++) sg[k] = (R)Store<S>::ldg(g[k * G.N + n]);
    } else {
#pragma unroll
        for (int i = 0; i < L::Q; i++) s[i] = (R)Store<S>::ldf(f[L::opp(i) * G.N + n - (L::ex(i) + L::ey(i) * sy + L::ez(i) * sz)]);
#pragma unroll
        for (int k = 0; k < L::QG; k++) sg[k] = (R)Store<S>::ldg(g[L::opp(k) * G.N + n - (L::ex(k) + L::ey(k) * sy + L::ez(k) * sz)]);
    }
}

// FP32 estimate of eps at integer offset (ix, iy, iz) from the particle's base
// node, centre at fractional offset c (both relative to the base node); the
// absolute error is below 1e-6 for radii up to a few hundred nodes.
__device__ __forceinline__ float eps_f32(int ix, int iy, int iz, const float* c, float Rp) {
    float dx = (float)ix - c[0], dy = (float)iy - c[1], dz = (float)iz - c[2];
    return Rp + 0.5f - sqrtf(dx * dx + dy * dy + dz * dz);
}

constexpr float EPS_GUARD = 1e-5f;  // FP32 decisions within this margin are re-taken in FP64

// FEAT: also accumulate, over the particle's owned nodes, the sums the learned
// surrogate's features need, weighted as the coupling weighs each node (w =
// eps rho for the velocity fit, eps for the temperature): sum w, sum w d, sum
// w d d^T (xx, yy, zz, xy, xz, yz), sum w u = sum eps j, sum w d x u = sum eps
// d x j, sum eps dT, sum eps, with d = r - X_p, j the raw momentum and dT = T0 -
// T_ref the raw temperature, into fsum[p][SG_NFSUM].
template <int D, typename S, bool FEAT>
__global__ void __launch_bounds__(CP_THREADS, (Lat<D>::dim == 2 && !FEAT) ? 4 : (FEAT ? 2 : 3)) k_footprint(Geo G, const S* __restrict__ f, const S* __restrict__ g,
                                                          typename Store<S>::V4* __restrict__ mk,
                                                          const double* __restrict__ X, const double* __restrict__ U,
                                                          const double* __restrict__ W, const double* __restrict__ Rr,
                                                          const double* __restrict__ Tp, const int* __restrict__ adj_start,
                                                          const int* __restrict__ adj_nb, double kappa, double Tref,
                                                          int parity, double* Fh, double* Th, double* Hh, double* fsum,
                                                          const int* __restrict__ order) {
    using L = Lat<D>;
    using R = typename Store<S>::R;
    __shared__ double sh_nb[CP_MAXNB][4];
    __shared__ float sh_nbf[CP_MAXNB][4];
    __shared__ int sh_id[CP_MAXNB];
    __shared__ double red[FEAT ? 7 + SG_NFSUM : 7][CP_THREADS / 32];
    float fa[FEAT ? SG_NFSUM : 1];
    for (int k = 0; k < (FEAT ? SG_NFSUM : 1); k++) fa[k] = 0.f;
    // per-particle constants, computed once by the first warp with one value per
    // lane, so that each FP64 operation (slow on this GPU) is one warp instruction:
    // lanes 0-2 the position axes, 3-5 U, 6-8 omega, 9 T_p - T_ref, 10 2 kappa, 11 R
    __shared__ int s_box[6], s_base[3];
    __shared__ float s_cf[3], s_U[3], s_W[3], s_misc[3];
    // the particle: block b takes the b-th of a spatially sorted order (the DEM's
    // cell list), so that blocks running together touch neighbouring nodes
    const int p = order ? order[blockIdx.x] : (int)blockIdx.x;
    const double Xp[3] = {X[3 * p], X[3 * p + 1], X[3 * p + 2]};
    const double Rp = Rr[p];
    const int a0 = adj_start[p];
    int nnb = adj_start[p + 1] - a0;
    if (nnb > CP_MAXNB) nnb = CP_MAXNB;  // the neighbour build rejects more
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double v = 0.0;
        if (lane < 3) v = Xp[lane];
        else if (lane < 6) v = U[3 * p + lane - 3];
        else if (lane < 9) v = W[3 * p + lane - 6];
        else if (lane == 9) v = Tp[p] - Tref;
        else if (lane == 10) v = 2.0 * kappa;
        else if (lane == 11) v = Rp;
        const float vf = (float)v;
        const float Rf = __shfl_sync(0xffffffffu, vf, 11);
        if (lane < 3) {
            int lo = 0, hi = 0, base = 0;
            const int n = lane == 0 ? G.nx : (lane == 1 ? G.ny : G.nz);
            if (lane < Lat<D>::dim) axis_box(v, vf, Rp, Rf, n, &lo, &hi, &base);
            s_box[lane] = lo;
            s_box[3 + lane] = hi;
            s_base[lane] = base;
            s_cf[lane] = (float)(v - (double)base);
        } else if (lane < 6) {
            s_U[lane - 3] = vf;
        } else if (lane < 9) {
            s_W[lane - 6] = vf;
        } else if (lane < 12) {
            s_misc[lane == 9 ? 0 : (lane == 10 ? 1 : 2)] = vf;
        }
    }
    // the neighbours' centres and radii, staged by the other warps while the first
    // sets up the particle: one (neighbour, axis or radius) per thread, with the
    // centre relative to p's base node floor(X_p) (each thread forms that axis's
    // base by the same exact rule as the set-up)
    for (int t = (int)threadIdx.x - 32; t >= 0 && t < 4 * nnb; t += (int)blockDim.x - 32) {
        const int k = t >> 2, a = t & 3;
        const int q = adj_nb[a0 + k];
        if (a == 0) sh_id[k] = q;
        const double v = a < 3 ? X[3 * q + a] : Rr[q];
        sh_nb[k][a] = v;
        if (a < 3) {
            int blo = 0, bhi = 0, b = 0;
            if (a < Lat<D>::dim) {
                const int n = a == 0 ? G.nx : (a == 1 ? G.ny : G.nz);
                axis_box(Xp[a], (float)Xp[a], Rp, (float)Rp, n, &blo, &bhi, &b);
            }
            sh_nbf[k][a] = (float)(v - (double)b);
        } else {
            sh_nbf[k][3] = (float)v;
        }
    }
    __syncthreads();
    const int base[3] = {s_base[0], s_base[1], s_base[2]};
    const float cf[3] = {s_cf[0], s_cf[1], s_cf[2]};
    const int lo[3] = {s_box[0], s_box[1], s_box[2]}, hi[3] = {s_box[3], s_box[4], s_box[5]};
    int ex = hi[0] - lo[0] + 1, ey = hi[1] - lo[1] + 1, ez = hi[2] - lo[2] + 1;
    const int cnt = (ex > 0 && ey > 0 && ez > 0) ? ex * ey * ez : 0;  // 32-bit: boxes of R <= 600
    const float Upf[3] = {s_U[0], s_U[1], s_U[2]};
    const float Wpf[3] = {s_W[0], s_W[1], s_W[2]};
    const R dTp = (R)s_misc[0];
    const R twok = (R)s_misc[1];
    const float Rpf = s_misc[2];
    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // per-thread partials; the block sum is FP64
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int qy = q / ex, qz = qy / ey;
        const int x = lo[0] + (q - qy * ex), y = lo[1] + (qy - qz * ey), z = lo[2] + qz;
        const int ix = x - base[0], iy = y - base[1], iz = z - base[2];
        const float ef = eps_f32(ix, iy, iz, cf, Rpf);
        if (ef <= -EPS_GUARD) continue;  // certainly not covered
        // eps: 1 deep inside (exact), the FP32 value in the open band, FP64 within
        // the guard of the clamp points 0 and 1 (there the decision must be exact)
        float eps;
        double eps64 = -1.0;  // the FP64 value once computed
        if (ef >= 1.0f + EPS_GUARD) {
            eps = 1.0f;
            eps64 = 1.0;
        } else if (ef > EPS_GUARD && ef < 1.0f - EPS_GUARD) {
            eps = ef;
        } else {
            eps64 = eps_of((double)x, (double)y, (double)z, Xp, Rp);
            if (!(eps64 > 0.0)) continue;
            eps = (float)eps64;
        }
        // ownership: the larger eps, ties to the lower index; FP32 decides
        // unless the two values are within the guard of each other
        bool own = true;
        for (int k = 0; k < nnb; k++) {
            const float e2r = eps_f32(ix, iy, iz, sh_nbf[k], sh_nbf[k][3]);
            const float e2f = e2r >= 1.0f + EPS_GUARD ? 1.0f : e2r;
            if (e2f < eps - 2.0f * EPS_GUARD) continue;  // certainly smaller: no contest
            if (!(eps == 1.0f && e2f == 1.0f) && e2f > eps + 2.0f * EPS_GUARD) {  // certainly larger
                own = false;
                break;
            }
            if (eps64 < 0.0) eps64 = eps_of((double)x, (double)y, (double)z, Xp, Rp);
            const double e2 = e2r >= 1.0f + EPS_GUARD ? 1.0 : eps_of((double)x, (double)y, (double)z, sh_nb[k], sh_nb[k][3]);
            if (e2 > eps64 || (e2 == eps64 && sh_id[k] < p)) {
                own = false;
                break;
            }
        }
        if (!own) continue;
        R s[L::Q], sg[L::QG];
        load_node_fast<D, S, R>(G, f, g, x, y, z, parity, s, sg);
        R drho = 0, j[3] = {0, 0, 0}, dT = 0;
#pragma unroll
        for (int i = 0; i < L::Q; i++) {
            drho += s[i];
            if (L::ex(i)) j[0] += L::ex(i) * s[i];
            if (L::ey(i)) j[1] += L::ey(i) * s[i];
            if (L::ez(i)) j[2] += L::ez(i) * s[i];
        }
#pragma unroll
        for (int k = 0; k < L::QG; k++) dT += sg[k];
        const R rho = (R)1 + drho;
        const float arm[3] = {(float)ix - cf[0], (float)iy - cf[1], (float)iz - cf[2]};  // r - X_p
        // U_l = U_p + omega_p x (r - X_p)
        const float Ul[3] = {Upf[0] + (Wpf[1] * arm[2] - Wpf[2] * arm[1]), Upf[1] + (Wpf[2] * arm[0] - Wpf[0] * arm[2]),
                             Upf[2] + (Wpf[0] * arm[1] - Wpf[1] * arm[0])};
        R e;
        if constexpr (sizeof(R) == 8) {  // FP64 storage: the exact value
            if (eps64 < 0.0) eps64 = eps_of((double)x, (double)y, (double)z, Xp, Rp);
            e = (R)eps64;
        } else {
            e = (R)eps;  // FP32 away from the clamp points (error ~1e-7 of eps)
        }
        R M[4];
#pragma unroll
        for (int a = 0; a < 3; a++) M[a] = e * (R)2 * (rho * (R)Ul[a] - j[a]);  // eps F_f (Eqs lbm7, lbm8)
        M[3] = e * twok * (dTp - dT);                                             // eps Q (Eq lbm7.5)
        if (D == 2) M[2] = 0;
        typename Store<S>::V4 mv;
        mv.x = M[0], mv.y = M[1], mv.z = M[2], mv.w = M[3];
        mk[node_index(G, x, y, z)] = mv;
        // Eq lbm13 and the torque about the centre
        const float MF[3] = {(float)M[0], (float)M[1], (float)M[2]};
        acc[0] -= MF[0];
        acc[1] -= MF[1];
        acc[2] -= MF[2];
        acc[3] -= arm[1] * MF[2] - arm[2] * MF[1];
        acc[4] -= arm[2] * MF[0] - arm[0] * MF[2];
        acc[5] -= arm[0] * MF[1] - arm[1] * MF[0];
        acc[6] += (float)M[3];
        if constexpr (FEAT) {
            const float ef = (float)e, w = ef * (float)rho;
            const float ej[3] = {ef * (float)j[0], ef * (float)j[1], Lat<D>::dim == 3 ? ef * (float)j[2] : 0.f};
            const float dz = Lat<D>::dim == 3 ? arm[2] : 0.f;
            const float wd[3] = {w * arm[0], w * arm[1], w * dz};
            fa[0] += w;
            fa[1] += wd[0], fa[2] += wd[1], fa[3] += wd[2];
            fa[4] += wd[0] * arm[0], fa[5] += wd[1] * arm[1], fa[6] += wd[2] * dz;
            fa[7] += wd[0] * arm[1], fa[8] += wd[0] * dz, fa[9] += wd[1] * dz;
            fa[10] += ej[0], fa[11] += ej[1], fa[12] += ej[2];
            fa[13] += arm[1] * ej[2] - dz * ej[1], fa[14] += dz * ej[0] - arm[0] * ej[2], fa[15] += arm[0] * ej[1] - arm[1] * ej[0];
            fa[16] += ef * (float)dT;
            fa[17] += ef;
        }
    }
    // warp sums in FP32 (32 partials, a butterfly: every lane gets the sum); lane
    // a keeps quantity a and the warp converts them all in one FP64 instruction;
    // the per-particle total over the warps is FP64
    const int lane = threadIdx.x & 31;
    float mine = 0.f;
#pragma unroll
    for (int a = 0; a < 7; a++) {
        float v = acc[a];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == a) mine = v;
    }
    if constexpr (FEAT) {
#pragma unroll
        for (int a = 0; a < SG_NFSUM; a++) {
            float v = fa[a];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 7 + a) mine = v;
        }
    }
    if (lane < (FEAT ? 7 + SG_NFSUM : 7)) red[lane][threadIdx.x >> 5] = (double)mine;
    __syncthreads();
    if (threadIdx.x < (FEAT ? 7 + SG_NFSUM : 7)) {
        double v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) v += red[threadIdx.x][w];
        if (threadIdx.x < 3) Fh[3 * p + threadIdx.x] = v;
        else if (threadIdx.x < 6) Th[3 * p + threadIdx.x - 3] = v;
        else if (threadIdx.x == 6) Hh[p] = v;
        else fsum[SG_NFSUM * (long long)p + threadIdx.x - 7] = v;
    }
}

// Spreading over the footprint grown by one node: the marker field of the
// region grown by two nodes is staged in shared memory, then every output node
// gathers its 3^D neighbours from there (Eqs lbm10-lbm12, lbm12.6).
constexpr int SPREAD_SMEM = 46 * 1024;  // plus a few static bytes: under the 48 KB default per CTA

// Shared memory the spread reserves per CTA: the x-summed buffer of the largest
// particle (the output x range, at most floor(2 R_max) + 4 nodes: the footprint
// grown by one node; the y/z ranges one node wider on each side), capped at
// SPREAD_SMEM; a smaller reservation lets more CTAs share an SM.
int spread_smem_bytes(int dim, double rmax, size_t v4) {
    const long long e = (long long)floor(2.0 * rmax) + 4;
    long long b = (long long)v4 * e;
    for (int a = 1; a < dim; a++) b *= e + 2;
    return (int)(b < SPREAD_SMEM ? b : SPREAD_SMEM);
}

template <int D, typename V>
__global__ void __launch_bounds__(CP_THREADS) k_spread(Geo G, const double* __restrict__ X, const double* __restrict__ Rr,
                                                       const V* __restrict__ mk, V* __restrict__ fb, uint8_t* flags, int* box,
                                                       int smem_bytes, const int* __restrict__ order) {
    extern __shared__ __align__(32) unsigned char sm_raw[];
    V* tile = reinterpret_cast<V*>(sm_raw);
    using T = decltype(V().x);
    const int p = order ? order[blockIdx.x] : (int)blockIdx.x;  // as in k_footprint
    __shared__ int s_b[12];  // output box lo/hi, staged box lo/hi, computed once (lane a: axis a)
    if (threadIdx.x < 3) {
        const int a = threadIdx.x;
        const double Xa = X[3 * p + a], R = Rr[p];
        const int n = a == 0 ? G.nx : (a == 1 ? G.ny : G.nz);
        int lo = 0, hi = 0, base = 0;
        if (a < Lat<D>::dim) axis_box(Xa, (float)Xa, R, (float)R, n, &lo, &hi, &base);
        int ilo = lo, ihi = hi;
        if (a < Lat<D>::dim) {
            lo = max(lo - 1, 0);
            hi = min(hi + 1, n - 1);
            ilo = max(lo - 1, 0);
            ihi = min(hi + 1, n - 1);
        }
        s_b[a] = lo, s_b[3 + a] = hi, s_b[6 + a] = ilo, s_b[9 + a] = ihi;
        box[6 * p + a] = lo;
        box[6 * p + 3 + a] = hi;
    }
    __syncthreads();
    const int lo[3] = {s_b[0], s_b[1], s_b[2]}, hi[3] = {s_b[3], s_b[4], s_b[5]};
    const int ilo[3] = {s_b[6], s_b[7], s_b[8]}, ihi[3] = {s_b[9], s_b[10], s_b[11]};
    int ex = hi[0] - lo[0] + 1, ey = hi[1] - lo[1] + 1, ez = hi[2] - lo[2] + 1;
    if (ex <= 0 || ey <= 0 || ez <= 0) return;
    const int sy = ihi[1] - ilo[1] + 1, sz = ihi[2] - ilo[2] + 1;
    // delta_h weights are separable (1/2 at 0, 1/4 at +-1 per axis, Eq lbm12):
    // pass 1 sums along x, from the marker field into shared memory, over the
    // output x range and the y/z range grown by one; pass 2 sums the 3 (2-D) or
    // 3x3 (3-D) y/z neighbours from there.  Every node's value is formed from the
    // same inputs in the same order by whichever CTA computes it, so overlapping
    // boxes still write identical values.
    const int na = ex * sy * sz;  // 32-bit: boxes of R <= 600
    const bool staged = (long long)na * (long long)sizeof(V) <= smem_bytes;
    // launched as a programmatic dependent of the footprint kernel: everything above
    // overlaps its tail; the marker field is read only once that grid has completed
    // and its writes are visible (a no-op when launched without the dependency)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (staged) {
        for (int q = threadIdx.x; q < na; q += blockDim.x) {
            const int qy = q / ex, qz = qy / sy;
            const int x = lo[0] + (q - qy * ex), y = ilo[1] + (qy - qz * sy), z = ilo[2] + qz;
            const long long n0 = node_index(G, x, y, z);
            const V c = mk[n0];
            T a0 = (T)0.5 * c.x, a1 = (T)0.5 * c.y, a2 = (T)0.5 * c.z, a3 = (T)0.5 * c.w;
            if (x > 0) {
                const V m = mk[n0 - 1];
                a0 += (T)0.25 * m.x, a1 += (T)0.25 * m.y, a2 += (T)0.25 * m.z, a3 += (T)0.25 * m.w;
            }
            if (x < G.nx - 1) {
                const V m = mk[n0 + 1];
                a0 += (T)0.25 * m.x, a1 += (T)0.25 * m.y, a2 += (T)0.25 * m.z, a3 += (T)0.25 * m.w;
            }
            V a;
            a.x = a0, a.y = a1, a.z = a2, a.w = a3;
            tile[q] = a;
        }
        __syncthreads();
    }
    const int cnt = ex * ey * ez;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int qy = q / ex, qz = qy / ey;
        const int x = lo[0] + (q - qy * ex), y = lo[1] + (qy - qz * ey), z = lo[2] + qz;
        T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
        if (staged) {
            for (int dz = (Lat<D>::dim == 3 ? -1 : 0); dz <= (Lat<D>::dim == 3 ? 1 : 0); dz++) {
                const int zz = z + dz;
                if (zz < 0 || zz >= G.nz) continue;
                const T wz = Lat<D>::dim == 3 ? (dz == 0 ? (T)0.5 : (T)0.25) : (T)1;
                for (int dy = -1; dy <= 1; dy++) {
                    const int yy = y + dy;
                    if (yy < 0 || yy >= G.ny) continue;
                    const T w = wz * (dy == 0 ? (T)0.5 : (T)0.25);
                    const V a = tile[((long long)(zz - ilo[2]) * sy + (yy - ilo[1])) * ex + (x - lo[0])];
                    s0 += w * a.x;
                    s1 += w * a.y;
                    s2 += w * a.z;
                    s3 += w * a.w;
                }
            }
        } else {  // a region beyond the reserved shared memory: the 27-point gather from global memory
            for (int dz = (Lat<D>::dim == 3 ? -1 : 0); dz <= (Lat<D>::dim == 3 ? 1 : 0); dz++) {
                int zz = z + dz;
                if (zz < 0 || zz >= G.nz) continue;
                for (int dy = -1; dy <= 1; dy++) {
                    int yy = y + dy;
                    if (yy < 0 || yy >= G.ny) continue;
                    for (int dx = -1; dx <= 1; dx++) {
                        int xx = x + dx;
                        if (xx < 0 || xx >= G.nx) continue;
                        T w = (dx == 0 ? (T)0.5 : (T)0.25) * (dy == 0 ? (T)0.5 : (T)0.25);
                        if (Lat<D>::dim == 3) w *= (dz == 0 ? (T)0.5 : (T)0.25);
                        V m = mk[node_index(G, xx, yy, zz)];
                        s0 += w * m.x;
                        s1 += w * m.y;
                        s2 += w * m.z;
                        s3 += w * m.w;
                    }
                }
            }
        }
        V out;
        out.x = s0, out.y = s1, out.z = s2, out.w = s3;
        fb[node_index(G, x, y, z)] = out;
        flags[((long long)z * G.ny + y) * G.ntx + (x >> 5)] = 1;
    }
}

// ------------------------------------------------------- static markers
template <int D, typename S>
__global__ void __launch_bounds__(CP_THREADS) k_markers(Geo G, const S* __restrict__ f, const S* __restrict__ g,
                                                        int nm, const double* __restrict__ MX, const double* __restrict__ MA,
                                                        const double* __restrict__ MT, double kappa, double Tref, int parity,
                                                        typename Store<S>::V4* Ml, double* nu_part) {
    using L = Lat<D>;
    using R = typename Store<S>::R;
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nm) return;
    double Xl[3] = {MX[3 * l], MX[3 * l + 1], MX[3 * l + 2]};
    double Lw[3][4];
    int base[3] = {0, 0, 0};
    for (int a = 0; a < Lat<D>::dim; a++) {
        base[a] = (int)floor(Xl[a]) - 1;
        for (int k = 0; k < 4; k++) {  // Eq lbm6, four points per axis
            double Lk = 1.0;
            for (int mm = 0; mm < 4; mm++)
                if (mm != k) Lk *= (Xl[a] - (base[a] + mm)) / (double)(k - mm);
            Lw[a][k] = Lk;
        }
    }
    R fl[L::Q], gl[L::QG];
#pragma unroll
    for (int i = 0; i < L::Q; i++) fl[i] = 0;
#pragma unroll
    for (int k = 0; k < L::QG; k++) gl[k] = 0;
    int nn[3] = {G.nx, G.ny, G.nz};
    for (int kz = 0; kz < (Lat<D>::dim == 3 ? 4 : 1); kz++)
        for (int ky = 0; ky < 4; ky++)
            for (int kx = 0; kx < 4; kx++) {
                int c[3] = {base[0] + kx, base[1] + ky, Lat<D>::dim == 3 ? base[2] + kz : 0};
                for (int a = 0; a < Lat<D>::dim; a++) c[a] = ((c[a] % nn[a]) + nn[a]) % nn[a];
                R wgt = (R)(Lw[0][kx] * Lw[1][ky] * (Lat<D>::dim == 3 ? Lw[2][kz] : 1.0));
                R s[L::Q], sg[L::QG];
                load_node<D, S, R>(G, f, g, c[0], c[1], c[2], parity, s, sg);
#pragma unroll
                for (int i = 0; i < L::Q; i++) fl[i] += wgt * s[i];
#pragma unroll
                for (int k = 0; k < L::QG; k++) gl[k] += wgt * sg[k];
            }
    R j[3] = {0, 0, 0}, dT = 0;
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        if (L::ex(i)) j[0] += L::ex(i) * fl[i];
        if (L::ey(i)) j[1] += L::ey(i) * fl[i];
        if (L::ez(i)) j[2] += L::ez(i) * fl[i];
    }
#pragma unroll
    for (int k = 0; k < L::QG; k++) dT += gl[k];
    const R A = (R)MA[l];
    const R dTp = (R)(MT[l] - Tref) - dT;  // T_p - T_l
    typename Store<S>::V4 mv;
    mv.x = A * (R)(-2) * j[0];  // static marker: U_l = 0, F_f = -2 j
    mv.y = A * (R)(-2) * j[1];
    mv.z = Lat<D>::dim == 3 ? A * (R)(-2) * j[2] : (R)0;
    mv.w = A * (R)2 * (R)kappa * dTp;
    Ml[l] = mv;
    nu_part[l] = (double)A * (double)dTp;
}

template <typename V>
__global__ void __launch_bounds__(CP_THREADS) k_marker_spread(int nn, const long long* __restrict__ node, const int* __restrict__ start,
                                                              const int* __restrict__ marker, const double* __restrict__ w,
                                                              const V* __restrict__ Ml, V* fb) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nn) return;
    decltype(V().x) s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (int k = start[q]; k < start[q + 1]; k++) {
        V m = Ml[marker[k]];
        decltype(V().x) wk = (decltype(V().x))w[k];
        s0 += wk * m.x;
        s1 += wk * m.y;
        s2 += wk * m.z;
        s3 += wk * m.w;
    }
    V out;
    out.x = s0, out.y = s1, out.z = s2, out.w = s3;
    fb[node[q]] = out;
}

__global__ void __launch_bounds__(CP_THREADS) k_nu_reduce(const double* part, int nm, double scale, double* out) {
    __shared__ double sh[CP_THREADS];
    double v = 0;
    for (int l = threadIdx.x; l < nm; l += blockDim.x) v += part[l];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = CP_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0] * scale;
}

// Sub-grid particles (d_p <= h, the paper's own regime): one PIBM point per
// particle at its centre, moving with it.  One thread per particle:
// Eq lbm6 with four points per axis (at a wall the stencil is shifted inside),
// Eqs lbm7, lbm8, lbm7.5 with A_p = pi d_p^2 / 4, Eq lbm13 for the particle, and
// the delta_h spreading of Eqs lbm10-lbm12 over the 4^D support by atomic
// additions (supports of nearby particles overlap; the order of the additions,
// and so the last bits of F_B, can differ between runs).  The support box is
// recorded for the next clear.
__device__ __forceinline__ double delta_h_dev(double a) { return fabs(a) <= 2.0 ? 0.25 * (1.0 + cospi(0.5 * a)) : 0.0; }

template <typename V> __device__ __forceinline__ void atomic_add4(V* p, double a, double b, double c, double d);
template <> __device__ __forceinline__ void atomic_add4<float4>(float4* p, double a, double b, double c, double d) {
    atomicAdd(&p->x, (float)a), atomicAdd(&p->y, (float)b), atomicAdd(&p->z, (float)c), atomicAdd(&p->w, (float)d);
}
template <> __device__ __forceinline__ void atomic_add4<double4_32a>(double4_32a* p, double a, double b, double c, double d) {
    atomicAdd(&p->x, a), atomicAdd(&p->y, b), atomicAdd(&p->z, c), atomicAdd(&p->w, d);
}

template <int D, typename S>
__global__ void __launch_bounds__(CP_THREADS) k_points(Geo G, const S* __restrict__ f, const S* __restrict__ g, int np,
                                                       const double* __restrict__ X, const double* __restrict__ U,
                                                       const double* __restrict__ Rr, const double* __restrict__ Tp,
                                                       double kappa, double Tref, int parity, typename Store<S>::V4* fb,
                                                       uint8_t* flags, int* box, double* Fh, double* Th, double* Hh) {
    using L = Lat<D>;
    using R = typename Store<S>::R;
    using V = typename Store<S>::V4;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const double Xl[3] = {X[3 * p], X[3 * p + 1], Lat<D>::dim == 3 ? X[3 * p + 2] : 0.0};
    const int nn[3] = {G.nx, G.ny, G.nz};
    double Lw[3][4];
    int base[3] = {0, 0, 0};
    for (int a = 0; a < Lat<D>::dim; a++) {
        int b = (int)floor(Xl[a]) - 1;
        b = b > nn[a] - 4 ? nn[a] - 4 : b;
        b = b < 0 ? 0 : b;
        base[a] = b;
        for (int k = 0; k < 4; k++) {
            double Lk = 1.0;
            for (int m = 0; m < 4; m++)
                if (m != k) Lk *= (Xl[a] - (b + m)) / (double)(k - m);
            Lw[a][k] = Lk;
        }
    }
    R fl[L::Q], gl[L::QG];
#pragma unroll
    for (int i = 0; i < L::Q; i++) fl[i] = 0;
#pragma unroll
    for (int k = 0; k < L::QG; k++) gl[k] = 0;
    for (int kz = 0; kz < (Lat<D>::dim == 3 ? 4 : 1); kz++)
        for (int ky = 0; ky < 4; ky++)
            for (int kx = 0; kx < 4; kx++) {
                const R w = (R)(Lw[0][kx] * Lw[1][ky] * (Lat<D>::dim == 3 ? Lw[2][kz] : 1.0));
                R s[L::Q], sg[L::QG];
                load_node<D, S, R>(G, f, g, base[0] + kx, base[1] + ky, Lat<D>::dim == 3 ? base[2] + kz : 0, parity, s, sg);
#pragma unroll
                for (int i = 0; i < L::Q; i++) fl[i] += w * s[i];
#pragma unroll
                for (int k = 0; k < L::QG; k++) gl[k] += w * sg[k];
            }
    R drho = 0, j[3] = {0, 0, 0}, dT = 0;
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        drho += fl[i];
        if (L::ex(i)) j[0] += L::ex(i) * fl[i];
        if (L::ey(i)) j[1] += L::ey(i) * fl[i];
        if (L::ez(i)) j[2] += L::ez(i) * fl[i];
    }
#pragma unroll
    for (int k = 0; k < L::QG; k++) dT += gl[k];
    const double rho = 1.0 + (double)drho;
    const double A = 3.14159265358979323846 * Rr[p] * Rr[p];
    double MF[3];
    for (int a = 0; a < 3; a++) MF[a] = A * 2.0 * (rho * U[3 * p + a] - (double)j[a]);
    if (D == 2) MF[2] = 0.0;
    const double MQ = A * 2.0 * kappa * ((Tp[p] - Tref) - (double)dT);
    for (int a = 0; a < 3; a++) {
        Fh[3 * p + a] = -MF[a];
        Th[3 * p + a] = 0.0;
    }
    Hh[p] = MQ;
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int a = 0; a < Lat<D>::dim; a++) {
        lo[a] = (int)ceil(Xl[a] - 2.0);
        hi[a] = (int)floor(Xl[a] + 2.0);
        lo[a] = lo[a] < 0 ? 0 : lo[a];
        hi[a] = hi[a] > nn[a] - 1 ? nn[a] - 1 : hi[a];
    }
    for (int a = 0; a < 3; a++) box[6 * p + a] = lo[a], box[6 * p + 3 + a] = hi[a];
    for (int z = lo[2]; z <= hi[2]; z++)
        for (int y = lo[1]; y <= hi[1]; y++)
            for (int x = lo[0]; x <= hi[0]; x++) {
                double w = delta_h_dev(x - Xl[0]) * delta_h_dev(y - Xl[1]);
                if (Lat<D>::dim == 3) w *= delta_h_dev(z - Xl[2]);
                const long long n = node_index(G, x, y, z);
                atomic_add4<V>(fb + n, w * MF[0], w * MF[1], w * MF[2], w * MQ);
                flags[((long long)z * G.ny + y) * G.ntx + (x >> 5)] = 1;
            }
}

// Threads per footprint CTA: in 2-D a box of the largest particle holds at most
// (floor(2 R_max) + 2)^2 nodes, so a block of that many threads (rounded up to
// whole warps, at least two: the set-up warp and a staging warp) covers it in one
// pass without idle warps in the barriers and the block reduction; 3-D boxes take
// several nodes per thread in blocks of CP_THREADS.
static int footprint_threads(const Ctx* c) {
    if (c->tune_coupling_threads > 0) return c->tune_coupling_threads;
    if (c->D != 2) return CP_THREADS;
    const long long e = (long long)floor(2.0 * c->rmax) + 2;
    const long long t = (e * e + 31) / 32 * 32;
    return (int)(t < 64 ? 64 : (t > CP_THREADS ? CP_THREADS : t));
}

template <int D, typename S>
static cudaError_t coupling_impl(Ctx* c, cudaStream_t s, int parity) {
    using V = typename Store<S>::V4;
    if (!c->desc.pibm) return cudaSuccess;
    if (c->np > 0 && c->point) {
        k_points<D, S><<<(c->np + CP_THREADS - 1) / CP_THREADS, CP_THREADS, 0, s>>>(
            c->G, (const S*)c->f, (const S*)c->g, c->np, c->X, c->U, c->R, c->Tp, c->desc.kappa_T, c->desc.T_ref, parity,
            (V*)c->fb[parity], c->flags[parity], c->box[parity], c->Fh, c->Th, c->Hh);
    } else if (c->np > 0) {
        // the DEM's cell list orders the particles in space (a full permutation
        // after every rebuild; the coupling runs after the DEM has finished)
        const int* order = c->tune_coupling_order ? c->cell_ids : nullptr;
        if (c->sg.enabled)  // the surrogate's feature sums ride along
            k_footprint<D, S, true><<<c->np, footprint_threads(c), 0, s>>>(
                c->G, (const S*)c->f, (const S*)c->g, (V*)c->mk[parity], c->X, c->U, c->W, c->R, c->Tp, c->adj_start,
                c->adj_nb, c->desc.kappa_T, c->desc.T_ref, parity, c->Fh, c->Th, c->Hh, c->sg.fsum, order);
        else
            k_footprint<D, S, false><<<c->np, footprint_threads(c), 0, s>>>(
                c->G, (const S*)c->f, (const S*)c->g, (V*)c->mk[parity], c->X, c->U, c->W, c->R, c->Tp, c->adj_start,
                c->adj_nb, c->desc.kappa_T, c->desc.T_ref, parity, c->Fh, c->Th, c->Hh, nullptr, order);
        // programmatic dependent launch: the spread's CTAs start (and set up their boxes)
        // as the footprint's CTAs finish, then wait for the whole footprint grid
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c->np, 1, 1);
        cfg.blockDim = dim3(c->tune_coupling_threads > 0 ? c->tune_coupling_threads : CP_THREADS, 1, 1);
        cfg.dynamicSmemBytes = c->spread_smem;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&cfg, k_spread<D, V>, c->G, (const double*)c->X, (const double*)c->R,
                                           (const V*)c->mk[parity], (V*)c->fb[parity], c->flags[parity], c->box[parity],
                                           c->spread_smem, order);
        if (e != cudaSuccess) return e;
    }
    if (c->nm > 0) {
        int nb = (c->nm + CP_THREADS - 1) / CP_THREADS;
        k_markers<D, S><<<nb, CP_THREADS, 0, s>>>(c->G, (const S*)c->f, (const S*)c->g, c->nm, c->MX, c->MA, c->MT,
                                                  c->desc.kappa_T, c->desc.T_ref, parity, (V*)c->Ml, c->nu_part);
        int nn = c->n_csr_nodes;
        if (nn > 0)
            k_marker_spread<V><<<(nn + CP_THREADS - 1) / CP_THREADS, CP_THREADS, 0, s>>>(nn, c->csr_node, c->csr_start, c->csr_marker,
                                                                                   c->csr_w, (const V*)c->Ml, (V*)c->fb[parity]);
        k_nu_reduce<<<1, CP_THREADS, 0, s>>>(c->nu_part, c->nm, 1.0 / (c->alpha * c->desc.nu_dT), c->nu_val);
    }
    return cudaGetLastError();
}

cudaError_t launch_coupling(Ctx* c, cudaStream_t s, int parity) { PIBM_DISPATCH(c, coupling_impl, c, s, parity); }

// The footprint pass alone with the feature sums (rewrites the same marker
// field and particle loads: the pass is deterministic).
template <int D, typename S>
static cudaError_t footprint_sums_impl(Ctx* c, cudaStream_t s, int parity) {
    using V = typename Store<S>::V4;
    if (!c->desc.pibm || c->np <= 0) return cudaSuccess;
    k_footprint<D, S, true><<<c->np, footprint_threads(c), 0, s>>>(c->G, (const S*)c->f, (const S*)c->g, (V*)c->mk[parity], c->X,
                                                         c->U, c->W, c->R, c->Tp, c->adj_start, c->adj_nb, c->desc.kappa_T,
                                                         c->desc.T_ref, parity, c->Fh, c->Th, c->Hh, c->sg.fsum,
                                                         c->tune_coupling_order ? c->cell_ids : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_footprint_sums(Ctx* c, cudaStream_t s, int parity) {
    PIBM_DISPATCH(c, footprint_sums_impl, c, s, parity);
}

// Zero the coupling fields of one parity on the boxes its last spread recorded.
template <int D, typename S>
static cudaError_t clear_impl(Ctx* c, cudaStream_t s, int parity) {
    using V = typename Store<S>::V4;
    if (!c->desc.pibm || c->np <= 0) return cudaSuccess;
    k_clear<V><<<c->np, CP_THREADS, 0, s>>>(c->G, c->box[parity], (V*)c->mk[parity], (V*)c->fb[parity], c->flags[parity]);
    return cudaGetLastError();
}

cudaError_t launch_coupling_clear(Ctx* c, cudaStream_t s, int parity) { PIBM_DISPATCH(c, clear_impl, c, s, parity); }

int coupling_kernel_count(Ctx* c) {
    if (!c->desc.pibm) return 0;
    // clear (on the DEM stream), footprint, spread; point particles: clear, k_points
    return (c->np > 0 ? (c->point ? 2 : 3) : 0) + (c->nm > 0 ? 3 : 0);
}

}  // namespace pibm

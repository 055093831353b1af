// Lattice kernels: the fused collide-and-stream update of the flow (D2Q9 /
// D3Q19) and thermal (D2Q5 / D3Q7) populations (Section 2.1), plus the
// initialisation, read-back and diagnostic kernels of the lattice state.
//
// Storage: structure of arrays, one plane of nx*ny*nz values per direction,
// x fastest.  Populations are kept as deviations s_i = f_i - w_i (density 1)
// and s_gk = g_k - w_k T_ref, so that the small velocity-carrying part keeps
// its relative precision in FP32.  Streaming follows the A-A pattern in place:
// even steps read and write the node's own slots (the post-collision value of
// direction i goes to the slot of its opposite), odd steps read from and write
// to the neighbours, so one array serves both time levels.
#include <float.h>

#include <type_traits>

#include "pibm_internal.cuh"

namespace pibm {

// Collision constants in the arithmetic type R (no per-thread conversions:
// GB300's FP64 pipe is slow, and a double-to-float conversion runs on it).
template <typename R>
struct CollideParams {
    R omf, omg;        // 1 / tau_f, 1 / tau_g
    R cf, cg;          // 1 - 1/(2 tau_f), 1 - 1/(2 tau_g)
    R buoy, Tref;      // U_c^2 / L_c, reference temperature
    R body[3];
    R abb[6];          // anti-bounce-back offset 2 w (T_w - T_ref) per face (w of a non-rest thermal direction)
    int gaxis, buoyancy;
};

// One node update: moments, forcing, BGK collision of f and g.
//   rho = 1 + sum s_i, j = sum e_i s_i, T = T_ref + sum s_gk + Q_B / 2
//   F = F_B + body + buoy (T - T_ref) e_up,  u = (j + F/2) / rho
//   Eq lbm2 + lbm3 + lbm9 in deviation form:
//     s_i* = s_i + (s_i^eq - s_i)/tau_f + (1 - 1/2tau_f) w_i [3 (e_i - u) + 9 (e_i.u) e_i] . F
//     s_i^eq = w_i (rho - 1 + rho (3 e.u + 4.5 (e.u)^2 - 1.5 u^2))
//   Eq lbm2.5 + lbm3.5 (linear, D2Q5 / D3Q7) + lbm12.5:
//     s_gk* = s_gk + (w_k (T - T_ref + T e.u / cs_T^2) - s_gk)/tau_g + (1 - 1/2tau_g) w_k Q_B
template <int D, typename R>
__device__ __forceinline__ void collide_node(R* s, R* sg, R fbx, R fby, R fbz, R qb, const CollideParams<R>& P) {
    using L = Lat<D>;
    R drho = 0, jx = 0, jy = 0, jz = 0, dT = 0;
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        drho += s[i];
        if (L::ex(i)) jx += L::ex(i) * s[i];
        if (L::ey(i)) jy += L::ey(i) * s[i];
        if (L::ez(i)) jz += L::ez(i) * s[i];
    }
#pragma unroll
    for (int k = 0; k < L::QG; k++) dT += sg[k];
    const R half = (R)0.5;
    dT += half * qb;                        // T - T_ref
    const R T = (R)P.Tref + dT;
    R Fx = fbx + (R)P.body[0], Fy = fby + (R)P.body[1], Fz = fbz + (R)P.body[2];
    if (P.buoyancy) {
        R fbu = (R)P.buoy * dT;
        if (P.gaxis == 0) Fx += fbu;
        else if (P.gaxis == 1) Fy += fbu;
        else Fz += fbu;
    }
    const R rho = (R)1 + drho;
    const R inv_rho = (R)1 / rho;
    const R ux = (jx + half * Fx) * inv_rho, uy = (jy + half * Fy) * inv_rho, uz = (jz + half * Fz) * inv_rho;
    const R uu = ux * ux + uy * uy + uz * uz;
    const R uF = ux * Fx + uy * Fy + uz * Fz;
    const R omf = (R)P.omf, cf = (R)P.cf;
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        const R wi = (R)L::w(i);
        R eu = 0, eF = 0;
        if (L::ex(i)) { eu += L::ex(i) * ux; eF += L::ex(i) * Fx; }
        if (L::ey(i)) { eu += L::ey(i) * uy; eF += L::ey(i) * Fy; }
        if (L::ez(i)) { eu += L::ez(i) * uz; eF += L::ez(i) * Fz; }
        const R seq = wi * (drho + rho * ((R)3 * eu + (R)4.5 * eu * eu - (R)1.5 * uu));
        const R Fi = cf * wi * ((R)3 * (eF - uF) + (R)9 * eu * eF);
        s[i] = s[i] + omf * (seq - s[i]) + Fi;
    }
    const R omg = (R)P.omg, gq = (R)P.cg * qb;
#pragma unroll
    for (int k = 0; k < L::QG; k++) {
        const R wk = (R)L::wg(k);
        R eu = 0;
        if (L::ex(k)) eu += L::ex(k) * ux;
        if (L::ey(k)) eu += L::ey(k) * uy;
        if (L::ez(k)) eu += L::ez(k) * uz;
        const R sgeq = wk * (dT + T * eu * (R)L::inv_csT2);
        sg[k] = sg[k] + omg * (sgeq - sg[k]) + wk * gq;
    }
}

// Odd-step source of direction i for a node whose y/z neighbours are all
// inside: only the x neighbour can leave the lattice.  Per-lane selects keep a
// warp that holds an x-boundary node on this path (no divergence into the
// generic boundary code).  Returns the flat index and sets bounce when the x
// neighbour lies beyond a wall (then the node's own slot of direction i holds
// the bounced value).
template <int D, int I>
__device__ __forceinline__ long long odd_src(const Geo& G, long long n, int x, long long sy, long long sz, bool& bounce) {
    using L = Lat<D>;
    constexpr int ex = L::ex(I);
    long long off = (long long)L::ey(I) * sy + (long long)L::ez(I) * sz;
    bounce = false;
    if (ex == 0) return (long long)L::opp(I) * G.N + n - off;
    int sx = x - ex;
    long long dx = ex;
    if (sx < 0 || sx >= G.nx) {
        if (G.per[0]) dx = ex + (sx < 0 ? -G.nx : G.nx);  // wrap: source at sx +- nx
        else bounce = true;
    }
    return bounce ? (long long)I * G.N + n : (long long)L::opp(I) * G.N + n - off - dx;
}

template <int D, int I>
__device__ __forceinline__ long long odd_dst(const Geo& G, long long n, int x, long long sy, long long sz, bool& bounce) {
    using L = Lat<D>;
    constexpr int ex = L::ex(I);
    long long off = (long long)L::ey(I) * sy + (long long)L::ez(I) * sz;
    bounce = false;
    if (ex == 0) return (long long)I * G.N + n + off;
    int tx = x + ex;
    long long dx = ex;
    if (tx < 0 || tx >= G.nx) {
        if (G.per[0]) dx = ex + (tx < 0 ? G.nx : -G.nx);
        else bounce = true;
    }
    return bounce ? (long long)L::opp(I) * G.N + n : (long long)I * G.N + n + off + dx;
}

template <int D, typename S, int I>
struct OddLoad {
    using R = typename Store<S>::R;
    static __device__ __forceinline__ void run(const Geo& G, const CollideParams<R>& P, const S* f, const S* g, long long n,
                                               int x, long long sy, long long sz, R* s, R* sg) {
        using L = Lat<D>;
        bool b;
        long long idx = odd_src<D, I>(G, n, x, sy, sz, b);
        s[I] = Store<S>::ldf(f[idx]);
        if (I < L::QG) {
            R v = Store<S>::ldg(g[idx]);
            constexpr int face = L::ex(I) > 0 ? 0 : 1;  // face crossed by x - e_I
            if (b && face_iso(G, face)) v = P.abb[face] - v;
            sg[I < L::QG ? I : 0] = v;
        }
        OddLoad<D, S, I + 1>::run(G, P, f, g, n, x, sy, sz, s, sg);
    }
};
template <typename S> struct OddLoad<2, S, 9> {
    using R = typename Store<S>::R;
    static __device__ __forceinline__ void run(const Geo&, const CollideParams<R>&, const S*, const S*, long long, int,
                                               long long, long long, R*, R*) {}
};
template <typename S> struct OddLoad<3, S, 19> {
    using R = typename Store<S>::R;
    static __device__ __forceinline__ void run(const Geo&, const CollideParams<R>&, const S*, const S*, long long, int,
                                               long long, long long, R*, R*) {}
};

template <int D, typename S, int I>
struct OddStore {
    using R = typename Store<S>::R;
    static __device__ __forceinline__ void run(const Geo& G, const CollideParams<R>& P, S* f, S* g, long long n, int x,
                                               long long sy, long long sz, const R* s, const R* sg) {
        using L = Lat<D>;
        bool b;
        long long idx = odd_dst<D, I>(G, n, x, sy, sz, b);
        f[idx] = Store<S>::stf(s[I]);
        if (I < L::QG) {
            R v = sg[I < L::QG ? I : 0];
            constexpr int face = L::ex(I) > 0 ? 1 : 0;  // face crossed by x + e_I
            if (b && face_iso(G, face)) v = P.abb[face] - v;
            g[idx] = Store<S>::stg(v);
        }
        OddStore<D, S, I + 1>::run(G, P, f, g, n, x, sy, sz, s, sg);
    }
};
template <typename S> struct OddStore<2, S, 9> {
    using R = typename Store<S>::R;
    static __device__ __forceinline__ void run(const Geo&, const CollideParams<R>&, S*, S*, long long, int, long long,
                                               long long, const R*, const R*) {}
};
template <typename S> struct OddStore<3, S, 19> {
    using R = typename Store<S>::R;
    static __device__ __forceinline__ void run(const Geo&, const CollideParams<R>&, S*, S*, long long, int, long long,
                                               long long, const R*, const R*) {}
};

// Flat offsets of the A-A slots relative to the node index n, per direction
// (uniform over the grid, computed once on the host): odd-step sources
// plane opp(i) at n - e_i, odd-step destinations plane i at n + e_i, even-step
// loads plane i at n and stores plane opp(i) at n.
struct AAOffsets {
    long long src[19], dst[19], ld[19], st[19];
};

template <int D, typename S, int PARITY>
__global__ void __launch_bounds__(256) k_stream_collide(Geo G, S* __restrict__ f, S* __restrict__ g,
                                                        const typename Store<S>::V4* __restrict__ fb,
                                                        const uint8_t* __restrict__ flags,
                                                        CollideParams<typename Store<S>::R> P, AAOffsets O) {
    using L = Lat<D>;
    using R = typename Store<S>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= G.nx) return;
    const long long n = node_index(G, x, y, z);
    const long long sy = G.nx, sz = (long long)G.nx * G.ny;
    // y and z are uniform across the block, so this test never splits a warp
    const bool inner_yz = y > 0 && y < G.ny - 1 && (D == 2 || (z > 0 && z < G.nz - 1));
    R s[L::Q], sg[L::QG];
    // lanes on the x faces need the wrap / bounce fix-up (warp-divergent only there)
    const bool xedge = x == 0 || x == G.nx - 1;
    if (PARITY == 0) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) s[i] = Store<S>::ldf(f[n + O.ld[i]]);
#pragma unroll
        for (int k = 0; k < L::QG; k++) sg[k] = Store<S>::ldg(g[n + O.ld[k]]);
    } else if (inner_yz && !xedge) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) s[i] = Store<S>::ldf(f[n + O.src[i]]);
#pragma unroll
        for (int k = 0; k < L::QG; k++) sg[k] = Store<S>::ldg(g[n + O.src[k]]);
    } else if (inner_yz) {
        OddLoad<D, S, 0>::run(G, P, f, g, n, x, sy, sz, s, sg);
    } else {
        load_node<D, S, R>(G, f, g, x, y, z, 1, s, sg);
    }
    R fbx = 0, fby = 0, fbz = 0, qb = 0;
    if (flags[((long long)z * G.ny + y) * G.ntx + (x >> 5)]) {
        const typename Store<S>::V4 v = fb[n];
        fbx = v.x;
        fby = v.y;
        fbz = v.z;
        qb = v.w;
    }
    collide_node<D, R>(s, sg, fbx, fby, fbz, qb, P);
    if (PARITY == 0) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) f[n + O.st[i]] = Store<S>::stf(s[i]);
#pragma unroll
        for (int k = 0; k < L::QG; k++) g[n + O.st[k]] = Store<S>::stg(sg[k]);
    } else if (inner_yz && !xedge) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) f[n + O.dst[i]] = Store<S>::stf(s[i]);
#pragma unroll
        for (int k = 0; k < L::QG; k++) g[n + O.dst[k]] = Store<S>::stg(sg[k]);
    } else if (inner_yz) {
        OddStore<D, S, 0>::run(G, P, f, g, n, x, sy, sz, s, sg);
    } else {
#pragma unroll
        for (int i = 0; i < L::Q; i++) {
            long long idx;
            post_slot(G, x, y, z, L::ex(i), L::ey(i), L::ez(i), i, L::opp(i), 1, idx);
            f[idx] = Store<S>::stf(s[i]);
        }
#pragma unroll
        for (int k = 0; k < L::QG; k++) {
            long long idx;
            int face = post_slot(G, x, y, z, L::ex(k), L::ey(k), L::ez(k), k, L::opp(k), 1, idx);
            R v = sg[k];
            if (face_iso(G, face)) v = P.abb[face] - v;
            g[idx] = Store<S>::stg(v);
        }
    }
}

template <typename R>
static CollideParams<R> collide_params(const Ctx* c) {
    CollideParams<R> P;
    P.omf = (R)(1.0 / c->tau_f);
    P.omg = (R)(1.0 / c->tau_g);
    P.cf = (R)(1.0 - 0.5 / c->tau_f);
    P.cg = (R)(1.0 - 0.5 / c->tau_g);
    P.buoy = (R)c->buoy;
    P.Tref = (R)c->desc.T_ref;
    for (int a = 0; a < 3; a++) P.body[a] = (R)c->desc.body_force[a];
    double wgk = c->D == 2 ? Lat<2>::wg(1) : Lat<3>::wg(1);
    for (int f = 0; f < 6; f++) P.abb[f] = (R)(2.0 * wgk * c->G.dTw[f]);
    P.gaxis = c->desc.gravity_axis;
    P.buoyancy = c->desc.buoyancy;
    return P;
}

// Generic odd-step store of one node's post-collision populations (any
// boundary).  side = -1 or +1 restricts it to the directions that leave the
// lattice through that x face (the rest were stored by the pair path).
template <int D, typename S>
__device__ __forceinline__ void store_node(const Geo& G, const CollideParams<typename Store<S>::R>& P, S* f, S* g, int x,
                                           int y, int z, const typename Store<S>::R* s, const typename Store<S>::R* sg,
                                           int side) {
    using L = Lat<D>;
    using R = typename Store<S>::R;
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        if (side != 0 && L::ex(i) != side) continue;
        long long idx;
        post_slot(G, x, y, z, L::ex(i), L::ey(i), L::ez(i), i, L::opp(i), 1, idx);
        f[idx] = Store<S>::stf(s[i]);
    }
#pragma unroll
    for (int k = 0; k < L::QG; k++) {
        if (side != 0 && L::ex(k) != side) continue;
        long long idx;
        int face = post_slot(G, x, y, z, L::ex(k), L::ey(k), L::ez(k), k, L::opp(k), 1, idx);
        R v = sg[k];
        if (face_iso(G, face)) v = P.abb[face] - v;
        g[idx] = Store<S>::stg(v);
    }
}

// ---------------------------------------------------------------------------
// 16-bit storage, two nodes per thread.  Populations of the pair (x0, x0+1)
// move as one 32-bit half2 / bfloat162 word with a packed conversion.  In odd
// steps a direction with e_x = +1 reads x-1 (the upper half of the left
// neighbour lane's aligned pair, via a warp shuffle) and e_x = -1 reads x+1
// (the lower half of the right lane's pair); the lanes at either end of the
// warp fetch the one element beyond it with a scalar access.  Stores mirror
// this.  Lanes holding a node on an x face run the generic path for that node
// as well (wrap or bounce-back); accesses that would cross the row end are
// skipped there.  Requires nx to be a multiple of 64 (whole warps per row).
template <typename S> struct Pair;
template <> struct Pair<__half> {
    using T = __half2;
    static __device__ __forceinline__ float2 ldf(T v) { float2 r = __half22float2(v); return make_float2(r.x * 0.0009765625f, r.y * 0.0009765625f); }
    static __device__ __forceinline__ float2 ldg(T v) { float2 r = __half22float2(v); return make_float2(r.x * 0.00390625f, r.y * 0.00390625f); }
    static __device__ __forceinline__ T stf(float a, float b) { return __floats2half2_rn(a * 1024.0f, b * 1024.0f); }
    static __device__ __forceinline__ T stg(float a, float b) { return __floats2half2_rn(a * 256.0f, b * 256.0f); }
};
template <> struct Pair<__nv_bfloat16> {
    using T = __nv_bfloat162;
    static __device__ __forceinline__ float2 ldf(T v) { return __bfloat1622float2(v); }
    static __device__ __forceinline__ float2 ldg(T v) { return __bfloat1622float2(v); }
    static __device__ __forceinline__ T stf(float a, float b) { return __floats2bfloat162_rn(a, b); }
    static __device__ __forceinline__ T stg(float a, float b) { return __floats2bfloat162_rn(a, b); }
};

template <int D, typename S, int PARITY>
__global__ void __launch_bounds__(256) k_stream_collide_pair(Geo G, S* __restrict__ f, S* __restrict__ g,
                                                             const float4* __restrict__ fb, const uint8_t* __restrict__ flags,
                                                             CollideParams<float> P, AAOffsets O) {
    using L = Lat<D>;
    using PT = typename Pair<S>::T;
    using St = Store<S>;
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y, z = blockIdx.z;
    const int lane = threadIdx.x & 31;
    if (x0 >= G.nx) return;  // whole warps only: nx / 2 is a multiple of 32
    const long long n0 = node_index(G, x0, y, z);
    const bool inner_yz = y > 0 && y < G.ny - 1 && (D == 2 || (z > 0 && z < G.nz - 1));
    const bool lo_edge = x0 == 0, hi_edge = x0 + 1 == G.nx - 1;
    float s0[L::Q], s1[L::Q], g0[L::QG], g1[L::QG];
    if (PARITY == 0) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) {
            float2 v = Pair<S>::ldf(*reinterpret_cast<const PT*>(f + n0 + O.ld[i]));
            s0[i] = v.x, s1[i] = v.y;
        }
#pragma unroll
        for (int k = 0; k < L::QG; k++) {
            float2 v = Pair<S>::ldg(*reinterpret_cast<const PT*>(g + n0 + O.ld[k]));
            g0[k] = v.x, g1[k] = v.y;
        }
    } else if (inner_yz) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) {
            const int ex = L::ex(i);
            const long long e = n0 + O.src[i];  // source element of node x0
            if (ex == 0) {
                float2 v = Pair<S>::ldf(*reinterpret_cast<const PT*>(f + e));
                s0[i] = v.x, s1[i] = v.y;
            } else if (ex == 1) {  // node x reads x-1: (x0-1, x0)
                float2 v = Pair<S>::ldf(*reinterpret_cast<const PT*>(f + e + 1));
                float left = __shfl_up_sync(0xffffffffu, v.y, 1);
                if (lane == 0) left = lo_edge ? 0.f : St::ldf(f[e]);
                s0[i] = left, s1[i] = v.x;
            } else {  // node x reads x+1: (x0+1, x0+2)
                float2 v = Pair<S>::ldf(*reinterpret_cast<const PT*>(f + e - 1));
                float right = __shfl_down_sync(0xffffffffu, v.x, 1);
                if (lane == 31) right = hi_edge ? 0.f : St::ldf(f[e + 1]);
                s0[i] = v.y, s1[i] = right;
            }
        }
#pragma unroll
        for (int k = 0; k < L::QG; k++) {
            const int ex = L::ex(k);
            const long long e = n0 + O.src[k];
            if (ex == 0) {
                float2 v = Pair<S>::ldg(*reinterpret_cast<const PT*>(g + e));
                g0[k] = v.x, g1[k] = v.y;
            } else if (ex == 1) {
                float2 v = Pair<S>::ldg(*reinterpret_cast<const PT*>(g + e + 1));
                float left = __shfl_up_sync(0xffffffffu, v.y, 1);
                if (lane == 0) left = lo_edge ? 0.f : St::ldg(g[e]);
                g0[k] = left, g1[k] = v.x;
            } else {
                float2 v = Pair<S>::ldg(*reinterpret_cast<const PT*>(g + e - 1));
                float right = __shfl_down_sync(0xffffffffu, v.x, 1);
                if (lane == 31) right = hi_edge ? 0.f : St::ldg(g[e + 1]);
                g0[k] = v.y, g1[k] = right;
            }
        }
        if (lo_edge) load_node<D, S, float>(G, f, g, x0, y, z, 1, s0, g0);
        if (hi_edge) load_node<D, S, float>(G, f, g, x0 + 1, y, z, 1, s1, g1);
    } else {
        load_node<D, S, float>(G, f, g, x0, y, z, 1, s0, g0);
        load_node<D, S, float>(G, f, g, x0 + 1, y, z, 1, s1, g1);
    }
    float b0[4] = {0.f, 0.f, 0.f, 0.f}, b1[4] = {0.f, 0.f, 0.f, 0.f};
    if (flags[((long long)z * G.ny + y) * G.ntx + (x0 >> 5)]) {  // x0 and x0+1 share a 32-node tile
        const float4 v0 = fb[n0], v1 = fb[n0 + 1];
        b0[0] = v0.x, b0[1] = v0.y, b0[2] = v0.z, b0[3] = v0.w;
        b1[0] = v1.x, b1[1] = v1.y, b1[2] = v1.z, b1[3] = v1.w;
    }
    collide_node<D, float>(s0, g0, b0[0], b0[1], b0[2], b0[3], P);
    collide_node<D, float>(s1, g1, b1[0], b1[1], b1[2], b1[3], P);
    if (PARITY == 0) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) *reinterpret_cast<PT*>(f + n0 + O.st[i]) = Pair<S>::stf(s0[i], s1[i]);
#pragma unroll
        for (int k = 0; k < L::QG; k++) *reinterpret_cast<PT*>(g + n0 + O.st[k]) = Pair<S>::stg(g0[k], g1[k]);
    } else if (inner_yz) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) {
            const int ex = L::ex(i);
            const long long e = n0 + O.dst[i];  // destination element of node x0
            if (ex == 0) {
                *reinterpret_cast<PT*>(f + e) = Pair<S>::stf(s0[i], s1[i]);
            } else if (ex == 1) {  // x0 -> x0+1, x0+1 -> x0+2: this lane owns the word (x0, x0+1)
                float left = __shfl_up_sync(0xffffffffu, s1[i], 1);
                if (lane > 0) *reinterpret_cast<PT*>(f + e - 1) = Pair<S>::stf(left, s0[i]);
                else f[e] = St::stf(s0[i]);
                if (lane == 31 && !hi_edge) f[e + 1] = St::stf(s1[i]);
            } else {  // x0 -> x0-1, x0+1 -> x0: this lane owns the word (x0, x0+1)
                float right = __shfl_down_sync(0xffffffffu, s0[i], 1);
                if (lane < 31) *reinterpret_cast<PT*>(f + e + 1) = Pair<S>::stf(s1[i], right);
                else f[e + 1] = St::stf(s1[i]);
                if (lane == 0 && !lo_edge) f[e] = St::stf(s0[i]);
            }
        }
#pragma unroll
        for (int k = 0; k < L::QG; k++) {
            const int ex = L::ex(k);
            const long long e = n0 + O.dst[k];
            if (ex == 0) {
                *reinterpret_cast<PT*>(g + e) = Pair<S>::stg(g0[k], g1[k]);
            } else if (ex == 1) {
                float left = __shfl_up_sync(0xffffffffu, g1[k], 1);
                if (lane > 0) *reinterpret_cast<PT*>(g + e - 1) = Pair<S>::stg(left, g0[k]);
                else g[e] = St::stg(g0[k]);
                if (lane == 31 && !hi_edge) g[e + 1] = St::stg(g1[k]);
            } else {
                float right = __shfl_down_sync(0xffffffffu, g0[k], 1);
                if (lane < 31) *reinterpret_cast<PT*>(g + e + 1) = Pair<S>::stg(g1[k], right);
                else g[e + 1] = St::stg(g1[k]);
                if (lane == 0 && !lo_edge) g[e] = St::stg(g0[k]);
            }
        }
        if (lo_edge) store_node<D, S>(G, P, f, g, x0, y, z, s0, g0, -1);
        if (hi_edge) store_node<D, S>(G, P, f, g, x0 + 1, y, z, s1, g1, +1);
    } else {
        store_node<D, S>(G, P, f, g, x0, y, z, s0, g0, 0);
        store_node<D, S>(G, P, f, g, x0 + 1, y, z, s1, g1, 0);
    }
}

template <int D>
static AAOffsets aa_offsets(const Geo& G) {
    using L = Lat<D>;
    AAOffsets O;
    const long long sy = G.nx, sz = (long long)G.nx * G.ny;
    for (int i = 0; i < 19; i++) O.src[i] = O.dst[i] = O.ld[i] = O.st[i] = 0;
    for (int i = 0; i < L::Q; i++) {
        long long off = L::ex(i) + L::ey(i) * sy + L::ez(i) * sz;
        O.src[i] = (long long)L::opp(i) * G.N - off;
        O.dst[i] = (long long)i * G.N + off;
        O.ld[i] = (long long)i * G.N;
        O.st[i] = (long long)L::opp(i) * G.N;
    }
    return O;
}

template <int D, typename S>
static cudaError_t pair_launch(Ctx* c, cudaStream_t s, int parity) {
    if constexpr (std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value) {
        const int pairs = c->G.nx / 2;
        dim3 block(pairs < 256 ? pairs : 256), grid((pairs + 255) / 256, c->G.ny, c->G.nz);
        CollideParams<float> P = collide_params<float>(c);
        AAOffsets O = aa_offsets<D>(c->G);
        if (parity == 0)
            k_stream_collide_pair<D, S, 0><<<grid, block, 0, s>>>(c->G, (S*)c->f, (S*)c->g, (const float4*)c->fb[parity],
                                                                  c->flags[parity], P, O);
        else
            k_stream_collide_pair<D, S, 1><<<grid, block, 0, s>>>(c->G, (S*)c->f, (S*)c->g, (const float4*)c->fb[parity],
                                                                  c->flags[parity], P, O);
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}

template <int D, typename S>
static cudaError_t sc_launch(Ctx* c, cudaStream_t s, int parity) {
    constexpr bool half = std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value;
    if (half && c->G.nx % 64 == 0 && !c->tune_scalar_lattice) return pair_launch<D, S>(c, s, parity);
    dim3 block(256), grid((c->G.nx + 255) / 256, c->G.ny, c->G.nz);
    if (c->G.nx <= 128) block.x = 128, grid.x = (c->G.nx + 127) / 128;
    using R = typename Store<S>::R;
    CollideParams<R> P = collide_params<R>(c);
    AAOffsets O = aa_offsets<D>(c->G);
    using V = typename Store<S>::V4;
    if (parity == 0)
        k_stream_collide<D, S, 0><<<grid, block, 0, s>>>(c->G, (S*)c->f, (S*)c->g, (const V*)c->fb[parity], c->flags[parity], P, O);
    else
        k_stream_collide<D, S, 1><<<grid, block, 0, s>>>(c->G, (S*)c->f, (S*)c->g, (const V*)c->fb[parity], c->flags[parity], P, O);
    return cudaGetLastError();
}

cudaError_t launch_stream_collide(Ctx* c, cudaStream_t s, int parity) { PIBM_DISPATCH(c, sc_launch, c, s, parity); }

// ----------------------------------------------------------- initialisation
// Rest equilibrium at density 1 and temperature T_init: s_i = 0, s_gk = w_k (T_init - T_ref).
template <int D, typename S>
__global__ void k_init(long long N, S* f, S* g, double dT0) {
    using L = Lat<D>;
    using R = typename Store<S>::R;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) f[i * N + n] = Store<S>::stf((R)0);
#pragma unroll
        for (int k = 0; k < L::QG; k++) g[k * N + n] = Store<S>::stg((R)(L::wg(k) * dT0));
    }
}

template <int D, typename S>
static cudaError_t init_launch(Ctx* c, double dT0) {
    k_init<D, S><<<1024, 256, 0, c->s0>>>(c->G.N, (S*)c->f, (S*)c->g, dT0);
    return cudaGetLastError();
}

cudaError_t launch_init_equilibrium(Ctx* c) {
    double dT0 = c->desc.T_init - c->desc.T_ref;
    PIBM_DISPATCH(c, init_launch, c, dT0);
}

// ------------------------------------------------- population read / write
// One plane (direction q) of the populations of the current time, as doubles.
template <int D, typename S>
__global__ void k_read_plane(Geo G, const S* __restrict__ arr, int thermal, int q, int parity, double* out, double Tref) {
    using L = Lat<D>;
    long long N = G.N;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        int x = (int)(n % G.nx), y = (int)((n / G.nx) % G.ny), z = (int)(n / ((long long)G.nx * G.ny));
        int ex = 0, ey = 0, ez = 0, io = 0;
        double w = 0;
#pragma unroll
        for (int i = 0; i < L::Q; i++)
            if (i == q) { ex = L::ex(i); ey = L::ey(i); ez = L::ez(i); io = L::opp(i); w = thermal ? L::wg(i) : L::w(i); }
        long long idx;
        int face = pop_slot(G, x, y, z, ex, ey, ez, q, io, parity, idx);
        double v = thermal ? (double)Store<S>::ldg(arr[idx]) : (double)Store<S>::ldf(arr[idx]);
        if (thermal && face_iso(G, face)) v = 2.0 * w * face_dTw(G, face) - v;
        out[n] = v + (thermal ? w * Tref : w);
    }
}

template <int D, typename S>
__global__ void k_write_plane(Geo G, S* __restrict__ arr, int thermal, int q, int parity, const double* in, double Tref) {
    using L = Lat<D>;
    long long N = G.N;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        int x = (int)(n % G.nx), y = (int)((n / G.nx) % G.ny), z = (int)(n / ((long long)G.nx * G.ny));
        int ex = 0, ey = 0, ez = 0, io = 0;
        double w = 0;
#pragma unroll
        for (int i = 0; i < L::Q; i++)
            if (i == q) { ex = L::ex(i); ey = L::ey(i); ez = L::ez(i); io = L::opp(i); w = thermal ? L::wg(i) : L::w(i); }
        long long idx;
        int face = pop_slot(G, x, y, z, ex, ey, ez, q, io, parity, idx);
        double v = in[n] - (thermal ? w * Tref : w);
        if (thermal && face_iso(G, face)) v = 2.0 * w * face_dTw(G, face) - v;
        using R = typename Store<S>::R;
        arr[idx] = thermal ? Store<S>::stg((R)v) : Store<S>::stf((R)v);
    }
}

template <int D, typename S>
static cudaError_t rw_plane(Ctx* c, int which, int q, int parity, bool write) {
    const S* arr = (const S*)(which == 0 ? c->f : c->g);
    if (write)
        k_write_plane<D, S><<<1024, 256, 0, c->s0>>>(c->G, (S*)arr, which, q, parity, c->plane, c->desc.T_ref);
    else
        k_read_plane<D, S><<<1024, 256, 0, c->s0>>>(c->G, arr, which, q, parity, c->plane, c->desc.T_ref);
    return cudaGetLastError();
}

cudaError_t launch_read_plane(Ctx* c, int which, int q, int parity) { PIBM_DISPATCH(c, rw_plane, c, which, q, parity, false); }

cudaError_t launch_write_plane(Ctx* c, int which, int q, int parity) { PIBM_DISPATCH(c, rw_plane, c, which, q, parity, true); }

// ------------------------------------------------------ macroscopic fields
template <int D, typename S>
__device__ void node_macro(const Geo& G, const S* f, const S* g, const typename Store<S>::V4* fb, const uint8_t* flags,
                           const CollideParams<double>& P, int x, int y, int z, int parity, double* out /*rho,ux,uy,uz,T,fbx,fby,fbz,qb,T0*/) {
    using L = Lat<D>;
    double s[L::Q], sg[L::QG];
    load_node<D, S, double>(G, f, g, x, y, z, parity, s, sg);
    long long n = node_index(G, x, y, z);
    double fbv[4] = {0, 0, 0, 0};
    if (flags[((long long)z * G.ny + y) * G.ntx + (x >> 5)]) {
        typename Store<S>::V4 v = fb[n];
        fbv[0] = v.x, fbv[1] = v.y, fbv[2] = v.z, fbv[3] = v.w;
    }
    double drho = 0, j[3] = {0, 0, 0}, dT = 0;
    for (int i = 0; i < L::Q; i++) {
        drho += s[i];
        j[0] += L::ex(i) * s[i];
        j[1] += L::ey(i) * s[i];
        j[2] += L::ez(i) * s[i];
    }
    for (int k = 0; k < L::QG; k++) dT += sg[k];
    double T0 = P.Tref + dT;
    dT += 0.5 * fbv[3];
    double F[3] = {fbv[0] + P.body[0], fbv[1] + P.body[1], fbv[2] + P.body[2]};
    if (P.buoyancy) F[P.gaxis] += P.buoy * dT;
    double rho = 1.0 + drho;
    out[0] = rho;
    for (int a = 0; a < 3; a++) out[1 + a] = (j[a] + 0.5 * F[a]) / rho;
    out[4] = P.Tref + dT;
    for (int a = 0; a < 4; a++) out[5 + a] = fbv[a];
    out[9] = T0;
}

template <int D, typename S>
__global__ void k_macro(Geo G, const S* f, const S* g, const typename Store<S>::V4* fb, const uint8_t* flags,
                        CollideParams<double> P, int field, int parity, double* out) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < G.N; n += (long long)gridDim.x * blockDim.x) {
        int x = (int)(n % G.nx), y = (int)((n / G.nx) % G.ny), z = (int)(n / ((long long)G.nx * G.ny));
        double m[10];
        node_macro<D, S>(G, f, g, fb, flags, P, x, y, z, parity, m);
        out[n] = m[field];
    }
}

template <int D, typename S>
static cudaError_t macro_launch(Ctx* c, int field, int parity) {
    using V = typename Store<S>::V4;
    k_macro<D, S><<<1024, 256, 0, c->s0>>>(c->G, (const S*)c->f, (const S*)c->g, (const V*)c->fb[parity], c->flags[parity],
                                           collide_params<double>(c), field, parity, c->plane);
    return cudaGetLastError();
}

cudaError_t launch_macro(Ctx* c, int field, int parity) { PIBM_DISPATCH(c, macro_launch, c, field, parity); }

// ------------------------------------------------------------ diagnostics
// Deterministic two-level reduction: a fixed grid of 512 blocks writes
// partials, one block combines them in a fixed order.
constexpr int DIAG_BLOCKS = 512;

template <int D, typename S>
__global__ void __launch_bounds__(256) k_diag_lattice(Geo G, const S* f, const S* g, const typename Store<S>::V4* fb,
                                                      const uint8_t* flags, CollideParams<double> P, int parity, double* part) {
    __shared__ double sh[4][256];
    double mass = 0, heat = 0, umax = 0, bad = 0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < G.N; n += (long long)gridDim.x * blockDim.x) {
        int x = (int)(n % G.nx), y = (int)((n / G.nx) % G.ny), z = (int)(n / ((long long)G.nx * G.ny));
        double m[10];
        node_macro<D, S>(G, f, g, fb, flags, P, x, y, z, parity, m);
        mass += m[0];
        heat += m[9];
        double um = sqrt(m[1] * m[1] + m[2] * m[2] + m[3] * m[3]);
        if (!(um <= umax)) umax = isfinite(um) ? um : umax;
        if (!isfinite(m[0]) || !isfinite(m[9]) || !isfinite(um)) bad = 1;
    }
    int t = threadIdx.x;
    sh[0][t] = mass, sh[1][t] = heat, sh[2][t] = umax, sh[3][t] = bad;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (t < s) {
            sh[0][t] += sh[0][t + s];
            sh[1][t] += sh[1][t + s];
            sh[2][t] = fmax(sh[2][t], sh[2][t + s]);
            sh[3][t] = fmax(sh[3][t], sh[3][t + s]);
        }
        __syncthreads();
    }
    if (t == 0)
        for (int a = 0; a < 4; a++) part[4 * blockIdx.x + a] = sh[a][0];
}

__global__ void __launch_bounds__(256) k_diag_final(const double* part, int nblocks, const double* U, const double* W,
                                                    const double* X, const double* m, const double* I, int np,
                                                    int gaxis, double* out) {
    __shared__ double sh[6][256];
    int t = threadIdx.x;
    double mass = 0, heat = 0, umax = 0, bad = 0, ke = 0, hmin = 1e300;
    for (int b = t; b < nblocks; b += 256) {
        mass += part[4 * b];
        heat += part[4 * b + 1];
        umax = fmax(umax, part[4 * b + 2]);
        bad = fmax(bad, part[4 * b + 3]);
    }
    for (int p = t; p < np; p += 256) {
        double v2 = U[3 * p] * U[3 * p] + U[3 * p + 1] * U[3 * p + 1] + U[3 * p + 2] * U[3 * p + 2];
        double w2 = W[3 * p] * W[3 * p] + W[3 * p + 1] * W[3 * p + 1] + W[3 * p + 2] * W[3 * p + 2];
        ke += 0.5 * m[p] * v2 + 0.5 * I[p] * w2;
        hmin = fmin(hmin, X[3 * p + gaxis]);
        if (!isfinite(v2) || !isfinite(w2)) bad = 1;
    }
    sh[0][t] = mass, sh[1][t] = heat, sh[2][t] = ke, sh[3][t] = hmin, sh[4][t] = umax, sh[5][t] = bad;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (t < s) {
            sh[0][t] += sh[0][t + s];
            sh[1][t] += sh[1][t + s];
            sh[2][t] += sh[2][t + s];
            sh[3][t] = fmin(sh[3][t], sh[3][t + s]);
            sh[4][t] = fmax(sh[4][t], sh[4][t + s]);
            sh[5][t] = fmax(sh[5][t], sh[5][t + s]);
        }
        __syncthreads();
    }
    if (t == 0) {
        for (int a = 0; a < 6; a++) out[a] = sh[a][0];
        if (np == 0) out[3] = 0.0;
    }
}

template <int D, typename S>
static cudaError_t diag_launch(Ctx* c, int parity) {
    using V = typename Store<S>::V4;
    k_diag_lattice<D, S><<<DIAG_BLOCKS, 256, 0, c->s0>>>(c->G, (const S*)c->f, (const S*)c->g, (const V*)c->fb[parity],
                                                         c->flags[parity], collide_params<double>(c), parity, c->red);
    k_diag_final<<<1, 256, 0, c->s0>>>(c->red, DIAG_BLOCKS, c->U, c->W, c->X, c->m, c->I, c->np,
                                       c->desc.gravity_axis, c->red + 4 * DIAG_BLOCKS);
    return cudaGetLastError();
}

cudaError_t launch_diagnostics(Ctx* c, int parity) { PIBM_DISPATCH(c, diag_launch, c, parity); }

}  // namespace pibm

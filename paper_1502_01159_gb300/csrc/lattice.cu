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
//
// One node per thread.  The collision is written with explicitly rounded
// operations, so its result does not depend on how the compiler schedules or
// fuses them.
#include <float.h>

#include <algorithm>
#include <type_traits>

#include "pibm_internal.cuh"

namespace pibm {

// Collision constants in the arithmetic type R (no per-thread conversions:
// GB300's FP64 pipe is slow, and a double-to-float conversion runs on it).
template <typename R>
struct CollideParams {
    R om1f, om1g;      // 1 - 1/tau_f, 1 - 1/tau_g
    R c9f, c3f, m3f;   // 9 (1 - 1/(2 tau_f)), 3 (1 - 1/(2 tau_f)), -3 (1 - 1/(2 tau_f))
    R cg;              // 1 - 1/(2 tau_g)
    R buoy, Tref;      // U_c^2 / L_c, reference temperature
    R body[3];
    R abb[6];          // anti-bounce-back offset 2 w (T_w - T_ref) per face (w of a non-rest thermal direction)
    int gaxis, buoyancy;
};

// ------------------------------------------------------ collision arithmetic
// Every add, subtract, multiply and fused multiply-add of the collision is
// written out with its rounding (float, or double for FP64 storage), so the
// compiler contracts nothing and the result is fixed by the source alone.
__device__ __forceinline__ float op_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float op_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float op_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float op_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float op_rcp(float a) { return __frcp_rn(a); }
__device__ __forceinline__ double op_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double op_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double op_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double op_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double op_rcp(double a) { return __drcp_rn(a); }
// a constant of the arithmetic type T
template <typename T> struct Bc;
template <> struct Bc<float> { static __device__ __forceinline__ float of(float v) { return v; } };
template <> struct Bc<double> { static __device__ __forceinline__ double of(double v) { return v; } };

// One node update: moments, forcing, BGK collision of f and g.
//   rho = 1 + sum s_i, j = sum e_i s_i, T = T_ref + sum s_gk + Q_B / 2
//   F = F_B + body + buoy (T - T_ref) e_up,  u = (j + F/2) / rho
//   Eq lbm2 + lbm3 + lbm9 in deviation form:
//     s_i* = s_i + (s_i^eq - s_i)/tau_f + (1 - 1/2tau_f) w_i [3 (e_i - u) + 9 (e_i.u) e_i] . F
//     s_i^eq = w_i (rho - 1 + rho (3 e.u + 4.5 (e.u)^2 - 1.5 u^2))
//   Eq lbm2.5 + lbm3.5 (linear, D2Q5 / D3Q7) + lbm12.5:
//     s_gk* = s_gk + (w_k (T - T_ref + T e.u / cs_T^2) - s_gk)/tau_g + (1 - 1/2tau_g) w_k Q_B
template <int D, typename T, typename R>
__device__ __forceinline__ void collide_node(T* s, T* sg, T fbx, T fby, T fbz, T qb, const CollideParams<R>& P) {
    using L = Lat<D>;
    using B = Bc<T>;
    T drho = s[0], jx = B::of(0), jy = B::of(0), jz = B::of(0);
#pragma unroll
    for (int i = 1; i < L::Q; i++) {
        drho = op_add(drho, s[i]);
        if (L::ex(i) > 0) jx = op_add(jx, s[i]);
        if (L::ex(i) < 0) jx = op_sub(jx, s[i]);
        if (L::ey(i) > 0) jy = op_add(jy, s[i]);
        if (L::ey(i) < 0) jy = op_sub(jy, s[i]);
        if (L::ez(i) > 0) jz = op_add(jz, s[i]);
        if (L::ez(i) < 0) jz = op_sub(jz, s[i]);
    }
    T dT = sg[0];
#pragma unroll
    for (int k = 1; k < L::QG; k++) dT = op_add(dT, sg[k]);
    const T half = B::of(0.5);
    dT = op_fma(half, qb, dT);  // T - T_ref
    const T Tt = op_add(B::of(P.Tref), dT);
    T Fx = op_add(fbx, B::of(P.body[0])), Fy = op_add(fby, B::of(P.body[1])), Fz = op_add(fbz, B::of(P.body[2]));
    if (P.buoyancy) {
        const T fbu = op_mul(B::of(P.buoy), dT);
        if (P.gaxis == 0) Fx = op_add(Fx, fbu);
        else if (P.gaxis == 1) Fy = op_add(Fy, fbu);
        else Fz = op_add(Fz, fbu);
    }
    const T rho = op_add(B::of(1), drho);
    const T inv_rho = op_rcp(rho);
    const T ux = op_mul(op_fma(half, Fx, jx), inv_rho);
    const T uy = op_mul(op_fma(half, Fy, jy), inv_rho);
    const T uz = op_mul(op_fma(half, Fz, jz), inv_rho);
    const T uu = op_fma(uz, uz, op_fma(uy, uy, op_mul(ux, ux)));
    const T uF = op_fma(uz, Fz, op_fma(uy, Fy, op_mul(ux, Fx)));
    const T om1 = B::of(P.om1f);
    // Opposite directions i, i' share e.u and e.F up to sign, so equilibrium
    // and forcing split into parts even and odd in e:
    //   s_i^eq = w (p0 + 4.5 rho (e.u)^2) + w 3 rho e.u,  p0 = drho - 1.5 rho u^2
    //   F_i    = w cf (9 (e.u)(e.F) - 3 u.F) + w 3 cf e.F
    // and the update keeps the non-equilibrium form (small correction added to
    // the equilibrium, no cancellation of two large terms):
    //   s_i* = s_i^eq + F_i + (1 - 1/tau) (s_i - s_i^eq)
    const T p0 = op_fma(B::of(-1.5), op_mul(rho, uu), drho);
    const T q0 = op_mul(B::of(4.5), rho), r0 = op_mul(B::of(3), rho);
    const T k0 = op_mul(B::of(P.m3f), uF), c9 = B::of(P.c9f), c3 = B::of(P.c3f);
    {
        const T w0 = B::of(L::w(0));
        const T seq = op_mul(w0, p0);
        s[0] = op_fma(om1, op_sub(s[0], seq), op_fma(w0, k0, seq));
    }
#pragma unroll
    for (int i = 1; i < L::Q; i++) {
        if (L::opp(i) < i) continue;
        const int io = L::opp(i);
        const T wi = B::of(L::w(i));
        // e.u and e.F: the sum of the non-zero components with their signs
        T eu = B::of(0), eF = B::of(0);
        bool first = true;
        if (L::ex(i)) { eu = L::ex(i) > 0 ? ux : op_sub(eu, ux); eF = L::ex(i) > 0 ? Fx : op_sub(eF, Fx); first = false; }
        if (L::ey(i)) {
            if (first) { eu = L::ey(i) > 0 ? uy : op_sub(eu, uy); eF = L::ey(i) > 0 ? Fy : op_sub(eF, Fy); }
            else { eu = L::ey(i) > 0 ? op_add(eu, uy) : op_sub(eu, uy); eF = L::ey(i) > 0 ? op_add(eF, Fy) : op_sub(eF, Fy); }
            first = false;
        }
        if (L::ez(i)) {
            if (first) { eu = L::ez(i) > 0 ? uz : op_sub(eu, uz); eF = L::ez(i) > 0 ? Fz : op_sub(eF, Fz); }
            else { eu = L::ez(i) > 0 ? op_add(eu, uz) : op_sub(eu, uz); eF = L::ez(i) > 0 ? op_add(eF, Fz) : op_sub(eF, Fz); }
        }
        const T es = op_mul(wi, op_fma(q0, op_mul(eu, eu), p0));  // even / odd equilibrium parts
        const T ea = op_mul(op_mul(wi, r0), eu);
        const T fs = op_mul(wi, op_fma(c9, op_mul(eu, eF), k0));  // even / odd forcing parts
        const T fa = op_mul(op_mul(wi, c3), eF);
        const T ni = op_sub(op_sub(s[i], es), ea);                // non-equilibrium parts
        const T no = op_add(op_sub(s[io], es), ea);
        const T a = op_add(es, fs), b = op_add(ea, fa);
        s[i] = op_fma(om1, ni, op_add(a, b));
        s[io] = op_fma(om1, no, op_sub(a, b));
    }
    // thermal, the same split: s_gk^eq = w_k dT + w_k (T / cs_T^2) e.u, source w_k cg Q_B
    const T om1g = B::of(P.om1g);
    const T gq = op_mul(B::of(P.cg), qb), kT = op_mul(Tt, B::of(L::inv_csT2));
    {
        const T w0 = B::of(L::wg(0));
        const T seq = op_mul(w0, dT);
        sg[0] = op_fma(om1g, op_sub(sg[0], seq), op_fma(w0, gq, seq));
    }
#pragma unroll
    for (int k = 1; k < L::QG; k++) {
        if (L::opp(k) < k) continue;
        const int ko = L::opp(k);
        const T wk = B::of(L::wg(k));
        T eu = L::ex(k) ? ux : (L::ey(k) ? uy : uz);
        if (L::ex(k) + L::ey(k) + L::ez(k) < 0) eu = op_sub(B::of(0), eu);
        const T es = op_mul(wk, dT), ea = op_mul(op_mul(wk, kT), eu), src = op_mul(wk, gq);
        const T ni = op_sub(op_sub(sg[k], es), ea), no = op_add(op_sub(sg[ko], es), ea);
        const T a = op_add(es, src);
        sg[k] = op_fma(om1g, ni, op_add(a, ea));
        sg[ko] = op_fma(om1g, no, op_sub(a, ea));
    }
}

// The first non-zero component of e_i is positive: one direction of each
// opposite pair (the other is opp(i)).
template <int D>
__host__ __device__ constexpr bool lead_positive(int i) {
    using L = Lat<D>;
    return L::ex(i) != 0 ? L::ex(i) > 0 : (L::ey(i) != 0 ? L::ey(i) > 0 : L::ez(i) > 0);
}

// The collision of the 16-bit storage forms, the same BGK update and Guo
// forcing as collide_node, in the storage's own units (deviations times 2^KF
// for f and 2^KG for g: FP16's exact scales; 0 for BF16) and regrouped so that
// an opposite pair (i, i') costs nine operations past e.u and e.F:
//   s_i* = om1 s_i + A + B,  s_i'* = om1 s_i' + A - B,  g = 1 - om1 = 1/tau
//   A = w_i [e.u (4.5 g rho e.u + 9 cf e.F) + g p0 - 3 cf u.F]   (even in e)
//   B = w_i [3 g rho e.u + 3 cf e.F]                              (odd in e)
// with p0 = drho - 1.5 rho u^2 and cf = 1 - 1/(2 tau); the moments come from
// the pair sums s_i + s_i' and differences s_i - s_i'.  collide_node's
// non-equilibrium grouping costs about twice the operations; the rounding it
// saves is FP32's, 2^-24 relative, against the 2^-8 (BF16) or 2^-11 (FP16) of
// the stored result.  Thermal, likewise: s_k* = om1g s_k + w_k (g_g dT + cg Q_B)
// +- w_k g_g (T / cs_T^2) e.u.
template <int D, int KF, int KG>
__device__ __forceinline__ void collide_lean(float* s, float* sg, float fbx, float fby, float fbz, float qb,
                                             const CollideParams<float>& P) {
    using L = Lat<D>;
    constexpr double sf = (double)(1 << KF), sgs = (double)(1 << KG);
    float drho = s[0], jx = 0.f, jy = 0.f, jz = 0.f;
    bool fx = true, fy = true, fz = true;
#pragma unroll
    for (int i = 1; i < L::Q; i++) {
        if (!lead_positive<D>(i)) continue;
        const int io = L::opp(i);
        const float sum = op_add(s[i], s[io]), dif = op_sub(s[i], s[io]);
        drho = op_add(drho, sum);
        if (L::ex(i)) { jx = fx ? (L::ex(i) > 0 ? dif : op_sub(0.f, dif)) : (L::ex(i) > 0 ? op_add(jx, dif) : op_sub(jx, dif)); fx = false; }
        if (L::ey(i)) { jy = fy ? (L::ey(i) > 0 ? dif : op_sub(0.f, dif)) : (L::ey(i) > 0 ? op_add(jy, dif) : op_sub(jy, dif)); fy = false; }
        if (L::ez(i)) { jz = fz ? (L::ez(i) > 0 ? dif : op_sub(0.f, dif)) : (L::ez(i) > 0 ? op_add(jz, dif) : op_sub(jz, dif)); fz = false; }
    }
    float dT = sg[0];
#pragma unroll
    for (int k = 1; k < L::QG; k++) dT = op_add(dT, sg[k]);
    if (KF != 0) {
        const float is = (float)(1.0 / sf);  // exact: a power of two
        drho = op_mul(drho, is);
        jx = op_mul(jx, is);
        jy = op_mul(jy, is);
        jz = op_mul(jz, is);
    }
    if (KG != 0) dT = op_mul(dT, (float)(1.0 / sgs));
    dT = op_fma(0.5f, qb, dT);  // T - T_ref
    const float Tt = op_add(P.Tref, dT);
    float Fx = op_add(fbx, P.body[0]), Fy = op_add(fby, P.body[1]), Fz = op_add(fbz, P.body[2]);
    if (P.buoyancy) {
        const float fbu = op_mul(P.buoy, dT);
        if (P.gaxis == 0) Fx = op_add(Fx, fbu);
        else if (P.gaxis == 1) Fy = op_add(Fy, fbu);
        else Fz = op_add(Fz, fbu);
    }
    const float rho = op_add(1.f, drho);
    const float inv_rho = op_rcp(rho);
    const float ux = op_mul(op_fma(0.5f, Fx, jx), inv_rho);
    const float uy = op_mul(op_fma(0.5f, Fy, jy), inv_rho);
    const float uz = op_mul(op_fma(0.5f, Fz, jz), inv_rho);
    const float uu = op_fma(uz, uz, op_fma(uy, uy, op_mul(ux, ux)));
    const float uF = op_fma(uz, Fz, op_fma(uy, Fy, op_mul(ux, Fx)));
    const float om1 = P.om1f, g = op_sub(1.f, om1);  // 1/tau, so that g + om1 = 1 in FP32
    const float p0 = op_fma(-1.5f, op_mul(rho, uu), drho);
    const float grho = op_mul(g, rho);
    const float Gq = op_mul(4.5f, grho), Gr = op_mul(3.f, grho);
    const float P0 = op_fma(g, p0, op_mul(P.m3f, uF));
    s[0] = op_fma(om1, s[0], op_mul((float)(L::w(0) * sf), P0));
#pragma unroll
    for (int i = 1; i < L::Q; i++) {
        if (!lead_positive<D>(i)) continue;
        const int io = L::opp(i);
        // per weight class (the compiler shares these between pairs of one class)
        const float wsf = (float)(L::w(i) * sf);
        const float aq = op_mul(wsf, Gq), ar = op_mul(wsf, Gr), ap = op_mul(wsf, P0);
        const float a9 = op_mul(wsf, P.c9f), a3 = op_mul(wsf, P.c3f);
        // e.u and e.F, the leading component positive
        float eu = ux, eF = Fx;
        if (L::ex(i) == 0) {
            eu = uy;
            eF = Fy;
            if (L::ey(i) == 0) {
                eu = uz;
                eF = Fz;
            } else if (L::ez(i)) {
                eu = L::ez(i) > 0 ? op_add(eu, uz) : op_sub(eu, uz);
                eF = L::ez(i) > 0 ? op_add(eF, Fz) : op_sub(eF, Fz);
            }
        } else {
            if (L::ey(i)) {
                eu = L::ey(i) > 0 ? op_add(eu, uy) : op_sub(eu, uy);
                eF = L::ey(i) > 0 ? op_add(eF, Fy) : op_sub(eF, Fy);
            }
            if (L::ez(i)) {
                eu = L::ez(i) > 0 ? op_add(eu, uz) : op_sub(eu, uz);
                eF = L::ez(i) > 0 ? op_add(eF, Fz) : op_sub(eF, Fz);
            }
        }
        const float A = op_fma(eu, op_fma(aq, eu, op_mul(a9, eF)), ap);
        const float B = op_fma(ar, eu, op_mul(a3, eF));
        s[i] = op_fma(om1, s[i], op_add(A, B));
        s[io] = op_fma(om1, s[io], op_sub(A, B));
    }
    const float om1g = P.om1g, gg = op_sub(1.f, om1g);
    const float Ag = op_fma(gg, dT, op_mul(P.cg, qb));
    const float Bg = op_mul(gg, op_mul(Tt, (float)L::inv_csT2));
    sg[0] = op_fma(om1g, sg[0], op_mul((float)(L::wg(0) * sgs), Ag));
#pragma unroll
    for (int k = 1; k < L::QG; k++) {
        if (!lead_positive<D>(k)) continue;
        const int ko = L::opp(k);
        const float wsg = (float)(L::wg(k) * sgs);
        const float a = op_mul(wsg, Ag), bw = op_mul(wsg, Bg);
        const float eu = L::ex(k) ? ux : (L::ey(k) ? uy : uz);
        const float b = op_mul(bw, eu);
        sg[k] = op_fma(om1g, sg[k], op_add(a, b));
        sg[ko] = op_fma(om1g, sg[ko], op_sub(a, b));
    }
}

// Loads and stores of the lattice kernel: in physical units (FP32, FP64), or
// in the storage's own units for the 16-bit forms, which collide_lean takes.
template <typename S, bool RAW> struct LatIo {
    using R = typename Store<S>::R;
    static __device__ __forceinline__ R ldf(S v) { return Store<S>::ldf(v); }
    static __device__ __forceinline__ R ldg(S v) { return Store<S>::ldg(v); }
    static __device__ __forceinline__ S stf(R v) { return Store<S>::stf(v); }
    static __device__ __forceinline__ S stg(R v) { return Store<S>::stg(v); }
    static __device__ __forceinline__ R gunit(R v) { return v; }  // a physical g value in these units
};
template <typename S> struct LatIo<S, true> {
    static __device__ __forceinline__ float ldf(S v) { return Store<S>::rawf(v); }
    static __device__ __forceinline__ float ldg(S v) { return Store<S>::rawf(v); }
    static __device__ __forceinline__ S stf(float v) { return Store<S>::raws(v); }
    static __device__ __forceinline__ S stg(float v) { return Store<S>::raws(v); }
    static __device__ __forceinline__ float gunit(float v) {
        return Store<S>::KG ? op_mul(v, (float)(1 << Store<S>::KG)) : v;
    }
};

// Flat offsets of the A-A slots relative to the node index n, per direction
// (uniform over the grid, computed once on the host): odd-step sources
// plane opp(i) at n - e_i, odd-step destinations plane i at n + e_i, even-step
// loads plane i at n and stores plane opp(i) at n.  IX = int when every offset
// fits in 32 bits (Q N < 2^31 elements): then each access is the thread's node
// pointer plus a 32-bit offset, one multiply-add.
template <typename IX>
struct AAOffsets {
    IX src[19], dst[19], ld[19], st[19];
};

// Odd-step loads and stores of a warp whose nodes can have a neighbour beyond
// a face: a warp holding an x-face node, or a row on a y or z face.  Every lane
// starts from the fast path's offset; per direction, a neighbour beyond a
// periodic face is taken from the periodic image (the offset shifted by the
// axis's extent times its stride), and a neighbour beyond a wall sends the
// access to the node's own slot of direction i (loads) / opp(i) (stores),
// where bounce-back left or leaves the value, with the anti-bounce-back of an
// isothermal face for g.  When a diagonal neighbour leaves through two faces
// the wall of the later axis (z, then y, then x) decides, as in pop_slot /
// post_slot.  y and z are uniform across a warp and x only selects, so no warp
// diverges; interior lanes get the fast path's offsets exactly.
template <int D, typename S, typename IX, bool RAW>
__device__ __forceinline__ void odd_load_face(const Geo& G, const CollideParams<typename Store<S>::R>& P, const S* fn,
                                              const S* gn, int x, int y, int z, const AAOffsets<IX>& O,
                                              typename Store<S>::R* s, typename Store<S>::R* sg) {
    using L = Lat<D>;
    using R = typename Store<S>::R;
    const bool xlo = x == 0, xhi = x == G.nx - 1, ylo = y == 0, yhi = y == G.ny - 1;
    const bool zlo = L::dim == 3 && z == 0, zhi = L::dim == 3 && z == G.nz - 1;
    const IX sx = (IX)G.nx, sy = (IX)G.nx * (IX)G.ny, sz = (IX)G.N;
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
        // x - e_i beyond a face, per axis
        const bool ox = (ex > 0 && xlo) || (ex < 0 && xhi);
        const bool oy = (ey > 0 && ylo) || (ey < 0 && yhi);
        const bool oz = (ez > 0 && zlo) || (ez < 0 && zhi);
        int face = -1;
        if (ox && !G.per[0]) face = ex > 0 ? 0 : 1;
        if (oy && !G.per[1]) face = ey > 0 ? 2 : 3;
        if (oz && !G.per[2]) face = ez > 0 ? 4 : 5;
        IX idx = O.src[i];
        if (ox) idx += (IX)ex * sx;
        if (oy) idx += (IX)ey * sy;
        if (oz) idx += (IX)ez * sz;
        if (face >= 0) idx = O.ld[i];
        s[i] = LatIo<S, RAW>::ldf(fn[idx]);
        if (i < L::QG) {
            R v = LatIo<S, RAW>::ldg(gn[idx]);
            if constexpr (RAW) {
                if (face_iso(G, face)) v = op_sub(LatIo<S, RAW>::gunit(P.abb[face]), v);
            } else {
                if (face_iso(G, face)) v = op_sub(P.abb[face], v);
            }
            sg[i < L::QG ? i : 0] = v;
        }
    }
}

template <int D, typename S, typename IX, bool RAW>
__device__ __forceinline__ void odd_store_face(const Geo& G, const CollideParams<typename Store<S>::R>& P, S* fn, S* gn,
                                               int x, int y, int z, const AAOffsets<IX>& O,
                                               const typename Store<S>::R* s, const typename Store<S>::R* sg) {
    using L = Lat<D>;
    using R = typename Store<S>::R;
    const bool xlo = x == 0, xhi = x == G.nx - 1, ylo = y == 0, yhi = y == G.ny - 1;
    const bool zlo = L::dim == 3 && z == 0, zhi = L::dim == 3 && z == G.nz - 1;
    const IX sx = (IX)G.nx, sy = (IX)G.nx * (IX)G.ny, sz = (IX)G.N;
#pragma unroll
    for (int i = 0; i < L::Q; i++) {
        const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
        // x + e_i beyond a face, per axis
        const bool ox = (ex > 0 && xhi) || (ex < 0 && xlo);
        const bool oy = (ey > 0 && yhi) || (ey < 0 && ylo);
        const bool oz = (ez > 0 && zhi) || (ez < 0 && zlo);
        int face = -1;
        if (ox && !G.per[0]) face = ex > 0 ? 1 : 0;
        if (oy && !G.per[1]) face = ey > 0 ? 3 : 2;
        if (oz && !G.per[2]) face = ez > 0 ? 5 : 4;
        IX idx = O.dst[i];
        if (ox) idx -= (IX)ex * sx;
        if (oy) idx -= (IX)ey * sy;
        if (oz) idx -= (IX)ez * sz;
        if (face >= 0) idx = O.st[i];
        fn[idx] = LatIo<S, RAW>::stf(s[i]);
        if (i < L::QG) {
            R v = sg[i < L::QG ? i : 0];
            if constexpr (RAW) {
                if (face_iso(G, face)) v = op_sub(LatIo<S, RAW>::gunit(P.abb[face]), v);
            } else {
                if (face_iso(G, face)) v = op_sub(P.abb[face], v);
            }
            gn[idx] = LatIo<S, RAW>::stg(v);
        }
    }
}

// One thread per node.  FP32 and FP64 storage: at most 64 registers for the
// odd step of FP32 (two 512-thread blocks per SM).  16-bit storage: the node's
// 26 populations occupy as many registers as in FP32 for half the bytes, so
// the kernel waits on memory with too few warps resident.  Bounded to 384
// threads and three blocks of them (56 registers, no spills) and launched in
// 128-thread blocks, nine blocks (36 warps) fit an SM instead of eight; at
// 384^3 (BF16) that took the kernel from 1.44 to 1.29 ms.  48 registers spill
// and lose.
template <typename S>
constexpr int sc_max_threads() { return sizeof(S) == 2 ? 384 : 512; }
template <typename S, int PARITY>
constexpr int sc_min_blocks() { return sizeof(S) == 2 ? 3 : ((PARITY == 1 && sizeof(S) != 8) ? 2 : 0); }

template <int D, typename S, int PARITY, typename IX>
__global__ void __launch_bounds__(sc_max_threads<S>(), (sc_min_blocks<S, PARITY>())) k_stream_collide(Geo G, S* __restrict__ f, S* __restrict__ g,
                                                        const typename Store<S>::V4* __restrict__ fb,
                                                        const uint8_t* __restrict__ flags,
                                                        CollideParams<typename Store<S>::R> P, AAOffsets<IX> O) {
    using L = Lat<D>;
    using R = typename Store<S>::R;
    // block: blockDim.x nodes of a row (a multiple of 32) x blockDim.y rows
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    if (x >= G.nx || y >= G.ny) return;
    const long long n = node_index(G, x, y, z);
    S* const fn = f + n;  // this node's slot in plane 0 of f and g: every fast-path access is one offset from here
    S* const gn = g + n;
    // y and z are uniform across a warp, so this test never splits one
    const bool inner_yz = y > 0 && y < G.ny - 1 && (D == 2 || (z > 0 && z < G.nz - 1));
    // 16-bit storage collides in its own units (collide_lean); FP32 and FP64 in
    // physical units with every rounding of collide_node
    constexpr bool LEAN = sizeof(S) == 2;
    using IO = LatIo<S, LEAN>;
    R s[L::Q], sg[L::QG];
    // warps holding a node on an x face take the per-lane-select path as a
    // whole (it is exact for interior lanes too), so no warp splits in two;
    // blockDim.x is a multiple of 32, so x & ~31 is the warp's first node
    const int xw = x & ~31;
    const bool xedge = xw == 0 || xw + 31 >= G.nx - 1;
    if (PARITY == 0) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) s[i] = IO::ldf(fn[O.ld[i]]);
#pragma unroll
        for (int k = 0; k < L::QG; k++) sg[k] = IO::ldg(gn[O.ld[k]]);
    } else if (inner_yz && !xedge) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) s[i] = IO::ldf(fn[O.src[i]]);
#pragma unroll
        for (int k = 0; k < L::QG; k++) sg[k] = IO::ldg(gn[O.src[k]]);
    } else {
        odd_load_face<D, S, IX, LEAN>(G, P, fn, gn, x, y, z, O, s, sg);
    }
    R fbx = 0, fby = 0, fbz = 0, qb = 0;
    if (flags[((long long)z * G.ny + y) * G.ntx + (x >> 5)]) {
        const typename Store<S>::V4 v = fb[n];
        fbx = v.x;
        fby = v.y;
        fbz = v.z;
        qb = v.w;
    }
    if constexpr (LEAN) collide_lean<D, Store<S>::KF, Store<S>::KG>(s, sg, fbx, fby, fbz, qb, P);
    else collide_node<D, R, R>(s, sg, fbx, fby, fbz, qb, P);
    if (PARITY == 0) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) fn[O.st[i]] = IO::stf(s[i]);
#pragma unroll
        for (int k = 0; k < L::QG; k++) gn[O.st[k]] = IO::stg(sg[k]);
    } else if (inner_yz && !xedge) {
#pragma unroll
        for (int i = 0; i < L::Q; i++) fn[O.dst[i]] = IO::stf(s[i]);
#pragma unroll
        for (int k = 0; k < L::QG; k++) gn[O.dst[k]] = IO::stg(sg[k]);
    } else {
        odd_store_face<D, S, IX, LEAN>(G, P, fn, gn, x, y, z, O, s, sg);
    }
}

// Two 16-bit values of x-adjacent nodes in one 32-bit word (the lower x in
// the low half): the storage-unit values and the round-to-nearest packing of
// two of them, bit for bit what the one-node path loads and stores.
template <typename S> struct Pair16;
template <> struct Pair16<__nv_bfloat16> {
    static __device__ __forceinline__ float lo(uint32_t w) { return __uint_as_float(w << 16); }
    static __device__ __forceinline__ float hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&v);
    }
};
template <> struct Pair16<__half> {
    static __device__ __forceinline__ float lo(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu))); }
    static __device__ __forceinline__ float hi(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }
    static __device__ __forceinline__ uint32_t pack(float a, float b) {
        const __half2 v = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&v);
    }
};

// The even (own-slot) step of 16-bit storage with two x-adjacent nodes per
// thread: one 32-bit load and one 32-bit store per population and node pair
// instead of two 16-bit ones, and twice the bytes in flight per warp.  The
// even step has no face logic (every node reads and writes its own slots), so
// the pair needs none either.  Needs an even row length (then n and every
// plane offset i N are even: 4-byte aligned words).  Each node goes through
// collide_lean as in the one-node kernel, so the results are identical.  The
// first node's results wait as packed pairs of directions while the second
// node collides; byte permutes then form the (first, second) words.
// At most 72 registers for BF16 (24 bytes of spills; 98 unbounded): at 384^3,
// one node per thread 1.323 ms per lattice step (mean of both parities), node
// pairs 1.303 / 1.254 / 1.281 ms at 64 / 72 / 80 registers, 1.41 unbounded
// (128-thread blocks of 128 pairs).  FP16 at most 80 (no spills; at 72 it
// spilled 52 bytes): 1.245 ms against 1.301 at 72.
#ifndef PIBM_EVEN2_REGS
#define PIBM_EVEN2_REGS 72
#endif
#ifndef PIBM_EVEN2_REGS_F16
#define PIBM_EVEN2_REGS_F16 80
#endif
template <int D, typename S, typename IX>
__global__ void __maxnreg__((std::is_same<S, __half>::value ? PIBM_EVEN2_REGS_F16 : PIBM_EVEN2_REGS))
    k_stream_collide_even2(Geo G, S* __restrict__ f, S* __restrict__ g,
                                                             const float4* __restrict__ fb,
                                                             const uint8_t* __restrict__ flags,
                                                             CollideParams<float> P, AAOffsets<IX> O) {
    using L = Lat<D>;
    using W = Pair16<S>;
    constexpr int QP = (L::Q + 1) / 2, QGP = (L::QG + 1) / 2;
    const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    if (x >= G.nx || y >= G.ny) return;
    const long long n = node_index(G, x, y, z);
    S* const fn = f + n;
    S* const gn = g + n;
    uint32_t wf[L::Q], wg[L::QG];
#pragma unroll
    for (int i = 0; i < L::Q; i++) wf[i] = *reinterpret_cast<const uint32_t*>(fn + O.ld[i]);
#pragma unroll
    for (int k = 0; k < L::QG; k++) wg[k] = *reinterpret_cast<const uint32_t*>(gn + O.ld[k]);
    // x and x + 1 share a 32-node tile (x is even)
    const bool flagged = flags[((long long)z * G.ny + y) * G.ntx + (x >> 5)] != 0;
    float s[L::Q], sg[L::QG];
    uint32_t pf[QP], pg[QGP];
    {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (flagged) v = fb[n];
#pragma unroll
        for (int i = 0; i < L::Q; i++) s[i] = W::lo(wf[i]);
#pragma unroll
        for (int k = 0; k < L::QG; k++) sg[k] = W::lo(wg[k]);
        collide_lean<D, Store<S>::KF, Store<S>::KG>(s, sg, v.x, v.y, v.z, v.w, P);
#pragma unroll
        for (int j = 0; j < QP; j++) pf[j] = W::pack(s[2 * j], 2 * j + 1 < L::Q ? s[2 * j + 1] : 0.f);
#pragma unroll
        for (int j = 0; j < QGP; j++) pg[j] = W::pack(sg[2 * j], 2 * j + 1 < L::QG ? sg[2 * j + 1] : 0.f);
    }
    {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (flagged) v = fb[n + 1];
#pragma unroll
        for (int i = 0; i < L::Q; i++) s[i] = W::hi(wf[i]);
#pragma unroll
        for (int k = 0; k < L::QG; k++) sg[k] = W::hi(wg[k]);
        collide_lean<D, Store<S>::KF, Store<S>::KG>(s, sg, v.x, v.y, v.z, v.w, P);
    }
#pragma unroll
    for (int j = 0; j < QP; j++) {
        const uint32_t q = W::pack(s[2 * j], 2 * j + 1 < L::Q ? s[2 * j + 1] : 0.f);
        *reinterpret_cast<uint32_t*>(fn + O.st[2 * j]) = __byte_perm(pf[j], q, 0x5410);
        if (2 * j + 1 < L::Q) *reinterpret_cast<uint32_t*>(fn + O.st[2 * j + 1]) = __byte_perm(pf[j], q, 0x7632);
    }
#pragma unroll
    for (int j = 0; j < QGP; j++) {
        const uint32_t q = W::pack(sg[2 * j], 2 * j + 1 < L::QG ? sg[2 * j + 1] : 0.f);
        *reinterpret_cast<uint32_t*>(gn + O.st[2 * j]) = __byte_perm(pg[j], q, 0x5410);
        if (2 * j + 1 < L::QG) *reinterpret_cast<uint32_t*>(gn + O.st[2 * j + 1]) = __byte_perm(pg[j], q, 0x7632);
    }
}

// The node-pair form applies: 16-bit storage, an even step, an even row
// length, and the tuning knob on.
template <typename S>
static bool even_pairs(const Ctx* c, int parity) {
    return sizeof(S) == 2 && parity == 0 && c->G.nx % 2 == 0 && c->tune_lattice_pairs;
}

template <int D, typename S, int PARITY, typename IX>
static void sc_go(const Ctx* c, cudaStream_t s, dim3 grid, dim3 block, int parity,
                  const CollideParams<typename Store<S>::R>& P, const AAOffsets<IX>& O) {
    using V = typename Store<S>::V4;
    if constexpr (sizeof(S) == 2 && PARITY == 0) {
        if (even_pairs<S>(c, parity)) {
            // the same threads per block over the node pairs, in blocks that
            // span the widest multiple of 32 pairs dividing both the row's
            // pairs rounded up to 32 and the threads (no idle tail warps: at
            // 384^3, 64 x 2 blocks; 128 x 1 left a quarter of every second
            // block idle and measured 2 % slower over both parities)
            const int pairs = c->G.nx / 2, p32 = (pairs + 31) / 32 * 32;
            const int threads = (int)(block.x * block.y);
            const int cap = (int)block.x < p32 ? (int)block.x : p32;
            int bx = 32;
            for (int cand = 32; cand <= cap; cand += 32)
                if (p32 % cand == 0 && threads % cand == 0) bx = cand;
            const int by = threads / bx;
            const dim3 b2(bx, by, 1), g2((pairs + bx - 1) / bx, (c->G.ny + by - 1) / by, grid.z);
            k_stream_collide_even2<D, S, IX><<<g2, b2, 0, s>>>(c->G, (S*)c->f, (S*)c->g, (const V*)c->fb[parity],
                                                                c->flags[parity], P, O);
            return;
        }
    }
    k_stream_collide<D, S, PARITY, IX><<<grid, block, 0, s>>>(c->G, (S*)c->f, (S*)c->g, (const V*)c->fb[parity],
                                                              c->flags[parity], P, O);
}

template <typename R>
static CollideParams<R> collide_params(const Ctx* c) {
    CollideParams<R> P;
    const double cf = 1.0 - 0.5 / c->tau_f;
    P.om1f = (R)(1.0 - 1.0 / c->tau_f);
    P.om1g = (R)(1.0 - 1.0 / c->tau_g);
    P.c9f = (R)(9.0 * cf);
    P.c3f = (R)(3.0 * cf);
    P.m3f = (R)(-3.0 * cf);
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

template <int D, typename IX>
static AAOffsets<IX> aa_offsets(const Geo& G) {
    using L = Lat<D>;
    AAOffsets<IX> O;
    const long long sy = G.nx, sz = (long long)G.nx * G.ny;
    for (int i = 0; i < 19; i++) O.src[i] = O.dst[i] = O.ld[i] = O.st[i] = 0;
    for (int i = 0; i < L::Q; i++) {
        long long off = L::ex(i) + L::ey(i) * sy + L::ez(i) * sz;
        O.src[i] = (IX)((long long)L::opp(i) * G.N - off);
        O.dst[i] = (IX)((long long)i * G.N + off);
        O.ld[i] = (IX)((long long)i * G.N);
        O.st[i] = (IX)((long long)L::opp(i) * G.N);
    }
    return O;
}

// 32-bit offsets hold when every slot of f (the larger array) is within 2^31 - 1
// elements of plane 0's node, with room for the periodic x shift
template <int D>
static bool narrow_offsets(const Geo& G) {
    return (long long)Lat<D>::Q * G.N + 2LL * G.nx < (1LL << 31) - 1;
}

// Block shape of the lattice kernel: bx threads along x (a multiple of 32) times
// by rows.  Default: bx = min(the row rounded up to 32, 256) and 256 threads per
// block for rows of 256 or more nodes, 128 for shorter rows and for 16-bit
// storage (its 56-register bound fits nine 128-thread blocks per SM, four of
// 256; a block of 16-bit storage has at most 384 threads, larger requests are
// cut to 384).  With
// PIBM_TUNE_LATTICE_ROW_TILES = 1, bx is the largest multiple of 32 (at most
// 256) that divides the row rounded up to 32, so that no block straddles a
// row end with idle warps (a 384-node row: 192, not 256 + 128).  The tuning
// knob PIBM_TUNE_LATTICE_THREADS sets the threads per block (32 .. 512).
static void lattice_shape(const Ctx* c, dim3& block, dim3& grid) {
    const int w32 = (c->G.nx + 31) / 32 * 32;
    const bool st16 = c->desc.storage == PIBM_STORE_F16 || c->desc.storage == PIBM_STORE_BF16;
    int threads = c->tune_lattice_threads > 0 ? c->tune_lattice_threads : (w32 >= 256 && !st16 ? 256 : 128);
    if (st16 && threads > sc_max_threads<__half>()) threads = sc_max_threads<__half>();
    int bx = w32 < threads ? w32 : (threads < 256 ? threads : 256);
    if (c->tune_lattice_row_tiles) {
        int best = 32;
        for (int cand = 32; cand <= bx; cand += 32)
            if (w32 % cand == 0) best = cand;
        bx = best;
    }
    const int by = threads / bx > 0 ? threads / bx : 1;
    block = dim3(bx, by, 1);
    grid = dim3((c->G.nx + bx - 1) / bx, (c->G.ny + by - 1) / by, c->G.nz);
}

template <int D, typename S>
static cudaError_t sc_launch(Ctx* c, cudaStream_t s, int parity) {
    dim3 block, grid;
    lattice_shape(c, block, grid);
    using R = typename Store<S>::R;
    CollideParams<R> P = collide_params<R>(c);
    if (narrow_offsets<D>(c->G) && !c->tune_wide_index) {
        const AAOffsets<int> O = aa_offsets<D, int>(c->G);
        if (parity == 0) sc_go<D, S, 0, int>(c, s, grid, block, parity, P, O);
        else sc_go<D, S, 1, int>(c, s, grid, block, parity, P, O);
    } else {
        const AAOffsets<long long> O = aa_offsets<D, long long>(c->G);
        if (parity == 0) sc_go<D, S, 0, long long>(c, s, grid, block, parity, P, O);
        else sc_go<D, S, 1, long long>(c, s, grid, block, parity, P, O);
    }
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

// --------------------------------------------------- surrogate features
// Per-particle features of the learned coupling surrogate.  Region S_p = the
// nodes particle p owns in the coupling (epsilon > 0, the larger epsilon, ties
// to the lower index): the footprint pass accumulates the sums over S_p of
// d = r - X_p, d d^T, the raw fluid velocity u = j / rho (moments before the
// coupling's correction), d x u and T0 - T_ref; here the velocity is fitted by
// a rigid motion V + Om x d about X_p (least squares):
//   n V - D x Om = sum u,  D x V + M Om = sum d x u,
//   D = sum d, M = sum (|d|^2 I - d d^T)   (2-D: unknowns V_x, V_y, Om_z).
// Features: U_p - V (3), omega_p - Om (3), T_p - mean T0 over S_p (1) here;
// the solid fraction sum_{q != p, |X_q - X_p| < 4 R_p} (R_q / 4 R_p)^D (1) and
// the four smallest surface gaps |X_q - X_p| - R_p - R_q capped at 2 R_p (4)
// in k_neighbour_features.

// Gaussian elimination with partial pivoting on an m x m system (m <= 6).
__device__ void solve_small(double* A, double* b, int m) {
    for (int k = 0; k < m; k++) {
        int piv = k;
        for (int i = k + 1; i < m; i++)
            if (fabs(A[i * 6 + k]) > fabs(A[piv * 6 + k])) piv = i;
        if (piv != k) {
            for (int j = 0; j < m; j++) {
                double t = A[k * 6 + j];
                A[k * 6 + j] = A[piv * 6 + j];
                A[piv * 6 + j] = t;
            }
            double t = b[k];
            b[k] = b[piv];
            b[piv] = t;
        }
        const double inv = 1.0 / A[k * 6 + k];
        for (int i = k + 1; i < m; i++) {
            const double l = A[i * 6 + k] * inv;
            for (int j = k; j < m; j++) A[i * 6 + j] -= l * A[k * 6 + j];
            b[i] -= l * b[k];
        }
    }
    for (int k = m - 1; k >= 0; k--) {
        double s = b[k];
        for (int j = k + 1; j < m; j++) s -= A[k * 6 + j] * b[j];
        b[k] = s / A[k * 6 + k];
    }
}

// Features 0-6 from the sums the footprint pass accumulates over the
// particle's owned nodes with the coupling's weights (fsum[p]: sum w, sum w d
// (3), sum w d d^T (xx, yy, zz, xy, xz, yz), sum w u (3), sum w d x u (3) with
// w = eps rho, then sum eps dT and sum eps): the weighted rigid-motion fit
//   m V - D x Om = sum w u,  D x V + M Om = sum w d x u
// (m = sum w, D = sum w d, M = sum w (|d|^2 I - d d^T)) and the eps-weighted
// mean temperature; one thread per particle.
template <int D>
__global__ void k_feature_solve(int n, const double* __restrict__ fsum, const double* __restrict__ U,
                                const double* __restrict__ W, const double* __restrict__ Tp, double Tref,
                                double* __restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double s[SG_NFSUM];
    for (int k = 0; k < SG_NFSUM; k++) s[k] = fsum[SG_NFSUM * (long long)p + k];
    double V[3] = {0, 0, 0}, Om[3] = {0, 0, 0};
    const double m = s[0];
    if (m > 0) {
        double A[36], b[6];
        if (Lat<D>::dim == 3) {
            const double Dd[3] = {s[1], s[2], s[3]};
            const double trace = s[4] + s[5] + s[6];
            const double M[9] = {trace - s[4], -s[7], -s[8], -s[7], trace - s[5], -s[9], -s[8], -s[9], trace - s[6]};
            const double Dx[9] = {0, -Dd[2], Dd[1], Dd[2], 0, -Dd[0], -Dd[1], Dd[0], 0};  // D x (cross-product matrix)
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) {
                    A[i * 6 + j] = i == j ? m : 0.0;
                    A[i * 6 + 3 + j] = -Dx[i * 3 + j];
                    A[(3 + i) * 6 + j] = Dx[i * 3 + j];
                    A[(3 + i) * 6 + 3 + j] = M[i * 3 + j];
                }
            b[0] = s[10], b[1] = s[11], b[2] = s[12], b[3] = s[13], b[4] = s[14], b[5] = s[15];
            solve_small(A, b, 6);
            V[0] = b[0], V[1] = b[1], V[2] = b[2], Om[0] = b[3], Om[1] = b[4], Om[2] = b[5];
        } else {
            A[0] = m, A[1] = 0.0, A[2] = -s[2];
            A[6] = 0.0, A[7] = m, A[8] = s[1];
            A[12] = -s[2], A[13] = s[1], A[14] = s[4] + s[5];
            b[0] = s[10], b[1] = s[11], b[2] = s[15];
            solve_small(A, b, 3);
            V[0] = b[0], V[1] = b[1], Om[2] = b[2];
        }
    }
    double* o = out + 12 * (long long)p;
    for (int a = 0; a < 3; a++) {
        o[a] = U[3 * p + a] - V[a];
        o[3 + a] = W[3 * p + a] - Om[a];
    }
    o[6] = Tp[p] - (s[17] > 0 ? Tref + s[16] / s[17] : 0.0);
}

// Neighbour features (solid fraction and the four smallest gaps), n-body
// style: one thread per particle, the other particles staged through shared
// memory in tiles of NB_T as FP32 (x, y, z, R).  The FP32 prefilter keeps the
// exact FP64 distance to the particles that can matter: centres closer than
// max(4 R_p, 3 R_p + R_q) (a larger gap is capped at 2 R_p anyway).
constexpr int NB_T = 128;
template <int D>
__global__ void __launch_bounds__(NB_T) k_neighbour_features(int n, int slice_len, const double* __restrict__ X,
                                                             const double* __restrict__ R, const float4* __restrict__ xr,
                                                             double* __restrict__ part) {
    // blockIdx.y: slice of the other particles [q0, q1); part[slice][p][5]: phi, four gaps
    __shared__ float4 tile[NB_T];
    const int p = blockIdx.x * NB_T + threadIdx.x;
    const bool live = p < n;
    const int q0 = blockIdx.y * slice_len, q1 = min(n, q0 + slice_len);
    const float4 me = live ? xr[p] : make_float4(0.f, 0.f, 0.f, 0.f);
    double xp = 0.0, yp = 0.0, zp = 0.0, Rp = 1.0;
    if (live) xp = X[3 * p], yp = X[3 * p + 1], zp = X[3 * p + 2], Rp = R[p];
    double phi = 0.0;
    double gd4[4] = {1e300, 1e300, 1e300, 1e300};
    for (int t0 = q0; t0 < q1; t0 += NB_T) {
        __syncthreads();
        if (t0 + threadIdx.x < q1) tile[threadIdx.x] = xr[t0 + threadIdx.x];
        __syncthreads();
        const int m = q1 - t0 < NB_T ? q1 - t0 : NB_T;
        if (!live) continue;
        for (int j = 0; j < m; j++) {
            const int q = t0 + j;
            if (q == p) continue;
            const float4 o = tile[j];
            const float fx = o.x - me.x, fy = o.y - me.y, fz = o.z - me.z;
            const float lim = fmaxf(4.f * me.w, 3.f * me.w + o.w) + 0.01f;
            if (fx * fx + fy * fy + fz * fz >= lim * lim) continue;
            const double ex = X[3 * q] - xp, ey = X[3 * q + 1] - yp, ez = X[3 * q + 2] - zp;
            const double dist = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)));
            const double Rq = R[q];
            if (dist < 4.0 * Rp) {
                const double sr = Rq / (4.0 * Rp);
                phi += Lat<D>::dim == 3 ? sr * sr * sr : sr * sr;
            }
            double gap = (dist - Rp) - Rq;
            for (int k = 0; k < 4; k++)  // insert into the sorted four
                if (gap < gd4[k]) {
                    const double tt = gd4[k];
                    gd4[k] = gap;
                    gap = tt;
                }
        }
    }
    if (!live) return;
    double* o = part + ((long long)blockIdx.y * n + p) * 5;
    o[0] = phi;
    for (int k = 0; k < 4; k++) o[1 + k] = gd4[k];
}

// slices combined in slice order (deterministic): phi summed, the four smallest gaps merged
__global__ void k_neighbour_merge(int n, int nslice, const double* __restrict__ R, const double* __restrict__ part,
                                  double* __restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double phi = 0.0, best[4] = {1e300, 1e300, 1e300, 1e300};
    for (int s = 0; s < nslice; s++) {
        const double* o = part + ((long long)s * n + p) * 5;
        phi += o[0];
        for (int j = 1; j < 5; j++) {
            double gap = o[j];
            for (int k = 0; k < 4; k++)
                if (gap < best[k]) {
                    const double tt = best[k];
                    best[k] = gap;
                    gap = tt;
                }
        }
    }
    double* out_p = out + 12 * (long long)p;
    out_p[7] = phi;
    const double cap = 2.0 * R[p];
    for (int k = 0; k < 4; k++) out_p[8 + k] = best[k] < cap ? best[k] : cap;
}

// Features 7-11 from the DEM's cell list instead of all pairs: one warp per
// particle scans the cells that can hold a particle within the feature range
// max(4 R_p, 3 R_p + R_max) of it, widened by half the neighbour skin (the list
// was built where the particles stood at the last rebuild, and none has moved
// more than that since).  The cells of an x-row are consecutive in the sorted
// list, so each lane takes whole rows (one id range each); the pair test is the
// all-pairs kernel's (FP32 prefilter, exact FP64 distance), so the same
// neighbours are found.  phi is summed per lane, then over the lanes in a fixed
// butterfly (last-bit differences from index order); the four smallest gaps are
// merged across the lanes exactly.
template <int D>
__global__ void k_neighbour_cells(int n, const double* __restrict__ X, const double* __restrict__ R,
                                  const float4* __restrict__ xr, const int* __restrict__ cell_start,
                                  const int* __restrict__ cell_ids, DemCfg C, double rmax, double* __restrict__ out) {
    const int p = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (p >= n) return;  // whole warps: p is uniform across the warp
    const float4 me = xr[p];
    const double xp = X[3 * p], yp = X[3 * p + 1], zp = X[3 * p + 2], Rp = R[p];
    const double Lr = fmax(4.0 * Rp, 3.0 * Rp + rmax) + 0.01 + 0.5 * C.skin + 1e-6;
    const double Xp[3] = {xp, yp, zp};
    int clo[3], chi[3];
    for (int a = 0; a < 3; a++) {
        if (a < Lat<D>::dim) {
            clo[a] = (int)floor((Xp[a] - Lr + 0.5) * C.inv[a]);
            chi[a] = (int)floor((Xp[a] + Lr + 0.5) * C.inv[a]);
            clo[a] = clo[a] < 0 ? 0 : clo[a];
            chi[a] = chi[a] > C.nc[a] - 1 ? C.nc[a] - 1 : chi[a];
        } else {
            clo[a] = chi[a] = 0;
        }
    }
    const int ny_rows = chi[1] - clo[1] + 1, nrows = (chi[2] - clo[2] + 1) * ny_rows;
    double phi = 0.0;
    double gd4[4] = {1e300, 1e300, 1e300, 1e300};
    for (int r = lane; r < nrows; r += 32) {
        const int cz = clo[2] + r / ny_rows, cy = clo[1] + r % ny_rows;
        const int row = (cz * C.nc[1] + cy) * C.nc[0];
        const int b = cell_start[row + clo[0]], e = cell_start[row + chi[0] + 1];
        for (int k = b; k < e; k++) {
            const int q = cell_ids[k];
            if (q == p) continue;
            const float4 o = xr[q];
            const float fx = o.x - me.x, fy = o.y - me.y, fz = o.z - me.z;
            const float lim = fmaxf(4.f * me.w, 3.f * me.w + o.w) + 0.01f;
            if (fx * fx + fy * fy + fz * fz >= lim * lim) continue;
            const double ex = X[3 * q] - xp, ey = X[3 * q + 1] - yp, ez = X[3 * q + 2] - zp;
            const double dist = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez)));
            const double Rq = R[q];
            if (dist < 4.0 * Rp) {
                const double sr = Rq / (4.0 * Rp);
                phi += Lat<D>::dim == 3 ? sr * sr * sr : sr * sr;
            }
            double gap = (dist - Rp) - Rq;
            for (int j = 0; j < 4; j++)  // insert into the sorted four
                if (gap < gd4[j]) {
                    const double tt = gd4[j];
                    gd4[j] = gap;
                    gap = tt;
                }
        }
    }
    // across the warp: phi by a butterfly sum, the four smallest gaps by merging
    // the two sorted fours of each pair of lanes (every lane ends with the result)
    for (int o = 16; o > 0; o >>= 1) {
        phi += __shfl_xor_sync(0xffffffffu, phi, o);
        double other[4];
        for (int j = 0; j < 4; j++) other[j] = __shfl_xor_sync(0xffffffffu, gd4[j], o);
        double merged[4];
        int ia = 0, ib = 0;
        for (int j = 0; j < 4; j++) {
            if (gd4[ia] <= other[ib]) merged[j] = gd4[ia++];
            else merged[j] = other[ib++];
        }
        for (int j = 0; j < 4; j++) gd4[j] = merged[j];
    }
    if (lane == 0) {
        double* out_p = out + 12 * (long long)p;
        out_p[7] = phi;
        const double cap = 2.0 * Rp;
        for (int k = 0; k < 4; k++) out_p[8 + k] = gd4[k] < cap ? gd4[k] : cap;
    }
}

__global__ void k_pos_f32(int n, const double* X, const double* R, float4* xr) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) xr[p] = make_float4((float)X[3 * p], (float)X[3 * p + 1], (float)X[3 * p + 2], (float)R[p]);
}

template <int D, typename S>
static cudaError_t features_launch(Ctx* c, cudaStream_t s, int parity, double* out) {
    if (c->np == 0) return cudaSuccess;
    k_pos_f32<<<(c->np + 255) / 256, 256, 0, s>>>(c->np, c->X, c->R, c->sg.xr);
    k_feature_solve<D><<<(c->np + 127) / 128, 128, 0, s>>>(c->np, c->sg.fsum, c->U, c->W, c->Tp, c->desc.T_ref, out);
    // through the DEM's cell list when the scan stays within a few cells per axis
    {
        const double L = 4.0 * c->rmax + 0.01 + 0.5 * c->dem.skin;
        bool cells = c->dem.ncell > 1;
        for (int a = 0; a < Lat<D>::dim; a++) cells = cells && L * c->dem.inv[a] < 3.5;
        if (cells) {
            k_neighbour_cells<D><<<(int)(((long long)c->np * 32 + 127) / 128), 128, 0, s>>>(c->np, c->X, c->R, c->sg.xr, c->cell_start,
                                                                     c->cell_ids, c->dem, c->rmax, out);
            return cudaGetLastError();
        }
    }
    // otherwise all pairs: the other particles in slices of at least 1024, so that large sets fill the GPU
    const int nslice = std::min(SG_NB_SLICES, std::max(1, (c->np + 1023) / 1024));
    const int slice_len = (c->np + nslice - 1) / nslice;
    k_neighbour_features<D><<<dim3((c->np + NB_T - 1) / NB_T, nslice), NB_T, 0, s>>>(c->np, slice_len, c->X, c->R,
                                                                                    c->sg.xr, c->sg.nbpart);
    k_neighbour_merge<<<(c->np + 127) / 128, 128, 0, s>>>(c->np, nslice, c->R, c->sg.nbpart, out);
    return cudaGetLastError();
}

cudaError_t launch_features(Ctx* c, cudaStream_t s, int parity, double* out) {
    PIBM_DISPATCH(c, features_launch, c, s, parity, out);
}

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

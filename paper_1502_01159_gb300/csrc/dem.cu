// DEM kernels (Section 2.3, Eq demgov; Hertz normal law and
// Mindlin-Deresiewicz loading stiffness, or a linear spring-dashpot law).
//
// One launch per lattice step runs as one thread-block cluster (up to 16 CTAs
// on 16 SMs).  Particle p belongs to CTA p / per.  Each CTA publishes the
// positions (FP64) and velocities (FP32) of its particles in shared memory,
// double-buffered by substep; every thread reads the published state of its
// particles' neighbours directly from the owning CTA's shared memory
// (distributed shared memory), so one hardware cluster barrier per substep
// is the only synchronisation:
//   substep: for each own particle, contact forces with every neighbour of
//   the neighbour list -- each pair is evaluated in its canonical order
//   (lower index first) by both partners with bit-identical inputs, so the two
//   contributions are exactly opposite and no atomics are needed; the lower
//   index writes the pair's tangential history into the other half of a
//   double buffer -- plus wall contacts, then the velocity Verlet kicks and
//   drift in FP64 and the publication of the new state.
// After the substeps: the thermosensitive update C_p dT_p = -H_p, and -- only
// when a particle has moved more than (skin - 1)/2 since the last build -- the
// rebuild: FP64 cell ids (no contraction, the oracle's operation order),
// counting sort stable by index, neighbour pairs within R_i + R_j + skin
// sorted by (i, j), histories carried over by binary search.  A move larger
// than half the skin within one lattice step raises a status word (contacts
// could be missed).
#include <cooperative_groups.h>

#include "pibm_internal.cuh"

namespace cg = cooperative_groups;

namespace pibm {

constexpr int DEM_T = 256;
constexpr int DEM_MAXNB = 64;

struct DemState {
    double *X, *U, *W, *Xb, *R, *m, *I, *im, *iI, *mg, *Tp, *Cp, *Fh, *Th, *Hh;
    float *Fc, *Tc;  // contact force and torque of the last evaluation (FP32, as the substeps form them)
    double *Fhp, *Thp, *Hhp;
    int* have_prev;
    int* adj_new;
    const uint8_t* fixed;
    int *cell_of, *cell_cnt, *cell_start, *cell_ids, *cnt_hi, *cnt_lo;
    int *nb_start0, *nb_start1, *nb_i0, *nb_i1, *nb_j0, *nb_j1;
    float4 *nb_ft0, *nb_ft1;  // per list: two substep buffers of cap entries (history xyz, substep stamp)
    double *nb_md0, *nb_md1;  // per list: two substep buffers of cap FP64 records (MD_REC doubles) of the
                              // Mindlin-Deresiewicz history of law PIBM_HERTZ_MD_HIST
    int* nb_cur;              // [0] current list, [1] global substep counter
    int *adj_start, *adj_nb, *adj_k;
    float* wall_ft;
    double* wall_md;  // [n][6][MD_REC]: the Mindlin-Deresiewicz history of the wall contacts
    int* dstat;
    int* flag;  // cluster-wide overflow flag
    int adj_cap;
};

// state a CTA publishes for each of its particles: FP64 position (exact
// contact test), FP32 copy of it (prefilter), FP32 velocities (force law)
struct Pub {
    double x[3];
    float u[3], w[3];
    float xf[3], rf;  // FP32 position and radius: one 16-byte load for the prefilter
};

__device__ __forceinline__ void set_error(int* dstat, int detail) {
    if (atomicCAS(dstat, 0, (int)PIBM_ERR_STATE) == 0) dstat[1] = detail;
}

// exclusive scan of in[0..M) into out[0..M] (out[M] = total) by one CTA
__device__ void cta_scan(const int* in, int* out, int M, int* sh) {
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

// FP64 squared distance with the oracle's operation order (no contraction)
__device__ __forceinline__ double dist2(const double* Xi, const double* Xj) {
    double dx = __dsub_rn(Xj[0], Xi[0]), dy = __dsub_rn(Xj[1], Xi[1]), dz = __dsub_rn(Xj[2], Xi[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__device__ __forceinline__ void ldX(const double* X, int p, double* o) {
    o[0] = __ldcg(X + 3 * p);
    o[1] = __ldcg(X + 3 * p + 1);
    o[2] = __ldcg(X + 3 * p + 2);
}

__device__ __forceinline__ float3 f3(float a, float b, float c) { return make_float3(a, b, c); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Contact law in FP32: returns F_n and the tangential stiffness.
__device__ __forceinline__ float normal_law(const DemCfg& C, float delta, float vn, float Rstar, float* kt_eff) {
    if (C.law != PIBM_SPRING_DASHPOT) {  // Hertz (with or without the Mindlin-Deresiewicz history)
        *kt_eff = 8.0f * C.G_star * sqrtf(delta * Rstar);
        return (4.0f / 3.0f) * C.E_star * sqrtf(Rstar) * delta * sqrtf(delta) + C.gn * vn;
    }
    *kt_eff = C.kt;
    return C.kn * delta + C.gn * vn;
}

// Tangential force: history projected on the tangent plane, incremented by
// -k_t v_t dt, capped at mu |F_n|; returns the total with tangential damping.
__device__ __forceinline__ float3 tangential(const DemCfg& C, float3& h, float3 n, float3 vt, float kt_eff, float Fn, float dt) {
    float hn = h.x * n.x + h.y * n.y + h.z * n.z;
    h = f3(h.x - hn * n.x - kt_eff * vt.x * dt, h.y - hn * n.y - kt_eff * vt.y * dt, h.z - hn * n.z - kt_eff * vt.z * dt);
    float mag = sqrtf(h.x * h.x + h.y * h.y + h.z * h.z);
    float cap = C.mu * fabsf(Fn);
    if (mag > cap) {
        float sc = mag > 0.f ? cap / mag : 0.f;
        h = f3(h.x * sc, h.y * sc, h.z * sc);
    }
    return f3(h.x - C.gt * vt.x, h.y - C.gt * vt.y, h.z - C.gt * vt.z);
}

// Tangential force with the Mindlin-Deresiewicz loading history (law
// PIBM_HERTZ_MD_HIST): increment 8 G* r_a theta_k dd_t + (-1)^k mu dF_n
// (1 - theta_k) with theta_k of Thornton and Yin for loading (k = 0),
// unloading (1) and reloading (2) along the contact's reference direction e
// (set at its first tangential displacement, kept in the tangent plane):
//   theta_0^3 = 1 - (T + mu dF_n)/(mu F_n), theta_1^3 = 1 - (T* - T + 2 mu dF_n)/(2 mu F_n),
//   theta_2^3 = 1 - (T - T** + 2 mu dF_n)/(2 mu F_n),
// T the force along e; the branch turns when the displacement along e
// reverses (reloading rejoins loading at T*); no history increment on a
// contact's first update; Coulomb cap on the total.  kt8a = 8 G* r_a.
//
// Evaluated in FP64 on an FP64 record: theta_k is the cube root of a
// difference that vanishes at full slip, so a relative error eps in T or
// mu F_n moves theta by about eps^(1/3) there (FP32: 4e-3 of the stiffness
// 8 G* r_a; FP64: 5e-6).  The inputs n, v_t, F_n and kt8a stay the kernel's
// FP32 values.
struct MdRec {
    double h[3], e[3], fnp, ts, tss, k;  // the MD_REC doubles of one contact
};

__device__ __forceinline__ void md_load(const double* p, MdRec& r) {
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 a = __ldcg(q), b = __ldcg(q + 1), c = __ldcg(q + 2), d = __ldcg(q + 3), e = __ldcg(q + 4);
    r.h[0] = a.x, r.h[1] = a.y, r.h[2] = b.x, r.e[0] = b.y, r.e[1] = c.x, r.e[2] = c.y;
    r.fnp = d.x, r.ts = d.y, r.tss = e.x, r.k = e.y;
}

__device__ __forceinline__ void md_store(double* p, const MdRec& r) {
    double2* q = reinterpret_cast<double2*>(p);
    q[0] = make_double2(r.h[0], r.h[1]), q[1] = make_double2(r.h[2], r.e[0]), q[2] = make_double2(r.e[1], r.e[2]);
    q[3] = make_double2(r.fnp, r.ts), q[4] = make_double2(r.tss, r.k);
}

__device__ __forceinline__ void md_zero(MdRec& r) {
    r.h[0] = r.h[1] = r.h[2] = r.e[0] = r.e[1] = r.e[2] = 0.0;
    r.fnp = r.ts = r.tss = r.k = 0.0;
}

__device__ __forceinline__ float3 tangential_md(const DemCfg& C, MdRec& r, float3 nf, float3 vtf, float kt8af, float Fnf,
                                                float dtf) {
    const double n[3] = {nf.x, nf.y, nf.z}, vt[3] = {vtf.x, vtf.y, vtf.z};
    const double kt8a = kt8af, dt = dtf;
    const double hn = r.h[0] * n[0] + r.h[1] * n[1] + r.h[2] * n[2];
    const double en = r.e[0] * n[0] + r.e[1] * n[1] + r.e[2] * n[2];
    for (int a = 0; a < 3; a++) {
        r.h[a] -= hn * n[a];
        r.e[a] -= en * n[a];
    }
    const double el = sqrt(r.e[0] * r.e[0] + r.e[1] * r.e[1] + r.e[2] * r.e[2]);
    const double ds[3] = {vt[0] * dt, vt[1] * dt, vt[2] * dt};
    const double dsl = sqrt(ds[0] * ds[0] + ds[1] * ds[1] + ds[2] * ds[2]);
    if (el > 0.0) {
        for (int a = 0; a < 3; a++) r.e[a] /= el;
    } else if (dsl > 0.0) {
        for (int a = 0; a < 3; a++) r.e[a] = -ds[a] / dsl;
    }
    const double mu = C.mu_d, N = fabs((double)Fnf);
    const double dFn = r.fnp > 0.0 ? N - r.fnp : 0.0;
    const double T = r.h[0] * r.e[0] + r.h[1] * r.e[1] + r.h[2] * r.e[2];
    const double sgn = -(ds[0] * r.e[0] + ds[1] * r.e[1] + ds[2] * r.e[2]);  // > 0: T increases
    int k = (int)r.k;
    if (k == 0 && sgn < 0.0) {
        k = 1;
        r.ts = T;
    } else if (k == 1 && sgn > 0.0) {
        k = 2;
        r.tss = T;
    } else if (k == 2) {
        if (sgn < 0.0) {
            k = 1;
            r.ts = T;
        } else if (T >= r.ts) {
            k = 0;
        }
    }
    double th3 = 0.0;
    if (mu * N > 0.0) {
        if (k == 0) th3 = 1.0 - (T + mu * dFn) / (mu * N);
        else if (k == 1) th3 = 1.0 - (r.ts - T + 2.0 * mu * dFn) / (2.0 * mu * N);
        else th3 = 1.0 - (T - r.tss + 2.0 * mu * dFn) / (2.0 * mu * N);
    }
    th3 = fmin(fmax(th3, 0.0), 1.0);
    const double th = cbrt(th3);
    const double sk = k == 1 ? -1.0 : 1.0;
    const double kd = kt8a * th, kn = sk * mu * dFn * (1.0 - th);
    for (int a = 0; a < 3; a++) r.h[a] += -kd * ds[a] + kn * r.e[a];
    const double mag = sqrt(r.h[0] * r.h[0] + r.h[1] * r.h[1] + r.h[2] * r.h[2]);
    const double cap = mu * N;
    if (mag > cap) {
        const double sc = mag > 0.0 ? cap / mag : 0.0;
        for (int a = 0; a < 3; a++) r.h[a] *= sc;
    }
    r.fnp = N;
    r.k = k;
    const double gt = C.gt;
    return f3((float)(r.h[0] - gt * vt[0]), (float)(r.h[1] - gt * vt[1]), (float)(r.h[2] - gt * vt[2]));
}

// Pair (a < b) in canonical order, in contact (d2 < SS): force on a, torques
// on a and b, new history.  d = X_b - X_a and d2 = |d|^2, SS = (R_a + R_b)^2
// come from the caller's exact FP64 contact test; the only FP64 operation left
// is the overlap S^2 - d^2, which cancels.  Both partners call this with the
// same inputs and get the same bits.
template <bool MDH>
__device__ __forceinline__ void pair_force(const DemCfg& C, const Pub& A, const Pub& B, const double* d, double d2,
                                           double SS, float Raf, float Rbf, float3& h, MdRec& md, float dtf,
                                           float3& Fa, float3& Ta, float3& Tb) {
    float distf = sqrtf((float)d2);
    const float Sf = Raf + Rbf;
    float delta = (float)(SS - d2) / (Sf + distf);
    float3 nn = f3((float)d[0] / distf, (float)d[1] / distf, (float)d[2] / distf);
    float ai = Raf - 0.5f * delta, aj = Rbf - 0.5f * delta;
    float3 wi = cross3(f3(A.w[0], A.w[1], A.w[2]), f3(ai * nn.x, ai * nn.y, ai * nn.z));
    float3 wj = cross3(f3(B.w[0], B.w[1], B.w[2]), f3(-aj * nn.x, -aj * nn.y, -aj * nn.z));
    float3 vr = f3(A.u[0] + wi.x - B.u[0] - wj.x, A.u[1] + wi.y - B.u[1] - wj.y, A.u[2] + wi.z - B.u[2] - wj.z);
    float vn = vr.x * nn.x + vr.y * nn.y + vr.z * nn.z;
    float3 vt = f3(vr.x - vn * nn.x, vr.y - vn * nn.y, vr.z - vn * nn.z);
    float Rstar = Raf * Rbf / Sf, kt_eff;
    float Fn = normal_law(C, delta, vn, Rstar, &kt_eff);
    float3 Ft;
    if constexpr (MDH) {
        Ft = tangential_md(C, md, nn, vt, kt_eff, Fn, dtf);
        h = f3((float)md.h[0], (float)md.h[1], (float)md.h[2]);
    } else {
        Ft = tangential(C, h, nn, vt, kt_eff, Fn, dtf);
    }
    Ta = cross3(f3(ai * nn.x, ai * nn.y, ai * nn.z), Ft);
    Tb = cross3(f3(aj * nn.x, aj * nn.y, aj * nn.z), Ft);
    Fa = f3(-Fn * nn.x + Ft.x, -Fn * nn.y + Ft.y, -Fn * nn.z + Ft.z);
}

// Hydrodynamic load over one lattice step: the mean of the couplings of time
// t and t-1 (the half-force fluid momentum advances by the mean of consecutive
// forcing terms; this also cancels the step-to-step sign flip of the
// bounce-back impulse on covered nodes).
__device__ __forceinline__ double hydro(const double* cur, const double* prev, int k, int hp) {
    return hp ? 0.5 * (cur[k] + prev[k]) : cur[k];
}

template <int D>
__device__ void cell_coords(const DemCfg& C, const double* Xp, int* c) {
    for (int a = 0; a < 3; a++) {
        int v = 0;
        if (a < D) {
            v = (int)floor(__dmul_rn(__dadd_rn(Xp[a], 0.5), C.inv[a]));
            if (v < 0) v = 0;
            if (v > C.nc[a] - 1) v = C.nc[a] - 1;
        }
        c[a] = v;
    }
}

// visit the particles of the 3^D cells around cell c
template <int D, typename F>
__device__ __forceinline__ void for_neighbours(const DemCfg& C, const DemState& S, const int* c, F&& fn) {
    for (int z = c[2] - 1; z <= c[2] + 1; z++) {
        if (z < 0 || z >= C.nc[2]) continue;
        for (int y = c[1] - 1; y <= c[1] + 1; y++) {
            if (y < 0 || y >= C.nc[1]) continue;
            for (int x = c[0] - 1; x <= c[0] + 1; x++) {
                if (x < 0 || x >= C.nc[0]) continue;
                int cell = (z * C.nc[1] + y) * C.nc[0] + x;
                int b = __ldcg(S.cell_start + cell), e = __ldcg(S.cell_start + cell + 1);
                for (int k = b; k < e; k++) fn(__ldcg(S.cell_ids + k));
            }
        }
    }
}

// wall contacts of particle p (same law, R_wall = infinity, wall at rest).
// mask: bit f set while face f holds a non-zero tangential history, so faces
// out of contact cost no memory traffic; hpre (or null): those histories,
// loaded ahead by the caller.
template <int D, bool MDH>
__device__ __forceinline__ void wall_forces(const DemCfg& C, const DemState& S, int p, const Pub& me, double Rp, float Rpf,
                                            float dtf, float* F, float* T, int& mask, const float* hpre) {
    for (int face = 0; face < 2 * D; face++) {
        int a = face >> 1, hi = face & 1;
        if (!C.walled[a]) continue;
        float* ftp = S.wall_ft + 3 * (6 * p + face);
        double* mdp = S.wall_md + MD_REC * (6 * p + face);
        // FP32 prefilter on the distance to the wall plane, exact FP64 test when close
        const float distf = hi ? C.hif[a] - me.xf[a] : me.xf[a] - C.lof[a];
        double dd = -1.0;
        if (distf < Rpf + 1e-3f) dd = Rp - (hi ? C.hi[a] - me.x[a] : me.x[a] - C.lo[a]);
        if (!(dd > 0.0)) {
            if (mask & (1 << face)) {
                ftp[0] = ftp[1] = ftp[2] = 0.f;
                if constexpr (MDH)
                    for (int q = 0; q < MD_REC; q++) mdp[q] = 0.0;
                mask &= ~(1 << face);
            }
            continue;
        }
        float delta = (float)dd;
        float3 nn = f3(0, 0, 0);
        if (a == 0) nn.x = hi ? 1.f : -1.f;
        else if (a == 1) nn.y = hi ? 1.f : -1.f;
        else nn.z = hi ? 1.f : -1.f;
        float ai = Rpf - 0.5f * delta;
        float3 ri = f3(ai * nn.x, ai * nn.y, ai * nn.z);
        float3 wi = cross3(f3(me.w[0], me.w[1], me.w[2]), ri);
        float3 vr = f3(me.u[0] + wi.x, me.u[1] + wi.y, me.u[2] + wi.z);
        float vn = vr.x * nn.x + vr.y * nn.y + vr.z * nn.z;
        float3 vt = f3(vr.x - vn * nn.x, vr.y - vn * nn.y, vr.z - vn * nn.z);
        float kt_eff;
        float Fn = normal_law(C, delta, vn, Rpf, &kt_eff);
        float3 h = f3(0.f, 0.f, 0.f);
        if (mask & (1 << face))
            h = hpre ? f3(hpre[3 * face], hpre[3 * face + 1], hpre[3 * face + 2]) : f3(__ldcg(ftp), __ldcg(ftp + 1), __ldcg(ftp + 2));
        float3 Ft;
        if constexpr (MDH) {
            MdRec md;
            if (mask & (1 << face)) md_load(mdp, md);
            else md_zero(md);
            Ft = tangential_md(C, md, nn, vt, kt_eff, Fn, dtf);
            md_store(mdp, md);
            h = f3((float)md.h[0], (float)md.h[1], (float)md.h[2]);
        } else {
            Ft = tangential(C, h, nn, vt, kt_eff, Fn, dtf);
        }
        ftp[0] = h.x, ftp[1] = h.y, ftp[2] = h.z;
        mask |= 1 << face;
        float3 Ti = cross3(ri, Ft);
        F[0] += -Fn * nn.x + Ft.x, F[1] += -Fn * nn.y + Ft.y, F[2] += -Fn * nn.z + Ft.z;
        T[0] += Ti.x, T[1] += Ti.y, T[2] += Ti.z;
    }
}

// private state of a particle while its CTA runs the substeps (shared memory)
struct Priv {
    double X[3], U[3], W[3];
    float a[3], al[3];       // external linear / angular acceleration: (hydro + buoyant weight)/m, hydro torque/I
    double im, iI, R;        // 1/m, 1/I, radius
    float Rf, imf;           // radius and 1/m in FP32
    float Fc[3], Tc[3];      // contact force / torque of the last evaluation
    int fixed, wall_mask;    // wall_mask: faces with a non-zero tangential history
    int nadj;                // neighbours in the adjacency
    float iIf;               // 1/I in FP32
};

// Velocity Verlet half or full kick.  J (optional, per particle: J_FU then
// J_TW, row-major) is a learned estimate of d(hydrodynamic force)/dU and
// d(hydrodynamic torque)/domega; the held hydrodynamic load is then corrected
// by J_FU (U - U0) and J_TW (omega - omega0), with U0, omega0 the velocities
// at the start of the lattice step.
//
// FP64 on this GPU issues at a small fraction of the FP32 rate, and every
// warp-wide FP64 instruction holds its scheduler for many cycles, so the
// substep does FP64 work only where the result needs it: the velocity and
// position sums.  The increment h (F_c/m + a_ext) is formed in FP32 (relative
// error ~1e-7 of a per-substep change) and added to the FP64 velocity in one
// operation.  In 2-D only U_x, U_y and omega_z can change: U_z, omega_x and
// omega_y are zero from the load on, and their FP64 operations are skipped.
template <int D>
__device__ __forceinline__ void kick_s(Priv& P, double h, float hf, const float* J, const double* U0, const double* W0) {
    constexpr int NU = D == 3 ? 3 : 2;  // velocity components that can change
    constexpr int W_LO = D == 3 ? 0 : 2;  // first spin component that can change
    // held hydrodynamic load corrected by J_FU (U - U0), J_TW (omega - omega0),
    // with the velocities before this kick
    double dF[3] = {0.0, 0.0, 0.0}, dT[3] = {0.0, 0.0, 0.0};
    if (J) {
        double du[3], dw[3];
        for (int b = 0; b < 3; b++) du[b] = P.U[b] - U0[b], dw[b] = P.W[b] - W0[b];
        for (int a = 0; a < NU; a++)
            for (int b = 0; b < NU; b++) dF[a] += (double)J[3 * a + b] * du[b];
        for (int a = W_LO; a < 3; a++)
            for (int b = W_LO; b < 3; b++) dT[a] += (double)J[9 + 3 * a + b] * dw[b];
    }
    for (int a = 0; a < NU; a++) P.U[a] += (double)(hf * (P.Fc[a] * P.imf + P.a[a]));
    for (int a = W_LO; a < 3; a++) P.W[a] += (double)(hf * (P.Tc[a] * P.iIf + P.al[a]));
    if (J) {
        for (int a = 0; a < NU; a++) P.U[a] += h * dF[a] * P.im;
        for (int a = W_LO; a < 3; a++) P.W[a] += h * dT[a] * P.iI;
    }
}

// drift and publication of the fields that change (the others were published
// into both buffers at the load)
template <int D>
__device__ __forceinline__ void drift_s(Priv& P, double dt, Pub& pub) {
    constexpr int NU = D == 3 ? 3 : 2;
    constexpr int W_LO = D == 3 ? 0 : 2;
    for (int a = 0; a < NU; a++) {
        P.X[a] += dt * P.U[a];
        pub.x[a] = P.X[a];
        pub.xf[a] = (float)P.X[a];
        pub.u[a] = (float)P.U[a];
    }
    for (int a = W_LO; a < 3; a++) pub.w[a] = (float)P.W[a];
}

// the published fields a free particle's substeps never change: in 2-D the
// out-of-plane position, velocity and in-plane spin; the radius
template <int D>
__device__ __forceinline__ void publish_const(const Priv& P, Pub& pub) {
    if (D == 2) {
        pub.x[2] = P.X[2];
        pub.xf[2] = (float)P.X[2];
        pub.u[2] = 0.f;
        pub.w[0] = pub.w[1] = 0.f;
    }
    pub.rf = P.Rf;
}

__device__ __forceinline__ void publish_s(const Priv& P, Pub& pub) {
    for (int a = 0; a < 3; a++) {
        pub.x[a] = P.X[a];
        pub.xf[a] = (float)P.X[a];
        pub.u[a] = (float)P.U[a];
        pub.w[a] = (float)P.W[a];
    }
    pub.rf = P.Rf;
}

constexpr int DEM_MAXA = 6;  // neighbours per particle staged in shared memory

// MDH: contact law PIBM_HERTZ_MD_HIST (the loading-history records); the other
// laws run an instantiation without them
template <int D, bool MDH>
__global__ void __launch_bounds__(DEM_T) k_dem(DemCfg C, DemState S, int nsub, int advance) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int sh[DEM_T];
    __shared__ int need_flag;
    cg::cluster_group cl = cg::this_cluster();
    const int per = C.per;
    Pub* pub = reinterpret_cast<Pub*>(smem);                     // [2][per]
    Priv* prv = reinterpret_cast<Priv*>(pub + 2 * per);          // [per]
    int2* adj = reinterpret_cast<int2*>(prv + per);              // [per][DEM_MAXA]: (neighbour, +-pair)
    const int n = C.n;
    const unsigned rank = cl.block_rank();
    const unsigned csize = cl.num_blocks();
    const int gt = rank * blockDim.x + threadIdx.x, gs = csize * blockDim.x;
    const int base = rank * per;
    const int nloc = max(0, min(per, n - base));
    const int cur = __ldcg(S.nb_cur);
    const int gbase = __ldcg(S.nb_cur + 1);  // global index of this launch's first substep
    const int* nb_start = cur ? S.nb_start1 : S.nb_start0;
    const int* nb_j = cur ? S.nb_j1 : S.nb_j0;
    float4* nb_ft = cur ? S.nb_ft1 : S.nb_ft0;
    double* nb_md = cur ? S.nb_md1 : S.nb_md0;
    const double dt = C.dt;
    const float dtf = (float)dt;
    int gnow = gbase;  // global substep counter after this launch

    // the learned hydrodynamic Jacobian, when set and passed by its gate
    const bool useJ = C.J != nullptr && __ldcg(C.J_on) != 0;
    if (advance) {
        const int hp = __ldcg(S.have_prev);
        // load the private state once; external accelerations are constant over the lattice step.
        // Every global load of a particle is issued before the first store: the stores go to
        // shared memory through pointers the compiler cannot separate from the global ones, so
        // interleaving them would expose one load latency per value.
        // Two passes: one thread per particle for the scalar state, then one thread per
        // (velocity component, particle) for the FP64 arithmetic of the opening half kick
        // and drift, so the FP64 chain is split over the warps as in the substeps.  The
        // second pass's loads are issued before the first pass (registers), so both
        // passes wait on memory once.
        constexpr int NU = D == 3 ? 3 : 2, NC = D == 3 ? 6 : 3;
        const int items = NC * nloc;
        double pre[3] = {0.0, 0.0, 0.0};  // hydrodynamic load now / before, m g (or 0) of item threadIdx.x
        if (threadIdx.x < items) {
            const int c = threadIdx.x / nloc, l = threadIdx.x - c * nloc, p = base + l;
            const bool lin = c < NU;
            const int a = lin ? c : (D == 3 ? c - 3 : 2);
            pre[0] = __ldcg((lin ? S.Fh : S.Th) + 3 * p + a);
            pre[1] = __ldcg((lin ? S.Fhp : S.Thp) + 3 * p + a);
            pre[2] = lin ? __ldcg(S.mg + p) : 0.0;
        }
        for (int l = threadIdx.x; l < nloc; l += blockDim.x) {
            const int p = base + l;
            double x[3], u[3], w[3];
            float fc[3], tc[3];
            for (int a = 0; a < 3; a++) {
                x[a] = __ldcg(S.X + 3 * p + a);
                u[a] = __ldcg(S.U + 3 * p + a);
                w[a] = __ldcg(S.W + 3 * p + a);
                fc[a] = __ldcg(S.Fc + 3 * p + a);
                tc[a] = __ldcg(S.Tc + 3 * p + a);
            }
            const double im = __ldcg(S.im + p), iI = __ldcg(S.iI + p), R = __ldcg(S.R + p);
            const int fixed = S.fixed[p];
            float wft[6][3];
            for (int f = 0; f < 2 * D; f++)
                for (int a = 0; a < 3; a++) wft[f][a] = __ldcg(S.wall_ft + 3 * (6 * p + f) + a);
            // the adjacency is fixed during the lattice step: stage it (up to DEM_MAXA entries)
            const int e0 = __ldcg(S.adj_start + p), ne = __ldcg(S.adj_start + p + 1) - e0;
            int2 ad[DEM_MAXA];
            for (int e = 0; e < DEM_MAXA; e++)
                ad[e] = e < ne ? make_int2(__ldcg(S.adj_nb + e0 + e), __ldcg(S.adj_k + e0 + e)) : make_int2(0, 0);
            Priv& P = prv[l];
            P.im = im;
            P.iI = iI;
            P.imf = (float)im;
            P.iIf = (float)iI;
            P.R = R;
            P.Rf = (float)R;
            P.fixed = fixed;
            P.wall_mask = 0;
            for (int f = 0; f < 2 * D; f++)
                if (wft[f][0] != 0.f || wft[f][1] != 0.f || wft[f][2] != 0.f) P.wall_mask |= 1 << f;
            for (int a = 0; a < 3; a++) {
                P.X[a] = x[a];
                P.U[a] = u[a];
                P.W[a] = w[a];
                P.Fc[a] = fc[a];
                P.Tc[a] = tc[a];
                P.a[a] = 0.f;
                P.al[a] = 0.f;
            }
            if (D == 2) {  // the components a 2-D particle cannot have
                P.U[2] = 0.0;
                P.W[0] = P.W[1] = 0.0;
            }
            P.nadj = ne;
            // staged as (owning CTA << 16 | slot in it, pair): the substeps need no division
            for (int e = 0; e < ne && e < DEM_MAXA; e++) {
                const int q = ad[e].x, rq = q / per;
                adj[l * DEM_MAXA + e] = make_int2((rq << 16) | (q - rq * per), ad[e].y);
            }
            // every published field, in both buffers; for a free particle the second pass
            // rewrites those that move
            publish_s(P, pub[l]);
            publish_s(P, pub[per + l]);
        }
        __syncthreads();
        // Accelerations and the opening half kick + drift, one (component, particle) per
        // thread.  The learned Jacobian's correction is zero here (U = U0 at the start of
        // the lattice step), so the kick is the plain one.
        const float hf0 = (float)(0.5 * dt);
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int c = it / nloc, l = it - c * nloc, p = base + l;
            const bool lin = c < NU;
            const int a = lin ? c : (D == 3 ? c - 3 : 2);
            if (it != threadIdx.x) {  // items beyond the first pass load here
                pre[0] = __ldcg((lin ? S.Fh : S.Th) + 3 * p + a);
                pre[1] = __ldcg((lin ? S.Fhp : S.Thp) + 3 * p + a);
                pre[2] = lin ? __ldcg(S.mg + p) : 0.0;
            }
            Priv& P = prv[l];
            const double hyd = hp ? 0.5 * (pre[0] + pre[1]) : pre[0];
            float acc;
            if (lin) {
                acc = (float)((hyd + pre[2] * C.g[a]) * P.im);
                P.a[a] = acc;
            } else {
                acc = (float)(hyd * P.iI);
                P.al[a] = acc;
            }
            if (P.fixed) continue;
            const float inc = lin ? hf0 * (P.Fc[a] * P.imf + acc) : hf0 * (P.Tc[a] * P.iIf + acc);
            double& V = lin ? P.U[a] : P.W[a];
            const double v = V + (double)inc;
            V = v;
            Pub& out = pub[l];
            Pub& out2 = pub[per + l];  // both buffers: substep 0 reads one, its drift writes the other
            if (lin) {
                const double xn = P.X[a] + dt * v;
                P.X[a] = xn;
                out.x[a] = out2.x[a] = xn;
                out.xf[a] = out2.xf[a] = (float)xn;
                out.u[a] = out2.u[a] = (float)v;
            } else {
                out.w[a] = out2.w[a] = (float)v;
            }
        }
        cl.sync();
        for (int sub = 0; sub < nsub; sub++) {
            const int rb = sub & 1;                      // published buffer read this substep
            // tangential history: entries carry the global substep that wrote them; a pair's
            // history is valid only if written in the previous substep (it was in contact),
            // so pairs out of contact cost no memory traffic
            const int gsub = gbase + sub;
            const float4* hist_old = nb_ft + (size_t)(gsub & 1) * C.cap;
            float4* hist_new = nb_ft + (size_t)((gsub + 1) & 1) * C.cap;
            const double* md_old = nb_md + (size_t)(gsub & 1) * MD_REC * C.cap;
            double* md_new = nb_md + (size_t)((gsub + 1) & 1) * MD_REC * C.cap;
            constexpr bool mdh = MDH;
            // tpp threads per particle (4 up to 64 particles per CTA, 2 up to 128, else
            // 1; 8 measured slower than 4 on 2-D beds): consecutive lanes, each taking
            // every tpp-th neighbour (the first also the walls, after the pairs);
            // warp-uniform loop so the shuffles below always see the whole warp
            const int tpp = per <= 64 ? 4 : (per <= 128 ? 2 : 1);
            const int ltpp = tpp == 8 ? 3 : (tpp == 4 ? 2 : (tpp == 2 ? 1 : 0));
            const int lane = threadIdx.x & 31, sl = lane & (tpp - 1);
            for (int l0 = (threadIdx.x >> 5) * (32 >> ltpp); l0 < nloc; l0 += (int)blockDim.x >> ltpp) {
                const int l = l0 + (lane >> ltpp);
                const bool active = l < nloc;
                float F[3] = {0.f, 0.f, 0.f}, T[3] = {0.f, 0.f, 0.f};  // contact sums (a few terms) in FP32
                if (active) {
                    const int p = base + l;
                    Priv& P = prv[l];
                    const Pub me = pub[rb * per + l];
                    const double Rp = P.R;
                    const float Rpf = P.Rf;
                    // 3-D: the wall histories are loaded now and used after the pairs (their
                    // latency hides behind the pair loop; in 2-D the extra registers cost more)
                    float hpre[D == 3 ? 18 : 1];
                    if (D == 3 && sl == 0) {
                        const float* wf = S.wall_ft + 18 * p;
#pragma unroll
                        for (int f = 0; f < 2 * D; f++)
#pragma unroll
                            for (int a = 0; a < 3; a++) hpre[3 * f + a] = (P.wall_mask >> f & 1) ? __ldcg(wf + 3 * f + a) : 0.f;
                    }
                    const int ne = P.nadj, e0 = ne > DEM_MAXA ? __ldcg(S.adj_start + p) : 0;
                    for (int e = sl; e < ne; e += tpp) {
                        int rq, lq, kk;
                        if (ne <= DEM_MAXA) {
                            const int2 a = adj[l * DEM_MAXA + e];
                            rq = a.x >> 16, lq = a.x & 0xffff, kk = a.y;
                        } else {
                            const int q = __ldcg(S.adj_nb + e0 + e);
                            kk = __ldcg(S.adj_k + e0 + e);
                            rq = q / per, lq = q - rq * per;
                        }
                        const bool first = kk >= 0;
                        const int k = first ? kk : ~kk;
                        // every load of the slot at once: the neighbour's published state and
                        // radius (distributed shared memory) and the pair's tangential history
                        // (global; used only in contact), so their latencies overlap
                        const float4 hv = __ldcg(hist_old + k);
                        const Pub other = cl.map_shared_rank(pub, rq)[rb * per + lq];
                        const double Rq = cl.map_shared_rank(prv, rq)[lq].R;
                        // FP32 prefilter from the published FP32 position and radius
                        const float dxf = other.xf[0] - me.xf[0], dyf = other.xf[1] - me.xf[1], dzf = other.xf[2] - me.xf[2];
                        const float sf = Rpf + other.rf + 1e-3f;
                        float3 Fa = f3(0.f, 0.f, 0.f), Ta = Fa, Tb = Fa, h = Fa;
                        MdRec md;
                        md_zero(md);
                        bool contact = false;
                        if (dxf * dxf + dyf * dyf + dzf * dzf < sf * sf) {
                            const Pub& A = first ? me : other;
                            const Pub& B = first ? other : me;
                            const double Ssum = first ? Rp + Rq : Rq + Rp;
                            // the exact FP64 contact test, in the oracle's operation order
                            const double d[3] = {__dsub_rn(B.x[0], A.x[0]), __dsub_rn(B.x[1], A.x[1]),
                                                 __dsub_rn(B.x[2], A.x[2])};
                            const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])),
                                                        __dmul_rn(d[2], d[2]));
                            const double SS = Ssum * Ssum;
                            contact = d2 < SS;
                            if (contact) {
                                if (__float_as_int(hv.w) == gsub - 1) {
                                    h = f3(hv.x, hv.y, hv.z);
                                    if (mdh) md_load(md_old + (size_t)MD_REC * k, md);
                                }
                                pair_force<MDH>(C, A, B, d, d2, SS, first ? Rpf : other.rf, first ? other.rf : Rpf, h, md, dtf,
                                           Fa, Ta, Tb);
                            }
                        }
                        if (first) {
                            if (contact) {
                                hist_new[k] = make_float4(h.x, h.y, h.z, __int_as_float(gsub));
                                if (mdh) md_store(md_new + (size_t)MD_REC * k, md);
                            }
                            F[0] += Fa.x, F[1] += Fa.y, F[2] += Fa.z;
                            T[0] += Ta.x, T[1] += Ta.y, T[2] += Ta.z;
                        } else {
                            F[0] -= Fa.x, F[1] -= Fa.y, F[2] -= Fa.z;
                            T[0] += Tb.x, T[1] += Tb.y, T[2] += Tb.z;
                        }
                    }
                    if (sl == 0) wall_forces<D, MDH>(C, S, p, me, Rp, Rpf, dtf, F, T, P.wall_mask, D == 3 ? hpre : nullptr);
                }
                // the tpp partial sums, in a fixed butterfly order: ((0 + 1) + (2 + 3)) + ...
                if (tpp > 1)
                    for (int a = 0; a < 3; a++) {
                        F[a] += __shfl_xor_sync(0xffffffffu, F[a], 1);
                        T[a] += __shfl_xor_sync(0xffffffffu, T[a], 1);
                    }
                if (tpp > 2)
                    for (int a = 0; a < 3; a++) {
                        F[a] += __shfl_xor_sync(0xffffffffu, F[a], 2);
                        T[a] += __shfl_xor_sync(0xffffffffu, T[a], 2);
                    }
                if (tpp > 4)
                    for (int a = 0; a < 3; a++) {
                        F[a] += __shfl_xor_sync(0xffffffffu, F[a], 4);
                        T[a] += __shfl_xor_sync(0xffffffffu, T[a], 4);
                    }
                if (!active) continue;
                const int p = base + l;
                Priv& P = prv[l];
                const bool last = sub + 1 == nsub;  // closing half kick only; else also the next opening one
                // the contact sums are read from shared memory only by the write-back (and by
                // the learned-Jacobian kick below); the per-component kick takes the registers
                if (sl == 0 && (last || useJ))
                    for (int a = 0; a < 3; a++) {
                        P.Fc[a] = F[a];
                        P.Tc[a] = T[a];
                    }
                if (P.fixed) continue;  // published into both buffers at the load
                if (useJ) {  // the learned Jacobian couples the components: one thread per particle
                    if (sl != 0) continue;
                    const float* Jp = C.J + SG_NJ * p;
                    if (!last) {
                        kick_s<D>(P, dt, dtf, Jp, S.U + 3 * p, S.W + 3 * p);
                        drift_s<D>(P, dt, pub[(rb ^ 1) * per + l]);
                    } else {
                        kick_s<D>(P, 0.5 * dt, (float)(0.5 * dt), Jp, S.U + 3 * p, S.W + 3 * p);
                    }
                    continue;
                }
                // one velocity component per thread of the particle: the same operations as
                // kick_s and drift_s, with the FP64 chain split over the tpp threads (2-D: U_x,
                // U_y, omega_z; 3-D: U then omega)
                const float hf = last ? (float)(0.5 * dt) : dtf;
                Pub& out = pub[(rb ^ 1) * per + l];
                constexpr int NU = D == 3 ? 3 : 2, NC = D == 3 ? 6 : 3;
                for (int c = sl; c < NC; c += tpp) {
                    const bool lin = c < NU;
                    const int a = lin ? c : (D == 3 ? c - 3 : 2);
                    const float Fa_ = a == 0 ? F[0] : (a == 1 ? F[1] : F[2]);
                    const float Ta_ = a == 0 ? T[0] : (a == 1 ? T[1] : T[2]);
                    const float inc = lin ? hf * (Fa_ * P.imf + P.a[a]) : hf * (Ta_ * P.iIf + P.al[a]);
                    double& V = lin ? P.U[a] : P.W[a];
                    const double v = V + (double)inc;
                    V = v;
                    if (!last) {
                        const float vf = (float)v;
                        if (lin) {
                            const double xn = P.X[a] + dt * v;
                            P.X[a] = xn;
                            out.x[a] = xn;
                            out.xf[a] = (float)xn;
                            out.u[a] = vf;
                        } else {
                            out.w[a] = vf;
                        }
                    }
                }
            }
            if (sub + 1 < nsub) cl.sync();
        }
        // After the last substep no CTA changes anything another reads (the last kick
        // publishes nothing), so a CTA barrier suffices; the write-back's loads are
        // issued before it.
        double wb[13];  // write-back inputs of this thread's first particle (C_p, T_p, H, H_prev, F_h, tau_h, X_build)
        if ((int)threadIdx.x < nloc) {
            const int p = base + threadIdx.x;
            wb[0] = __ldcg(S.Cp + p), wb[1] = __ldcg(S.Tp + p), wb[2] = __ldcg(S.Hh + p);
            wb[3] = __ldcg(S.Hhp + p);
            for (int a = 0; a < 3; a++) {
                wb[4 + a] = __ldcg(S.Fh + 3 * p + a);
                wb[7 + a] = __ldcg(S.Th + 3 * p + a);
                wb[10 + a] = __ldcg(S.Xb + 3 * p + a);
            }
        }
        __syncthreads();
        gnow = gbase + nsub;
        // write back; thermosensitive particles: C_p dT_p / dt = -H_p over one
        // lattice step, with the learned Jacobian in use C_p (T_new - T) =
        // -(H + J_HT (T_new - T)) (J_HT < 0 counts as 0); keep this step's
        // coupling as the previous one
        int moved = 0;
        const double thr2 = 0.25 * (C.skin - 1.0) * (C.skin - 1.0);
        const double err2 = 0.25 * C.skin * C.skin;
        for (int l = threadIdx.x; l < nloc; l += blockDim.x) {
            const int p = base + l;
            const Priv& P = prv[l];
            // loads first (the stores below may alias them as far as the compiler knows);
            // the first particle of each thread was loaded before the barrier
            if (l != (int)threadIdx.x) {
                wb[0] = __ldcg(S.Cp + p), wb[1] = __ldcg(S.Tp + p), wb[2] = __ldcg(S.Hh + p);
                wb[3] = __ldcg(S.Hhp + p);
                for (int a = 0; a < 3; a++) {
                    wb[4 + a] = __ldcg(S.Fh + 3 * p + a);
                    wb[7 + a] = __ldcg(S.Th + 3 * p + a);
                    wb[10 + a] = __ldcg(S.Xb + 3 * p + a);
                }
            }
            const double cp = wb[0], tp = wb[1], hh = wb[2], hhp = hp ? wb[3] : 0.0;
            const double fh[3] = {wb[4], wb[5], wb[6]}, th[3] = {wb[7], wb[8], wb[9]}, xb[3] = {wb[10], wb[11], wb[12]};
            if (cp > 0.0) {
                double jh = useJ ? (double)__ldcg(C.J + SG_NJ * (long long)p + 18) : 0.0;
                if (!(jh > 0.0)) jh = 0.0;
                S.Tp[p] = tp - (hp ? 0.5 * (hh + hhp) : hh) / (cp + jh);
            }
            double d2 = 0;
            for (int a = 0; a < 3; a++) {
                S.X[3 * p + a] = P.X[a];
                S.U[3 * p + a] = P.U[a];
                S.W[3 * p + a] = P.W[a];
                S.Fc[3 * p + a] = P.Fc[a];
                S.Tc[3 * p + a] = P.Tc[a];
                S.Fhp[3 * p + a] = fh[a];
                S.Thp[3 * p + a] = th[a];
            }
            for (int a = 0; a < (D == 3 ? 3 : 2); a++) {  // a 2-D particle does not move out of plane
                double dd = P.X[a] - xb[a];
                d2 += dd * dd;
            }
            S.Hhp[p] = hh;
            if (d2 > thr2) moved = 1;
            if (d2 > err2) set_error(S.dstat, 2);
        }
        moved = __syncthreads_or(moved);
        if (threadIdx.x == 0) need_flag = moved;
        if (gt == 0) *S.have_prev = 1;
        cl.sync();
        // thread r reads CTA r's flag (16 remote loads per CTA, not one per thread and CTA)
        const int need = __syncthreads_or(threadIdx.x < csize ? *cl.map_shared_rank(&need_flag, threadIdx.x) : 0);
        if (!need) {
            cl.sync();  // no CTA may exit while others still read its shared memory
            if (gt == 0) S.nb_cur[1] = gnow;
            return;
        }
    }

    // ------------------------------------------------ rebuild at new positions
    for (int p = gt; p < n; p += gs) {
        double Xp[3];
        ldX(S.X, p, Xp);
        int c[3];
        cell_coords<D>(C, Xp, c);
        S.cell_of[p] = (c[2] * C.nc[1] + c[1]) * C.nc[0] + c[0];
    }
    for (int cidx = gt; cidx < C.ncell; cidx += gs) S.cell_cnt[cidx] = 0;
    if (gt == 0) *S.flag = 0;
    cl.sync();
    for (int p = gt; p < n; p += gs) atomicAdd(S.cell_cnt + __ldcg(S.cell_of + p), 1);
    cl.sync();
    if (rank == 0) {
        cta_scan(S.cell_cnt, S.cell_start, C.ncell, sh);
        for (int cidx = threadIdx.x; cidx < C.ncell; cidx += blockDim.x) S.cell_cnt[cidx] = 0;
    }
    cl.sync();
    for (int p = gt; p < n; p += gs) {
        int cidx = __ldcg(S.cell_of + p);
        int pos = atomicAdd(S.cell_cnt + cidx, 1);
        S.cell_ids[__ldcg(S.cell_start + cidx) + pos] = p;
    }
    cl.sync();
    for (int cidx = gt; cidx < C.ncell; cidx += gs) {  // stable order: by particle index
        int b = __ldcg(S.cell_start + cidx), e = __ldcg(S.cell_start + cidx + 1);
        for (int a = b + 1; a < e; a++) {
            int v = __ldcg(S.cell_ids + a), q = a - 1;
            while (q >= b && __ldcg(S.cell_ids + q) > v) {
                S.cell_ids[q + 1] = __ldcg(S.cell_ids + q);
                q--;
            }
            S.cell_ids[q + 1] = v;
        }
    }
    cl.sync();
    // neighbour counts (pairs within R_i + R_j + skin)
    for (int i = gt; i < n; i += gs) {
        double Xi[3];
        ldX(S.X, i, Xi);
        int c[3];
        cell_coords<D>(C, Xi, c);
        int hi = 0, lo = 0;
        double Ri = S.R[i];
        for_neighbours<D>(C, S, c, [&](int j) {
            if (j == i) return;
            double Xj[3];
            ldX(S.X, j, Xj);
            double cut = Ri + S.R[j] + C.skin;
            if (dist2(Xi, Xj) < cut * cut) {
                if (j > i) hi++;
                else lo++;
            }
        });
        S.cnt_hi[i] = hi;
        S.cnt_lo[i] = lo;
        if (hi + lo > DEM_MAXNB) {
            set_error(S.dstat, 1);
            atomicExch(S.flag, 1);
        }
    }
    cl.sync();
    int* nst = cur ? S.nb_start0 : S.nb_start1;
    int* ni = cur ? S.nb_i0 : S.nb_i1;
    int* nj = cur ? S.nb_j0 : S.nb_j1;
    // histories written in the last substep (stamp gnow - 1) live in buffer gnow & 1 of the
    // old list; the new list gets them in the same buffer with the same stamp
    float4* nft = (cur ? S.nb_ft0 : S.nb_ft1) + (size_t)(gnow & 1) * C.cap;
    const float4* oft = nb_ft + (size_t)(gnow & 1) * C.cap;
    double* nmd = (cur ? S.nb_md0 : S.nb_md1) + (size_t)(gnow & 1) * MD_REC * C.cap;
    const double* omd = (cur ? S.nb_md1 : S.nb_md0) + (size_t)(gnow & 1) * MD_REC * C.cap;
    if (rank == 0) {
        cta_scan(S.cnt_hi, nst, n, sh);
        for (int i = threadIdx.x; i < n; i += blockDim.x) S.cnt_lo[i] += S.cnt_hi[i];
        __syncthreads();
        cta_scan(S.cnt_lo, S.adj_new, n, sh);
        if (threadIdx.x == 0 && (nst[n] > C.cap || S.adj_new[n] > S.adj_cap)) {
            set_error(S.dstat, 3);
            *S.flag = 1;
        }
    }
    cl.sync();
    if (__ldcg(S.flag)) {  // keep the previous list and adjacency; the host reports the status
        if (gt == 0) S.nb_cur[1] = gnow;
        return;
    }
    for (int i = gt; i < n; i += gs) {
        double Xi[3];
        ldX(S.X, i, Xi);
        int c[3];
        cell_coords<D>(C, Xi, c);
        int cand[DEM_MAXNB], cnt = 0;
        double Ri = S.R[i];
        for_neighbours<D>(C, S, c, [&](int j) {
            if (j <= i) return;
            double Xj[3];
            ldX(S.X, j, Xj);
            double cut = Ri + S.R[j] + C.skin;
            if (dist2(Xi, Xj) < cut * cut && cnt < DEM_MAXNB) cand[cnt++] = j;
        });
        for (int a = 1; a < cnt; a++) {
            int v = cand[a], q = a - 1;
            while (q >= 0 && cand[q] > v) {
                cand[q + 1] = cand[q];
                q--;
            }
            cand[q + 1] = v;
        }
        int o = __ldcg(nst + i);
        int ob = nb_start[i], oe = nb_start[i + 1];
        for (int r = 0; r < cnt; r++) {
            int j = cand[r];
            ni[o + r] = i;
            nj[o + r] = j;
            int L = ob, Hh = oe - 1, found = -1;
            while (L <= Hh) {
                int mid = (L + Hh) >> 1, v = nb_j[mid];
                if (v == j) { found = mid; break; }
                if (v < j) L = mid + 1;
                else Hh = mid - 1;
            }
            nft[o + r] = found >= 0 ? __ldcg(oft + found) : make_float4(0.f, 0.f, 0.f, __int_as_float(-2));
            if constexpr (MDH) {  // (a pair without history is stamped invalid above)
                MdRec md;
                if (found >= 0) md_load(omd + (size_t)MD_REC * found, md);
                else md_zero(md);
                md_store(nmd + (size_t)MD_REC * (o + r), md);
            }
        }
    }
    cl.sync();
    // adjacency of each particle: partners j < i (pair found in j's segment), then j > i
    for (int i = gt; i < n; i += gs) {
        double Xi[3];
        ldX(S.X, i, Xi);
        int c[3];
        cell_coords<D>(C, Xi, c);
        int cand[DEM_MAXNB], cnt = 0;
        double Ri = S.R[i];
        for_neighbours<D>(C, S, c, [&](int j) {
            if (j >= i) return;
            double Xj[3];
            ldX(S.X, j, Xj);
            double cut = Ri + S.R[j] + C.skin;
            if (dist2(Xi, Xj) < cut * cut && cnt < DEM_MAXNB) cand[cnt++] = j;
        });
        for (int a = 1; a < cnt; a++) {
            int v = cand[a], q = a - 1;
            while (q >= 0 && cand[q] > v) {
                cand[q + 1] = cand[q];
                q--;
            }
            cand[q + 1] = v;
        }
        int e0 = __ldcg(S.adj_new + i);
        for (int r = 0; r < cnt; r++) {
            int j = cand[r];
            int L = __ldcg(nst + j), Hh = __ldcg(nst + j + 1) - 1, found = -1;
            while (L <= Hh) {
                int mid = (L + Hh) >> 1, v = __ldcg(nj + mid);
                if (v == i) { found = mid; break; }
                if (v < i) L = mid + 1;
                else Hh = mid - 1;
            }
            if (found < 0) set_error(S.dstat, 4);
            S.adj_nb[e0 + r] = j;
            S.adj_k[e0 + r] = ~found;
        }
        int o = __ldcg(nst + i), oc = __ldcg(nst + i + 1) - o;
        for (int r = 0; r < oc; r++) {
            S.adj_nb[e0 + cnt + r] = __ldcg(nj + o + r);
            S.adj_k[e0 + cnt + r] = o + r;
        }
        for (int a = 0; a < 3; a++) S.Xb[3 * i + a] = Xi[a];
    }
    cl.sync();
    for (int i = gt; i <= n; i += gs) S.adj_start[i] = __ldcg(S.adj_new + i);
    if (gt == 0) {
        S.nb_cur[0] = cur ^ 1;
        S.nb_cur[1] = gnow;
    }
}

// cluster size: up to 16 CTAs of DEM_T threads, at most DEM_MAXPER particles per CTA
constexpr int DEM_MAXPER = 640;  // (2 * 64 + 168 + 48) B per particle: 220 KB of shared memory

static size_t dem_smem(int per) { return (size_t)per * (2 * sizeof(Pub) + sizeof(Priv) + DEM_MAXA * sizeof(int2)); }

// the DEM kernel of the context's dimension and contact law
using DemKernel = void (*)(DemCfg, DemState, int, int);
static DemKernel dem_kernel(const Ctx* c) {
    const bool h = c->dem.law == PIBM_HERTZ_MD_HIST;
    if (c->D == 2) return h ? k_dem<2, true> : k_dem<2, false>;
    return h ? k_dem<3, true> : k_dem<3, false>;
}

int dem_cluster_size(Ctx* c) {
    int n = c->np;
    int cs = c->tune_dem_particles_per_cta > 0 ? (n + c->tune_dem_particles_per_cta - 1) / c->tune_dem_particles_per_cta
                                               : (n + 31) / 32;
    cs = cs < 1 ? 1 : (cs > 16 ? 16 : cs);
    if (cs > 8) {
        int max16 = 0;  // is a 16-CTA cluster with this much shared memory schedulable here?
        {
            auto kern = dem_kernel(c);
            int per = (n + 15) / 16;
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dem_smem(DEM_MAXPER)) == cudaSuccess) {
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(16, 1, 1);
                cfg.blockDim = dim3(DEM_T, 1, 1);
                cfg.dynamicSmemBytes = dem_smem(per);
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = 16;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                int clusters = 0;
                if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) == cudaSuccess && clusters > 0) max16 = 1;
            }
            cudaGetLastError();
        }
        if (!max16) cs = 8;
    }
    return cs;
}

int dem_max_particles() { return 16 * DEM_MAXPER; }
int dem_max_per_cta() { return DEM_MAXPER; }

static DemState dem_state(Ctx* c) {
    DemState S;
    S.X = c->X, S.U = c->U, S.W = c->W, S.Xb = c->Xb, S.R = c->R, S.m = c->m, S.I = c->I, S.mg = c->mg;
    S.im = c->im, S.iI = c->iI;
    S.Tp = c->Tp, S.Cp = c->Cp, S.Fh = c->Fh, S.Th = c->Th, S.Hh = c->Hh, S.Fc = c->Fc, S.Tc = c->Tc;
    S.Fhp = c->Fh_prev, S.Thp = c->Th_prev, S.Hhp = c->Hh_prev, S.have_prev = c->have_prev;
    S.adj_new = c->adj_start_new;
    S.fixed = c->fixed;
    S.cell_of = c->cell_of, S.cell_cnt = c->cell_cnt, S.cell_start = c->cell_start, S.cell_ids = c->cell_ids;
    S.cnt_hi = c->cnt_hi, S.cnt_lo = c->cnt_lo;
    S.nb_start0 = c->nb_start[0], S.nb_start1 = c->nb_start[1];
    S.nb_i0 = c->nb_i[0], S.nb_i1 = c->nb_i[1];
    S.nb_j0 = c->nb_j[0], S.nb_j1 = c->nb_j[1];
    S.nb_ft0 = (float4*)c->nb_ft[0], S.nb_ft1 = (float4*)c->nb_ft[1];
    S.nb_md0 = c->nb_md[0], S.nb_md1 = c->nb_md[1];
    S.wall_md = c->wall_md;
    S.nb_cur = c->nb_cur;
    S.adj_start = c->adj_start, S.adj_nb = c->adj_nb, S.adj_k = c->adj_k;
    S.wall_ft = c->wall_ft;
    S.dstat = c->dstat;
    S.flag = c->dstat + 2;
    S.adj_cap = c->adj_cap;
    return S;
}

cudaError_t launch_dem(Ctx* c, cudaStream_t s, int nsub) {
    if (c->np <= 0) return cudaSuccess;
    int cs = c->dem_cs;
    DemCfg C = c->dem;
    C.per = (c->np + cs - 1) / cs;
    auto kern = dem_kernel(c);
    size_t smem = dem_smem(C.per);
    const int variant = 1 << ((c->D == 2 ? 0 : 2) + (c->dem.law == PIBM_HERTZ_MD_HIST ? 1 : 0));
    if (!(c->dem_attr_ok & variant)) {  // once per context and kernel: host calls, not needed per launch
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dem_smem(DEM_MAXPER));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        c->dem_attr_ok |= variant;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(DEM_T, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    DemState S = dem_state(c);
    int advance = nsub > 0 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, C, S, nsub, advance);
}

// ---------------------------------------------------- contacts for read-back
// Pairs of the current neighbour list with |X_i - X_j| < R_i + R_j (FP64, the
// oracle's operation order), in list order, i.e. sorted by (i, j).
__global__ void __launch_bounds__(DEM_T) k_contacts(int n, const double* X, const double* R, const int* nb_cur,
                                                    const int* st0, const int* st1, const int* j0, const int* j1,
                                                    int* cnt, int* pairs, int cap, int* total) {
    __shared__ int sh[DEM_T];
    const int cur = *nb_cur;
    const int* st = cur ? st1 : st0;
    const int* nj = cur ? j1 : j0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int c = 0;
        for (int k = st[i]; k < st[i + 1]; k++) {
            int j = nj[k];
            double s = R[i] + R[j];
            if (dist2(X + 3 * i, X + 3 * j) < s * s) c++;
        }
        cnt[i] = c;
    }
    __syncthreads();
    cta_scan(cnt, cnt + n + 1, n, sh);
    const int* off = cnt + n + 1;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int o = off[i];
        for (int k = st[i]; k < st[i + 1]; k++) {
            int j = nj[k];
            double s = R[i] + R[j];
            if (dist2(X + 3 * i, X + 3 * j) < s * s) {
                if (o < cap) {
                    pairs[2 * o] = i;
                    pairs[2 * o + 1] = j;
                }
                o++;
            }
        }
    }
    if (threadIdx.x == 0) *total = off[n];
}

cudaError_t launch_contacts(Ctx* c, int* d_pairs, int cap, int* d_count) {
    // d_count: total, then per-particle counts (n) and their offsets (n + 1)
    k_contacts<<<1, DEM_T, 0, c->s0>>>(c->np, c->X, c->R, c->nb_cur, c->nb_start[0], c->nb_start[1], c->nb_j[0],
                                       c->nb_j[1], d_count + 1, d_pairs, cap, d_count);
    return cudaGetLastError();
}

// cell of each particle at the current positions (same definition as the rebuild)
template <int D>
__global__ void k_cells(DemCfg C, const double* X, int n, int* cell) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        double Xp[3] = {X[3 * p], X[3 * p + 1], X[3 * p + 2]};
        int c[3];
        cell_coords<D>(C, Xp, c);
        cell[p] = (c[2] * C.nc[1] + c[1]) * C.nc[0] + c[0];
    }
}

cudaError_t launch_cells(Ctx* c, int* d_cell) {
    if (c->np <= 0) return cudaSuccess;
    int blocks = (c->np + 255) / 256;
    if (c->D == 2) k_cells<2><<<blocks, 256, 0, c->s0>>>(c->dem, c->X, c->np, d_cell);
    else k_cells<3><<<blocks, 256, 0, c->s0>>>(c->dem, c->X, c->np, d_cell);
    return cudaGetLastError();
}

}  // namespace pibm

// mmx_box_res.cuh -- the H/M half steps of the magnetic box (Sec. 3.2.2,
// Steps 1 and 3: Eqs. llg_tra4-llg_tra6, N() and Eq. iterate_H iterated to
// the domain-wide tolerance) with every magnetic face's iteration records
// held in shared memory for the whole launch.
//
// Same scheme, same arithmetic and same device-side loop control as
// k_hm_box (the list-driven kernel of mmx_kernels.cuh); what differs is where
// the per-face records live.  k_hm_box keeps them in global memory, so every
// phase of every half step reloads and rewrites them (about 100 bytes per
// magnetic face per phase through L2); here block b owns the faces
// b F 256 ... (b+1) F 256 - 1 of the magnetic list (F per thread), loads
// their list entries and M^n once, and keeps M^n / e0, beta / C', the
// current increment DeltaM and the curl sum of each face in shared memory
// across both half steps of a launch.  A phase then reads only the
// neighbours' H iterates (box-local arrays in L2) and the read-only face
// constants.  It applies while the box's magnetic faces fit in the GPU's
// shared memory: F <= kResMaxF faces per thread over one resident wave of
// blocks (the 128x128x512 waveguide's 0.354 M faces take F = 2).
#pragma once
#include "mmx_kernels.cuh"

namespace mmx {

constexpr int kResThreads = 256;
constexpr int kResMaxF = 3;

// Code-size and occupancy settings of the resident kernel, measured on the
// 128x128x512 waveguide (two-half-step launch, FP32): the LLG solve written
// once for a run-time face family and inlined at its two call sites, 5
// blocks/SM (48 registers, F = 2): 44.3 us; the list-driven kernel 47.8 us;
// the first version, with the solve inlined for each family and half step
// (18 copies; its largest stall was instruction fetch), 47.1 us.  One
// non-inlined copy of the solve and of the half step (MMX_RES_NOINLINE)
// spills under the 48-register bound: 69.7 us (76.7 us with 4 blocks/SM and
// F = 3); inlined with 4 blocks/SM and F = 3, 49.7 us.  All bit-identical.
#ifndef MMX_RES_NOINLINE
#define MMX_RES_NOINLINE 0
#endif
#ifndef MMX_RES_MINB
#define MMX_RES_MINB 5
#endif
#if MMX_RES_NOINLINE
#define MMX_RES_FN __noinline__
#else
#define MMX_RES_FN __forceinline__
#endif

// Shared-memory bytes of a block with F faces per thread: list entry (int4),
// M^n and e0, beta and C', DeltaM (Q4 each) and the curl sum (T).
template <typename T> constexpr size_t res_smem_bytes(int F)
{
    return (size_t)F * kResThreads * (sizeof(int4) + 3 * sizeof(Q4<T>) + sizeof(T));
}

template <typename T> struct ResSmem {
    int4 *ent;
    Q4<T> *mn, *bc, *dm;
    T *curl;
};

template <typename T> __device__ __forceinline__ ResSmem<T> res_smem(int F)
{
    extern __shared__ __align__(16) unsigned char res_raw[];
    const int n = F * kResThreads;
    ResSmem<T> r;
    r.ent = reinterpret_cast<int4 *>(res_raw);
    r.mn = reinterpret_cast<Q4<T> *>(res_raw + (size_t)n * sizeof(int4));
    r.bc = r.mn + n;
    r.dm = r.bc + n;
    r.curl = reinterpret_cast<T *>(r.dm + n);
    return r;
}

// Component d (0, 1, 2 at run time) of a register vector, by selects, so
// that no register array is indexed at run time.
template <typename T> __device__ __forceinline__ T pick(const T v[3], int d)
{
    return d == 0 ? v[0] : d == 1 ? v[1] : v[2];
}

// The four-point H vector at a face of run-time family d (the gather is the
// only part that differs between families; one short inlined copy each).
template <typename T, typename SG>
__device__ __forceinline__ void h_vector_rt(const Geo &g, const Box<T> &b, SG *const Hg[3], T *const Hb[3], int mode,
                                            const FaceOf &fo, T h[3], T sH)
{
    if (fo.d == 0)
        h_vector<0>(g, b, Hg, Hb, mode, fo.i, fo.j, fo.k, h, sH);
    else if (fo.d == 1)
        h_vector<1>(g, b, Hg, Hb, mode, fo.i, fo.j, fo.k, h, sH);
    else
        h_vector<2>(g, b, Hg, Hb, mode, fo.i, fo.j, fo.k, h, sH);
}

// Three components passed by value (in registers) to the non-inlined solves.
template <typename T> struct V3 {
    T x, y, z;
};

// The closed-form solve of llg_iterate (Eqs. llg_tra4-llg_tra6, N(),
// Eq. iterate_H in increment form) for a run-time family d: the same
// operations in the same order, with the component-d terms picked by
// selects.  Non-inlined so that one copy serves every phase and family.
// Returns (DeltaM, the on-sphere increment of component d).
template <typename T>
__device__ MMX_RES_FN Q4<T> llg_solve_rt(V3<T> mn, V3<T> bt, V3<T> he, T kap, T s, T Ms, T e0, int d)
{
    const T Mn[3] = {mn.x, mn.y, mn.z}, beta[3] = {bt.x, bt.y, bt.z};
    T u[3] = {kap * he.x, kap * he.y, kap * he.z};
    T m2 = Ms * Ms - e0;
    T p = u[0] * Mn[0] + u[1] * Mn[1] + u[2] * Mn[2];
    T q = (u[0] + s * Mn[0]) * beta[0] + (u[1] + s * Mn[1]) * beta[1] + (u[2] + s * Mn[2]) * beta[2];
    T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    T c_u = p + s * m2 + q;
    T c_m = s * q - s * p - uu;
    T uxm[3] = {u[1] * Mn[2] - u[2] * Mn[1], u[2] * Mn[0] - u[0] * Mn[2], u[0] * Mn[1] - u[1] * Mn[0]};
    T uxb[3] = {u[1] * beta[2] - u[2] * beta[1], u[2] * beta[0] - u[0] * beta[2], u[0] * beta[1] - u[1] * beta[0]};
    T mxb[3] = {Mn[1] * beta[2] - Mn[2] * beta[1], Mn[2] * beta[0] - Mn[0] * beta[2],
                Mn[0] * beta[1] - Mn[1] * beta[0]};
    T inv = llg_rcp(T(1) + uu + T(2) * s * p + s * s * m2);
    T del[3];
#pragma unroll
    for (int c = 0; c < 3; c++)
        del[c] = (beta[c] + c_u * u[c] + c_m * Mn[c] + uxm[c] + uxb[c] + s * mxb[c]) * inv;
    // renormalised_increment with the component-d term by select
    T md = Mn[0] * del[0] + Mn[1] * del[1] + Mn[2] * del[2];
    T dd = del[0] * del[0] + del[1] * del[1] + del[2] * del[2];
    T q0 = -(T(2) * md + dd);
    T qv = e0 + q0;
    T xn = llg_sqrt(Ms * Ms - qv);
    T den = llg_rcp(xn * (Ms + xn));
    T sm1 = qv * den;
    T dM[3];
#pragma unroll
    for (int c = 0; c < 3; c++) dM[c] = del[c] + (del[c] + Mn[c]) * sm1;
    const T deld = pick(del, d), mnd = pick(Mn, d);
    return q4(dM[0], dM[1], dM[2], deld + (deld + mnd) * (q0 * den));
}

// The first-order update of llg_euler for a run-time family d.
template <typename T>
__device__ MMX_RES_FN Q4<T> llg_euler_rt(V3<T> mn, V3<T> he, T c1, T c2, T Ms, T e0, int d)
{
    const T Mn[3] = {mn.x, mn.y, mn.z}, heff[3] = {he.x, he.y, he.z};
    T mxh[3] = {Mn[1] * heff[2] - Mn[2] * heff[1], Mn[2] * heff[0] - Mn[0] * heff[2],
                Mn[0] * heff[1] - Mn[1] * heff[0]};
    T mxmxh[3] = {Mn[1] * mxh[2] - Mn[2] * mxh[1], Mn[2] * mxh[0] - Mn[0] * mxh[2],
                  Mn[0] * mxh[1] - Mn[1] * mxh[0]};
    T del[3];
#pragma unroll
    for (int c = 0; c < 3; c++) del[c] = -c1 * mxh[c] - c2 * mxmxh[c];
    T md = Mn[0] * del[0] + Mn[1] * del[1] + Mn[2] * del[2];
    T dd = del[0] * del[0] + del[1] * del[1] + del[2] * del[2];
    T q0 = -(T(2) * md + dd);
    T qv = e0 + q0;
    T xn = llg_sqrt(Ms * Ms - qv);
    T den = llg_rcp(xn * (Ms + xn));
    T sm1 = qv * den;
    T dM[3];
#pragma unroll
    for (int c = 0; c < 3; c++) dM[c] = del[c] + (del[c] + Mn[c]) * sm1;
    const T deld = pick(del, d), mnd = pick(Mn, d);
    return q4(dM[0], dM[1], dM[2], deld + (deld + mnd) * (q0 * den));
}

template <typename T> __device__ __forceinline__ T *pick_ptr(T *const p[3], int d)
{
    return d == 0 ? p[0] : d == 1 ? p[1] : p[2];
}

// Phase 0 on one magnetic face (list position t, slot s): C' = H^n -
// dt/(2 mu0) curl E, beta = -kappa M^n x H_eff^n, e0 and the first iterate
// (or the first-order update); H^1 into Hw.  second: H^n from the previous
// half step's iterate buffer Hp, M^n = M^n + DeltaM of that half step, and
// the curl sum stored by the first half step.
template <int ORD, typename T, typename S>
__device__ __forceinline__ T res_first(const Geo &g, const Fields<T, S> &f, const Box<T> &b, S *const Hin[3],
                                       T *const Hp[3], T *const Hw[3], const ResSmem<T> &sm, int s,
                                       const FaceOf &fo, int t, const T h0[3], bool second, bool write,
                                       S *const Hout[3], bool &ok)
{
    const Q4<T> cs = q4_load(b.cst + t);
    const int d = fo.d;
    T Mn[3], hn, csum, h[3];
    const Q4<T> m0 = sm.mn[s];
    if (second) {
        const Q4<T> d0 = sm.dm[s];
        Mn[0] = m0.x + d0.x;
        Mn[1] = m0.y + d0.y;
        Mn[2] = m0.z + d0.z;
        hn = pick_ptr(Hp, d)[fo.l];
        csum = sm.curl[s];
        h_vector_rt(g, b, Hin, Hp, 1, fo, h, f.sH);
    } else {
        Mn[0] = m0.x;
        Mn[1] = m0.y;
        Mn[2] = m0.z;
        const unsigned q = gidx32(g, fo.i, fo.j, fo.k);
        T rest, zp;
        curl_e32(g, f.E, f.inv_d, d, q, rest, zp, f.sE);
        csum = rest + zp;
        sm.curl[s] = csum;
        hn = ld_s(pick_ptr(Hin, d) + q, f.sH);
        h_vector_rt(g, b, Hin, Hp, 0, fo, h, f.sH);
    }
    const T Ms = cs.x, k1 = cs.y, k2 = cs.z;
    const T cp = hn - b.cfar * csum;
    const T e0 = norm_defect(Ms, Mn[0], Mn[1], Mn[2]);
    T heff[3];
#pragma unroll
    for (int c = 0; c < 3; c++) heff[c] = h0[c] + h[c];
    T beta[3] = {T(0), T(0), T(0)};
    Q4<T> r;
    const V3<T> mn = {Mn[0], Mn[1], Mn[2]}, he = {heff[0], heff[1], heff[2]};
    if constexpr (ORD == 2) {
        beta[0] = -k1 * (Mn[1] * heff[2] - Mn[2] * heff[1]);
        beta[1] = -k1 * (Mn[2] * heff[0] - Mn[0] * heff[2]);
        beta[2] = -k1 * (Mn[0] * heff[1] - Mn[1] * heff[0]);
        r = llg_solve_rt(mn, V3<T>{beta[0], beta[1], beta[2]}, he, k1, k2, Ms, e0, d);
    } else {
        r = llg_euler_rt(mn, he, k1, k2, Ms, e0, d);
    }
    sm.bc[s] = q4(beta[0], beta[1], beta[2], cp);
    sm.mn[s] = q4(Mn[0], Mn[1], Mn[2], e0);
    sm.dm[s] = q4(r.x, r.y, r.z, T(0));
    const bool wall = wall_node(g, d, d == 0 ? fo.i : d == 1 ? fo.j : fo.k);
    const T hv = wall ? T(0) : cp - r.w;
    pick_ptr(Hw, d)[fo.l] = hv;
    if (write) ok &= res_store(g, f, b, Hout, fo, t, hv, q4(Mn[0], Mn[1], Mn[2], e0), q4(r.x, r.y, r.z, T(0)));
    return max(abs(r.x), max(abs(r.y), abs(r.z))) * cs.w;
}

// Iterate r >= 2 on one magnetic face from the neighbours' iterate r-1 in
// Hprev: DeltaM^r replaces DeltaM^(r-1) in shared memory, H^r into Hcur.
// Returns max_c |DeltaM^r_c - DeltaM^(r-1)_c| / Ms.
template <typename T, typename S>
__device__ __forceinline__ T res_next(const Geo &g, const Fields<T, S> &f, const Box<T> &b, T *const Hprev[3],
                                      T *const Hcur[3], const ResSmem<T> &sm, int s, const FaceOf &fo, int t,
                                      const T h0[3], bool write, S *const Hout[3], bool &ok)
{
    const Q4<T> cs = q4_load(b.cst + t);
    const int d = fo.d;
    T h[3];
    h_vector_rt(g, b, Hprev, Hprev, 1, fo, h, T(1));
    const Q4<T> mq = sm.mn[s], bq = sm.bc[s], pq = sm.dm[s];
    const V3<T> he = {h0[0] + h[0], h0[1] + h[1], h0[2] + h[2]};
    const Q4<T> r = llg_solve_rt(V3<T>{mq.x, mq.y, mq.z}, V3<T>{bq.x, bq.y, bq.z}, he, cs.y, cs.z, cs.x, mq.w, d);
    const bool wall = wall_node(g, d, d == 0 ? fo.i : d == 1 ? fo.j : fo.k);
    const T hv = wall ? T(0) : bq.w - r.w;
    pick_ptr(Hcur, d)[fo.l] = hv;
    sm.dm[s] = q4(r.x, r.y, r.z, T(0));
    if (write) ok &= res_store(g, f, b, Hout, fo, t, hv, mq, q4(r.x, r.y, r.z, T(0)));
    return max(abs(r.x - pq.x), max(abs(r.y - pq.y), abs(r.z - pq.z))) * cs.w;
}

// Phase 0 on a non-magnetic face of run-time family d: its final H in both
// iterate buffers.
template <typename T, typename S>
__device__ __forceinline__ T res_non_first(const Geo &g, const Fields<T, S> &f, S *const Hin[3], T *const Hp[3],
                                           T *const W0[3], T *const W1[3], const FaceOf &fo, bool second)
{
    const int d = fo.d;
    const T hn = second ? pick_ptr(Hp, d)[fo.l] : ld_s(pick_ptr(Hin, d) + gidx32(g, fo.i, fo.j, fo.k), f.sH);
    const T v = h_face_nonmag_val(g, f, d, fo.i, fo.j, fo.k, hn);
    pick_ptr(W0, d)[fo.l] = v;
    pick_ptr(W1, d)[fo.l] = v;
    return v;
}

// When the half step writes back: H^r and M^(n+1/2,r) of one magnetic face
// into Hout and its global record after every iterate r (the last write
// stands, so no separate write-back phase is needed; the kernel reads M^n
// from shared memory, never from the global record).  Returns false if a
// value is not finite.
template <typename T, typename S>
__device__ __forceinline__ bool res_store(const Geo &g, const Fields<T, S> &f, const Box<T> &b, S *const Hout[3],
                                          const FaceOf &fo, int t, T h, const Q4<T> &mq, const Q4<T> &dq)
{
    st_s(pick_ptr(Hout, fo.d) + gidx32(g, fo.i, fo.j, fo.k), h, f.isH);
    const T m0 = mq.x + dq.x, m1 = mq.y + dq.y, m2 = mq.z + dq.z;
    b.mn[t] = q4(m0, m1, m2, T(0));
    return isfinite(h) && isfinite(m0) && isfinite(m1) && isfinite(m2);
}

// One H/M half step with the records in shared memory (the counterpart of
// hm_half_step; the same phases, votes and iteration log).  Magnetic face
// slot s = f 256 + threadIdx.x of this block is list position
// (blockIdx.x F + f) 256 + threadIdx.x.  second / write as SECOND / WRITE of
// hm_half_step, at run time: one copy of the code serves all three half
// steps of the launches, which keeps the kernel's instruction footprint
// small.  Returns the final iterate parity, or -1 if a barrier timed out.
template <int F, int ORD, typename T, typename S>
__device__ MMX_RES_FN int hm_half_step_res(const Geo &g, const Fields<T, S> &f, const Box<T> &b, S *const Hin[3],
                                             S *const Hout[3], int fprev, unsigned long long *res,
                                             const ResSmem<T> sm, bool second, bool write)
{
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int tb = blockIdx.x * F * kResThreads + threadIdx.x;
    const T h0[3] = {(T)b.h0[0], (T)b.h0[1], (T)b.h0[2]};
    const int hs = second ? 1 : 0;
    T *const W0[3] = {hs ? b.Hit2[0][0] : b.Hit[0][0], hs ? b.Hit2[0][1] : b.Hit[0][1],
                      hs ? b.Hit2[0][2] : b.Hit[0][2]};
    T *const W1[3] = {hs ? b.Hit2[1][0] : b.Hit[1][0], hs ? b.Hit2[1][1] : b.Hit[1][1],
                      hs ? b.Hit2[1][2] : b.Hit[1][2]};
    T *const Hp[3] = {b.Hit[fprev & 1][0], b.Hit[fprev & 1][1], b.Hit[fprev & 1][2]};

    // Writing back into another buffer than the one read (the fused path's
    // ping-pong), every iterate's H and M go to Hout and the global records
    // at once and the last write stands: no write-back phase.  In place
    // (Hout = Hin) that would race with other blocks still reading H^n, so
    // the final iterate is written after the last barrier instead.
    const bool spec = write && (const void *)Hout[0] != (const void *)Hin[0];
    // ---- phase 0: r = 1 (a non-magnetic face has its final H here)
    bool ok = true;
    for (int t = t0; t < b.nnon; t += stride) {
        const FaceOf fo = face_of(b.nonmag[t]);
        const T v = res_non_first(g, f, Hin, Hp, W0, W1, fo, second);
        if (spec) {
            st_s(pick_ptr(Hout, fo.d) + gidx32(g, fo.i, fo.j, fo.k), v, f.isH);
            ok &= isfinite(v);
        }
    }
    T rmax = T(0);
#pragma unroll 1
    for (int q = 0; q < F; q++) {
        const int t = tb + q * kResThreads, s = q * kResThreads + threadIdx.x;
        if (t >= b.nmag) break;
        rmax = max(rmax, res_first<ORD>(g, f, b, Hin, Hp, W1, sm, s, face_of(sm.ent[s]), t, h0, second, spec, Hout,
                                        ok));
    }
    rmax = block_max(rmax);
    publish_residual(&res[1], rmax);
    unsigned long long *const vote = res + kVoteRows * (kMaxIter + 1);
    const int v1 = grid_vote(&vote[1], rmax > T(0) && !((double)rmax < b.tol), b.err);
    if (v1 < 0) return -1;

    int r = 1;
    bool conv = v1 == 1 || ORD == 1;
    while (!conv && r < b.max_iter) {
        r++;
        const int pr = (r - 1) & 1, cr = r & 1;
        T *const Hprev[3] = {pr ? W1[0] : W0[0], pr ? W1[1] : W0[1], pr ? W1[2] : W0[2]};
        T *const Hcur[3] = {cr ? W1[0] : W0[0], cr ? W1[1] : W0[1], cr ? W1[2] : W0[2]};
        rmax = T(0);
#pragma unroll 1
        for (int q = 0; q < F; q++) {
            const int t = tb + q * kResThreads, s = q * kResThreads + threadIdx.x;
            if (t >= b.nmag) break;
            rmax = max(rmax, res_next(g, f, b, Hprev, Hcur, sm, s, face_of(sm.ent[s]), t, h0, spec, Hout, ok));
        }
        rmax = block_max(rmax);
        publish_residual(&res[r], rmax);
        const int vr = grid_vote(&vote[r], rmax > T(0) && !((double)rmax < b.tol), b.err);
        if (vr < 0) return -1;
        conv = vr == 1;
    }

    const int fr = r & 1;
    if (write && !spec) {
        // ---- write back H (all box faces) and M^(n+1/2) (global records)
        T *const Hfin[3] = {fr ? W1[0] : W0[0], fr ? W1[1] : W0[1], fr ? W1[2] : W0[2]};
        for (int t = t0; t < b.nnon; t += stride) {
            const FaceOf fo = face_of(b.nonmag[t]);
            const T v = pick_ptr(Hfin, fo.d)[fo.l];
            st_s(pick_ptr(Hout, fo.d) + gidx32(g, fo.i, fo.j, fo.k), v, f.isH);
            ok &= isfinite(v);
        }
#pragma unroll 1
        for (int q = 0; q < F; q++) {
            const int t = tb + q * kResThreads, s = q * kResThreads + threadIdx.x;
            if (t >= b.nmag) break;
            const FaceOf fo = face_of(sm.ent[s]);
            ok &= res_store(g, f, b, Hout, fo, t, pick_ptr(Hfin, fo.d)[fo.l], sm.mn[s], sm.dm[s]);
        }
    }
    // with spec the last iterate's H and M are already in Hout and the records
    if (write && !ok) atomicOr(b.err, kErrNonFinite);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (!conv && ORD == 2) atomicOr(b.err, kErrNotConverged);
        unsigned long long n = *b.halfsteps;
        b.iterlog[n % kIterLogCap] = r;
        *b.halfsteps = n + 1;
        *b.last_res = ORD == 2 ? __longlong_as_double((long long)res[r]) : 0.0;
    }
    return fr;
}

// Cooperative launch over the magnetic box with the records in shared memory
// (F faces per thread, res_smem_bytes<T>(F) bytes of dynamic shared memory
// per block); nsub and slot as for k_hm_box.  Requires gridDim.x F 256 >=
// nmag.
template <typename T, typename S, int F, int ORD>
__global__ void __launch_bounds__(kResThreads, MMX_RES_MINB)
    k_hm_box_res(const __grid_constant__ Geo g, const __grid_constant__ Fields<T, S> f,
                 const __grid_constant__ Box<T> b, const __grid_constant__ Ptr3<S> Hout, int nsub, int slot)
{
    const int W = kMaxIter + 1;
    if (timeout_latched(b.err)) return;   // see k_hm_box
    if (blockIdx.x == 0) {
        unsigned long long *other = b.res + 2 * (1 - slot) * W;
        for (int r = threadIdx.x; r < 2 * W; r += blockDim.x) {
            other[r] = 0ull;
            other[kVoteRows * W + r] = 0ull;
        }
    }
    const ResSmem<T> sm = res_smem<T>(F);
    const int tb = blockIdx.x * F * kResThreads + threadIdx.x;
#pragma unroll
    for (int q = 0; q < F; q++) {
        const int t = tb + q * kResThreads, s = q * kResThreads + threadIdx.x;
        if (t < b.nmag) {
            sm.ent[s] = b.mag[t];
            sm.mn[s] = q4_load(b.mn + t);
        }
    }
    // each thread reads back only its own slots: no block barrier needed.
    // nsub = 2: the first half step keeps its result in the iterate buffers
    // and shared memory, the second starts from there and writes back.
    const int fr = hm_half_step_res<F, ORD>(g, f, b, f.H, Hout.p, 0, b.res + 2 * slot * W, sm, false, nsub != 2);
    if (fr < 0 || nsub != 2) return;
    hm_half_step_res<F, ORD>(g, f, b, f.H, Hout.p, fr, b.res + (2 * slot + 1) * W, sm, true, true);
}

} // namespace mmx

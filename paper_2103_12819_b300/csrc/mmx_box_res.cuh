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
constexpr int kResMaxF = 2;

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

// Phase 0 on one magnetic face of family D (list position t, slot s): C' =
// H^n - dt/(2 mu0) curl E, beta = -kappa M^n x H_eff^n, e0 and the first
// iterate (or the first-order update); H^1 into Hw.  SECOND: H^n from the
// previous half step's iterate buffer Hp, M^n = M^n + DeltaM of that half step
// (updated in place), and the curl sum stored by the first half step.
template <int D, bool SECOND, typename T, typename S>
__device__ __forceinline__ T res_first(const Geo &g, const Fields<T, S> &f, const Box<T> &b, S *const Hin[3],
                                       T *const Hp[3], T *const Hw[3], const ResSmem<T> &sm, int s,
                                       const FaceOf &fo, int t, const T h0[3])
{
    const Q4<T> cs = q4_load(b.cst + t);
    T Mn[3], hn, csum, h[3];
    Q4<T> m0 = sm.mn[s];
    if (SECOND) {
        const Q4<T> d0 = sm.dm[s];
        Mn[0] = m0.x + d0.x;
        Mn[1] = m0.y + d0.y;
        Mn[2] = m0.z + d0.z;
        hn = Hp[D][fo.l];
        csum = sm.curl[s];
        h_vector<D>(g, b, Hin, Hp, 1, fo.i, fo.j, fo.k, h);
    } else {
        Mn[0] = m0.x;
        Mn[1] = m0.y;
        Mn[2] = m0.z;
        const unsigned q = gidx32(g, fo.i, fo.j, fo.k);
        T rest, zp;
        curl_e32(g, f.E, f.inv_d, D, q, rest, zp, f.sE);
        csum = rest + zp;
        sm.curl[s] = csum;
        hn = ld_s(Hin[D] + q, f.sH);
        h_vector<D>(g, b, Hin, Hp, 0, fo.i, fo.j, fo.k, h, f.sH);
    }
    const T Ms = cs.x, k1 = cs.y, k2 = cs.z;
    const T cp = hn - b.cfar * csum;
    const T e0 = norm_defect(Ms, Mn[0], Mn[1], Mn[2]);
    T heff[3];
#pragma unroll
    for (int c = 0; c < 3; c++) heff[c] = h0[c] + h[c];
    T dM[3], dMh;
    T beta[3] = {T(0), T(0), T(0)};
    if (b.order == 2) {
        beta[0] = -k1 * (Mn[1] * heff[2] - Mn[2] * heff[1]);
        beta[1] = -k1 * (Mn[2] * heff[0] - Mn[0] * heff[2]);
        beta[2] = -k1 * (Mn[0] * heff[1] - Mn[1] * heff[0]);
        llg_iterate(Mn, beta, heff, k1, k2, Ms, e0, D, dM, dMh);
    } else {
        llg_euler(Mn, heff, k1, k2, Ms, e0, D, dM, dMh);
    }
    sm.bc[s] = q4(beta[0], beta[1], beta[2], cp);
    sm.mn[s] = q4(Mn[0], Mn[1], Mn[2], e0);
    sm.dm[s] = q4(dM[0], dM[1], dM[2], T(0));
    const bool wall = wall_node(g, D, D == 0 ? fo.i : D == 1 ? fo.j : fo.k);
    Hw[D][fo.l] = wall ? T(0) : cp - dMh;
    return max(abs(dM[0]), max(abs(dM[1]), abs(dM[2]))) * cs.w;
}

// Iterate r >= 2 on one magnetic face from the neighbours' iterate r-1 in
// Hprev: DeltaM^r replaces DeltaM^(r-1) in shared memory, H^r into Hcur.
// Returns max_c |DeltaM^r_c - DeltaM^(r-1)_c| / Ms.
template <int D, typename T>
__device__ __forceinline__ T res_next(const Geo &g, const Box<T> &b, T *const Hprev[3], T *const Hcur[3],
                                      const ResSmem<T> &sm, int s, const FaceOf &fo, int t, const T h0[3])
{
    const Q4<T> cs = q4_load(b.cst + t);
    T h[3];
    h_vector<D>(g, b, Hprev, Hprev, 1, fo.i, fo.j, fo.k, h);
    const Q4<T> mq = sm.mn[s], bq = sm.bc[s], pq = sm.dm[s];
    const T Mn[3] = {mq.x, mq.y, mq.z};
    const T beta[3] = {bq.x, bq.y, bq.z};
    T heff[3];
#pragma unroll
    for (int c = 0; c < 3; c++) heff[c] = h0[c] + h[c];
    T dM[3], dMh;
    llg_iterate(Mn, beta, heff, cs.y, cs.z, cs.x, mq.w, D, dM, dMh);
    const bool wall = wall_node(g, D, D == 0 ? fo.i : D == 1 ? fo.j : fo.k);
    Hcur[D][fo.l] = wall ? T(0) : bq.w - dMh;
    sm.dm[s] = q4(dM[0], dM[1], dM[2], T(0));
    return max(abs(dM[0] - pq.x), max(abs(dM[1] - pq.y), abs(dM[2] - pq.z))) * cs.w;
}

// One H/M half step with the records in shared memory (the counterpart of
// hm_half_step; the same phases, votes and iteration log).  Magnetic face
// slot s = f 256 + threadIdx.x of this block is list position
// (blockIdx.x F + f) 256 + threadIdx.x.  Returns the final iterate parity,
// or -1 if a barrier timed out.
template <bool SECOND, bool WRITE, int F, typename T, typename S>
__device__ int hm_half_step_res(const Geo &g, const Fields<T, S> &f, const Box<T> &b, S *const Hin[3],
                                S *const Hout[3], int fprev, unsigned long long *res, const ResSmem<T> &sm)
{
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int tb = blockIdx.x * F * kResThreads + threadIdx.x;
    const T h0[3] = {(T)b.h0[0], (T)b.h0[1], (T)b.h0[2]};
    T *const W0[3] = {SECOND ? b.Hit2[0][0] : b.Hit[0][0], SECOND ? b.Hit2[0][1] : b.Hit[0][1],
                      SECOND ? b.Hit2[0][2] : b.Hit[0][2]};
    T *const W1[3] = {SECOND ? b.Hit2[1][0] : b.Hit[1][0], SECOND ? b.Hit2[1][1] : b.Hit[1][1],
                      SECOND ? b.Hit2[1][2] : b.Hit[1][2]};
    T *const Hp[3] = {b.Hit[fprev & 1][0], b.Hit[fprev & 1][1], b.Hit[fprev & 1][2]};

    // ---- phase 0: r = 1
    for (int t = t0; t < b.nnon; t += stride) {
        const FaceOf fo = face_of(b.nonmag[t]);
        if (fo.d == 0)
            non_first<0, SECOND>(g, f, Hin, Hp, W0, W1, fo);
        else if (fo.d == 1)
            non_first<1, SECOND>(g, f, Hin, Hp, W0, W1, fo);
        else
            non_first<2, SECOND>(g, f, Hin, Hp, W0, W1, fo);
    }
    T rmax = T(0);
#pragma unroll
    for (int q = 0; q < F; q++) {
        const int t = tb + q * kResThreads, s = q * kResThreads + threadIdx.x;
        if (t >= b.nmag) break;
        const FaceOf fo = face_of(sm.ent[s]);
        T rv;
        if (fo.d == 0)
            rv = res_first<0, SECOND>(g, f, b, Hin, Hp, W1, sm, s, fo, t, h0);
        else if (fo.d == 1)
            rv = res_first<1, SECOND>(g, f, b, Hin, Hp, W1, sm, s, fo, t, h0);
        else
            rv = res_first<2, SECOND>(g, f, b, Hin, Hp, W1, sm, s, fo, t, h0);
        rmax = max(rmax, rv);
    }
    rmax = block_max(rmax);
    publish_residual(&res[1], rmax);
    unsigned long long *const vote = res + kVoteRows * (kMaxIter + 1);
    const int v1 = grid_vote(&vote[1], rmax > T(0) && !((double)rmax < b.tol), b.err);
    if (v1 < 0) return -1;

    int r = 1;
    bool conv = v1 == 1 || b.order == 1;
    while (!conv && r < b.max_iter) {
        r++;
        const int pr = (r - 1) & 1, cr = r & 1;
        T *const Hprev[3] = {pr ? W1[0] : W0[0], pr ? W1[1] : W0[1], pr ? W1[2] : W0[2]};
        T *const Hcur[3] = {cr ? W1[0] : W0[0], cr ? W1[1] : W0[1], cr ? W1[2] : W0[2]};
        rmax = T(0);
#pragma unroll
        for (int q = 0; q < F; q++) {
            const int t = tb + q * kResThreads, s = q * kResThreads + threadIdx.x;
            if (t >= b.nmag) break;
            const FaceOf fo = face_of(sm.ent[s]);
            T rv;
            if (fo.d == 0)
                rv = res_next<0>(g, b, Hprev, Hcur, sm, s, fo, t, h0);
            else if (fo.d == 1)
                rv = res_next<1>(g, b, Hprev, Hcur, sm, s, fo, t, h0);
            else
                rv = res_next<2>(g, b, Hprev, Hcur, sm, s, fo, t, h0);
            rmax = max(rmax, rv);
        }
        rmax = block_max(rmax);
        publish_residual(&res[r], rmax);
        const int vr = grid_vote(&vote[r], rmax > T(0) && !((double)rmax < b.tol), b.err);
        if (vr < 0) return -1;
        conv = vr == 1;
    }

    const int fr = r & 1;
    if (WRITE) {
        // ---- write back H (all box faces) and M^(n+1/2) (global records)
        T *const Hfin[3] = {fr ? W1[0] : W0[0], fr ? W1[1] : W0[1], fr ? W1[2] : W0[2]};
        bool ok = true;
        for (int t = t0; t < b.nnon; t += stride) {
            const FaceOf fo = face_of(b.nonmag[t]);
            const T v = Hfin[fo.d][fo.l];
            S *const Ho = fo.d == 0 ? Hout[0] : fo.d == 1 ? Hout[1] : Hout[2];
            st_s(Ho + gidx32(g, fo.i, fo.j, fo.k), v, f.isH);
            ok &= isfinite(v);
        }
#pragma unroll
        for (int q = 0; q < F; q++) {
            const int t = tb + q * kResThreads, s = q * kResThreads + threadIdx.x;
            if (t >= b.nmag) break;
            const FaceOf fo = face_of(sm.ent[s]);
            const T v = Hfin[fo.d][fo.l];
            S *const Ho = fo.d == 0 ? Hout[0] : fo.d == 1 ? Hout[1] : Hout[2];
            st_s(Ho + gidx32(g, fo.i, fo.j, fo.k), v, f.isH);
            const Q4<T> mq = sm.mn[s], dq = sm.dm[s];
            const T m0 = mq.x + dq.x, m1 = mq.y + dq.y, m2 = mq.z + dq.z;
            b.mn[t] = q4(m0, m1, m2, T(0));
            ok &= isfinite(v) && isfinite(m0) && isfinite(m1) && isfinite(m2);
        }
        if (!ok) atomicOr(b.err, kErrNonFinite);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (!conv && b.order == 2) atomicOr(b.err, kErrNotConverged);
        unsigned long long hs = *b.halfsteps;
        b.iterlog[hs % kIterLogCap] = r;
        *b.halfsteps = hs + 1;
        *b.last_res = b.order == 2 ? __longlong_as_double((long long)res[r]) : 0.0;
    }
    return fr;
}

// Cooperative launch over the magnetic box with the records in shared memory
// (F faces per thread, res_smem_bytes<T>(F) bytes of dynamic shared memory
// per block); nsub and slot as for k_hm_box.  Requires gridDim.x F 256 >=
// nmag.
template <typename T, typename S, int F>
__global__ void __launch_bounds__(kResThreads, BoxMinBlocks<T>::value)
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
    // each thread reads back only its own slots: no block barrier needed
    if (nsub == 2) {
        const int fr = hm_half_step_res<false, false, F>(g, f, b, f.H, Hout.p, 0, b.res + 2 * slot * W, sm);
        if (fr < 0) return;
        hm_half_step_res<true, true, F>(g, f, b, f.H, Hout.p, fr, b.res + (2 * slot + 1) * W, sm);
    } else {
        hm_half_step_res<false, true, F>(g, f, b, f.H, Hout.p, 0, b.res + 2 * slot * W, sm);
    }
}

} // namespace mmx

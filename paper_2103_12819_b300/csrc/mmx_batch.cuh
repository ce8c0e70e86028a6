// mmx_batch.cuh -- the H/M half steps of many independent grids (instances)
// in one cooperative launch, for the batched path (e.g. a bias sweep of
// small devices).  The magnetic and non-magnetic box faces of all instances
// are concatenated into two lists, each entry tagged with its instance; the
// same thread takes the same faces in every phase.  Every instance keeps its
// own residual (Sec. 3.2.2: max over its magnetic faces of
// |DeltaM^r - DeltaM^(r-1)|/Ms) and stops at its own first r with residual
// < tol; the launch iterates while any instance is still active, and an
// instance that has stopped does no further work.  Residuals are reduced per
// block in shared memory (one atomicMax per instance per block, on the FP64
// bit pattern) and meet at the bounded grid barrier.
#pragma once
#include "mmx_kernels.cuh"

namespace mmx {

// One instance of a batch, for one parity of the E/H ping-pong.
template <typename T, typename S> struct BoxInst {
    Geo g;
    Fields<T, S> f;     // E^(n+1) and H^(n+1/2) of the instance
    Box<T> b;
    Ptr3<S> Hout;       // where H^(n+3/2) (or H^(n+1)) goes
    int base_mag;       // first entry of the instance in the magnetic list
};

// The batched magnetic-face list packs each entry and its instance q into
// 8 bytes, d << 62 | q << 48 | i << 32 | j << 16 | k (q below 2^14, every
// index below 2^16), against 20 bytes for the single-instance entry
// {l | d << 30, i, j, k} and a separate instance index; the box index l
// comes back from i, j, k and the instance's box with multiply-adds, so the
// neighbour addresses (from i, j, k) wait on no load of the instance.
__global__ void k_pack_faces(const int4 *__restrict__ in, unsigned long long *__restrict__ out, int n, int q)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int4 e = in[t];
    out[t] = (unsigned long long)((unsigned)e.x >> 30) << 62 | (unsigned long long)(unsigned)q << 48 |
             (unsigned long long)(unsigned)e.y << 32 | (unsigned long long)(unsigned)e.z << 16 |
             (unsigned long long)(unsigned)e.w;
}

__device__ __forceinline__ int inst_of64(unsigned long long e)
{
    return (int)((e >> 48) & 0x3fffu);
}

template <typename T> __device__ __forceinline__ FaceOf face_of64(unsigned long long e, const Box<T> &b)
{
    FaceOf fo;
    fo.d = (int)(e >> 62);
    fo.i = (int)((e >> 32) & 0xffffu);
    fo.j = (int)((e >> 16) & 0xffffu);
    fo.k = (int)(e & 0xffffu);
    fo.l = (unsigned)(fo.i - b.lo[0]) +
           (unsigned)b.bx * ((unsigned)(fo.j - b.lo[1]) + (unsigned)b.by * (unsigned)(fo.k - b.lo[2]));
    return fo;
}

// Per-block state of a batched half step, in dynamic shared memory.
struct BatchShared {
    unsigned long long *res;   // [ninst] block partial residuals (bit patterns)
    int *done;                 // [ninst] iteration the instance stopped at (0: active)
    int *fprev;                // [ninst] iterate the previous half step stopped at
};

__device__ __forceinline__ void batch_publish(const BatchShared &sh, int ninst, unsigned long long *res, int r,
                                              int stride_inst)
{
    __syncthreads();
    for (int q = threadIdx.x; q < ninst; q += blockDim.x) {
        const unsigned long long v = sh.res[q];
        if (v) atomicMax(&res[(size_t)q * stride_inst + r], v);
        sh.res[q] = 0ull;
    }
}

// After the barrier of iteration r: every block marks the instances that
// stop at r (residual below tol, or max_iter reached); returns whether any
// instance goes on.
template <typename T, typename S>
__device__ __forceinline__ bool batch_update(const BatchShared &sh, const BoxInst<T, S> *inst, int ninst,
                                             const unsigned long long *res, int r, int stride_inst)
{
    int any = 0;
    for (int q = threadIdx.x; q < ninst; q += blockDim.x) {
        if (sh.done[q]) continue;
        const Box<T> &b = inst[q].b;
        const double v = __longlong_as_double((long long)*(volatile const unsigned long long *)&res[
            (size_t)q * stride_inst + r]);
        if (b.order == 1 || v < b.tol || r >= b.max_iter)
            sh.done[q] = r;
        else
            any = 1;
    }
    return __syncthreads_or(any) != 0;
}

// ORD: the scheme order of every instance (2 or 1), or 0 when they differ.
template <bool SECOND, bool WRITE, int ORD, typename T, typename S>
__device__ bool hm_half_step_batch(const BoxInst<T, S> *inst, int ninst, const unsigned long long *mag,
                                   int nmag, const int4 *non, const int *non_inst, int nnon,
                                   unsigned long long *res, unsigned long long *bar, int *berr,
                                   const BatchShared &sh)
{
    constexpr int W = kMaxIter + 1;
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (int q = threadIdx.x; q < ninst; q += blockDim.x) {
        sh.res[q] = 0ull;
        sh.done[q] = 0;
    }
    __syncthreads();

    // ---- phase 0: r = 1
    for (int t = t0; t < nnon; t += stride) {
        const int qi = non_inst[t];
        const BoxInst<T, S> &I = inst[qi];
        const int fp = sh.fprev[qi] & 1;
        T *const W0[3] = {SECOND ? I.b.Hit2[0][0] : I.b.Hit[0][0], SECOND ? I.b.Hit2[0][1] : I.b.Hit[0][1],
                          SECOND ? I.b.Hit2[0][2] : I.b.Hit[0][2]};
        T *const W1[3] = {SECOND ? I.b.Hit2[1][0] : I.b.Hit[1][0], SECOND ? I.b.Hit2[1][1] : I.b.Hit[1][1],
                          SECOND ? I.b.Hit2[1][2] : I.b.Hit[1][2]};
        T *const Hp[3] = {I.b.Hit[fp][0], I.b.Hit[fp][1], I.b.Hit[fp][2]};
        S *const Hin[3] = {I.f.H[0], I.f.H[1], I.f.H[2]};
        const FaceOf fo = face_of(non[t]);
        if (fo.d == 0)
            non_first<0, SECOND>(I.g, I.f, Hin, Hp, W0, W1, fo);
        else if (fo.d == 1)
            non_first<1, SECOND>(I.g, I.f, Hin, Hp, W0, W1, fo);
        else
            non_first<2, SECOND>(I.g, I.f, Hin, Hp, W0, W1, fo);
    }
    for (int t = t0; t < nmag; t += stride) {
        const unsigned long long e = mag[t];
        const int qi = inst_of64(e);
        const BoxInst<T, S> &I = inst[qi];
        const int tl = t - I.base_mag;
        const int fp = sh.fprev[qi] & 1;
        T *const W1[3] = {SECOND ? I.b.Hit2[1][0] : I.b.Hit[1][0], SECOND ? I.b.Hit2[1][1] : I.b.Hit[1][1],
                          SECOND ? I.b.Hit2[1][2] : I.b.Hit[1][2]};
        T *const Hp[3] = {I.b.Hit[fp][0], I.b.Hit[fp][1], I.b.Hit[fp][2]};
        S *const Hin[3] = {I.f.H[0], I.f.H[1], I.f.H[2]};
        const T h0[3] = {(T)I.b.h0[0], (T)I.b.h0[1], (T)I.b.h0[2]};
        const FaceOf fo = face_of64(e, I.b);
        FirstIn<T> in;
        T rv;
        if (fo.d == 0) {
            first_load<0, SECOND>(I.g, I.f, I.b, Hin, Hp, I.b.dm[fp], fo, tl, in);
            rv = first_finish<0, SECOND, ORD>(I.g, I.b, W1, fo, tl, in, h0, sh.fprev[qi] > 1);
        } else if (fo.d == 1) {
            first_load<1, SECOND>(I.g, I.f, I.b, Hin, Hp, I.b.dm[fp], fo, tl, in);
            rv = first_finish<1, SECOND, ORD>(I.g, I.b, W1, fo, tl, in, h0, sh.fprev[qi] > 1);
        } else {
            first_load<2, SECOND>(I.g, I.f, I.b, Hin, Hp, I.b.dm[fp], fo, tl, in);
            rv = first_finish<2, SECOND, ORD>(I.g, I.b, W1, fo, tl, in, h0, sh.fprev[qi] > 1);
        }
        if (rv > T(0)) atomicMax(&sh.res[qi], (unsigned long long)__double_as_longlong((double)rv));
    }
    batch_publish(sh, ninst, res, 1, W);
    if (!grid_barrier(bar, berr)) return false;
    int r = 1;
    bool more = batch_update(sh, inst, ninst, res, 1, W);
    while (more && r < kMaxIter) {
        r++;
        const int pr = (r - 1) & 1, cr = r & 1;
        // one copy of the sweep per source of beta and C' (RecomputeBC), each
        // register-allocated on its own: the record, or at iterate 2 of an
        // instance whose phase 0 stored none, beta and C' formed again
        auto sweep = [&](auto have) {
            constexpr bool HB = decltype(have)::value;
            for (int t = t0; t < nmag; t += stride) {
                const unsigned long long e = mag[t];
                const int qi = inst_of64(e);
                if (sh.done[qi]) continue;
                if (RecomputeBC<T>::value && (sh.fprev[qi] > 1 || r > 2) != HB) continue;
                const BoxInst<T, S> &I = inst[qi];
                const int tl = t - I.base_mag;
                T *const Wp[3] = {SECOND ? I.b.Hit2[pr][0] : I.b.Hit[pr][0], SECOND ? I.b.Hit2[pr][1] : I.b.Hit[pr][1],
                                  SECOND ? I.b.Hit2[pr][2] : I.b.Hit[pr][2]};
                T *const Wc[3] = {SECOND ? I.b.Hit2[cr][0] : I.b.Hit[cr][0], SECOND ? I.b.Hit2[cr][1] : I.b.Hit[cr][1],
                                  SECOND ? I.b.Hit2[cr][2] : I.b.Hit[cr][2]};
                const T h0[3] = {(T)I.b.h0[0], (T)I.b.h0[1], (T)I.b.h0[2]};
                const int fp = sh.fprev[qi] & 1;
                T *const Hp[3] = {I.b.Hit[fp][0], I.b.Hit[fp][1], I.b.Hit[fp][2]};
                S *const Hin[3] = {I.f.H[0], I.f.H[1], I.f.H[2]};
                const FaceOf fo = face_of64(e, I.b);
                NextIn<T> in;
                T rv;
                if (fo.d == 0) {
                    next_load<0, SECOND, HB>(I.g, I.b, fo, tl, Wp, pr, in, &I.f, Hin, Hp);
                    rv = next_finish<0, HB>(I.g, I.b, fo, tl, Wc, cr, in, h0);
                } else if (fo.d == 1) {
                    next_load<1, SECOND, HB>(I.g, I.b, fo, tl, Wp, pr, in, &I.f, Hin, Hp);
                    rv = next_finish<1, HB>(I.g, I.b, fo, tl, Wc, cr, in, h0);
                } else {
                    next_load<2, SECOND, HB>(I.g, I.b, fo, tl, Wp, pr, in, &I.f, Hin, Hp);
                    rv = next_finish<2, HB>(I.g, I.b, fo, tl, Wc, cr, in, h0);
                }
                if (rv > T(0)) atomicMax(&sh.res[qi], (unsigned long long)__double_as_longlong((double)rv));
            }
        };
        sweep(std::true_type{});
        if (RecomputeBC<T>::value && r == 2) {
            // the second copy only where an active instance has no record
            int rc = 0;
            for (int q = threadIdx.x; q < ninst; q += blockDim.x)
                if (!sh.done[q] && sh.fprev[q] <= 1) rc = 1;
            if (__syncthreads_or(rc)) sweep(std::false_type{});
        }
        batch_publish(sh, ninst, res, r, W);
        if (!grid_barrier(bar, berr)) return false;
        more = batch_update(sh, inst, ninst, res, r, W);
    }

    if (WRITE) {
        // ---- write back H (all box faces) and M (face records), each
        // instance from the iterate it stopped at
        bool ok = true;
        for (int t = t0; t < nnon; t += stride) {
            const int qi = non_inst[t];
            const BoxInst<T, S> &I = inst[qi];
            const int fr = sh.done[qi] & 1;
            const FaceOf fo = face_of(non[t]);
            T *const *Wf = SECOND ? I.b.Hit2[fr] : I.b.Hit[fr];
            const T v = Wf[fo.d][fo.l];
            S *const Ho = fo.d == 0 ? I.Hout.p[0] : fo.d == 1 ? I.Hout.p[1] : I.Hout.p[2];
            st_s(Ho + gidx32(I.g, fo.i, fo.j, fo.k), v, I.f.isH);
            ok &= isfinite(v);
        }
        for (int t = t0; t < nmag; t += stride) {
            const unsigned long long e = mag[t];
            const int qi = inst_of64(e);
            const BoxInst<T, S> &I = inst[qi];
            const int tl = t - I.base_mag;
            const int fr = sh.done[qi] & 1;
            T *const Hfin[3] = {SECOND ? I.b.Hit2[fr][0] : I.b.Hit[fr][0], SECOND ? I.b.Hit2[fr][1] : I.b.Hit[fr][1],
                                SECOND ? I.b.Hit2[fr][2] : I.b.Hit[fr][2]};
            S *const Ho[3] = {I.Hout.p[0], I.Hout.p[1], I.Hout.p[2]};
            const FaceOf fo = face_of64(e, I.b);
            ok &= fo.d == 0   ? mag_store<0>(I.g, I.b, fo, tl, Hfin, Ho, fr, I.f.isH)
                  : fo.d == 1 ? mag_store<1>(I.g, I.b, fo, tl, Hfin, Ho, fr, I.f.isH)
                              : mag_store<2>(I.g, I.b, fo, tl, Hfin, Ho, fr, I.f.isH);
        }
        if (!ok) atomicOr(berr, kErrNonFinite);
    }
    // per-instance iteration log, status and last residual
    if (blockIdx.x == 0)
        for (int q = threadIdx.x; q < ninst; q += blockDim.x) {
            const Box<T> &b = inst[q].b;
            const int rq = sh.done[q] ? sh.done[q] : r;
            const double v = __longlong_as_double((long long)res[(size_t)q * W + rq]);
            if (b.order == 2 && !(v < b.tol)) atomicOr(b.err, kErrNotConverged);
            unsigned long long hs = *b.halfsteps;
            b.iterlog[hs % kIterLogCap] = rq;
            *b.halfsteps = hs + 1;
            *b.last_res = b.order == 2 ? v : 0.0;
        }
    __syncthreads();
    for (int q = threadIdx.x; q < ninst; q += blockDim.x) sh.fprev[q] = sh.done[q] ? sh.done[q] : r;
    __syncthreads();
    return true;
}

// nsub H/M half steps of every instance with one E.  res holds, for launch
// parity `slot`, rows [2 slot + h][instance][kMaxIter + 1] (h = half step);
// the other parity's rows are cleared here for the next launch.
template <typename T, typename S = T, int ORD = 0>
__global__ void __launch_bounds__(256, BoxMinBlocks<T>::value)
    k_hm_box_batch(const BoxInst<T, S> *__restrict__ inst, int ninst, const unsigned long long *__restrict__ mag,
                   int nmag, const int4 *__restrict__ non,
                   const int *__restrict__ non_inst, int nnon, unsigned long long *res, unsigned long long *bar,
                   int *berr, int nsub, int slot)
{
    if (timeout_latched(berr)) return;   // see k_hm_box
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BatchShared sh;
    sh.res = reinterpret_cast<unsigned long long *>(smem_raw);
    sh.done = reinterpret_cast<int *>(sh.res + ninst);
    sh.fprev = sh.done + ninst;
    const size_t rows = (size_t)ninst * (kMaxIter + 1);
    if (blockIdx.x == 0) {
        unsigned long long *other = res + 2 * (1 - slot) * rows;
        for (size_t q = threadIdx.x; q < 2 * rows; q += blockDim.x) other[q] = 0ull;
    }
    // each instance's last logged iterate count (2 when none is): read
    // before block 0 logs this launch's first half step, which it does only
    // after that half step's grid barriers, which every block joins after
    // this
    for (int q = threadIdx.x; q < ninst; q += blockDim.x) {
        const Box<T> &bq = inst[q].b;
        const unsigned long long hs = *bq.halfsteps;
        sh.fprev[q] = hs == 0 ? 2 : bq.iterlog[(hs - 1) % kIterLogCap];
    }
    __syncthreads();
    unsigned long long *r0 = res + 2 * slot * rows;
    if (nsub == 2) {
        if (!hm_half_step_batch<false, false, ORD>(inst, ninst, mag, nmag, non, non_inst, nnon, r0, bar, berr,
                                              sh))
            return;
        hm_half_step_batch<true, true, ORD>(inst, ninst, mag, nmag, non, non_inst, nnon, r0 + rows, bar, berr,
                                       sh);
    } else {
        hm_half_step_batch<false, true, ORD>(inst, ninst, mag, nmag, non, non_inst, nnon, r0, bar, berr, sh);
    }
}

} // namespace mmx

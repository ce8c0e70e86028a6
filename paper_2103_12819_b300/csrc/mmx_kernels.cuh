// mmx_kernels.cuh -- CUDA kernels of the coupled Maxwell-LLG step for
// sm_103a: setup (cell -> edge/face averaging, coefficients, initial M), the
// streaming E and H updates, and the cooperative H/M kernel of the magnetic
// box with the device-side residual reduction and loop control.
#pragma once
#include "mmx_device.cuh"

namespace mmx {

template <typename T> struct Ptr3 {
    T *p[3];
};

// ====================================================================== setup

// Mean of the existing cells adjacent to edge (c; i, j, k) (up to 4) or face
// (d; i, j, k) (2), periodic axes wrapped (Sec. 3.1).
__device__ __forceinline__ double edge_mean(const Geo &g, const double *cell, int c, int i, int j, int k)
{
    int ix[3] = {i, j, k};
    int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
    double sum = 0.0;
    int cnt = 0;
    for (int o1 = -1; o1 <= 0; o1++)
        for (int o2 = -1; o2 <= 0; o2++) {
            int cc[3];
            cc[c] = ix[c];
            cc[a1] = cell_nb(g, a1, ix[a1] + o1);
            cc[a2] = cell_nb(g, a2, ix[a2] + o2);
            if (cc[a1] < 0 || cc[a2] < 0) continue;
            sum += cell[(size_t)cc[0] + (size_t)g.n[0] * ((size_t)cc[1] + (size_t)g.n[1] * cc[2])];
            cnt++;
        }
    return sum / cnt;
}

__device__ __forceinline__ double face_mean(const Geo &g, const double *cell, int d, int i, int j, int k)
{
    int ix[3] = {i, j, k};
    double sum = 0.0;
    int cnt = 0;
    for (int o = -1; o <= 0; o++) {
        int cc[3] = {i, j, k};
        cc[d] = cell_nb(g, d, ix[d] + o);
        if (cc[d] < 0) continue;
        sum += cell[(size_t)cc[0] + (size_t)g.n[0] * ((size_t)cc[1] + (size_t)g.n[1] * cc[2])];
        cnt++;
    }
    return sum / cnt;
}

// Decode a thread of a 3-D launch over node indices [0,n0] x [0,n1] x [0,n2].
__device__ __forceinline__ bool node_of_thread(const Geo &g, int &i, int &j, int &k)
{
    i = blockIdx.x * blockDim.x + threadIdx.x;
    j = blockIdx.y * blockDim.y + threadIdx.y;
    k = blockIdx.z;
    return i <= g.n[0] && j <= g.n[1] && k <= g.n[2];
}

__device__ __forceinline__ bool edge_valid(const Geo &g, int c, int i, int j, int k)
{
    int ix[3] = {i, j, k};
    return ix[c] < g.n[c];
}

__device__ __forceinline__ bool face_valid(const Geo &g, int d, int i, int j, int k)
{
    int ix[3] = {i, j, k};
    for (int a = 0; a < 3; a++)
        if (a != d && ix[a] >= g.n[a]) return false;
    return true;
}

// which: 0 edge mean of component c, 1 face mean of family c.  Writes the
// mean (double) into out at the padded index.
__global__ void k_mean(const Geo g, const double *__restrict__ cell, int which, int c, double *out)
{
    int i, j, k;
    if (!node_of_thread(g, i, j, k)) return;
    if (which == 0) {
        if (!edge_valid(g, c, i, j, k)) return;
        out[gidx(g, i, j, k)] = cell ? edge_mean(g, cell, c, i, j, k) : 0.0;
    } else {
        if (!face_valid(g, c, i, j, k)) return;
        out[gidx(g, i, j, k)] = cell ? face_mean(g, cell, c, i, j, k) : 0.0;
    }
}

// E coefficients of edge component c from cell eps_r (NULL: 1) and sigma
// (NULL: 0): cb = 1/(eps/dt + sigma/2), ca = (eps/dt - sigma/2) cb.
template <typename T>
__global__ void k_e_coef(const Geo g, const double *__restrict__ eps_c, const double *__restrict__ sig_c,
                         int c, T *ca, T *cb)
{
    int i, j, k;
    if (!node_of_thread(g, i, j, k) || !edge_valid(g, c, i, j, k)) return;
    double eps0 = 1.0 / (kMu0 * kC0 * kC0);
    double eps = eps0 * (eps_c ? edge_mean(g, eps_c, c, i, j, k) : 1.0);
    double sg = sig_c ? edge_mean(g, sig_c, c, i, j, k) : 0.0;
    double den = sg / 2.0 + eps / g.dt;
    double keep = sg / 2.0 - eps / g.dt;
    size_t q = gidx(g, i, j, k);
    cb[q] = (T)(1.0 / den);
    if (ca) ca[q] = (T)(-keep / den);
}

// eps_r per cell in the padded layout (cell (i, j, k) at the padded index of
// node (i, j, k)); 1 where no cell is (the padding and the i = nx, j = ny,
// k = nz planes), eps_c NULL meaning 1 everywhere.
template <typename T> __global__ void k_eps_cells(const Geo g, const double *__restrict__ eps_c, T *out)
{
    int i, j, k;
    if (!node_of_thread(g, i, j, k)) return;
    const bool cell = i < g.n[0] && j < g.n[1] && k < g.n[2];
    out[gidx(g, i, j, k)] =
        (cell && eps_c) ? (T)eps_c[(size_t)i + (size_t)g.n[0] * ((size_t)j + (size_t)g.n[1] * k)] : T(1);
}

// H coefficient fh = dt/(2 mu0 mu_r,face) of face family d.
template <typename T>
__global__ void k_h_coef(const Geo g, const double *__restrict__ mu_c, int d, T *fh)
{
    int i, j, k;
    if (!node_of_thread(g, i, j, k) || !face_valid(g, d, i, j, k)) return;
    fh[gidx(g, i, j, k)] = (T)(g.dt / (2.0 * kMu0 * face_mean(g, mu_c, d, i, j, k)));
}

// Face materials of the magnetic box (family d): Ms, and either
// (kappa = mu0|gamma|dt/4, alpha/Ms) for the trapezoidal scheme or
// ((dt/2) mu0 gamma_L, (dt/2) alpha mu0 gamma_L/Ms) for the first-order one;
// M^n reset to Ms zhat.
template <typename T>
__global__ void k_box_materials(const Geo g, Box<T> b, int d, const double *__restrict__ ms_c,
                                const double *__restrict__ al_c, const double *__restrict__ ga_c)
{
    long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= b.nb) return;
    int bi = (int)(l % b.bx);
    int bj = (int)((l / b.bx) % b.by);
    int bk = (int)(l / ((long long)b.bx * b.by));
    int i = b.lo[0] + bi, j = b.lo[1] + bj, k = b.lo[2] + bk;
    T *ms = const_cast<T *>(b.ms[d]), *k1 = const_cast<T *>(b.k1[d]), *k2 = const_cast<T *>(b.k2[d]);
    double Ms = 0.0, al = 0.0, ga = 0.0;
    if (face_valid(g, d, i, j, k) && i <= g.n[0] && j <= g.n[1] && k <= g.n[2]) {
        Ms = ms_c ? face_mean(g, ms_c, d, i, j, k) : 0.0;
        al = al_c ? face_mean(g, al_c, d, i, j, k) : 0.0;
        ga = ga_c ? face_mean(g, ga_c, d, i, j, k) : 0.0;
    }
    ms[l] = (T)Ms;
    if (Ms > 0.0) {
        if (b.order == 2) {
            k1[l] = (T)(kMu0 * ga * g.dt / 4.0);
            k2[l] = (T)(al / Ms);
        } else {
            double gL = ga / (1.0 + al * al);
            k1[l] = (T)((g.dt / 2.0) * (kMu0 * gL));
            k2[l] = (T)((g.dt / 2.0) * (al * kMu0 * gL / Ms));
        }
    } else {
        k1[l] = T(0);
        k2[l] = T(0);
    }
    b.M[3 * d + 0][l] = T(0);
    b.M[3 * d + 1][l] = T(0);
    b.M[3 * d + 2][l] = (T)Ms;
}

// Initial M from cell-centred values: face average, renormalised to Ms
// (Sec. 3.1); a face whose average is below 1e-6 Ms takes the lower-index
// cell's direction (else the upper one's); none at all is an input error.
template <typename T>
__global__ void k_box_init_m(const Geo g, Box<T> b, int d, const double *__restrict__ mx,
                             const double *__restrict__ my, const double *__restrict__ mz)
{
    long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= b.nb) return;
    int bi = (int)(l % b.bx);
    int bj = (int)((l / b.bx) % b.by);
    int bk = (int)(l / ((long long)b.bx * b.by));
    int ix[3] = {b.lo[0] + bi, b.lo[1] + bj, b.lo[2] + bk};
    double Ms = (double)b.ms[d][l];
    double m[3] = {0.0, 0.0, 0.0};
    if (Ms > 0.0) {
        const double *mc[3] = {mx, my, mz};
        for (int c = 0; c < 3; c++) m[c] = face_mean(g, mc[c], d, ix[0], ix[1], ix[2]);
        double nrm = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
        if (!(nrm >= 1e-6 * Ms)) {
            bool found = false;
            for (int o = -1; o <= 0 && !found; o++) {
                int cc[3] = {ix[0], ix[1], ix[2]};
                cc[d] = cell_nb(g, d, ix[d] + o);
                if (cc[d] < 0) continue;
                size_t cq = (size_t)cc[0] + (size_t)g.n[0] * ((size_t)cc[1] + (size_t)g.n[1] * cc[2]);
                double v[3] = {mx[cq], my[cq], mz[cq]};
                if (v[0] * v[0] + v[1] * v[1] + v[2] * v[2] > 0.0) {
                    m[0] = v[0]; m[1] = v[1]; m[2] = v[2];
                    found = true;
                }
            }
            if (!found) {
                atomicOr(b.err, kErrBadInput);
                return;
            }
        }
        double n2 = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
        double f = Ms / n2;
        for (int c = 0; c < 3; c++) m[c] *= f;
    }
    for (int c = 0; c < 3; c++) b.M[3 * d + c][l] = (T)m[c];
}

// Per-magnetic-face constants in list order: Ms, k1, k2 from the box arrays
// and 1/Ms, which scales the iteration residual.
template <typename T> __global__ void k_box_cst(Box<T> b)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= b.nmag) return;
    const int4 e = b.mag[t];
    const unsigned l = (unsigned)e.x & 0x3fffffffu;
    const int d = (int)((unsigned)e.x >> 30);
    Q4<T> c;
    c.x = b.ms[d][l];
    c.y = b.k1[d][l];
    c.z = b.k2[d][l];
    c.w = c.x > T(0) ? T(1) / c.x : T(0);   // the residual's 1/Ms
    const_cast<Q4<T> *>(b.cst)[t] = c;
}

// M between the box arrays (read and written through the API) and the
// magnetic-face records (used while stepping): to_rec copies box -> records,
// otherwise records -> box.
template <typename T> __global__ void k_box_m_sync(Box<T> b, int to_rec)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= b.nmag) return;
    const int4 e = b.mag[t];
    const unsigned l = (unsigned)e.x & 0x3fffffffu;
    const int d = (int)((unsigned)e.x >> 30);
    if (to_rec) {
        Q4<T> q;
        q.x = b.M[3 * d][l];
        q.y = b.M[3 * d + 1][l];
        q.z = b.M[3 * d + 2][l];
        q.w = T(0);
        b.mn[t] = q;
    } else {
        const Q4<T> q = b.mn[t];
        b.M[3 * d][l] = q.x;
        b.M[3 * d + 1][l] = q.y;
        b.M[3 * d + 2][l] = q.z;
    }
}

// Point probes: row[p] = E component probe[p].x at padded index probe[p].y.
template <typename S, typename T>
__global__ void k_probe(Ptr3<S> E, T sE, const int2 *__restrict__ probe, int np, double *row)
{
    const int p = threadIdx.x;
    if (p < np) {
        const int2 q = probe[p];
        row[p] = (double)ld_s(E.p[q.x] + q.y, sE);
    }
}

// ============================================================ field copies

// Gather a padded device field (or a box-local M component) into a compact
// float64 array of extents e[3]; or scatter the other way (dir = 1).
template <typename T>
__global__ void k_copy_field(const Geo g, T *dev, const Box<T> b, int boxed, int e0, int e1, int e2,
                             double *host_like, int dir)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long N = (long long)e0 * e1 * e2;
    if (t >= N) return;
    int i = (int)(t % e0);
    int j = (int)((t / e0) % e1);
    int k = (int)(t / ((long long)e0 * e1));
    if (!boxed) {
        size_t q = gidx(g, i, j, k);
        if (dir == 0) host_like[t] = (double)dev[q];
        else dev[q] = (T)host_like[t];
        return;
    }
    bool in = i >= b.lo[0] && i < b.lo[0] + b.bx && j >= b.lo[1] && j < b.lo[1] + b.by &&
              k >= b.lo[2] && k < b.lo[2] + b.bz;
    if (dir == 0) {
        host_like[t] = in ? (double)dev[bidx(b.lo, b.bx, b.by, i, j, k)] : 0.0;
    } else if (in) {
        dev[bidx(b.lo, b.bx, b.by, i, j, k)] = (T)host_like[t];
    }
}

// Scatter a compact float64 copy of the box region [lo, lo + ce) of an M
// component (x fastest) into its box-local array.
template <typename T>
__global__ void k_box_region_in(const Box<T> b, int ce0, int ce1, int ce2, const double *__restrict__ src, T *dev)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)ce0 * ce1 * ce2) return;
    const int i = (int)(t % ce0), j = (int)((t / ce0) % ce1), k = (int)(t / ((long long)ce0 * ce1));
    dev[(size_t)i + (size_t)b.bx * ((size_t)j + (size_t)b.by * k)] = (T)src[t];
}

// The same for an FP16-stored E/H field: value = stored * scale.
__global__ void k_copy_field_h(const Geo g, __half *dev, float scale, int e0, int e1, int e2, double *host_like,
                               int dir)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long N = (long long)e0 * e1 * e2;
    if (t >= N) return;
    int i = (int)(t % e0);
    int j = (int)((t / e0) % e1);
    int k = (int)(t / ((long long)e0 * e1));
    size_t q = gidx(g, i, j, k);
    if (dir == 0)
        host_like[t] = (double)__half2float(dev[q]) * (double)scale;
    else
        dev[q] = __float2half_rn((float)(host_like[t] / (double)scale));
}

// On a periodic axis the node index n repeats node index 0 (padded arrays).
template <typename T>
__global__ void k_sync_periodic(const Geo g, T *dev, int e0, int e1, int e2, int axis)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int e[3] = {e0, e1, e2};
    int b = (axis + 1) % 3, c = (axis + 2) % 3;
    long long N = (long long)e[b] * e[c];
    if (t >= N) return;
    int ix[3], src[3];
    ix[axis] = g.n[axis];
    ix[b] = (int)(t % e[b]);
    ix[c] = (int)(t / e[b]);
    src[axis] = 0;
    src[b] = ix[b];
    src[c] = ix[c];
    dev[gidx(g, ix[0], ix[1], ix[2])] = dev[gidx(g, src[0], src[1], src[2])];
}

// ======================================================= streaming updates

// Step 2 on every edge; one thread per node (i, j, k) updates Ex, Ey, Ez
// there.  Soft J at t = (step + 1/2) dt.
template <typename T>
__global__ void __launch_bounds__(256) k_e_update(const __grid_constant__ Geo g,
                                                  const __grid_constant__ Fields<T> f,
                                                  const Src<T> *__restrict__ src, int nsrc)
{
    int i, j, k;
    if (!node_of_thread(g, i, j, k)) return;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        if (!edge_valid(g, c, i, j, k)) continue;
        T J = nsrc ? j_source(g, f, src, nsrc, c, i, j, k) : T(0);
        e_edge(g, f, c, i, j, k, J);
    }
}

// Steps 1/3 on every face outside the magnetic box (those are all
// non-magnetic); in place.
template <typename T, typename S = T>
__global__ void __launch_bounds__(256) k_h_update(const __grid_constant__ Geo g,
                                                  const __grid_constant__ Fields<T, S> f, int blo0, int blo1,
                                                  int blo2, int bhi0, int bhi1, int bhi2)
{
    int i, j, k;
    if (!node_of_thread(g, i, j, k)) return;
    bool inbox = i >= blo0 && i < bhi0 && j >= blo1 && j < bhi1 && k >= blo2 && k < bhi2;
    if (inbox) return;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (!face_valid(g, d, i, j, k)) continue;
        size_t q = gidx(g, i, j, k);
        T v = h_face_nonmag(g, f, d, i, j, k, f.H[d]);
        st_s(f.H[d] + q, v, f.isH);
        if (!isfinite(v)) atomicOr(f.err, kErrNonFinite);
    }
}

// Hard sources (Sec. 3.2): overwrite one field value with g(t).
template <typename T>
__global__ void k_hard(const Geo g, Ptr3<T> F, const Src<T> *__restrict__ src, int nsrc, int kind, double t)
{
    int s = threadIdx.x;
    if (s >= nsrc) return;
    const Src<T> &q = src[s];
    if (q.kind != kind) return;
    F.p[q.comp][gidx(g, q.i, q.j, q.k)] = (T)waveform(q.amp, q.f0, q.tp, q.t0, t);
}

// ================================================== magnetic box kernel

// Grid barrier on one monotonic 64-bit arrival counter.  After the block's
// __syncthreads, thread 0 arrives with a release add at GPU scope (which
// publishes every write the block made before the barrier) and spins with
// acquire loads; the barrier round a block is in completes when the counter
// reaches the next multiple of gridDim.x, which the block derives from the
// value its own add returned, so no reset or generation word is needed.  The
// wait is bounded (~2^31 cycles): on expiry the block latches kErrTimeout
// and returns false (the other blocks then time out at the next barrier).
// (A two-level arrival over 16 group counters measured slower: the last
// block then makes two dependent atomic round trips.)
constexpr int kBarWords = 2;   // u64 words: the barrier's count, a probe's decision word

// True once a bounded wait has latched kErrTimeout in the status word (read
// at kernel entry, before any barrier; the word only changes between
// launches except through this launch's own timeouts).
__device__ __forceinline__ bool timeout_latched(const int *err)
{
    return (*(const volatile int *)err & kErrTimeout) != 0;
}
constexpr int kVoteRows = 4;   // decision words sit this many residual rows past them

__device__ __forceinline__ bool grid_barrier(unsigned long long *bar, int *err, int nblocks = -1)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long nb = nblocks < 0 ? gridDim.x : (unsigned)nblocks;
        unsigned long long old;
        asm volatile("atom.add.release.gpu.global.u64 %0, [%1], 1;" : "=l"(old) : "l"(bar) : "memory");
        const unsigned long long target = (old / nb + 1) * nb;
        const long long t0 = clock64();
        for (;;) {
            unsigned long long cur;
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(cur) : "l"(bar) : "memory");
            if (cur >= target) break;
            if (clock64() - t0 > (1LL << 31)) {
                atomicOr(err, kErrTimeout);
                ok = 0;
                break;
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Grid barrier that also takes the convergence decision of one iteration:
// every block adds 2^32 plus its not-converged flag to the iteration's own
// word (zeroed before the launch) with acquire-release semantics and polls
// it with acquire loads, 32 ns apart, until all blocks have arrived; the low
// half then counts the blocks that did not converge.  The decision thus comes
// with the barrier instead of a second read of the reduced residual after it
// (134.8 -> 133.4 us per waveguide step).  Returns 1 if no block flagged, 0
// if some did, -1 if the bounded wait (~2^31 cycles) expired, with
// kErrTimeout latched.
__device__ __forceinline__ int grid_vote(unsigned long long *word, bool flag, int *err, int nblocks = -1)
{
    __shared__ int s_v;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long nb = nblocks < 0 ? gridDim.x : (unsigned)nblocks;
        const unsigned long long add = (1ull << 32) | (flag ? 1ull : 0ull);
        unsigned long long v;
        asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;" : "=l"(v) : "l"(word), "l"(add) : "memory");
        v += add;
        const long long t0 = clock64();
        int res;
        for (;;) {
            if ((v >> 32) >= nb) {
                res = (v & 0xffffffffull) == 0 ? 1 : 0;
                break;
            }
            if (clock64() - t0 > (1LL << 31)) {
                atomicOr(err, kErrTimeout);
                res = -1;
                break;
            }
            __nanosleep(32);
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(word) : "memory");
        }
        s_v = res;
    }
    __syncthreads();
    return s_v;
}

// Block-wide max: warp shuffle, then one warp over the per-warp maxima.
template <typename T> __device__ __forceinline__ T block_max(T v)
{
    __shared__ T s_part[32];
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) s_part[w] = v;
    __syncthreads();
    if (w == 0) {
        int nw = (blockDim.x + 31) >> 5;
        v = l < nw ? s_part[l] : T(0);
        for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;   // valid in thread 0
}

// Publish a block's residual maximum: atomicMax on the bit pattern of the
// non-negative FP64 value (non-negative doubles order like their bits).
template <typename T>
__device__ __forceinline__ void publish_residual(unsigned long long *slot, T rblock)
{
    if (threadIdx.x == 0 && rblock > T(0))
        atomicMax(slot, (unsigned long long)__double_as_longlong((double)rblock));
}


struct FaceOf {
    int d, i, j, k;
    unsigned l;
};

// A face from its packed word alone: i, j, k from the box index l =
// (i - lo0) + bx ((j - lo1) + by (k - lo2)), the inverse of the list build.
template <typename T> __device__ __forceinline__ FaceOf face_of32(unsigned e, const Box<T> &b)
{
    FaceOf fo;
    fo.l = e & 0x3fffffffu;
    fo.d = (int)(e >> 30);
    const unsigned bx = (unsigned)b.bx, bxy = bx * (unsigned)b.by;
    const unsigned bk = fo.l / bxy, r = fo.l - bk * bxy;
    const unsigned bj = r / bx;
    fo.i = b.lo[0] + (int)(r - bj * bx);
    fo.j = b.lo[1] + (int)bj;
    fo.k = b.lo[2] + (int)bk;
    return fo;
}

__device__ __forceinline__ FaceOf face_of(int4 e)
{
    FaceOf fo;
    fo.l = (unsigned)e.x & 0x3fffffffu;
    fo.d = (int)((unsigned)e.x >> 30);
    fo.i = e.y;
    fo.j = e.z;
    fo.k = e.w;
    return fo;
}

// H vector at a face of family D (i, j, k): own normal value and the
// four-point means of the two transverse families (Sec. 3.1), from the padded
// global H (mode 0) or from box-local iterates (mode 1).  The family is a
// template argument so that every index below is in registers.
template <int D, typename T, typename SG>
__device__ __forceinline__ void h_vector(const Geo &g, const Box<T> &b, SG *const Hg[3], T *const Hb[3],
                                         int mode, int i, int j, int k, T h[3], T sH = T(1))
{
    const int ix[3] = {i, j, k};
    // the face's index and the strides of the layout read: every neighbour
    // is the face's index plus its offsets times the strides (a periodic wrap
    // along D is an offset of n - 1 cells; unsigned arithmetic is modular)
    const unsigned base = mode == 0 ? gidx32(g, i, j, k) : bidx32(b.lo, b.bx, b.by, i, j, k);
    const unsigned s1 = mode == 0 ? (unsigned)g.X : (unsigned)b.bx;
    const unsigned st[3] = {1u, s1, s1 * (mode == 0 ? (unsigned)g.Y : (unsigned)b.by)};
    h[D] = mode == 0 ? ld_s(Hg[D] + base, sH) : Hb[D][base];
#pragma unroll
    for (int t = 0; t < 3; t++) {
        if (t == D) continue;
        T sum = T(0);
        int cnt = 0;
#pragma unroll
        for (int od = -1; od <= 0; od++) {
            int nd = cell_nb(g, D, ix[D] + od);
            if (nd < 0) continue;
            const unsigned qd = base + (unsigned)(nd - ix[D]) * st[D];
#pragma unroll
            for (int ot = 0; ot <= 1; ot++) {
                const unsigned q = qd + (unsigned)ot * st[t];
                sum += mode == 0 ? ld_s(Hg[t] + q, sH) : Hb[t][q];
                cnt++;
            }
        }
        h[t] = sum * (cnt == 4 ? T(0.25) : T(0.5));
    }
}

template <typename T> __device__ __forceinline__ Q4<T> q4_load(const Q4<T> *p)
{
    return *p;
}

template <typename T> __device__ __forceinline__ Q4<T> q4(T x, T y, T z, T w)
{
    Q4<T> q;
    q.x = x;
    q.y = y;
    q.z = z;
    q.w = w;
    return q;
}

// Everything phase 0 reads for one magnetic face.
template <typename T> struct FirstIn {
    Q4<T> cs;       // Ms, k1, k2
    T Mn[3];
    T hn, rest, zp;
    T h[3];
};

// Where the iterates r >= 2 get beta and C'.  Phase 0 stores them in a
// 16-byte record per face for the iterates to read back.  The batched launch
// in FP32 skips that store for an instance whose previous half step stopped
// at its first iterate (then this one most likely does too, and the record
// would never be read); an iterate 2 of such an instance forms beta and C'
// again from H^n and E and stores them for any later iterate.  The
// single-instance launches always keep the record: the second copy of the
// iterate sweep would cost them instruction fetch where the box is
// L2-resident, and their benchmark boxes take two iterates per half step.
// FP64, bound by its arithmetic, always keeps the record.
template <typename T> struct RecomputeBC {
    static constexpr bool value = sizeof(T) == 4;
};

// C' = H^n - dt/(2 mu0) curl E (curl E = rest + zp) and
// beta = -kappa M^n x H_eff^n: one expression each for phase 0 and for the
// iterates that form them again, so both round alike.
template <typename T> __device__ __forceinline__ T c_prime(const Box<T> &b, T hn, T rest, T zp)
{
    return hn - b.cfar * (rest + zp);
}

template <typename T> __device__ __forceinline__ void beta_of(const T Mn[3], const T heff[3], T k1, T beta[3])
{
    beta[0] = -k1 * (Mn[1] * heff[2] - Mn[2] * heff[1]);
    beta[1] = -k1 * (Mn[2] * heff[0] - Mn[0] * heff[2]);
    beta[2] = -k1 * (Mn[0] * heff[1] - Mn[1] * heff[0]);
}

// The H^n and curl E loads of phase 0 on a magnetic face of family D: H^n is
// the global H (SECOND false) or the previous half step's box-local iterate
// Hp (SECOND true); h gets the four-point H vector at the face.
template <int D, bool SECOND, typename T, typename S>
__device__ __forceinline__ void hn_loads(const Geo &g, const Fields<T, S> &f, const Box<T> &b, S *const Hin[3],
                                         T *const Hp[3], const FaceOf &fo, T &hn, T &rest, T &zp, T h[3])
{
    const unsigned q = gidx32(g, fo.i, fo.j, fo.k);
    curl_e32(g, f.E, f.inv_d, D, q, rest, zp, f.sE);
    if (SECOND) {
        hn = Hp[D][fo.l];
        h_vector<D>(g, b, Hin, Hp, 1, fo.i, fo.j, fo.k, h);
    } else {
        hn = ld_s(Hin[D] + q, f.sH);
        h_vector<D>(g, b, Hin, Hp, 0, fo.i, fo.j, fo.k, h, f.sH);
    }
}

// Loads of phase 0 on a magnetic face of family D (list position t): H^n and
// curl E as hn_loads; M^n is the face record, plus the previous half step's
// converged increment dmp when SECOND.
template <int D, bool SECOND, typename T, typename S>
__device__ __forceinline__ void first_load(const Geo &g, const Fields<T, S> &f, const Box<T> &b, S *const Hin[3],
                                           T *const Hp[3], const Q4<T> *dmp, const FaceOf &fo, int t,
                                           FirstIn<T> &in)
{
    in.cs = q4_load(b.cst + t);
    const Q4<T> m0 = q4_load(b.mn + t);
    if (SECOND) {
        const Q4<T> d0 = q4_load(dmp + t);
        in.Mn[0] = m0.x + d0.x;
        in.Mn[1] = m0.y + d0.y;
        in.Mn[2] = m0.z + d0.z;
    } else {
        in.Mn[0] = m0.x;
        in.Mn[1] = m0.y;
        in.Mn[2] = m0.z;
    }
    hn_loads<D, SECOND>(g, f, b, Hin, Hp, fo, in.hn, in.rest, in.zp, in.h);
}

// Arithmetic and stores of phase 0: C' = H^n - dt/(2 mu0) curl E,
// beta = -kappa M^n x H_eff^n, e0 and DeltaM^1; H^1 into Hw.  e0 rides in
// the w slot of the increment record, which every iterate rewrites anyway,
// so a first half step (SECOND false, M^n unchanged in its record) writes
// no M record; the {beta, C'} record is stored when store_bc is true (see
// RecomputeBC).  Returns max_c |DeltaM^1_c| / Ms.
template <int D, bool SECOND, int ORD = 0, typename T>
__device__ __forceinline__ T first_finish(const Geo &g, const Box<T> &b, T *const Hw[3], const FaceOf &fo, int t,
                                          const FirstIn<T> &in, const T h0[3], bool store_bc = true)
{
    const T Ms = in.cs.x, k1 = in.cs.y, k2 = in.cs.z;
    const T *Mn = in.Mn;
    const T cp = c_prime(b, in.hn, in.rest, in.zp);
    const T e0 = norm_defect(Ms, Mn[0], Mn[1], Mn[2]);
    T heff[3];
#pragma unroll
    for (int c = 0; c < 3; c++) heff[c] = h0[c] + in.h[c];
    T dM[3], dMh;
    T beta[3] = {T(0), T(0), T(0)};
    if (ORD == 0 ? b.order == 2 : ORD == 2) {
        beta_of(Mn, heff, k1, beta);
        llg_iterate(Mn, beta, heff, k1, k2, Ms, e0, D, dM, dMh);
    } else {
        llg_euler(Mn, heff, k1, k2, Ms, e0, D, dM, dMh);
    }
    if (!RecomputeBC<T>::value || store_bc) b.bc[t] = q4(beta[0], beta[1], beta[2], cp);
    if (SECOND) b.mn[t] = q4(Mn[0], Mn[1], Mn[2], T(0));
    b.dm[1][t] = q4(dM[0], dM[1], dM[2], e0);
    const bool wall = wall_node(g, D, D == 0 ? fo.i : D == 1 ? fo.j : fo.k);
    Hw[D][fo.l] = wall ? T(0) : cp - dMh;
    return max(abs(dM[0]), max(abs(dM[1]), abs(dM[2]))) * in.cs.w;
}

// Phase 0 on a non-magnetic face of family D: its final H in both iterate
// buffers W0, W1.
template <int D, bool SECOND, typename T, typename S>
__device__ __forceinline__ void non_first(const Geo &g, const Fields<T, S> &f, S *const Hin[3], T *const Hp[3],
                                          T *const W0[3], T *const W1[3], const FaceOf &fo)
{
    const T hn = SECOND ? Hp[D][fo.l] : ld_s(Hin[D] + gidx32(g, fo.i, fo.j, fo.k), f.sH);
    const T v = h_face_nonmag_val(g, f, D, fo.i, fo.j, fo.k, hn);
    W0[D][fo.l] = v;
    W1[D][fo.l] = v;
}

// Everything iteration r reads for one magnetic face: the {beta, C'} record
// bq, or (HAVE_BC false) what phase 0 formed it from.
template <typename T> struct NextIn {
    Q4<T> cs, mq, bq, pq;
    T h[3];
    T hn, rest, zp, hN[3];
};

// Loads of iterate r on a magnetic face of family D; without the record
// (HAVE_BC false) the H^n and curl E loads of phase 0 instead, with H^n
// from Hin or Hp as in phase 0 (SECOND).
template <int D, bool SECOND = false, bool HAVE_BC = true, typename T, typename S = T>
__device__ __forceinline__ void next_load(const Geo &g, const Box<T> &b, const FaceOf &fo, int t, T *const Hprev[3],
                                          int pr, NextIn<T> &in, const Fields<T, S> *f = nullptr,
                                          S *const *Hin = nullptr, T *const *Hp = nullptr)
{
    in.cs = q4_load(b.cst + t);
    in.mq = q4_load(b.mn + t);
    if constexpr (HAVE_BC)
        in.bq = q4_load(b.bc + t);
    else
        hn_loads<D, SECOND>(g, *f, b, Hin, Hp, fo, in.hn, in.rest, in.zp, in.hN);
    in.pq = q4_load(b.dm[pr] + t);
    h_vector<D>(g, b, Hprev, Hprev, 1, fo.i, fo.j, fo.k, in.h);
}

// Iterate r >= 2 from the neighbours' iterate r-1: DeltaM^r into dm[cr]
// (e0 carried on in its w slot), H^r into Hcur; without the record
// (HAVE_BC false) beta and C' are formed first and stored.  Returns
// max_c |DeltaM^r_c - DeltaM^(r-1)_c| / Ms.
template <int D, bool HAVE_BC = true, typename T>
__device__ __forceinline__ T next_finish(const Geo &g, const Box<T> &b, const FaceOf &fo, int t, T *const Hcur[3],
                                         int cr, const NextIn<T> &in, const T h0[3])
{
    const T Ms = in.cs.x, k1 = in.cs.y, k2 = in.cs.z;
    const T Mn[3] = {in.mq.x, in.mq.y, in.mq.z};
    Q4<T> bq = in.bq;
    if constexpr (!HAVE_BC) {
        T heffn[3], bt[3];
#pragma unroll
        for (int c = 0; c < 3; c++) heffn[c] = h0[c] + in.hN[c];
        beta_of(Mn, heffn, k1, bt);
        bq = q4(bt[0], bt[1], bt[2], c_prime(b, in.hn, in.rest, in.zp));
        b.bc[t] = bq;
    }
    const T beta[3] = {bq.x, bq.y, bq.z};
    T heff[3];
#pragma unroll
    for (int c = 0; c < 3; c++) heff[c] = h0[c] + in.h[c];
    T dM[3], dMh;
    llg_iterate(Mn, beta, heff, k1, k2, Ms, in.pq.w, D, dM, dMh);
    const bool wall = wall_node(g, D, D == 0 ? fo.i : D == 1 ? fo.j : fo.k);
    Hcur[D][fo.l] = wall ? T(0) : bq.w - dMh;
    b.dm[cr][t] = q4(dM[0], dM[1], dM[2], in.pq.w);
    return max(abs(dM[0] - in.pq.x), max(abs(dM[1] - in.pq.y), abs(dM[2] - in.pq.z))) * in.cs.w;
}

// Final H and M^(n+1/2) on one magnetic face of family D: H to the global
// Hout, M into the face record (the box M is refreshed from the records at
// the end of every mmx_step call).  Returns false if a value is not finite.
template <int D, typename T, typename S>
__device__ __forceinline__ bool mag_store(const Geo &g, const Box<T> &b, const FaceOf &fo, int t,
                                          T *const Hfin[3], S *const Hout[3], int fr, T isH)
{
    const T v = Hfin[D][fo.l];
    st_s(Hout[D] + gidx32(g, fo.i, fo.j, fo.k), v, isH);
    const Q4<T> mq = q4_load(b.mn + t);
    const Q4<T> dq = q4_load(b.dm[fr] + t);
    const T m0 = mq.x + dq.x, m1 = mq.y + dq.y, m2 = mq.z + dq.z;
    b.mn[t] = q4(m0, m1, m2, T(0));
    return isfinite(v) && isfinite(m0) && isfinite(m1) && isfinite(m2);
}

// One H/M half step on every face of the magnetic box (Sec. 3.2.2 Step 1 or
// Step 3) with the E in f.E.  Work comes from two lists built when the
// materials are set, each ordered by family: the magnetic faces and the
// other faces of the box; the same thread takes the same faces in every
// phase.  Phase 0 gives
// non-magnetic faces their final H and forms the first iterate on magnetic
// faces; each further iteration r updates every magnetic face from the
// neighbours' iterate r-1 (Jacobi), reduces max |DeltaM^r - DeltaM^(r-1)|/Ms
// into res[r] (warp shuffle, block max, one atomicMax on the FP64 bit
// pattern per block) and meets at a bounded grid barrier; all blocks then
// read res[r] and stop together at the first r with res[r] < tol (or at
// max_iter, latching kErrNotConverged).  M lives in the face records.
//   SECOND false: H^n comes from the global H (Hin), M^n from the records.
//   SECOND true:  both come from the previous half step of this launch,
//                 which ended in iterate buffer fprev without writing back.
//   WRITE true:   H^(n+1/2) goes to the global Hout and M^(n+1/2) into the
//                 records; otherwise both stay in the iterate buffers.
// Returns the final iterate parity, or -1 if a barrier timed out.
//   ORD:          the scheme order (2 or 1) as a compile-time constant, or
//                 0 to read it from the box descriptor.
template <bool SECOND, bool WRITE, int ORD = 0, typename T, typename S>
__device__ int hm_half_step(const Geo &g, const Fields<T, S> &f, const Box<T> &b, S *const Hin[3], S *const Hout[3],
                            int fprev, unsigned long long *res, int bid = -1, int nblocks = -1)
{
    const bool second_order = ORD == 0 ? b.order == 2 : ORD == 2;
    // the blocks taking part: the whole grid, or blocks 0 .. nblocks-1 of an
    // overlap launch
    if (bid < 0) {
        bid = blockIdx.x;
        nblocks = gridDim.x;
    }
    const int stride = nblocks * blockDim.x;
    const int t0 = bid * blockDim.x + threadIdx.x;
    const T h0[3] = {(T)b.h0[0], (T)b.h0[1], (T)b.h0[2]};
    // iterate buffers of this half step; H^n of a second half step
    T *const W0[3] = {SECOND ? b.Hit2[0][0] : b.Hit[0][0], SECOND ? b.Hit2[0][1] : b.Hit[0][1],
                      SECOND ? b.Hit2[0][2] : b.Hit[0][2]};
    T *const W1[3] = {SECOND ? b.Hit2[1][0] : b.Hit[1][0], SECOND ? b.Hit2[1][1] : b.Hit[1][1],
                      SECOND ? b.Hit2[1][2] : b.Hit[1][2]};
    T *const Hp[3] = {b.Hit[fprev & 1][0], b.Hit[fprev & 1][1], b.Hit[fprev & 1][2]};
    const Q4<T> *dmp = b.dm[fprev & 1];

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
    {
        unsigned nx = t0 < b.nmag ? b.mag32[t0] : 0u;
        for (int t = t0; t < b.nmag; t += stride) {
            const FaceOf fo = face_of32(nx, b);
            if (t + stride < b.nmag) nx = b.mag32[t + stride];
            FirstIn<T> in;
            T rv;
            if (fo.d == 0) {
                first_load<0, SECOND>(g, f, b, Hin, Hp, dmp, fo, t, in);
                rv = first_finish<0, SECOND, ORD>(g, b, W1, fo, t, in, h0);
            } else if (fo.d == 1) {
                first_load<1, SECOND>(g, f, b, Hin, Hp, dmp, fo, t, in);
                rv = first_finish<1, SECOND, ORD>(g, b, W1, fo, t, in, h0);
            } else {
                first_load<2, SECOND>(g, f, b, Hin, Hp, dmp, fo, t, in);
                rv = first_finish<2, SECOND, ORD>(g, b, W1, fo, t, in, h0);
            }
            rmax = max(rmax, rv);
        }
    }
    rmax = block_max(rmax);
    publish_residual(&res[1], rmax);
    // the decision words of this half step: the row kVoteRows rows past res.
    // A block votes "not converged" when its maximum is at or above tol; the
    // maximum over blocks is below tol exactly when no block votes so.  A
    // block whose maximum is not positive (NaN included) publishes nothing
    // and does not vote, as it does not raise the published maximum.
    unsigned long long *const vote = res + kVoteRows * (kMaxIter + 1);
    const int v1 = grid_vote(&vote[1], rmax > T(0) && !((double)rmax < b.tol), b.err, nblocks);
    if (v1 < 0) return -1;

    int r = 1;
    bool conv = v1 == 1 || !second_order;
    while (!conv && r < b.max_iter) {
        r++;
        const int pr = (r - 1) & 1, cr = r & 1;
        T *const Hprev[3] = {pr ? W1[0] : W0[0], pr ? W1[1] : W0[1], pr ? W1[2] : W0[2]};
        T *const Hcur[3] = {cr ? W1[0] : W0[0], cr ? W1[1] : W0[1], cr ? W1[2] : W0[2]};
        rmax = T(0);
        unsigned nx = t0 < b.nmag ? b.mag32[t0] : 0u;
        for (int t = t0; t < b.nmag; t += stride) {
            const FaceOf fo = face_of32(nx, b);
            if (t + stride < b.nmag) nx = b.mag32[t + stride];
            NextIn<T> in;
            T rv;
            if (fo.d == 0) {
                next_load<0>(g, b, fo, t, Hprev, pr, in);
                rv = next_finish<0>(g, b, fo, t, Hcur, cr, in, h0);
            } else if (fo.d == 1) {
                next_load<1>(g, b, fo, t, Hprev, pr, in);
                rv = next_finish<1>(g, b, fo, t, Hcur, cr, in, h0);
            } else {
                next_load<2>(g, b, fo, t, Hprev, pr, in);
                rv = next_finish<2>(g, b, fo, t, Hcur, cr, in, h0);
            }
            rmax = max(rmax, rv);
        }
        rmax = block_max(rmax);
        publish_residual(&res[r], rmax);
        const int vr = grid_vote(&vote[r], rmax > T(0) && !((double)rmax < b.tol), b.err, nblocks);
        if (vr < 0) return -1;
        conv = vr == 1;
    }

    const int fr = r & 1;
    if (WRITE) {
        // ---- write back H (all box faces) and M (magnetic-face records)
        T *const Hfin[3] = {fr ? W1[0] : W0[0], fr ? W1[1] : W0[1], fr ? W1[2] : W0[2]};
        bool ok = true;
        for (int t = t0; t < b.nnon; t += stride) {
            const FaceOf fo = face_of(b.nonmag[t]);
            const T v = Hfin[fo.d][fo.l];
            S *const Ho = fo.d == 0 ? Hout[0] : fo.d == 1 ? Hout[1] : Hout[2];
            st_s(Ho + gidx32(g, fo.i, fo.j, fo.k), v, f.isH);
            ok &= isfinite(v);
        }
        for (int t = t0; t < b.nmag; t += stride) {
            const FaceOf fo = face_of32(b.mag32[t], b);
            ok &= fo.d == 0   ? mag_store<0>(g, b, fo, t, Hfin, Hout, fr, f.isH)
                  : fo.d == 1 ? mag_store<1>(g, b, fo, t, Hfin, Hout, fr, f.isH)
                              : mag_store<2>(g, b, fo, t, Hfin, Hout, fr, f.isH);
        }
        if (!ok) atomicOr(b.err, kErrNonFinite);
    }
    if (bid == 0 && threadIdx.x == 0) {
        if (!conv && second_order) atomicOr(b.err, kErrNotConverged);
        unsigned long long hs = *b.halfsteps;
        b.iterlog[hs % kIterLogCap] = r;
        *b.halfsteps = hs + 1;
        *b.last_res = second_order ? __longlong_as_double((long long)res[r]) : 0.0;
    }
    return fr;
}

// Resident blocks per SM the box kernels are compiled for.  The H/M phases
// are bound by load latency and grid barriers, so FP32 trades registers for
// occupancy: 5 blocks of 256 threads (48 registers) against 2 at the
// unconstrained 99 registers, 15% faster on the 128x128x512 waveguide; FP64
// is bound by FP64 arithmetic and needs at most 128 registers for its two
// blocks (at 130 it fell to one block and a step took 1% longer).
template <typename T> struct BoxMinBlocks {
    static constexpr int value = sizeof(T) == 4 ? 5 : 2;
};

// Cooperative launch over the magnetic box: nsub = 1 runs one H/M half step
// from f.H into Hout; nsub = 2 runs Step 3 of step n and Step 1 of step n+1
// back to back (both use the same E^(n+1)), the second reading the first's
// result.  Residual words: launch parity `slot` uses rows 2 slot and
// 2 slot + 1 of res (residual maxima) and the rows kVoteRows further on
// (decision words), and clears the other parity's rows for the next launch.
template <typename T, typename S = T, int ORD = 0>
__global__ void __launch_bounds__(256, BoxMinBlocks<T>::value) k_hm_box(const __grid_constant__ Geo g,
                                                const __grid_constant__ Fields<T, S> f,
                                                const __grid_constant__ Box<T> b,
                                                const __grid_constant__ Ptr3<S> Hout, int nsub, int slot)
{
    const int W = kMaxIter + 1;
    // a bounded wait that gave up earlier in this mmx_step call left the
    // barrier counter out of step: every later launch of the call returns at
    // once instead of spending its wait budget at each barrier (the host
    // reads the latched timeout and resets the counter)
    if (timeout_latched(b.err)) return;
    if (blockIdx.x == 0) {
        unsigned long long *other = b.res + 2 * (1 - slot) * W;
        for (int r = threadIdx.x; r < 2 * W; r += blockDim.x) {
            other[r] = 0ull;
            other[kVoteRows * W + r] = 0ull;
        }
    }
    if (nsub == 2) {
        // two half steps with one E; the first keeps its result in the
        // iterate buffers, the second starts from there and writes back
        const int fr = hm_half_step<false, false, ORD>(g, f, b, f.H, Hout.p, 0, b.res + 2 * slot * W);
        if (fr < 0) return;
        hm_half_step<true, true, ORD>(g, f, b, f.H, Hout.p, fr, b.res + (2 * slot + 1) * W);
    } else {
        hm_half_step<false, true, ORD>(g, f, b, f.H, Hout.p, 0, b.res + 2 * slot * W);
    }
}

// ========================================================== fused pass

// One pass per time step over the whole grid: E^(n+1) on every edge from
// (E^n, H^(n+1/2)) and, on every face outside the magnetic box, H from
// H^(n+1/2) by nhalf half steps of -fh curl E^(n+1) (two for H^(n+3/2):
// Step 3 of step n then Step 1 of step n+1, both with E^(n+1); one for
// H^(n+1) on the last step of a call).  Reads Eo/Ho/Zo, writes En/Hn/Zn
// (ping-pong: every recomputed halo value sees consistent old data); the
// H PML parts are private to their face and updated in place.
//
// Blocking (2.5-D): a block of BX x BY threads owns an x-y tile of
// (BX-1) x (BY-1) columns plus a one-column high-side halo and marches over
// a z chunk [k0, k1).  At plane k it stages H^(n+1/2) of layer/plane k (with
// a one-cell low-side halo) in shared memory, computes E^(n+1) at plane k
// for tile + halo, then H at plane k (Hz) and layer k-1 (Hx, Hy) for the
// tile.  The next plane's column values are loaded into registers before
// the first barrier so their latency overlaps this plane's work; the shared
// tiles are double-buffered (two barriers per plane).  Everything that does
// not depend on k (offsets, wall and box flags, sources) is set up once per
// column, and offsets are 32-bit (a grid of up to 2^31 padded elements).
// The chunk's last iteration k = k1 recomputes the next chunk's E plane
// without writing it.
// Compile-time variants: NH half steps of H (1 or 2), PMLK a z-PML is
// present, GEN per-edge ca / per-face fh arrays exist (sigma or mu_r varies).
template <typename T, int BX, int BY, int NH, bool PMLK, bool GEN>
__global__ void __launch_bounds__(BX *BY, sizeof(T) == 4 ? 4 : 2) k_fused(const __grid_constant__ Geo g, const __grid_constant__ Fields<T> f,
                                                 Ptr3<T> Eo, Ptr3<T> Ho, Ptr3<T> En, Ptr3<T> Hn, Ptr3<T> Zo,
                                                 Ptr3<T> Zn, const Src<T> *__restrict__ src, int nsrc,
                                                 int chunk, int blo0, int blo1, int blo2, int bhi0, int bhi1,
                                                 int bhi2)
{
    constexpr int nhalf = NH;
    __shared__ T sH[2][3][BY + 1][BX + 1];
    __shared__ T sE[2][2][BY][BX];
    __shared__ T sEz[2][BY][BX];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.x * (BX - 1) + tx;
    const int j = blockIdx.y * (BY - 1) + ty;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int k0 = blockIdx.z * chunk;
    const int k1 = min(k0 + chunk, nz);
    const bool last_chunk = k1 == nz;
    const bool halo = tx == BX - 1 || ty == BY - 1;
    const bool col = i <= nx && j <= ny;
    const T idx = f.inv_d[0], idy = f.inv_d[1], idz = f.inv_d[2];
    const unsigned XY = (unsigned)g.X * (unsigned)g.Y;

    // ---- per-column set-up
    const int ci = cell_nb(g, 0, i), cj = cell_nb(g, 1, j);
    const int cim = cell_nb(g, 0, i - 1), cjm = cell_nb(g, 1, j - 1);
    const unsigned qc = (unsigned)i + (unsigned)g.X * (unsigned)j;          // this column
    const bool hx_ok = col && cj >= 0, hy_ok = col && ci >= 0, hz_ok = col && ci >= 0 && cj >= 0;
    const unsigned ohx = (unsigned)i + (unsigned)g.X * (unsigned)max(cj, 0);
    const unsigned ohy = (unsigned)max(ci, 0) + (unsigned)g.X * (unsigned)j;
    const unsigned ohz = (unsigned)max(ci, 0) + (unsigned)g.X * (unsigned)max(cj, 0);
    const bool hym_ok = col && tx == 0 && cim >= 0, hzm_ok = hym_ok && cj >= 0;
    const unsigned ohym = (unsigned)max(cim, 0) + (unsigned)g.X * (unsigned)j;
    const unsigned ohzm = (unsigned)max(cim, 0) + (unsigned)g.X * (unsigned)max(cj, 0);
    const bool hxj_ok = col && ty == 0 && cjm >= 0, hzj_ok = hxj_ok && ci >= 0;
    const unsigned ohxj = (unsigned)i + (unsigned)g.X * (unsigned)max(cjm, 0);
    const unsigned ohzj = (unsigned)max(ci, 0) + (unsigned)g.X * (unsigned)max(cjm, 0);
    const bool wx = wall_node(g, 0, i), wy = wall_node(g, 1, j);
    const bool ex_on = col && i < nx && !wy;          // Ex edge exists and is not on a y wall
    const bool ey_on = col && j < ny && !wx;
    const bool ez_on = col && !wx && !wy;
    const bool ex_has = col && i < nx, ey_has = col && j < ny;
    const bool tile = col && !halo;
    const bool hz_on = tile && i < nx && j < ny && !(i >= blo0 && i < bhi0 && j >= blo1 && j < bhi1);
    const bool hz_box = tile && i < nx && j < ny && (i >= blo0 && i < bhi0 && j >= blo1 && j < bhi1);
    const bool hx_on = tile && j < ny, hy_on = tile && i < nx;
    const bool xy_box = i >= blo0 && i < bhi0 && j >= blo1 && j < bhi1;
    const bool hx_wall = wx, hy_wall = wy;
    // z range of the soft sources touching this column (empty: klo > khi)
    int src_klo = 1 << 30, src_khi = -1;
    if (col)
        for (int s = 0; s < nsrc; s++) {
            const Src<T> &q = src[s];
            if (q.kind == 1 || (q.kind == 0 && q.i == ((g.per[0] && q.comp != 0 && i == nx) ? 0 : i) &&
                                q.j == ((g.per[1] && q.comp != 1 && j == ny) ? 0 : j))) {
                src_klo = min(src_klo, q.k);
                src_khi = max(src_khi, q.k);
                if (g.per[2] && q.k == 0) src_khi = max(src_khi, nz);
            }
        }
    const T fh0 = f.fh0;

    // ---- next-plane register set
    T nhx, nhy, nhz, nhym, nhzm, nhxj, nhzj, neo0, neo1, neo2, ncb0, ncb1, ncb2, nca0, nca1, nca2, nz0, nz1;
    auto fetch = [&](int k) {
        const int ck = cell_nb(g, 2, k);
        const bool kin = k <= k1;
        const unsigned kz = (unsigned)max(ck, 0) * XY, kn = (unsigned)k * XY;
        const bool ckok = ck >= 0 && kin;
        nhx = (hx_ok && ckok) ? Ho.p[0][ohx + kz] : T(0);
        nhy = (hy_ok && ckok) ? Ho.p[1][ohy + kz] : T(0);
        nhz = (hz_ok && kin) ? Ho.p[2][ohz + kn] : T(0);
        nhym = (hym_ok && ckok) ? Ho.p[1][ohym + kz] : T(0);
        nhzm = (hzm_ok && kin) ? Ho.p[2][ohzm + kn] : T(0);
        nhxj = (hxj_ok && ckok) ? Ho.p[0][ohxj + kz] : T(0);
        nhzj = (hzj_ok && kin) ? Ho.p[2][ohzj + kn] : T(0);
        const unsigned q = qc + kn;
        const bool ok = col && kin;
        neo0 = (ok && ex_has) ? Eo.p[0][q] : T(0);
        neo1 = (ok && ey_has) ? Eo.p[1][q] : T(0);
        neo2 = (ok && k < nz) ? Eo.p[2][q] : T(0);
        ncb0 = (ok && ex_has) ? f.cb[0][q] : T(0);
        ncb1 = (ok && ey_has) ? f.cb[1][q] : T(0);
        ncb2 = (ok && k < nz) ? f.cb[2][q] : T(0);
        if (GEN) {
            nca0 = (f.ca[0] && ok && ex_has) ? f.ca[0][q] : T(1);
            nca1 = (f.ca[1] && ok && ey_has) ? f.ca[1][q] : T(1);
            nca2 = (f.ca[2] && ok && k < nz) ? f.ca[2][q] : T(1);
        } else {
            nca0 = nca1 = nca2 = T(1);
        }
        if (PMLK) {
            const bool pz = ok && pml_e_plane(g, k);
            nz0 = (pz && ex_has) ? Zo.p[0][q] : T(0);
            nz1 = (pz && ey_has) ? Zo.p[1][q] : T(0);
        } else {
            nz0 = nz1 = T(0);
        }
    };

    T hx_prev = T(0), hy_prev = T(0), ex_prev = T(0), ey_prev = T(0);
    {
        const int ckm = cell_nb(g, 2, k0 - 1);
        const unsigned kz = (unsigned)max(ckm, 0) * XY;
        hx_prev = (hx_ok && ckm >= 0) ? Ho.p[0][ohx + kz] : T(0);
        hy_prev = (hy_ok && ckm >= 0) ? Ho.p[1][ohy + kz] : T(0);
    }
    fetch(k0);
    T acc = T(0);        // sum of everything written: NaN/Inf propagate into it
    int b = 0;
    for (int k = k0; k <= k1; k++, b ^= 1) {
        // ---- stage H^(n+1/2) of plane k; take this plane's registers
        const T hx = nhx, hy = nhy, hz = nhz;
        const T eo0 = neo0, eo1 = neo1, eo2 = neo2, cb0 = ncb0, cb1 = ncb1, cb2 = ncb2;
        const T ca0 = nca0, ca1 = nca1, ca2 = nca2, zo0 = nz0, zo1 = nz1;
        sH[b][0][ty + 1][tx + 1] = hx;
        sH[b][1][ty + 1][tx + 1] = hy;
        sH[b][2][ty + 1][tx + 1] = hz;
        if (tx == 0) {
            sH[b][1][ty + 1][0] = nhym;
            sH[b][2][ty + 1][0] = nhzm;
        }
        if (ty == 0) {
            sH[b][0][0][tx + 1] = nhxj;
            sH[b][2][0][tx + 1] = nhzj;
        }
        fetch(k + 1);
        __syncthreads();

        // ---- E^(n+1) at plane k (Ex, Ey) and layer k (Ez)
        const bool own_plane = k < k1 || last_chunk;
        const bool wz = wall_node(g, 2, k);
        const bool pml = PMLK && pml_e_plane(g, k);
        const unsigned q = qc + (unsigned)k * XY;
        T J0 = T(0), J1 = T(0), J2 = T(0);
        if (k >= src_klo && k <= src_khi) {
            J0 = j_source(g, f, src, nsrc, 0, i, j, k);
            J1 = j_source(g, f, src, nsrc, 1, i, j, k);
            J2 = j_source(g, f, src, nsrc, 2, i, j, k);
        }
        T ex = T(0), ey = T(0), ez = T(0);
        T zn0 = T(0), zn1 = T(0);
        if (ex_on && !wz) {
            const T rest = (hz - sH[b][2][ty][tx + 1]) * idy;
            const T zp = -(hy - hy_prev) * idz;
            if (pml) {
                const T h = f.dampE[k];
                zn0 = (ca0 * (zo0 * h) + cb0 * zp) * h;
                ex = ca0 * (eo0 - zo0) + cb0 * (rest - J0) + zn0;
            } else {
                ex = ca0 * eo0 + cb0 * (rest + zp - J0);
            }
        }
        if (ey_on && !wz) {
            const T zp = (hx - hx_prev) * idz;
            const T rest = -(hz - sH[b][2][ty + 1][tx]) * idx;
            if (pml) {
                const T h = f.dampE[k];
                zn1 = (ca1 * (zo1 * h) + cb1 * zp) * h;
                ey = ca1 * (eo1 - zo1) + cb1 * (rest - J1) + zn1;
            } else {
                ey = ca1 * eo1 + cb1 * (rest + zp - J1);
            }
        }
        if (ez_on && k < nz) {
            const T rest = (hy - sH[b][1][ty + 1][tx]) * idx - (hx - sH[b][0][ty][tx + 1]) * idy;
            ez = ca2 * eo2 + cb2 * (rest - J2);
        }
        if (tile && own_plane) {
            if (ex_has) En.p[0][q] = ex;
            if (ey_has) En.p[1][q] = ey;
            if (k < nz) En.p[2][q] = ez;
            if (pml) {
                if (ex_has) Zn.p[0][q] = zn0;
                if (ey_has) Zn.p[1][q] = zn1;
            }
            acc += ex + ey + ez;
        }
        sE[b][0][ty][tx] = ex;
        sE[b][1][ty][tx] = ey;
        sEz[b][ty][tx] = ez;
        __syncthreads();

        // ---- H for the tile: Hz at plane k, Hx and Hy at layer k-1
        if (own_plane && (hz_on || (hz_box && !(k >= blo2 && k < bhi2)))) {
            T v = T(0);
            if (!wz) {
                const T cz = (sE[b][1][ty][tx + 1] - ey) * idx - (sE[b][0][ty + 1][tx] - ex) * idy;
                const T fh = (GEN && f.fh[2]) ? f.fh[2][q] : fh0;
                v = hz - fh * cz;
                if (nhalf == 2) v = v - fh * cz;
            }
            Hn.p[2][q] = v;
            acc += v;
        }
        if (k > k0) {
            const int kl = k - 1;
            const unsigned ql = q - XY;
            const bool inbox = xy_box && kl >= blo2 && kl < bhi2;
            const bool hp = PMLK && pml_h_plane(g, kl);
            const int pb = b ^ 1;
            if (hx_on && !inbox) {      // Hx (i, j+1/2, k-1/2)
                T v = T(0);
                if (!hx_wall) {
                    const T rest = (sEz[pb][ty + 1][tx] - sEz[pb][ty][tx]) * idy;
                    const T zp = -(ey - ey_prev) * idz;
                    const T fh = (GEN && f.fh[0]) ? f.fh[0][ql] : fh0;
                    if (hp) {
                        const T h = f.dampH[kl];
                        T hzp = f.Hzp[0][ql];
                        T hr = hx_prev - hzp;
                        for (int s = 0; s < nhalf; s++) {
                            hzp = (hzp * h - fh * zp) * h;
                            hr = hr - fh * rest;
                        }
                        f.Hzp[0][ql] = hzp;
                        v = hr + hzp;
                    } else {
                        v = hx_prev - fh * (rest + zp);
                        if (nhalf == 2) v = v - fh * (rest + zp);
                    }
                } else if (hp) {
                    f.Hzp[0][ql] = T(0);
                }
                Hn.p[0][ql] = v;
                acc += v;
            }
            if (hy_on && !inbox) {      // Hy (i+1/2, j, k-1/2)
                T v = T(0);
                if (!hy_wall) {
                    const T zp = (ex - ex_prev) * idz;
                    const T rest = -(sEz[pb][ty][tx + 1] - sEz[pb][ty][tx]) * idx;
                    const T fh = (GEN && f.fh[1]) ? f.fh[1][ql] : fh0;
                    if (hp) {
                        const T h = f.dampH[kl];
                        T hzp = f.Hzp[1][ql];
                        T hr = hy_prev - hzp;
                        for (int s = 0; s < nhalf; s++) {
                            hzp = (hzp * h - fh * zp) * h;
                            hr = hr - fh * rest;
                        }
                        f.Hzp[1][ql] = hzp;
                        v = hr + hzp;
                    } else {
                        v = hy_prev - fh * (rest + zp);
                        if (nhalf == 2) v = v - fh * (rest + zp);
                    }
                } else if (hp) {
                    f.Hzp[1][ql] = T(0);
                }
                Hn.p[1][ql] = v;
                acc += v;
            }
        }
        hx_prev = hx;
        hy_prev = hy;
        ex_prev = ex;
        ey_prev = ey;
    }
    if (!isfinite(acc)) atomicOr(f.err, kErrNonFinite);
}

} // namespace mmx

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
template <typename T>
__global__ void __launch_bounds__(256) k_h_update(const __grid_constant__ Geo g,
                                                  const __grid_constant__ Fields<T> f, int blo0, int blo1,
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
        f.H[d][q] = v;
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

// Bounded grid-wide barrier for a cooperative launch (all blocks resident).
// Returns false (and latches kErrTimeout) if the others did not arrive
// within ~2^31 clock cycles.
__device__ __forceinline__ bool grid_barrier(unsigned int *bar, int *err)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int *vgen = bar + 1;
        unsigned int gen = *vgen;
        __threadfence();
        unsigned int arrived = atomicAdd(bar, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long t0 = clock64();
            while (*vgen == gen) {
                __nanosleep(64);
                if (clock64() - t0 > (1LL << 31)) {
                    atomicOr(err, kErrTimeout);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok && !(*(volatile int *)err & kErrTimeout);
    }
    __syncthreads();
    return s_ok != 0;
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

// All blocks read the reduced residual after the barrier; thread 0 decides.
__device__ __forceinline__ bool residual_below(const unsigned long long *slot, double tol)
{
    __shared__ int s_conv;
    if (threadIdx.x == 0)
        s_conv = __longlong_as_double((long long)*(volatile const unsigned long long *)slot) < tol;
    __syncthreads();
    return s_conv != 0;
}

struct FaceOf {
    int d, i, j, k;
    long long l;
};

template <typename T>
__device__ __forceinline__ bool box_face(const Geo &g, const Box<T> &b, long long t, FaceOf &fo)
{
    fo.d = (int)(t / b.nb);
    fo.l = t - (long long)fo.d * b.nb;
    int bi = (int)(fo.l % b.bx);
    int bj = (int)((fo.l / b.bx) % b.by);
    int bk = (int)(fo.l / ((long long)b.bx * b.by));
    fo.i = b.lo[0] + bi;
    fo.j = b.lo[1] + bj;
    fo.k = b.lo[2] + bk;
    if (fo.i > g.n[0] || fo.j > g.n[1] || fo.k > g.n[2]) return false;
    return face_valid(g, fo.d, fo.i, fo.j, fo.k);
}

// H vector at face (d; i, j, k): own normal value and the four-point means of
// the two transverse families (Sec. 3.1), from the padded global H (mode 0)
// or from box-local iterates (mode 1).
template <typename T>
__device__ __forceinline__ void h_vector(const Geo &g, const Box<T> &b, T *const Hg[3], T *const Hb[3],
                                         int mode, int d, int i, int j, int k, T h[3])
{
    int ix[3] = {i, j, k};
    h[d] = mode == 0 ? Hg[d][gidx(g, i, j, k)] : Hb[d][bidx(b.lo, b.bx, b.by, i, j, k)];
#pragma unroll
    for (int t = 0; t < 3; t++) {
        if (t == d) continue;
        T sum = T(0);
        int cnt = 0;
#pragma unroll
        for (int od = -1; od <= 0; od++) {
            int nd = cell_nb(g, d, ix[d] + od);
            if (nd < 0) continue;
#pragma unroll
            for (int ot = 0; ot <= 1; ot++) {
                int q[3] = {ix[0], ix[1], ix[2]};
                q[d] = nd;
                q[t] = ix[t] + ot;
                sum += mode == 0 ? Hg[t][gidx(g, q[0], q[1], q[2])]
                                 : Hb[t][bidx(b.lo, b.bx, b.by, q[0], q[1], q[2])];
                cnt++;
            }
        }
        h[t] = sum * (cnt == 4 ? T(0.25) : T(0.5));
    }
}

// One H/M half step on every face of the magnetic box (Sec. 3.2.2 Step 1 or
// Step 3) with the E in f.E, from H^n in Hin to H^(n+1/2) in Hout (the same
// array for the in-place plain path).  Phase 0 forms Cp = H^n - dt/(2 mu0)
// curl E, beta, e0 and the first iterate on magnetic faces and the final H
// on non-magnetic ones; each further iteration r updates every magnetic face
// from the neighbours' iterate r-1 (Jacobi), reduces
// max |DeltaM^r - DeltaM^(r-1)|/Ms into res[r] (warp shuffle, block max, one
// atomicMax on the FP64 bit pattern per block) and meets at a bounded grid
// barrier; all blocks then read res[r] and stop together at the first r with
// res[r] < tol (or at max_iter, latching kErrNotConverged).  Returns false
// if a barrier timed out.
template <typename T>
__device__ bool hm_half_step(const Geo &g, const Fields<T> &f, const Box<T> &b, const T *Hin, T *const Hout[3],
                             unsigned long long *res)
{
    const long long F = 3 * b.nb;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const T h0[3] = {(T)b.h0[0], (T)b.h0[1], (T)b.h0[2]};
    T *const Hb0[3] = {b.Hit[0][0], b.Hit[0][1], b.Hit[0][2]};
    T *const Hg[3] = {const_cast<T *>(Hin) , nullptr, nullptr};
    (void)Hg;

    // ---- phase 0: r = 1
    T rmax = T(0);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < F; t += stride) {
        FaceOf fo;
        if (!box_face(g, b, t, fo)) continue;
        const int d = fo.d;
        const long long l = fo.l;
        T Ms = b.ms[d][l];
        if (!(Ms > T(0))) {
            T v = h_face_nonmag(g, f, d, fo.i, fo.j, fo.k, f.H[d]);
            b.Hit[0][d][l] = v;
            b.Hit[1][d][l] = v;
            continue;
        }
        T rest, zp;
        curl_e(g, f.E, f.inv_d, d, fo.i, fo.j, fo.k, rest, zp);
        size_t q = gidx(g, fo.i, fo.j, fo.k);
        T cp = f.H[d][q] - b.cfar * (rest + zp);
        T Mn[3] = {b.M[3 * d][l], b.M[3 * d + 1][l], b.M[3 * d + 2][l]};
        T e0 = norm_defect(Ms, Mn[0], Mn[1], Mn[2]);
        T h[3], heff[3];
        h_vector(g, b, f.H, Hb0, 0, d, fo.i, fo.j, fo.k, h);
#pragma unroll
        for (int c = 0; c < 3; c++) heff[c] = h0[c] + h[c];
        T dM[3], dMh;
        T k1 = b.k1[d][l], k2 = b.k2[d][l];
        if (b.order == 2) {
            T beta[3] = {-k1 * (Mn[1] * heff[2] - Mn[2] * heff[1]), -k1 * (Mn[2] * heff[0] - Mn[0] * heff[2]),
                         -k1 * (Mn[0] * heff[1] - Mn[1] * heff[0])};
            llg_iterate(Mn, beta, heff, k1, k2, Ms, e0, d, dM, dMh);
            for (int c = 0; c < 3; c++) b.beta[3 * d + c][l] = beta[c];
        } else {
            llg_euler(Mn, heff, k1, k2, Ms, e0, d, dM, dMh);
        }
        b.Cp[d][l] = cp;
        b.e0[d][l] = e0;
        bool wall = wall_node(g, d, d == 0 ? fo.i : d == 1 ? fo.j : fo.k);
        b.Hit[1][d][l] = wall ? T(0) : cp - dMh;
        T amax = T(0);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            b.dM[1][3 * d + c][l] = dM[c];
            amax = max(amax, abs(dM[c]));
        }
        rmax = max(rmax, amax / Ms);
    }
    rmax = block_max(rmax);
    publish_residual(&res[1], rmax);
    if (!grid_barrier(b.bar, b.err)) return false;

    int r = 1;
    bool conv = residual_below(&res[1], b.tol) || b.order == 1;
    while (!conv && r < b.max_iter) {
        r++;
        const int pr = (r - 1) & 1, cr = r & 1;
        T *const Hprev[3] = {b.Hit[pr][0], b.Hit[pr][1], b.Hit[pr][2]};
        rmax = T(0);
        for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < F; t += stride) {
            FaceOf fo;
            if (!box_face(g, b, t, fo)) continue;
            const int d = fo.d;
            const long long l = fo.l;
            T Ms = b.ms[d][l];
            if (!(Ms > T(0))) continue;
            T Mn[3] = {b.M[3 * d][l], b.M[3 * d + 1][l], b.M[3 * d + 2][l]};
            T beta[3] = {b.beta[3 * d][l], b.beta[3 * d + 1][l], b.beta[3 * d + 2][l]};
            T h[3], heff[3];
            h_vector(g, b, f.H, Hprev, 1, d, fo.i, fo.j, fo.k, h);
#pragma unroll
            for (int c = 0; c < 3; c++) heff[c] = h0[c] + h[c];
            T dM[3], dMh;
            llg_iterate(Mn, beta, heff, b.k1[d][l], b.k2[d][l], Ms, b.e0[d][l], d, dM, dMh);
            bool wall = wall_node(g, d, d == 0 ? fo.i : d == 1 ? fo.j : fo.k);
            b.Hit[cr][d][l] = wall ? T(0) : b.Cp[d][l] - dMh;
            T amax = T(0);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                T prev = b.dM[pr][3 * d + c][l];
                b.dM[cr][3 * d + c][l] = dM[c];
                amax = max(amax, abs(dM[c] - prev));
            }
            rmax = max(rmax, amax / Ms);
        }
        rmax = block_max(rmax);
        publish_residual(&res[r], rmax);
        if (!grid_barrier(b.bar, b.err)) return false;
        conv = residual_below(&res[r], b.tol);
    }

    // ---- write back H (all box faces) and M (magnetic faces)
    const int fr = r & 1;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < F; t += stride) {
        FaceOf fo;
        if (!box_face(g, b, t, fo)) continue;
        const int d = fo.d;
        const long long l = fo.l;
        T v = b.Hit[fr][d][l];
        Hout[d][gidx(g, fo.i, fo.j, fo.k)] = v;
        bool bad = !isfinite(v);
        if (b.ms[d][l] > T(0)) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                T m = b.M[3 * d + c][l] + b.dM[fr][3 * d + c][l];
                b.M[3 * d + c][l] = m;
                bad |= !isfinite(m);
            }
        }
        if (bad) atomicOr(b.err, kErrNonFinite);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (!conv && b.order == 2) atomicOr(b.err, kErrNotConverged);
        unsigned long long hs = *b.halfsteps;
        b.iterlog[hs % kIterLogCap] = r;
        *b.halfsteps = hs + 1;
        *b.last_res = b.order == 2 ? __longlong_as_double((long long)res[r]) : 0.0;
    }
    return true;
}

// Cooperative launch over the magnetic box: nsub = 1 runs one H/M half step
// from f.H into Hout; nsub = 2 runs Step 3 of step n and Step 1 of step n+1
// back to back (both use the same E^(n+1)), the second reading the first's
// result.  Residual words: launch parity `slot` uses rows 2 slot and
// 2 slot + 1 of res and clears the other parity's rows for the next launch.
template <typename T>
__global__ void __launch_bounds__(256) k_hm_box(const __grid_constant__ Geo g,
                                                const __grid_constant__ Fields<T> f,
                                                const __grid_constant__ Box<T> b, Ptr3<T> Hout, int nsub,
                                                int slot)
{
    const int W = kMaxIter + 1;
    if (blockIdx.x == 0) {
        unsigned long long *other = b.res + 2 * (1 - slot) * W;
        for (int r = threadIdx.x; r < 2 * W; r += blockDim.x) other[r] = 0ull;
    }
    if (!hm_half_step(g, f, b, f.H[0], Hout.p, b.res + 2 * slot * W)) return;
    if (nsub == 2) {
        if (!grid_barrier(b.bar, b.err)) return;
        Fields<T> f2 = f;
        for (int a = 0; a < 3; a++) f2.H[a] = Hout.p[a];
        hm_half_step(g, f2, b, f2.H[0], Hout.p, b.res + (2 * slot + 1) * W);
    }
}

// ========================================================== fused pass

// Values of one column at one z plane that the fused pass loads ahead.
template <typename T> struct ColPlane {
    T hx, hy, hz;          // H^(n+1/2): Hx, Hy of layer k, Hz of plane k
    T hy_m, hz_m;          // column i-1 (loaded by tx == 0)
    T hx_jm, hz_jm;        // row j-1 (loaded by ty == 0)
    T eo[3];               // E^n of Ex, Ey (plane k), Ez (layer k)
    T cb[3], ca[3];        // E coefficients
    T zo[2];               // PML z parts of Ex, Ey (old buffer)
};

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
// tile; the next plane's column values are loaded into registers before the
// first barrier so their latency overlaps this plane's work.  The chunk's
// last iteration k = k1 recomputes the next chunk's E plane without writing.
template <typename T, int BX, int BY>
__global__ void __launch_bounds__(BX *BY) k_fused(const __grid_constant__ Geo g, const __grid_constant__ Fields<T> f,
                                                 Ptr3<T> Eo, Ptr3<T> Ho, Ptr3<T> En, Ptr3<T> Hn, Ptr3<T> Zo,
                                                 Ptr3<T> Zn, const Src<T> *__restrict__ src, int nsrc, int nhalf,
                                                 int chunk, int blo0, int blo1, int blo2, int bhi0, int bhi1,
                                                 int bhi2)
{
    __shared__ T sH[3][BY + 1][BX + 1];
    __shared__ T sE[2][BY][BX];
    __shared__ T sEz[2][BY][BX];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.x * (BX - 1) + tx;
    const int j = blockIdx.y * (BY - 1) + ty;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int k0 = blockIdx.z * chunk;
    const int k1 = min(k0 + chunk, nz);
    const bool last_chunk = k1 == nz;
    const int kend = k1;                     // inclusive
    const bool halo = tx == BX - 1 || ty == BY - 1;
    const bool col = i <= nx && j <= ny;     // a node column of the grid
    const T idx = f.inv_d[0], idy = f.inv_d[1], idz = f.inv_d[2];
    // wrapped cell-centred indices of this column (-1: outside a wall)
    const int ci = cell_nb(g, 0, i), cj = cell_nb(g, 1, j);
    const int cim = cell_nb(g, 0, i - 1), cjm = cell_nb(g, 1, j - 1);
    const bool has_ex = i < nx, has_ey = j < ny;

    auto loadH = [&](int c, int ii, int jj, int kk) -> T {
        if (ii < 0 || jj < 0 || kk < 0) return T(0);
        return Ho.p[c][gidx(g, ii, jj, kk)];
    };
    auto fetch = [&](int k, ColPlane<T> &v) {
        const int ck = cell_nb(g, 2, k);
        v.hx = v.hy = v.hz = v.hy_m = v.hz_m = v.hx_jm = v.hz_jm = T(0);
        v.eo[0] = v.eo[1] = v.eo[2] = T(0);
        v.cb[0] = v.cb[1] = v.cb[2] = T(0);
        v.ca[0] = v.ca[1] = v.ca[2] = T(1);
        v.zo[0] = v.zo[1] = T(0);
        if (!col || k > kend) return;
        v.hx = loadH(0, i, cj, ck);
        v.hy = loadH(1, ci, j, ck);
        v.hz = loadH(2, ci, cj, k);
        if (tx == 0) {
            v.hy_m = loadH(1, cim, j, ck);
            v.hz_m = loadH(2, cim, cj, k);
        }
        if (ty == 0) {
            v.hx_jm = loadH(0, i, cjm, ck);
            v.hz_jm = loadH(2, ci, cjm, k);
        }
        const size_t q = gidx(g, i, j, k);
        if (has_ex) { v.eo[0] = Eo.p[0][q]; v.cb[0] = f.cb[0][q]; if (f.ca[0]) v.ca[0] = f.ca[0][q]; }
        if (has_ey) { v.eo[1] = Eo.p[1][q]; v.cb[1] = f.cb[1][q]; if (f.ca[1]) v.ca[1] = f.ca[1][q]; }
        if (k < nz) { v.eo[2] = Eo.p[2][q]; v.cb[2] = f.cb[2][q]; if (f.ca[2]) v.ca[2] = f.ca[2][q]; }
        if (pml_e_plane(g, k)) {
            if (has_ex) v.zo[0] = Zo.p[0][q];
            if (has_ey) v.zo[1] = Zo.p[1][q];
        }
    };

    // H of layer k0-1 in this column (for E at plane k0)
    T hx_prev = T(0), hy_prev = T(0), ex_prev = T(0), ey_prev = T(0);
    if (col) {
        int ckm = cell_nb(g, 2, k0 - 1);
        hx_prev = loadH(0, i, cj, ckm);
        hy_prev = loadH(1, ci, j, ckm);
    }
    ColPlane<T> cur, nxt;
    fetch(k0, cur);
    int zb = 0;
    for (int k = k0; k <= kend; k++) {
        // ---- stage H^(n+1/2) of plane k
        sH[0][ty + 1][tx + 1] = cur.hx;
        sH[1][ty + 1][tx + 1] = cur.hy;
        sH[2][ty + 1][tx + 1] = cur.hz;
        if (tx == 0) {
            sH[1][ty + 1][0] = cur.hy_m;
            sH[2][ty + 1][0] = cur.hz_m;
        }
        if (ty == 0) {
            sH[0][0][tx + 1] = cur.hx_jm;
            sH[2][0][tx + 1] = cur.hz_jm;
        }
        // ---- issue the next plane's loads (consumed next iteration)
        fetch(k + 1, nxt);
        __syncthreads();

        // ---- E^(n+1) at plane k (Ex, Ey) and layer k (Ez)
        const bool own_plane = k < k1 || last_chunk;
        T ex = T(0), ey = T(0), ez = T(0);
        if (col) {
            const size_t q = gidx(g, i, j, k);
            const bool wx = wall_node(g, 0, i), wy = wall_node(g, 1, j), wz = wall_node(g, 2, k);
            const bool pml = pml_e_plane(g, k);
            if (has_ex && !wy && !wz) {
                T rest = (sH[2][ty + 1][tx + 1] - sH[2][ty][tx + 1]) * idy;
                T zp = -(sH[1][ty + 1][tx + 1] - hy_prev) * idz;
                T J = nsrc ? j_source(g, f, src, nsrc, 0, i, j, k) : T(0);
                if (pml) {
                    T h = f.dampE[k];
                    T ez1 = (cur.ca[0] * (cur.zo[0] * h) + cur.cb[0] * zp) * h;
                    ex = cur.ca[0] * (cur.eo[0] - cur.zo[0]) + cur.cb[0] * (rest - J) + ez1;
                    if (!halo && own_plane) Zn.p[0][q] = ez1;
                } else {
                    ex = cur.ca[0] * cur.eo[0] + cur.cb[0] * (rest + zp - J);
                }
            } else if (pml && has_ex && !halo && own_plane) {
                Zn.p[0][q] = T(0);
            }
            if (has_ey && !wx && !wz) {
                T zp = (sH[0][ty + 1][tx + 1] - hx_prev) * idz;
                T rest = -(sH[2][ty + 1][tx + 1] - sH[2][ty + 1][tx]) * idx;
                T J = nsrc ? j_source(g, f, src, nsrc, 1, i, j, k) : T(0);
                if (pml) {
                    T h = f.dampE[k];
                    T ez1 = (cur.ca[1] * (cur.zo[1] * h) + cur.cb[1] * zp) * h;
                    ey = cur.ca[1] * (cur.eo[1] - cur.zo[1]) + cur.cb[1] * (rest - J) + ez1;
                    if (!halo && own_plane) Zn.p[1][q] = ez1;
                } else {
                    ey = cur.ca[1] * cur.eo[1] + cur.cb[1] * (rest + zp - J);
                }
            } else if (pml && has_ey && !halo && own_plane) {
                Zn.p[1][q] = T(0);
            }
            if (k < nz && !wx && !wy) {
                T rest = (sH[1][ty + 1][tx + 1] - sH[1][ty + 1][tx]) * idx
                       - (sH[0][ty + 1][tx + 1] - sH[0][ty][tx + 1]) * idy;
                T J = nsrc ? j_source(g, f, src, nsrc, 2, i, j, k) : T(0);
                ez = cur.ca[2] * cur.eo[2] + cur.cb[2] * (rest - J);
            }
            if (!halo && own_plane) {
                if (has_ex) En.p[0][q] = ex;
                if (has_ey) En.p[1][q] = ey;
                if (k < nz) En.p[2][q] = ez;
                if (!(isfinite(ex) && isfinite(ey) && isfinite(ez))) atomicOr(f.err, kErrNonFinite);
            }
        }
        sE[0][ty][tx] = ex;
        sE[1][ty][tx] = ey;
        sEz[zb][ty][tx] = ez;
        __syncthreads();

        // ---- H for the tile: Hz at plane k, Hx and Hy at layer k-1
        if (col && !halo) {
            if (own_plane && has_ex && has_ey) {
                const bool inbox = i >= blo0 && i < bhi0 && j >= blo1 && j < bhi1 && k >= blo2 && k < bhi2;
                if (!inbox) {
                    const size_t q = gidx(g, i, j, k);
                    T v = T(0);
                    if (!wall_node(g, 2, k)) {
                        T cz = (sE[1][ty][tx + 1] - sE[1][ty][tx]) * idx - (sE[0][ty + 1][tx] - sE[0][ty][tx]) * idy;
                        T fh = f.fh[2] ? f.fh[2][q] : f.fh0;
                        v = sH[2][ty + 1][tx + 1] - fh * cz;
                        if (nhalf == 2) v = v - fh * cz;
                    }
                    Hn.p[2][q] = v;
                    if (!isfinite(v)) atomicOr(f.err, kErrNonFinite);
                }
            }
            if (k > k0) {
                const int kl = k - 1;
                const size_t q = gidx(g, i, j, kl);
                const bool inbox = i >= blo0 && i < bhi0 && j >= blo1 && j < bhi1 && kl >= blo2 && kl < bhi2;
                const bool pml = pml_h_plane(g, kl);
                if (has_ey && !inbox) {      // Hx (i, j+1/2, k-1/2)
                    T v = T(0);
                    if (!wall_node(g, 0, i)) {
                        T rest = (sEz[zb ^ 1][ty + 1][tx] - sEz[zb ^ 1][ty][tx]) * idy;
                        T zp = -(sE[1][ty][tx] - ey_prev) * idz;
                        T fh = f.fh[0] ? f.fh[0][q] : f.fh0;
                        if (pml) {
                            T h = f.dampH[kl];
                            T hzp = f.Hzp[0][q];
                            T hr = hx_prev - hzp;
                            for (int s = 0; s < nhalf; s++) {
                                hzp = (hzp * h - fh * zp) * h;
                                hr = hr - fh * rest;
                            }
                            f.Hzp[0][q] = hzp;
                            v = hr + hzp;
                        } else {
                            v = hx_prev - fh * (rest + zp);
                            if (nhalf == 2) v = v - fh * (rest + zp);
                        }
                    } else if (pml) {
                        f.Hzp[0][q] = T(0);
                    }
                    Hn.p[0][q] = v;
                    if (!isfinite(v)) atomicOr(f.err, kErrNonFinite);
                }
                if (has_ex && !inbox) {      // Hy (i+1/2, j, k-1/2)
                    T v = T(0);
                    if (!wall_node(g, 1, j)) {
                        T zp = (sE[0][ty][tx] - ex_prev) * idz;
                        T rest = -(sEz[zb ^ 1][ty][tx + 1] - sEz[zb ^ 1][ty][tx]) * idx;
                        T fh = f.fh[1] ? f.fh[1][q] : f.fh0;
                        if (pml) {
                            T h = f.dampH[kl];
                            T hzp = f.Hzp[1][q];
                            T hr = hy_prev - hzp;
                            for (int s = 0; s < nhalf; s++) {
                                hzp = (hzp * h - fh * zp) * h;
                                hr = hr - fh * rest;
                            }
                            f.Hzp[1][q] = hzp;
                            v = hr + hzp;
                        } else {
                            v = hy_prev - fh * (rest + zp);
                            if (nhalf == 2) v = v - fh * (rest + zp);
                        }
                    } else if (pml) {
                        f.Hzp[1][q] = T(0);
                    }
                    Hn.p[1][q] = v;
                    if (!isfinite(v)) atomicOr(f.err, kErrNonFinite);
                }
            }
        }
        // ---- roll the column registers and the Ez buffers
        hx_prev = cur.hx;
        hy_prev = cur.hy;
        ex_prev = ex;
        ey_prev = ey;
        zb ^= 1;
        cur = nxt;
        __syncthreads();
    }
}

} // namespace mmx

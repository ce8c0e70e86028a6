// mmx_kernels.cuh -- CUDA kernels of the coupled Maxwell-LLG step for
// sm_103a: setup (cell -> edge/face averaging, coefficients, initial M), the
// streaming E and H updates, and the cooperative H/M kernel of the magnetic
// box with the device-side residual reduction and loop control.
#pragma once
#include "mmx_device.cuh"

namespace mmx {

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
                                                  const Src<T> *__restrict__ src, int nsrc, long long step)
{
    int i, j, k;
    if (!node_of_thread(g, i, j, k)) return;
    double t = ((double)step + 0.5) * g.dt;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        if (!edge_valid(g, c, i, j, k)) continue;
        double J = nsrc ? j_source(g, src, nsrc, c, i, j, k, t) : 0.0;
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
        if (!isfinite((double)v)) atomicOr(f.err, kErrNonFinite);
    }
}

// Hard sources (Sec. 3.2): overwrite one field value with g(t).
template <typename T> struct Ptr3 {
    T *p[3];
};

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

__device__ __forceinline__ double block_max(double v)
{
    __shared__ double s_part[32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) s_part[w] = v;
    __syncthreads();
    if (w == 0) {
        int nw = (blockDim.x + 31) >> 5;
        v = l < nw ? s_part[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;   // valid in thread 0
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
// Step 3, whichever E is current).  Cooperative launch: phase 0 forms
// Cp = H^n - dt/(2 mu0) curl E, beta, e0 and the first iterate for magnetic
// faces and the final H for non-magnetic ones; each further iteration r
// updates every magnetic face from the neighbours' iterate r-1 (Jacobi),
// reduces max |DeltaM^r - DeltaM^(r-1)|/Ms into res[r] (warp shuffle, block
// max, one atomicMax on the FP64 bit pattern per block) and meets at a
// bounded grid barrier; all blocks then read res[r] and stop together at the
// first r with res[r] < tol (or at max_iter, latching kErrNotConverged).
template <typename T>
__global__ void __launch_bounds__(256) k_hm_box(const __grid_constant__ Geo g,
                                                const __grid_constant__ Fields<T> f,
                                                const __grid_constant__ Box<T> b, int slot)
{
    unsigned long long *res = b.res + slot * (kMaxIter + 1);
    if (blockIdx.x == 0) {
        unsigned long long *other = b.res + (1 - slot) * (kMaxIter + 1);
        for (int r = threadIdx.x; r <= kMaxIter; r += blockDim.x) other[r] = 0ull;
    }
    const long long F = 3 * b.nb;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const T h0[3] = {(T)b.h0[0], (T)b.h0[1], (T)b.h0[2]};
    T *const Hb0[3] = {b.Hit[0][0], b.Hit[0][1], b.Hit[0][2]};
    T *const Hb1[3] = {b.Hit[1][0], b.Hit[1][1], b.Hit[1][2]};

    // ---- phase 0: r = 1
    double rmax = 0.0;
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
        curl_e(g, f.E, d, fo.i, fo.j, fo.k, rest, zp);
        size_t q = gidx(g, fo.i, fo.j, fo.k);
        T cp = f.H[d][q] - b.cfar * (rest + zp);
        T Mn[3] = {b.M[3 * d][l], b.M[3 * d + 1][l], b.M[3 * d + 2][l]};
        double md = (double)Mn[0] * Mn[0] + (double)Mn[1] * Mn[1] + (double)Mn[2] * Mn[2];
        T e0 = (T)((double)Ms * (double)Ms - md);
        T h[3], heff[3];
        h_vector(g, b, f.H, Hb0, 0, d, fo.i, fo.j, fo.k, h);
#pragma unroll
        for (int c = 0; c < 3; c++) heff[c] = h0[c] + h[c];
        T dM[3];
        T k1 = b.k1[d][l], k2 = b.k2[d][l];
        if (b.order == 2) {
            T beta[3] = {-k1 * (Mn[1] * heff[2] - Mn[2] * heff[1]), -k1 * (Mn[2] * heff[0] - Mn[0] * heff[2]),
                         -k1 * (Mn[0] * heff[1] - Mn[1] * heff[0])};
            llg_iterate(Mn, beta, heff, k1, k2, Ms, e0, dM);
            for (int c = 0; c < 3; c++) b.beta[3 * d + c][l] = beta[c];
        } else {
            llg_euler(Mn, heff, k1, k2, Ms, e0, dM);
        }
        b.Cp[d][l] = cp;
        b.e0[d][l] = e0;
        bool wall = wall_node(g, d, d == 0 ? fo.i : d == 1 ? fo.j : fo.k);
        b.Hit[1][d][l] = wall ? T(0) : cp - dM[d];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            b.dM[1][3 * d + c][l] = dM[c];
            rmax = fmax(rmax, fabs((double)dM[c]) / (double)Ms);
        }
    }
    rmax = block_max(rmax);
    if (threadIdx.x == 0 && rmax > 0.0) atomicMax(&res[1], (unsigned long long)__double_as_longlong(rmax));
    if (!grid_barrier(b.bar, b.err)) return;

    int r = 1;
    bool conv = b.order == 1 || __longlong_as_double((long long)*(volatile unsigned long long *)&res[1]) < b.tol;
    while (!conv && r < b.max_iter) {
        r++;
        const int pr = (r - 1) & 1, cr = r & 1;
        T *const Hprev[3] = {b.Hit[pr][0], b.Hit[pr][1], b.Hit[pr][2]};
        rmax = 0.0;
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
            T dM[3];
            llg_iterate(Mn, beta, heff, b.k1[d][l], b.k2[d][l], Ms, b.e0[d][l], dM);
            bool wall = wall_node(g, d, d == 0 ? fo.i : d == 1 ? fo.j : fo.k);
            b.Hit[cr][d][l] = wall ? T(0) : b.Cp[d][l] - dM[d];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                T prev = b.dM[pr][3 * d + c][l];
                b.dM[cr][3 * d + c][l] = dM[c];
                rmax = fmax(rmax, fabs((double)dM[c] - (double)prev) / (double)Ms);
            }
        }
        rmax = block_max(rmax);
        if (threadIdx.x == 0 && rmax > 0.0) atomicMax(&res[r], (unsigned long long)__double_as_longlong(rmax));
        if (!grid_barrier(b.bar, b.err)) return;
        conv = __longlong_as_double((long long)*(volatile unsigned long long *)&res[r]) < b.tol;
    }

    // ---- write back H (all box faces) and M (magnetic faces)
    const int fr = r & 1;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < F; t += stride) {
        FaceOf fo;
        if (!box_face(g, b, t, fo)) continue;
        const int d = fo.d;
        const long long l = fo.l;
        T v = b.Hit[fr][d][l];
        f.H[d][gidx(g, fo.i, fo.j, fo.k)] = v;
        bool bad = !isfinite((double)v);
        if (b.ms[d][l] > T(0)) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                T m = b.M[3 * d + c][l] + b.dM[fr][3 * d + c][l];
                b.M[3 * d + c][l] = m;
                bad |= !isfinite((double)m);
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
}

} // namespace mmx

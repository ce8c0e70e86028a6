// mmx_device.cuh -- device-side data structures and per-point arithmetic of
// the coupled Maxwell-LLG scheme (Yao, Jambunathan, Zeng & Nonaka,
// arXiv 2103.12819, Sec. 3) for sm_103a.  Everything here is templated on
// the storage/arithmetic type T (double or float).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mmx {

// CODATA 2018 mu0 and the exact speed of light.
constexpr double kMu0 = 1.25663706212e-6;
constexpr double kC0 = 299792458.0;
constexpr double kPi = 3.14159265358979323846;

constexpr int kMaxIter = 64;
constexpr int kMaxSources = 32;
constexpr int kIterLogCap = 65536;

// Latched device status bits.
constexpr int kErrNotConverged = 1;
constexpr int kErrNonFinite = 2;
constexpr int kErrTimeout = 4;
constexpr int kErrBadInput = 8;

// Grid geometry.  All Yee arrays share one padded layout: element (i, j, k)
// at i + X*(j + Y*k) with X = nx+1 rounded up to a multiple of 8 and
// Y = ny+1, so a neighbour is +-1, +-X or +-X*Y for every component.
struct Geo {
    int n[3];
    int X, Y;
    int per[3];        // 1 on a periodic axis
    int npml;          // PML cells at each z end (0: none)
    double dt;
    double inv_d[3];
    double d[3];
};

__device__ __forceinline__ size_t gidx(const Geo &g, int i, int j, int k)
{
    return (size_t)i + (size_t)g.X * ((size_t)j + (size_t)g.Y * (size_t)k);
}

// Cell-centred neighbour index along axis a (idx in [-1, n]): wrapped on a
// periodic axis, -1 outside a non-periodic one.
__device__ __forceinline__ int cell_nb(const Geo &g, int a, int idx)
{
    int n = g.n[a];
    if (idx < 0) return g.per[a] ? idx + n : -1;
    if (idx >= n) return g.per[a] ? idx - n : -1;
    return idx;
}

__device__ __forceinline__ bool wall_node(const Geo &g, int a, int idx)
{
    return !g.per[a] && (idx == 0 || idx == g.n[a]);
}

// z planes inside the PML: E (nodal in z) at node k, H x/y faces at k+1/2.
__device__ __forceinline__ bool pml_e_plane(const Geo &g, int k)
{
    return g.npml > 0 && (k < g.npml || k > g.n[2] - g.npml);
}
__device__ __forceinline__ bool pml_h_plane(const Geo &g, int k)
{
    return g.npml > 0 && (k < g.npml || k >= g.n[2] - g.npml);
}

template <typename T> struct Src {
    int kind, comp, i, j, k;
    double amp, f0, tp, t0;
};

// Field storage: S is the stored type of E, H and their PML split parts, T
// the arithmetic type.  FP16 storage (S = __half, T = float) holds each value
// divided by a per-field scale (sE for E, sH for H) so that the fields sit in
// FP16's range; ld_s / st_s convert.  With S = T the scales are not applied.
__device__ __forceinline__ float ld_s(const __half *p, float sc)
{
    return __half2float(*p) * sc;
}
template <typename T> __device__ __forceinline__ T ld_s(const T *p, T)
{
    return *p;
}
__device__ __forceinline__ void st_s(__half *p, float v, float isc)
{
    *p = __float2half_rn(v * isc);
}
template <typename T> __device__ __forceinline__ void st_s(T *p, T v, T)
{
    *p = v;
}

template <typename T, typename S = T> struct Fields {
    S *E[3];
    S *H[3];
    S *Ezp[2];          // z-derivative parts of Ex, Ey in the PML (else null)
    S *Hzp[2];          // z-derivative parts of Hx, Hy in the PML (else null)
    const T *ca[3];     // E update: E' = ca E + cb (curl H - J); ca null -> 1
    const T *cb[3];
    const T *fh[3];     // H update: H' = H - fh curl E; fh null -> fh0
    T fh0;
    const T *dampE;     // per z node: exp(-sigma_z dt/(2 eps0)) (PML planes)
    const T *dampH;     // per z cell: exp(-sigma_z dt/(4 eps0))
    T inv_d[3];         // 1/dx, 1/dy, 1/dz in T (no FP64 in FP32 kernels)
    const T *src_amp;   // g(t) of every source for the current step
    const T *prof[2];   // TE10 profile sin(pi x/W): [0] at x = i dx, [1] at (i+1/2) dx
    int *err;
    T sE, sH, isE, isH; // storage scales and their inverses (FP16 storage only)
    const T *epsc;      // FP32 arithmetic: eps_r per cell in the padded layout (1 in
                        // the padding), from which the vectorised kernel forms cb
    T kcb;              // 4 dt / eps0: cb = kcb / (sum of the edge's four cells' eps_r)
};

// Magnetic box: the bounding box of the magnetic faces grown by one face on
// every side (so every neighbour a magnetic face reads lies inside), stored
// box-locally with dims (bx, by, bz), element (i,j,k) at
// (i-lo0) + bx*((j-lo1) + by*(k-lo2)).
// Four values of one magnetic face, moved as one 16-byte (FP32) or two
// 16-byte (FP64) accesses.
template <typename T> struct alignas(4 * sizeof(T)) Q4 {
    T x, y, z, w;
};

template <typename T> struct Box {
    int lo[3];
    int bx, by, bz;
    long long nb;
    T *M[9];            // M per face family: M[3*fam + comp] (box layout)
    T *Hit[2][3];       // H iterates (box layout; neighbours read them)
    T *Hit2[2][3];      // H iterates of the second half step of a launch
    // per magnetic face, in the order of the magnetic-face list:
    const Q4<T> *cst;   // Ms, k1, k2, 1/Ms
    Q4<T> *mn;          // M^n (w unused)
    Q4<T> *bc;          // beta = -kappa M^n x Heff^n, C' = H^n - dt/(2 mu0) curl E
    Q4<T> *dm[2];       // iterates of DeltaM = M^r - M^n; w: e0 = Ms^2 - |M^n|^2
    const T *ms[3];     // Ms on faces
    const T *k1[3];     // order 2: kappa = mu0|gamma|dt/4; order 1: (dt/2) mu0 gamma_L
    const T *k2[3];     // order 2: alpha/Ms;               order 1: (dt/2) alpha mu0 gamma_L / Ms
    double h0[3];
    double tol;
    int max_iter;
    int order;
    T cfar;             // dt/(2 mu0)
    unsigned long long *res;   // [8][kMaxIter+1]: residual bit patterns, then decision words
    unsigned long long *bar;   // grid barrier: monotonic arrival count
    int *iterlog;
    unsigned long long *halfsteps;
    double *last_res;
    int *err;
    // work lists: {box index | family << 30, i, j, k} of the magnetic faces
    // and of the other (non-magnetic) faces of the box
    const int4 *mag;
    const int4 *nonmag;
    // the magnetic list's first words alone (box index | family << 30): the
    // list-driven kernel rebuilds i, j, k from the box index, reading 4 bytes
    // per face and phase instead of 16
    const unsigned *mag32;
    int nmag, nnon;
};

__device__ __forceinline__ size_t bidx(const int lo[3], int bx, int by, int i, int j, int k)
{
    return (size_t)(i - lo[0]) + (size_t)bx * ((size_t)(j - lo[1]) + (size_t)by * (size_t)(k - lo[2]));
}

// 32-bit forms for the box kernel (box and grid below 2^32 elements)
__device__ __forceinline__ unsigned bidx32(const int lo[3], int bx, int by, int i, int j, int k)
{
    return (unsigned)(i - lo[0]) + (unsigned)bx * ((unsigned)(j - lo[1]) + (unsigned)by * (unsigned)(k - lo[2]));
}

__device__ __forceinline__ unsigned gidx32(const Geo &g, int i, int j, int k)
{
    return (unsigned)i + (unsigned)g.X * ((unsigned)j + (unsigned)g.Y * (unsigned)k);
}

// ---------------------------------------------------------------- curls

// (curl H) on an E edge split into the z-derivative part and the rest
// (Sec. 3.1: 2nd-order central differences of the face values).
template <typename T>
__device__ __forceinline__ void curl_h(const Geo &g, T *const H[3], const T inv_d[3], int c, int i, int j,
                                       int k, T &rest, T &zp)
{
    const T idx = inv_d[0], idy = inv_d[1], idz = inv_d[2];
    if (c == 0) {
        int jm = cell_nb(g, 1, j - 1), jp = cell_nb(g, 1, j);
        int km = cell_nb(g, 2, k - 1), kp = cell_nb(g, 2, k);
        rest = (H[2][gidx(g, i, jp, k)] - H[2][gidx(g, i, jm, k)]) * idy;
        zp = -(H[1][gidx(g, i, j, kp)] - H[1][gidx(g, i, j, km)]) * idz;
    } else if (c == 1) {
        int im = cell_nb(g, 0, i - 1), ip = cell_nb(g, 0, i);
        int km = cell_nb(g, 2, k - 1), kp = cell_nb(g, 2, k);
        zp = (H[0][gidx(g, i, j, kp)] - H[0][gidx(g, i, j, km)]) * idz;
        rest = -(H[2][gidx(g, ip, j, k)] - H[2][gidx(g, im, j, k)]) * idx;
    } else {
        int im = cell_nb(g, 0, i - 1), ip = cell_nb(g, 0, i);
        int jm = cell_nb(g, 1, j - 1), jp = cell_nb(g, 1, j);
        rest = (H[1][gidx(g, ip, j, k)] - H[1][gidx(g, im, j, k)]) * idx
             - (H[0][gidx(g, i, jp, k)] - H[0][gidx(g, i, jm, k)]) * idy;
        zp = T(0);
    }
}

// (curl E) on an H face of family d, split the same way.
template <typename T, typename S>
__device__ __forceinline__ void curl_e(const Geo &g, S *const E[3], const T inv_d[3], int d, int i, int j,
                                       int k, T &rest, T &zp, T sE = T(1))
{
    const T idx = inv_d[0], idy = inv_d[1], idz = inv_d[2];
    auto e = [&](int c, int a, int b2, int c2) { return ld_s(E[c] + gidx(g, a, b2, c2), sE); };
    if (d == 0) {
        rest = (e(2, i, j + 1, k) - e(2, i, j, k)) * idy;
        zp = -(e(1, i, j, k + 1) - e(1, i, j, k)) * idz;
    } else if (d == 1) {
        zp = (e(0, i, j, k + 1) - e(0, i, j, k)) * idz;
        rest = -(e(2, i + 1, j, k) - e(2, i, j, k)) * idx;
    } else {
        rest = (e(1, i + 1, j, k) - e(1, i, j, k)) * idx - (e(0, i, j + 1, k) - e(0, i, j, k)) * idy;
        zp = T(0);
    }
}

// The same for the face at 32-bit padded index q (grids below 2^32
// elements): its four edges are q plus one-element, row or plane offsets,
// with the operations of curl_e in the same order.
template <typename T, typename S>
__device__ __forceinline__ void curl_e32(const Geo &g, S *const E[3], const T inv_d[3], int d, unsigned q, T &rest,
                                         T &zp, T sE = T(1))
{
    const unsigned X = (unsigned)g.X, XY = (unsigned)g.X * (unsigned)g.Y;
    const T idx = inv_d[0], idy = inv_d[1], idz = inv_d[2];
    if (d == 0) {
        rest = (ld_s(E[2] + q + X, sE) - ld_s(E[2] + q, sE)) * idy;
        zp = -(ld_s(E[1] + q + XY, sE) - ld_s(E[1] + q, sE)) * idz;
    } else if (d == 1) {
        zp = (ld_s(E[0] + q + XY, sE) - ld_s(E[0] + q, sE)) * idz;
        rest = -(ld_s(E[2] + q + 1u, sE) - ld_s(E[2] + q, sE)) * idx;
    } else {
        rest = (ld_s(E[1] + q + 1u, sE) - ld_s(E[1] + q, sE)) * idx - (ld_s(E[0] + q + X, sE) - ld_s(E[0] + q, sE)) * idy;
        zp = T(0);
    }
}

// ------------------------------------------------------------ sources

__device__ __forceinline__ double waveform(double amp, double f0, double tp, double t0, double t)
{
    double u = t - t0;
    return amp * exp(-u * u / (2.0 * tp * tp)) * cos(2.0 * kPi * f0 * t);
}

// Soft J on edge (c, i, j, k) for the current step: point sources and
// TE10-shaped plane sources (profile sin(pi x / W) across x), with the
// waveform value of each source precomputed for the step.  Indices on
// periodic axes are compared modulo n so that a duplicate node receives the
// same current.
template <typename T, typename S>
__device__ __forceinline__ T j_source_a(const Geo &g, const Fields<T, S> &f, const T *amp, const Src<T> *src,
                                        int nsrc, int c, int i, int j, int k);

template <typename T, typename S>
__device__ __forceinline__ T j_source(const Geo &g, const Fields<T, S> &f, const Src<T> *src, int nsrc, int c,
                                      int i, int j, int k)
{
    return j_source_a(g, f, f.src_amp, src, nsrc, c, i, j, k);
}

// The same with this step's source amplitudes amp[s] given explicitly.
template <typename T, typename S>
__device__ __forceinline__ T j_source_a(const Geo &g, const Fields<T, S> &f, const T *amp, const Src<T> *src,
                                        int nsrc, int c, int i, int j, int k)
{
    T J = T(0);
    int ci = (g.per[0] && c != 0 && i == g.n[0]) ? 0 : i;
    int cj = (g.per[1] && c != 1 && j == g.n[1]) ? 0 : j;
    int ck = (g.per[2] && c != 2 && k == g.n[2]) ? 0 : k;
    for (int s = 0; s < nsrc; s++) {
        const Src<T> &q = src[s];
        if (q.comp != c) continue;
        if (q.kind == 0) {
            if (q.i == ci && q.j == cj && q.k == ck) J += amp[s];
        } else if (q.kind == 1) {
            if (q.k == ck) J += amp[s] * f.prof[c == 0 ? 1 : 0][ci];
        }
    }
    return J;
}

// ------------------------------------------------ Step 2: the E update

// E^(n+1) = ca E^n + cb (curl H^(n+1/2) - J^(n+1/2)), ca = (eps/dt - s/2)/
// (eps/dt + s/2), cb = 1/(eps/dt + s/2) (Sec. 3.2.1, Step 2); PEC edges are
// held at zero; in the z-PML the z part is damped before and after its
// update (time-centred split field).
template <typename T>
__device__ __forceinline__ void e_edge(const Geo &g, const Fields<T> &f, int c, int i, int j, int k, T J)
{
    size_t q = gidx(g, i, j, k);
    bool wall = (c != 0 && wall_node(g, 0, i)) || (c != 1 && wall_node(g, 1, j)) ||
                (c != 2 && wall_node(g, 2, k));
    if (wall) {
        f.E[c][q] = T(0);
        if (c < 2 && f.Ezp[c]) f.Ezp[c][q] = T(0);
        return;
    }
    T rest, zp;
    curl_h(g, f.H, f.inv_d, c, i, j, k, rest, zp);
    T ca = f.ca[c] ? f.ca[c][q] : T(1);
    T cb = f.cb[c][q];
    T v;
    if (c < 2 && pml_e_plane(g, k)) {
        T h = f.dampE[k];
        T ez = f.Ezp[c][q];
        T er = f.E[c][q] - ez;
        T ez1 = (ca * (ez * h) + cb * zp) * h;
        T er1 = ca * er + cb * (rest - J);
        f.Ezp[c][q] = ez1;
        v = er1 + ez1;
    } else {
        v = ca * f.E[c][q] + cb * (rest + zp - J);
    }
    f.E[c][q] = v;
    if (!isfinite(v)) atomicOr(f.err, kErrNonFinite);
}

// ------------------------------------------- Steps 1/3: non-magnetic faces

// H^(n+1/2) = H^n - dt/(2 mu) curl E (Eq. iterate_H with mu for mu0, Ms = 0),
// PEC wall faces zero, time-centred z-PML split.  Reads Hin, writes Hout
// (the same array for the streaming kernel).
// The same with the old value hn passed in (the box kernel's second half
// step takes it from its box-local iterate).
template <typename T, typename S>
__device__ __forceinline__ T h_face_nonmag_val(const Geo &g, const Fields<T, S> &f, int d, int i, int j, int k,
                                               T hn)
{
    size_t q = gidx(g, i, j, k);
    int ix[3] = {i, j, k};
    if (wall_node(g, d, ix[d])) {
        if (d < 2 && f.Hzp[d]) st_s(f.Hzp[d] + q, T(0), f.isH);
        return T(0);
    }
    T rest, zp;
    curl_e(g, f.E, f.inv_d, d, i, j, k, rest, zp, f.sE);
    T fh = f.fh[d] ? f.fh[d][q] : f.fh0;
    T v;
    if (d < 2 && pml_h_plane(g, k)) {
        T h = f.dampH[k];
        T hz = ld_s(f.Hzp[d] + q, f.sH);
        T hr = hn - hz;
        T hz1 = (hz * h - fh * zp) * h;
        T hr1 = hr - fh * rest;
        st_s(f.Hzp[d] + q, hz1, f.isH);
        v = hr1 + hz1;
    } else {
        v = hn - fh * (rest + zp);
    }
    return v;
}

template <typename T, typename S>
__device__ __forceinline__ T h_face_nonmag(const Geo &g, const Fields<T, S> &f, int d, int i, int j, int k,
                                           const S *Hin)
{
    return h_face_nonmag_val(g, f, d, i, j, k, ld_s(Hin + gidx(g, i, j, k), f.sH));
}

// ------------------------------------------------ LLG: one iterate

// e0 = Ms^2 - |M^n|^2, the norm defect of the stored M^n that N() removes.
// |M^n| equals Ms up to rounding, so this is a difference of two nearly equal
// ~1e10 numbers; FP64: every square is split exactly with an FMA
// (a*a = p + e) and the eight terms are summed with Neumaier compensation;
// FP32: the float products are exact in FP64.
__device__ __forceinline__ void two_sum_acc(double &s, double &c, double x)
{
    double t = s + x;
    c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
    s = t;
}

__device__ __forceinline__ double norm_defect(double Ms, double mx, double my, double mz)
{
    double v[4] = {Ms, mx, my, mz};
    double s = 0.0, c = 0.0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        double p = v[q] * v[q];
        double e = fma(v[q], v[q], -p);
        double sg = q == 0 ? 1.0 : -1.0;
        two_sum_acc(s, c, sg * p);
        two_sum_acc(s, c, sg * e);
    }
    return s + c;
}

__device__ __forceinline__ void two_sum_accf(float &s, float &c, float x)
{
    float t = s + x;
    c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
}

// FP32 path: the same exact splitting with FMA in float; the compensated
// sum keeps e0 to ~1e-14 relative to Ms^2, which FP64 would also give,
// without FP64 instructions (1/64 of the FP32 rate on this part).
__device__ __forceinline__ float norm_defect(float Ms, float mx, float my, float mz)
{
    float v[4] = {Ms, mx, my, mz};
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        float p = v[q] * v[q];
        float e = fmaf(v[q], v[q], -p);
        float sg = q == 0 ? 1.f : -1.f;
        two_sum_accf(s, c, sg * p);
        two_sum_accf(s, c, sg * e);
    }
    return s + c;
}

// The quotient and square root of the FP32 LLG solve in the hardware's
// approximate forms (reciprocal and square root to about 2 ulp).  Their
// error enters the increment delta and the N() correction relative to
// those small terms, not relative to |M|; FP64 keeps the IEEE forms.
template <typename T> __device__ __forceinline__ T llg_rcp(T x)
{
    return T(1) / x;
}
template <> __device__ __forceinline__ float llg_rcp<float>(float x)
{
    return __fdividef(1.0f, x);
}
template <typename T> __device__ __forceinline__ T llg_sqrt(T x)
{
    return sqrt(x);
}
template <> __device__ __forceinline__ float llg_sqrt<float>(float x)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// N(M^n + delta) - M^n without cancellation against |M| ~ Ms:
// DeltaM = delta + (delta + M^n)(s - 1), s - 1 = q/(|x|(Ms + |x|)),
// q = Ms^2 - |x|^2 = e0 - 2 M^n.delta - |delta|^2.  The H update (Eq.
// iterate_H) takes the change along the sphere through the stored M^n
// (the same with e0 = 0): component d of it is returned in dMh, so the
// rounding of the stored M^n, which N() also removes, does not enter H.
template <typename T>
__device__ __forceinline__ void renormalised_increment(const T Mn[3], const T del[3], T Ms, T e0, int d,
                                                       T dM[3], T &dMh)
{
    T md = Mn[0] * del[0] + Mn[1] * del[1] + Mn[2] * del[2];
    T dd = del[0] * del[0] + del[1] * del[1] + del[2] * del[2];
    T q0 = -(T(2) * md + dd);
    T qv = e0 + q0;
    T xn = llg_sqrt(Ms * Ms - qv);
    T den = llg_rcp(xn * (Ms + xn));
    T sm1 = qv * den;
#pragma unroll
    for (int c = 0; c < 3; c++) dM[c] = del[c] + (del[c] + Mn[c]) * sm1;
    dMh = del[d] + (del[d] + Mn[d]) * (q0 * den);
}

// One solve of the trapezoidal LLG step (Eqs. llg_tra4-llg_tra6) written for
// the increment.  With b = M^n + beta, beta = -kappa M^n x Heff^n and
// a = -(u + s M^n), u = kappa Heff^(r-1), s = alpha/Ms, the closed form
// x = (b + (a.b) a - a x b)/(1+|a|^2) gives
//   delta = x - M^n = (beta + (a.b) a - |a|^2 M^n - a x b)/(1+|a|^2).
// a is dominated by its damping part s M^n, parallel to M^n; expanding
//   (a.b) a - |a|^2 M^n = (p + s m2 + q) u + (s q - s p - |u|^2) M^n,
//   a x b = -(u x M^n + u x beta + s M^n x beta),
// with p = u.M^n, q = (u + s M^n).beta, m2 = |M^n|^2 = Ms^2 - e0, drops the
// terms that cancel identically (M^n x M^n and the s^2 m2 pair), so every
// remaining term is small and keeps its relative precision (FP32 included).
// N(x) = x Ms/|x| then gives DeltaM = delta + (delta + M^n)(s_N - 1) with
// s_N - 1 = q'/(|x|(Ms + |x|)), q' = Ms^2 - |x|^2 = e0 - 2 M^n.delta - |delta|^2.
template <typename T>
__device__ __forceinline__ void llg_iterate(const T Mn[3], const T beta[3], const T heff[3], T kap,
                                            T s, T Ms, T e0, int d, T dM[3], T &dMh)
{
    T u[3] = {kap * heff[0], kap * heff[1], kap * heff[2]};
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
    renormalised_increment(Mn, del, Ms, e0, d, dM, dMh);
}

// First-order scheme (Sec. 3.2.1, Steps 1/3): forward Euler of Eq. LLG_scalar
// over the half step, delta = -c1 M^n x H - c2 M^n x (M^n x H), then N().
template <typename T>
__device__ __forceinline__ void llg_euler(const T Mn[3], const T heff[3], T c1, T c2, T Ms, T e0, int d,
                                          T dM[3], T &dMh)
{
    T mxh[3] = {Mn[1] * heff[2] - Mn[2] * heff[1], Mn[2] * heff[0] - Mn[0] * heff[2],
                Mn[0] * heff[1] - Mn[1] * heff[0]};
    T mxmxh[3] = {Mn[1] * mxh[2] - Mn[2] * mxh[1], Mn[2] * mxh[0] - Mn[0] * mxh[2],
                  Mn[0] * mxh[1] - Mn[1] * mxh[0]};
    T del[3];
#pragma unroll
    for (int c = 0; c < 3; c++) del[c] = -c1 * mxh[c] - c2 * mxmxh[c];
    renormalised_increment(Mn, del, Ms, e0, d, dM, dMh);
}

} // namespace mmx

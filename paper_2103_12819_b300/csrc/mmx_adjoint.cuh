// mmx_adjoint.cuh -- discrete adjoint of the second-order scheme (Sec. 3.2:
// H/M half step, E update with the time-centred split-field z-PML, H/M half
// step) for grids without periodic axes, with respect to eps_r of every cell
// and to the bias H0, for the loss
//   L = sum_n dt P(E^n, H^n),   P = sum (Ex <Hy>_z - Ey <Hx>_z) dx dy
// through a z node plane (the flux monitor's formula).  Every electromagnetic
// kernel is the exact transpose of its forward counterpart, written as a
// gather so that no atomics are needed: the adjoint of a curl is collected
// per edge (or face) from the per-face (per-edge) adjoint curl parts it fed.
//
// Notation per location: lam* are adjoints (dL/d value) of the state after
// an update on entry and before it on exit; fR/fZ (eR/eZ) the adjoints of
// the curl parts a face (edge) update consumed, in the padded layout, zero
// where no face (edge) exists.
//
// The magnetic half of each H half step (Sec. 3.2.2, Steps 1 and 3) is
// transposed through its converged fixed point rather than iterate by
// iterate.  On a magnetic face the half step solves
//   M = N(X(a(Heff(H)), b)),  H_perp = C' + M^n_perp - M_perp,
// with X(a, b) = (b + (a.b) a - a x b)/(1 + |a|^2) (Eqs. llg_tra4-6),
// a = -(kappa Heff + alpha/Ms M^n), b = M^n - kappa M^n x Heff^n, and the
// Jacobi iteration only finds that fixed point; by the implicit-function
// theorem the adjoint mu of M solves the transposed linear system
//   mu = gM + (dM/dM)^T mu,  gM = lamM - e_perp lamH_perp,
// which the same Jacobi sweep solves (same contraction: the transpose of the
// forward linearisation).  The transposed four-point means of Sec. 3.1 are
// gathers over the faces that read a given face (weights 1/4, or 1/2 next to
// a wall).  The loss does not see the norm |M| (M stays on the sphere), so
// the on-sphere H increment of the forward path and H = C' + M^n - M agree
// on every perturbation that occurs.
#pragma once
#include "mmx_kernels.cuh"

namespace mmx {

template <typename T> struct AdjState {
    T *lE[3];
    T *lH[3];
    T *lEz[2];        // adjoint of the PML split part of Ex, Ey (null without PML)
    T *lHz[2];        // adjoint of the PML split part of Hx, Hy
    T *fR[3], *fZ[3]; // per face family
    T *eR[3], *eZ[3]; // per edge component
    double *gcb[3];   // dL/dcb per edge, accumulated over the steps
    double *gca[3];   // dL/dca per edge
};

// Transpose of one H half step on every face (k_h_update with no box):
// H' = H - fh (R + Z), or in a PML plane hz' = (hz h - fh Z) h,
// H' = (H - hz) - fh R + hz'; wall faces are zero.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_h(const Geo g, const Fields<T> f, AdjState<T> a)
{
    int i, j, k;
    if (!node_of_thread(g, i, j, k)) return;
    const int ix[3] = {i, j, k};
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (!face_valid(g, d, i, j, k)) continue;
        const size_t q = gidx(g, i, j, k);
        if (wall_node(g, d, ix[d])) {
            a.lH[d][q] = T(0);
            if (d < 2 && a.lHz[d]) a.lHz[d][q] = T(0);
            a.fR[d][q] = T(0);
            a.fZ[d][q] = T(0);
            continue;
        }
        const T fh = f.fh[d] ? f.fh[d][q] : f.fh0;
        const T lh = a.lH[d][q];
        if (d < 2 && pml_h_plane(g, k)) {
            const T h = f.dampH[k];
            const T lz = a.lHz[d][q];
            a.lHz[d][q] = (h * h - T(1)) * lh + h * h * lz;
            a.fR[d][q] = -fh * lh;
            a.fZ[d][q] = -fh * h * (lh + lz);
        } else {
            a.fR[d][q] = -fh * lh;
            a.fZ[d][q] = -fh * lh;
        }
        // lH[d][q] stays lh: dH'/dH = 1 in both branches
    }
}

// lE += curl_e^T (fR, fZ): every E edge collects what the faces whose curl
// it entered owe it (curl_e of Sec. 3.1, split in rest / z parts).
template <typename T> __global__ void __launch_bounds__(256) k_adj_curl_e(const Geo g, AdjState<T> a)
{
    int i, j, k;
    if (!node_of_thread(g, i, j, k)) return;
    const T idx = (T)g.inv_d[0], idy = (T)g.inv_d[1], idz = (T)g.inv_d[2];
    const size_t q = gidx(g, i, j, k);
    const size_t X = g.X, XY = (size_t)g.X * g.Y;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    // Ex (i+1/2, j, k): Z of face y (i, j, k) and (i, j, k-1); R of face z (i, j, k) and (i, j-1, k)
    if (i < nx) {
        T v = T(0);
        if (k < nz) v -= a.fZ[1][q] * idz;
        if (k > 0) v += a.fZ[1][q - XY] * idz;
        if (j < ny) v += a.fR[2][q] * idy;
        if (j > 0) v -= a.fR[2][q - X] * idy;
        a.lE[0][q] += v;
    }
    // Ey (i, j+1/2, k): Z of face x (i, j, k), (i, j, k-1); R of face z (i, j, k), (i-1, j, k)
    if (j < ny) {
        T v = T(0);
        if (k < nz) v += a.fZ[0][q] * idz;
        if (k > 0) v -= a.fZ[0][q - XY] * idz;
        if (i < nx) v -= a.fR[2][q] * idx;
        if (i > 0) v += a.fR[2][q - 1] * idx;
        a.lE[1][q] += v;
    }
    // Ez (i, j, k+1/2): R of face x (i, j, k), (i, j-1, k); R of face y (i, j, k), (i-1, j, k)
    if (k < nz) {
        T v = T(0);
        if (j < ny) v -= a.fR[0][q] * idy;
        if (j > 0) v += a.fR[0][q - X] * idy;
        if (i < nx) v += a.fR[1][q] * idx;
        if (i > 0) v -= a.fR[1][q - 1] * idx;
        a.lE[2][q] += v;
    }
}

// Transpose of the E update on every edge (k_e_update), given the H^(n+1/2)
// it used (Hh), E^n and the PML part ez^n it started from (E0, Z0) and this
// step's source amplitudes; accumulates dL/dcb and dL/dca.
template <typename T>
__global__ void __launch_bounds__(256)
    k_adj_e(const Geo g, const Fields<T> f, Ptr3<T> Hh, Ptr3<T> E0, Ptr3<T> Z0, const Src<T> *__restrict__ src,
            int nsrc, AdjState<T> a)
{
    int i, j, k;
    if (!node_of_thread(g, i, j, k)) return;
    const size_t q = gidx(g, i, j, k);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        if (!edge_valid(g, c, i, j, k)) continue;
        const bool wall = (c != 0 && wall_node(g, 0, i)) || (c != 1 && wall_node(g, 1, j)) ||
                          (c != 2 && wall_node(g, 2, k));
        if (wall) {
            a.lE[c][q] = T(0);
            if (c < 2 && a.lEz[c]) a.lEz[c][q] = T(0);
            a.eR[c][q] = T(0);
            a.eZ[c][q] = T(0);
            continue;
        }
        T rest, zp;
        curl_h(g, Hh.p, f.inv_d, c, i, j, k, rest, zp);
        const T J = nsrc ? j_source(g, f, src, nsrc, c, i, j, k) : T(0);
        const T ca = f.ca[c] ? f.ca[c][q] : T(1);
        const T cb = f.cb[c][q];
        const T le = a.lE[c][q];
        if (c < 2 && pml_e_plane(g, k)) {
            const T h = f.dampE[k];
            const T lz = a.lEz[c][q];
            const T ez = Z0.p[c][q];
            a.lE[c][q] = ca * le;
            a.lEz[c][q] = ca * (h * h - T(1)) * le + ca * h * h * lz;
            a.eR[c][q] = cb * le;
            a.eZ[c][q] = cb * h * (le + lz);
            a.gcb[c][q] += (double)le * (double)(rest - J) + (double)(le + lz) * (double)h * (double)zp;
            a.gca[c][q] += (double)le * (double)(E0.p[c][q] - ez) + (double)(le + lz) * (double)(h * h) * (double)ez;
        } else {
            a.lE[c][q] = ca * le;
            a.eR[c][q] = cb * le;
            a.eZ[c][q] = cb * le;
            a.gcb[c][q] += (double)le * (double)(rest + zp - J);
            a.gca[c][q] += (double)le * (double)E0.p[c][q];
        }
    }
}

// lH += curl_h^T (eR, eZ): every H face collects from the edges whose curl
// it entered (curl_h of Sec. 3.1; wall edges carry zero).
template <typename T> __global__ void __launch_bounds__(256) k_adj_curl_h(const Geo g, AdjState<T> a)
{
    int i, j, k;
    if (!node_of_thread(g, i, j, k)) return;
    const T idx = (T)g.inv_d[0], idy = (T)g.inv_d[1], idz = (T)g.inv_d[2];
    const size_t q = gidx(g, i, j, k);
    const size_t X = g.X, XY = (size_t)g.X * g.Y;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    // Hx (i, j+1/2, k+1/2): Z of Ey (i, j, k), (i, j, k+1); R of Ez (i, j, k), (i, j+1, k)
    if (j < ny && k < nz) {
        T v = a.eZ[1][q] * idz - a.eZ[1][q + XY] * idz;
        v += -a.eR[2][q] * idy + a.eR[2][q + X] * idy;
        a.lH[0][q] += v;
    }
    // Hy (i+1/2, j, k+1/2): Z of Ex (i, j, k), (i, j, k+1); R of Ez (i, j, k), (i+1, j, k)
    if (i < nx && k < nz) {
        T v = -a.eZ[0][q] * idz + a.eZ[0][q + XY] * idz;
        v += a.eR[2][q] * idx - a.eR[2][q + 1] * idx;
        a.lH[1][q] += v;
    }
    // Hz (i+1/2, j+1/2, k): R of Ex (i, j, k), (i, j+1, k); R of Ey (i, j, k), (i+1, j, k)
    if (i < nx && j < ny) {
        T v = a.eR[0][q] * idy - a.eR[0][q + X] * idy;
        v += -a.eR[1][q] * idx + a.eR[1][q + 1] * idx;
        a.lH[2][q] += v;
    }
}

// dL/d(E^n, H^n) of the step's flux term dt P(E^n, H^n) through node plane kp.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_flux(const Geo g, Ptr3<T> E, Ptr3<T> H, int kp, T w, AdjState<T> a)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = p % g.X, j = p / g.X;
    if (j > g.n[1] || i > g.n[0]) return;
    const size_t XY = (size_t)g.X * g.Y;
    const size_t q = (size_t)i + (size_t)g.X * j;
    const int km = kp - 1;
    const bool lo = km >= 0, hi = kp < g.n[2];
    // w = dt dx dy; P = sum Ex <Hy> - Ey <Hx>, <.> the mean of the faces below and above
    if (i < g.n[0]) {
        const T ex = E.p[0][q + kp * XY];
        T hy = T(0);
        if (lo) hy += T(0.5) * H.p[1][q + km * XY];
        if (hi) hy += T(0.5) * H.p[1][q + kp * XY];
        a.lE[0][q + kp * XY] += w * hy;
        if (lo) a.lH[1][q + km * XY] += w * T(0.5) * ex;
        if (hi) a.lH[1][q + kp * XY] += w * T(0.5) * ex;
    }
    if (j < g.n[1]) {
        const T ey = E.p[1][q + kp * XY];
        T hx = T(0);
        if (lo) hx += T(0.5) * H.p[0][q + km * XY];
        if (hi) hx += T(0.5) * H.p[0][q + kp * XY];
        a.lE[1][q + kp * XY] -= w * hx;
        if (lo) a.lH[0][q + km * XY] -= w * T(0.5) * ey;
        if (hi) a.lH[0][q + kp * XY] -= w * T(0.5) * ey;
    }
}

// dL/d eps_r of every cell from dL/dcb, dL/dca of its 12 edges:
// eps_e = eps0 mean(eps_r), cb = 1/(eps_e/dt + sigma_e/2), ca = (eps_e/dt -
// sigma_e/2) cb; dcb/deps_r = -(eps0/dt) cb^2 / cnt, dca/deps_r =
// (eps0/dt) cb (1 - ca) / cnt per edge mean over cnt cells.
__global__ void __launch_bounds__(256)
    k_adj_eps(const Geo g, const double *__restrict__ eps_c, const double *__restrict__ sig_c,
              const double *const *gcb, const double *const *gca, double *grad)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
    if (t >= ncell) return;
    const int ci = (int)(t % g.n[0]), cj = (int)((t / g.n[0]) % g.n[1]), ck = (int)(t / ((long long)g.n[0] * g.n[1]));
    const double eps0 = 1.0 / (kMu0 * kC0 * kC0);
    double s = 0.0;
    for (int c = 0; c < 3; c++) {
        const int a1 = (c + 1) % 3, a2 = (c + 2) % 3;
        for (int o1 = 0; o1 <= 1; o1++)
            for (int o2 = 0; o2 <= 1; o2++) {
                int e[3] = {ci, cj, ck};
                e[a1] += o1;
                e[a2] += o2;
                // the edge's cells: count those that exist
                int cnt = 0;
                for (int p1 = -1; p1 <= 0; p1++)
                    for (int p2 = -1; p2 <= 0; p2++) {
                        const int v1 = e[a1] + p1, v2 = e[a2] + p2;
                        if (v1 >= 0 && v1 < g.n[a1] && v2 >= 0 && v2 < g.n[a2]) cnt++;
                    }
                const double epsm = eps0 * (eps_c ? edge_mean(g, eps_c, c, e[0], e[1], e[2]) : 1.0);
                const double sg = sig_c ? edge_mean(g, sig_c, c, e[0], e[1], e[2]) : 0.0;
                const double cb = 1.0 / (sg / 2.0 + epsm / g.dt);
                const double ca = (epsm / g.dt - sg / 2.0) * cb;
                const size_t q = gidx(g, e[0], e[1], e[2]);
                s += (gcb[c][q] * (-(eps0 / g.dt) * cb * cb) + gca[c][q] * ((eps0 / g.dt) * cb * (1.0 - ca))) / cnt;
            }
    }
    grad[t] = s;
}

// ------------------------------------------------------------ magnetic part

// Scratch of the magnetic adjoint, per face family and component in the box
// layout of the magnetic box (index 3 family + component), zero on faces
// that are not magnetic.
template <typename T> struct AdjMag {
    T *lM[9];    // adjoint of M (after a half step on entry, before it on exit)
    T *gM[9];    // right-hand side gM of the fixed-point adjoint
    T *mu[9];    // its solution, iterated in place
    T *A[9];     // a at the converged iterate
    T *B[9];     // b
    T *lHe[9];   // adjoint of Heff of the iteration: -kappa Ja^T JN^T mu
    T *lHn[9];   // adjoint of Heff^n (the b path): -kappa (lam_b x M^n)
    unsigned long long *res;   // per sweep: max |mu' - mu|, max |mu'| (FP64 bit patterns)
    double *gh0;               // dL/dH0, accumulated
    int *nc;                   // set when a half step's sweeps missed eps
    int kmax;                  // sweeps per half step at most
    double eps;                // stop when max |mu' - mu| <= eps max |mu'|
};

template <typename T> struct MPtr {
    T *p[9];
};

__device__ __forceinline__ bool box_pos(const Geo &g, const int lo[3], int bx, int by, long long nb, long long l,
                                        int ix[3])
{
    if (l >= nb) return false;
    ix[0] = lo[0] + (int)(l % bx);
    ix[1] = lo[1] + (int)((l / bx) % by);
    ix[2] = lo[2] + (int)(l / ((long long)bx * by));
    return true;
}

template <typename T> __device__ __forceinline__ bool in_box(const Box<T> &b, const int ix[3])
{
    return ix[0] >= b.lo[0] && ix[0] < b.lo[0] + b.bx && ix[1] >= b.lo[1] && ix[1] < b.lo[1] + b.by &&
           ix[2] >= b.lo[2] && ix[2] < b.lo[2] + b.bz;
}

// Transpose of the H vector of h_vector (own normal value plus the two
// four-point means) for the face of family t at q: the sum, over the
// magnetic faces whose H_eff reads this face, of their H_eff adjoint L
// (component t) times the weight they read it with.  A face of family
// D != t at ix reads q when q is one of the cells ix[D]-1, ix[D] along D
// and one of the nodes ix[t], ix[t]+1 along t; the weight is 1/4 with both
// cells present, 1/2 at a wall node (non-periodic axes).
template <typename T>
__device__ T adj_gather(const Geo &g, const Box<T> &b, T *const L[9], int t, const int q[3])
{
    T v = L[3 * t + t][bidx(b.lo, b.bx, b.by, q[0], q[1], q[2])];
    for (int D = 0; D < 3; D++) {
        if (D == t) continue;
        for (int od = -1; od <= 0; od++) {
            const int iD = q[D] - od;
            if (iD < 0 || iD > g.n[D]) continue;
            for (int ot = 0; ot <= 1; ot++) {
                const int it = q[t] - ot;
                if (it < 0 || it >= g.n[t]) continue;
                int ix[3] = {q[0], q[1], q[2]};
                ix[D] = iD;
                ix[t] = it;
                if (!in_box(b, ix)) continue;
                const T w = (iD > 0 && iD < g.n[D]) ? T(0.25) : T(0.5);
                v += w * L[3 * D + t][bidx(b.lo, b.bx, b.by, ix[0], ix[1], ix[2])];
            }
        }
    }
    return v;
}

template <typename T> __device__ __forceinline__ void cross3(const T a[3], const T b[3], T o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

template <typename T> __device__ __forceinline__ T dot3(const T a[3], const T b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// x = X(a, b) of Eq. llg_tra4 and the transposed Jacobians of N(x) = Ms x/|x|
// and of X with respect to a and b, applied to the adjoint m of M:
//   lx = JN^T m = (Ms/|x|)(m - xh (xh.m)),
//   la = (b (a.lx) + (a.b) lx - b x lx - 2 (x.lx) a)/(1 + |a|^2),
//   lb = (lx + a (a.lx) + a x lx)/(1 + |a|^2).
template <typename T>
__device__ __forceinline__ void llg_transpose(const T a[3], const T bv[3], T Ms, const T m[3], T la[3], T lb[3])
{
    const T aa = dot3(a, a), ab = dot3(a, bv);
    const T inv = T(1) / (T(1) + aa);
    T axb[3], x[3];
    cross3(a, bv, axb);
    for (int c = 0; c < 3; c++) x[c] = (bv[c] + ab * a[c] - axb[c]) * inv;
    const T r = sqrt(dot3(x, x));
    const T xm = dot3(x, m) / (r * r);
    T lx[3];
    for (int c = 0; c < 3; c++) lx[c] = (Ms / r) * (m[c] - x[c] * xm);
    const T alx = dot3(a, lx), xlx = dot3(x, lx);
    T bxl[3], axl[3];
    cross3(bv, lx, bxl);
    cross3(a, lx, axl);
    for (int c = 0; c < 3; c++) {
        la[c] = (bv[c] * alx + ab * lx[c] - bxl[c] - T(2) * xlx * a[c]) * inv;
        lb[c] = (lx[c] + a[c] * alx + axl[c]) * inv;
    }
}

template <typename T>
__device__ __forceinline__ void heff_at(const Geo &g, const Box<T> &b, T *const H[3], int D, const int ix[3],
                                        T h[3])
{
    if (D == 0)
        h_vector<0>(g, b, H, H, 0, ix[0], ix[1], ix[2], h);
    else if (D == 1)
        h_vector<1>(g, b, H, H, 0, ix[0], ix[1], ix[2], h);
    else
        h_vector<2>(g, b, H, H, 0, ix[0], ix[1], ix[2], h);
    for (int c = 0; c < 3; c++) h[c] += (T)b.h0[c];
}

// Set-up of one magnetic half step's adjoint: a from the H the half step
// ended with (Hs), b from the H and M it started from (Hn, Mn); gM and the
// first sweep's mu = gM; clears the sweep residual words.
template <typename T>
__global__ void __launch_bounds__(256)
    k_adjm_prep(const Geo g, const Box<T> b, Ptr3<T> Hn, MPtr<T> Mn, Ptr3<T> Hs, AdjState<T> a, AdjMag<T> m)
{
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l < 2LL * m.kmax) m.res[l] = 0ull;
    int ix[3];
    if (!box_pos(g, b.lo, b.bx, b.by, b.nb, l, ix)) return;
    for (int D = 0; D < 3; D++) {
        const T Ms = b.ms[D][l];
        if (!(Ms > T(0))) continue;
        const T kap = b.k1[D][l], s = b.k2[D][l];
        T mn[3], hn[3], hs[3], mxh[3];
        for (int c = 0; c < 3; c++) mn[c] = Mn.p[3 * D + c][l];
        heff_at(g, b, Hn.p, D, ix, hn);
        heff_at(g, b, Hs.p, D, ix, hs);
        cross3(mn, hn, mxh);
        const bool wall = wall_node(g, D, ix[D]);
        const T lh = wall ? T(0) : a.lH[D][gidx(g, ix[0], ix[1], ix[2])];
        for (int c = 0; c < 3; c++) {
            m.A[3 * D + c][l] = -(kap * hs[c] + s * mn[c]);
            m.B[3 * D + c][l] = mn[c] - kap * mxh[c];
            const T gv = m.lM[3 * D + c][l] - (c == D ? lh : T(0));
            m.gM[3 * D + c][l] = gv;
            m.mu[3 * D + c][l] = gv;
        }
    }
}

// Has sweep `it - 1` already met the stopping rule?
__device__ __forceinline__ bool adjm_done(const unsigned long long *res, int it, double eps)
{
    if (it < 1) return false;
    const double d = __longlong_as_double((long long)res[2 * (it - 1)]);
    const double mx = __longlong_as_double((long long)res[2 * (it - 1) + 1]);
    return d <= eps * mx;
}

// lHe = -kappa Ja^T JN^T mu on every magnetic face (it < 0: unconditionally).
template <typename T> __global__ void __launch_bounds__(256) k_adjm_heff(const Box<T> b, AdjMag<T> m, int it)
{
    if (it >= 0 && adjm_done(m.res, it, m.eps)) return;
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= b.nb) return;
    for (int D = 0; D < 3; D++) {
        const T Ms = b.ms[D][l];
        if (!(Ms > T(0))) continue;
        T av[3], bv[3], mu[3], la[3], lb[3];
        for (int c = 0; c < 3; c++) {
            av[c] = m.A[3 * D + c][l];
            bv[c] = m.B[3 * D + c][l];
            mu[c] = m.mu[3 * D + c][l];
        }
        llg_transpose(av, bv, Ms, mu, la, lb);
        const T kap = b.k1[D][l];
        for (int c = 0; c < 3; c++) m.lHe[3 * D + c][l] = -kap * la[c];
    }
}

// One Jacobi sweep of the fixed-point adjoint: mu = gM - e_perp (gathered
// lHe)_perp on magnetic faces off the walls (a wall face's H is held at zero,
// so its M does not feed back); residual words of sweep it.
template <typename T>
__global__ void __launch_bounds__(256) k_adjm_sweep(const Geo g, const Box<T> b, AdjMag<T> m, int it)
{
    if (adjm_done(m.res, it, m.eps)) return;
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int ix[3];
    double dmax = 0.0, vmax = 0.0;
    if (box_pos(g, b.lo, b.bx, b.by, b.nb, l, ix)) {
        for (int D = 0; D < 3; D++) {
            if (!(b.ms[D][l] > T(0))) continue;
            const bool wall = wall_node(g, D, ix[D]);
            const T gl = wall ? T(0) : adj_gather(g, b, m.lHe, D, ix);
            for (int c = 0; c < 3; c++) {
                const T v = m.gM[3 * D + c][l] - (c == D ? gl : T(0));
                dmax = fmax(dmax, fabs((double)(v - m.mu[3 * D + c][l])));
                vmax = fmax(vmax, fabs((double)v));
                m.mu[3 * D + c][l] = v;
            }
        }
    }
    dmax = block_max(dmax);
    vmax = block_max(vmax);
    publish_residual(&m.res[2 * it], dmax);
    publish_residual(&m.res[2 * it + 1], vmax);
}

// Close one magnetic half step's adjoint: lH += gathered lHe on every box
// face off the walls (the adjoint of C' on magnetic faces, of the final H
// on the others); lM becomes the adjoint of M^n; lHn the adjoint of Heff^n;
// dL/dH0 collects both H_eff adjoints.  Sets *nc if no sweep met the
// stopping rule.
template <typename T>
__global__ void __launch_bounds__(256)
    k_adjm_close(const Geo g, const Box<T> b, Ptr3<T> Hn, MPtr<T> Mn, AdjState<T> a, AdjMag<T> m)
{
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l == 0) {
        bool conv = false;
        for (int it = 0; it < m.kmax && !conv; it++) conv = adjm_done(m.res, it + 1, m.eps);
        if (!conv) atomicOr(m.nc, 1);
    }
    int ix[3];
    double h0[3] = {0.0, 0.0, 0.0};
    if (box_pos(g, b.lo, b.bx, b.by, b.nb, l, ix)) {
        for (int D = 0; D < 3; D++) {
            if (!face_valid(g, D, ix[0], ix[1], ix[2])) continue;
            const bool wall = wall_node(g, D, ix[D]);
            const size_t q = gidx(g, ix[0], ix[1], ix[2]);
            T lh = T(0);
            if (!wall) {
                lh = a.lH[D][q] + adj_gather(g, b, m.lHe, D, ix);
                a.lH[D][q] = lh;
            }
            const T Ms = b.ms[D][l];
            if (!(Ms > T(0))) continue;
            const T kap = b.k1[D][l], s = b.k2[D][l];
            T av[3], bv[3], mu[3], mn[3], hn[3], la[3], lb[3];
            for (int c = 0; c < 3; c++) {
                av[c] = m.A[3 * D + c][l];
                bv[c] = m.B[3 * D + c][l];
                mu[c] = m.mu[3 * D + c][l];
                mn[c] = Mn.p[3 * D + c][l];
            }
            heff_at(g, b, Hn.p, D, ix, hn);
            llg_transpose(av, bv, Ms, mu, la, lb);
            T hxl[3], lxm[3];
            cross3(hn, lb, hxl);
            cross3(lb, mn, lxm);
            for (int c = 0; c < 3; c++) {
                m.lM[3 * D + c][l] = -s * la[c] + lb[c] - kap * hxl[c] + (c == D ? lh : T(0));
                const T ln = -kap * lxm[c];
                m.lHn[3 * D + c][l] = ln;
                h0[c] += (double)(-kap * la[c]) + (double)ln;
            }
        }
    }
    for (int c = 0; c < 3; c++) {
        __shared__ double part[256];
        part[threadIdx.x] = h0[c];
        __syncthreads();
        for (int h = blockDim.x / 2; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0 && part[0] != 0.0) atomicAdd(&m.gh0[c], part[0]);
        __syncthreads();
    }
}

// After k_adj_h: magnetic faces took C' = H^n - dt/(2 mu0) curl E (mu0, no
// PML split), so their curl adjoints are -dt/(2 mu0) lH; then the b path
// adds the gathered lHn to lH (the adjoint of H^n) on every box face off
// the walls.
template <typename T> __global__ void __launch_bounds__(256) k_adjm_curl(const Geo g, const Box<T> b, AdjState<T> a, AdjMag<T> m)
{
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int ix[3];
    if (!box_pos(g, b.lo, b.bx, b.by, b.nb, l, ix)) return;
    for (int D = 0; D < 3; D++) {
        if (!face_valid(g, D, ix[0], ix[1], ix[2]) || wall_node(g, D, ix[D])) continue;
        const size_t q = gidx(g, ix[0], ix[1], ix[2]);
        if (b.ms[D][l] > T(0)) {
            const T v = -b.cfar * a.lH[D][q];
            a.fR[D][q] = v;
            a.fZ[D][q] = v;
        }
        a.lH[D][q] += adj_gather(g, b, m.lHn, D, ix);
    }
}

} // namespace mmx

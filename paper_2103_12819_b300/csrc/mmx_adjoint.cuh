// mmx_adjoint.cuh -- discrete adjoint of the electromagnetic update of the
// scheme (Sec. 3.2: H half step, E update with the time-centred split-field
// z-PML, H half step) for grids without magnetic material and without
// periodic axes, with respect to eps_r of every cell, for the loss
//   L = sum_n dt P(E^n, H^n),   P = sum (Ex <Hy>_z - Ey <Hx>_z) dx dy
// through a z node plane (the flux monitor's formula).  Every kernel is the
// exact transpose of its forward counterpart, written as a gather so that
// no atomics are needed: the adjoint of a curl is collected per edge (or
// face) from the per-face (per-edge) adjoint curl parts it fed.
//
// Notation per location: lam* are adjoints (dL/d value) of the state after
// an update on entry and before it on exit; fR/fZ (eR/eZ) the adjoints of
// the curl parts a face (edge) update consumed, in the padded layout, zero
// where no face (edge) exists.
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

} // namespace mmx

// mmx_monitor.cuh -- energy and Poynting-flux monitors with FP64
// Neumaier-compensated sums, whatever the storage precision of the fields.
//
// Energy: the discrete electromagnetic energy of the half-step leapfrog,
//   W = 1/2 sum_edges eps E^2 + 1/2 sum_faces mu (H^2 - (dt/(2 mu) curl E)^2),
// with E and H at the same integer time level (H^n the mean of H^(n+-1/2)),
// which the scheme of Sec. 3.2 conserves exactly in lossless, source-free,
// non-magnetic media.  mu is mu0 mu_r on non-magnetic faces and mu0 on
// magnetic ones (Sec. 5.1).
//
// Flux: the Poynting power through the z node plane k,
//   P = sum (Ex <Hy>_z - Ey <Hx>_z) dx dy,
// with each E edge paired with the two H faces above and below it in z
// (no x/y interpolation is needed: Ex and Hy share their x and y position,
// as do Ey and Hx), H taken at the time level of E.
#pragma once
#include "mmx_kernels.cuh"

namespace mmx {

constexpr int kMonitorBlocks = 1184;   // 8 x 148 SMs, grid-stride
constexpr int kMonitorThreads = 256;
constexpr int kMaxFluxPlanes = 4;

// (s, c) += (s2, c2), Neumaier.
__device__ __forceinline__ void nsum_merge(double &s, double &c, double s2, double c2)
{
    two_sum_acc(s, c, s2);
    c += c2;
}

// Block-wide compensated sum; thread 0 writes (s, c) to out.
__device__ __forceinline__ void block_nsum(double s, double c, double2 *out)
{
    __shared__ double ss[kMonitorThreads], sc[kMonitorThreads];
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int h = kMonitorThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            double a = ss[threadIdx.x], b = sc[threadIdx.x];
            nsum_merge(a, b, ss[threadIdx.x + h], sc[threadIdx.x + h]);
            ss[threadIdx.x] = a;
            sc[threadIdx.x] = b;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = make_double2(ss[0], sc[0]);
}

// On a periodic axis node index n repeats node index 0: count it once.
__device__ __forceinline__ bool unique_node(const Geo &g, int a, int idx)
{
    return !(g.per[a] && idx == g.n[a]);
}

template <typename T, typename S = T>
__global__ void __launch_bounds__(kMonitorThreads)
    k_energy(const Geo g, Fields<T, S> f, const double *__restrict__ eps_cell, const double *__restrict__ mu_cell,
             const double *__restrict__ ms_cell, double2 *partial)
{
    const double eps0 = 1.0 / (kMu0 * kC0 * kC0);
    const long long XY = (long long)g.X * g.Y;
    const long long total = XY * (g.n[2] + 1);
    double s = 0.0, c = 0.0;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % g.X), j = (int)((q / g.X) % g.Y), k = (int)(q / XY);
        if (i > g.n[0]) continue;
        const int ix[3] = {i, j, k};
        for (int a = 0; a < 3; a++) {
            // edge of E_a: cell index along a, node index along the others
            bool ok = ix[a] < g.n[a];
            for (int b = 0; b < 3; b++)
                if (b != a) ok = ok && unique_node(g, b, ix[b]);
            if (ok) {
                const double e = (double)ld_s(f.E[a] + q, f.sE);
                const double eps = eps0 * (eps_cell ? edge_mean(g, eps_cell, a, i, j, k) : 1.0);
                two_sum_acc(s, c, 0.5 * eps * e * e);
            }
            // face of H_a: node index along a, cell index along the others
            ok = unique_node(g, a, ix[a]);
            for (int b = 0; b < 3; b++)
                if (b != a) ok = ok && ix[b] < g.n[b];
            if (ok) {
                const double h = (double)ld_s(f.H[a] + q, f.sH);
                const bool mag = ms_cell && face_mean(g, ms_cell, a, i, j, k) > 0.0;
                const double mu = kMu0 * ((mu_cell && !mag) ? face_mean(g, mu_cell, a, i, j, k) : 1.0);
                double cu = 0.0;
                if (!wall_node(g, a, ix[a])) {
                    T rest, zp;
                    curl_e(g, f.E, f.inv_d, a, i, j, k, rest, zp, f.sE);
                    cu = (double)rest + (double)zp;
                }
                const double r = g.dt / (2.0 * mu) * cu;
                two_sum_acc(s, c, 0.5 * mu * (h * h - r * r));
            }
        }
    }
    block_nsum(s, c, partial + blockIdx.x);
}

// Poynting power through z node plane k, H at the time level of E taken as
// the mean of Ha and Hb (equal arrays when H is already there).
template <typename S, typename T>
__global__ void __launch_bounds__(kMonitorThreads)
    k_flux_partial(const Geo g, Ptr3<S> E, Ptr3<S> Ha, Ptr3<S> Hb, T sE, T sH, int k, double2 *partial)
{
    const int km = cell_nb(g, 2, k - 1), kp = cell_nb(g, 2, k);
    const long long XY = (long long)g.X * g.Y;
    const int npt = g.X * (g.n[1] + 1);
    const double area = g.d[0] * g.d[1];
    double s = 0.0, c = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npt; p += gridDim.x * blockDim.x) {
        const int i = p % g.X, j = p / g.X;
        if (i > g.n[0]) continue;
        const long long q = (long long)i + (long long)g.X * j;
        auto hv = [&](const Ptr3<S> &A, int comp, long long off) { return (double)ld_s(A.p[comp] + off, sH); };
        auto hmean = [&](const Ptr3<S> &A, const Ptr3<S> &B, int comp) {
            double v = 0.0;
            if (km >= 0) v += 0.5 * (0.5 * (hv(A, comp, q + km * XY) + hv(B, comp, q + km * XY)));
            if (kp >= 0) v += 0.5 * (0.5 * (hv(A, comp, q + kp * XY) + hv(B, comp, q + kp * XY)));
            return v;
        };
        // Ex (i+1/2, j, k) with Hy (i+1/2, j, k+-1/2)
        if (i < g.n[0] && j < g.n[1] + (g.per[1] ? 0 : 1))
            two_sum_acc(s, c, area * (double)ld_s(E.p[0] + q + (long long)k * XY, sE) * hmean(Ha, Hb, 1));
        // Ey (i, j+1/2, k) with Hx (i, j+1/2, k+-1/2)
        if (j < g.n[1] && i < g.n[0] + (g.per[0] ? 0 : 1))
            two_sum_acc(s, c, -area * (double)ld_s(E.p[1] + q + (long long)k * XY, sE) * hmean(Ha, Hb, 0));
    }
    block_nsum(s, c, partial + blockIdx.x);
}

// acc = {sum, correction, last power}: adds dt * P of this step.
__global__ void __launch_bounds__(kMonitorThreads)
    k_flux_accumulate(const double2 *partial, int nblocks, double dt, double *acc)
{
    double s = 0.0, c = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) nsum_merge(s, c, partial[b].x, partial[b].y);
    __shared__ double2 tot;
    block_nsum(s, c, &tot);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double P = tot.x + tot.y;
        double as = acc[0], ac = acc[1];
        two_sum_acc(as, ac, dt * P);
        acc[0] = as;
        acc[1] = ac;
        acc[2] = P;
    }
}

} // namespace mmx

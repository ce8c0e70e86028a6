// mmx_fused.cuh -- the vectorised one-pass E/H kernel of the coupled
// Maxwell-LLG step (arXiv 2103.12819, Sec. 3.2.2 Steps 2 and 3 with the next
// step's Step 1 folded in), for grids whose x and y boundaries are PEC walls.
//
// Work decomposition.  A CTA owns a strip of W = 32 V columns (V = 16 bytes /
// sizeof(T): 4 floats or 2 doubles per lane, moved with one 16-byte load or
// store; with FP16 storage the same 4 columns move as 8 bytes) by BY rows,
// and marches its z chunk plane by plane.  Lane L of warp
// w holds columns x0 + V L ... x0 + V L + V-1 of row y0 + w.  Neighbours
// along x come from warp shuffles; neighbours along y from double-buffered
// shared-memory rows.  Warp BY is a halo warp: it computes E^(n+1) of row
// y0 + BY, which the H update of row y0 + BY - 1 needs, and stores nothing.
// A strip narrower than the grid (nx > W) likewise treats lane 31 as a halo
// lane and the strips overlap by V columns.
//
// Per plane k of the chunk: H^(n+1/2) of plane k is staged for the warp
// below; E^(n+1) of plane k (Ex, Ey at node k; Ez at layer k+1/2) is formed
// and staged for the warp above, while the next planes are in flight into
// a ring of shared-memory stages (bulk tensor copies, or per-lane cp.async);
// then Hz at plane k and Hx, Hy at layer k-1/2 take NH half steps
// (Steps 3 and the next step's 1, both with E^(n+1)).  Faces of the magnetic
// box are written here too and overwritten by the H/M box kernel, which runs
// after this one from the old H buffer.  Walls: Ey, Ez at x = 0, Ex, Ez at
// y = 0 and every component at z walls are written as zero; the wall column
// x = nx and wall row y = ny are never written (the host keeps them zero).
#pragma once
#include <cuda.h>
#include <type_traits>

#include "mmx_kernels.cuh"

namespace mmx {


template <typename S> struct FusedIO {
    const S *Eo[3];
    const S *Ho[3];
    S *En[3];
    S *Hn[3];
    const S *Zo[2];     // PML split part of Ex, Ey (old)
    S *Zn[2];           // (new)
};

template <typename T> struct Lanes;
template <> struct Lanes<float> { static constexpr int V = 4; };
template <> struct Lanes<double> { static constexpr int V = 2; };

// 16-byte vector loads (read-only path) and stores.
__device__ __forceinline__ void vload(float (&r)[4], const float *p)
{
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
}
__device__ __forceinline__ void vload(double (&r)[2], const double *p)
{
    const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    r[0] = v.x; r[1] = v.y;
}
// coherent load for arrays this kernel also writes (the PML split H)
__device__ __forceinline__ void vload_rw(float (&r)[4], const float *p)
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
}
__device__ __forceinline__ void vload_rw(double (&r)[2], const double *p)
{
    const double2 v = *reinterpret_cast<const double2 *>(p);
    r[0] = v.x; r[1] = v.y;
}
// shared-memory 16-byte load
__device__ __forceinline__ void sload(float (&r)[4], const float *p)
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
}
__device__ __forceinline__ void sload(double (&r)[2], const double *p)
{
    const double2 v = *reinterpret_cast<const double2 *>(p);
    r[0] = v.x; r[1] = v.y;
}
__device__ __forceinline__ void vstore(float *p, const float (&r)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(r[0], r[1], r[2], r[3]);
}
__device__ __forceinline__ void vstore(double *p, const double (&r)[2])
{
    *reinterpret_cast<double2 *>(p) = make_double2(r[0], r[1]);
}

template <typename T, int V> __device__ __forceinline__ void vzero(T (&r)[V])
{
#pragma unroll
    for (int e = 0; e < V; e++) r[e] = T(0);
}
template <typename T, int V> __device__ __forceinline__ void vfill(T (&r)[V], T x)
{
#pragma unroll
    for (int e = 0; e < V; e++) r[e] = x;
}
template <typename T, int V> __device__ __forceinline__ void vcopy(T (&d)[V], const T (&s)[V])
{
#pragma unroll
    for (int e = 0; e < V; e++) d[e] = s[e];
}

// Paired FP32 arithmetic on a lane's 4 columns: columns (0, 1) and (2, 3)
// each go through one two-wide instruction (FADD2 / FMUL2 / FFMA2 of
// sm_100 and later), halving the FP32 instruction count of the updates.
// All round to nearest; a - b is formed as fma(-1, b, a), which is exact
// before its single rounding, as a subtraction is.
struct Pair4 {
    __device__ static float2 lo(const float (&x)[4]) { return make_float2(x[0], x[1]); }
    __device__ static float2 hi(const float (&x)[4]) { return make_float2(x[2], x[3]); }
    __device__ static void put(float (&r)[4], float2 a, float2 b)
    {
        r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y;
    }
    // r = a - b
    __device__ static void sub(float (&r)[4], const float (&a)[4], const float (&b)[4])
    {
        const float2 m = make_float2(-1.f, -1.f);
        put(r, __ffma2_rn(m, lo(b), lo(a)), __ffma2_rn(m, hi(b), hi(a)));
    }
    // r = a + b
    __device__ static void add(float (&r)[4], const float (&a)[4], const float (&b)[4])
    {
        put(r, __fadd2_rn(lo(a), lo(b)), __fadd2_rn(hi(a), hi(b)));
    }
    // r = a * s
    __device__ static void mul(float (&r)[4], const float (&a)[4], float s)
    {
        const float2 s2 = make_float2(s, s);
        put(r, __fmul2_rn(lo(a), s2), __fmul2_rn(hi(a), s2));
    }
    // r = a * b
    __device__ static void mulv(float (&r)[4], const float (&a)[4], const float (&b)[4])
    {
        put(r, __fmul2_rn(lo(a), lo(b)), __fmul2_rn(hi(a), hi(b)));
    }
    // r = a * s + c
    __device__ static void fma(float (&r)[4], const float (&a)[4], float s, const float (&c)[4])
    {
        const float2 s2 = make_float2(s, s);
        put(r, __ffma2_rn(lo(a), s2, lo(c)), __ffma2_rn(hi(a), s2, hi(c)));
    }
    // r = a * b + c
    __device__ static void fmav(float (&r)[4], const float (&a)[4], const float (&b)[4], const float (&c)[4])
    {
        put(r, __ffma2_rn(lo(a), lo(b), lo(c)), __ffma2_rn(hi(a), hi(b), hi(c)));
    }
};

// V stored values (S) -> V values of T times sc, and back (times isc): 16-byte
// moves for FP32/FP64 storage, 8-byte moves of 4 halves for FP16 storage.
template <typename S> struct SV;
template <> struct SV<float> {
    __device__ static void gld(float (&r)[4], const float *p, float) { vload(r, p); }
    __device__ static void gld_rw(float (&r)[4], const float *p, float) { vload_rw(r, p); }
    __device__ static void sld(float (&r)[4], const float *p, float) { sload(r, p); }
    __device__ static void gst(float *p, const float (&r)[4], float) { vstore(p, r); }
};
template <> struct SV<double> {
    __device__ static void gld(double (&r)[2], const double *p, double) { vload(r, p); }
    __device__ static void gld_rw(double (&r)[2], const double *p, double) { vload_rw(r, p); }
    __device__ static void sld(double (&r)[2], const double *p, double) { sload(r, p); }
    __device__ static void gst(double *p, const double (&r)[2], double) { vstore(p, r); }
};
template <> struct SV<__half> {
    __device__ static void cvt(float (&r)[4], uint2 u, float sc)
    {
        __half2 a, b;
        memcpy(&a, &u.x, 4);
        memcpy(&b, &u.y, 4);
        const float2 fa = __half22float2(a), fb = __half22float2(b);
        r[0] = fa.x * sc; r[1] = fa.y * sc; r[2] = fb.x * sc; r[3] = fb.y * sc;
    }
    __device__ static void gld(float (&r)[4], const __half *p, float sc)
    {
        cvt(r, __ldg(reinterpret_cast<const uint2 *>(p)), sc);
    }
    __device__ static void gld_rw(float (&r)[4], const __half *p, float sc)
    {
        cvt(r, *reinterpret_cast<const uint2 *>(p), sc);
    }
    __device__ static void sld(float (&r)[4], const __half *p, float sc)
    {
        cvt(r, *reinterpret_cast<const uint2 *>(p), sc);
    }
    __device__ static void gst(__half *p, const float (&r)[4], float isc)
    {
        const __half2 a = __floats2half2_rn(r[0] * isc, r[1] * isc), b = __floats2half2_rn(r[2] * isc, r[3] * isc);
        uint2 u;
        memcpy(&u.x, &a, 4);
        memcpy(&u.y, &b, 4);
        *reinterpret_cast<uint2 *>(p) = u;
    }
};

// Asynchronous global -> shared copies (cp.async): 16 bytes, 8 or 4 bytes;
// a false predicate zero-fills the destination and reads nothing (the
// source operand is then the array base, always valid).
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp16(void *dst, const void *src, const void *base, bool on)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)),
                 "l"(on ? src : base), "r"(on ? 16 : 0)
                 : "memory");
}
template <int N> __device__ __forceinline__ void cpn(void *dst, const void *src, const void *base, bool on)
{
    if constexpr (N == 16) {
        cp16(dst, src, base, on);
    } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_u32(dst)),
                     "l"(on ? src : base), "n"(N), "r"(on ? N : 0)
                     : "memory");
    }
}
// The same with the destination given as a 32-bit shared-memory address.
__device__ __forceinline__ void cp16a(unsigned dst, const void *src, const void *base, bool on)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(on ? src : base),
                 "r"(on ? 16 : 0)
                 : "memory");
}
template <int N> __device__ __forceinline__ void cpna(unsigned dst, const void *src, const void *base, bool on)
{
    if constexpr (N == 16) {
        cp16a(dst, src, base, on);
    } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(dst), "l"(on ? src : base), "n"(N),
                     "r"(on ? N : 0)
                     : "memory");
    }
}
// Tensor maps of the planes the TMA variant stages: the three H and three E
// arrays it reads and the cell eps_r array, each a 3-D (x, y, z) view of the
// padded layout whose box is one plane of the CTA's rows (H and eps_r from
// row y0-1, E from row y0).
struct VecMaps {
    CUtensorMap h[3];
    CUtensorMap e[3];
    CUtensorMap eps;
};

// mbarrier and bulk tensor copy primitives (PTX), shared addresses 32-bit.
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}
// One box of a 3-D tensor map at (x, y, z) into shared memory at dst; the
// copy's bytes complete on the mbarrier bar.  Coordinates outside the tensor
// read zero (x is always a multiple of 16 bytes here).
__device__ __forceinline__ void tma_load3(unsigned dst, const CUtensorMap *map, int x, int y, int z, unsigned bar)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
                 "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void cp_commit()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
// Wait until at most N of this thread's copy groups are still in flight.
template <int N> __device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Shared-memory layout of the vectorised kernel, a ring of ST plane stages
// (byte offsets, every region a multiple of 16 bytes):
//   sst [ST][6][R][W] of S  per plane: Hx, Hy (layer k+1/2), Hz (node k),
//                           Ex, Ey, Ez of rows y0..y0+BY
//   cst [ST][NC][R][W] of T cbx, cby, cbz [, cax, cay, caz]; with CBF the
//                           eps_r row of cell plane k instead
//   (CBF) eu [ST][W], el [ST][2][R] of T  eps_r of row y0-1 and of column
//                           x0-1 (rows y and y-1) of cell plane k
//   up  [ST][2][W] of S     Hx, Hz of row y0-1
//   left [ST][2][R][LW] of S  Hy, Hz of column x0-1 (FP16: the 4-byte pair
//                           ending there), one entry per row
//   sEx, sEz [2][R][W] of T E^(n+1) exchanged between rows
template <typename T, typename S, int BY, bool GEN, int ST, bool TMA = false> struct VecLayout {
    static constexpr int V = Lanes<T>::V;
    static constexpr int W = 32 * V;
    static constexpr int R = BY + 1;
    // rows per staged slab: the TMA variant also stages row y0-1 (row 0)
    static constexpr int RR = TMA ? R + 1 : R;
    static constexpr int OFF = TMA ? 1 : 0;   // slab row of row y0
    // FP32 arithmetic without sigma or mu_r: cb is formed from staged cell
    // eps_r (one value per cell instead of three per-edge coefficients)
    // (FP32 storage; with FP16 storage the kernel is bound by instruction
    // issue and the added arithmetic costs more than the bytes it saves)
    static constexpr bool CBF = !GEN && sizeof(T) == 4 && sizeof(S) == 4;
    static constexpr int NC = GEN ? 6 : (CBF ? 1 : 3);
    static constexpr int LW = sizeof(S) >= 4 ? 1 : 4 / (int)sizeof(S);
    // regions start on 128-byte boundaries where bulk tensor copies land
    static constexpr size_t al(size_t x) { return TMA ? (x + 127) / 128 * 128 : (x + 15) / 16 * 16; }
    static constexpr size_t sst = 0;
    static constexpr size_t cst = sst + al((size_t)ST * 6 * RR * W * sizeof(S));
    static constexpr size_t up = cst + al((size_t)ST * NC * RR * W * sizeof(T));
    static constexpr size_t left = up + (TMA ? 0 : al((size_t)ST * 2 * W * sizeof(S)));
    static constexpr size_t ex = left + al((size_t)ST * 2 * R * LW * sizeof(S));
    // Ez rows of the last planes: the H update of plane k reads plane k-1's
    // after the mid-plane barrier.  Two buffers when a barrier at the top of
    // every plane keeps a warp from writing plane k+1's meanwhile; three in
    // the TMA variant, which has no such barrier
    static constexpr int NEZ = TMA ? 3 : 2;
    static_assert(!TMA || NEZ >= 3, "one barrier per plane needs three Ez exchange buffers");
    static constexpr size_t ez = ex + al((size_t)2 * R * W * sizeof(T));
    static constexpr size_t eu = ez + al((size_t)NEZ * R * W * sizeof(T));
    static constexpr size_t el = eu + (CBF && !TMA ? al((size_t)ST * W * sizeof(T)) : 0);
    static constexpr size_t mb = el + (CBF ? al((size_t)ST * 2 * R * sizeof(T)) : 0);
    static constexpr size_t bytes = mb + (TMA ? al((size_t)ST * 8) : 0);
    // bytes one stage's bulk copies deliver (H 3 and eps_r with RR rows, E 3 with R)
    static constexpr unsigned tx = (unsigned)((3 * RR + 3 * R) * W * sizeof(S) + (CBF ? RR * W * sizeof(T) : 0));
};

// The kernel body for the CTA at tile (bx, by) and z range [k0, k1) of one
// grid: the single grid launch passes its block index and chunk bounds, the
// batched launch the entry of its work table; amp holds this step's source
// amplitudes.
template <typename T, typename S, int BY, int ST, int NH, bool PMLK, bool GEN, bool TMA = false>
__device__ __forceinline__ void fused_vec_body(const Geo &g, const Fields<T, S> &f, const FusedIO<S> &io,
                                               const Src<T> *__restrict__ src, int nsrc, const T *amp,
                                               int k0, int k1, int xstride, int bx, int by,
                                               const VecMaps *maps = nullptr)
{
    using L = VecLayout<T, S, BY, GEN, ST, TMA>;
    using P = SV<S>;
    constexpr int V = L::V, W = L::W, R = L::R, NC = L::NC, LW = L::LW, RR = L::RR, OFF = L::OFF;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // S-typed stage fields 0-5: Hx Hy Hz Ex Ey Ez; T-typed 0-5: cb, ca (or
    // eps_r); row r of the CTA (r = -1 the row below y0 in the TMA variant)
    auto SS = [&](int st, int fld, int row) -> S * {
        return reinterpret_cast<S *>(smem_raw + L::sst) + ((st * 6 + fld) * RR + row + OFF) * W;
    };
    auto SC = [&](int st, int fld, int row) -> T * {
        return reinterpret_cast<T *>(smem_raw + L::cst) + ((st * NC + fld) * RR + row + OFF) * W;
    };
    auto U = [&](int st, int fld) -> S * { return reinterpret_cast<S *>(smem_raw + L::up) + (st * 2 + fld) * W; };
    auto Lf = [&](int st, int fld) -> S * {
        return reinterpret_cast<S *>(smem_raw + L::left) + (st * 2 + fld) * R * LW;
    };
    auto SEx = [&](int bb, int row) -> T * { return reinterpret_cast<T *>(smem_raw + L::ex) + (bb * R + row) * W; };
    auto SEz = [&](int bb, int row) -> T * { return reinterpret_cast<T *>(smem_raw + L::ez) + (bb * R + row) * W; };
    constexpr bool CBF = L::CBF;
    // FP16 storage (FP32 arithmetic, 4 columns per lane): the updates run on
    // column pairs.  With FP32 storage the paired form executed 15% fewer
    // instructions but ran 6% slower (longer dependent chains in a kernel
    // bound by issue latency), so it keeps one column per instruction.
    constexpr bool PAIRED = std::is_same<T, float>::value && V == 4 && sizeof(S) == 2;
    auto EU = [&](int st) -> T * { return reinterpret_cast<T *>(smem_raw + L::eu) + st * W; };
    auto EL = [&](int st, int r2) -> T * { return reinterpret_cast<T *>(smem_raw + L::el) + (st * 2 + r2) * R; };
    const T sE = f.sE, sH = f.sH, isE = f.isE, isH = f.isH;
    constexpr int VB = V * (int)sizeof(S);      // bytes of one lane's S values

    // lane and warp from the linear thread index: the same for the (32,
    // BY+1) blocks of the plain launches and the 1-D blocks of the overlap
    // launch
    const int lin = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = lin & 31, w = lin >> 5;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int x0 = bx * xstride;
    const int i0 = x0 + V * lane;
    const int col = V * lane;
    const int j = by * BY + w;
    const bool last_chunk = k1 == nz;
    const bool lane_on = j < ny && i0 < nx;
    const bool up_on = w == 0 && j > 0 && j <= ny && i0 < nx;
    const bool left_on = lane == 0 && x0 > 0 && j < ny;
    const bool store = lane_on && w < BY && (lane < 31 || x0 + W >= nx);
    const unsigned XY = (unsigned)g.X * (unsigned)g.Y;
    const unsigned rb = (unsigned)i0 + (unsigned)g.X * (unsigned)j;
    const unsigned rbu = rb - (unsigned)g.X;
    const unsigned rbl = (unsigned)(x0 - 1) + (unsigned)g.X * (unsigned)j;
    const T idx = f.inv_d[0], idy = f.inv_d[1], idz = f.inv_d[2];
    const T fh0 = f.fh0;
    const bool wy = j == 0;
    bool cin[V], xw[V];
#pragma unroll
    for (int e = 0; e < V; e++) {
        cin[e] = i0 + e < nx;
        xw[e] = i0 + e == 0;
    }
    // z range of the soft sources touching this lane's columns
    int src_klo = 1 << 30, src_khi = -1;
    if (lane_on)
        for (int s = 0; s < nsrc; s++) {
            const Src<T> &q = src[s];
            if (q.kind == 1 || (q.kind == 0 && q.j == j && q.i >= i0 && q.i < i0 + V)) {
                src_klo = min(src_klo, q.k);
                src_khi = max(src_khi, q.k);
                if (g.per[2] && q.k == 0) src_khi = max(src_khi, nz);
            }
        }

    // copies of everything plane k needs into stage st
    // this thread's copy destinations as 32-bit shared addresses of stage 0;
    // stage st adds st times the stage stride, a field a multiple of its slab
    constexpr unsigned SF = RR * W * sizeof(S), SST = 6 * SF;   // S fields
    constexpr unsigned CF = RR * W * sizeof(T), CST = NC * CF;  // material words
    constexpr unsigned UF = W * sizeof(S), UST = 2 * UF;        // row y0-1
    constexpr unsigned LFB = R * LW * sizeof(S), LST = 2 * LFB; // column x0-1
    const unsigned sS = smem_u32(SS(0, 0, w) + col), sC = smem_u32(SC(0, 0, w) + col);
    // TMA variant: one mbarrier per stage, armed by thread (0, 0) with the
    // stage's byte count; every thread waits on its phase
    const unsigned mbar0 = TMA ? smem_u32(smem_raw + L::mb) : 0u;
    const bool leader = lin == 0;
    if constexpr (TMA) {
        if (leader) {
#pragma unroll
            for (int q = 0; q < ST; q++) mbar_init(mbar0 + 8 * q, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }
    auto issue = [&](int k, int st) {
        const int ck = cell_nb(g, 2, k);
        const unsigned kn = (unsigned)k * XY, kc = (unsigned)max(ck, 0) * XY;
        const bool lay = ck >= 0;
        if constexpr (TMA) {
            if (leader) {
                // planes of H (rows y0-1 .. y0+BY; cell plane ck or node k),
                // E (rows y0 .. y0+BY, node k) and eps_r (cell plane ck); a
                // missing cell plane (ck < 0) is read as zero
                const unsigned bar = mbar0 + 8 * st;
                const unsigned s0 = smem_u32(smem_raw + L::sst) + (unsigned)st * SST;
                const unsigned c0 = smem_u32(smem_raw + L::cst) + (unsigned)st * CST;
                const int yh = by * BY - 1, ye = by * BY, zc = ck;
                mbar_expect_tx(bar, L::tx);
                tma_load3(s0, &maps->h[0], x0, yh, zc, bar);
                tma_load3(s0 + SF, &maps->h[1], x0, yh, zc, bar);
                tma_load3(s0 + 2 * SF, &maps->h[2], x0, yh, k, bar);
#pragma unroll
                for (int c = 0; c < 3; c++) tma_load3(s0 + (3 + c) * SF + W * sizeof(S), &maps->e[c], x0, ye, k, bar);
                if constexpr (CBF) tma_load3(c0, &maps->eps, x0, yh, zc, bar);
            }
            if (lane == 0) {
                constexpr int CB = LW * (int)sizeof(S);
                const unsigned l0 = smem_u32(Lf(0, 0) + w * LW) + (unsigned)st * LST;
                cpna<CB>(l0, io.Ho[1] + rbl + kc - (LW - 1), io.Ho[1], left_on && lay);
                cpna<CB>(l0 + LFB, io.Ho[2] + rbl + kn - (LW - 1), io.Ho[2], left_on);
                if constexpr (CBF) {
                    cpn<4>(EL(st, 0) + w, f.epsc + rbl + kc, f.epsc, left_on && lay);
                    cpn<4>(EL(st, 1) + w, f.epsc + rbl - (unsigned)g.X + kc, f.epsc, left_on && j > 0 && lay);
                }
            }
            cp_commit();
            return;
        }
        const unsigned s0 = sS + (unsigned)st * SST, c0 = sC + (unsigned)st * CST;
        cpna<VB>(s0, io.Ho[0] + rb + kc, io.Ho[0], lane_on && lay);
        cpna<VB>(s0 + SF, io.Ho[1] + rb + kc, io.Ho[1], lane_on && lay);
        cpna<VB>(s0 + 2 * SF, io.Ho[2] + rb + kn, io.Ho[2], lane_on);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            cpna<VB>(s0 + (3 + c) * SF, io.Eo[c] + rb + kn, io.Eo[c], lane_on);
            if (!CBF) cp16a(c0 + c * CF, f.cb[c] + rb + kn, f.cb[c], lane_on);
            if (GEN && f.ca[c]) cp16a(c0 + (3 + c) * CF, f.ca[c] + rb + kn, f.ca[c], lane_on);
        }
        if constexpr (CBF) {
            // eps_r of cell plane k: this row, the row below, and column x0-1
            cp16a(c0, f.epsc + rb + kc, f.epsc, lane_on && lay);
            if (w == 0) cp16(EU(st) + col, f.epsc + rbu + kc, f.epsc, up_on && lay);
            if (lane == 0) {
                cpn<4>(EL(st, 0) + w, f.epsc + rbl + kc, f.epsc, left_on && lay);
                cpn<4>(EL(st, 1) + w, f.epsc + rbl - (unsigned)g.X + kc, f.epsc, left_on && j > 0 && lay);
            }
        }
        if (w == 0) {
            const unsigned u0 = smem_u32(U(0, 0) + col) + (unsigned)st * UST;
            cpna<VB>(u0, io.Ho[0] + rbu + kc, io.Ho[0], up_on && lay);
            cpna<VB>(u0 + UF, io.Ho[2] + rbu + kn, io.Ho[2], up_on);
        }
        if (lane == 0) {
            // the LW-element group ending at column x0-1 (one element unless
            // the element is narrower than the 4-byte minimum copy)
            constexpr int CB = LW * (int)sizeof(S);
            const unsigned l0 = smem_u32(Lf(0, 0) + w * LW) + (unsigned)st * LST;
            cpna<CB>(l0, io.Ho[1] + rbl + kc - (LW - 1), io.Ho[1], left_on && lay);
            cpna<CB>(l0 + LFB, io.Ho[2] + rbl + kn - (LW - 1), io.Ho[2], left_on);
        }
        cp_commit();
    };

    // CBF: eps_r pair sums of cell plane k-1 along y (cells j-1, j: Ex) and
    // along x (cells i-1, i: Ey), carried up the z march
    T pyxp[V], pxyp[V];
    vfill<T, V>(pyxp, T(2));
    vfill<T, V>(pxyp, T(2));
    if constexpr (CBF) {
        const int ckm = cell_nb(g, 2, k0 - 1);
        T a[V], au[V];
        vfill<T, V>(a, T(1));
        vfill<T, V>(au, T(1));
        if (lane_on && ckm >= 0) {
            vload(a, f.epsc + rb + (unsigned)ckm * XY);
            if (j > 0) vload(au, f.epsc + rbu + (unsigned)ckm * XY);
        }
        T al = __shfl_up_sync(0xffffffffu, a[V - 1], 1);
        if (lane == 0) al = (left_on && ckm >= 0) ? f.epsc[rbl + (unsigned)ckm * XY] : T(1);
#pragma unroll
        for (int e = 0; e < V; e++) {
            pyxp[e] = au[e] + a[e];
            pxyp[e] = (e > 0 ? a[e > 0 ? e - 1 : 0] : al) + a[e];
        }
    }
    T hxp[V], hyp[V];                 // Hx, Hy at layer k-1/2
    T exq[V], eyq[V], ezq[V];         // E^(n+1) of plane k-1 (Ez: layer k-1/2)
    vzero<T, V>(exq);
    vzero<T, V>(eyq);
    vzero<T, V>(ezq);
    {
        const int ckm = cell_nb(g, 2, k0 - 1);
        if (lane_on && ckm >= 0) {
            P::gld(hxp, io.Ho[0] + rb + (unsigned)ckm * XY, sH);
            P::gld(hyp, io.Ho[1] + rb + (unsigned)ckm * XY, sH);
        } else {
            vzero<T, V>(hxp);
            vzero<T, V>(hyp);
        }
    }
    // prologue: planes k0 .. k0+ST-2 in flight (k0 .. k0+ST-1 with bulk
    // copies, which refill a stage as soon as its plane has been read); one
    // copy group per plane, empty groups past the chunk keep the group count
    // uniform
    constexpr int PRE = TMA ? ST : ST - 1;
#pragma unroll
    for (int s = 0; s < PRE; s++) {
        if (k0 + s <= k1)
            issue(k0 + s, s);
        else
            cp_commit();
    }
    T acc = T(0);
    bool nonfin = false;
    bool tma_bad = false;
    int b = 0, st = 0;
    int ze = 0, zq = L::NEZ - 1;      // Ez buffers of planes k and k-1
    for (int k = k0; k <= k1; k++, b ^= 1, st = st + 1 == ST ? 0 : st + 1, zq = ze, ze = ze + 1 == L::NEZ ? 0 : ze + 1) {
        if constexpr (TMA) {
            // bounded wait for plane k's bulk copies (stage st, use (k-k0)/ST)
            if (!tma_bad) {
                const unsigned par = (unsigned)((k - k0) / ST) & 1u;
                const long long t0 = clock64();
                while (!mbar_try_wait(mbar0 + 8 * st, par)) {
                    if (clock64() - t0 > (1LL << 31)) {
                        tma_bad = true;
                        atomicOr(f.err, kErrTimeout);
                        break;
                    }
                }
            }
        }
        if constexpr (TMA) {
            // this warp's lane-0 halo copies of plane k (read by lane 0 only)
            cp_wait<ST - 1>();
        } else {
            cp_wait<ST - 2>();
            __syncthreads();      // plane k staged; every thread is done with plane k-1
            // plane k+ST-1 into the stage plane k-1 used
            const int sn = st == 0 ? ST - 1 : st - 1;
            if (k + ST - 1 <= k1)
                issue(k + ST - 1, sn);
            else
                cp_commit();
        }

        T hx[V], hy[V], hz[V], hzu[V], hxu[V];
        P::sld(hx, SS(st, 0, w) + col, sH);
        P::sld(hy, SS(st, 1, w) + col, sH);
        P::sld(hz, SS(st, 2, w) + col, sH);
        if (w == 0 && !TMA) {
            P::sld(hxu, U(st, 0) + col, sH);
            P::sld(hzu, U(st, 1) + col, sH);
        } else {
            P::sld(hxu, SS(st, 0, w - 1) + col, sH);
            P::sld(hzu, SS(st, 2, w - 1) + col, sH);
        }
        // column i-1 of element 0: previous lane's last element, or the halo
        T hzl = __shfl_up_sync(0xffffffffu, hz[V - 1], 1);
        T hyl = __shfl_up_sync(0xffffffffu, hy[V - 1], 1);
        if (lane == 0) {
            hyl = ld_s(Lf(st, 0) + w * LW + (LW - 1), sH);
            hzl = ld_s(Lf(st, 1) + w * LW + (LW - 1), sH);
        }

        // ---- E^(n+1) at plane k
        const bool own_plane = k < k1 || last_chunk;
        const bool wz = wall_node(g, 2, k);
        const bool pml = PMLK && pml_e_plane(g, k);
        const unsigned q = rb + (unsigned)k * XY;
        T ex[V], ey[V], ez[V], zn0[V], zn1[V];
        {
            T eo[3][V], cb[3][V], ca[3][V];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                P::sld(eo[c], SS(st, 3 + c, w) + col, sE);
                if (!CBF) sload(cb[c], SC(st, c, w) + col);
                if (GEN && f.ca[c])
                    sload(ca[c], SC(st, 3 + c, w) + col);
                else
                    vfill<T, V>(ca[c], T(1));
            }
            if constexpr (CBF) {
                // cb = dt/(eps0 mean eps_r) over the edge's four cells: Ex
                // (i, j-1..j, k-1..k), Ey (i-1..i, j, k-1..k), Ez (i-1..i,
                // j-1..j, k); only interior edges use it (walls are zeroed)
                T er[V], eu[V];
                sload(er, SC(st, 0, w) + col);
                if (w == 0 && !TMA)
                    sload(eu, EU(st) + col);
                else
                    sload(eu, SC(st, 0, w - 1) + col);
                T el = __shfl_up_sync(0xffffffffu, er[V - 1], 1);
                T elu = __shfl_up_sync(0xffffffffu, eu[V - 1], 1);
                if (lane == 0) {
                    el = EL(st, 0)[w];
                    elu = EL(st, 1)[w];
                }
#pragma unroll
                for (int e = 0; e < V; e++) {
                    const T erl = e > 0 ? er[e > 0 ? e - 1 : 0] : el;
                    const T eul = e > 0 ? eu[e > 0 ? e - 1 : 0] : elu;
                    const T pyx = eu[e] + er[e], pxy = erl + er[e];
                    // one reciprocal for the three edges (Montgomery's
                    // simultaneous inversion, 1987): t = kcb/(sx sy sz), then
                    // kcb/sx = t sy sz and so on
                    const T sx = pyxp[e] + pyx, sy = pxyp[e] + pxy, sz = pxy + eul + eu[e];
                    const T sxy = sx * sy;
                    const T t = __fdividef(f.kcb, sxy * sz);
                    const T u = t * sz;
                    cb[0][e] = u * sy;
                    cb[1][e] = u * sx;
                    cb[2][e] = t * sxy;
                    pyxp[e] = pyx;
                    pxyp[e] = pxy;
                }
            }
            T zo0[V], zo1[V];
            if (pml && lane_on) {
                P::gld(zo0, io.Zo[0] + q, sE);
                P::gld(zo1, io.Zo[1] + q, sE);
            } else {
                vzero<T, V>(zo0);
                vzero<T, V>(zo1);
            }
            const T hdamp = pml ? f.dampE[k] : T(1);
            const bool src_here = k >= src_klo && k <= src_khi;
            bool paired = false;
            if constexpr (PAIRED && !GEN) {
                if (!pml) {
                    // FP32 outside the PML planes (ca = 1): columns in pairs
                    T J0[V], J1[V], J2[V];
                    vzero<T, V>(J0);
                    vzero<T, V>(J1);
                    vzero<T, V>(J2);
                    if (src_here) {
#pragma unroll
                        for (int e = 0; e < V; e++)
                            if (cin[e]) {
                                J0[e] = j_source_a(g, f, amp, src, nsrc, 0, i0 + e, j, k);
                                J1[e] = j_source_a(g, f, amp, src, nsrc, 1, i0 + e, j, k);
                                J2[e] = j_source_a(g, f, amp, src, nsrc, 2, i0 + e, j, k);
                            }
                    }
                    const T hzm[V] = {hzl, hz[0], hz[1], hz[2]};
                    const T hym[V] = {hyl, hy[0], hy[1], hy[2]};
                    T t1[V], t2[V], v[V];
                    // Ex = eo + cb ((hz - hzu) idy + (hyp - hy) idz - J)
                    Pair4::sub(t1, hz, hzu);
                    Pair4::mul(t1, t1, idy);
                    Pair4::sub(t2, hyp, hy);
                    Pair4::fma(t1, t2, idz, t1);
                    Pair4::sub(t1, t1, J0);
                    Pair4::fmav(v, cb[0], t1, eo[0]);
#pragma unroll
                    for (int e = 0; e < V; e++) {
                        ex[e] = (lane_on && cin[e] && !wy && !wz) ? v[e] : T(0);
                        zn0[e] = T(0);
                    }
                    // Ey = eo + cb ((hx - hxp) idz + (hzm - hz) idx - J)
                    Pair4::sub(t1, hx, hxp);
                    Pair4::mul(t1, t1, idz);
                    Pair4::sub(t2, hzm, hz);
                    Pair4::fma(t1, t2, idx, t1);
                    Pair4::sub(t1, t1, J1);
                    Pair4::fmav(v, cb[1], t1, eo[1]);
#pragma unroll
                    for (int e = 0; e < V; e++) {
                        ey[e] = (lane_on && cin[e] && !xw[e] && !wz) ? v[e] : T(0);
                        zn1[e] = T(0);
                    }
                    // Ez = eo + cb ((hy - hym) idx + (hxu - hx) idy - J)
                    Pair4::sub(t1, hy, hym);
                    Pair4::mul(t1, t1, idx);
                    Pair4::sub(t2, hxu, hx);
                    Pair4::fma(t1, t2, idy, t1);
                    Pair4::sub(t1, t1, J2);
                    Pair4::fmav(v, cb[2], t1, eo[2]);
#pragma unroll
                    for (int e = 0; e < V; e++) ez[e] = (lane_on && cin[e] && !xw[e] && !wy && k < nz) ? v[e] : T(0);
                    paired = true;
                }
            }
            // one copy without source terms (J = 0 folds away) and one with,
            // each with and without the PML split update: the plane's kind
            // is uniform, and a run-time test inside the unrolled columns
            // was if-converted (both updates computed, one selected)
            auto e_cols = [&](auto with_src, auto with_pml) {
                constexpr bool SRC = decltype(with_src)::value;
                constexpr bool PML = decltype(with_pml)::value == 1;
#pragma unroll
            for (int e = 0; e < V; e++) {
                T J0 = T(0), J1 = T(0), J2 = T(0);
                if (SRC && cin[e]) {
                    J0 = j_source_a(g, f, amp, src, nsrc, 0, i0 + e, j, k);
                    J1 = j_source_a(g, f, amp, src, nsrc, 1, i0 + e, j, k);
                    J2 = j_source_a(g, f, amp, src, nsrc, 2, i0 + e, j, k);
                }
                const T hzm = e > 0 ? hz[e > 0 ? e - 1 : 0] : hzl;
                const T hym = e > 0 ? hy[e > 0 ? e - 1 : 0] : hyl;
                // Ex (i+1/2, j, k)
                {
                    const T rest = (hz[e] - hzu[e]) * idy;
                    const T zp = -(hy[e] - hyp[e]) * idz;
                    T v, z = T(0);
                    if constexpr (PML) {
                        z = (ca[0][e] * (zo0[e] * hdamp) + cb[0][e] * zp) * hdamp;
                        v = ca[0][e] * (eo[0][e] - zo0[e]) + cb[0][e] * (rest - J0) + z;
                    } else {
                        v = ca[0][e] * eo[0][e] + cb[0][e] * (rest + zp - J0);
                    }
                    const bool on = lane_on && cin[e] && !wy && !wz;
                    ex[e] = on ? v : T(0);
                    zn0[e] = on ? z : T(0);
                }
                // Ey (i, j+1/2, k)
                {
                    const T zp = (hx[e] - hxp[e]) * idz;
                    const T rest = -(hz[e] - hzm) * idx;
                    T v, z = T(0);
                    if constexpr (PML) {
                        z = (ca[1][e] * (zo1[e] * hdamp) + cb[1][e] * zp) * hdamp;
                        v = ca[1][e] * (eo[1][e] - zo1[e]) + cb[1][e] * (rest - J1) + z;
                    } else {
                        v = ca[1][e] * eo[1][e] + cb[1][e] * (rest + zp - J1);
                    }
                    const bool on = lane_on && cin[e] && !xw[e] && !wz;
                    ey[e] = on ? v : T(0);
                    zn1[e] = on ? z : T(0);
                }
                // Ez (i, j, k+1/2)
                {
                    const T rest = (hy[e] - hym) * idx - (hx[e] - hxu[e]) * idy;
                    const T v = ca[2][e] * eo[2][e] + cb[2][e] * (rest - J2);
                    const bool on = lane_on && cin[e] && !xw[e] && !wy && k < nz;
                    ez[e] = on ? v : T(0);
                }
            }
            };
            if (!paired) {
                auto e_pml = [&](auto with_src) {
                    if (pml)
                        e_cols(with_src, std::integral_constant<int, 1>{});
                    else
                        e_cols(with_src, std::integral_constant<int, 0>{});
                };
                // FP32 arithmetic: the copy without source terms on every
                // plane, then on the few planes that hold sources their
                // -cb J added to the finished E (a second, source-carrying
                // copy of the update in the loop cost the source-free planes
                // 4 % of their instructions: 84.4 against 85.3 us per
                // launch); FP64 keeps the copy with source terms only (a
                // second copy's registers cost it more than the subtractions
                // it saves).  Hoisting the PML test out of the columns cut
                // the FP32 launch from 56.9 M to 50.4 M warp instructions
                // and 87.6 to 85.7 us on the waveguide.
                if (sizeof(T) == 8) {
                    e_pml(std::true_type{});
                } else {
                    e_pml(std::false_type{});
                    if (src_here) {
#pragma unroll
                        for (int e = 0; e < V; e++) {
                            if (!cin[e] || !lane_on) continue;
                            const int i = i0 + e;
                            const T J0 = j_source_a(g, f, amp, src, nsrc, 0, i, j, k);
                            const T J1 = j_source_a(g, f, amp, src, nsrc, 1, i, j, k);
                            const T J2 = j_source_a(g, f, amp, src, nsrc, 2, i, j, k);
                            if (!wy && !wz) ex[e] -= cb[0][e] * J0;
                            if (!xw[e] && !wz) ey[e] -= cb[1][e] * J1;
                            if (!xw[e] && !wy && k < nz) ez[e] -= cb[2][e] * J2;
                        }
                    }
                }
            }
        }
        vstore(SEx(b, w) + col, ex);
        vstore(SEz(ze, w) + col, ez);
        if (store && own_plane) {
            P::gst(io.En[0] + q, ex, isE);
            P::gst(io.En[1] + q, ey, isE);
            if (k < nz) P::gst(io.En[2] + q, ez, isE);
            if (pml) {
                P::gst(io.Zn[0] + q, zn0, isE);
                P::gst(io.Zn[1] + q, zn1, isE);
            }
            // non-finite check on E^(n+1) only: H^(n+3/2) is formed from it,
            // so a non-finite H shows in E one step later
#pragma unroll
            for (int e = 0; e < V; e++) {
                if constexpr (sizeof(T) == 8) {
                    // FP64 (bound by the FP64 pipe): test the exponent bits
                    // on the integer pipe instead of summing
                    const unsigned a0 = (unsigned)__double2hiint((double)ex[e]) & 0x7ff00000u;
                    const unsigned a1 = (unsigned)__double2hiint((double)ey[e]) & 0x7ff00000u;
                    const unsigned a2 = (unsigned)__double2hiint((double)ez[e]) & 0x7ff00000u;
                    nonfin |= (a0 == 0x7ff00000u) | (a1 == 0x7ff00000u) | (a2 == 0x7ff00000u);
                } else {
                    acc += ex[e] + ey[e] + ez[e];
                }
            }
        }
        // E^(n+1) of plane k visible to the row above.  In the TMA variant
        // this is the only block barrier of a plane, so a warp can run at
        // most one plane ahead of the slowest warp (it cannot pass the next
        // plane's barrier before every warp has arrived at it).  Under that
        // bound: (1) the refill of stage st below is safe, since every read
        // of stage st precedes this barrier and the H part after it reads
        // registers, the SEx/SEz exchange rows and lane-0 halos only (the
        // halos are read by the warp that copied them, after its own
        // cp_wait); (2) SEx rows of planes k and k-1 (b and b^1) suffice, as
        // a warp writing plane k+1's rows waits at plane k+1's barrier
        // before anyone reads them, while a slower warp may still read plane
        // k-1's SEz rows after plane k's barrier: hence three SEz buffers
        // (NEZ) for the variant without a top-of-plane barrier.
        __syncthreads();
        if constexpr (TMA) {
            // every thread has read stage st (all its reads precede the
            // barrier above): plane k+ST into it, half a plane earlier than
            // a refill at the top of the next plane, and no barrier there
            if (k + ST <= k1)
                issue(k + ST, st);
            else
                cp_commit();
        }

        // ---- H: Hz at plane k, Hx and Hy at layer k-1/2
        const T eyr = __shfl_down_sync(0xffffffffu, ey[0], 1);
        const T ezr = __shfl_down_sync(0xffffffffu, ezq[0], 1);
        if (w < BY) {
            if (store && own_plane) {
                T fh[V], exd[V];
                if (GEN && f.fh[2])
                    vload(fh, f.fh[2] + q);
                else
                    vfill<T, V>(fh, fh0);
                sload(exd, SEx(b, w + 1) + col);
                T hn[V];
                if constexpr (PAIRED) {
                    // cz = (eyn - ey) idx + (ex - exd) idy; NH half steps of
                    // -fh curl E with the same E in one FMA
                    const T eyn[V] = {ey[1], ey[2], ey[3], lane < 31 ? eyr : T(0)};
                    T t1[V], t2[V], nf[V], v[V];
                    Pair4::sub(t1, eyn, ey);
                    Pair4::mul(t1, t1, idx);
                    Pair4::sub(t2, ex, exd);
                    Pair4::fma(t1, t2, idy, t1);
                    Pair4::mul(nf, fh, -T(NH));
                    Pair4::fmav(v, t1, nf, hz);
#pragma unroll
                    for (int e = 0; e < V; e++) hn[e] = (cin[e] && !wz) ? v[e] : T(0);
                } else {
#pragma unroll
                    for (int e = 0; e < V; e++) {
                        const T eyn = e < V - 1 ? ey[e < V - 1 ? e + 1 : 0] : (lane < 31 ? eyr : T(0));
                        const T cz = (eyn - ey[e]) * idx - (exd[e] - ex[e]) * idy;
                        // NH half steps of -fh curl E with the same E: one FMA
                        const T v = hz[e] - (T(NH) * fh[e]) * cz;
                        hn[e] = (cin[e] && !wz) ? v : T(0);
                    }
                }
                P::gst(io.Hn[2] + q, hn, isH);
            }
            if (store && k > k0) {
                const int kl = k - 1;
                const unsigned ql = q - XY;
                const bool hp = PMLK && pml_h_plane(g, kl);
                const T hdh = hp ? f.dampH[kl] : T(1);
                T fhx[V], fhy[V], sx[V], sy[V], ezd[V];
                if (GEN && f.fh[0])
                    vload(fhx, f.fh[0] + ql);
                else
                    vfill<T, V>(fhx, fh0);
                if (GEN && f.fh[1])
                    vload(fhy, f.fh[1] + ql);
                else
                    vfill<T, V>(fhy, fh0);
                if (hp) {
                    P::gld_rw(sx, f.Hzp[0] + ql, sH);
                    P::gld_rw(sy, f.Hzp[1] + ql, sH);
                } else {
                    vzero<T, V>(sx);
                    vzero<T, V>(sy);
                }
                sload(ezd, SEz(zq, w + 1) + col);
                T hxn[V], hyn[V];
                bool hpaired = false;
                if constexpr (PAIRED) {
                    if (!hp) {
                        // Hx = hxp - NH fhx ((ezd - ezq) idy + (eyq - ey) idz)
                        // Hy = hyp - NH fhy ((ex - exq) idz + (ezq - ezn) idx)
                        const T ezn[V] = {ezq[1], ezq[2], ezq[3], lane < 31 ? ezr : T(0)};
                        T t1[V], t2[V], nf[V], v[V];
                        Pair4::sub(t1, ezd, ezq);
                        Pair4::mul(t1, t1, idy);
                        Pair4::sub(t2, eyq, ey);
                        Pair4::fma(t1, t2, idz, t1);
                        Pair4::mul(nf, fhx, -T(NH));
                        Pair4::fmav(v, t1, nf, hxp);
#pragma unroll
                        for (int e = 0; e < V; e++) hxn[e] = (cin[e] && !xw[e]) ? v[e] : T(0);
                        Pair4::sub(t1, ex, exq);
                        Pair4::mul(t1, t1, idz);
                        Pair4::sub(t2, ezq, ezn);
                        Pair4::fma(t1, t2, idx, t1);
                        Pair4::mul(nf, fhy, -T(NH));
                        Pair4::fmav(v, t1, nf, hyp);
#pragma unroll
                        for (int e = 0; e < V; e++) hyn[e] = (cin[e] && !wy) ? v[e] : T(0);
                        hpaired = true;
                    }
                }
                // with and without the split update, as for E
                auto h_cols = [&](auto with_pml) {
                    constexpr bool PML = decltype(with_pml)::value;
#pragma unroll
                for (int e = 0; e < V; e++) {
                    // Hx (i, j+1/2, k-1/2)
                    {
                        const T rest = (ezd[e] - ezq[e]) * idy;
                        const T zp = -(ey[e] - eyq[e]) * idz;
                        T v;
                        if constexpr (PML) {
                            T hzp = sx[e];
                            T hr = hxp[e] - hzp;
#pragma unroll
                            for (int s = 0; s < NH; s++) {
                                hzp = (hzp * hdh - fhx[e] * zp) * hdh;
                                hr = hr - fhx[e] * rest;
                            }
                            sx[e] = (cin[e] && !xw[e]) ? hzp : T(0);
                            v = hr + hzp;
                        } else {
                            v = hxp[e] - (T(NH) * fhx[e]) * (rest + zp);
                        }
                        hxn[e] = (cin[e] && !xw[e]) ? v : T(0);
                    }
                    // Hy (i+1/2, j, k-1/2)
                    {
                        const T ezn = e < V - 1 ? ezq[e < V - 1 ? e + 1 : 0] : (lane < 31 ? ezr : T(0));
                        const T zp = (ex[e] - exq[e]) * idz;
                        const T rest = -(ezn - ezq[e]) * idx;
                        T v;
                        if constexpr (PML) {
                            T hzp = sy[e];
                            T hr = hyp[e] - hzp;
#pragma unroll
                            for (int s = 0; s < NH; s++) {
                                hzp = (hzp * hdh - fhy[e] * zp) * hdh;
                                hr = hr - fhy[e] * rest;
                            }
                            sy[e] = (cin[e] && !wy) ? hzp : T(0);
                            v = hr + hzp;
                        } else {
                            v = hyp[e] - (T(NH) * fhy[e]) * (rest + zp);
                        }
                        hyn[e] = (cin[e] && !wy) ? v : T(0);
                    }
                }
                };
                if (!hpaired) {
                    if (hp)
                        h_cols(std::true_type{});
                    else
                        h_cols(std::false_type{});
                }
                P::gst(io.Hn[0] + ql, hxn, isH);
                P::gst(io.Hn[1] + ql, hyn, isH);
                if (hp) {
                    P::gst(f.Hzp[0] + ql, sx, isH);
                    P::gst(f.Hzp[1] + ql, sy, isH);
                }
            }
        }
        // ---- advance
        vcopy<T, V>(hxp, hx);
        vcopy<T, V>(hyp, hy);
        vcopy<T, V>(exq, ex);
        vcopy<T, V>(eyq, ey);
        vcopy<T, V>(ezq, ez);
    }
    if (!isfinite(acc) || nonfin) atomicOr(f.err, kErrNonFinite);
}

// Resident CTAs per SM the vectorised kernel is compiled for: two when two
// copies of its shared memory fit in the SM's 228 KB (1 KB per CTA reserved).
// z ranges of the fused pass: chunk c (blockIdx.z) marches planes
// b[c] .. b[c+1]-1 and recomputes plane b[c+1] without storing it.  The host
// places the bounds so the chunks carry equal work: PML planes and planes
// holding a plane source cost more than the others, and the one resident
// wave ends with its slowest chunk.
constexpr int kMaxZChunks = 512;
struct ZChunks {
    int b[kMaxZChunks + 1];
};

template <typename T, typename S, int BY, int ST, bool GEN, bool TMA = false> struct VecMinBlocks {
    static constexpr int value = 2 * (VecLayout<T, S, BY, GEN, ST, TMA>::bytes + 1024) <= 228 * 1024 ? 2 : 1;
};

template <typename T, typename S, int BY, int ST, int NH, bool PMLK, bool GEN>
__global__ void __launch_bounds__(32 * (BY + 1), (VecMinBlocks<T, S, BY, ST, GEN>::value))
    k_fused_vec(const __grid_constant__ Geo g, const __grid_constant__ Fields<T, S> f,
                const __grid_constant__ FusedIO<S> io, const Src<T> *__restrict__ src, int nsrc,
                const __grid_constant__ ZChunks zc, int xstride)
{
    if (timeout_latched(f.err)) return;   // the state is already void; see k_hm_box
    fused_vec_body<T, S, BY, ST, NH, PMLK, GEN>(g, f, io, src, nsrc, f.src_amp, zc.b[blockIdx.z],
                                                zc.b[blockIdx.z + 1], xstride, blockIdx.x, blockIdx.y);
}

// The same pass with the planes staged by bulk tensor copies (TMA): one
// thread per CTA issues each plane's tiles against a per-stage mbarrier, so
// the other threads spend no instructions on copy addresses.  FP32 storage
// without sigma or mu_r; maps are the tensor maps of the buffers read.
template <typename T, typename S, int BY, int ST, int NH, bool PMLK, bool GEN>
__global__ void __launch_bounds__(32 * (BY + 1), (VecMinBlocks<T, S, BY, ST, GEN, true>::value))
    k_fused_vec_tma(const __grid_constant__ Geo g, const __grid_constant__ Fields<T, S> f,
                    const __grid_constant__ FusedIO<S> io, const __grid_constant__ VecMaps maps,
                    const Src<T> *__restrict__ src, int nsrc, const __grid_constant__ ZChunks zc, int xstride)
{
    if (timeout_latched(f.err)) return;
    fused_vec_body<T, S, BY, ST, NH, PMLK, GEN, true>(g, f, io, src, nsrc, f.src_amp, zc.b[blockIdx.z],
                                                      zc.b[blockIdx.z + 1], xstride, blockIdx.x, blockIdx.y, &maps);
}

// One grid of a batch: what the batched fused launch needs per instance, for
// one parity of the E/H ping-pong.
template <typename T, typename S> struct VecInst {
    Geo g;
    Fields<T, S> f;
    FusedIO<S> io;
    const Src<T> *src;
    const T *amp;        // source amplitudes, [step][source]
    int nsrc;
    int chunk, xstride;
};

// Batched fused step: CTA b takes work[b] = {instance, bx, by, bz}.
template <typename T, typename S, int BY, int ST, int NH, bool PMLK, bool GEN>
__global__ void __launch_bounds__(32 * (BY + 1), (VecMinBlocks<T, S, BY, ST, GEN>::value))
    k_fused_vec_batch(const VecInst<T, S> *__restrict__ inst, const int4 *__restrict__ work, int step)
{
    const int4 wk = work[blockIdx.x];
    const VecInst<T, S> &I = inst[wk.x];
    const int k0 = wk.w * I.chunk;
    fused_vec_body<T, S, BY, ST, NH, PMLK, GEN>(I.g, I.f, I.io, I.src, I.nsrc, I.amp + (size_t)step * I.nsrc, k0,
                                                min(k0 + I.chunk, I.g.n[2]), I.xstride, wk.y, wk.z);
}

// Rows per CTA (+1 halo warp), chosen by measurement on the 128x128x512
// waveguide: FP32 7 rows (8 warps, 2 CTAs/SM, no spills: 110 us; 8 rows 123,
// 15 rows 122), FP64 8 rows (1269 us; 7 rows 1316).
#ifndef MMX_VEC_F32_ROWS
#define MMX_VEC_F32_ROWS 7
#endif
#ifndef MMX_VEC_F32_STAGES
#define MMX_VEC_F32_STAGES 2
#endif
template <typename T> struct VecRows;
template <> struct VecRows<float> { static constexpr int value = MMX_VEC_F32_ROWS; };
template <> struct VecRows<double> { static constexpr int value = 8; };
// Plane stages in the shared-memory ring (2: two CTAs per SM; more: one CTA
// per SM with ST-1 planes in flight).  Variants that also stage the ca
// arrays (sigma != 0) keep two stages to fit in shared memory.
template <typename T, bool GEN> struct VecStages { static constexpr int value = 2; };
template <> struct VecStages<float, false> { static constexpr int value = MMX_VEC_F32_STAGES; };

// One H half step (Steps 1/3 on non-magnetic faces, Eq. iterate_H with mu;
// the same operations as k_h_update / h_face_nonmag_val) on every face
// outside the magnetic box, in place, for grids with PEC x and y walls: the
// first H half step of an mmx_step call on the fused path.  A lane owns V
// consecutive columns of one row j of one plane k (16-byte vectors, 8 bytes
// with FP16 storage) and updates Hx, Hy at layer k+1/2 and Hz at node k;
// the column to its right comes from the next lane (lane 31 loads it).  A
// warp covers W = 32 V columns; blocks are (32, 8): eight rows of one plane.
template <typename T, typename S, bool PMLK, bool GEN>
__global__ void __launch_bounds__(256) k_h_half_vec(const __grid_constant__ Geo g,
                                                    const __grid_constant__ Fields<T, S> f, int blo0, int blo1,
                                                    int blo2, int bhi0, int bhi1, int bhi2)
{
    using P = SV<S>;
    constexpr int V = Lanes<T>::V, W = 32 * V;
    const int lane = threadIdx.x;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int x0 = blockIdx.x * W, i0 = x0 + V * lane;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    const bool on = j <= ny && i0 <= nx;   // some column of this lane is a node column
    const T sE = f.sE, sH = f.sH, isH = f.isH;
    const T idx = f.inv_d[0], idy = f.inv_d[1], idz = f.inv_d[2];
    const unsigned X = (unsigned)g.X, XY = (unsigned)g.X * (unsigned)g.Y;
    const unsigned q = (unsigned)i0 + X * (unsigned)j + XY * (unsigned)k;
    const bool kin = k < nz, jin = j < ny;           // a cell layer above / row after exists
    const bool zwall = !g.per[2] && (k == 0 || k == nz);
    const bool pml = PMLK && kin && pml_h_plane(g, k);
    T ex[V], ey[V], ez[V], eyk[V], exk[V], ezj[V], exj[V];
    vzero<T, V>(ex);
    vzero<T, V>(ey);
    vzero<T, V>(ez);
    vzero<T, V>(eyk);
    vzero<T, V>(exk);
    vzero<T, V>(ezj);
    vzero<T, V>(exj);
    if (on) {
        P::gld(ex, f.E[0] + q, sE);
        P::gld(ey, f.E[1] + q, sE);
        if (kin) {
            P::gld(ez, f.E[2] + q, sE);
            P::gld(eyk, f.E[1] + q + XY, sE);
            P::gld(exk, f.E[0] + q + XY, sE);
            if (jin) P::gld(ezj, f.E[2] + q + X, sE);
        }
        if (jin) P::gld(exj, f.E[0] + q + X, sE);
    }
    // column i0 + V: the next lane's first element, lane 31 loads it
    T eyr = __shfl_down_sync(0xffffffffu, ey[0], 1);
    T ezr = __shfl_down_sync(0xffffffffu, ez[0], 1);
    if (lane == 31) {
        const bool rin = on && x0 + W <= nx;
        eyr = rin ? ld_s(f.E[1] + q + V, sE) : T(0);
        ezr = (rin && kin) ? ld_s(f.E[2] + q + V, sE) : T(0);
    }
    bool bad = false;
    const bool yrow_box = j >= blo1 && j < bhi1, k_box = k >= blo2 && k < bhi2;
    // every H this thread reads before any of its stores: the three
    // components (and the PML split parts) are then in flight together
    // instead of one round trip per component.  No other thread reads or
    // writes them.
    const bool onx = on && jin && kin, ony = on && kin, onz = on && jin;
    T hn0[V], hn1[V], hn2[V], sp0[V], sp1[V];
    if (onx) P::gld(hn0, f.H[0] + q, sH); else vzero<T, V>(hn0);
    if (ony) P::gld(hn1, f.H[1] + q, sH); else vzero<T, V>(hn1);
    if (onz) P::gld(hn2, f.H[2] + q, sH); else vzero<T, V>(hn2);
    if (pml && onx) P::gld_rw(sp0, f.Hzp[0] + q, sH); else vzero<T, V>(sp0);
    if (pml && ony) P::gld_rw(sp1, f.Hzp[1] + q, sH); else vzero<T, V>(sp1);
    // Hx and Hy with and without the PML split update, chosen per plane
    // (block) rather than inside the unrolled columns
    auto hxy = [&](auto with_pml) {
        constexpr bool PML = decltype(with_pml)::value;
        // ---- Hx (i, j+1/2, k+1/2): j < ny, k < nz
        if (onx) {
            T fh[V], v[V];
            T (&hn)[V] = hn0;
            T (&sp)[V] = sp0;
            if (GEN && f.fh[0]) vload(fh, f.fh[0] + q); else vfill<T, V>(fh, f.fh0);
            bool any = false;
#pragma unroll
            for (int e = 0; e < V; e++) {
                const int i = i0 + e;
                const bool skip = i > nx || (i >= blo0 && i < bhi0 && yrow_box && k_box);
                T val = hn[e];
                if (!skip) {
                    if (i == 0 || i == nx) {
                        val = T(0);
                        sp[e] = T(0);
                    } else {
                        const T rest = (ezj[e] - ez[e]) * idy;
                        const T zp = -(eyk[e] - ey[e]) * idz;
                        if constexpr (PML) {
                            const T h = f.dampH[k];
                            const T hz = sp[e];
                            const T hr = hn[e] - hz;
                            const T hz1 = (hz * h - fh[e] * zp) * h;
                            const T hr1 = hr - fh[e] * rest;
                            sp[e] = hz1;
                            val = hr1 + hz1;
                        } else {
                            val = hn[e] - fh[e] * (rest + zp);
                        }
                    }
                    any = true;
                    bad |= !isfinite(val);
                }
                v[e] = val;
            }
            if (any) {
                P::gst(f.H[0] + q, v, isH);
                if constexpr (PML) P::gst(f.Hzp[0] + q, sp, isH);
            }
        }
        // ---- Hy (i+1/2, j, k+1/2): i < nx, k < nz
        if (ony) {
            T fh[V], v[V];
            T (&hn)[V] = hn1;
            T (&sp)[V] = sp1;
            if (GEN && f.fh[1]) vload(fh, f.fh[1] + q); else vfill<T, V>(fh, f.fh0);
            bool any = false;
#pragma unroll
            for (int e = 0; e < V; e++) {
                const int i = i0 + e;
                const bool skip = i >= nx || (i >= blo0 && i < bhi0 && yrow_box && k_box);
                T val = hn[e];
                if (!skip) {
                    if (j == 0 || j == ny) {
                        val = T(0);
                        sp[e] = T(0);
                    } else {
                        const T ezn = e < V - 1 ? ez[e < V - 1 ? e + 1 : 0] : ezr;
                        const T zp = (exk[e] - ex[e]) * idz;
                        const T rest = -(ezn - ez[e]) * idx;
                        if constexpr (PML) {
                            const T h = f.dampH[k];
                            const T hz = sp[e];
                            const T hr = hn[e] - hz;
                            const T hz1 = (hz * h - fh[e] * zp) * h;
                            const T hr1 = hr - fh[e] * rest;
                            sp[e] = hz1;
                            val = hr1 + hz1;
                        } else {
                            val = hn[e] - fh[e] * (rest + zp);
                        }
                    }
                    any = true;
                    bad |= !isfinite(val);
                }
                v[e] = val;
            }
            if (any) {
                P::gst(f.H[1] + q, v, isH);
                if constexpr (PML) P::gst(f.Hzp[1] + q, sp, isH);
            }
        }
    };
    if (pml)
        hxy(std::true_type{});
    else
        hxy(std::false_type{});
    // ---- Hz (i+1/2, j+1/2, k): i < nx, j < ny
    if (onz) {
        T fh[V], v[V];
        T (&hn)[V] = hn2;
        if (GEN && f.fh[2]) vload(fh, f.fh[2] + q); else vfill<T, V>(fh, f.fh0);
        bool any = false;
#pragma unroll
        for (int e = 0; e < V; e++) {
            const int i = i0 + e;
            const bool skip = i >= nx || (i >= blo0 && i < bhi0 && yrow_box && k_box);
            T val = hn[e];
            if (!skip) {
                if (zwall) {
                    val = T(0);
                } else {
                    const T eyn = e < V - 1 ? ey[e < V - 1 ? e + 1 : 0] : eyr;
                    const T rest = (eyn - ey[e]) * idx - (exj[e] - ex[e]) * idy;
                    const T zp = T(0);
                    val = hn[e] - fh[e] * (rest + zp);
                }
                any = true;
                bad |= !isfinite(val);
            }
            v[e] = val;
        }
        if (any) P::gst(f.H[2] + q, v, isH);
    }
    if (bad) atomicOr(f.err, kErrNonFinite);
}

// Zero the wall column x = nx and the wall row y = ny (all planes) of up to
// 16 Yee arrays: every component there is either a PEC wall value or does
// not exist, and the vectorised kernel never writes it.
template <typename T> struct WallList {
    T *p[16];
    int n;
};

template <typename T> __global__ void k_zero_walls(const Geo g, WallList<T> L)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    size_t q;
    if (t < g.Y)
        q = gidx(g, g.n[0], t, k);
    else if (t < g.Y + g.X)
        q = gidx(g, t - g.Y, g.n[1], k);
    else
        return;
    for (int a = 0; a < L.n; a++) L.p[a][q] = T(0);
}

} // namespace mmx

// mmx.cu -- host side of the C ABI declared in include/mmx.h: context
// lifetime, device memory, material/field setup and the per-step launch
// sequence of the coupled Maxwell-LLG scheme (arXiv 2103.12819, Sec. 3).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "mmx.h"
#include "mmx_fused.cuh"
#include "mmx_box_res.cuh"
#include "mmx_monitor.cuh"
#include "mmx_batch.cuh"
#include "mmx_adjoint.cuh"

using namespace mmx;

namespace {

// Kernel kinds timed by the optional profiler.
enum KernelKind {
    KK_HM_BOX = 0, KK_H_UPDATE, KK_E_UPDATE, KK_HARD, KK_FUSED, KK_FUSED_VEC, KK_FUSED_VEC_TMA, KK_ZERO_WALLS,
    KK_M_SYNC, KK_HM_BOX_RES, KK_H_HALF_VEC, KK_COUNT
};
// fused_eh_vec is k_fused_vec (per-lane cp.async staging), fused_eh_vec_tma
// k_fused_vec_tma (bulk tensor copies); fused_eh the one-column kernel
const char *const kKernelNames[KK_COUNT] = {"hm_box",       "h_update",         "e_update",
                                            "hard_source",  "fused_eh",         "fused_eh_vec",
                                            "fused_eh_vec_tma", "zero_walls",   "box_m_sync",
                                            "hm_box_res",   "h_half_vec"};

struct ProfRec {
    int kind;
    cudaEvent_t a, b;
};

} // namespace

struct mmx_ctx {
    mmx_grid_desc desc;
    Geo g;
    size_t npad = 0;            // padded elements per Yee array
    int esz = 8;                // bytes per element of the arithmetic type
    int ssz = 8;                // bytes per stored E/H element
    double sE = 1.0, sH = 1.0;  // FP16 storage scales
    bool touched = false;       // a field was set or a step taken
    cudaStream_t stream = nullptr;
    int path = MMX_PATH_FUSED;
    std::string err;

    // Yee state (current) and the second set the fused path ping-pongs with
    void *E[3] = {}, *H[3] = {}, *Ezp[2] = {}, *Hzp[2] = {};
    void *Ealt[3] = {}, *Halt[3] = {}, *Ezpalt[2] = {};
    int fused_chunk = 0;
    int fused_grid_z = 0;
    // vectorised fused kernel: plan (0 chunk = not planned) and wall state
    int vec_chunk = 0;
    dim3 vec_grid;
    ZChunks vec_z;           // chunk bounds along z (weighted by plane cost)
    int vec_xstride = 0;
    bool walls_dirty = false;
    // bulk-tensor (TMA) staging of the vectorised kernel: -1 not planned,
    // 0 not used, 1 used; one map set per E/H ping-pong parity, keyed by the
    // H array it reads
    int vec_tma = -1;
    int bulk_staging = 1;    // caller's choice (mmx_set_fused_staging)
    int tma_fallback = 0;    // 1: bulk copies apply but their set-up failed
    int last_fused = 0;      // kernel of the last fused step (mmx_info.fused_kernel)
    bool inject_timeout = false;   // test hook: see mmx_inject_timeout
    VecMaps vmaps[2];
    void *vmap_key[2] = {};
    // coefficients
    void *ca[3] = {}, *cb[3] = {}, *fh[3] = {};
    void *epsc = nullptr;                  // FP32 arithmetic: eps_r per cell, padded
    void *dampE = nullptr, *dampH = nullptr;
    bool any_sigma = false, any_mu = false;
    // cell-centred materials (double, compact nx*ny*nz; null = default)
    double *cell[6] = {};
    double h0[3] = {0, 0, 0};

    // magnetic box
    bool magnetic = false;
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    int bx = 0, by = 0, bz = 0;
    long long nb = 0;
    std::vector<void *> box_allocs;
    void *bM[9] = {}, *bHit[2][3] = {}, *bHit2[2][3] = {};
    void *fcst = nullptr, *fmn = nullptr, *fbc = nullptr, *fdm[2] = {};   // per magnetic face (list order)
    void *bms[3] = {}, *bk1[3] = {}, *bk2[3] = {};
    // arrays placed by dalloc, each with its guard bytes after `second` bytes
    std::vector<std::pair<void *, size_t>> guards;
    int4 *dmag = nullptr, *dnon = nullptr;
    unsigned *dmag32 = nullptr;   // the magnetic list's packed first words
    int nmag = 0, nnon = 0;
    int coop_blocks = 0;
    // H/M box kernel with the records in shared memory (k_hm_box_res): faces
    // per thread (0: the magnetic faces do not fit, k_hm_box runs) and blocks
    int res_faces = 0, res_blocks = 0;
    int box_resident = 1;    // caller's choice (mmx_set_box_kernel)
    bool h_half_vec = true;  // the fused path's first H half step vectorised
    // M lives in two places: the box arrays (read and written through the
    // API) and the magnetic-face records (used while stepping).  Each copy
    // is refreshed from the other only when something reads it.
    bool m_rec_stale = true;   // the box arrays hold a newer M than the records
    bool m_box_stale = false;  // the records hold a newer M than the box arrays
    int last_box = 0;        // kernel of the last box launch (mmx_info.box_kernel)

    // point probes of E: (field, padded index) per probe and a device table
    // of samples, one row of nprobe doubles per completed time step
    std::vector<int2> probes;
    int2 *dprobe = nullptr;
    double *probe_buf = nullptr;
    long long probe_rows = 0;

    // monitors: block partial sums, flux planes and their accumulators
    // ({sum, correction, last power, unused} per plane)
    double2 *mon_partial = nullptr;
    std::vector<int> flux_k;
    double *flux_acc = nullptr;

    // control words (device)
    unsigned long long *res = nullptr;     // [8][kMaxIter+1]: residual maxima, then decision words
    unsigned long long *bar = nullptr;     // grid-barrier arrival count
    int *iterlog = nullptr;                // [kIterLogCap]
    unsigned long long *halfsteps = nullptr;
    double *last_res = nullptr;
    int *errw = nullptr;
    int box_slot = 0;

    // sources: descriptors, per-step waveform table (T, kAmpChunk x nsrc)
    // and the TE10 profile tables (T, nx+1 each)
    std::vector<mmx_source_desc> src;
    void *dsrc = nullptr;
    void *damp = nullptr;
    void *dprof[2] = {};

    // staging
    double *stage = nullptr;
    size_t stage_elems = 0;

    long long steps = 0;

    // optional per-kernel profile
    bool prof_on = false;
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> prof_pool;
    long long prof_launches[KK_COUNT] = {};
    double prof_ms[KK_COUNT] = {};
    int prof_open = -1;
    bool nvtx_open = false;  // an NVTX range of the current launch is open
};

// ------------------------------------------------------------- helpers

static int fail(mmx_ctx *c, int code, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

#define CK_RAW(call)                                                                              \
    do {                                                                                          \
        if ((call) != cudaSuccess) return MMX_ERR_CUDA;                                            \
    } while (0)

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? MMX_ERR_OOM : MMX_ERR_CUDA,        \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);     \
    } while (0)

static bool is_fp64(const mmx_ctx *c) { return c->desc.prec == MMX_FP64; }
static bool is_fp16(const mmx_ctx *c) { return c->desc.prec == MMX_FP16; }

constexpr int kAmpChunk = 1024;   // steps whose source values are uploaded at once

static cudaEvent_t prof_event(mmx_ctx *c)
{
    if (!c->prof_pool.empty()) {
        cudaEvent_t e = c->prof_pool.back();
        c->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket the next launch with events when profiling is enabled.
// Every timed launch is also an NVTX range named like its profile entry, so
// that a timeline tool shows the kernels of a step by name (the calls do
// nothing when no tool is attached).
static void prof_begin(mmx_ctx *c, int kind)
{
    nvtxRangePushA(kKernelNames[kind]);
    c->nvtx_open = true;
    if (!c->prof_on) return;
    ProfRec r;
    r.kind = kind;
    r.a = prof_event(c);
    r.b = prof_event(c);
    cudaEventRecord(r.a, c->stream);
    c->prof_recs.push_back(r);
    c->prof_open = (int)c->prof_recs.size() - 1;
}

static void prof_end(mmx_ctx *c)
{
    if (c->nvtx_open) {
        nvtxRangePop();
        c->nvtx_open = false;
    }
    if (!c->prof_on || c->prof_open < 0) return;
    cudaEventRecord(c->prof_recs[c->prof_open].b, c->stream);
    c->prof_open = -1;
}

static void prof_collect(mmx_ctx *c)
{
    for (ProfRec &r : c->prof_recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            c->prof_ms[r.kind] += ms;
            c->prof_launches[r.kind] += 1;
        }
        c->prof_pool.push_back(r.a);
        c->prof_pool.push_back(r.b);
    }
    c->prof_recs.clear();
}

static void edge_ext(const mmx_ctx *c, int comp, int e[3])
{
    for (int a = 0; a < 3; a++) e[a] = c->desc.n[a] + (a == comp ? 0 : 1);
}
static void face_ext(const mmx_ctx *c, int fam, int e[3])
{
    for (int a = 0; a < 3; a++) e[a] = c->desc.n[a] + (a == fam ? 1 : 0);
}

// Extents of a field id; returns false for an unknown id.
static size_t gidx_host(const mmx_ctx *c, int i, int j, int k)
{
    return (size_t)i + (size_t)c->g.X * ((size_t)j + (size_t)c->g.Y * (size_t)k);
}

constexpr int kMaxProbes = 16;
constexpr long long kProbeRows = 1 << 16;

static bool field_ext(const mmx_ctx *c, int id, int e[3])
{
    if (id >= 0 && id < 3) { edge_ext(c, id, e); return true; }
    if (id >= 3 && id < 6) { face_ext(c, id - 3, e); return true; }
    if (id >= 6 && id < 15) { face_ext(c, (id - 6) / 3, e); return true; }
    if (id == 15 || id == 16) { edge_ext(c, id - 15, e); return true; }
    if (id == 17 || id == 18) { face_ext(c, id - 17, e); return true; }
    return false;
}

static dim3 node_block() { return dim3(32, 8, 1); }
static dim3 node_grid(const mmx_ctx *c)
{
    return dim3((c->desc.n[0] + 1 + 31) / 32, (c->desc.n[1] + 1 + 7) / 8, c->desc.n[2] + 1);
}

// Every array dalloc places is followed by kGuardBytes of a fixed pattern;
// mmx_check_guards reads them back, so that a kernel writing past the end
// of one of the context's arrays is caught (the canary check of the tests,
// in place of a memory sanitizer).
constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xC3;

static int dalloc(mmx_ctx *ctx, void **p, size_t bytes)
{
    const size_t n = bytes > 0 ? bytes : 1;
    CK(cudaMalloc(p, n + kGuardBytes));
    CK(cudaMemsetAsync(*p, 0, n, ctx->stream));
    CK(cudaMemsetAsync((unsigned char *)*p + n, kGuardByte, kGuardBytes, ctx->stream));
    ctx->guards.push_back({*p, n});
    return MMX_OK;
}

// Free an array dalloc placed before the context ends (its guard goes too).
static void dfree(mmx_ctx *ctx, void *p)
{
    if (!p) return;
    for (size_t q = 0; q < ctx->guards.size(); q++)
        if (ctx->guards[q].first == p) {
            ctx->guards.erase(ctx->guards.begin() + (long)q);
            break;
        }
    cudaFree(p);
}

template <typename T, typename S = T> static Fields<T, S> make_fields(mmx_ctx *c)
{
    Fields<T, S> f;
    for (int a = 0; a < 3; a++) {
        f.E[a] = (S *)c->E[a];
        f.H[a] = (S *)c->H[a];
        f.ca[a] = (const T *)c->ca[a];
        f.cb[a] = (const T *)c->cb[a];
        f.fh[a] = (const T *)c->fh[a];
    }
    for (int a = 0; a < 2; a++) {
        f.Ezp[a] = (S *)c->Ezp[a];
        f.Hzp[a] = (S *)c->Hzp[a];
    }
    f.sE = (T)c->sE;
    f.sH = (T)c->sH;
    f.isE = (T)(1.0 / c->sE);
    f.isH = (T)(1.0 / c->sH);
    f.fh0 = (T)(c->desc.dt / (2.0 * kMu0));
    f.dampE = (const T *)c->dampE;
    f.dampH = (const T *)c->dampH;
    for (int a = 0; a < 3; a++) f.inv_d[a] = (T)(1.0 / c->desc.d[a]);
    f.src_amp = (const T *)c->damp;
    f.prof[0] = (const T *)c->dprof[0];
    f.prof[1] = (const T *)c->dprof[1];
    f.err = c->errw;
    f.epsc = sizeof(T) == 4 ? (const T *)c->epsc : nullptr;
    f.kcb = (T)(4.0 * c->desc.dt * kMu0 * kC0 * kC0);
    return f;
}

template <typename T> static Box<T> make_box(mmx_ctx *c)
{
    Box<T> b;
    memset(&b, 0, sizeof b);
    for (int a = 0; a < 3; a++) b.lo[a] = c->lo[a];
    b.bx = c->bx; b.by = c->by; b.bz = c->bz; b.nb = c->nb;
    for (int q = 0; q < 9; q++) b.M[q] = (T *)c->bM[q];
    b.cst = (const Q4<T> *)c->fcst;
    b.mn = (Q4<T> *)c->fmn;
    b.bc = (Q4<T> *)c->fbc;
    b.dm[0] = (Q4<T> *)c->fdm[0];
    b.dm[1] = (Q4<T> *)c->fdm[1];
    for (int a = 0; a < 3; a++) {
        b.Hit[0][a] = (T *)c->bHit[0][a];
        b.Hit[1][a] = (T *)c->bHit[1][a];
        b.Hit2[0][a] = (T *)c->bHit2[0][a];
        b.Hit2[1][a] = (T *)c->bHit2[1][a];
        b.ms[a] = (const T *)c->bms[a];
        b.k1[a] = (const T *)c->bk1[a];
        b.k2[a] = (const T *)c->bk2[a];
        b.h0[a] = c->h0[a];
    }
    b.tol = c->desc.tol;
    b.max_iter = c->desc.max_iter;
    b.order = c->desc.order;
    b.cfar = (T)(c->desc.dt / (2.0 * kMu0));
    b.res = c->res;
    b.bar = c->bar;
    b.iterlog = c->iterlog;
    b.halfsteps = c->halfsteps;
    b.last_res = c->last_res;
    b.err = c->errw;
    b.mag = c->dmag;
    b.nonmag = c->dnon;
    b.mag32 = c->dmag32;
    b.nmag = c->nmag;
    b.nnon = c->nnon;
    return b;
}

// PML damping tables: E at z node k, H at z cell centre k + 1/2; identical
// to 1 outside the layers.  sigma_z = smax (depth/L)^3 with
// smax = -(m+1) eps0 c ln(R0)/(2 L), m = 3, R0 = 1e-8, L = npml dz.
static void pml_tables(const mmx_ctx *c, std::vector<double> &dE, std::vector<double> &dH)
{
    int nz = c->desc.n[2], np = c->g.npml;
    double dz = c->desc.d[2], dt = c->desc.dt;
    double e0 = 1.0 / (kMu0 * kC0 * kC0);
    dE.assign(nz + 1, 1.0);
    dH.assign(nz, 1.0);
    if (np <= 0) return;
    double L = np * dz;
    double zlo = L, zhi = (nz - np) * dz;
    double smax = -(3.0 + 1.0) * e0 * kC0 * std::log(1e-8) / (2.0 * L);
    auto sig = [&](double z) {
        double depth;
        if (z < zlo) depth = (zlo - z) / L;
        else if (z > zhi) depth = (z - zhi) / L;
        else return 0.0;
        return smax * depth * depth * depth;
    };
    for (int k = 0; k <= nz; k++) {
        double s = sig(k * dz);
        if (s > 0.0) dE[k] = std::exp(-s * dt / (2.0 * e0));
    }
    for (int k = 0; k < nz; k++) {
        double s = sig((k + 0.5) * dz);
        if (s > 0.0) dH[k] = std::exp(-s * (dt / 4.0) / e0);
    }
}

// Waveform of a source, g(t) = amp exp(-(t-t0)^2/(2 tp^2)) cos(2 pi f0 t).
static double host_waveform(const mmx_source_desc &q, double t)
{
    double u = t - q.t0;
    return q.amp * std::exp(-u * u / (2.0 * q.tp * q.tp)) * std::cos(2.0 * kPi * q.f0 * t);
}

// Soft-source values at t = (n + 1/2) dt for steps n0 .. n0+cnt-1.
template <typename T> static int upload_amplitudes(mmx_ctx *ctx, long long n0, int cnt)
{
    size_t ns = ctx->src.size();
    if (ns == 0) return MMX_OK;
    std::vector<T> v((size_t)cnt * ns);
    for (int s = 0; s < cnt; s++)
        for (size_t q = 0; q < ns; q++) {
            const mmx_source_desc &d = ctx->src[q];
            double val = (d.kind == 0 || d.kind == 1) ? host_waveform(d, ((double)(n0 + s) + 0.5) * ctx->desc.dt) : 0.0;
            v[(size_t)s * ns + q] = (T)val;
        }
    CK(cudaMemcpyAsync(ctx->damp, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    // the host vector dies at return: wait for the copy
    CK(cudaStreamSynchronize(ctx->stream));
    return MMX_OK;
}

template <typename T> static int upload_table(mmx_ctx *ctx, void **dst, const std::vector<double> &v)
{
    std::vector<T> t(v.begin(), v.end());
    int rc = dalloc(ctx, dst, t.size() * sizeof(T));
    if (rc) return rc;
    CK(cudaMemcpyAsync(*dst, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MMX_OK;
}

static int ensure_stage(mmx_ctx *ctx, size_t elems)
{
    if (ctx->stage_elems >= elems) return MMX_OK;
    if (ctx->stage) cudaFree(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_elems = 0;
    CK(cudaMalloc((void **)&ctx->stage, elems * sizeof(double)));
    ctx->stage_elems = elems;
    return MMX_OK;
}

static void free_box(mmx_ctx *c)
{
    for (void *p : c->box_allocs) dfree(c, p);
    c->box_allocs.clear();
    c->magnetic = false;
    c->nb = 0;
    c->dmag = c->dnon = nullptr;
    c->dmag32 = nullptr;
    c->nmag = c->nnon = 0;
    c->fcst = c->fmn = c->fbc = c->fdm[0] = c->fdm[1] = nullptr;
}

// Work lists of the box kernel: every valid face of the box, split into
// magnetic faces (an adjacent cell has Ms > 0, i.e. Ms_face > 0) and the rest;
// entries {box index | family << 30, i, j, k}.
static int build_box_lists(mmx_ctx *ctx, const double *Ms)
{
    const int *n = ctx->desc.n;
    std::vector<int4> mag, non;
    auto cell_ms = [&](int i, int j, int k) {
        return Ms[(size_t)i + (size_t)n[0] * ((size_t)j + (size_t)n[1] * k)];
    };
    for (int d = 0; d < 3; d++)
        for (int k = ctx->lo[2]; k < ctx->hi[2]; k++)
            for (int j = ctx->lo[1]; j < ctx->hi[1]; j++)
                for (int i = ctx->lo[0]; i < ctx->hi[0]; i++) {
                    int ix[3] = {i, j, k};
                    bool valid = true;
                    for (int a = 0; a < 3; a++)
                        if (ix[a] > n[a] || (a != d && ix[a] >= n[a])) valid = false;
                    if (!valid) continue;
                    bool magnetic = false;
                    for (int o = -1; o <= 0; o++) {
                        int cc[3] = {i, j, k};
                        int v = ix[d] + o;
                        if (v < 0 || v >= n[d]) {
                            if (!ctx->g.per[d]) continue;
                            v = (v + n[d]) % n[d];
                        }
                        cc[d] = v;
                        if (cell_ms(cc[0], cc[1], cc[2]) > 0) magnetic = true;
                    }
                    unsigned l = (unsigned)(i - ctx->lo[0]) +
                                 (unsigned)ctx->bx * ((unsigned)(j - ctx->lo[1]) + (unsigned)ctx->by * (unsigned)(k - ctx->lo[2]));
                    int4 e = make_int4((int)(l | ((unsigned)d << 30)), i, j, k);
                    (magnetic ? mag : non).push_back(e);
                }
    ctx->nmag = (int)mag.size();
    ctx->nnon = (int)non.size();
    void *pm = nullptr, *pn = nullptr;
    int rc = dalloc(ctx, &pm, std::max<size_t>(1, mag.size()) * sizeof(int4));
    if (rc) return rc;
    ctx->box_allocs.push_back(pm);
    rc = dalloc(ctx, &pn, std::max<size_t>(1, non.size()) * sizeof(int4));
    if (rc) return rc;
    ctx->box_allocs.push_back(pn);
    if (!mag.empty()) CK(cudaMemcpy(pm, mag.data(), mag.size() * sizeof(int4), cudaMemcpyHostToDevice));
    if (!non.empty()) CK(cudaMemcpy(pn, non.data(), non.size() * sizeof(int4), cudaMemcpyHostToDevice));
    ctx->dmag = (int4 *)pm;
    ctx->dnon = (int4 *)pn;
    std::vector<unsigned> m32(mag.size());
    for (size_t q = 0; q < mag.size(); q++) m32[q] = (unsigned)mag[q].x;
    void *p32 = nullptr;
    rc = dalloc(ctx, &p32, std::max<size_t>(1, m32.size()) * sizeof(unsigned));
    if (rc) return rc;
    ctx->box_allocs.push_back(p32);
    if (!m32.empty()) CK(cudaMemcpy(p32, m32.data(), m32.size() * sizeof(unsigned), cudaMemcpyHostToDevice));
    ctx->dmag32 = (unsigned *)p32;
    return MMX_OK;
}

static int box_alloc(mmx_ctx *ctx, void **p)
{
    int rc = dalloc(ctx, p, (size_t)ctx->nb * ctx->esz);
    if (rc == MMX_OK) ctx->box_allocs.push_back(*p);
    return rc;
}

// Resident blocks per SM of the shared-memory H/M kernel with F faces per
// thread: the smaller of its second- and first-order instantiations.
template <typename T, typename S, int F> static int res_occupancy(int *per)
{
    const size_t sm = res_smem_bytes<T>(F);
    int p1 = 0, p2 = 0;
    CK_RAW(cudaFuncSetAttribute(k_hm_box_res<T, S, F, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    CK_RAW(cudaFuncSetAttribute(k_hm_box_res<T, S, F, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    CK_RAW(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p1, k_hm_box_res<T, S, F, 1>, kResThreads, sm));
    CK_RAW(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p2, k_hm_box_res<T, S, F, 2>, kResThreads, sm));
    *per = std::min(p1, p2);
    return MMX_OK;
}

template <typename T, typename S = T> static int compute_coop(mmx_ctx *ctx)
{
    int dev = 0, nsm = 0, per = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    {
        int p1 = 0, p2 = 0;   // first- and second-order instantiations
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p1, k_hm_box<T, S, 1>, 256, 0));
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p2, k_hm_box<T, S, 2>, 256, 0));
        per = std::min(p1, p2);
    }
    if (per < 1) return fail(ctx, MMX_ERR_CUDA, "H/M kernel cannot be resident");
    long long need = (std::max(ctx->nmag, ctx->nnon) + 255) / 256;
    long long cap = (long long)per * nsm;
    ctx->coop_blocks = (int)std::max(1LL, std::min(need, cap));
    // the records in shared memory: the fewest faces per thread (up to
    // kResMaxF, FP32 arithmetic) with which one resident wave covers every
    // magnetic face
    ctx->res_faces = ctx->res_blocks = 0;
    if constexpr (sizeof(T) == 4) {
        for (int F = 1; F <= kResMaxF && ctx->nmag > 0; F++) {
            int pr = 0;
            int rc = F == 1 ? res_occupancy<T, S, 1>(&pr) : F == 2 ? res_occupancy<T, S, 2>(&pr)
                                                                   : res_occupancy<T, S, 3>(&pr);
            if (rc) {
                cudaGetLastError();
                break;
            }
            const long long blocks = ((long long)ctx->nmag + (long long)F * kResThreads - 1) / ((long long)F * kResThreads);
            if (pr >= 1 && blocks <= (long long)pr * nsm) {
                ctx->res_faces = F;
                ctx->res_blocks = (int)blocks;
                break;
            }
        }
    }
    return MMX_OK;
}

// ------------------------------------------------------------ materials

template <typename T, typename S = T> static int set_materials_t(mmx_ctx *ctx)
{
    const Geo &g = ctx->g;
    dim3 B = node_block(), G = node_grid(ctx);
    double *eps_c = ctx->cell[0], *sig_c = ctx->cell[1], *mu_c = ctx->cell[2];
    if (ctx->epsc && sizeof(T) == 4) {
        k_eps_cells<T><<<G, B, 0, ctx->stream>>>(g, eps_c, (T *)ctx->epsc);
        CK(cudaGetLastError());
    }
    for (int c = 0; c < 3; c++) {
        k_e_coef<T><<<G, B, 0, ctx->stream>>>(g, eps_c, sig_c, c, (T *)ctx->ca[c], (T *)ctx->cb[c]);
        CK(cudaGetLastError());
        if (ctx->fh[c]) {
            k_h_coef<T><<<G, B, 0, ctx->stream>>>(g, mu_c, c, (T *)ctx->fh[c]);
            CK(cudaGetLastError());
        }
    }
    if (ctx->magnetic) {
        Box<T> b = make_box<T>(ctx);
        int nblk = (int)((ctx->nb + 255) / 256);
        for (int d = 0; d < 3; d++) {
            k_box_materials<T><<<nblk, 256, 0, ctx->stream>>>(g, b, d, ctx->cell[3], ctx->cell[4], ctx->cell[5]);
            CK(cudaGetLastError());
        }
        if (ctx->nmag > 0) {
            k_box_cst<T><<<(ctx->nmag + 255) / 256, 256, 0, ctx->stream>>>(b);
            CK(cudaGetLastError());
        }
        int rc = compute_coop<T, S>(ctx);
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return MMX_OK;
}

// ------------------------------------------------------------ stepping

// One cooperative launch over the magnetic box: nsub H/M half steps with
// the E in f.E, starting from the H in f.H and ending in Hout.
template <typename T, typename S>
static int launch_box(mmx_ctx *ctx, const Fields<T, S> &f, const Box<T> &b, Ptr3<S> Hout, int nsub)
{
    int slot = ctx->box_slot;
    ctx->box_slot ^= 1;
    void *args[] = {(void *)&ctx->g, (void *)&f, (void *)&b, (void *)&Hout, (void *)&nsub, (void *)&slot};
    cudaError_t e = cudaSuccess;
    bool done = false;
    if constexpr (sizeof(T) == 4) {   // the resident kernel exists for FP32 arithmetic only
        if (ctx->res_faces > 0 && ctx->box_resident) {
            // the scheme order is a template argument: with a run-time test
            // the first-order branch cost the second-order launch 1.5 us
            const bool o2 = ctx->desc.order == 2;
            const void *fn = ctx->res_faces == 1   ? (o2 ? (const void *)k_hm_box_res<T, S, 1, 2>
                                                         : (const void *)k_hm_box_res<T, S, 1, 1>)
                             : ctx->res_faces == 2 ? (o2 ? (const void *)k_hm_box_res<T, S, 2, 2>
                                                         : (const void *)k_hm_box_res<T, S, 2, 1>)
                                                   : (o2 ? (const void *)k_hm_box_res<T, S, 3, 2>
                                                         : (const void *)k_hm_box_res<T, S, 3, 1>);
            ctx->last_box = 2;
            prof_begin(ctx, KK_HM_BOX_RES);
            e = cudaLaunchCooperativeKernel(fn, dim3(ctx->res_blocks), dim3(kResThreads), args,
                                            res_smem_bytes<T>(ctx->res_faces), ctx->stream);
            done = true;
        }
    }
    if (!done) {
        ctx->last_box = 1;
        prof_begin(ctx, KK_HM_BOX);
        const void *fn = ctx->desc.order == 2 ? (const void *)k_hm_box<T, S, 2> : (const void *)k_hm_box<T, S, 1>;
        e = cudaLaunchCooperativeKernel(fn, dim3(ctx->coop_blocks), dim3(256), args, 0, ctx->stream);
    }
    prof_end(ctx);
    CK(e);
    return MMX_OK;
}

// The vectorised H half step (PEC x and y walls) outside the box [lo, hi).
template <typename T, typename S>
static void launch_h_half_vec(mmx_ctx *ctx, const Fields<T, S> &f, const int lo[3], const int hi[3])
{
    constexpr int W = 32 * Lanes<T>::V;
    const int *n = ctx->desc.n;
    // Columns 0 .. nx-1 and rows 0 .. ny-1: the only faces beyond them, Hx on
    // the wall x = nx and Hy on the wall y = ny, are PEC zeros that zero_walls
    // (after a set_field) or the previous steps left in place.  With nx a
    // multiple of the strip width the wall column alone would take a strip of
    // nearly idle blocks: 110 -> 69 us per launch on the 128x128x512 guide.
    dim3 B(32, 8), G((n[0] + W - 1) / W, (n[1] + 7) / 8, n[2] + 1);
    const bool pml = ctx->g.npml > 0, gen = ctx->any_sigma || ctx->any_mu;
    prof_begin(ctx, KK_H_HALF_VEC);
#define MMX_HHV(PV, GV)                                                                                   \
    if (pml == PV && gen == GV)                                                                           \
        k_h_half_vec<T, S, PV, GV><<<G, B, 0, ctx->stream>>>(ctx->g, f, lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]);
    MMX_HHV(false, false) MMX_HHV(false, true) MMX_HHV(true, false) MMX_HHV(true, true)
#undef MMX_HHV
    prof_end(ctx);
}

// One H/M half step in place: the box kernel on the magnetic box, then the
// non-magnetic update on every other face (the vectorised kernel when vec:
// PEC x and y walls, as on the fused path).
template <typename T, typename S>
static int half_step(mmx_ctx *ctx, const Fields<T, S> &f, const Box<T> &b, double t_end, bool vec = false)
{
    dim3 B = node_block(), G = node_grid(ctx);
    const int none[3] = {0, 0, 0};
    if (ctx->magnetic) {
        Ptr3<S> Hout = {{f.H[0], f.H[1], f.H[2]}};
        int rc = launch_box<T, S>(ctx, f, b, Hout, 1);
        if (rc) return rc;
        if (vec) {
            launch_h_half_vec<T, S>(ctx, f, ctx->lo, ctx->hi);
        } else {
            prof_begin(ctx, KK_H_UPDATE);
            k_h_update<T, S><<<G, B, 0, ctx->stream>>>(ctx->g, f, ctx->lo[0], ctx->lo[1], ctx->lo[2], ctx->hi[0],
                                                        ctx->hi[1], ctx->hi[2]);
            prof_end(ctx);
        }
    } else if (vec) {
        launch_h_half_vec<T, S>(ctx, f, none, none);
    } else {
        prof_begin(ctx, KK_H_UPDATE);
        k_h_update<T, S><<<G, B, 0, ctx->stream>>>(ctx->g, f, 0, 0, 0, 0, 0, 0);
        prof_end(ctx);
    }
    CK(cudaGetLastError());
    bool hardH = false;
    for (auto &s : ctx->src) hardH |= s.kind == 3;
    if constexpr (std::is_same<T, S>::value)
    if (hardH) {
        Ptr3<T> F = {{f.H[0], f.H[1], f.H[2]}};
        prof_begin(ctx, KK_HARD);
        k_hard<T><<<1, 32, 0, ctx->stream>>>(ctx->g, F, (const Src<T> *)ctx->dsrc, (int)ctx->src.size(), 3, t_end);
        prof_end(ctx);
        CK(cudaGetLastError());
    }
    return MMX_OK;
}

// Record the probes after a completed time step (E^(n+1) in ctx->E).
template <typename T, typename S = T> static int record_probes(mmx_ctx *ctx)
{
    if (ctx->probes.empty() || ctx->probe_rows >= kProbeRows) return MMX_OK;
    Ptr3<S> E = {{(S *)ctx->E[0], (S *)ctx->E[1], (S *)ctx->E[2]}};
    const int np = (int)ctx->probes.size();
    k_probe<S, T><<<1, 64, 0, ctx->stream>>>(E, (T)ctx->sE, ctx->dprobe, np,
                                             ctx->probe_buf + ctx->probe_rows * np);
    CK(cudaGetLastError());
    ctx->probe_rows++;
    return MMX_OK;
}

// Add this step's Poynting power x dt to every flux plane's accumulator; H
// at the time level of E is the mean of Ha and Hb.
template <typename T, typename S = T> static int record_flux(mmx_ctx *ctx, Ptr3<S> E, Ptr3<S> Ha, Ptr3<S> Hb)
{
    const int npt = ctx->g.X * (ctx->desc.n[1] + 1);
    const int nblk = std::min(kMonitorBlocks, (npt + kMonitorThreads - 1) / kMonitorThreads);
    for (size_t p = 0; p < ctx->flux_k.size(); p++) {
        k_flux_partial<S, T><<<nblk, kMonitorThreads, 0, ctx->stream>>>(ctx->g, E, Ha, Hb, (T)ctx->sE, (T)ctx->sH,
                                                                          ctx->flux_k[p], ctx->mon_partial);
        k_flux_accumulate<<<1, kMonitorThreads, 0, ctx->stream>>>(ctx->mon_partial, nblk, ctx->desc.dt,
                                                                  ctx->flux_acc + 4 * p);
        CK(cudaGetLastError());
    }
    return MMX_OK;
}

template <typename T> static int step_plain(mmx_ctx *ctx, int nsteps)
{
    Fields<T> f = make_fields<T>(ctx);
    Box<T> b = make_box<T>(ctx);
    dim3 B = node_block(), G = node_grid(ctx);
    int nsrc = (int)ctx->src.size();
    bool hardE = false;
    for (auto &s : ctx->src) hardE |= s.kind == 2;
    const T *amp0 = (const T *)ctx->damp;
    for (int s = 0; s < nsteps; s++) {
        long long n = ctx->steps;
        double dt = ctx->desc.dt;
        if (s % kAmpChunk == 0) {
            int rc = upload_amplitudes<T>(ctx, n, std::min(kAmpChunk, nsteps - s));
            if (rc) return rc;
        }
        f.src_amp = amp0 + (size_t)(s % kAmpChunk) * nsrc;
        int rc = half_step<T, T>(ctx, f, b, (n + 0.5) * dt);
        if (rc) return rc;
        prof_begin(ctx, KK_E_UPDATE);
        k_e_update<T><<<G, B, 0, ctx->stream>>>(ctx->g, f, (const Src<T> *)ctx->dsrc, nsrc);
        prof_end(ctx);
        CK(cudaGetLastError());
        if (hardE) {
            Ptr3<T> F = {{f.E[0], f.E[1], f.E[2]}};
            prof_begin(ctx, KK_HARD);
            k_hard<T><<<1, 32, 0, ctx->stream>>>(ctx->g, F, (const Src<T> *)ctx->dsrc, nsrc, 2, (n + 1.0) * dt);
            prof_end(ctx);
            CK(cudaGetLastError());
        }
        rc = half_step<T, T>(ctx, f, b, (n + 1.0) * dt);
        if (rc) return rc;
        ctx->steps++;
        rc = record_probes<T, T>(ctx);
        if (!rc && !ctx->flux_k.empty()) {
            Ptr3<T> E = {{f.E[0], f.E[1], f.E[2]}}, H = {{f.H[0], f.H[1], f.H[2]}};
            rc = record_flux<T, T>(ctx, E, H, H);
        }
        if (rc) return rc;
    }
    return MMX_OK;
}

// ------------------------------------------------------------ fused path

constexpr int kFBX = 32, kFBY = 8;   // fused block: 31 x 7 output columns + halo

// M between the box arrays and the magnetic-face records (see k_box_m_sync).
template <typename T> static int box_m_sync(mmx_ctx *ctx, int to_rec)
{
    if (!ctx->magnetic || ctx->nmag == 0) return MMX_OK;
    prof_begin(ctx, KK_M_SYNC);
    k_box_m_sync<T><<<(ctx->nmag + 255) / 256, 256, 0, ctx->stream>>>(make_box<T>(ctx), to_rec);
    prof_end(ctx);
    CK(cudaGetLastError());
    return MMX_OK;
}

// Bring the box arrays up to date before anything reads or writes them
// there (field copies of M, the adjoint, a batch call); after stepping the
// records hold the current M.
static int ensure_box_m(mmx_ctx *ctx)
{
    if (!ctx->m_box_stale) return MMX_OK;
    int rc = is_fp64(ctx) ? box_m_sync<double>(ctx, 0) : box_m_sync<float>(ctx, 0);
    if (!rc) ctx->m_box_stale = false;
    return rc;
}

// z chunk of the fused kernel: as many chunks as fill one resident wave of
// blocks (each block marches its whole chunk, so a second wave would double
// the time).
template <typename T> static int plan_fused(mmx_ctx *ctx)
{
    int dev = 0, nsm = 0, per = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fused<T, kFBX, kFBY, 2, true, true>, kFBX * kFBY, 0));
    per = std::max(per, 1);
    const int *n = ctx->desc.n;
    long long tiles = (long long)((n[0] + 1 + kFBX - 2) / (kFBX - 1)) * ((n[1] + 1 + kFBY - 2) / (kFBY - 1));
    // as many z chunks as fit in one resident wave
    long long nch = std::max(1LL, ((long long)per * nsm) / tiles);
    int chunk = (int)std::max(2LL, (n[2] + nch - 1) / nch);
    chunk = std::min(chunk, n[2]);
    ctx->fused_chunk = chunk;
    ctx->fused_grid_z = (n[2] + chunk - 1) / chunk;
    return MMX_OK;
}

template <typename T> static void swap_buffers(mmx_ctx *ctx)
{
    for (int a = 0; a < 3; a++) {
        std::swap(ctx->E[a], ctx->Ealt[a]);
        std::swap(ctx->H[a], ctx->Halt[a]);
    }
    for (int a = 0; a < 2; a++) std::swap(ctx->Ezp[a], ctx->Ezpalt[a]);
}

template <typename T, int NH, bool PMLK, bool GEN>
static void launch_fused_v(mmx_ctx *ctx, dim3 G, dim3 B, const Fields<T> &f, Ptr3<T> Eo, Ptr3<T> Ho, Ptr3<T> En,
                           Ptr3<T> Hn, Ptr3<T> Zo, Ptr3<T> Zn, int nsrc)
{
    k_fused<T, kFBX, kFBY, NH, PMLK, GEN><<<G, B, 0, ctx->stream>>>(
        ctx->g, f, Eo, Ho, En, Hn, Zo, Zn, (const Src<T> *)ctx->dsrc, nsrc, ctx->fused_chunk, ctx->lo[0],
        ctx->lo[1], ctx->lo[2], ctx->hi[0], ctx->hi[1], ctx->hi[2]);
}

// Pick the compile-time variant of the fused kernel.
template <typename T>
static void launch_fused(mmx_ctx *ctx, dim3 G, dim3 B, const Fields<T> &f, Ptr3<T> Eo, Ptr3<T> Ho, Ptr3<T> En,
                         Ptr3<T> Hn, Ptr3<T> Zo, Ptr3<T> Zn, int nsrc, int nhalf)
{
    const bool pml = ctx->g.npml > 0, gen = ctx->any_sigma || ctx->any_mu;
#define MMX_FUSED_CASE(NHV, PV, GV)                                                                  \
    if (nhalf == NHV && pml == PV && gen == GV) {                                                    \
        launch_fused_v<T, NHV, PV, GV>(ctx, G, B, f, Eo, Ho, En, Hn, Zo, Zn, nsrc);                  \
        return;                                                                                      \
    }
    MMX_FUSED_CASE(2, true, false) MMX_FUSED_CASE(2, false, false) MMX_FUSED_CASE(2, true, true)
    MMX_FUSED_CASE(2, false, true) MMX_FUSED_CASE(1, true, false) MMX_FUSED_CASE(1, false, false)
    MMX_FUSED_CASE(1, true, true) MMX_FUSED_CASE(1, false, true)
#undef MMX_FUSED_CASE
}

// ------------------------------------------- vectorised fused kernel (PEC x, y)

template <typename T, typename S, bool GEN> constexpr size_t vec_smem_bytes()
{
    constexpr int BY = VecRows<T>::value, ST = VecStages<T, GEN>::value;
    constexpr size_t b = VecLayout<T, S, BY, GEN, ST>::bytes;
    static_assert(b <= 227 * 1024, "vectorised kernel shared memory above the per-CTA limit");
    return b;
}

// The vectorised kernel covers grids with PEC x and y walls whose magnetic
// box stays clear of the PML layers (it writes box faces for the box kernel
// to overwrite, which the in-place PML split parts would not survive).
static bool vec_usable(const mmx_ctx *ctx)
{
    if (ctx->g.per[0] || ctx->g.per[1]) return false;
    if (ctx->magnetic && ctx->g.npml > 0 &&
        (ctx->lo[2] < ctx->g.npml + 1 || ctx->hi[2] > ctx->desc.n[2] - ctx->g.npml - 1))
        return false;
    return true;
}

// Opt every variant in to its dynamic shared memory (above the 48 KB default).
template <typename T, typename S, int NH, bool PMLK, bool GEN> static cudaError_t set_vec_smem_v()
{
    constexpr int BY = VecRows<T>::value, ST = VecStages<T, GEN>::value;
    return cudaFuncSetAttribute(k_fused_vec<T, S, BY, ST, NH, PMLK, GEN>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem_bytes<T, S, GEN>());
}

template <typename T, typename S> static cudaError_t set_vec_smem()
{
    cudaError_t e = cudaSuccess;
    cudaError_t r[8] = {set_vec_smem_v<T, S, 1, false, false>(), set_vec_smem_v<T, S, 1, false, true>(),
                        set_vec_smem_v<T, S, 1, true, false>(),  set_vec_smem_v<T, S, 1, true, true>(),
                        set_vec_smem_v<T, S, 2, false, false>(), set_vec_smem_v<T, S, 2, false, true>(),
                        set_vec_smem_v<T, S, 2, true, false>(),  set_vec_smem_v<T, S, 2, true, true>()};
    for (cudaError_t x : r)
        if (x != cudaSuccess) e = x;
    return e;
}

#ifndef MMX_VEC_TMA
#define MMX_VEC_TMA 1
#endif

template <typename T, typename S, int NH, bool PMLK> static cudaError_t set_vec_tma_smem_v()
{
    constexpr int BY = VecRows<T>::value, ST = VecStages<T, false>::value;
    constexpr size_t b = VecLayout<T, S, BY, false, ST, true>::bytes;
    static_assert(b <= 227 * 1024, "TMA variant shared memory above the per-CTA limit");
    return cudaFuncSetAttribute(k_fused_vec_tma<T, S, BY, ST, NH, PMLK, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
}

// Tensor maps for the TMA variant (FP32 storage, no sigma or mu_r): the
// padded arrays as (X, Y, nz+1) float tensors, boxes of one plane of W
// columns by BY+2 rows (H, eps_r) or BY+1 rows (E).  Returns false (and the
// vectorised kernel keeps its cp.async staging) if the driver entry point
// or an encoding is unavailable.
static bool encode_vec_maps(mmx_ctx *ctx)
{
    using Enc = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                             const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return false;
    Enc enc = (Enc)fn;
    constexpr int BY = VecRows<float>::value, W = 32 * Lanes<float>::V;
    const cuuint64_t dim[3] = {(cuuint64_t)ctx->g.X, (cuuint64_t)ctx->g.Y, (cuuint64_t)ctx->desc.n[2] + 1};
    const cuuint64_t str[2] = {(cuuint64_t)ctx->g.X * 4, (cuuint64_t)ctx->g.X * ctx->g.Y * 4};
    const cuuint32_t boxh[3] = {(cuuint32_t)W, (cuuint32_t)(BY + 2), 1}, boxe[3] = {(cuuint32_t)W, (cuuint32_t)(BY + 1), 1};
    const cuuint32_t es[3] = {1, 1, 1};
    auto one = [&](CUtensorMap *m, void *p, const cuuint32_t *box) {
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, p, dim, str, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    for (int p = 0; p < 2; p++) {
        void *const *Eb = p == 0 ? ctx->E : ctx->Ealt, *const *Hb = p == 0 ? ctx->H : ctx->Halt;
        VecMaps &m = ctx->vmaps[p];
        bool ok = true;
        for (int a = 0; a < 3; a++) {
            ok = ok && one(&m.h[a], Hb[a], boxh);
            ok = ok && one(&m.e[a], Eb[a], boxe);
        }
        ok = ok && one(&m.eps, ctx->epsc, boxh);
        if (!ok) return false;
        ctx->vmap_key[p] = Hb[0];
    }
    return true;
}

// Extra cost of a fused-pass plane inside the z-PML (split-field loads,
// stores and updates) and of a plane holding a plane source, relative to an
// interior plane.  On the 128x128x512 waveguide (FP32) a step took 146.1 us
// with equal chunks and 134.5 us with these weights; 0.5-3 for the PML and
// 0-5 for the source bracket them (flat within 0.3 us from 0.8 to 1.2).
// With the PML update of a plane chosen at compile time (a cheaper PML
// plane), 0.5 and 0.75 measured 91.8 and 88.1 us per launch against 85.8.
constexpr double kZWeightPml = 1.0, kZWeightSrc = 1.0;

// Chunk bounds of the fused pass along z for at most nch chunks (the count
// that fills one resident wave): the max over chunks of the summed plane
// weights is minimised (binary search on the bound, greedy fill), with a
// plane weighing 1, plus kZWeightPml inside the z-PML and kZWeightSrc where
// a plane source sits.  Every chunk keeps at least 2 planes.  Returns the
// chunk count.
static int plan_zchunks(mmx_ctx *ctx, int nch)
{
    const int nz = ctx->desc.n[2], np = ctx->g.npml;
    nch = std::max(1, std::min({nch, kMaxZChunks, nz / 2}));
    std::vector<double> w(nz, 1.0);
    for (int k = 0; k < nz; k++) {
        if (np > 0 && (k < np || k >= nz - np)) w[k] += kZWeightPml;
    }
    for (const mmx_source_desc &q : ctx->src)
        if (q.kind == 1) w[std::min(q.k, nz - 1)] += kZWeightSrc;
    // chunks a bound B needs, each closed once adding a plane would pass B
    auto fill = [&](double B, int *b) {
        int c = 0, k0 = 0;
        double acc = 0.0;
        for (int k = 0; k < nz; k++) {
            if (k - k0 >= 2 && acc + w[k] > B) {
                if (b) b[c] = k0;
                c++;
                k0 = k;
                acc = 0.0;
            }
            acc += w[k];
        }
        if (b) {
            b[c] = k0;
            b[c + 1] = nz;
        }
        return c + 1;
    };
    double lo = 0.0, hi = 0.0;
    for (double x : w) hi += x;
    for (int it = 0; it < 60; it++) {
        const double mid = 0.5 * (lo + hi);
        if (fill(mid, nullptr) <= nch) hi = mid; else lo = mid;
    }
    const int c = fill(hi, ctx->vec_z.b);
    // a trailing chunk of fewer than 2 planes joins the one before it
    if (c > 1 && ctx->vec_z.b[c] - ctx->vec_z.b[c - 1] < 2) {
        ctx->vec_z.b[c - 1] = nz;
        return c - 1;
    }
    return c;
}

template <typename T, typename S> static int plan_vec(mmx_ctx *ctx)
{
    constexpr int W = 32 * Lanes<T>::V;
    int dev = 0, nsm = 0, per = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    {
        cudaError_t e = set_vec_smem<T, S>();
        CK(e);
    }
    constexpr int BY = VecRows<T>::value, ST = VecStages<T, false>::value;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fused_vec<T, S, BY, ST, 2, true, false>,
                                                     32 * (BY + 1), vec_smem_bytes<T, S, false>()));
    per = std::max(per, 1);
    const int *n = ctx->desc.n;
    const int xs = W - Lanes<T>::V;
    const int ntx = n[0] <= W ? 1 : 1 + (n[0] - W + xs - 1) / xs;
    const int nty = (n[1] + BY - 1) / BY;
    long long nch = std::max(1LL, ((long long)per * nsm) / ((long long)ntx * nty));
    int chunk = (int)std::max(2LL, (n[2] + nch - 1) / nch);
    chunk = std::min(chunk, n[2]);
    ctx->vec_chunk = chunk;
    ctx->vec_xstride = xs;
    ctx->vec_grid = dim3(ntx, nty, plan_zchunks(ctx, (n[2] + chunk - 1) / chunk));
    ctx->vec_tma = 0;
    ctx->tma_fallback = 0;
    if constexpr (std::is_same<T, float>::value && std::is_same<S, float>::value) {
        const bool applies = MMX_VEC_TMA && ctx->bulk_staging && !(ctx->any_sigma || ctx->any_mu) && ctx->epsc;
        if (applies && encode_vec_maps(ctx)) {
            cudaError_t r[4] = {set_vec_tma_smem_v<T, S, 1, false>(), set_vec_tma_smem_v<T, S, 1, true>(),
                                set_vec_tma_smem_v<T, S, 2, false>(), set_vec_tma_smem_v<T, S, 2, true>()};
            bool ok = true;
            for (cudaError_t x : r) ok = ok && x == cudaSuccess;
            int pt = 0;
            if (ok && cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                          &pt, k_fused_vec_tma<T, S, BY, ST, 2, true, false>, 32 * (BY + 1),
                          VecLayout<T, S, BY, false, ST, true>::bytes) == cudaSuccess &&
                pt >= per)
                ctx->vec_tma = 1;
            cudaGetLastError();
        }
        // recorded, so that the caller (mmx_get_info) sees which staging runs
        if (applies && ctx->vec_tma != 1) ctx->tma_fallback = 1;
    }
    return MMX_OK;
}

template <typename T> static int zero_walls(mmx_ctx *ctx)   // T: the stored type
{
    WallList<T> L;
    L.n = 0;
    for (int a = 0; a < 3; a++) {
        L.p[L.n++] = (T *)ctx->E[a];
        L.p[L.n++] = (T *)ctx->Ealt[a];
        L.p[L.n++] = (T *)ctx->H[a];
        L.p[L.n++] = (T *)ctx->Halt[a];
    }
    for (int a = 0; a < 2; a++) {
        if (ctx->Ezp[a]) L.p[L.n++] = (T *)ctx->Ezp[a];
        if (ctx->Ezpalt[a]) L.p[L.n++] = (T *)ctx->Ezpalt[a];
    }
    dim3 G((ctx->g.X + ctx->g.Y + 255) / 256, ctx->desc.n[2] + 1);
    prof_begin(ctx, KK_ZERO_WALLS);
    k_zero_walls<T><<<G, 256, 0, ctx->stream>>>(ctx->g, L);
    if (ctx->Hzp[0]) {
        WallList<T> P;
        P.n = 0;
        for (int a = 0; a < 2; a++) P.p[P.n++] = (T *)ctx->Hzp[a];
        k_zero_walls<T><<<G, 256, 0, ctx->stream>>>(ctx->g, P);
    }
    prof_end(ctx);
    CK(cudaGetLastError());
    return MMX_OK;
}

template <typename T, typename S, int NH, bool PMLK, bool GEN>
static void launch_vec_v(mmx_ctx *ctx, const Fields<T, S> &f, const FusedIO<S> &io, int nsrc)
{
    constexpr int BY = VecRows<T>::value, ST = VecStages<T, GEN>::value;
    if constexpr (std::is_same<T, float>::value && std::is_same<S, float>::value && !GEN) {
        if (ctx->vec_tma == 1) {
            // the map set of the buffers this step reads
            const int p = (void *)io.Ho[0] == ctx->vmap_key[0] ? 0 : 1;
            k_fused_vec_tma<T, S, BY, ST, NH, PMLK, GEN>
                <<<ctx->vec_grid, dim3(32, BY + 1), VecLayout<T, S, BY, GEN, ST, true>::bytes, ctx->stream>>>(
                    ctx->g, f, io, ctx->vmaps[p], (const Src<T> *)ctx->dsrc, nsrc, ctx->vec_z, ctx->vec_xstride);
            return;
        }
    }
    k_fused_vec<T, S, BY, ST, NH, PMLK, GEN><<<ctx->vec_grid, dim3(32, BY + 1), vec_smem_bytes<T, S, GEN>(),
                                               ctx->stream>>>(
        ctx->g, f, io, (const Src<T> *)ctx->dsrc, nsrc, ctx->vec_z, ctx->vec_xstride);
}

template <typename T, typename S>
static void launch_vec(mmx_ctx *ctx, const Fields<T, S> &f, const FusedIO<S> &io, int nsrc, int nhalf)
{
    const bool pml = ctx->g.npml > 0, gen = ctx->any_sigma || ctx->any_mu;
#define MMX_VEC_CASE(NHV, PV, GV)                                                                    \
    if (nhalf == NHV && pml == PV && gen == GV) {                                                    \
        launch_vec_v<T, S, NHV, PV, GV>(ctx, f, io, nsrc);                                           \
        return;                                                                                      \
    }
    MMX_VEC_CASE(2, true, false) MMX_VEC_CASE(2, false, false) MMX_VEC_CASE(2, true, true)
    MMX_VEC_CASE(2, false, true) MMX_VEC_CASE(1, true, false) MMX_VEC_CASE(1, false, false)
    MMX_VEC_CASE(1, true, true) MMX_VEC_CASE(1, false, true)
#undef MMX_VEC_CASE
}

template <typename T, typename S = T> static int step_fused(mmx_ctx *ctx, int nsteps)
{
    constexpr bool same = std::is_same<T, S>::value;
    const bool vec = vec_usable(ctx);
    if (!same && !vec) return fail(ctx, MMX_ERR_INVALID, "FP16 storage needs PEC x and y walls");
    if (vec) {
        if (!ctx->vec_chunk) {
            int rc = plan_vec<T, S>(ctx);
            if (rc) return rc;
        }
    }
    if constexpr (same) {
        if (!ctx->fused_chunk) {
            int rc = plan_fused<T>(ctx);
            if (rc) return rc;
        }
    }
    Box<T> b = make_box<T>(ctx);
    int nsrc = (int)ctx->src.size();
    const T *amp0 = (const T *)ctx->damp;
    // Step 1 of the first step in place: H^n -> H^(n+1/2)
    {
        Fields<T, S> f = make_fields<T, S>(ctx);
        int rc = half_step<T, S>(ctx, f, b, (ctx->steps + 0.5) * ctx->desc.dt, vec && ctx->h_half_vec);
        if (rc) return rc;
    }
    // Wall values set through mmx_set_field have been used by that half step
    // (as the per-update path uses them); from here on they are zero, which
    // the vectorised kernel relies on for the x = nx column and y = ny row.
    if (vec && ctx->walls_dirty) {
        int rc = zero_walls<S>(ctx);
        if (rc) return rc;
        ctx->walls_dirty = false;
    }
    const int *n = ctx->desc.n;
    dim3 B(kFBX, kFBY, 1);
    dim3 G((n[0] + 1 + kFBX - 2) / (kFBX - 1), (n[1] + 1 + kFBY - 2) / (kFBY - 1), ctx->fused_grid_z);
    for (int s = 0; s < nsteps; s++) {
        if (s % kAmpChunk == 0) {
            int rc = upload_amplitudes<T>(ctx, ctx->steps, std::min(kAmpChunk, nsteps - s));
            if (rc) return rc;
        }
        const int nhalf = s == nsteps - 1 ? 1 : 2;
        Fields<T, S> f = make_fields<T, S>(ctx);
        f.src_amp = amp0 + (size_t)(s % kAmpChunk) * nsrc;
        Ptr3<S> Eo = {{(S *)ctx->E[0], (S *)ctx->E[1], (S *)ctx->E[2]}};
        Ptr3<S> Ho = {{(S *)ctx->H[0], (S *)ctx->H[1], (S *)ctx->H[2]}};
        Ptr3<S> En = {{(S *)ctx->Ealt[0], (S *)ctx->Ealt[1], (S *)ctx->Ealt[2]}};
        Ptr3<S> Hn = {{(S *)ctx->Halt[0], (S *)ctx->Halt[1], (S *)ctx->Halt[2]}};
        Ptr3<S> Zo = {{(S *)ctx->Ezp[0], (S *)ctx->Ezp[1], nullptr}};
        Ptr3<S> Zn = {{(S *)ctx->Ezpalt[0], (S *)ctx->Ezpalt[1], nullptr}};
        // the same test launch_vec_v applies
        const bool tma = vec && ctx->vec_tma == 1 && std::is_same<T, float>::value &&
                         std::is_same<S, float>::value && !(ctx->any_sigma || ctx->any_mu);
        ctx->last_fused = vec ? (tma ? 3 : 2) : 1;
        prof_begin(ctx, vec ? (tma ? KK_FUSED_VEC_TMA : KK_FUSED_VEC) : KK_FUSED);
        if (vec) {
            FusedIO<S> io;
            for (int a = 0; a < 3; a++) {
                io.Eo[a] = Eo.p[a];
                io.Ho[a] = Ho.p[a];
                io.En[a] = En.p[a];
                io.Hn[a] = Hn.p[a];
            }
            for (int a = 0; a < 2; a++) {
                io.Zo[a] = Zo.p[a];
                io.Zn[a] = Zn.p[a];
            }
            launch_vec<T, S>(ctx, f, io, nsrc, nhalf);
        } else {
            if constexpr (same) launch_fused<T>(ctx, G, B, f, Eo, Ho, En, Hn, Zo, Zn, nsrc, nhalf);
        }
        prof_end(ctx);
        CK(cudaGetLastError());
        if (ctx->magnetic) {
            Fields<T, S> fb = f;
            for (int a = 0; a < 3; a++) fb.E[a] = En.p[a];   // E^(n+1); fb.H = H^(n+1/2)
            int rc = launch_box<T, S>(ctx, fb, b, Hn, nhalf);
            if (rc) return rc;
        }
        if (!ctx->flux_k.empty()) {
            // E^(n+1) with H^(n+1) = mean of H^(n+1/2) and H^(n+3/2), or
            // H^(n+1) itself after the single half step of a call's last step
            int rc = record_flux<T, S>(ctx, En, nhalf == 2 ? Ho : Hn, Hn);
            if (rc) return rc;
        }
        swap_buffers<T>(ctx);
        ctx->steps++;
        int rc = record_probes<T, S>(ctx);
        if (rc) return rc;
    }
    return MMX_OK;
}

// ------------------------------------------------------------ field copy

// FP16-stored E, H and PML split parts (ids 0-5, 15-18) of an MMX_FP16
// context; value = stored * scale.
static int copy_field_half(mmx_ctx *ctx, int id, double *host, long long N, const int e[3], int dir)
{
    __half *dev = id < 3 ? (__half *)ctx->E[id] : id < 6 ? (__half *)ctx->H[id - 3]
                : id < 17 ? (__half *)ctx->Ezp[id - 15] : (__half *)ctx->Hzp[id - 17];
    const float scale = (float)(id < 3 || id == 15 || id == 16 ? ctx->sE : ctx->sH);
    int blocks = (int)((N + 255) / 256);
    if (!dev) {
        if (dir == 0) {
            memset(host, 0, (size_t)N * sizeof(double));
            return MMX_OK;
        }
        return fail(ctx, MMX_ERR_INVALID, "field %d exists only with a z-PML", id);
    }
    if (dir == 1)
        CK(cudaMemcpyAsync(ctx->stage, host, (size_t)N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    k_copy_field_h<<<blocks, 256, 0, ctx->stream>>>(ctx->g, dev, scale, e[0], e[1], e[2], ctx->stage, dir);
    CK(cudaGetLastError());
    if (dir == 0)
        CK(cudaMemcpyAsync(host, ctx->stage, (size_t)N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MMX_OK;
}

template <typename T> static int copy_field_t(mmx_ctx *ctx, int id, double *host, long long n, int dir)
{
    int e[3];
    field_ext(ctx, id, e);
    long long N = (long long)e[0] * e[1] * e[2];
    int rc = ensure_stage(ctx, (size_t)N);
    if (rc) return rc;
    if (is_fp16(ctx) && (id < 6 || id >= 15)) return copy_field_half(ctx, id, host, N, e, dir);
    T *dev = nullptr;
    int boxed = 0;
    if (id < 3) dev = (T *)ctx->E[id];
    else if (id < 6) dev = (T *)ctx->H[id - 3];
    else if (id < 15) {
        boxed = 1;
        dev = ctx->magnetic ? (T *)ctx->bM[id - 6] : nullptr;
        if (dev) {
            rc = ensure_box_m(ctx);
            if (rc) return rc;
            if (dir == 1) ctx->m_rec_stale = true;   // the box arrays are written
        }
    } else if (id < 17) dev = (T *)ctx->Ezp[id - 15];
    else dev = (T *)ctx->Hzp[id - 17];
    Box<T> b = make_box<T>(ctx);
    int blocks = (int)((N + 255) / 256);
    if (dir == 0) {
        if (!dev) {
            memset(host, 0, (size_t)N * sizeof(double));
            return MMX_OK;
        }
        k_copy_field<T><<<blocks, 256, 0, ctx->stream>>>(ctx->g, dev, b, boxed, e[0], e[1], e[2], ctx->stage, 0);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(host, ctx->stage, (size_t)N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return MMX_OK;
    }
    if (!dev) {
        if (id >= 15) return fail(ctx, MMX_ERR_INVALID, "field %d exists only with a z-PML", id);
        for (long long q = 0; q < N; q++)
            if (host[q] != 0.0) return fail(ctx, MMX_ERR_INVALID, "M can only be set on magnetic faces");
        return MMX_OK;
    }
    if (boxed) {
        // M lives on the magnetic box only (values elsewhere are ignored):
        // move just the box region, [lo, min(lo + box, e)) per axis
        int ce[3];
        const int bd[3] = {ctx->bx, ctx->by, ctx->bz};
        for (int a = 0; a < 3; a++) ce[a] = std::min(ctx->lo[a] + bd[a], e[a]) - ctx->lo[a];
        if (ce[0] <= 0 || ce[1] <= 0 || ce[2] <= 0) return MMX_OK;
        cudaMemcpy3DParms p = {};
        p.srcPtr = make_cudaPitchedPtr(host, (size_t)e[0] * sizeof(double), (size_t)e[0], (size_t)e[1]);
        p.srcPos = make_cudaPos((size_t)ctx->lo[0] * sizeof(double), (size_t)ctx->lo[1], (size_t)ctx->lo[2]);
        p.dstPtr = make_cudaPitchedPtr(ctx->stage, (size_t)ce[0] * sizeof(double), (size_t)ce[0], (size_t)ce[1]);
        p.extent = make_cudaExtent((size_t)ce[0] * sizeof(double), (size_t)ce[1], (size_t)ce[2]);
        p.kind = cudaMemcpyHostToDevice;
        CK(cudaMemcpy3DAsync(&p, ctx->stream));
        const long long nbox = (long long)ce[0] * ce[1] * ce[2];
        k_box_region_in<T><<<(int)((nbox + 255) / 256), 256, 0, ctx->stream>>>(b, ce[0], ce[1], ce[2], ctx->stage, dev);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(ctx->stream));
        return MMX_OK;
    }
    CK(cudaMemcpyAsync(ctx->stage, host, (size_t)N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    k_copy_field<T><<<blocks, 256, 0, ctx->stream>>>(ctx->g, dev, b, boxed, e[0], e[1], e[2], ctx->stage, 1);
    CK(cudaGetLastError());
    if (!boxed) {
        for (int a = 0; a < 3; a++) {
            if (!ctx->g.per[a] || e[a] != ctx->desc.n[a] + 1) continue;
            int bb = (a + 1) % 3, cc = (a + 2) % 3;
            long long P = (long long)e[bb] * e[cc];
            k_sync_periodic<T><<<(int)((P + 255) / 256), 256, 0, ctx->stream>>>(ctx->g, dev, e[0], e[1], e[2], a);
            CK(cudaGetLastError());
        }
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return MMX_OK;
}

static int read_status(mmx_ctx *ctx)
{
    int w = 0;
    CK(cudaMemcpyAsync(&w, ctx->errw, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (w) {
        int z = 0;
        CK(cudaMemcpyAsync(ctx->errw, &z, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (w & kErrTimeout) {
        // launches after the timeout returned at entry without clearing the
        // residual and decision rows of the next launch's parity: clear all
        CK(cudaMemsetAsync(ctx->bar, 0, kBarWords * sizeof(unsigned long long), ctx->stream));
        CK(cudaMemsetAsync(ctx->res, 0, 2 * kVoteRows * (kMaxIter + 1) * sizeof(unsigned long long), ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return fail(ctx, MMX_ERR_TIMEOUT, "a device-side wait gave up");
    }
    if (w & kErrNonFinite) return fail(ctx, MMX_ERR_NONFINITE, "a field became non-finite");
    if (w & kErrBadInput) return fail(ctx, MMX_ERR_INVALID, "invalid input detected on the device");
    if (w & kErrNotConverged)
        return fail(ctx, MMX_ERR_NOT_CONVERGED, "an H/M half step reached max_iter=%d", ctx->desc.max_iter);
    return MMX_OK;
}

// ================================================================= C ABI

static int ensure_monitor(mmx_ctx *ctx)
{
    if (ctx->mon_partial) return MMX_OK;
    int rc = dalloc(ctx, (void **)&ctx->mon_partial, kMonitorBlocks * sizeof(double2));
    if (!rc) rc = dalloc(ctx, (void **)&ctx->flux_acc, 4 * kMaxFluxPlanes * sizeof(double));
    return rc;
}

template <typename T, typename S = T> static int energy_t(mmx_ctx *ctx, double *out)
{
    int rc = ensure_monitor(ctx);
    if (rc) return rc;
    Fields<T, S> f = make_fields<T, S>(ctx);
    k_energy<T, S><<<kMonitorBlocks, kMonitorThreads, 0, ctx->stream>>>(ctx->g, f, ctx->cell[0], ctx->cell[2],
                                                                     ctx->cell[3], ctx->mon_partial);
    CK(cudaGetLastError());
    std::vector<double2> part(kMonitorBlocks);
    CK(cudaMemcpyAsync(part.data(), ctx->mon_partial, kMonitorBlocks * sizeof(double2), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    double s = 0.0, c = 0.0;
    for (const double2 &v : part) {
        const double t = s + v.x;
        c += std::fabs(s) >= std::fabs(v.x) ? (s - t) + v.x : (v.x - t) + s;
        s = t;
        c += v.y;
    }
    *out = s + c;
    return MMX_OK;
}

// ============================================================ adjoint
//
// Gradient of the time-integrated Poynting flux through a z node plane with
// respect to eps_r of every cell, by the discrete adjoint of the per-update
// path (mmx_adjoint.cuh), with the forward states checkpointed every C steps
// and each segment recomputed once in the reverse sweep.

// The state a step starts from: E, H, the PML split parts and, on grids
// with magnetic material, M (the nine box arrays).
constexpr int kSnapArrays = 19;
struct AdjSnap {
    void *a[kSnapArrays] = {};
};

template <typename T> static void snap_ptrs(mmx_ctx *c, void *p[kSnapArrays], size_t bytes[kSnapArrays])
{
    for (int q = 0; q < kSnapArrays; q++) {
        p[q] = nullptr;
        bytes[q] = c->npad * sizeof(T);
    }
    for (int a = 0; a < 3; a++) {
        p[a] = c->E[a];
        p[3 + a] = c->H[a];
    }
    for (int a = 0; a < 2; a++) {
        p[6 + a] = c->Ezp[a];
        p[8 + a] = c->Hzp[a];
    }
    if (c->magnetic)
        for (int q = 0; q < 9; q++) {
            p[10 + q] = c->bM[q];
            bytes[10 + q] = (size_t)c->nb * sizeof(T);
        }
}

// Copy the live state into s (save) or back; M is taken from (and left in)
// the box arrays.
template <typename T> static int snap_copy(mmx_ctx *ctx, AdjSnap &s, bool save)
{
    mmx_ctx *const c = ctx;
    void *live[kSnapArrays];
    size_t bytes[kSnapArrays];
    snap_ptrs<T>(c, live, bytes);
    for (int q = 0; q < kSnapArrays; q++) {
        if (!live[q]) continue;
        if (save)
            CK(cudaMemcpyAsync(s.a[q], live[q], bytes[q], cudaMemcpyDeviceToDevice, c->stream));
        else
            CK(cudaMemcpyAsync(live[q], s.a[q], bytes[q], cudaMemcpyDeviceToDevice, c->stream));
    }
    return MMX_OK;
}

template <typename T> static Ptr3<T> snap3(const AdjSnap &s, int base)
{
    Ptr3<T> p = {{(T *)s.a[base], (T *)s.a[base + 1], (T *)s.a[base + 2]}};
    return p;
}

template <typename T> static MPtr<T> snapM(const AdjSnap &s)
{
    MPtr<T> p;
    for (int q = 0; q < 9; q++) p.p[q] = (T *)s.a[10 + q];
    return p;
}

// Largest iteration count among the last `count` logged H/M half steps.
static int logged_iter_max(mmx_ctx *ctx, long long count)
{
    unsigned long long hs = 0;
    if (cudaMemcpy(&hs, ctx->halfsteps, sizeof hs, cudaMemcpyDeviceToHost) != cudaSuccess) return kMaxIter;
    const long long m = std::min<long long>(std::min<long long>((long long)hs, kIterLogCap), count);
    std::vector<int> v(kIterLogCap);
    if (cudaMemcpy(v.data(), ctx->iterlog, kIterLogCap * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return kMaxIter;
    int mx = 1;
    for (long long q = 0; q < m; q++) mx = std::max(mx, v[(hs - 1 - q) % kIterLogCap]);
    return mx;
}

// One magnetic half step's adjoint, before its k_adj_h: the fixed-point
// adjoint of the LLG solve from the state it started from (Hn, Mn) and the
// H it ended with (Hs).
template <typename T>
static int adj_mag_half(mmx_ctx *ctx, const Box<T> &b, Ptr3<T> Hn, MPtr<T> Mn, Ptr3<T> Hs, const AdjState<T> &a,
                        const AdjMag<T> &m)
{
    const int nblk = (int)((std::max<long long>(b.nb, 2LL * m.kmax) + 255) / 256);
    k_adjm_prep<T><<<nblk, 256, 0, ctx->stream>>>(ctx->g, b, Hn, Mn, Hs, a, m);
    for (int it = 0; it < m.kmax; it++) {
        k_adjm_heff<T><<<nblk, 256, 0, ctx->stream>>>(b, m, it);
        k_adjm_sweep<T><<<nblk, 256, 0, ctx->stream>>>(ctx->g, b, m, it);
    }
    k_adjm_heff<T><<<nblk, 256, 0, ctx->stream>>>(b, m, -1);
    k_adjm_close<T><<<nblk, 256, 0, ctx->stream>>>(ctx->g, b, Hn, Mn, a, m);
    CK(cudaGetLastError());
    return MMX_OK;
}

template <typename T>
static int flux_gradient_t(mmx_ctx *ctx, int kp, int nsteps, int every, double *loss, double *grad, double *grad_h0)
{
    std::vector<void *> mem;
    auto cleanup = [&]() {
        cudaStreamSynchronize(ctx->stream);
        for (void *p : mem) cudaFree(p);
    };
    auto alloc = [&](size_t bytes, void **p) {
        if (cudaMalloc(p, bytes) != cudaSuccess) return fail(ctx, MMX_ERR_OOM, "adjoint: out of device memory");
        mem.push_back(*p);
        if (cudaMemsetAsync(*p, 0, bytes, ctx->stream) != cudaSuccess) return fail(ctx, MMX_ERR_CUDA, "memset");
        return MMX_OK;
    };
    const size_t fb = ctx->npad * sizeof(T), db = ctx->npad * sizeof(double);
    const bool pml = ctx->g.npml > 0, mag = ctx->magnetic && ctx->nmag > 0;
    const int nseg = (nsteps + every - 1) / every;
    int rc = MMX_OK;
    auto snap_alloc = [&](AdjSnap &sn) {
        void *live[kSnapArrays];
        size_t bytes[kSnapArrays];
        snap_ptrs<T>(ctx, live, bytes);
        for (int q = 0; q < kSnapArrays && !rc; q++)
            if (live[q]) rc = alloc(bytes[q], &sn.a[q]);
    };
    std::vector<AdjSnap> ck(nseg + 1), seg(every);
    for (auto &sn : ck) snap_alloc(sn);
    for (auto &sn : seg) snap_alloc(sn);
    AdjSnap half;                     // the state after the first H/M half step
    snap_alloc(half);
    AdjState<T> a = {};
    for (int c = 0; c < 3 && !rc; c++) {
        rc = alloc(fb, (void **)&a.lE[c]);
        if (!rc) rc = alloc(fb, (void **)&a.lH[c]);
        if (!rc) rc = alloc(fb, (void **)&a.fR[c]);
        if (!rc) rc = alloc(fb, (void **)&a.fZ[c]);
        if (!rc) rc = alloc(fb, (void **)&a.eR[c]);
        if (!rc) rc = alloc(fb, (void **)&a.eZ[c]);
        if (!rc) rc = alloc(db, (void **)&a.gcb[c]);
        if (!rc) rc = alloc(db, (void **)&a.gca[c]);
    }
    for (int c = 0; c < 2 && !rc && pml; c++) {
        rc = alloc(fb, (void **)&a.lEz[c]);
        if (!rc) rc = alloc(fb, (void **)&a.lHz[c]);
    }
    AdjMag<T> am = {};
    if (mag && !rc) {
        const size_t bb = (size_t)ctx->nb * sizeof(T);
        T **sets[7] = {am.lM, am.gM, am.mu, am.A, am.B, am.lHe, am.lHn};
        for (int q = 0; q < 7 && !rc; q++)
            for (int c = 0; c < 9 && !rc; c++) rc = alloc(bb, (void **)&sets[q][c]);
        if (!rc) rc = alloc(2 * kMaxIter * sizeof(unsigned long long), (void **)&am.res);
        if (!rc) rc = alloc(sizeof(int), (void **)&am.nc);
        am.eps = sizeof(T) == 8 ? 1e-13 : 1e-6;
    }
    double *dh0 = nullptr;
    if (!rc) rc = alloc(3 * sizeof(double), (void **)&dh0);
    am.gh0 = dh0;
    if (rc) {
        cleanup();
        return rc;
    }
    const long long n0 = ctx->steps;
    // ---- forward: checkpoints every `every` steps, loss by the flux monitor
    std::vector<int> saved_flux = ctx->flux_k;
    ctx->flux_k.assign(1, kp);
    rc = ensure_monitor(ctx);
    if (!rc && cudaMemsetAsync(ctx->flux_acc, 0, 4 * sizeof(double), ctx->stream) != cudaSuccess)
        rc = fail(ctx, MMX_ERR_CUDA, "memset");
    if (!rc && cudaMemsetAsync(ctx->bar, 0, kBarWords * sizeof(unsigned long long), ctx->stream) != cudaSuccess)
        rc = fail(ctx, MMX_ERR_CUDA, "memset");
    if (!rc) rc = snap_copy<T>(ctx, ck[0], true);
    if (!rc) rc = box_m_sync<T>(ctx, 1);
    for (int s = 0; s < nseg && !rc; s++) {
        rc = step_plain<T>(ctx, std::min(every, nsteps - s * every));
        if (!rc) rc = box_m_sync<T>(ctx, 0);
        if (!rc) rc = snap_copy<T>(ctx, ck[s + 1], true);
    }
    double acc[4] = {0, 0, 0, 0};
    if (!rc) {
        CK(cudaMemcpyAsync(acc, ctx->flux_acc, sizeof acc, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    ctx->flux_k = saved_flux;
    if (!rc) rc = read_status(ctx);
    if (rc) {
        cleanup();
        return rc;
    }
    *loss = acc[0] + acc[1];
    // the fixed-point adjoint contracts like the forward iteration: allow it
    // the forward's largest sweep count plus a margin (it stops on its own)
    if (mag) am.kmax = std::min(ctx->desc.max_iter, logged_iter_max(ctx, 2LL * nsteps) + 8);
    // ---- reverse sweep
    dim3 B = node_block(), G = node_grid(ctx);
    const int npt = ctx->g.X * (ctx->desc.n[1] + 1);
    const T w = (T)(ctx->desc.dt * ctx->desc.d[0] * ctx->desc.d[1]);
    const int nsrc = (int)ctx->src.size();
    const Box<T> bx = make_box<T>(ctx);
    for (int s = nseg - 1; s >= 0 && !rc; s--) {
        const int len = std::min(every, nsteps - s * every);
        // recompute the segment, keeping the state before each step
        rc = snap_copy<T>(ctx, ck[s], false);
        if (!rc) rc = box_m_sync<T>(ctx, 1);
        ctx->steps = n0 + (long long)s * every;
        for (int m = 0; m < len && !rc; m++) {
            rc = box_m_sync<T>(ctx, 0);
            if (!rc) rc = snap_copy<T>(ctx, seg[m], true);
            if (!rc) rc = step_plain<T>(ctx, 1);
        }
        for (int m = len - 1; m >= 0 && !rc; m--) {
            const long long n = n0 + (long long)s * every + m;
            const AdjSnap &before = seg[m];
            const AdjSnap &after = m + 1 < len ? seg[m + 1] : ck[s + 1];
            Fields<T> f = make_fields<T>(ctx);
            // H^(n+1/2) (and M^(n+1/2)) recomputed from the state before
            const size_t bytes = ctx->npad * sizeof(T);
            for (int q = 3; q < 6; q++)
                CK(cudaMemcpyAsync(half.a[q], before.a[q], bytes, cudaMemcpyDeviceToDevice, ctx->stream));
            for (int q = 8; q < 10; q++)
                if (before.a[q]) CK(cudaMemcpyAsync(half.a[q], before.a[q], bytes, cudaMemcpyDeviceToDevice, ctx->stream));
            Fields<T> fh = f;
            for (int c = 0; c < 3; c++) {
                fh.E[c] = (T *)before.a[c];
                fh.H[c] = (T *)half.a[3 + c];
            }
            for (int c = 0; c < 2; c++) fh.Hzp[c] = (T *)half.a[8 + c];
            if (mag) {
                const size_t mb = (size_t)ctx->nb * sizeof(T);
                for (int q = 0; q < 9; q++)
                    CK(cudaMemcpyAsync(ctx->bM[q], before.a[10 + q], mb, cudaMemcpyDeviceToDevice, ctx->stream));
                rc = box_m_sync<T>(ctx, 1);
                if (!rc) rc = half_step<T, T>(ctx, fh, bx, (n + 0.5) * ctx->desc.dt);
                if (!rc) rc = box_m_sync<T>(ctx, 0);
                for (int q = 0; q < 9 && !rc; q++)
                    CK(cudaMemcpyAsync(half.a[10 + q], ctx->bM[q], mb, cudaMemcpyDeviceToDevice, ctx->stream));
                if (rc) break;
            } else {
                k_h_update<T><<<G, B, 0, ctx->stream>>>(ctx->g, fh, 0, 0, 0, 0, 0, 0);
            }
            // loss term of time n+1
            k_adj_flux<T><<<(npt + 255) / 256, 256, 0, ctx->stream>>>(ctx->g, snap3<T>(after, 0), snap3<T>(after, 3),
                                                                      kp, w, a);
            // second H/M half step (with E^(n+1)), from the half state to after
            if (mag) rc = adj_mag_half<T>(ctx, bx, snap3<T>(half, 3), snapM<T>(half), snap3<T>(after, 3), a, am);
            if (rc) break;
            k_adj_h<T><<<G, B, 0, ctx->stream>>>(ctx->g, f, a);
            if (mag) k_adjm_curl<T><<<(int)((ctx->nb + 255) / 256), 256, 0, ctx->stream>>>(ctx->g, bx, a, am);
            k_adj_curl_e<T><<<G, B, 0, ctx->stream>>>(ctx->g, a);
            // E update: needs H^(n+1/2)
            {
                rc = upload_amplitudes<T>(ctx, n, 1);
                if (rc) break;
                Fields<T> fe = f;
                fe.src_amp = (const T *)ctx->damp;
                Ptr3<T> Z0 = {{(T *)before.a[6], (T *)before.a[7], nullptr}};
                k_adj_e<T><<<G, B, 0, ctx->stream>>>(ctx->g, fe, snap3<T>(half, 3), snap3<T>(before, 0), Z0,
                                                     (const Src<T> *)ctx->dsrc, nsrc, a);
                k_adj_curl_h<T><<<G, B, 0, ctx->stream>>>(ctx->g, a);
            }
            // first H/M half step (with E^n), from before to the half state
            if (mag) rc = adj_mag_half<T>(ctx, bx, snap3<T>(before, 3), snapM<T>(before), snap3<T>(half, 3), a, am);
            if (rc) break;
            k_adj_h<T><<<G, B, 0, ctx->stream>>>(ctx->g, f, a);
            if (mag) k_adjm_curl<T><<<(int)((ctx->nb + 255) / 256), 256, 0, ctx->stream>>>(ctx->g, bx, a, am);
            k_adj_curl_e<T><<<G, B, 0, ctx->stream>>>(ctx->g, a);
            if (cudaGetLastError() != cudaSuccess) rc = fail(ctx, MMX_ERR_CUDA, "adjoint launch failed");
        }
    }
    // gradient per cell, and the context back at the end of the forward run
    if (!rc) {
        double *dgrad = nullptr;
        const long long ncell = (long long)ctx->desc.n[0] * ctx->desc.n[1] * ctx->desc.n[2];
        rc = alloc((size_t)ncell * sizeof(double), (void **)&dgrad);
        const double **gtab = nullptr;
        if (!rc) rc = alloc(6 * sizeof(double *), (void **)&gtab);
        if (!rc) {
            const double *h[6] = {a.gcb[0], a.gcb[1], a.gcb[2], a.gca[0], a.gca[1], a.gca[2]};
            CK(cudaMemcpyAsync((void *)gtab, h, sizeof h, cudaMemcpyHostToDevice, ctx->stream));
            k_adj_eps<<<(int)((ncell + 255) / 256), 256, 0, ctx->stream>>>(ctx->g, ctx->cell[0], ctx->cell[1], gtab,
                                                                           gtab + 3, dgrad);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(grad, dgrad, (size_t)ncell * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
            if (grad_h0) CK(cudaMemcpyAsync(grad_h0, dh0, 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        }
        if (!rc) rc = snap_copy<T>(ctx, ck[nseg], false);
        ctx->steps = n0 + nsteps;
    }
    int nc = 0;
    if (!rc && mag) {
        CK(cudaMemcpyAsync(&nc, am.nc, sizeof nc, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    cleanup();
    if (!rc && nc)
        rc = fail(ctx, MMX_ERR_NOT_CONVERGED, "adjoint: a fixed-point sweep of an H/M half step missed its tolerance");
    return rc ? rc : read_status(ctx);
}

// Failure-detection probe: two blocks meet at a grid barrier and block
// `absent` returns without arriving, so the other one waits out the bounded
// wait and latches kErrTimeout (nothing faults, nothing hangs).
__global__ void k_barrier_probe(unsigned long long *bar, int *err, int absent, int vote)
{
    if ((int)blockIdx.x == absent) return;
    if (vote)
        grid_vote(bar + 1, false, err);
    else
        grid_barrier(bar, err);
}

extern "C" {

int mmx_create(const mmx_grid_desc *desc, void *cuda_stream, mmx_ctx **out)
{
    if (!desc || !out) return MMX_ERR_INVALID;
    *out = nullptr;
    mmx_ctx *ctx = new (std::nothrow) mmx_ctx();
    if (!ctx) return MMX_ERR_OOM;
    ctx->desc = *desc;
    const mmx_grid_desc &d = *desc;
    int rc = MMX_OK;
    for (int a = 0; a < 3; a++) {
        if (d.n[a] < 1 || !(d.d[a] > 0)) rc = fail(ctx, MMX_ERR_INVALID, "n and d must be positive");
        if (d.bc[a] < 0 || d.bc[a] > 2) rc = fail(ctx, MMX_ERR_INVALID, "bad boundary type");
        if (d.bc[a] == MMX_BC_PML && a != 2) rc = fail(ctx, MMX_ERR_INVALID, "PML only on the z axis");
    }
    if (!(d.dt > 0)) rc = fail(ctx, MMX_ERR_INVALID, "dt must be positive");
    if (d.order != 1 && d.order != 2) rc = fail(ctx, MMX_ERR_INVALID, "order must be 1 or 2");
    if (!(d.tol > 0)) rc = fail(ctx, MMX_ERR_INVALID, "tol must be positive");
    if (d.max_iter < 1 || d.max_iter > kMaxIter) rc = fail(ctx, MMX_ERR_INVALID, "max_iter must be 1..64");
    if (d.prec != MMX_FP64 && d.prec != MMX_FP32 && d.prec != MMX_FP16)
        rc = fail(ctx, MMX_ERR_INVALID, "bad precision");
    if (d.bc[2] == MMX_BC_PML && (d.pml_cells < 1 || 2 * d.pml_cells >= d.n[2]))
        rc = fail(ctx, MMX_ERR_INVALID, "pml_cells must be in [1, nz/2)");
    long long X = ((long long)d.n[0] + 1 + 7) / 8 * 8;
    long long npad = X * (d.n[1] + 1LL) * (d.n[2] + 1LL);
    if (npad > (1LL << 40)) rc = fail(ctx, MMX_ERR_INVALID, "grid too large");
    if (rc) {
        // keep the message reachable through *out
        *out = ctx;
        return rc;
    }
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->esz = d.prec == MMX_FP64 ? 8 : 4;
    ctx->ssz = d.prec == MMX_FP64 ? 8 : d.prec == MMX_FP32 ? 4 : 2;
    if (d.prec == MMX_FP16) {
        ctx->sH = 64.0;
        ctx->sE = kMu0 * kC0 * ctx->sH;
    }
    Geo &g = ctx->g;
    for (int a = 0; a < 3; a++) {
        g.n[a] = d.n[a];
        g.per[a] = d.bc[a] == MMX_BC_PERIODIC;
        g.d[a] = d.d[a];
        g.inv_d[a] = 1.0 / d.d[a];
    }
    g.X = (int)X;
    g.Y = d.n[1] + 1;
    g.npml = d.bc[2] == MMX_BC_PML ? d.pml_cells : 0;
    g.dt = d.dt;
    ctx->npad = (size_t)npad;
    size_t fb = ctx->npad * ctx->esz, sb = ctx->npad * ctx->ssz;
    for (int a = 0; a < 3 && !rc; a++) {
        rc = dalloc(ctx, &ctx->E[a], sb);
        if (!rc) rc = dalloc(ctx, &ctx->H[a], sb);
        if (!rc) rc = dalloc(ctx, &ctx->Ealt[a], sb);
        if (!rc) rc = dalloc(ctx, &ctx->Halt[a], sb);
        if (!rc) rc = dalloc(ctx, &ctx->cb[a], fb);
        if (!rc && a == 0 && ctx->esz == 4) rc = dalloc(ctx, &ctx->epsc, fb);
    }
    if (!rc && g.npml > 0)
        for (int a = 0; a < 2 && !rc; a++) {
            rc = dalloc(ctx, &ctx->Ezp[a], sb);
            if (!rc) rc = dalloc(ctx, &ctx->Ezpalt[a], sb);
            if (!rc) rc = dalloc(ctx, &ctx->Hzp[a], sb);
        }
    if (!rc) rc = dalloc(ctx, (void **)&ctx->res, 2 * kVoteRows * (kMaxIter + 1) * sizeof(unsigned long long));
    if (!rc) rc = dalloc(ctx, (void **)&ctx->bar, kBarWords * sizeof(unsigned long long));
    if (!rc) rc = dalloc(ctx, (void **)&ctx->iterlog, kIterLogCap * sizeof(int));
    if (!rc) rc = dalloc(ctx, (void **)&ctx->halfsteps, sizeof(unsigned long long));
    if (!rc) rc = dalloc(ctx, (void **)&ctx->last_res, sizeof(double));
    if (!rc) rc = dalloc(ctx, (void **)&ctx->errw, sizeof(int));
    if (!rc) rc = dalloc(ctx, &ctx->dsrc, kMaxSources * sizeof(Src<double>));
    if (!rc) rc = dalloc(ctx, &ctx->damp, (size_t)kAmpChunk * kMaxSources * ctx->esz);
    if (!rc) {
        // TE10 profile sin(pi x / W) at x = i dx and (i + 1/2) dx, W = nx dx
        std::vector<double> p0(d.n[0] + 1), p1(d.n[0] + 1);
        double W = d.n[0] * d.d[0];
        for (int i = 0; i <= d.n[0]; i++) {
            double x0 = (double)i * d.d[0], x1 = (i + 0.5) * d.d[0];
            p0[i] = std::sin(kPi * x0 / W);
            p1[i] = std::sin(kPi * x1 / W);
        }
        rc = is_fp64(ctx) ? upload_table<double>(ctx, &ctx->dprof[0], p0) : upload_table<float>(ctx, &ctx->dprof[0], p0);
        if (!rc) rc = is_fp64(ctx) ? upload_table<double>(ctx, &ctx->dprof[1], p1) : upload_table<float>(ctx, &ctx->dprof[1], p1);
    }
    if (!rc) {
        std::vector<double> dE, dH;
        pml_tables(ctx, dE, dH);
        rc = is_fp64(ctx) ? upload_table<double>(ctx, &ctx->dampE, dE) : upload_table<float>(ctx, &ctx->dampE, dE);
        if (!rc) rc = is_fp64(ctx) ? upload_table<double>(ctx, &ctx->dampH, dH) : upload_table<float>(ctx, &ctx->dampH, dH);
    }
    if (!rc)
        rc = is_fp64(ctx) ? set_materials_t<double>(ctx)
             : is_fp16(ctx) ? set_materials_t<float, __half>(ctx) : set_materials_t<float>(ctx);
    if (rc) {
        *out = ctx;
        return rc;
    }
    *out = ctx;
    return MMX_OK;
}

void mmx_destroy(mmx_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->E[0]) cudaStreamSynchronize(ctx->stream);
    for (int a = 0; a < 3; a++) {
        cudaFree(ctx->E[a]); cudaFree(ctx->H[a]); cudaFree(ctx->ca[a]); cudaFree(ctx->cb[a]); cudaFree(ctx->fh[a]);
        cudaFree(ctx->Ealt[a]); cudaFree(ctx->Halt[a]);
    }
    for (int a = 0; a < 2; a++) { cudaFree(ctx->Ezp[a]); cudaFree(ctx->Hzp[a]); cudaFree(ctx->Ezpalt[a]); }
    for (int a = 0; a < 6; a++) cudaFree(ctx->cell[a]);
    free_box(ctx);
    cudaFree(ctx->dampE); cudaFree(ctx->dampH); cudaFree(ctx->epsc);
    cudaFree(ctx->probe_buf); cudaFree(ctx->dprobe);
    cudaFree(ctx->mon_partial); cudaFree(ctx->flux_acc);
    cudaFree(ctx->res); cudaFree(ctx->bar); cudaFree(ctx->iterlog); cudaFree(ctx->halfsteps);
    cudaFree(ctx->last_res); cudaFree(ctx->errw); cudaFree(ctx->dsrc); cudaFree(ctx->stage);
    cudaFree(ctx->damp); cudaFree(ctx->dprof[0]); cudaFree(ctx->dprof[1]);
    for (ProfRec &r : ctx->prof_recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
    delete ctx;
}

const char *mmx_last_error(const mmx_ctx *ctx)
{
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

int mmx_set_materials(mmx_ctx *ctx, const double *eps_r, const double *sigma, const double *mu_r,
                      const double *Ms, const double *alpha, const double *gamma_abs)
{
    if (!ctx || !ctx->E[0]) return MMX_ERR_INVALID;
    const int *n = ctx->desc.n;
    size_t nc = (size_t)n[0] * n[1] * n[2];
    const double *in[6] = {eps_r, sigma, mu_r, Ms, alpha, gamma_abs};
    for (size_t q = 0; q < nc; q++) {
        if (eps_r && !(eps_r[q] > 0)) return fail(ctx, MMX_ERR_INVALID, "eps_r must be > 0");
        if (mu_r && !(mu_r[q] > 0)) return fail(ctx, MMX_ERR_INVALID, "mu_r must be > 0");
        if (sigma && !(sigma[q] >= 0)) return fail(ctx, MMX_ERR_INVALID, "sigma must be >= 0");
        if (Ms && !(Ms[q] == 0 || (Ms[q] >= 1e-20 && Ms[q] <= 1e20)))
            return fail(ctx, MMX_ERR_INVALID, "Ms must be 0 or in [1e-20, 1e20] A/m");
        if (alpha && !(alpha[q] >= 0)) return fail(ctx, MMX_ERR_INVALID, "alpha must be >= 0");
        if (gamma_abs && !(gamma_abs[q] >= 0)) return fail(ctx, MMX_ERR_INVALID, "gamma must be >= 0");
    }
    // magnetic bounding box (cells with Ms > 0)
    int c0[3] = {n[0], n[1], n[2]}, c1[3] = {-1, -1, -1};
    if (Ms) {
        for (int k = 0; k < n[2]; k++)
            for (int j = 0; j < n[1]; j++)
                for (int i = 0; i < n[0]; i++)
                    if (Ms[(size_t)i + (size_t)n[0] * ((size_t)j + (size_t)n[1] * k)] > 0) {
                        int ix[3] = {i, j, k};
                        for (int a = 0; a < 3; a++) {
                            c0[a] = std::min(c0[a], ix[a]);
                            c1[a] = std::max(c1[a], ix[a]);
                        }
                    }
    }
    bool magnetic = c1[0] >= 0;
    if (magnetic && ctx->g.npml > 0 && (c0[2] < ctx->g.npml || c1[2] >= n[2] - ctx->g.npml))
        return fail(ctx, MMX_ERR_INVALID, "Ms must be 0 inside the PML layers");
    // upload cell arrays
    for (int a = 0; a < 6; a++) {
        cudaFree(ctx->cell[a]);
        ctx->cell[a] = nullptr;
        if (!in[a]) continue;
        CK(cudaMalloc((void **)&ctx->cell[a], nc * sizeof(double)));
        CK(cudaMemcpyAsync(ctx->cell[a], in[a], nc * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    }
    bool any_sigma = false, any_mu = false;
    for (size_t q = 0; q < nc; q++) {
        if (sigma && sigma[q] != 0.0) any_sigma = true;
        if (mu_r && mu_r[q] != 1.0) any_mu = true;
    }
    size_t fb = ctx->npad * ctx->esz;
    for (int a = 0; a < 3; a++) {
        if (any_sigma && !ctx->ca[a]) { int rc = dalloc(ctx, &ctx->ca[a], fb); if (rc) return rc; }
        if (!any_sigma && ctx->ca[a]) { dfree(ctx, ctx->ca[a]); ctx->ca[a] = nullptr; }
        if (any_mu && !ctx->fh[a]) { int rc = dalloc(ctx, &ctx->fh[a], fb); if (rc) return rc; }
        if (!any_mu && ctx->fh[a]) { dfree(ctx, ctx->fh[a]); ctx->fh[a] = nullptr; }
    }
    ctx->any_sigma = any_sigma;
    ctx->any_mu = any_mu;
    // (re)build the magnetic box
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->m_rec_stale = true;    // the rebuilt box arrays hold M = Ms zhat
    ctx->m_box_stale = false;
    free_box(ctx);
    if (magnetic) {
        for (int a = 0; a < 3; a++) {
            if (ctx->g.per[a] && (c0[a] == 0 || c1[a] == n[a] - 1)) {
                ctx->lo[a] = 0;
                ctx->hi[a] = n[a] + 1;
            } else {
                ctx->lo[a] = std::max(c0[a] - 1, 0);
                ctx->hi[a] = std::min(c1[a] + 2, n[a] + 1);
            }
        }
        ctx->bx = ctx->hi[0] - ctx->lo[0];
        ctx->by = ctx->hi[1] - ctx->lo[1];
        ctx->bz = ctx->hi[2] - ctx->lo[2];
        ctx->nb = (long long)ctx->bx * ctx->by * ctx->bz;
        int rc = MMX_OK;
        for (int q = 0; q < 9 && !rc; q++) rc = box_alloc(ctx, &ctx->bM[q]);
        for (int a = 0; a < 3 && !rc; a++) {
            rc = box_alloc(ctx, &ctx->bHit[0][a]);
            if (!rc) rc = box_alloc(ctx, &ctx->bHit[1][a]);
            if (!rc) rc = box_alloc(ctx, &ctx->bHit2[0][a]);
            if (!rc) rc = box_alloc(ctx, &ctx->bHit2[1][a]);
            if (!rc) rc = box_alloc(ctx, &ctx->bms[a]);
            if (!rc) rc = box_alloc(ctx, &ctx->bk1[a]);
            if (!rc) rc = box_alloc(ctx, &ctx->bk2[a]);
        }
        if (!rc && (ctx->nb >= (1LL << 30) || (long long)ctx->g.X * ctx->g.Y * (ctx->desc.n[2] + 1LL) >= (1LL << 32)))
            rc = fail(ctx, MMX_ERR_INVALID, "magnetic box or grid too large for 32-bit box indexing");
        if (!rc) rc = build_box_lists(ctx, Ms);
        {
            // per magnetic face records: 4 values of the storage type each
            const size_t fb = (size_t)std::max(ctx->nmag, 1) * 4 * ctx->esz;
            void **rec[5] = {&ctx->fcst, &ctx->fmn, &ctx->fbc, &ctx->fdm[0], &ctx->fdm[1]};
            for (int q = 0; q < 5 && !rc; q++) {
                rc = dalloc(ctx, rec[q], fb);
                if (!rc) ctx->box_allocs.push_back(*rec[q]);
            }
        }
        if (rc) {
            free_box(ctx);
            return rc;
        }
        ctx->magnetic = true;
    } else {
        for (int a = 0; a < 3; a++) ctx->lo[a] = ctx->hi[a] = 0;
    }
    return is_fp64(ctx) ? set_materials_t<double>(ctx)
           : is_fp16(ctx) ? set_materials_t<float, __half>(ctx) : set_materials_t<float>(ctx);
}

int mmx_set_bias(mmx_ctx *ctx, double hx, double hy, double hz)
{
    if (!ctx || !ctx->E[0]) return MMX_ERR_INVALID;
    ctx->h0[0] = hx; ctx->h0[1] = hy; ctx->h0[2] = hz;
    return MMX_OK;
}

int mmx_set_M_cells(mmx_ctx *ctx, const double *mx, const double *my, const double *mz)
{
    if (!ctx || !ctx->E[0] || !mx || !my || !mz) return MMX_ERR_INVALID;
    if (!ctx->magnetic) return MMX_OK;
    const int *n = ctx->desc.n;
    size_t nc = (size_t)n[0] * n[1] * n[2];
    double *dm[3] = {};
    const double *in[3] = {mx, my, mz};
    int rc = MMX_OK;
    for (int c = 0; c < 3 && !rc; c++) {
        cudaError_t e = cudaMalloc((void **)&dm[c], nc * sizeof(double));
        if (e != cudaSuccess) rc = fail(ctx, MMX_ERR_OOM, "cudaMalloc: %s", cudaGetErrorString(e));
        else if (cudaMemcpyAsync(dm[c], in[c], nc * sizeof(double), cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
            rc = fail(ctx, MMX_ERR_CUDA, "copy of M cells failed");
    }
    if (!rc) {
        int nblk = (int)((ctx->nb + 255) / 256);
        for (int d = 0; d < 3; d++) {
            if (is_fp64(ctx))
                k_box_init_m<double><<<nblk, 256, 0, ctx->stream>>>(ctx->g, make_box<double>(ctx), d, dm[0], dm[1], dm[2]);
            else
                k_box_init_m<float><<<nblk, 256, 0, ctx->stream>>>(ctx->g, make_box<float>(ctx), d, dm[0], dm[1], dm[2]);
        }
        if (cudaGetLastError() != cudaSuccess) rc = fail(ctx, MMX_ERR_CUDA, "init M launch failed");
    }
    cudaStreamSynchronize(ctx->stream);
    for (int c = 0; c < 3; c++) cudaFree(dm[c]);
    ctx->m_rec_stale = true;
    ctx->m_box_stale = false;
    if (rc) return rc;
    rc = read_status(ctx);
    if (rc == MMX_ERR_INVALID) return fail(ctx, rc, "a magnetic face has no magnetisation direction");
    return rc;
}

int mmx_set_field(mmx_ctx *ctx, int id, const double *host, long long n)
{
    if (!ctx || !ctx->E[0] || !host) return MMX_ERR_INVALID;
    int e[3];
    if (!field_ext(ctx, id, e)) return fail(ctx, MMX_ERR_INVALID, "bad field id %d", id);
    if (n != (long long)e[0] * e[1] * e[2]) return fail(ctx, MMX_ERR_INVALID, "field %d needs %lld values", id, (long long)e[0] * e[1] * e[2]);
    ctx->walls_dirty = true;
    ctx->touched = true;
    return is_fp64(ctx) ? copy_field_t<double>(ctx, id, const_cast<double *>(host), n, 1)
                        : copy_field_t<float>(ctx, id, const_cast<double *>(host), n, 1);
}

int mmx_get_field(mmx_ctx *ctx, int id, double *host, long long n)
{
    if (!ctx || !ctx->E[0] || !host) return MMX_ERR_INVALID;
    int e[3];
    if (!field_ext(ctx, id, e)) return fail(ctx, MMX_ERR_INVALID, "bad field id %d", id);
    if (n != (long long)e[0] * e[1] * e[2]) return fail(ctx, MMX_ERR_INVALID, "field %d needs %lld values", id, (long long)e[0] * e[1] * e[2]);
    int rc = is_fp64(ctx) ? copy_field_t<double>(ctx, id, host, n, 0) : copy_field_t<float>(ctx, id, host, n, 0);
    if (rc) return rc;
    return read_status(ctx);
}

int mmx_get_material(mmx_ctx *ctx, int which, double *host, long long n)
{
    if (!ctx || !ctx->E[0] || !host || which < 0 || which > 17) return MMX_ERR_INVALID;
    int c = which % 3, kind = which / 3;
    int e[3];
    if (kind < 2) edge_ext(ctx, c, e); else face_ext(ctx, c, e);
    long long N = (long long)e[0] * e[1] * e[2];
    if (n != N) return fail(ctx, MMX_ERR_INVALID, "material %d needs %lld values", which, N);
    static const int cell_of_kind[6] = {0, 1, 2, 3, 4, 5};
    static const double dflt[6] = {1.0, 0.0, 1.0, 0.0, 0.0, 0.0};
    double *cellp = ctx->cell[cell_of_kind[kind]];
    if (!cellp) {
        for (long long q = 0; q < N; q++) host[q] = dflt[kind];
        return MMX_OK;
    }
    int rc = ensure_stage(ctx, ctx->npad);
    if (rc) return rc;
    double *tmp = nullptr;
    CK(cudaMalloc((void **)&tmp, ctx->npad * sizeof(double)));
    k_mean<<<node_grid(ctx), node_block(), 0, ctx->stream>>>(ctx->g, cellp, kind < 2 ? 0 : 1, c, tmp);
    cudaError_t le = cudaGetLastError();
    // compact into the staging buffer as a double field
    if (le == cudaSuccess) {
        Box<double> b = make_box<double>(ctx);
        int blocks = (int)((N + 255) / 256);
        k_copy_field<double><<<blocks, 256, 0, ctx->stream>>>(ctx->g, tmp, b, 0, e[0], e[1], e[2], ctx->stage, 0);
        le = cudaGetLastError();
    }
    if (le == cudaSuccess) le = cudaMemcpyAsync(host, ctx->stage, (size_t)N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(tmp);
    if (le != cudaSuccess) return fail(ctx, MMX_ERR_CUDA, "material readback: %s", cudaGetErrorString(le));
    return MMX_OK;
}

int mmx_add_source(mmx_ctx *ctx, const mmx_source_desc *s)
{
    if (!ctx || !ctx->E[0] || !s) return MMX_ERR_INVALID;
    if ((int)ctx->src.size() >= kMaxSources) return fail(ctx, MMX_ERR_INVALID, "at most %d sources", kMaxSources);
    if (s->kind < 0 || s->kind > 3 || s->comp < 0 || s->comp > 2 || !(s->tp > 0))
        return fail(ctx, MMX_ERR_INVALID, "bad source kind/comp/tp");
    int e[3];
    if (s->kind == 3) face_ext(ctx, s->comp, e); else edge_ext(ctx, s->comp, e);
    int ix[3] = {s->i, s->j, s->k};
    if (s->kind == 1) {
        if (s->comp == 2 || s->k < 0 || s->k > ctx->desc.n[2]) return fail(ctx, MMX_ERR_INVALID, "bad plane source");
        if (ctx->g.per[2] && s->k == ctx->desc.n[2]) return fail(ctx, MMX_ERR_INVALID, "use node 0, not n, on a periodic axis");
    } else {
        for (int a = 0; a < 3; a++) {
            if (ix[a] < 0 || ix[a] >= e[a]) return fail(ctx, MMX_ERR_INVALID, "source index out of range");
            bool nodal = e[a] == ctx->desc.n[a] + 1;
            if (ctx->g.per[a] && nodal && ix[a] == ctx->desc.n[a])
                return fail(ctx, MMX_ERR_INVALID, "use node 0, not n, on a periodic axis");
            if ((s->kind == 2 || s->kind == 3) && ctx->g.per[a] && nodal && ix[a] == 0)
                return fail(ctx, MMX_ERR_INVALID, "hard sources may not sit on a periodic seam");
        }
    }
    ctx->src.push_back(*s);
    std::vector<Src<double>> hs(ctx->src.size());
    for (size_t q = 0; q < ctx->src.size(); q++) {
        const mmx_source_desc &d = ctx->src[q];
        hs[q].kind = d.kind; hs[q].comp = d.comp; hs[q].i = d.i; hs[q].j = d.j; hs[q].k = d.k;
        hs[q].amp = d.amp; hs[q].f0 = d.f0; hs[q].tp = d.tp; hs[q].t0 = d.t0;
    }
    // Src<T> has the same layout for both T (only doubles and ints)
    CK(cudaMemcpyAsync(ctx->dsrc, hs.data(), hs.size() * sizeof(Src<double>), cudaMemcpyHostToDevice, ctx->stream));
    // a plane source changes the cost of its plane: re-place the chunk bounds
    if (s->kind == 1 && ctx->vec_chunk)
        ctx->vec_grid.z = plan_zchunks(ctx, (ctx->desc.n[2] + ctx->vec_chunk - 1) / ctx->vec_chunk);
    CK(cudaStreamSynchronize(ctx->stream));
    return MMX_OK;
}

int mmx_set_path(mmx_ctx *ctx, int path)
{
    if (!ctx || (path != MMX_PATH_PLAIN && path != MMX_PATH_FUSED)) return MMX_ERR_INVALID;
    ctx->path = path;
    return MMX_OK;
}

int mmx_step(mmx_ctx *ctx, int nsteps)
{
    if (!ctx || !ctx->E[0] || nsteps < 0) return MMX_ERR_INVALID;
    if (nsteps == 0) return MMX_OK;
    CK(cudaMemsetAsync(ctx->bar, 0, kBarWords * sizeof(unsigned long long), ctx->stream));
    if (ctx->inject_timeout) {
        // the state a bounded wait leaves when it gives up at the start of
        // this call: the timeout latched, the arrival counter one ahead
        ctx->inject_timeout = false;
        const int e = kErrTimeout;
        const unsigned long long one = 1;
        CK(cudaMemcpyAsync(ctx->errw, &e, sizeof e, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->bar, &one, sizeof one, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    bool hard = false;
    for (auto &q : ctx->src) hard |= q.kind >= 2;
    const bool fp64 = is_fp64(ctx);
    // M lives in the magnetic-face records while stepping and in the box
    // arrays where the API reads and writes it; the records are refreshed
    // only if the box arrays were written since the last step
    int rc = MMX_OK;
    if (ctx->m_rec_stale) {
        rc = fp64 ? box_m_sync<double>(ctx, 1) : box_m_sync<float>(ctx, 1);
        if (rc) return rc;
        ctx->m_rec_stale = false;
    }
    ctx->touched = true;
    if (is_fp16(ctx)) {
        if (ctx->path != MMX_PATH_FUSED || hard)
            rc = fail(ctx, MMX_ERR_INVALID, "FP16 storage runs the fused path without hard sources");
        else
            rc = step_fused<float, __half>(ctx, nsteps);
    } else if (ctx->path == MMX_PATH_FUSED && !hard)
        rc = fp64 ? step_fused<double>(ctx, nsteps) : step_fused<float>(ctx, nsteps);
    else
        rc = fp64 ? step_plain<double>(ctx, nsteps) : step_plain<float>(ctx, nsteps);
    // the records now hold M; the box arrays are refreshed when read
    if (ctx->magnetic) ctx->m_box_stale = true;
    return rc;
}

int mmx_sync(mmx_ctx *ctx)
{
    if (!ctx || !ctx->E[0]) return MMX_ERR_INVALID;
    CK(cudaStreamSynchronize(ctx->stream));
    return read_status(ctx);
}

int mmx_check_bounded_wait(mmx_ctx *ctx)
{
    if (!ctx || !ctx->E[0]) return MMX_ERR_INVALID;
    int rc = read_status(ctx);
    if (rc) return rc;
    // the grid barrier, then the voting barrier of the H/M iteration
    for (int vote = 0; vote < 2; vote++) {
        CK(cudaMemsetAsync(ctx->bar, 0, kBarWords * sizeof(unsigned long long), ctx->stream));
        k_barrier_probe<<<2, 32, 0, ctx->stream>>>(ctx->bar, ctx->errw, 1, vote);
        CK(cudaGetLastError());
        rc = read_status(ctx);
        if (rc != MMX_ERR_TIMEOUT) return rc;
    }
    return rc;
}

int mmx_inject_timeout(mmx_ctx *ctx)
{
    if (!ctx || !ctx->E[0]) return MMX_ERR_INVALID;
    ctx->inject_timeout = true;
    return MMX_OK;
}

int mmx_set_fused_staging(mmx_ctx *ctx, int bulk)
{
    if (!ctx || !ctx->E[0] || (bulk != 0 && bulk != 1)) return MMX_ERR_INVALID;
    if (ctx->bulk_staging != bulk) {
        ctx->bulk_staging = bulk;
        ctx->vec_chunk = 0;     // plan the vectorised pass again at the next step
    }
    return MMX_OK;
}

int mmx_check_guards(mmx_ctx *ctx)
{
    if (!ctx || !ctx->E[0]) return MMX_ERR_INVALID;
    CK(cudaStreamSynchronize(ctx->stream));
    unsigned char h[kGuardBytes];
    int bad = 0;
    size_t first = 0;
    for (size_t q = 0; q < ctx->guards.size(); q++) {
        const unsigned char *g = (const unsigned char *)ctx->guards[q].first + ctx->guards[q].second;
        CK(cudaMemcpy(h, g, kGuardBytes, cudaMemcpyDeviceToHost));
        for (size_t u = 0; u < kGuardBytes; u++)
            if (h[u] != kGuardByte) {
                if (!bad) first = q;
                bad++;
                break;
            }
    }
    if (bad)
        return fail(ctx, MMX_ERR_INVALID, "%d of %zu device arrays were written past their end (first: %zu bytes)",
                    bad, ctx->guards.size(), ctx->guards[first].second);
    return MMX_OK;
}

int mmx_set_box_kernel(mmx_ctx *ctx, int resident)
{
    if (!ctx || !ctx->E[0] || (resident != 0 && resident != 1)) return MMX_ERR_INVALID;
    ctx->box_resident = resident;
    return MMX_OK;
}

int mmx_get_info(mmx_ctx *ctx, mmx_info *out)
{
    if (!ctx || !ctx->E[0] || !out) return MMX_ERR_INVALID;
    memset(out, 0, sizeof *out);
    out->box_kernel = ctx->last_box;
    out->box_resident_faces_per_thread = ctx->magnetic ? ctx->res_faces : 0;
    out->fused_kernel = ctx->last_fused;
    out->tma_fallback = ctx->tma_fallback;
    out->bulk_staging = ctx->bulk_staging;
    out->box_blocks = !ctx->magnetic ? 0 : ctx->last_box == 2 ? ctx->res_blocks : ctx->coop_blocks;
    out->box_faces_magnetic = ctx->magnetic ? ctx->nmag : 0;
    out->box_faces_other = ctx->magnetic ? ctx->nnon : 0;
    return MMX_OK;
}

int mmx_kernel_binary_version(void)
{
    cudaFuncAttributes a;
    constexpr int BY = VecRows<float>::value, ST = VecStages<float, false>::value;
    if (cudaFuncGetAttributes(&a, k_fused_vec_tma<float, float, BY, ST, 2, true, false>) != cudaSuccess) {
        cudaGetLastError();
        return MMX_ERR_CUDA;
    }
    return a.binaryVersion;
}

int mmx_set_step_count(mmx_ctx *ctx, long long steps)
{
    if (!ctx || !ctx->E[0] || steps < 0) return MMX_ERR_INVALID;
    ctx->steps = steps;
    return MMX_OK;
}

int mmx_get_stats(mmx_ctx *ctx, mmx_stats *out)
{
    if (!ctx || !ctx->E[0] || !out) return MMX_ERR_INVALID;
    CK(cudaStreamSynchronize(ctx->stream));
    unsigned long long hs = 0;
    double lr = 0.0;
    CK(cudaMemcpy(&hs, ctx->halfsteps, sizeof hs, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&lr, ctx->last_res, sizeof lr, cudaMemcpyDeviceToHost));
    out->steps = ctx->steps;
    out->half_steps = ctx->magnetic ? (long long)hs : 2 * ctx->steps;
    out->last_residual = lr;
    out->iters_min = 0;
    out->iters_max = 0;
    if (ctx->magnetic && hs > 0) {
        long long m = std::min<long long>((long long)hs, kIterLogCap);
        std::vector<int> v(kIterLogCap);
        CK(cudaMemcpy(v.data(), ctx->iterlog, kIterLogCap * sizeof(int), cudaMemcpyDeviceToHost));
        int mn = 1 << 30, mx = 0;
        for (long long q = 0; q < m; q++) {
            mn = std::min(mn, v[q]);
            mx = std::max(mx, v[q]);
        }
        out->iters_min = mn;
        out->iters_max = mx;
    }
    out->status = read_status(ctx);
    return MMX_OK;
}

long long mmx_get_iter_log(mmx_ctx *ctx, int *host, long long cap)
{
    if (!ctx || !ctx->E[0] || (cap > 0 && !host)) return MMX_ERR_INVALID;
    CK(cudaStreamSynchronize(ctx->stream));
    if (!ctx->magnetic) return 0;
    unsigned long long hs = 0;
    CK(cudaMemcpy(&hs, ctx->halfsteps, sizeof hs, cudaMemcpyDeviceToHost));
    long long avail = std::min<long long>((long long)hs, kIterLogCap);
    long long m = std::min(avail, cap);
    std::vector<int> v(kIterLogCap);
    CK(cudaMemcpy(v.data(), ctx->iterlog, kIterLogCap * sizeof(int), cudaMemcpyDeviceToHost));
    long long first = (long long)hs - avail;   // oldest kept
    for (long long q = 0; q < m; q++) host[q] = v[(first + q) % kIterLogCap];
    return m;
}

int mmx_set_profiling(mmx_ctx *ctx, int enable)
{
    if (!ctx || !ctx->E[0]) return MMX_ERR_INVALID;
    ctx->prof_on = enable != 0;
    return MMX_OK;
}

int mmx_get_profile(mmx_ctx *ctx, mmx_kernel_profile *out, int cap, int reset)
{
    if (!ctx || !ctx->E[0] || (cap > 0 && !out)) return MMX_ERR_INVALID;
    CK(cudaStreamSynchronize(ctx->stream));
    prof_collect(ctx);
    int m = 0;
    for (int k = 0; k < KK_COUNT; k++) {
        if (ctx->prof_launches[k] == 0) continue;
        if (m < cap) {
            memset(out[m].name, 0, sizeof out[m].name);
            strncpy(out[m].name, kKernelNames[k], sizeof out[m].name - 1);
            out[m].launches = ctx->prof_launches[k];
            out[m].total_ms = ctx->prof_ms[k];
        }
        m++;
    }
    if (reset)
        for (int k = 0; k < KK_COUNT; k++) {
            ctx->prof_launches[k] = 0;
            ctx->prof_ms[k] = 0.0;
        }
    return m;
}

int mmx_set_storage_scale(mmx_ctx *ctx, double sE, double sH)
{
    if (!ctx || !ctx->E[0]) return MMX_ERR_INVALID;
    if (!is_fp16(ctx)) return fail(ctx, MMX_ERR_INVALID, "storage scales apply to MMX_FP16 contexts");
    if (ctx->touched) return fail(ctx, MMX_ERR_INVALID, "set the storage scales before any field or step");
    if (!(sE > 0) || !(sH > 0) || !std::isfinite(sE) || !std::isfinite(sH))
        return fail(ctx, MMX_ERR_INVALID, "storage scales must be positive and finite");
    ctx->sE = sE;
    ctx->sH = sH;
    return MMX_OK;
}

int mmx_flux_gradient(mmx_ctx *ctx, int kp, int nsteps, int checkpoint_every, double *loss, double *grad_eps,
                      double *grad_h0)
{
    if (!ctx || !ctx->E[0] || !loss || !grad_eps) return MMX_ERR_INVALID;
    if (ctx->magnetic && ctx->desc.order != 2)
        return fail(ctx, MMX_ERR_INVALID, "the adjoint of magnetic grids covers the second-order scheme");
    for (int a = 0; a < 3; a++)
        if (ctx->g.per[a]) return fail(ctx, MMX_ERR_INVALID, "the adjoint covers grids without periodic axes");
    if (is_fp16(ctx)) return fail(ctx, MMX_ERR_INVALID, "the adjoint runs in FP32 or FP64");
    for (auto &q : ctx->src)
        if (q.kind >= 2) return fail(ctx, MMX_ERR_INVALID, "the adjoint covers soft sources only");
    if (!ctx->probes.empty() || !ctx->flux_k.empty())
        return fail(ctx, MMX_ERR_INVALID, "remove probes and flux planes before the adjoint");
    if (kp < 0 || kp > ctx->desc.n[2]) return fail(ctx, MMX_ERR_INVALID, "flux plane k must be in [0, nz]");
    if (nsteps < 1 || checkpoint_every < 1) return fail(ctx, MMX_ERR_INVALID, "nsteps and checkpoint_every >= 1");
    if (grad_h0) grad_h0[0] = grad_h0[1] = grad_h0[2] = 0.0;
    int rc = ensure_box_m(ctx);   // the adjoint works from and on the box arrays
    if (rc) return rc;
    rc = is_fp64(ctx) ? flux_gradient_t<double>(ctx, kp, nsteps, checkpoint_every, loss, grad_eps, grad_h0)
                      : flux_gradient_t<float>(ctx, kp, nsteps, checkpoint_every, loss, grad_eps, grad_h0);
    ctx->m_rec_stale = true;
    ctx->m_box_stale = false;
    return rc;
}

int mmx_add_probe(mmx_ctx *ctx, int field, int i, int j, int k)
{
    if (!ctx || !ctx->E[0]) return MMX_ERR_INVALID;
    if (field < 0 || field > 2) return fail(ctx, MMX_ERR_INVALID, "probes record E components (fields 0-2)");
    if ((int)ctx->probes.size() >= kMaxProbes) return fail(ctx, MMX_ERR_INVALID, "at most %d probes", kMaxProbes);
    int e[3];
    field_ext(ctx, field, e);
    const int ix[3] = {i, j, k};
    for (int a = 0; a < 3; a++)
        if (ix[a] < 0 || ix[a] >= e[a]) return fail(ctx, MMX_ERR_INVALID, "probe index out of range");
    if (!ctx->probe_buf) {
        int rc = dalloc(ctx, (void **)&ctx->probe_buf, (size_t)kProbeRows * kMaxProbes * sizeof(double));
        if (!rc) rc = dalloc(ctx, (void **)&ctx->dprobe, kMaxProbes * sizeof(int2));
        if (rc) return rc;
    }
    // samples so far were recorded with the old probe count: start afresh
    ctx->probe_rows = 0;
    ctx->probes.push_back(make_int2(field, (int)gidx_host(ctx, i, j, k)));
    CK(cudaMemcpyAsync(ctx->dprobe, ctx->probes.data(), ctx->probes.size() * sizeof(int2), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return (int)ctx->probes.size() - 1;
}

long long mmx_get_probes(mmx_ctx *ctx, double *out, long long max_rows, int reset)
{
    if (!ctx || !ctx->E[0] || (max_rows > 0 && !out) || max_rows < 0) return MMX_ERR_INVALID;
    const long long np = (long long)ctx->probes.size();
    const long long rows = std::min(ctx->probe_rows, max_rows);
    if (np > 0 && rows > 0)
        CK(cudaMemcpyAsync(out, ctx->probe_buf, (size_t)(rows * np) * sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (reset) ctx->probe_rows = 0;
    return rows;
}

int mmx_energy(mmx_ctx *ctx, double *out)
{
    if (!ctx || !ctx->E[0] || !out) return MMX_ERR_INVALID;
    int rc = is_fp64(ctx) ? energy_t<double>(ctx, out)
             : is_fp16(ctx) ? energy_t<float, __half>(ctx, out) : energy_t<float>(ctx, out);
    return rc ? rc : read_status(ctx);
}

int mmx_add_flux_plane(mmx_ctx *ctx, int k)
{
    if (!ctx || !ctx->E[0]) return MMX_ERR_INVALID;
    if (k < 0 || k > ctx->desc.n[2]) return fail(ctx, MMX_ERR_INVALID, "flux plane k must be in [0, nz]");
    if ((int)ctx->flux_k.size() >= kMaxFluxPlanes)
        return fail(ctx, MMX_ERR_INVALID, "at most %d flux planes", kMaxFluxPlanes);
    int rc = ensure_monitor(ctx);
    if (rc) return rc;
    const int idx = (int)ctx->flux_k.size();
    CK(cudaMemsetAsync(ctx->flux_acc + 4 * idx, 0, 4 * sizeof(double), ctx->stream));
    ctx->flux_k.push_back(k);
    return idx;
}

int mmx_get_flux(mmx_ctx *ctx, int index, double out[2], int reset)
{
    if (!ctx || !ctx->E[0] || !out || index < 0 || index >= (int)ctx->flux_k.size()) return MMX_ERR_INVALID;
    double acc[4];
    CK(cudaMemcpyAsync(acc, ctx->flux_acc + 4 * index, sizeof acc, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    out[0] = acc[0] + acc[1];
    out[1] = acc[2];
    if (reset) CK(cudaMemsetAsync(ctx->flux_acc + 4 * index, 0, 4 * sizeof(double), ctx->stream));
    return MMX_OK;
}

int mmx_get_field_device(mmx_ctx *ctx, int id, void **ptr, long long *sx, long long *sy)
{
    if (!ctx || !ctx->E[0] || !ptr || !sx || !sy) return MMX_ERR_INVALID;
    if (id < 0 || id > 5) return fail(ctx, MMX_ERR_INVALID, "device views exist for E and H (ids 0-5)");
    *ptr = id < 3 ? ctx->E[id] : ctx->H[id - 3];
    *sx = ctx->g.X;
    *sy = (long long)ctx->g.X * ctx->g.Y;
    return MMX_OK;
}


} // extern "C"

// ============================================================ batches
//
// A batch advances independent contexts (instances) together: per time step
// one fused launch over every instance's tiles and one cooperative H/M launch
// over every instance's box faces, the whole mmx_batch_step call captured as
// one CUDA graph.  Instances are ordinary contexts, set up and read back
// through the per-context calls; the batch only gathers their device
// pointers into tables (rebuilt at every call, since the E/H buffers of a
// context alternate from step to step).

struct mmx_batch {
    std::vector<mmx_ctx *> ctx;
    cudaStream_t stream = nullptr;
    bool own_stream = false;               // created here (graph capture needs a non-default stream)
    int prec = MMX_FP32;
    bool pml = false, gen = false, magnetic = false;
    int planes = 0;                        // z planes per fused CTA (0: whole grid)
    std::vector<int> chunk, xstride;       // per instance, from the batch's plan
    // fused launch
    void *vinst[2] = {};                   // VecInst<T, S>[ninst] per parity
    int4 *work = nullptr;
    int nwork = 0;
    // box launch
    void *binst[2] = {};                   // BoxInst<T, S>[ninst] per parity
    unsigned long long *mag = nullptr;   // packed magnetic-face list (k_pack_faces)
    int4 *non = nullptr;
    int *non_inst = nullptr;
    int nmag = 0, nnon = 0;
    unsigned long long *res = nullptr, *bar = nullptr;
    int *err = nullptr;
    int coop_blocks = 0;
    size_t box_smem = 0;
    int order = 0;           // every instance's scheme order, or 0 if they differ
    // H/M launch size: blocks needed, resident blocks per SM, SMs, and the
    // caller's cap per SM (0: as many as are resident)
    long long box_need = 0;
    int box_per = 0, nsm = 0, box_per_sm = 0;
    // source amplitudes of every instance for one call: [inst][step][source]
    void *amp = nullptr;
    long long amp_cap = 0;                 // elements allocated
    // graph of the last call length
    cudaGraphExec_t graph = nullptr;
    int graph_steps = -1;
    std::vector<void *> allocs;
    std::string errmsg;
};

static int bfail(mmx_batch *b, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    b->errmsg = buf;
    return code;
}

#define BCK(call)                                                                                    \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return bfail(b, MMX_ERR_CUDA, "CUDA %s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                         __LINE__);                                                                  \
    } while (0)

static int balloc(mmx_batch *b, void **p, size_t bytes)
{
    BCK(cudaMalloc(p, bytes > 0 ? bytes : 16));
    BCK(cudaMemsetAsync(*p, 0, bytes > 0 ? bytes : 16, b->stream));
    b->allocs.push_back(*p);
    return MMX_OK;
}

// Work table of the fused launch: every (instance, strip, row tile, z chunk).
template <typename T> static int batch_plan(mmx_batch *b)
{
    constexpr int BY = VecRows<T>::value;
    constexpr int W = 32 * Lanes<T>::V;
    std::vector<int4> work;
    b->chunk.assign(b->ctx.size(), 0);
    b->xstride.assign(b->ctx.size(), 0);
    for (size_t q = 0; q < b->ctx.size(); q++) {
        mmx_ctx *c = b->ctx[q];
        const int *n = c->desc.n;
        const int xs = W - Lanes<T>::V;
        const int ntx = n[0] <= W ? 1 : 1 + (n[0] - W + xs - 1) / xs;
        const int nty = (n[1] + BY - 1) / BY;
        const int chunk = b->planes > 0 ? std::min(b->planes, n[2]) : n[2];
        const int nch = (n[2] + chunk - 1) / chunk;
        b->chunk[q] = chunk;
        b->xstride[q] = xs;
        for (int z = 0; z < nch; z++)
            for (int y = 0; y < nty; y++)
                for (int x = 0; x < ntx; x++) work.push_back(make_int4((int)q, x, y, z));
    }
    if (b->work) {
        cudaFree(b->work);
        b->allocs.erase(std::find(b->allocs.begin(), b->allocs.end(), (void *)b->work));
        b->work = nullptr;
    }
    int rc = balloc(b, (void **)&b->work, work.size() * sizeof(int4));
    if (rc) return rc;
    BCK(cudaMemcpyAsync(b->work, work.data(), work.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    b->nwork = (int)work.size();
    return MMX_OK;
}

// Concatenated face lists with their instance tags, per-instance residual
// rows, the barrier word and the cooperative grid size.
// Blocks of the batched H/M launch: enough for the larger face list, at
// most the resident wave, or box_per_sm blocks per SM if the caller capped it.
static void batch_box_grid(mmx_batch *b)
{
    const int per = b->box_per_sm > 0 ? std::min(b->box_per_sm, b->box_per) : b->box_per;
    b->coop_blocks = (int)std::max(1LL, std::min(b->box_need, (long long)per * b->nsm));
}

template <typename T, typename S> static int batch_box_setup(mmx_batch *b)
{
    const int ninst = (int)b->ctx.size();
    std::vector<int> ni;
    long long nm = 0, nn = 0;
    for (mmx_ctx *c : b->ctx) {
        nm += c->magnetic ? c->nmag : 0;
        nn += c->magnetic ? c->nnon : 0;
    }
    if (nm >= (1LL << 31) || nn >= (1LL << 31)) return bfail(b, MMX_ERR_INVALID, "batch has too many box faces");
    b->nmag = (int)nm;
    b->nnon = (int)nn;
    for (mmx_ctx *c : b->ctx)
        for (int a = 0; a < 3; a++)
            if (c->desc.n[a] >= (1 << 16)) return bfail(b, MMX_ERR_INVALID, "batched instance wider than 65535 cells");
    if (ninst > (1 << 14)) return bfail(b, MMX_ERR_INVALID, "more than 16384 batched instances");
    int rc = balloc(b, (void **)&b->mag, (size_t)std::max(1LL, nm) * sizeof(unsigned long long));
    if (!rc) rc = balloc(b, (void **)&b->non, (size_t)std::max(1LL, nn) * sizeof(int4));
    if (!rc) rc = balloc(b, (void **)&b->non_inst, (size_t)std::max(1LL, nn) * sizeof(int));
    if (!rc) rc = balloc(b, (void **)&b->res, 4 * (size_t)ninst * (kMaxIter + 1) * sizeof(unsigned long long));
    if (!rc) rc = balloc(b, (void **)&b->bar, kBarWords * sizeof(unsigned long long));
    if (!rc) rc = balloc(b, (void **)&b->err, sizeof(int));
    if (rc) return rc;
    long long om = 0, on = 0;
    ni.reserve(nn);
    for (int q = 0; q < ninst; q++) {
        mmx_ctx *c = b->ctx[q];
        if (!c->magnetic) continue;
        if (c->nmag) {
            k_pack_faces<<<(unsigned)((c->nmag + 255) / 256), 256, 0, b->stream>>>(c->dmag, b->mag + om, c->nmag, q);
            BCK(cudaGetLastError());
        }
        if (c->nnon)
            BCK(cudaMemcpyAsync(b->non + on, c->dnon, (size_t)c->nnon * sizeof(int4), cudaMemcpyDeviceToDevice,
                                b->stream));
        ni.insert(ni.end(), c->nnon, q);
        om += c->nmag;
        on += c->nnon;
    }
    if (nn) BCK(cudaMemcpyAsync(b->non_inst, ni.data(), ni.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    b->box_smem = (size_t)ninst * (sizeof(unsigned long long) + 2 * sizeof(int));
    // the H/M launch is specialised for the scheme order when every instance
    // has the same one
    b->order = b->ctx[0]->desc.order;
    for (mmx_ctx *c : b->ctx)
        if (c->desc.order != b->order) b->order = 0;
    const void *boxk = b->order == 2 ? (const void *)k_hm_box_batch<T, S, 2>
                     : b->order == 1 ? (const void *)k_hm_box_batch<T, S, 1>
                                     : (const void *)k_hm_box_batch<T, S, 0>;
    if (b->box_smem > 48 * 1024)
        BCK(cudaFuncSetAttribute(boxk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->box_smem));
    int dev = 0, nsm = 0, per = 0;
    BCK(cudaGetDevice(&dev));
    BCK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, boxk, 256, b->box_smem));
    if (per < 1) return bfail(b, MMX_ERR_CUDA, "batched H/M kernel cannot be resident");
    b->box_need = (std::max(nm, nn) + 255) / 256;
    b->box_per = per;
    b->nsm = nsm;
    batch_box_grid(b);
    return MMX_OK;
}

// Instance tables for parity p: p = 0 reads the contexts' current E/H and
// writes their second set; p = 1 the other way round.
template <typename T, typename S> static int batch_tables(mmx_batch *b, long long steps)
{
    const int ninst = (int)b->ctx.size();
    std::vector<VecInst<T, S>> vi[2];
    std::vector<BoxInst<T, S>> bi[2];
    long long base = 0;
    for (int p = 0; p < 2; p++) {
        vi[p].resize(ninst);
        bi[p].resize(ninst);
    }
    long long ampoff = 0;
    for (int q = 0; q < ninst; q++) {
        mmx_ctx *c = b->ctx[q];
        for (int p = 0; p < 2; p++) {
            void *const *Ea = p == 0 ? c->E : c->Ealt, *const *Eb = p == 0 ? c->Ealt : c->E;
            void *const *Ha = p == 0 ? c->H : c->Halt, *const *Hb = p == 0 ? c->Halt : c->H;
            void *const *Za = p == 0 ? c->Ezp : c->Ezpalt, *const *Zb = p == 0 ? c->Ezpalt : c->Ezp;
            VecInst<T, S> &v = vi[p][q];
            v.g = c->g;
            v.f = make_fields<T, S>(c);
            for (int a = 0; a < 3; a++) {
                v.io.Eo[a] = (const S *)Ea[a];
                v.io.Ho[a] = (const S *)Ha[a];
                v.io.En[a] = (S *)Eb[a];
                v.io.Hn[a] = (S *)Hb[a];
            }
            for (int a = 0; a < 2; a++) {
                v.io.Zo[a] = (const S *)Za[a];
                v.io.Zn[a] = (S *)Zb[a];
            }
            v.src = (const Src<T> *)c->dsrc;
            v.nsrc = (int)c->src.size();
            v.amp = (const T *)b->amp + ampoff;
            v.chunk = b->chunk[q];
            v.xstride = b->xstride[q];
            BoxInst<T, S> &x = bi[p][q];
            x.g = c->g;
            x.f = make_fields<T, S>(c);
            for (int a = 0; a < 3; a++) {
                x.f.E[a] = (S *)Eb[a];   // E^(n+1)
                x.f.H[a] = (S *)Ha[a];   // H^(n+1/2)
                x.Hout.p[a] = (S *)Hb[a];
            }
            x.b = make_box<T>(c);
            x.base_mag = (int)base;
        }
        ampoff += (long long)c->src.size() * steps;
        base += c->magnetic ? c->nmag : 0;
    }
    for (int p = 0; p < 2; p++) {
        BCK(cudaMemcpyAsync(b->vinst[p], vi[p].data(), ninst * sizeof(VecInst<T, S>), cudaMemcpyHostToDevice,
                            b->stream));
        BCK(cudaMemcpyAsync(b->binst[p], bi[p].data(), ninst * sizeof(BoxInst<T, S>), cudaMemcpyHostToDevice,
                            b->stream));
    }
    BCK(cudaStreamSynchronize(b->stream));
    return MMX_OK;
}

// Source amplitudes of every instance for steps [n0, n0 + steps) of its clock.
template <typename T> static int batch_amplitudes(mmx_batch *b, long long steps)
{
    long long total = 0;
    for (mmx_ctx *c : b->ctx) total += (long long)c->src.size() * steps;
    if (total > b->amp_cap) {
        if (b->amp) {
            cudaFree(b->amp);
            b->allocs.erase(std::find(b->allocs.begin(), b->allocs.end(), b->amp));
            b->amp = nullptr;
        }
        int rc = balloc(b, &b->amp, (size_t)std::max(1LL, total) * sizeof(T));
        if (rc) return rc;
        b->amp_cap = total;
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
            b->graph_steps = -1;
        }
    }
    std::vector<T> v((size_t)total);
    long long off = 0;
    for (mmx_ctx *c : b->ctx) {
        const size_t ns = c->src.size();
        for (long long s = 0; s < steps; s++)
            for (size_t q = 0; q < ns; q++) {
                const mmx_source_desc &d = c->src[q];
                const double t = ((double)(c->steps + s) + 0.5) * c->desc.dt;
                v[off + s * ns + q] = (T)((d.kind == 0 || d.kind == 1) ? host_waveform(d, t) : 0.0);
            }
        off += (long long)ns * steps;
    }
    if (total) BCK(cudaMemcpyAsync(b->amp, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return MMX_OK;
}

template <typename T, typename S, int NH, bool PMLK, bool GEN>
static void batch_fused_v(mmx_batch *b, int parity, int step)
{
    constexpr int BY = VecRows<T>::value, ST = VecStages<T, GEN>::value;
    k_fused_vec_batch<T, S, BY, ST, NH, PMLK, GEN><<<b->nwork, dim3(32, BY + 1), vec_smem_bytes<T, S, GEN>(),
                                                     b->stream>>>((const VecInst<T, S> *)b->vinst[parity],
                                                                  b->work, step);
}

template <typename T, typename S> static void batch_fused(mmx_batch *b, int parity, int step, int nhalf)
{
#define MMX_BATCH_CASE(NHV, PV, GV)                                                                  \
    if (nhalf == NHV && b->pml == PV && b->gen == GV) {                                              \
        batch_fused_v<T, S, NHV, PV, GV>(b, parity, step);                                           \
        return;                                                                                      \
    }
    MMX_BATCH_CASE(2, true, false) MMX_BATCH_CASE(2, false, false) MMX_BATCH_CASE(2, true, true)
    MMX_BATCH_CASE(2, false, true) MMX_BATCH_CASE(1, true, false) MMX_BATCH_CASE(1, false, false)
    MMX_BATCH_CASE(1, true, true) MMX_BATCH_CASE(1, false, true)
#undef MMX_BATCH_CASE
}

template <typename T, typename S, int NH, bool PMLK, bool GEN> static cudaError_t batch_smem_v()
{
    constexpr int BY = VecRows<T>::value, ST = VecStages<T, GEN>::value;
    return cudaFuncSetAttribute(k_fused_vec_batch<T, S, BY, ST, NH, PMLK, GEN>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vec_smem_bytes<T, S, GEN>());
}

template <typename T, typename S> static cudaError_t batch_smem()
{
    cudaError_t r[8] = {batch_smem_v<T, S, 1, false, false>(), batch_smem_v<T, S, 1, false, true>(),
                        batch_smem_v<T, S, 1, true, false>(),  batch_smem_v<T, S, 1, true, true>(),
                        batch_smem_v<T, S, 2, false, false>(), batch_smem_v<T, S, 2, false, true>(),
                        batch_smem_v<T, S, 2, true, false>(),  batch_smem_v<T, S, 2, true, true>()};
    for (cudaError_t x : r)
        if (x != cudaSuccess) return x;
    return cudaSuccess;
}

// The launches of steps [0, nsteps) on the batch stream (captured into the
// call's graph).
template <typename T, typename S> static int batch_enqueue(mmx_batch *b, int nsteps)
{
    const int ninst = (int)b->ctx.size();
    for (int s = 0; s < nsteps; s++) {
        const int p = s & 1, nhalf = s == nsteps - 1 ? 1 : 2;
        batch_fused<T, S>(b, p, s, nhalf);
        BCK(cudaGetLastError());
        if (b->magnetic) {
            const BoxInst<T, S> *inst = (const BoxInst<T, S> *)b->binst[p];
            int nsub = nhalf, slot = s & 1;
            void *args[] = {(void *)&inst,       (void *)&ninst,       (void *)&b->mag,
                            (void *)&b->nmag,    (void *)&b->non,      (void *)&b->non_inst, (void *)&b->nnon,
                            (void *)&b->res,     (void *)&b->bar,      (void *)&b->err, (void *)&nsub,
                            (void *)&slot};
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.gridDim = dim3(b->coop_blocks);
            cfg.blockDim = dim3(256);
            cfg.dynamicSmemBytes = b->box_smem;
            cfg.stream = b->stream;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            const void *boxk = b->order == 2 ? (const void *)k_hm_box_batch<T, S, 2>
                             : b->order == 1 ? (const void *)k_hm_box_batch<T, S, 1>
                                             : (const void *)k_hm_box_batch<T, S, 0>;
            BCK(cudaLaunchKernelExC(&cfg, boxk, args));
        }
    }
    return MMX_OK;
}

template <typename T, typename S> static int batch_step_t(mmx_batch *b, int nsteps)
{
    // per-instance start of the call: M into the records, the first H half
    // step, wall clean-up (all on the batch stream)
    std::vector<cudaStream_t> saved;
    for (mmx_ctx *c : b->ctx) {
        // work already queued on the instance's own stream comes first
        BCK(cudaStreamSynchronize(c->stream));
        saved.push_back(c->stream);
        c->stream = b->stream;
    }
    auto restore = [&]() {
        for (size_t q = 0; q < b->ctx.size(); q++) b->ctx[q]->stream = saved[q];
    };
    int rc = MMX_OK;
    for (mmx_ctx *c : b->ctx) {
        // the instance's M may sit in its records after a standalone step
        rc = ensure_box_m(c);
        if (!rc) rc = box_m_sync<T>(c, 1);
        if (!rc) {
            Fields<T, S> f = make_fields<T, S>(c);
            rc = half_step<T, S>(c, f, make_box<T>(c), (c->steps + 0.5) * c->desc.dt);
        }
        if (!rc && c->walls_dirty) {
            rc = zero_walls<S>(c);
            c->walls_dirty = false;
        }
        if (rc) {
            restore();
            return bfail(b, rc, "instance setup: %s", c->err.c_str());
        }
    }
    rc = batch_amplitudes<T>(b, nsteps);
    if (!rc) rc = batch_tables<T, S>(b, nsteps);
    if (rc) {
        restore();
        return rc;
    }
    BCK(cudaMemsetAsync(b->res, 0, 4 * b->ctx.size() * (kMaxIter + 1) * sizeof(unsigned long long), b->stream));
    if (!b->graph || b->graph_steps != nsteps) {
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        rc = batch_enqueue<T, S>(b, nsteps);
        cudaError_t ec = cudaStreamEndCapture(b->stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            restore();
            return rc;
        }
        BCK(ec);
        cudaError_t ei = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        BCK(ei);
        b->graph_steps = nsteps;
    }
    BCK(cudaGraphLaunch(b->graph, b->stream));
    for (mmx_ctx *c : b->ctx) {
        if (nsteps & 1) swap_buffers<T>(c);
        c->steps += nsteps;
        rc = box_m_sync<T>(c, 0);
        if (rc) break;
        c->m_rec_stale = c->m_box_stale = false;   // both copies hold the new M
    }
    restore();
    return rc;
}

template <typename T, typename S> static int batch_init(mmx_batch *b)
{
    const int ninst = (int)b->ctx.size();
    for (int p = 0; p < 2; p++) {
        int rc = balloc(b, &b->vinst[p], ninst * sizeof(VecInst<T, S>));
        if (!rc) rc = balloc(b, &b->binst[p], ninst * sizeof(BoxInst<T, S>));
        if (rc) return rc;
    }
    {
        cudaError_t e = batch_smem<T, S>();
        BCK(e);
    }
    int rc = batch_plan<T>(b);
    if (!rc && b->magnetic) rc = batch_box_setup<T, S>(b);
    return rc;
}

extern "C" {

int mmx_batch_create(mmx_ctx *const *ctxs, int count, void *cuda_stream, mmx_batch **out)
{
    if (!out) return MMX_ERR_INVALID;
    *out = nullptr;
    if (!ctxs || count < 1) return MMX_ERR_INVALID;
    mmx_batch *b = new (std::nothrow) mmx_batch;
    if (!b) return MMX_ERR_OOM;
    *out = b;
    b->stream = (cudaStream_t)cuda_stream;
    if (!b->stream) {
        BCK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        b->own_stream = true;
    }
    for (int q = 0; q < count; q++) {
        mmx_ctx *c = ctxs[q];
        if (!c || !c->E[0]) return bfail(b, MMX_ERR_INVALID, "instance %d is not a context", q);
        for (int r = 0; r < q; r++)
            if (ctxs[r] == c) return bfail(b, MMX_ERR_INVALID, "instance %d appears twice", q);
        if (q == 0) {
            b->prec = c->desc.prec;
            b->pml = c->g.npml > 0;
            b->gen = c->any_sigma || c->any_mu;
        }
        if (c->desc.prec != b->prec) return bfail(b, MMX_ERR_INVALID, "instances mix precisions");
        if ((c->g.npml > 0) != b->pml || (c->any_sigma || c->any_mu) != b->gen)
            return bfail(b, MMX_ERR_INVALID, "instances mix PML or conductive/permeable material variants");
        if (!vec_usable(c)) return bfail(b, MMX_ERR_INVALID, "instance %d needs PEC x and y walls", q);
        for (auto &s : c->src)
            if (s.kind >= 2) return bfail(b, MMX_ERR_INVALID, "instance %d has a hard source", q);
        if (!c->probes.empty() || !c->flux_k.empty())
            return bfail(b, MMX_ERR_INVALID, "instance %d has probes or flux planes (not recorded in batches)", q);
        b->magnetic |= c->magnetic;
        b->ctx.push_back(c);
    }
    return b->prec == MMX_FP64 ? batch_init<double, double>(b)
           : b->prec == MMX_FP16 ? batch_init<float, __half>(b) : batch_init<float, float>(b);
}

int mmx_batch_set_planes(mmx_batch *b, int planes)
{
    if (!b || b->ctx.empty() || planes < 0) return MMX_ERR_INVALID;
    b->planes = planes;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_steps = -1;
    }
    return b->prec == MMX_FP64 ? batch_plan<double>(b) : batch_plan<float>(b);
}

int mmx_batch_set_box_blocks(mmx_batch *b, int per_sm)
{
    if (!b || b->ctx.empty() || per_sm < 0) return MMX_ERR_INVALID;
    b->box_per_sm = per_sm;
    batch_box_grid(b);
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_steps = -1;
    }
    return MMX_OK;
}

int mmx_batch_step(mmx_batch *b, int nsteps)
{
    if (!b || b->ctx.empty() || nsteps < 0) return MMX_ERR_INVALID;
    if (nsteps == 0) return MMX_OK;
    for (mmx_ctx *c : b->ctx) {
        if (!vec_usable(c) || !c->probes.empty() || !c->flux_k.empty() || (c->g.npml > 0) != b->pml ||
            (c->any_sigma || c->any_mu) != b->gen)
            return bfail(b, MMX_ERR_INVALID, "an instance changed since the batch was made");
        for (auto &s : c->src)
            if (s.kind >= 2) return bfail(b, MMX_ERR_INVALID, "an instance has a hard source");
    }
    BCK(cudaMemsetAsync(b->bar, 0, kBarWords * sizeof(unsigned long long), b->stream));
    return b->prec == MMX_FP64 ? batch_step_t<double, double>(b, nsteps)
           : b->prec == MMX_FP16 ? batch_step_t<float, __half>(b, nsteps) : batch_step_t<float, float>(b, nsteps);
}

int mmx_batch_sync(mmx_batch *b)
{
    if (!b || b->ctx.empty()) return MMX_ERR_INVALID;
    BCK(cudaStreamSynchronize(b->stream));
    int w = 0;
    BCK(cudaMemcpy(&w, b->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (w) {
        int z = 0;
        BCK(cudaMemcpy(b->err, &z, sizeof(int), cudaMemcpyHostToDevice));
        BCK(cudaMemset(b->bar, 0, kBarWords * sizeof(unsigned long long)));
        if (w & kErrTimeout) return bfail(b, MMX_ERR_TIMEOUT, "a device-side wait gave up");
        if (w & kErrNonFinite) return bfail(b, MMX_ERR_NONFINITE, "a field became non-finite");
    }
    int first = MMX_OK;
    for (size_t q = 0; q < b->ctx.size(); q++) {
        int rc = read_status(b->ctx[q]);
        if (rc && first == MMX_OK) {
            first = rc;
            bfail(b, rc, "instance %d: %s", (int)q, b->ctx[q]->err.c_str());
        }
    }
    return first;
}

const char *mmx_batch_last_error(mmx_batch *b)
{
    return b ? b->errmsg.c_str() : "null batch";
}

int mmx_batch_destroy(mmx_batch *b)
{
    if (!b) return MMX_ERR_INVALID;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (void *p : b->allocs) cudaFree(p);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return MMX_OK;
}

} // extern "C"

// ====================================================== no-allocation entry

// Scratch of mmx_material_average_noalloc: the padded intermediate of the
// edge/face mean lives in this file-scope device array, so that the entry
// point allocates nothing.  Every GPU that loads the library holds it until
// the process exits.  In host code the name is only a stand-in: its device
// address is looked up once per device with cudaGetSymbolAddress.
constexpr size_t kNoAllocMaxElems = (size_t)1 << 20;   // 1,048,576 doubles = 8 MiB
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxElems];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_dev_ptr[kNoAllocMaxDevices] = {};
CUcontext g_noalloc_ctx[kNoAllocMaxDevices] = {};

// The CUDA context current on the calling thread (driver entry point, so
// the library needs no link against the driver library); null if unknown.
CUcontext current_context()
{
    using Fn = CUresult (*)(CUcontext *);
    static Fn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (Fn)p;
    });
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

// Device address of the scratch array on the current device.  It is looked
// up on the first call for that device, and again whenever the device's
// context has changed since (after cudaDeviceReset the runtime creates a new
// primary context, and the array gets a new address in it).
int noalloc_scratch(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MMX_ERR_CUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return MMX_ERR_INVALID;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    // cudaGetSymbolAddress makes the device's primary context current if no
    // context is yet, so the context is read after it on a first call
    const CUcontext before = current_context();
    if (!g_noalloc_dev_ptr[dev] || !before || before != g_noalloc_ctx[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MMX_ERR_CUDA;
        g_noalloc_dev_ptr[dev] = (double *)p;
        g_noalloc_ctx[dev] = current_context();
    }
    *out = g_noalloc_dev_ptr[dev];
    return MMX_OK;
}
} // namespace

extern "C" int mmx_material_average_noalloc(const mmx_grid_desc *desc, int location, const double *cell,
                                            double *out, long long n, void *cuda_stream)
{
    if (!desc || !cell || !out || location < 0 || location > 5) return MMX_ERR_INVALID;
    Geo g;
    memset(&g, 0, sizeof g);
    for (int a = 0; a < 3; a++) {
        if (desc->n[a] < 1 || desc->bc[a] < 0 || desc->bc[a] > 2) return MMX_ERR_INVALID;
        g.n[a] = desc->n[a];
        g.per[a] = desc->bc[a] == MMX_BC_PERIODIC;
    }
    long long X = ((long long)desc->n[0] + 1 + 7) / 8 * 8;
    long long padded = X * (desc->n[1] + 1LL) * (desc->n[2] + 1LL);
    if (padded > (long long)kNoAllocMaxElems) return MMX_ERR_INVALID;   // grid too large for the scratch
    if (desc->n[2] + 1 > 65535) return MMX_ERR_INVALID;                  // one launch row per z node
    g.X = (int)X;
    g.Y = desc->n[1] + 1;
    const int c = location % 3, kind = location < 3 ? 0 : 1;
    int e[3];
    for (int a = 0; a < 3; a++) e[a] = desc->n[a] + (kind == 0 ? (a == c ? 0 : 1) : (a == c ? 1 : 0));
    if (n != (long long)e[0] * e[1] * e[2]) return MMX_ERR_INVALID;
    double *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // clear an earlier, unrelated launch error so that the checks below see
    // only this call's launches
    cudaGetLastError();
    dim3 B(32, 8, 1), G((desc->n[0] + 1 + 31) / 32, (desc->n[1] + 1 + 7) / 8, desc->n[2] + 1);
    // every scratch element the gather reads is written by k_mean first, so
    // nothing has to be cleared between calls
    k_mean<<<G, B, 0, st>>>(g, cell, kind, c, scratch);
    if (cudaGetLastError() != cudaSuccess) return MMX_ERR_CUDA;
    Box<double> nobox;
    memset(&nobox, 0, sizeof nobox);
    k_copy_field<double><<<(int)((n + 255) / 256), 256, 0, st>>>(g, scratch, nobox, 0, e[0], e[1], e[2], out, 0);
    if (cudaGetLastError() != cudaSuccess) return MMX_ERR_CUDA;
    return MMX_OK;
}

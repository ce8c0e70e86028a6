/*
 * mmx.h -- C ABI of the B300 (sm_103a) coupled electrodynamics-micromagnetics
 * solver: the Yee-grid Ampere update of E and the iterated trapezoidal
 * Maxwell-LLG update of H and M of Yao, Jambunathan, Zeng & Nonaka,
 * "A Massively Parallel Time-Domain Coupled Electrodynamics-Micromagnetics
 * Solver" (arXiv 2103.12819), Sec. 3.
 *
 * Conventions used by every entry point
 *   - Grid: nx x ny x nz cells of size dx x dy x dz.  Cell (i, j, k) spans
 *     [i dx, (i+1) dx] x ... ; node indices run 0..n on each axis.
 *   - Yee locations (Sec. 3.1, Fig. 1): Ex (i+1/2, j, k), Ey (i, j+1/2, k),
 *     Ez (i, j, k+1/2) on edges; Hx (i, j+1/2, k+1/2), Hy (i+1/2, j, k+1/2),
 *     Hz (i+1/2, j+1/2, k) on faces; all three components of M on every face
 *     of all three face families.
 *   - Host arrays are float64, x fastest: element (i, j, k) of an array with
 *     extents (ex, ey, ez) is at i + ex*(j + ey*k).  Extents: Ex nx x (ny+1) x
 *     (nz+1), Ey (nx+1) x ny x (nz+1), Ez (nx+1) x (ny+1) x nz; x-face arrays
 *     (Hx and the x-face M) (nx+1) x ny x nz, y-face nx x (ny+1) x nz, z-face
 *     nx x ny x (nz+1).  Cell-centred arrays nx x ny x nz.
 *   - Field ids: 0-2 Ex, Ey, Ez; 3-5 Hx, Hy, Hz; 6-14 M as (x-face Mx, My,
 *     Mz), (y-face Mx, My, Mz), (z-face Mx, My, Mz); 15/16 the z-derivative
 *     parts of Ex/Ey inside the z-PML, 17/18 those of Hx/Hy (zero elsewhere).
 *   - Units SI: E V/m, H M and the bias A/m, J A/m^2, sigma S/m, |gamma|
 *     rad/(s T), dt s.
 *   - Ownership: the library owns all device memory of a context; host
 *     buffers belong to the caller and are only read (set_*) or written
 *     (get_*) during the call.
 *   - Errors: every int-returning entry point returns MMX_OK (0) or a
 *     negative MMX_ERR_* code; mmx_last_error() gives a message.  Device-side
 *     conditions (iteration cap reached, non-finite values, a bounded wait
 *     that gave up) latch in the context and are returned by the next
 *     synchronising call (mmx_sync, mmx_get_field, mmx_get_stats).  No call
 *     blocks without bound: every device wait carries an iteration limit.
 *   - Streams: work is enqueued on the stream given to mmx_create (NULL =
 *     the legacy default stream).  mmx_step is asynchronous.
 */
#ifndef MMX_H_
#define MMX_H_

#if defined(__GNUC__)
#define MMX_API __attribute__((visibility("default")))
#else
#define MMX_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define MMX_OK 0
#define MMX_ERR_INVALID (-1)        /* bad argument or state */
#define MMX_ERR_OOM (-2)            /* device allocation failed */
#define MMX_ERR_CUDA (-3)           /* a CUDA runtime call failed */
#define MMX_ERR_NOT_CONVERGED (-4)  /* a H/M half step hit max_iter */
#define MMX_ERR_NONFINITE (-5)      /* a field became NaN/Inf */
#define MMX_ERR_TIMEOUT (-6)        /* a bounded device wait gave up */

/* MMX_FP16: E, H and their PML split parts stored in FP16 (each value divided
 * by a per-context scale, see mmx_set_storage_scale), all arithmetic in FP32;
 * materials, M and the H/M iteration state stay FP32.  Supported on the
 * fused path for grids with PEC x and y walls and no hard sources; other
 * configurations make mmx_step return MMX_ERR_INVALID. */
typedef enum { MMX_FP64 = 0, MMX_FP32 = 1, MMX_FP16 = 2 } mmx_precision;
typedef enum { MMX_BC_PERIODIC = 0, MMX_BC_PEC = 1, MMX_BC_PML = 2 } mmx_bc;
typedef enum { MMX_PATH_PLAIN = 0, MMX_PATH_FUSED = 1 } mmx_path;

typedef struct mmx_ctx mmx_ctx;

/* Grid, time step and scheme (Sec. 3.1-3.2.3).
 *   n[3], d[3]  cells and cell size per axis (x, y, z).
 *   dt          time step (> 0; the caller applies its CFL rule).
 *   bc[3]       boundary per axis, same on both ends: periodic (Sec. 3.2.3,
 *               guard-cell exchange), PEC (tangential E and normal H held at
 *               0), or PML (z axis only: split-field, time-centred PML-2SC
 *               layers of pml_cells cells inside the grid, PEC behind them).
 *   order       2 = iterated trapezoidal scheme (Sec. 3.2.2), 1 = first-order
 *               forward-Euler scheme (Sec. 3.2.1).
 *   tol         stopping tolerance of the H/M iteration on the domain-wide
 *               max of |M^r - M^(r-1)|/Ms (Sec. 3.2.2; the paper uses 1e-6).
 *   max_iter    iteration cap (>= 1, <= 64).
 *   prec        arithmetic and storage precision of the fields. */
typedef struct {
    int n[3];
    double d[3];
    double dt;
    int bc[3];
    int pml_cells;
    int order;
    double tol;
    int max_iter;
    int prec;
} mmx_grid_desc;

/* Source (Sec. 3.2, "soft and hard sources"; waveform of Eq. gaulssian):
 *   g(t) = amp exp(-(t - t0)^2 / (2 tp^2)) cos(2 pi f0 t).
 *   kind 0  soft point current J_comp on the edge (i, j, k) of component
 *           comp, entering the E update at t = (n+1/2) dt.
 *   kind 1  soft plane current J_comp (comp 0 or 1) on every comp-edge of the
 *           z node plane k, shaped sin(pi x / (nx dx)) across x (TE10).
 *   kind 2  hard E: E_comp at edge (i, j, k) is overwritten with g(t^(n+1))
 *           after every E update.
 *   kind 3  hard H: H_comp at face (i, j, k) is overwritten with g(t) after
 *           every H/M half step, t its end time. */
typedef struct {
    int kind, comp, i, j, k;
    double amp, f0, tp, t0;
} mmx_source_desc;

typedef struct {
    long long steps;           /* full time steps done */
    long long half_steps;      /* H/M half steps logged */
    int iters_min, iters_max;  /* iteration counts over the logged half steps */
    double last_residual;      /* residual of the last H/M half step */
    int status;                /* latched device status (MMX_OK or MMX_ERR_*) */
} mmx_stats;

/* Create a context for the grid in *desc on the current CUDA device.
 * cuda_stream is a cudaStream_t (NULL = default stream); it must outlive the
 * context.  All fields start at zero and all materials at vacuum (eps_r 1,
 * sigma 0, mu_r 1, Ms 0).  Returns MMX_ERR_INVALID for an inconsistent
 * descriptor, MMX_ERR_OOM when device memory runs out; on failure *out may
 * still hold a context, usable only with mmx_last_error and mmx_destroy. */
MMX_API int mmx_create(const mmx_grid_desc *desc, void *cuda_stream, mmx_ctx **out);

/* Cell-centred materials -> Yee locations (Sec. 3.1): eps_r and sigma are
 * averaged to edges over the adjacent cells, mu_r, Ms, alpha and |gamma| to
 * faces over the two adjacent cells (existing cells only at non-periodic
 * walls; periodic axes wrap).  Each pointer is a host array of nx*ny*nz
 * doubles or NULL for the default (eps_r 1, sigma 0, mu_r 1, Ms 0, alpha 0,
 * |gamma| 0).  A face is magnetic iff its averaged Ms > 0; magnetic faces
 * restart at M = Ms zhat.  Ms must be 0 in the PML slabs (the paper's PML is
 * non-magnetic); every cell's Ms is 0 or in [1e-20, 1e20] A/m, eps_r and mu_r
 * > 0, sigma, alpha and |gamma| >= 0, else MMX_ERR_INVALID.  The magnetic box
 * must hold fewer than 2^30 faces per family.  Synchronises the context
 * stream. */
MMX_API int mmx_set_materials(mmx_ctx *ctx, const double *eps_r, const double *sigma,
                      const double *mu_r, const double *Ms, const double *alpha,
                      const double *gamma_abs);

/* Uniform bias field H0 (A/m) added to the effective field of every magnetic
 * face (Sec. 2: H_eff = H + H0). */
MMX_API int mmx_set_bias(mmx_ctx *ctx, double h0x, double h0y, double h0z);

/* Initial M from cell-centred values (Sec. 3.1): averaged to each face and
 * renormalised to the face's Ms (a face whose average is below 1e-6 Ms takes
 * the lower-index cell's direction).  Host arrays of nx*ny*nz doubles. */
MMX_API int mmx_set_M_cells(mmx_ctx *ctx, const double *mx, const double *my, const double *mz);

/* Copy a Yee-located field (ids above) from a host float64 array of exactly
 * n elements (its extent).  On periodic axes node index n is set equal to
 * node index 0.  FP32 contexts round to nearest.  M (ids 6-14) is stored on
 * the magnetic box only (the bounding box of the magnetic faces grown by one
 * face): only that region of the host array is read and moved, values
 * outside it are ignored and read back as zero; without magnetic material
 * every M value must be zero. */
MMX_API int mmx_set_field(mmx_ctx *ctx, int field_id, const double *host, long long n);

/* Copy a Yee-located field to a host float64 array of exactly n elements.
 * Synchronises the context stream and returns the latched device status. */
MMX_API int mmx_get_field(mmx_ctx *ctx, int field_id, double *host, long long n);

/* Edge/face material values after averaging: which = 0-2 eps_r on Ex/Ey/Ez
 * edges, 3-5 sigma on edges, 6-8 mu_r on x/y/z faces, 9-11 Ms, 12-14 alpha,
 * 15-17 |gamma| on faces.  Host float64 array of the edge/face extent. */
MMX_API int mmx_get_material(mmx_ctx *ctx, int which, double *host, long long n);

/* Register a source (see mmx_source_desc).  At most 32 per context. */
MMX_API int mmx_add_source(mmx_ctx *ctx, const mmx_source_desc *src);

/* Select the kernel path: MMX_PATH_PLAIN runs one kernel per update (H/M
 * half step, E update, H/M half step); MMX_PATH_FUSED (default) makes one
 * streaming pass per step (E update plus the two non-magnetic H half steps
 * that share curl E^(n+1)) and one launch for the magnetic box.  Both
 * compute the same scheme; contexts with hard sources always take the plain
 * path. */
MMX_API int mmx_set_path(mmx_ctx *ctx, int path);

/* Advance nsteps full time steps (Sec. 3.2: H/M half step with E^n, E
 * update with J at t^(n+1/2), H/M half step with E^(n+1)).  Asynchronous:
 * returns after enqueueing; the H/M iteration runs to the domain-wide
 * tolerance on the device with no host round trip.  Device conditions latch
 * (see mmx_sync). */
MMX_API int mmx_step(mmx_ctx *ctx, int nsteps);

/* Wait for the context stream and return the latched device status:
 * MMX_OK, MMX_ERR_NOT_CONVERGED (some half step reached max_iter; the step
 * went on with the last iterate), MMX_ERR_NONFINITE or MMX_ERR_TIMEOUT.
 * Reading the status clears it. */
MMX_API int mmx_sync(mmx_ctx *ctx);

/* Set the count of full time steps done, the time t = steps dt at which the
 * next step starts (the source waveforms are evaluated from it).  With
 * mmx_get_field / mmx_set_field over every field id (E, H, the 9 M
 * components and the PML split parts) this restores a checkpoint into a
 * context built with the same descriptor, materials, bias and sources.
 * MMX_ERR_INVALID for steps < 0. */
MMX_API int mmx_set_step_count(mmx_ctx *ctx, long long steps);

/* Statistics since creation; synchronises. */
MMX_API int mmx_get_stats(mmx_ctx *ctx, mmx_stats *out);

/* Check of the bounded device waits (failure detection without a fault):
 * launches, one after the other, the two grid-wide waits the H/M kernels
 * use (the grid barrier, and the voting barrier that also takes the
 * convergence decision), each in a two-block grid in which one block leaves
 * without arriving.  The other block gives up after its wait budget (about
 * 2^31 clock cycles, one second at the B300's clock), latches the timeout
 * and returns.  Returns MMX_ERR_TIMEOUT when both waits gave up as designed
 * (any other code means one did not); the barrier and error words are then
 * reset, so the context stays usable.  Synchronises; a status pending from
 * earlier work is returned first, without the check. */
MMX_API int mmx_check_bounded_wait(mmx_ctx *ctx);

/* Guard check: every device array the context allocates for its state,
 * coefficients, box records and work lists is followed by 256 bytes of a
 * fixed pattern; this reads them all back.  Returns MMX_OK when every guard
 * is intact, MMX_ERR_INVALID (with a message naming how many arrays and the
 * size of the first) when a kernel wrote past the end of an array, or
 * MMX_ERR_CUDA.  Synchronises the context's stream; no kernel is launched. */
MMX_API int mmx_check_guards(mmx_ctx *ctx);

/* Failure-detection test hook (the failure is made on the host, no GPU
 * fault): the next mmx_step call starts as if a bounded wait had given up in
 * its first launch, with MMX_ERR_TIMEOUT latched in the device status word
 * and the grid-barrier arrival counter one arrival ahead.  Every launch of
 * that call then returns at its entry instead of spending a wait budget at
 * each barrier, and the next synchronising call returns MMX_ERR_TIMEOUT and
 * resets the barrier words (the fields are then void).  Returns MMX_OK. */
MMX_API int mmx_inject_timeout(mmx_ctx *ctx);

/* Which kernels the fused path runs.
 *   fused_kernel        kernel of the last fused step: 0 none yet (or the
 *                       per-update path), 1 the one-column kernel (periodic x
 *                       or y, or a magnetic box reaching into the PML), 2 the
 *                       vectorised kernel with per-lane cp.async staging, 3
 *                       the vectorised kernel with bulk tensor copies (TMA).
 *   tma_fallback        1 if the bulk-copy staging applies (FP32 storage, no
 *                       sigma or mu_r, allowed by mmx_set_fused_staging) but
 *                       could not be set up (tensor-map encoding or its shared
 *                       memory), so the cp.async staging runs instead.
 *   bulk_staging        the setting of mmx_set_fused_staging (1 by default).
 *   box_blocks          blocks of the last cooperative H/M launch (0: no
 *                       magnetic material).
 *   box_faces_magnetic, box_faces_other   faces of the magnetic box with and
 *                       without Ms > 0.
 *   box_kernel          kernel of the last H/M launch: 0 none yet, 1 the
 *                       list-driven kernel (per-face records in global
 *                       memory), 2 the kernel with the records in shared
 *                       memory (see mmx_set_box_kernel).
 *   box_resident_faces_per_thread   magnetic faces per thread of the
 *                       shared-memory kernel (0: the box's magnetic faces do
 *                       not fit in one resident wave, or FP64 arithmetic). */
typedef struct {
    int fused_kernel;
    int tma_fallback;
    int bulk_staging;
    int box_blocks;
    long long box_faces_magnetic;
    long long box_faces_other;
    int box_kernel;
    int box_resident_faces_per_thread;
} mmx_info;
MMX_API int mmx_get_info(mmx_ctx *ctx, mmx_info *out);

/* Kernel of the H/M half steps.  resident = 1 (default): where the magnetic
 * faces fit in the GPU's shared memory (FP32 arithmetic, at most 3 faces per
 * thread over one resident wave of 256-thread blocks; about 0.45 M faces on
 * a B300), every block keeps its faces' iteration records (M^n, beta, C',
 * the current increment) in shared memory for the whole launch; elsewhere,
 * and with resident = 0, the list-driven kernel keeps them in global memory.
 * Both evaluate the same operations in the same order.  Takes effect at the
 * next mmx_step; MMX_ERR_INVALID for any other value. */
MMX_API int mmx_set_box_kernel(mmx_ctx *ctx, int resident);

/* Staging of the vectorised fused kernel: bulk = 1 (default) stages the planes
 * with bulk tensor copies where they apply, bulk = 0 always with per-lane
 * cp.async copies.  Both compute the same updates; the switch exists to
 * compare them.  Takes effect at the next mmx_step.  MMX_ERR_INVALID for any
 * other value. */
MMX_API int mmx_set_fused_staging(mmx_ctx *ctx, int bulk);

/* The SM architecture the library's kernels were compiled for, as the CUDA
 * runtime reports it for the current device (major * 10 + minor: 103 for
 * sm_103a), or MMX_ERR_CUDA if the kernels cannot run on it. */
MMX_API int mmx_kernel_binary_version(void);

/* Iteration count of each H/M half step, oldest first (up to cap entries of
 * the most recent 65536 half steps).  Returns the number written (>= 0) or a
 * negative error.  Synchronises. */
MMX_API long long mmx_get_iter_log(mmx_ctx *ctx, int *host, long long cap);

/* Device pointer and element strides of an E or H field's storage (ids
 * 0-5): element (i, j, k) is at ptr[i + sx*j + sy*k] with elements of 8 (FP64)
 * or 4 (FP32) bytes.  Valid until the next mmx_step, which may move the field
 * to the context's second buffer set. */
MMX_API int mmx_get_field_device(mmx_ctx *ctx, int field_id, void **ptr, long long *sx, long long *sy);

/* Per-kernel timing, the counterpart of the per-routine profile of the
 * paper's Table 1 ("Evolve HM", "Evolve E"): while enabled, every kernel the
 * context launches is bracketed by CUDA events on the context stream.
 * mmx_get_profile synchronises, fills up to cap records (kernel name,
 * launches, total device milliseconds) and returns the number of kernel
 * kinds seen; reset = 1 clears the accumulated records afterwards. */
typedef struct {
    char name[32];
    long long launches;
    double total_ms;
} mmx_kernel_profile;

/* Discrete adjoint of the second-order scheme (Sec. 3.2: H/M half step,
 * E update with the time-centred split-field z-PML, H/M half step), for
 * grids without periodic axes, FP32 or FP64, soft sources only, no probes
 * or flux planes registered; with magnetic material, the second-order
 * scheme (order 2).  From the current state the context runs nsteps steps
 * (the per-update path), accumulating
 *   loss = sum_(n=1..nsteps) dt P(E^n, H^n)
 * with P the Poynting power through z node plane kp as in mmx_add_flux_plane,
 * then sweeps back through the steps, recomputing each checkpoint_every-step
 * segment from its checkpoint, and writes d loss / d eps_r of every cell
 * (host array of nx*ny*nz doubles, x fastest) to grad_eps, d loss / d H0
 * (the uniform bias of mmx_set_bias, host array of 3 doubles; zero without
 * magnetic material) to grad_h0 unless it is NULL, and the loss to *loss.
 * The magnetic half steps are transposed through their converged fixed
 * point (implicit-function adjoint of Eqs. llg_tra4-6 with N() and
 * Eq. iterate_H), solved by the same Jacobi sweep as the forward iteration
 * to a relative change of 1e-13 (FP64) or 1e-6 (FP32); a sweep that does not
 * get there within the forward's largest iteration count + 8 (at most
 * max_iter) returns MMX_ERR_NOT_CONVERGED.  The context ends advanced by
 * nsteps, as after mmx_step.  Device memory: about (nsteps/checkpoint_every
 * + checkpoint_every + 2) copies of the E/H(/M) state plus 22 grid arrays
 * and 63 magnetic-box arrays.  Synchronises the context stream.
 * MMX_ERR_INVALID for a context it does not cover, MMX_ERR_OOM when the
 * checkpoints do not fit. */
MMX_API int mmx_flux_gradient(mmx_ctx *ctx, int kp, int nsteps, int checkpoint_every, double *loss,
                              double *grad_eps, double *grad_h0);

/* FP16 storage scales: E is stored as E / sE and H (with its PML split part)
 * as H / sH, so that the fields of a problem sit inside FP16's range
 * (|value / scale| < 65504, full precision above 6.1e-5).  Defaults:
 * sH = 64 A/m, sE = 376.73 * sH V/m (the vacuum impedance times sH).  Only
 * for MMX_FP16 contexts, and only before any field value is set or any step
 * is taken (MMX_ERR_INVALID otherwise); both scales must be positive. */
MMX_API int mmx_set_storage_scale(mmx_ctx *ctx, double sE, double sH);

/* Point probes of E: the time series from which the paper's air-filled guide
 * analysis (Sec. 5.2.1) takes the Fourier transform of E on the guide's
 * central line.
 * mmx_add_probe registers E component `field` (0-2) at (i, j, k) within that
 * component's extent and returns the probe's index (0-15), or
 * MMX_ERR_INVALID (bad field or index, more than 16 probes).  Adding a probe
 * discards the samples recorded so far.  After every completed time step the
 * context appends one row of samples (E^(n+1) of every probe, converted to
 * double) to a device table of 65536 rows; later steps are not recorded
 * until the table is read with reset.  mmx_get_probes copies up to max_rows
 * rows, row-major (out[r * nprobe + p], row r = the r-th step since the last
 * reset), into the host array out, synchronises the context stream, clears
 * the table if reset is nonzero, and returns the number of rows copied (or a
 * negative error code). */
MMX_API int mmx_add_probe(mmx_ctx *ctx, int field, int i, int j, int k);
MMX_API long long mmx_get_probes(mmx_ctx *ctx, double *out, long long max_rows, int reset);

/* Discrete electromagnetic energy of the grid, in joules per the units of
 * the inputs: W = 1/2 sum_edges eps E^2 + 1/2 sum_faces mu (H^2 -
 * (dt/(2 mu) curl E)^2), the quantity the half-step leapfrog of Sec. 3.2
 * conserves exactly in lossless, source-free, non-magnetic media (mu = mu0
 * mu_r on non-magnetic faces, mu0 on magnetic faces; periodic duplicates
 * counted once).  Valid between mmx_step calls, where E and H share a time
 * level.  Summed in FP64 with Neumaier compensation whatever the storage
 * precision; synchronises the context stream. */
MMX_API int mmx_energy(mmx_ctx *ctx, double *out);

/* Poynting flux monitors.  mmx_add_flux_plane registers the z node plane k
 * (0 <= k <= nz; at most 4 planes) and returns its index.  After every time
 * step the context adds dt * P to the plane's accumulator, where
 * P = sum (Ex <Hy>_z - Ey <Hx>_z) dx dy is the power through the plane in
 * +z, each E edge paired with the mean of the two H faces above and below it
 * and H taken at the time level of E (on the fused path the mean of the two
 * half-step values, exact on non-magnetic faces outside the PML).  The sum
 * and the accumulation are FP64 with Neumaier compensation.
 * mmx_get_flux writes out[0] = the time-integrated flux (J) since the plane
 * was added or last reset and out[1] = P of the last step (W), synchronising
 * the context stream; reset = 1 then clears the accumulator. */
MMX_API int mmx_add_flux_plane(mmx_ctx *ctx, int k);
MMX_API int mmx_get_flux(mmx_ctx *ctx, int index, double out[2], int reset);

MMX_API int mmx_set_profiling(mmx_ctx *ctx, int enable);
MMX_API int mmx_get_profile(mmx_ctx *ctx, mmx_kernel_profile *out, int cap, int reset);

/* Batches: independent contexts (instances, e.g. the devices of a bias
 * sweep) advanced together.  Per time step one fused E/H launch covers every
 * instance's tiles and one cooperative H/M launch every instance's box
 * faces; each instance keeps its own iteration residual and stops at its
 * own first iterate below its tolerance (Sec. 3.2.2), and the launches of a
 * whole mmx_batch_step call are captured as one CUDA graph (re-captured when
 * the call length changes).
 * mmx_batch_create gathers count contexts (owned by the caller, which must
 * keep them alive and not step them through mmx_step while a batch call is
 * in flight).  All instances must share the precision and the PML /
 * conductive-or-permeable variant, have PEC x and y walls, no hard sources,
 * probes or flux planes, and fewer than 65536 cells along every axis, with
 * count at most 16384 (the batched magnetic-face list packs each face's
 * indices and instance into 8 bytes); otherwise MMX_ERR_INVALID (with *out
 * holding a batch
 * usable only with mmx_batch_last_error and mmx_batch_destroy).  Between
 * batch calls every instance can be read, written and stepped on its own.
 * cuda_stream is the batch's stream (NULL: the batch creates and owns a
 * non-blocking stream, since graph capture needs one); every launch of a
 * batch call, including each instance's per-call set-up, goes there, after
 * the work queued on the instances' own streams.
 * mmx_batch_set_planes sets the z planes each fused CTA marches (0: a whole
 * grid; the tuning knob of the batch).  mmx_batch_step enqueues nsteps steps
 * of every instance and returns; mmx_batch_sync waits, reports the first
 * instance error (or a batch-level timeout / non-finite value) and clears
 * the latched status words. */
typedef struct mmx_batch mmx_batch;
MMX_API int mmx_batch_create(mmx_ctx *const *ctxs, int count, void *cuda_stream, mmx_batch **out);
MMX_API int mmx_batch_set_planes(mmx_batch *b, int planes);
/* mmx_batch_set_box_blocks caps the cooperative H/M launch of a batch at
 * per_sm blocks of 256 threads per SM (0, the default: as many as are
 * resident, at most one per 256 faces).  Fewer blocks mean fewer arrivals at
 * each grid-wide vote and more faces per thread; the second tuning knob of
 * the batch.  MMX_ERR_INVALID for per_sm < 0. */
MMX_API int mmx_batch_set_box_blocks(mmx_batch *b, int per_sm);
MMX_API int mmx_batch_step(mmx_batch *b, int nsteps);
MMX_API int mmx_batch_sync(mmx_batch *b);
MMX_API const char *mmx_batch_last_error(mmx_batch *b);
MMX_API int mmx_batch_destroy(mmx_batch *b);

/* Edge or face mean of a cell-centred array with no memory allocation, for
 * callers that cannot call cudaMalloc: code whose device memory is all owned
 * by its own arena or pool, or that runs where an allocation (which may
 * synchronise the device) is not acceptable.  The paper has no counterpart;
 * the computation is the one mmx_get_material reads back.
 *   desc       only n[3] and bc[3] are used.
 *   location   0-2: mean over the edges of Ex, Ey, Ez (up to 4 cells);
 *              3-5: mean over the x, y, z faces (2 cells).
 *   cell       device array, nx*ny*nz doubles, x fastest (read).
 *   out        device array of n doubles, the edge/face extent (written).
 *   cuda_stream  cudaStream_t of the two kernel launches (NULL = default).
 * The padded intermediate lives in a fixed 8 MiB device array inside the
 * library (1,048,576 doubles; every GPU that loads the library holds it until
 * exit): grids with (round_up(nx+1, 8))(ny+1)(nz+1) > 1,048,576 or with
 * nz + 1 > 65535 return MMX_ERR_INVALID, as do bad arguments; MMX_ERR_CUDA
 * reports a failed launch of this call.
 * The first call on a device looks up that array's device address, so make it
 * before any stream capture; a call after the device's context was destroyed
 * and re-created (cudaDeviceReset) looks it up again.  All calls share the
 * array: calls whose kernels overlap on the GPU (other streams, other
 * threads) race.  Asynchronous: the result is ready when the stream has
 * finished. */
MMX_API int mmx_material_average_noalloc(const mmx_grid_desc *desc, int location, const double *cell,
                                         double *out, long long n, void *cuda_stream);

/* Message of the last error on this context (never NULL). */
MMX_API const char *mmx_last_error(const mmx_ctx *ctx);

/* Free all device memory of the context (synchronises its stream). */
MMX_API void mmx_destroy(mmx_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* MMX_H_ */

/*
 * vloc.h -- C ABI of the GB300 (sm_103a) local-potential action library.
 *
 * The library applies the local potential of a plane-wave Kohn-Sham
 * Hamiltonian to a block of wave functions (Gao, Mo, Fang & Wang,
 * arXiv:1601.07378, Sec. 2, Eqs. 2-3 and the two-FFT recipe after them):
 * each band's coefficients on the cut-off sphere are scattered onto the
 * n1 x n2 x n3 grid, transformed to real space by a compact 3-D FFT
 * (Sec. 4.3, Fig. 5: z-pass on the occupied sticks, y-pass on the planes
 * that meet them, x-pass on the whole grid), multiplied by the real V(r),
 * transformed back and gathered onto the sphere:
 *
 *     out = A c,   A = (1/N) S^T F- diag(V) F+ S,   N = n1 n2 n3,
 *
 * with S the scatter G -> grid point (h mod n1, k mod n2, l mod n3),
 * F+ the unnormalised transform with kernel exp(+2 pi i m.j / n) and
 * F- = F+^H.  (Eq. 2 as printed uses exp(-iG.r); that is the same operator
 * applied to the negated G-list.)
 *
 * Conventions for every entry point below:
 *  - Layouts.  Coefficients and outputs are band-major [nbands][npw], in the
 *    caller's G-list order, complex interleaved (re, im).  V and grad_V are
 *    real [n1][n2][n3] with i3 fastest.  Complex64 + float32 for a VLOC_F32
 *    plan, complex128 + float64 for a VLOC_F64 plan.
 *  - Pointers passed to the hot-path calls are device pointers aligned to
 *    their element size (8 B for complex64, 16 B for complex128, 4 or 8 B
 *    for the real V) unless stated otherwise.  out == coeffs (exact alias) is
 *    allowed; any other overlap between an input and an output is an error.
 *  - Ownership.  The caller owns every buffer it passes.  A plan owns its
 *    index tables, twiddles and workspace; no device memory is allocated by
 *    vloc_apply, vloc_apply_adjoint, vloc_backward or vloc_apply_batched.
 *  - Streams.  Work is enqueued on the caller's stream (a cudaStream_t passed
 *    as void*, NULL = legacy default stream) and the call returns without
 *    synchronising, except where stated.  A plan must not be used by two
 *    streams at the same time.
 *  - Errors.  Every int-returning call returns VLOC_OK (0) or a negative
 *    VLOC_ERR_* code; no exception crosses this boundary.  On error nothing
 *    has been enqueued unless the code is VLOC_ERR_CUDA.
 */
#ifndef VLOC_H
#define VLOC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes -------------------------------------------------------- */
#define VLOC_OK            0
#define VLOC_ERR_ARG      (-1)  /* null/misaligned pointer, bad count, overlap      */
#define VLOC_ERR_SIZE     (-2)  /* grid not 2/3/5-smooth, n < 2 or n > 256, too big  */
#define VLOC_ERR_GLIST    (-3)  /* duplicate G, index outside [-n/2, (n+1)/2 - 1]   */
#define VLOC_ERR_ALLOC    (-4)  /* device or host allocation failed                 */
#define VLOC_ERR_CUDA     (-5)  /* a CUDA runtime call failed                        */
#define VLOC_ERR_TIMEOUT  (-6)  /* a bounded device-side wait gave up                */
#define VLOC_ERR_STATE    (-7)  /* plan flags do not allow this call                 */

/* ---- plan flags ---------------------------------------------------------- */
#define VLOC_F32                0x001  /* complex64 data, FP32 arithmetic           */
#define VLOC_F64                0x002  /* complex128 data, FP64 arithmetic          */
#define VLOC_PARTITION_GREEDY   0x000  /* Sec. 3.2 sorted round-robin (default)     */
#define VLOC_PARTITION_BASIC    0x010  /* Sec. 4.1 cyclic row/column groups         */
#define VLOC_PARTITION_IMPROVED 0x020  /* Sec. 4.2 plane-sorted row/column groups   */
#define VLOC_GRAPH              0x100  /* replay apply chains as CUDA graphs: the    */
                                       /* first call with a given set of pointers   */
                                       /* and band count captures the launches into */
                                       /* a graph (kept per plan, 8 most recent),   */
                                       /* later calls replay it with one launch.    */
                                       /* Buffers must stay valid while cached.     */
#define VLOC_GENERIC_KERNELS    0x400  /* use the runtime-radix kernels for every   */
                                       /* axis (the compile-time-length kernels are */
                                       /* the default where one exists)             */
#define VLOC_GAMMA              0x1000 /* Gamma-point real mode (Sec. 4.3): g_hkl is */
                                       /* half of a G -> -G symmetric list (never    */
                                       /* both G and -G); coefficients c(-G) =      */
                                       /* conj c(G) are implied, c(0) is taken real; */
                                       /* bands are real in r-space and travel two  */
                                       /* per complex transform.  Apply / adjoint / */
                                       /* batched only.                             */
#define VLOC_DOUBLE_FLOAT       0x2000 /* with VLOC_F64: apply in double-float       */
                                       /* arithmetic (hi + lo FP32 pairs, ~48 bits,  */
                                       /* on the FP32 pipes); FP64 data in and out.  */
                                       /* Used when every axis length has compiled   */
                                       /* kernels (info.path bit 3), else native FP64*/
                                       /* (apply / adjoint / H / batched only).      */
#define VLOC_X_TMA              0x4000 /* FP32: x-pass by a persistent kernel whose  */
                                       /* slab tiles move by TMA tensor copies,      */
                                       /* double-buffered on mbarriers (compiled x   */
                                       /* length, even n3; info.path bit 4).  Same   */
                                       /* results bit for bit; measured slower than  */
                                       /* the default x-pass at 96^3, kept opt-in.   */
                                       /* Its waits are bounded: see                 */
                                       /* vloc_device_status.                        */
#define VLOC_Z_WARP             0x20000 /* FP32, n3 = 32, 64, 96 or 128, not Gamma: */
                                       /* z-passes as warp-register transforms (one */
                                       /* warp per stick pair, 32-point DFTs across */
                                       /* the lanes by warp shuffles; info.path bit */
                                       /* 8).  Measured slower than the tile z-      */
                                       /* passes on GB300, kept opt-in.             */
#define VLOC_Z_BULK             0x40000 /* FP32, every |l| <= n3/4, each stick's    */
                                       /* plane waves consecutive in the caller's   */
                                       /* list with l ascending: the inverse z-pass */
                                       /* stages each stick's coefficients by one   */
                                       /* 1-D bulk copy on an mbarrier (info.path   */
                                       /* bit 9).  Measured slower than the direct  */
                                       /* loads on GB300, kept opt-in.  Its wait is */
                                       /* bounded: see vloc_device_status.          */
#define VLOC_POISON_WORKSPACE   0x10000 /* test aid: fill the plan's cylinder and   */
                                       /* slab workspace with NaN bytes before every */
                                       /* workspace chunk, so a pass that reads a    */
                                       /* cell its chunk never wrote shows up as a   */
                                       /* non-finite result (slower; not for use)    */
#define VLOC_HOST_ONLY          0x200  /* build host tables only (no device memory, */
                                       /* no CUDA call); for introspection: the     */
                                       /* device calls then return VLOC_ERR_STATE   */

typedef struct vloc_plan_s* vloc_plan;

/* Plan information filled by vloc_get_info. */
typedef struct vloc_info {
    int32_t n1, n2, n3;          /* grid                                          */
    int32_t precision;           /* VLOC_F32 or VLOC_F64                          */
    int64_t npw;                 /* plane waves per band                          */
    int32_t nsticks;             /* occupied (h, k) z-sticks (the cylinder)       */
    int32_t nplanes;             /* occupied x-planes h (the cuboid)              */
    int32_t nparts;              /* stick parts (one z-pass CTA each)             */
    int32_t lines_per_tile;      /* FFT lines per CTA                             */
    int64_t chunk_bands;         /* bands per workspace chunk                     */
    int64_t workspace_bytes;     /* device workspace owned by the plan            */
    int32_t radix[3][4];         /* per-axis radix schedule (0 = unused)          */
    int32_t nstages[3];
    int32_t path;                /* bit 0: compile-time-length kernels enabled;   */
                                 /* bit 2: Gamma-point real mode;                 */
                                 /* bit 3: double-float FP64 apply in use;        */
                                 /* bit 4: TMA x-pass in use;                     */
                                 /* bit 5: the x-planes are the quarter-sphere    */
                                 /* set x = 0..n1/4, n1 - n1/4 .. n1 - 1, and the */
                                 /* x-pass kernels take them at compile time;     */
                                 /* bit 6: every |l| <= n3/4, and the z-pass       */
                                 /* kernels skip the rows outside that band;      */
                                 /* bit 7: Gamma-point pairs are formed and       */
                                 /* separated inside the z-passes (no pack pass); */
                                 /* bit 8: the z-passes run as warp-register      */
                                 /* transforms (VLOC_Z_WARP);                     */
                                 /* bit 9: the inverse z-pass stages each stick's */
                                 /* coefficients by one bulk copy (VLOC_Z_BULK)   */
} vloc_info;

/*
 * vloc_plan_create -- build a plan for one grid and one G-list.
 * Sec. 2 Eqs. 2-3 (which plane waves exist), Sec. 3.2 / Fig. 2 (stick
 * workloads and the greedy sorted round-robin partition, here dealing
 * z-sticks to z-pass thread blocks), Sec. 4.3 / Fig. 5 (cylinder and cuboid
 * supports).
 *   out        : receives the plan handle (host pointer, not null).
 *   n1, n2, n3 : grid, each 2..256 and 2/3/5-smooth.
 *   g_hkl      : HOST pointer, npw x 3 int32 Miller indices (h, k, l), each
 *                in [-(n/2), (n+1)/2 - 1]; no duplicates.  Copied; the caller
 *                may free it after the call.
 *   npw        : number of plane waves, >= 1.
 *   flags      : exactly one of VLOC_F32 / VLOC_F64, optionally one
 *                partition flag, VLOC_GRAPH, VLOC_HOST_ONLY,
 *                VLOC_GENERIC_KERNELS, VLOC_GAMMA, VLOC_DOUBLE_FLOAT (with
 *                VLOC_F64 only, else VLOC_ERR_ARG) and VLOC_X_TMA.  With VLOC_GAMMA every
 *                -G must be a valid index too (else VLOC_ERR_GLIST), and
 *                npw counts the half list (the caller's arrays).
 *   max_bands_per_chunk : bands per workspace chunk (<= 0: automatic, a
 *                6 GiB workspace capped at 1/16 of the free device memory
 *                and at 2048 bands; large chunks keep every kernel many
 *                waves deep).
 *   stream     : stream used for the one-time table uploads (synchronised
 *                before return).
 * Errors: VLOC_ERR_ARG, VLOC_ERR_SIZE, VLOC_ERR_GLIST, VLOC_ERR_ALLOC,
 * VLOC_ERR_CUDA.  Must be called with the target device current.
 */
int vloc_plan_create(vloc_plan* out, int n1, int n2, int n3, const int32_t* g_hkl, int64_t npw,
                     int flags, int64_t max_bands_per_chunk, void* stream);

/*
 * vloc_plan_set_schedule -- replace the radix schedule of one axis (0: n1,
 * 1: n2, 2: n3) of a plan: nst stages (1..4) with radices from
 * {2,3,4,5,6,8,9,10,12,15,16} whose product is that axis's length.  The
 * plan then runs the runtime-radix kernels (the compile-time-length kernels
 * have their schedule built in).  Used by the autotuner.  Not while the plan
 * has work in flight.  Errors: VLOC_ERR_ARG (bad axis, radix or product).
 */
int vloc_plan_set_schedule(vloc_plan plan, int axis, int nst, const int32_t* radix);

/* vloc_plan_destroy -- free the plan's device and host memory (synchronises
 * the device first).  NULL is accepted.  Returns VLOC_OK or VLOC_ERR_CUDA. */
int vloc_plan_destroy(vloc_plan plan);

/*
 * vloc_apply -- out = A c for nbands bands (Sec. 2: G->r FFT, multiply by
 * V_loc(r), r->G FFT; compact passes of Sec. 4.3).
 *   coeffs : device [nbands][npw] complex.   V : device [n1][n2][n3] real.
 *   out    : device [nbands][npw] complex (may equal coeffs).
 *   nbands : >= 0 (0 is a no-op).
 * Errors: VLOC_ERR_ARG (null/misaligned pointer, nbands < 0, partial
 * overlap), VLOC_ERR_CUDA.
 */
int vloc_apply(vloc_plan plan, const void* coeffs, const void* V, int64_t nbands, void* out,
               void* stream);

/*
 * vloc_apply_h -- out = (diag(d) + A) c: the local-potential action plus a
 * term diagonal in G, added in the gather of the last kernel (for a
 * Kohn-Sham Hamiltonian d(G) = |k + G|^2 / 2, the kinetic energy, Eq. 1).
 *   diag : device real [npw] (plan precision), in the caller's G order; NULL
 *          gives vloc_apply.  Must not overlap out.
 * Other arguments, aliasing and errors as vloc_apply (Gamma-point plans
 * included: d is given on the half list).
 */
int vloc_apply_h(vloc_plan plan, const void* coeffs, const void* V, const void* diag, int64_t nbands,
                 void* out, void* stream);

/* vloc_apply_adjoint -- out = A^H c.  With real V the operator is Hermitian
 * (A^H = A), so this is the same action; it is a separate entry so that the
 * operator contract used by the backward pass is explicit.  Arguments and
 * errors as vloc_apply. */
int vloc_apply_adjoint(vloc_plan plan, const void* coeffs, const void* V, int64_t nbands,
                       void* out, void* stream);

/*
 * vloc_backward -- gradients of a real loss L through out = A c.
 * grad_out holds dL/dRe(out) + i dL/dIm(out) (PyTorch's convention).
 *   grad_coeffs (nullable) = A^H grad_out = A grad_out.
 *   grad_V      (nullable, overwritten, real [n1][n2][n3]) =
 *       (1/N) sum_n Re( conj(F+ S grad_out_n) * F+ S c_n ),
 *   with psi_n = F+ S c_n recomputed band by band (no grid is stored).
 *   The band sum runs in groups of at most 16 bands (FP32 sums in the FP32
 *   path, FP64 in the FP64 path) whose partial sums are added in FP64 in a
 *   fixed order, so the result is deterministic.
 * Errors as vloc_apply; VLOC_ERR_STATE for a VLOC_GAMMA plan; VLOC_ERR_SIZE
 * when the dL/dV x-pass does not fit in shared memory (FP64, n1 > ~170).
 */
int vloc_backward(vloc_plan plan, const void* coeffs, const void* grad_out, const void* V,
                  int64_t nbands, void* grad_coeffs, void* grad_V, void* stream);

/*
 * vloc_to_real -- the G -> r half of the action on its own (Sec. 2, the
 * first FFT of the two-FFT recipe): psi_n = F+ S c_n on the full grid, the
 * unnormalised e^{+} transform through the same compact z- and y-passes.
 *   coeffs : device [nbands][npw] complex.
 *   psi    : device [nbands][n1][n2][n3] complex, i3 fastest (written).
 * No overlap between the two.  Not for VLOC_GAMMA plans (VLOC_ERR_STATE).
 * Errors as vloc_apply.
 */
int vloc_to_real(vloc_plan plan, const void* coeffs, int64_t nbands, void* psi, void* stream);

/*
 * vloc_to_recip -- the r -> G half on its own (the second FFT of the
 * recipe): out_n(G) = (1/N) sum_r u_n(r) e^{-2 pi i G.r/n} at the plan's G,
 * through the output-pruned x-pass, the y-pass and the z-pass + gather.
 *   u   : device [nbands][n1][n2][n3] complex (read only).
 *   out : device [nbands][npw] complex (written).
 * to_recip(to_real(c)) = c.  Not for VLOC_GAMMA plans.  Errors as vloc_apply.
 */
int vloc_to_recip(vloc_plan plan, const void* u, int64_t nbands, void* out, void* stream);

/*
 * vloc_density -- the charge density of Sec. 3.1, rho(r) = sum_n f_n
 * |psi_n(r)|^2 with psi_n = F+ S c_n (unnormalised transform).
 *   coeffs : device [nbands][npw] complex (the half list for VLOC_GAMMA
 *            plans, whose bands are real: two travel per complex transform).
 *   occ    : device [nbands] real weights f_n, or NULL for f_n = 1.
 *   rho    : device real [n1][n2][n3], overwritten.
 * The band sum runs as in vloc_backward (groups of at most 16 bands, their
 * partial sums added in FP64 in a fixed order): deterministic.  No grid is
 * stored.  nbands = 0 writes zeros.
 * Errors as vloc_apply; VLOC_ERR_SIZE when the density x-pass does not fit
 * in shared memory (FP64, n1 > ~170).
 */
int vloc_density(vloc_plan plan, const void* coeffs, const void* occ, int64_t nbands, void* rho,
                 void* stream);

/*
 * vloc_apply_batched -- ninst independent applies (plans of different grids
 * and spheres).  Without VLOC_GRAPH they are enqueued back to back on the
 * stream.  When every plan has VLOC_GRAPH the whole batch is captured once
 * (per pointer set) into one CUDA graph whose instances run as up to four
 * parallel branches (instances sharing a plan share a branch), and each
 * call is one graph launch.  Arrays have ninst entries each; plans must
 * share a precision.  Errors as vloc_apply, per instance.
 */
int vloc_apply_batched(int ninst, const vloc_plan* plans, const void* const* coeffs,
                       const void* const* V, const int64_t* nbands, void* const* out,
                       void* stream);

/*
 * vloc_apply_host -- vloc_apply with HOST buffers: copies the coefficients
 * and V to the device in chunks, applies, and copies the result back,
 * overlapping copies with compute on the plan's copy stream.  Pinned host
 * memory gives asynchronous copies.  Synchronises `stream` before return.
 * The first call allocates the plan's staging buffers (once).
 * Errors: VLOC_ERR_ARG, VLOC_ERR_ALLOC, VLOC_ERR_CUDA.
 */
int vloc_apply_host(vloc_plan plan, const void* coeffs_host, const void* V_host, int64_t nbands,
                    void* out_host, void* stream);

/*
 * vloc_apply_host_async -- vloc_apply_host without the synchronisation: the
 * copies and the applies are enqueued and the call returns; `stream` is made
 * to wait for the last copy out, so the results are in out_host once the
 * caller's stream has reached that point (synchronise it before reading
 * them).  coeffs_host, V_host and out_host must stay untouched until then.
 * Consecutive calls on one plan overlap one call's last copies with the
 * next call's first (the staging slots' state carries over), which is how a
 * stream of band blocks keeps the host link busy.  Pinned host memory is
 * required for the copies to be asynchronous.  Same errors as
 * vloc_apply_host.
 */
int vloc_apply_host_async(vloc_plan plan, const void* coeffs_host, const void* V_host, int64_t nbands,
                          void* out_host, void* stream);

/* vloc_get_index_map -- grid_index[p] = ((h mod n1) n2 + (k mod n2)) n3 +
 * (l mod n3) for every G of the plan's list (host array of npw int64).
 * Eqs. 2-3. */
int vloc_get_index_map(vloc_plan plan, int64_t* grid_index);

/* vloc_get_partition -- stick_part[s] = part (z-pass thread block) of the
 * s-th occupied stick, sticks in ascending (h mod n1) n2 + (k mod n2) order
 * (host array of nsticks int32); *nparts_out receives the number of parts.
 * Sec. 3.2 / Fig. 2 (or Sec. 4.1 / 4.2 with the partition flags). */
int vloc_get_partition(vloc_plan plan, int32_t* stick_part, int32_t* nparts_out);

/* vloc_get_info -- fill *info (host pointer). */
int vloc_get_info(vloc_plan plan, vloc_info* info);

/*
 * vloc_apply_noalloc -- vloc_apply that allocates nothing.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- code running while another runtime owns the device's memory
 * (a framework that reserves the GPU up front and forbids outside
 * allocations), or a process that must not allocate after start-up.
 * Instead of the plan's workspace it uses one fixed scratch array compiled
 * into the library: 48 MiB of device memory per GPU that loads the library,
 * held until the process exits.  The index tables and twiddles are rebuilt
 * in that array on every call from the plan's host-side data (a block the
 * plan keeps unchanged until it is destroyed), so `plan` may be a
 * VLOC_HOST_ONLY plan (which made no CUDA call at all); together the two
 * never allocate device memory.  The caller passes inputs and outputs as
 * for vloc_apply (same layouts, alignment, alias and overlap rules).
 *   Kernels: the plan's own choice -- compile-time-length or runtime-radix
 *   kernels (VLOC_GENERIC_KERNELS, vloc_plan_set_schedule), and the
 *   double-float kernels for a VLOC_DOUBLE_FLOAT plan.
 *   Not for VLOC_GAMMA plans: they return VLOC_ERR_STATE before any CUDA
 *   call is made.
 *   Limit: the tables, twiddles (for a double-float plan also V as hi + lo
 *   pairs, 8 bytes per grid point) and the workspace of at least one band
 *   must fit in the 48 MiB (index tables at most 8 MiB); otherwise the call
 *   returns VLOC_ERR_SIZE before doing any device work.  Bands are
 *   processed in chunks that fit.
 *   Set-up: the first call on each device looks up the array's device
 *   address (with that device current); make that first call before any
 *   stream capture.
 *   Sharing: every call uses the same array and leaves its contents behind;
 *   nothing in it needs to start at zero.  Calls that overlap on the GPU
 *   (different streams, or interleaved work from several host threads) race
 *   on the array and must be serialised by the caller.
 * Errors: VLOC_ERR_ARG, VLOC_ERR_SIZE, VLOC_ERR_STATE (Gamma plan),
 * VLOC_ERR_CUDA.
 */
int vloc_apply_noalloc(vloc_plan plan, const void* coeffs, const void* V, int64_t nbands, void* out,
                       void* stream);

/* ---- tracing --------------------------------------------------------------
 * Per-kernel timing with CUDA events recorded on the launching stream around
 * every kernel of a plan's calls, for the roofline and profile reports.
 * Kernel slots: 0 scatter + inverse z-pass, 1 inverse y-pass, 2 x-pass with
 * V(r), 3 forward y-pass, 4 forward z-pass + gather, 5 dL/dV x-pass,
 * 6 auxiliary (zero / convert / reduce), 7 Gamma-point pack / unpack,
 * 8 inverse x-pass to a full grid, 9 forward x-pass from a full grid,
 * 10 density x-pass, 11 unused. */
#define VLOC_NKERNELS 12
typedef struct vloc_kernel_stat {
    int64_t launches;
    double total_ms;
} vloc_kernel_stat;

/* vloc_profile -- enable (1) or disable (0) per-launch event timing and clear
 * the recorded launches.  Timing costs two event records per launch. */
int vloc_profile(vloc_plan plan, int enable);

/* vloc_get_profile -- synchronise on the recorded events, fill
 * stats[VLOC_NKERNELS] (host array) with launches and summed device time per
 * kernel slot since the last vloc_profile / vloc_get_profile, then clear. */
int vloc_get_profile(vloc_plan plan, vloc_kernel_stat* stats);

/* vloc_get_launch_count -- kernels launched by this plan since creation
 * (always counted, profiling or not). */
int vloc_get_launch_count(vloc_plan plan, int64_t* count);

/* vloc_device_status -- synchronise the device and report whether a kernel
 * of this plan gave up a bounded wait since the last call (a bulk copy that
 * did not land within about a second): VLOC_ERR_TIMEOUT (and the flag is
 * cleared), else VLOC_OK.  Results of the affected calls are undefined. */
int vloc_device_status(vloc_plan plan);

/* ---- measurement aids ----------------------------------------------------
 * The paper has no counterpart.  The FP64 chain is bound by the GPU's FP64
 * rate and the double-float chain by its FP32 pipe, so their roofline
 * fractions divide by arithmetic ceilings measured with these probes rather
 * than nominal figures. */
#define VLOC_PEAK_DFMA   0  /* FP64 fused multiply-add (2 flops)               */
#define VLOC_PEAK_DADD   1  /* FP64 add (1 flop)                               */
#define VLOC_PEAK_FFMA   2  /* FP32 fused multiply-add (2 flops)               */
#define VLOC_PEAK_FFMA2  3  /* paired FP32 fused multiply-add (4 flops)        */
#define VLOC_PEAK_FADD2  4  /* paired FP32 add (2 flops)                       */
#define VLOC_PEAK_NKINDS 5
/*
 * vloc_alu_peak -- run one probe kernel of `kind`: 8 blocks of 256 threads
 * per SM, each thread 16 independent dependent chains of `iters` steps of
 * that one instruction; timed with CUDA events on `stream` (synchronises).
 *   sink  : device pointer to one double (never written in practice; keeps
 *           the chains live).
 *   flops : receives the floating-point operations the launch performed.
 *   ms    : receives the launch's event time in milliseconds.
 * Errors: VLOC_ERR_ARG (bad kind, iters <= 0, null pointer), VLOC_ERR_CUDA.
 */
int vloc_alu_peak(int kind, int64_t iters, void* sink, double* flops, double* ms, void* stream);

/* vloc_strerror -- static string for a return code (never NULL). */
const char* vloc_strerror(int code);

/* vloc_version -- library version, major*10000 + minor*100 + patch. */
int vloc_version(void);

/* vloc_last_cuda_error -- text of the last CUDA error seen by this thread in
 * a call that returned VLOC_ERR_CUDA or VLOC_ERR_ALLOC ("" if none). */
const char* vloc_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VLOC_H */

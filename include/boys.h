/*
 * libboys — batched Boys-function evaluation on NVIDIA GB300 (sm_103a).
 *
 * Implements the evaluation algorithm of Vikhamar-Sandberg & Repisky,
 * "Efficient Boys function evaluation using minimax approximation"
 * (arXiv:2512.10059): Section II.C / Eq. 3 define
 *     F_k(x) = \int_0^1 t^{2k} e^{-x t^2} dt,  x >= 0,
 * and Algorithm 1 evaluates F_0..F_kmax by splitting [0, inf) into
 *     A = [0, x_0)   rational minimax anchor r_{A,kmax}, downward recurrence
 *     B = [x_0, x_1) rational minimax r_B for F_0, upward recurrence
 *     C = [x_1, inf) asymptotic F_0 = sqrt(pi)/2 x^{-1/2}, upward recurrence
 * with x_0, x_1 and all FP64 coefficients from the paper's Appendix D
 * (eps_tol = 5e-14 absolute for every order k <= 32).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Array pointers are DEVICE pointers (CUDA global memory) owned by the
 *    caller; the library never frees or retains them beyond the call.
 *  * `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every compute entry point only enqueues work on it and
 *    returns; results are ready when the stream reaches that point.
 *  * Output layout is order-major ("SoA"): F_k(x_i) is stored at
 *    out[k * ld + i], 0 <= k <= kmax, 0 <= i < n, with ld >= n.  Offsets
 *    are 64-bit.
 *  * Argument errors are reported synchronously by the return value and
 *    enqueue nothing.  n == 0 is a no-op that returns BOYS_OK.
 *  * Domain conventions (the paper defines x >= 0 only): x < 0 or NaN
 *    gives NaN for every order; x = +inf gives 0; -0.0 is treated as 0.
 *    These are not errors (detecting them would need a synchronisation).
 *  * Launch failures return BOYS_ERR_CUDA; boys_last_error() then holds
 *    the CUDA error text for the calling thread.
 */
#ifndef LIBBOYS_BOYS_H
#define LIBBOYS_BOYS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum boys_status {
    BOYS_OK = 0,
    BOYS_ERR_INVALID_ARG = 1, /* NULL pointer, n < 0, ld < n, size overflow  */
    BOYS_ERR_KMAX = 2,        /* kmax outside the range the entry point supports */
    BOYS_ERR_ALIGNMENT = 3,   /* pointer not aligned to its element size      */
    BOYS_ERR_CUDA = 4         /* a CUDA runtime call or launch failed          */
} boys_status;

/* Human-readable name of a status code (static string, never NULL). */
const char* boys_status_string(int status);

/* Text of the last BOYS_ERR_* raised on the calling thread ("" if none). */
const char* boys_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int boys_version(void);

/* Highest kmax accepted by the FP64 entry points (32, the paper's table set). */
int boys_kmax_limit(void);

/*
 * Diagnostic (no counterpart in the paper): applies one of the library's own
 * FP64 elementary functions elementwise, out[i] = f(a[i]):
 *   fn 0: e^{-a} (0 <= a <= 700)  1: 1/a  2: b[i]/a  3: a^{-1/2}   (a normal)
 *   fn 4: e^{-a} on the integer pipes (0 <= a < 32), rounded to nearest double
 *   fn 5: a^{-1/2} on the integer pipes (a normal), rounded to nearest double
 * so that their accuracy can be measured against CUDA's functions.
 */
boys_status boys_diag_math(int fn, const double* a, const double* b, int64_t n, double* out, void* stream);

/*
 * FP64 stored mode — Algorithm 1 for every x_i.
 *   x    [n]            input arguments (8-byte aligned)
 *   n                   number of arguments, n >= 0
 *   kmax                highest order, 0 <= kmax <= 32
 *   out  [kmax+1][ld]   F_k(x_i) at out[k*ld + i]; ld >= n
 * Accuracy: |F_k - exact| <= 5e-14 absolute for every k (the paper's
 * eps_tol; at x = x_1 exactly the asymptotic form's own error exceeds it by
 * ~1e-29, see the design notes).  Results are bitwise deterministic.
 */
boys_status boys_eval(const double* x, int64_t n, int kmax, double* out, int64_t ld,
                      void* stream);

/*
 * FP64 stored mode on HOST buffers: x and out live in host memory that the
 * GPU can address (pinned with cudaHostAlloc / cudaHostRegister, or pageable
 * memory on systems with pageable-memory access).  The evaluation kernel
 * reads x and writes F over the host link itself (on GB300: NVLink-C2C, ~210
 * GB/s in, ~193 GB/s out, the same as copy engines reach), so no staging
 * buffer, copy or device allocation is involved.  Same arguments, layout and
 * results as boys_eval; asynchronous on `stream`; a buffer the GPU cannot
 * address returns BOYS_ERR_INVALID_ARG.
 */
boys_status boys_eval_host(const double* x, int64_t n, int kmax, double* out, int64_t ld, void* stream);

/*
 * FP64 fused consumer — the F_k never leave the SM (registers and 16 KB of
 * shared memory per 128-thread block at kmax 32):
 *   out[i] = sum_{k=0}^{kmax} (-2 rho_i)^k F_k(x_i)
 * (the McMurchie-Davidson-style scaling of an electron-repulsion-integral
 * kernel; the F_k are evaluated as boys_eval does, to the same accuracy).
 * The sum is formed as two Horner sums in a = -2 rho joined by a^(kmax/2+1),
 * so |2 rho|^(kmax/2+1) must be finite in double precision.
 *   x, rho [n] inputs; out [n] output; 0 <= kmax <= 32.
 */
boys_status boys_eval_fused(const double* x, const double* rho, int64_t n, int kmax,
                            double* out, void* stream);

/*
 * FP32 tier: Algorithm 1 in single precision with this library's own rational
 * minimax tables (generated by a rational Remez code in extended precision,
 * Section II.B, degrees chosen from the Walsh table as in Section II.D), one
 * set per kmax: x0(kmax) from Eq. x0, x1(kmax) from Eq. x1 with a 3e-7
 * asymptotic budget.  Absolute accuracy 1e-6 for every order against the
 * exact F_k at the (float) input.  x float [n]; out float [kmax+1][ld];
 * 0 <= kmax <= 32.  Alignment and kmax choose the access width, never the
 * results: below kmax 8, 16-byte aligned x and out with ld % 4 == 0 give
 * 128-bit accesses (four arguments per thread); otherwise 8-byte aligned x
 * and out with even ld give 64-bit accesses (two per thread); anything else
 * 32-bit accesses.
 */
boys_status boys_eval_f32(const float* x, int64_t n, int kmax, float* out, int64_t ld, void* stream);

/*
 * Backward pass: dF_k/dx = -F_{k+1} (Eq. 3 differentiated under the integral
 * sign), so for upstream gradients g_k = dL/dF_k
 *   dx[i] = -sum_{k=0}^{kmax} g[k*ldg + i] * F_{k+1}(x_i).
 * F_0..F_{kmax+1} are re-evaluated in-kernel at order kmax+1, hence
 * 0 <= kmax <= 31.  x [n], g [kmax+1][ldg] (ldg >= n), dx [n] (overwritten).
 */
boys_status boys_grad(const double* x, int64_t n, int kmax, const double* g, int64_t ldg,
                      double* dx, void* stream);

/*
 * Ragged batches — many segments with their own kmax in ONE persistent
 * launch (e.g. the shell quartets of an ERI batch, kmax_s = la+lb+lc+ld).
 *   x        [total]    all arguments, segment s owning x[seg_off[s] .. seg_off[s+1])
 *   seg_off  [nseg+1]   int64, seg_off[0] = 0, non-decreasing (empty segments allowed)
 *   seg_kmax [nseg]     int32 in [0, 32]
 *   out_off  [nseg]     int64 element offset of segment s's output block
 *   out                 F_k(x[seg_off[s] + j]) at out[out_off[s] + k*len_s + j],
 *                       len_s = seg_off[s+1] - seg_off[s]  (an order-major block)
 *   workspace           device scratch owned by the caller, 16-byte aligned, of
 *                       workspace_bytes >= boys_ragged_workspace_size() (256);
 *                       calls that share a workspace must not overlap on the GPU.
 *                         * 256 bytes: one persistent launch over flat tiles,
 *                           taking tiles from a work counter in the workspace;
 *                         * boys_ragged_workspace_size_grouped(nseg, total)
 *                           bytes (more than 528 in general): the kmax-grouped
 *                           shape of a plan without a plan.  The call builds a
 *                           table of tiles (up to 128 arguments of one segment)
 *                           grouped by kmax in the workspace on the device,
 *                           then launches one kernel per kmax.  If the table
 *                           exceeds a smaller workspace (any size of at least
 *                           528 bytes selects this shape), those kernels do
 *                           nothing and a persistent launch runs instead.
 *                       Either way everything is enqueued on `stream` with no
 *                       synchronisation (about 38 launches for the grouped shape).
 * Every argument is evaluated by the same code as boys_eval at its segment's
 * kmax, so results are bitwise identical to per-segment boys_eval calls, for
 * either shape.  Descriptors live on the device and are not validated on the
 * host; a non-empty segment whose kmax is outside [0, 32] is skipped and
 * flags the workspace (see boys_ragged_status).
 */
size_t boys_ragged_workspace_size(void);
/* Workspace bytes for the kmax-grouped shape of nseg segments holding `total`
 * arguments in all (0 for negative arguments). */
size_t boys_ragged_workspace_size_grouped(int32_t nseg, int64_t total);
boys_status boys_eval_ragged(const double* x, const int64_t* seg_off, const int32_t* seg_kmax,
                             int32_t nseg, double* out, const int64_t* out_off, void* workspace,
                             size_t workspace_bytes, void* stream);

/* Reads the error word of a ragged workspace after the stream's work so far
 * (synchronises `stream`): *bad_kmax = 1 if a segment had kmax outside [0, 32]. */
boys_status boys_ragged_status(const void* workspace, int* bad_kmax, void* stream);

/*
 * Ragged plan: fixes the buffers and descriptors of a ragged batch, picks the
 * launch shape and captures it into a CUDA graph; boys_ragged_plan_launch then
 * replays it with one cudaGraphLaunch.  Shapes: the persistent kernel (block
 * size 64/128/256, 1 or 2 arguments per thread, 1 or 2 resident waves), or
 * waves = 0: one kernel per kmax present, each over a table of tiles of
 * `block` arguments built at creation, as parallel branches of the graph.
 * Every shape gives the same bits.  Creation reads the descriptors back (it
 * synchronises the device), validates them (seg_off[0] = 0, non-decreasing,
 * kmax in [0, 32]) and allocates a 256-byte workspace, and for waves = 0 the
 * tile table (16 bytes per tile), that the plan owns.
 *   flags & BOYS_PLAN_AUTOTUNE      time every candidate shape on these very
 *                                   buffers (outputs are overwritten) and
 *                                   keep the fastest; results are cached per
 *                                   device/driver/library/workload key in
 *                                   memory and, if the environment variable
 *                                   BOYS_AUTOTUNE_CACHE names a file, on disk.
 *   flags & BOYS_PLAN_FORCE_CONFIG  take the shape from BOYS_FORCE_CONFIG =
 *                                   "block,xpt,waves" (for tests; waves 0
 *                                   selects the per-kmax launches).
 * Without flags the default shape (128, 1, 1) is used.
 */
#define BOYS_PLAN_AUTOTUNE 1
#define BOYS_PLAN_FORCE_CONFIG 2
typedef struct boys_ragged_plan boys_ragged_plan;
boys_status boys_ragged_plan_create(const double* x, const int64_t* seg_off, const int32_t* seg_kmax,
                                    int32_t nseg, double* out, const int64_t* out_off, int flags,
                                    boys_ragged_plan** plan);
boys_status boys_ragged_plan_launch(boys_ragged_plan* plan, void* stream);
boys_status boys_ragged_plan_config(const boys_ragged_plan* plan, int* block, int* xpt, int* waves);
void boys_ragged_plan_destroy(boys_ragged_plan* plan);

/*
 * The paper's benchmark workload (Section III, Algorithm 2):
 *   z[i] = sum_{l=0}^{k} c[l] * sum_{j=0}^{n-1} F_l(x[i] + x[j]) * y[j]
 * for every i, F_l by the three-region Algorithm 1 in FP64 accuracy.
 *   x, y, z [n]; c [k+1]; 0 <= k <= 32; n <= 2^40.
 * Work is n^2 (k+1) evaluations.  Sorting x ascending (permuting y alongside)
 * keeps each warp's arguments in one region and is several times faster; the
 * result is the same up to summation rounding.
 */
boys_status boys_pairwise(const double* x, const double* y, int64_t n, const double* c, int k, double* z,
                          void* stream);

/*
 * Ragged batch that allocates nothing.  The paper has no counterpart; this is
 * for callers that cannot provide device memory of their own, e.g. code that
 * must not call cudaMalloc because a framework or an application's fixed
 * memory budget owns every device allocation, or a latency-critical loop that
 * cannot take cudaMalloc's implicit synchronisation.  Same arguments, layout
 * and results as boys_eval_ragged, without the workspace: the persistent
 * kernel's scratch (a 16-byte tile counter and error word) lives in a 256-byte
 * array inside the library's device image, held by every GPU that loads the
 * library until the process exits.  The scratch need does not grow with nseg
 * or the argument count, so no call exceeds the array (the check is kept).
 *  * The first call on each device, with that device current, looks up the
 *    array's device address (cudaGetSymbolAddress, which may load the
 *    library's device code).
 *  * Every call on a device shares the one array and re-zeroes its counter on
 *    `stream` first: calls that overlap on the GPU (other streams, other host
 *    threads) race with each other and produce wrong output.
 *  * No cudaMalloc, cudaFree or other allocating routine is called.
 *  * A segment whose kmax is outside [0, 32] is skipped (its output block is
 *    left as it was) and sets the array's error word, which the next call
 *    clears; boys_ragged_noalloc_status reads it.
 */
boys_status boys_eval_ragged_noalloc(const double* x, const int64_t* seg_off, const int32_t* seg_kmax,
                                     int32_t nseg, double* out, const int64_t* out_off, void* stream);

/* Error word of the latest boys_eval_ragged_noalloc call on the current
 * device, read after the work enqueued on `stream` so far (synchronises
 * `stream`; copies 8 bytes from the static array, allocates nothing):
 * *bad_kmax = 1 if a segment had kmax outside [0, 32], else 0.  Like the
 * evaluation itself it has no counterpart in the paper. */
boys_status boys_ragged_noalloc_status(int* bad_kmax, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LIBBOYS_BOYS_H */

/*
 * lmg.h -- C ABI of the least-misfit gridding library for GB300 (sm_103a).
 *
 * Method: Ye, Gull, Tan & Nikolic, "Optimal gridding and degridding in radio
 * interferometry imaging", MNRAS 2019 (arXiv:1906.07102). Section and equation numbers
 * below refer to that paper (equations numbered in order of appearance: Eq. 3 DFT dirty
 * image, Eq. 4 FFT dirty image, Eq. 5 gridding sum, Eq. 6 support set, Eq. 8 misfit
 * bound, Eq. 11 map error, Eq. 12/15 optimal correction, Eq. 16 integrated misfit,
 * Eqs. 17-19 the linear system for C).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Visibility positions uv are float64 pairs (u, v) in wavelengths, array [nvis][2].
 *    They are converted to grid cells by the float64 product u_cells = u * (N * pixel_scale)
 *    (Section 2.1: u' = u L with the FFT field L = N * pixel_scale radians).
 *  - x0 is the kept fraction of the FFT image width: the image has n_image pixels per
 *    side and the grid N = n_image / x0 cells (N must be an even integer). The paper's
 *    x0 (half width of the kept field in normalised coordinates) is x0 / 2.
 *  - Grid arrays are [N][N] complex, row = v, column = u, index i = n + N/2 for the grid
 *    coordinate n in [-N/2, N/2) (Eq. 4); support points outside wrap modulo N.
 *  - Images are [n_image][n_image] complex, pixel p at x = (p - n_image/2) / N.
 *  - Imaging uses exp(+i 2 pi n x) with no normalisation (Eqs. 3-4); prediction uses
 *    exp(-i 2 pi (u l + v m)) (Eq. 2). Weights are real; NULL means all ones.
 *  - dtype LMG_C64: complex64 data, float32 table and float32 arithmetic;
 *    dtype LMG_C128: complex128 data, float64 table and float64 arithmetic.
 *  - Complex arrays are interleaved (re, im) pairs. Grids ([N][N] arrays that the sweeps
 *    and transforms read or write) are 16-byte aligned (16-byte vector accesses); images
 *    and visibility arrays are aligned to their element (8 bytes C64, 16 bytes C128),
 *    weights to theirs (4 or 8 bytes), uv arrays to 16 bytes. A call given a misaligned
 *    array returns LMG_EINVAL and does nothing. All data pointers are DEVICE pointers
 *    owned by the caller unless a parameter says "host". The library owns only the
 *    opaque table and plan objects (and the device buffers inside a plan); free them
 *    with lmg_*_free.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream). Every call
 *    that takes a stream only enqueues work and returns without synchronising, except
 *    where a comment says otherwise.
 *  - Positions that are not finite or lie 2^30 or more cells from the origin are dropped
 *    (they contribute nothing when gridding and are predicted as 0); lmg_plan_dropped
 *    reports how many were dropped by the last binning.
 *  - The support rule (Eq. 6): a position u (cells) is quantised to 2^-32 cell (round
 *    half to even) and covers the W grid points n_start .. n_start+W-1 with
 *    n_start = ceil(u - W/2); its table coordinate is s = n_start - (u - W/2) in [0, 1).
 *
 * Errors: every function returns LMG_OK (0) or a negative lmg_status; no call throws or
 * aborts. lmg_last_error() returns a message for the calling thread's last failure.
 */
#ifndef LMG_H
#define LMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LMG_OK = 0,
  LMG_EINVAL = -1,        /* invalid argument (range, null pointer, size) */
  LMG_ENOMEM = -2,        /* host or device allocation failed */
  LMG_ECUDA = -3,         /* a CUDA runtime call or kernel launch failed */
  LMG_ECUFFT = -4,        /* a cuFFT call failed */
  LMG_EUNSUPPORTED = -5,  /* valid request that this library does not implement */
  LMG_ENOCONV = -6,       /* the least-misfit optimisation did not converge */
  LMG_EDEVICE = -7        /* a kernel's own check found an anomaly (lmg_plan_status) */
} lmg_status;

enum { LMG_C64 = 0, LMG_C128 = 1 };
enum { LMG_INTERP_NEAREST = 0, LMG_INTERP_LINEAR = 1, LMG_INTERP_QUADRATIC = 2, LMG_INTERP_CUBIC = 3,
       LMG_INTERP_DIRECT = 4 };
enum { LMG_CORR_HOPT = 0, LMG_CORR_INV_C = 1 };
enum { LMG_ACCUM_PLAIN = 0, LMG_ACCUM_COMPENSATED = 1 };
enum { LMG_CROP = 0, LMG_PAD = 1 };
enum { LMG_FFT_IMAGE = +1, LMG_FFT_MODEL = -1 };

typedef struct lmg_table lmg_table; /* least-misfit function (host float64) */
typedef struct lmg_plan lmg_plan;   /* device state for one (table, n_image, x0, pixel_scale) */
typedef struct lmg_batch lmg_batch; /* many independent channels gridded together */

/* lmg_kernel_table -- build the least-misfit gridding function and its look-up table.
 *
 * Section 2.1 and Appendices A, B, E: h(x) is represented on Ng+1 = 33 nodes in
 * [0, x0_paper] with h(0) = 1 and optimised by Levenberg-Marquardt to minimise the
 * integrated map error E (Eq. 16), with C_r(s) solved per offset set from the normal
 * equations (Eqs. 17-19, W <= 11) or by QR least squares (Appendix B, W > 11). Initial
 * guesses: h = 1 for W <= 4, h_W = h_{W-1}^2 / h_{W-2} above (Appendix A). The table holds
 * rows s_i = i / oversample, i = 0..oversample, of the W values C(j - W/2 + s_i)
 * (Appendix E; one guard row at s = 1 so interpolation never crosses the odd-W jump of
 * Appendix C). Host-only float64 work; no GPU is touched.
 *
 *   W          support width, 1..16
 *   x0         kept fraction of the FFT image, 0 < x0 <= 1 (paper's x0 = x0 / 2)
 *   oversample table sampling rate M_s per cell, 2..1000000
 *   interp     table interpolation of degree d (Appendix F): LMG_INTERP_NEAREST (d = 0),
 *              LMG_INTERP_LINEAR (d = 1), LMG_INTERP_QUADRATIC (d = 2) or LMG_INTERP_CUBIC
 *              (d = 3). For d >= 2, t = s * oversample is interpolated through rows
 *              k0 .. k0 + d, k0 = floor(t - (d - 1) / 2) clamped to [0, oversample - d],
 *              with the Lagrange basis on those rows; the table error falls as
 *              oversample^-(d+1), so d = 3 reaches linear's accuracy with a far smaller
 *              table (oversample >= d required). LMG_INTERP_DIRECT: no table lookup;
 *              the gridding weights of every visibility are calculated directly from the
 *              normal equations, C(s) = A^-1 B(s) (Section 5.2, Eqs. 17-19), with A^-1 and
 *              the node sums folded into W x 33 cosine and sine coefficients on the host;
 *              exact function values at a higher cost. float64 plans and W <= 11 only (the
 *              normal equations' range, Appendix B); tables from lmg_table_from_values
 *              cannot use it (they carry no h)
 *   correction LMG_CORR_HOPT (h = c / D, Eqs. 12, 15) or LMG_CORR_INV_C (h = 1/c)
 *   out        receives the new table (caller frees with lmg_table_free)
 * Returns LMG_EINVAL on a bad argument, LMG_ENOMEM, LMG_ENOCONV if the optimiser fails.
 */
int lmg_kernel_table(int W, double x0, int oversample, int interp, int correction,
                     lmg_table** out);

/* lmg_table_from_values -- a table from caller-supplied host values C[(oversample+1)][W]
 * in the layout lmg_kernel_table builds (row i at s = i / oversample, entry j is
 * C(j - W/2 + s)). Lets any separable gridding function be used with the same kernels.
 * The values are copied. */
int lmg_table_from_values(int W, double x0, int oversample, int interp, int correction,
                          const double* C_host, lmg_table** out);

int lmg_table_free(lmg_table* t);

/* lmg_table_export -- copy host float64 data out of a table (any pointer may be NULL).
 *   C_host   [(oversample+1)][W] table values, nC = capacity in doubles
 *   h_host   [Ng+1] node values of h on [0, x0_paper] (all zero for a caller table),
 *            nh = capacity in doubles
 *   E        integrated misfit E at the optimum (Eq. 16; NaN for a caller table)
 *   info     [4] ints: W, oversample, Ng, iterations of the optimiser */
int lmg_table_export(const lmg_table* t, double* C_host, size_t nC, double* h_host,
                     size_t nh, double* E, int* info);

/* lmg_correction_export -- the grid-correction factors h(x_p) (host float64) at the
 * n_image kept pixels x_p = (p - n_image/2) / N, N = n_image / x0, for the table function
 * actually used (c and D integrated over s with 8-point Gauss-Legendre per table piece;
 * Eqs. 12-15). If single_precision is nonzero the table values are first rounded to
 * float32, as the LMG_C64 path uses them. h_host has n_image doubles. */
int lmg_correction_export(const lmg_table* t, int64_t n_image, int single_precision,
                          double* h_host);

/* lmg_plan_create -- device state for imaging with one table at one image size.
 *   n_image      kept image side (pixels); N = n_image / x0 must be an even integer,
 *                a multiple of 64 (LMG_C64) or 32 (LMG_C128), and at least 64
 *   pixel_scale  image pixel size in radians (u_cells = u * N * pixel_scale)
 *   max_vis      capacity: the largest nvis later passed to lmg_plan_bin (>= 1)
 *   dtype        LMG_C64 or LMG_C128
 * Allocates the device table, correction factors, binning buffers sized for max_vis, a
 * work grid [N][N] and a cuFFT plan; uses the current CUDA device. Synchronous.
 * Returns LMG_EINVAL, LMG_ENOMEM, LMG_ECUDA or LMG_ECUFFT on failure. */
int lmg_plan_create(const lmg_table* t, int64_t n_image, double pixel_scale,
                    int64_t max_vis, int dtype, lmg_plan** out);

/* lmg_plan_create_ex -- lmg_plan_create with flags. LMG_PLAN_NO_WORK_GRIDS leaves out the
 * plan's two [N][N] grids (work and model, 2 N^2 complex: 268 MB for a complex64 4096^2
 * grid); such a plan images and predicts only through lmg_dirty_image_ws and
 * lmg_predict_vis_ws with caller workspace (lmg_dirty_image / lmg_predict_vis return
 * LMG_EINVAL on it, lmg_work_grid returns NULL). Unknown flags are LMG_EINVAL. */
#define LMG_PLAN_NO_WORK_GRIDS 1
int lmg_plan_create_ex(const lmg_table* t, int64_t n_image, double pixel_scale,
                       int64_t max_vis, int dtype, int flags, lmg_plan** out);
int lmg_plan_free(lmg_plan* p);

/* lmg_plan_bin -- bin visibility positions for gridding and degridding (support rule of
 * Eq. 6; sort into strips of 64 columns (LMG_C64) or 32 columns (LMG_C128) by support-start
 * row; balanced work items). Must be called before lmg_grid / lmg_degrid / lmg_dirty_image /
 * lmg_predict_vis and again whenever the positions change. uv: device float64 [nvis][2] in
 * wavelengths, 16-byte aligned, 0 <= nvis <= max_vis; read by two kernels of this call
 * (counting, then placing the records), so it must stay unchanged until the stream has run
 * them. Allocates nothing. */
int lmg_plan_bin(lmg_plan* p, const double* uv, int64_t nvis, void* stream);

/* lmg_plan_bin_tracks -- lmg_plan_bin for positions stored sample-major: visibility
 * k = t * tracks + b is sample t of track b (one baseline of one channel), as a correlator
 * writes one integration of every baseline after another; a last partial sample row is
 * allowed (nvis need not be a multiple of tracks). Each binning thread follows one track
 * over 32 consecutive samples, and samples that share a bucket take one counter update and
 * one offset lookup per run instead of one per record. The binning is the same for any
 * tracks >= 1 (the order of the records within a bucket, and so the rounding order of the
 * sums, may differ); the hint only changes the cost. LMG_EINVAL for tracks < 1. */
int lmg_plan_bin_tracks(lmg_plan* p, const double* uv, int64_t nvis, int64_t tracks, void* stream);

/* lmg_plan_dropped -- number of positions dropped by the last lmg_plan_bin (not finite
 * or 2^30 cells or more from the origin). Synchronises the given stream. */
int lmg_plan_dropped(lmg_plan* p, int64_t* dropped, void* stream);

/* lmg_grid -- G_n = sum_k w_k V_k C(n - u_k) C(m - v_k) over each support (Eqs. 5-6).
 *   vis      device complex [nvis] of the plan's dtype
 *   weights  device real [nvis] (float for C64, double for C128) or NULL (all ones)
 *   accum    LMG_ACCUM_PLAIN, or LMG_ACCUM_COMPENSATED (C64 only: each accumulator is
 *            a float pair updated with an error-free sum)
 *   grid     device complex [N][N]; every cell is overwritten (no pre-zeroing needed)
 * Allocates nothing. Where work items are shorter than W - 1 rows (dense rows), the partial
 * rows of two items are added into the same cells by atomics in either order, so two calls
 * on the same input may differ at the rounding level of the dtype. */
int lmg_grid(lmg_plan* p, const void* vis, const void* weights, int accum, void* grid,
             void* stream);

/* lmg_degrid -- V_k = sum_{i,j} C(n_i - u_k) C(m_j - v_k) G[m_j][n_i] (Section 4, the
 * transpose of lmg_grid without weights). grid: device complex [N][N];
 * vis_out: device complex [nvis], every entry overwritten. Allocates nothing. The result
 * is the same bits on every call (each entry is one sum, or two added onto zero when the
 * support crosses a 64-column strip, 32 for complex128). */
int lmg_degrid(lmg_plan* p, const void* grid, void* vis_out, void* stream);

/* lmg_degrid_add -- lmg_degrid that adds the predictions to vis_inout instead of
 * overwriting it (Section 4; e.g. the sum of the predictions from several grids, or an
 * output zeroed earlier on another stream). Dropped positions leave their entries as they
 * are. Same arguments, alignment and errors as lmg_degrid. The two adds of a visibility
 * whose support crosses a strip may land in either order. */
int lmg_degrid_add(lmg_plan* p, const void* grid, void* vis_inout, void* stream);

/* lmg_fft -- unnormalised in-place 2-D FFT of a device grid [N][N] in grid index order.
 * direction LMG_FFT_IMAGE computes sum_i G[i] exp(+i 2 pi i q / N) (cuFFT inverse);
 * LMG_FFT_MODEL computes sum_q P[q] exp(-i 2 pi i q / N) (cuFFT forward). */
int lmg_fft(lmg_plan* p, int direction, void* grid, void* stream);

/* lmg_fft_pruned -- the transform lmg_dirty_image (LMG_FFT_IMAGE) or lmg_predict_vis
 * (LMG_FFT_MODEL) applies to the work grid, in place on `grid` ([N][N], plan dtype). Only
 * the kept field of Eq. 4 (|x| <= x0 / 2, n_image pixels per axis) is needed there, so:
 * LMG_FFT_IMAGE transforms every row, then only the n_image kept columns (index q mod N in
 * [0, n_image/2) or [N - n_image/2, N)); its result equals lmg_fft's at the kept rows and
 * columns and is partial elsewhere. LMG_FFT_MODEL transforms only the n_image kept rows,
 * then every column; its result equals lmg_fft's when every other row is zero (as after
 * lmg_grid_correct with LMG_PAD). */
int lmg_fft_pruned(lmg_plan* p, int direction, void* grid, void* stream);

/* lmg_grid_correct -- grid correction and crop (Eqs. 4, 15), or its adjoint, with the
 * plan's device copy of the correction factors (the table object is host-only and holds no
 * device memory; lmg_correct_factors takes the factors from the caller instead).
 *   LMG_CROP: in = FFT output [N][N] of a grid in index order, out = image
 *             [n_image][n_image] with out[p][q] = h(y_p) h(x_q) F(x_q, y_p).
 *   LMG_PAD:  in = image [n_image][n_image], out = [N][N] array that LMG_FFT_MODEL turns
 *             into the model grid in index order (zero outside the kept pixels).
 * Allocates nothing. */
int lmg_grid_correct(lmg_plan* p, int direction, const void* in, void* out, void* stream);

/* lmg_dirty_image -- grid, FFT (+i), correct and crop into image_out [n_image][n_image],
 * using the plan's work grid (lmg_dirty_image_ws takes a caller workspace). Allocates
 * nothing. */
int lmg_dirty_image(lmg_plan* p, const void* vis, const void* weights, int accum,
                    void* image_out, void* stream);

/* lmg_predict_vis -- pad and correct image [n_image][n_image], FFT (-i), degrid into
 * vis_out [nvis], using the plan's work grid. Allocates nothing. */
int lmg_predict_vis(lmg_plan* p, const void* image, void* vis_out, void* stream);

/* lmg_workspace_bytes -- bytes of caller workspace that lmg_dirty_image_ws and
 * lmg_predict_vis_ws need for this plan: one [N][N] complex grid of the plan's dtype
 * (N^2 * 8 bytes for LMG_C64, N^2 * 16 for LMG_C128). 0 for a NULL plan. */
size_t lmg_workspace_bytes(const lmg_plan* p);

/* lmg_dirty_image_ws -- lmg_dirty_image with a caller-owned device workspace in place of
 * the plan's work grid (Eqs. 4-6: grid, FFT (+i) pruned to the kept columns, correct and
 * crop). workspace: device, 256-byte aligned, ws_bytes >= lmg_workspace_bytes(p); its
 * contents on entry do not matter and on return are the partially transformed grid.
 * Allocates nothing. LMG_EINVAL for a NULL, misaligned or short workspace. */
int lmg_dirty_image_ws(lmg_plan* p, const void* vis, const void* weights, int accum,
                       void* image_out, void* workspace, size_t ws_bytes, void* stream);

/* lmg_predict_vis_ws -- lmg_predict_vis with a caller-owned device workspace (Section 4:
 * pad and correct into the whole workspace, zero outside the kept field; FFT (-i) of the
 * kept rows then every column, in place; degrid). Same workspace rules as
 * lmg_dirty_image_ws. Allocates nothing. */
int lmg_predict_vis_ws(lmg_plan* p, const void* image, void* vis_out, void* workspace,
                       size_t ws_bytes, void* stream);

/* lmg_correct_factors -- the grid correction of lmg_grid_correct with caller-supplied
 * factors instead of a plan (Eqs. 4, 15): h is a device array of n_image reals (float for
 * LMG_C64, double for LMG_C128), h[p] = h(x_p) at x_p = (p - n_image/2) / N, for example
 * lmg_correction_export's values copied to the device. LMG_CROP: in [N][N] FFT output,
 * out [n_image][n_image]; LMG_PAD: in [n_image][n_image], out [N][N] (zero outside the
 * kept pixels). n_image even, N even in [n_image, 65536]. Allocates nothing. */
int lmg_correct_factors(int direction, const void* in, void* out, const void* h, int64_t n_image,
                        int64_t N, int dtype, void* stream);

/* lmg_image_from_grid -- the dirty image from a gridded [N][N] array: the transform of
 * Eq. 4 with the correction and crop of Eq. 15, the same result as lmg_fft_pruned
 * (LMG_FFT_IMAGE) followed by lmg_grid_correct (LMG_CROP). For LMG_C64 plans with N = 4096
 * it runs fused transform kernels (two launches: the rows, keeping the n_image kept columns
 * in a scratch array, then four kept columns per CTA with the correction applied as the
 * image is written); grid is left unchanged, image_out must be 16-byte aligned and scratch
 * is a device array of lmg_transform_scratch_bytes bytes (16-byte aligned), or NULL for the
 * plan's own (which concurrent calls on other streams must not share; a plan created with
 * LMG_PLAN_NO_WORK_GRIDS has none: LMG_EINVAL). Otherwise grid is transformed in place with
 * the library's pruned transforms and scratch is not used. */
int lmg_image_from_grid(lmg_plan* p, void* grid, void* image_out, void* scratch, void* stream);

/* lmg_grid_from_image -- the adjoint: the [N][N] grid that lmg_degrid reads for a model
 * image (pad, correction, transform of Eq. 2), the same result as lmg_grid_correct (LMG_PAD)
 * followed by lmg_fft_pruned (LMG_FFT_MODEL); every cell of grid_out is written. Fused
 * kernels, alignment and scratch as for lmg_image_from_grid. */
int lmg_grid_from_image(lmg_plan* p, const void* image, void* grid_out, void* scratch, void* stream);

/* lmg_transform_scratch_bytes -- bytes of the scratch of the fused transforms
 * (N x n_image complex64 values), or 0 where the plan uses the library transforms. */
size_t lmg_transform_scratch_bytes(const lmg_plan* p);

/* lmg_plan_status -- device status of the plan's last binning. The kernels check their own
 * bounds and record what they could not do in a status word instead of faulting (today:
 * more work items than the plan's capacity, whose excess is dropped; the capacity is sized
 * so that this does not happen for any input within max_vis). Synchronises the stream,
 * writes the status bits to *status_bits (may be NULL) and returns LMG_OK when they are
 * zero, LMG_EDEVICE with a message otherwise. */
int lmg_plan_status(lmg_plan* p, int* status_bits, void* stream);

/* lmg_fp32_fma_rate -- measured float32 FMA throughput of the current device in flop/s (a
 * kernel of independent fmaf chains filling every SM, best of three timed launches after
 * one warm-up; synchronises the stream). A measurement helper for the arithmetic side of the
 * sweeps' roofline (8 W^2 flops per visibility for gridding plus degridding); not part of the
 * paper's method. */
int lmg_fp32_fma_rate(double* flops_per_s, void* stream);

/* lmg_plan_info -- sizes of a plan: out[0] = N, out[1] = n_image, out[2] = W,
 * out[3] = nvis of the last binning, out[4] = records, out[5] = work items (records and
 * items need a synchronised stream to be current), out[6] = dtype. */
int lmg_plan_info(lmg_plan* p, int64_t* out, void* stream);

/* lmg_work_grid -- device pointer of the plan's internal [N][N] work grid (valid until
 * lmg_plan_free). lmg_dirty_image and lmg_predict_vis transform it with FFTs pruned to
 * the outputs they use: afterwards it holds the transform at the kept rows and columns
 * (dirty image) or the transformed model grid (prediction; the plan pads the model into a
 * second internal grid whose rows outside the kept field stay zero and transforms it out of
 * place into the work grid). */
void* lmg_work_grid(lmg_plan* p);

/* lmg_grid_static -- binning plus gridding (the work of lmg_plan_bin + lmg_grid, complex64)
 * without allocating any memory, for callers that cannot call cudaMalloc: for example a
 * process whose device memory is owned by another allocator or reserved at start-up, or
 * a real-time pipeline that must not allocate while it runs. The paper has no
 * counterpart; this is a deployment variant of the existing path.
 *
 * All working memory (bucket ranks, records, bucket counts, work items,
 * spill rows and the float32 copy of the table) lives in one fixed-size __device__ array
 * of this library, about 16 MB, which every GPU that loads the library holds until the
 * process exits.
 * Limits: nvis <= LMG_STATIC_MAX_VIS, grid N = n_image / x0 a multiple of 64 in
 * [64, LMG_STATIC_MAX_N], table oversample <= LMG_STATIC_MAX_OVERSAMPLE; larger sizes
 * return LMG_EINVAL with a message and do nothing.
 *   t            table (host object from lmg_kernel_table or lmg_table_from_values)
 *   n_image, pixel_scale, uv, nvis   as for lmg_plan_create / lmg_plan_bin
 *   vis          device complex64 [nvis]; weights device float32 [nvis] or NULL
 *   grid         device complex64 [N][N]; every cell is overwritten
 * The first call on a device (with that device current) looks up the array's device
 * address and records it; make that first call before any stream capture. The recorded
 * address belongs to the device's current context: do not call lmg_grid_static again after
 * cudaDeviceReset on that device (the array then lives at a new address that this library
 * does not look up again). Each device keeps the float32 copy of the table of its latest
 * call; a call with a table whose values differ uploads it from host memory (and returns
 * LMG_EUNSUPPORTED if its stream is being captured), a call with the same table skips
 * the upload. All calls share the one array: calls whose GPU work overlaps (other streams,
 * other host threads) race on it and must be serialised by the caller. Nothing else is
 * carried between calls (bucket counts and counters are cleared on the stream by each
 * call). */
#define LMG_STATIC_MAX_VIS 262144
#define LMG_STATIC_MAX_N 2048
#define LMG_STATIC_MAX_OVERSAMPLE 4096
int lmg_grid_static(const lmg_table* t, int64_t n_image, double pixel_scale, const double* uv,
                    int64_t nvis, const void* vis, const void* weights, void* grid, void* stream);

/* ---------------------------------------------------------------------------------------
 * Multi-channel batches. Channels (for example frequency channels, each with its own uv
 * set in wavelengths) are independent problems of Sections 2-4, each with its own table
 * (so its own W), grid size and pixel scale. A batch runs them together: every channel is
 * binned as by lmg_plan_bin, then the sweeps of all channels with the same W run as ONE
 * persistent kernel launch, whose warps take work items of every such channel from one
 * counter. FFTs run as one batched cuFFT plan per distinct grid size. The launch sequence
 * of each operation is captured once into a CUDA graph on the batch's own stream (ordered
 * after and before the caller's stream by events) and replayed while the caller passes the
 * same buffers; new buffers trigger a new capture.
 * Complex64 only. Arrays of per-channel arguments are HOST arrays of length n_chan whose
 * entries are DEVICE pointers (complex64 vis/grids/images, float32 weights, float64 uv).
 * The batch copies what it needs from the arrays during the call.
 * --------------------------------------------------------------------------------------- */
#define LMG_BATCH_MAX_CHANNELS 1024

/* lmg_batch_create -- per channel c: table tables[c] (not owned; must outlive the batch),
 * image size n_image[c], pixel scale pixel_scale[c] (radians) and capacity max_vis[c].
 * Same argument rules as lmg_plan_create for each channel, with nearest or linear tables
 * (LMG_EUNSUPPORTED otherwise); 1 <= n_chan <=
 * LMG_BATCH_MAX_CHANNELS. Allocates every channel's binning buffers, one work grid per
 * channel (contiguous per grid size) and one batched FFT plan per grid size. */
int lmg_batch_create(int n_chan, const lmg_table* const* tables, const int64_t* n_image,
                     const double* pixel_scale, const int64_t* max_vis, lmg_batch** out);
int lmg_batch_free(lmg_batch* b);

/* lmg_batch_bin -- bins channel c's uv[c] (device float64 [nvis[c]][2], 16-byte aligned)
 * for every c; uv[c] may be NULL when nvis[c] == 0. As for lmg_plan_bin, each uv[c] is
 * read by two kernels on the stream and must stay unchanged until the stream has run
 * them. Invalidates captured graphs. */
int lmg_batch_bin(lmg_batch* b, const double* const* uv, const int64_t* nvis, void* stream);

/* lmg_batch_grid -- grid[c] = gridded vis[c] (x weights[c]) for every channel, as lmg_grid
 * with plain accumulation. weights may be NULL (all unweighted) or hold NULL entries. */
int lmg_batch_grid(lmg_batch* b, const void* const* vis, const void* const* weights, void* const* grid,
                   void* stream);

/* lmg_batch_degrid -- vis_out[c] = degridded grid[c] for every channel, as lmg_degrid. */
int lmg_batch_degrid(lmg_batch* b, const void* const* grid, void* const* vis_out, void* stream);

/* lmg_batch_dirty_image -- image[c] ([n_image[c]]^2) = dirty image of vis[c], as
 * lmg_dirty_image (plain accumulation) for every channel, through the batch's work grids. */
int lmg_batch_dirty_image(lmg_batch* b, const void* const* vis, const void* const* weights,
                          void* const* image, void* stream);

/* lmg_batch_predict_vis -- vis_out[c] = predicted visibilities of image[c], as
 * lmg_predict_vis for every channel. */
int lmg_batch_predict_vis(lmg_batch* b, const void* const* image, void* const* vis_out, void* stream);

/* lmg_batch_tune -- autotuner. Times gridding plus degridding of the current binned uv
 * sets with vis[c] (device complex64 [nvis[c]], used read-only) for each candidate of: rows
 * per work item bin (64, 128, 256, 512), records per work item (256, 512, 1024, 2048), warps
 * per CTA (4, 8) and table placement (shared or global memory, where the tables fit),
 * keeps the fastest, re-bins every channel with it and writes it to chosen[4] (rows,
 * records, warps, table in shared memory) when chosen is not NULL. Requires a prior
 * lmg_batch_bin with the same uv (its pointers are reused for re-binning). Synchronises
 * the stream; allocates and frees scratch output. Not capturable. */
int lmg_batch_tune(lmg_batch* b, const void* const* vis, void* stream, int* chosen);

/* lmg_batch_info -- out[0] channels, out[1] distinct W, out[2] distinct grid sizes,
 * out[3] total visibilities binned, out[4] rows per bin, out[5] records per item,
 * out[6] warps per CTA, out[7] graphs captured so far. */
int lmg_batch_info(lmg_batch* b, int64_t* out);

/* lmg_last_error -- message for the calling thread's most recent failure ("" if none). */
const char* lmg_last_error(void);

/* lmg_version -- library version string. */
const char* lmg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LMG_H */

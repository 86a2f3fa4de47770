/*
 * mmsar.h -- C ABI of the GB300 multi-planar multistatic MIMO-SAR imager.
 *
 * The library forms a complex 3-D reflectivity volume from irregularly
 * sampled MIMO-SAR echoes by the method of Smith & Torlak, "Efficient 3-D
 * Near-Field MIMO-SAR Imaging for Irregular Scanning Geometries" (IEEE
 * Access 2022):
 *
 *   1. per-sample multi-planar multistatic phase compensation (Sec. II-C,
 *      Eq. 11-12) onto a virtual planar monostatic array (Eq. 3-4, Eq. 10);
 *   2. Gaussian gridding of the compensated samples onto the regular planar
 *      aperture and a 2-D FFT (the FGG-NUFFT form of FT_2D in Eq. 16, Sec. III);
 *   3. the k_z weight and phase of Eq. 15 (P(f) = 1) and the Stolt step S of
 *      Eq. 16, done as a 1-D Gaussian gridding over k_z plus an FFT;
 *   4. the inverse 2-D FFT over (k_x, k_y) (IFT_3D of Eq. 16).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All pointers named "device" are CUDA device pointers the caller owns
 *   (PyTorch tensors, cudaMalloc, ...).  The library allocates no device
 *   memory: every intermediate lives in the caller's workspace.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Calls are stream-ordered and asynchronous: argument
 *   validation errors return synchronously; conditions found on the device
 *   (non-finite input, an unusable reference plane) are recorded in an
 *   error word inside the workspace and read with mmsar_poll_error().
 * - Geometry in metres, frequencies in Hz, c = 299792458 m/s.
 * - Sample order l = (t, r, p): echo[t][r][p][k], k fastest, with the Tx at
 *   pos[p] + tx[t] and the Rx at pos[p] + rx[r].
 * - +z points from the scan plane toward the scene (the scene lies at
 *   z > z_ref).  With this orientation the residual of Eq. 12 reads
 *   beta = -2 d^z + ((d^x)^2 + (d^y)^2) / (4 Z_c), Z_c = z_scene - z_ref.
 * - Output voxel (i, j, q) has centre (x0 + i dx, y0 + j dy, z0 + q dz) and
 *   is stored at vol[(i * ny + j) * nz + q] (z fastest), complex64.
 * - The image is normalised by 1 / (n_tx n_rx n_pos n_k).
 * - No C++ exception crosses this boundary.  The imaging calls only read
 *   the plan, so one plan may serve several streams or threads at once as
 *   long as every call in flight has its own workspace.  The calls that
 *   change a plan (mmsar_plan_set_tiles, mmsar_plan_set_stage_events,
 *   mmsar_plan_destroy) must not run while another thread uses that plan;
 *   stage events set on a plan are recorded by every call that uses it.
 */
#ifndef MMSAR_H
#define MMSAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MMSAR_OK = 0,
    MMSAR_ERR_INVALID_ARG = 1,      /* null pointer, non-positive pitch, ...     */
    MMSAR_ERR_UNSUPPORTED_SIZE = 2, /* a size outside the supported ranges       */
    MMSAR_ERR_OUT_OF_MEMORY = 3,    /* workspace smaller than required           */
    MMSAR_ERR_CUDA = 4,             /* a CUDA runtime call failed                */
    MMSAR_ERR_DEVICE_TIMEOUT = 5,   /* a bounded device-side wait gave up        */
    MMSAR_ERR_NONFINITE = 6         /* NaN/Inf in the echo or the geometry       */
} mmsar_status;

/* Storage type of the echo tensor.  Arithmetic is FP32 in every case. */
typedef enum {
    MMSAR_ECHO_C64 = 0,          /* interleaved float (re, im)                       */
    MMSAR_ECHO_F16X2_SCALED = 1, /* interleaved __half (re, im) times a per-scan scale */
    MMSAR_ECHO_BF16X2_SCALED = 2 /* interleaved bf16 (re, im) times a per-scan scale   */
} mmsar_echo_dtype;

/* Acquisition shape.  The stepped/FMCW frequency grid is uniform,
 * f_k = f0_hz + k * df_hz (Sec. II-C, Eq. 9; sampling rule Sec. III). */
typedef struct {
    int n_tx;                 /* Tx elements, >= 1                      */
    int n_rx;                 /* Rx elements, >= 1                      */
    int n_pos;                /* scan positions, >= 0                   */
    int n_k;                  /* frequency samples, 1 .. 1024           */
    double f0_hz;             /* first frequency, > 0                   */
    double df_hz;             /* frequency step, > 0 (ignored if n_k=1) */
    mmsar_echo_dtype dtype;   /* echo storage                           */
} mmsar_shape;

/* Output voxel grid (centres).  nx, ny in 1 .. 1024, nz in 1 .. 256. */
typedef struct {
    double x0, y0, z0;        /* centre of voxel (0, 0, 0)              */
    double dx, dy, dz;        /* pitches, > 0                           */
    int nx, ny, nz;
} mmsar_grid;

typedef struct {
    double z_ref;      /* virtual plane Z0 (Eq. 4); NaN => mean of z_l over samples    */
    double z_scene;    /* scene depth for the MIMO term of Eq. 12; NaN => grid z centre */
    int compensate;    /* 1 = Eq. 11-12 applied (paper: Eq. 7's on-axis residual);      *
                        * 2 = Eq. 11 with the residual of Eq. 5 evaluated at the scene   *
                        *     centre (x_c, y_c, z_scene) for each virtual element, i.e.   *
                        *     with the off-axis terms Eq. 7 drops;                       *
                        * 0 = beta = 0 (RMA ablation).  Other values: INVALID_ARG.       */
    double nufft_tol;  /* Gaussian gridding accuracy per transform; <= 0 => 1e-3        */
    int mx, my;        /* spectral grid (power of two >= nx, ny, 16..1024); 0 => auto  */
} mmsar_options;

typedef struct mmsar_plan mmsar_plan;

/* Fill `opt` with the defaults listed above.  Never fails for non-NULL opt. */
void mmsar_options_default(mmsar_options *opt);

/* Validate sizes and build a host-side plan (no device memory, no CUDA
 * calls).  On success *out owns the plan; release it with
 * mmsar_plan_destroy.  Returns MMSAR_ERR_INVALID_ARG / _UNSUPPORTED_SIZE
 * with a message in mmsar_last_error() otherwise. */
mmsar_status mmsar_plan_create(mmsar_plan **out, const mmsar_shape *shape,
                               const mmsar_grid *grid, const mmsar_options *opt);

/* Bytes of device workspace one mmsar_image call on this plan needs. */
mmsar_status mmsar_plan_workspace_bytes(const mmsar_plan *plan, size_t *bytes);

/* The Gaussian kernel width (taps per axis), the spectral grid and the
 * number of kernels one mmsar_image call launches.  Any output may be NULL. */
mmsar_status mmsar_plan_info(const mmsar_plan *plan, int *kernel_width, int *mx, int *my,
                             int *kernels_per_image);

/* Launch shape of the gridding stage (the spreading step of Sec. III's
 * Gaussian gridding).  The shapes compute the same image: bit for bit among
 * the per-sample shapes, to rounding between the per-sample and the grouped
 * form (another summation order); they differ in speed, which depends on the
 * scan (small scans fill the GPU better with smaller CTAs; arrays whose Tx
 * and Rx lie on one line along y give large groups).  The tensor-core form
 * agrees with them to FP32 rounding.  Defaults: 2, 4, 0, 5 (the
 * warp-specialised tensor-core form; the first three fields then unused). */
typedef struct {
    int grid_freqs_per_lane;   /* 1: a CTA covers 32 frequencies; 2: 64; 4: 128,   *
                                * in 4 x 2-cell warp blocks (fewer taps outside   *
                                * the support; per-sample form only)              */
    int grid_warps_per_cta;    /* 4: an 8 x 8-cell tile (8 x 4 for 4 frequencies  *
                                * per lane); 8: 16 x 8 (16 x 4)                   */
    int grid_grouped;          /* 1: the samples of one position whose Tx/Rx pairs *
                                * share the x offset (Eq. 3: the same x') are     *
                                * gridded together, the x weights applied once to *
                                * their y-weighted sum (needs n_tx n_rx <= 16);   *
                                * 0: sample by sample                              */
    int grid_tensor_cores;     /* 1 .. 5: the gridding runs on the tensor cores as *
                                * a per-tile product weights x samples, FP32-     *
                                * accurate (FP16 hi/lo operands, FP32             *
                                * accumulation); the value picks the pipeline:    *
                                * 64-frequency groups per work item 4 (1, 2, 5)   *
                                * or 2 (3, 4); the sample rows staged through     *
                                * registers (1, 4) or by asynchronous copies with *
                                * two (2) or four (3) shared-memory stages, all   *
                                * giving the same bits; 5: one CTA per SM whose   *
                                * warps list, gather, multiply and write back     *
                                * concurrently (its own list segments: the same  *
                                * sums to FP32 rounding, deterministic); the     *
                                * three fields above are then ignored.  0: the    *
                                * FP32 FMA forms above                             */
} mmsar_tiles;

/* Set (or read) the plan's gridding launch shape; the autotuner of the
 * Python package times the shapes on the caller's data and sets the
 * fastest.  INVALID_ARG for other values.  Changes the plan: not while another
 * thread images with it. */
mmsar_status mmsar_plan_set_tiles(mmsar_plan *plan, const mmsar_tiles *tiles);
mmsar_status mmsar_plan_get_tiles(const mmsar_plan *plan, mmsar_tiles *tiles);

/* Test of the bounded device-side waits (no counterpart in the paper).  With
 * on == 1, the next images of this plan run the warp-specialised tensor-core
 * gridding (grid_tensor_cores = 5) with one MMA thread per CTA waiting on a
 * barrier that nothing completes: the wait runs out after about half a
 * second, the CTA's other warps stop at their next wait, every copy and MMA in
 * flight is waited for and the tensor memory freed, and the error word gets
 * MMSAR_ERR_DEVICE_TIMEOUT (mmsar_poll_error returns it; the image is void).
 * The context stays usable: with on == 0 the next image is normal.  Other
 * gridding forms ignore it.  INVALID_ARG for other values. */
mmsar_status mmsar_plan_set_wait_test(mmsar_plan *plan, int on);

/* Stages of mmsar_image, in launch order: 0 "prep" (reference plane,
 * geometry of Eq. 3-4 and 12, binning), 1 "compensate" (Eq. 11),
 * 2 "grid" (Gaussian gridding), 3 "fft_x", 4 "fft_y" (FT_2D of Eq. 16 with
 * deconvolution), 5 "stolt" (Eq. 15 weight + Stolt + z transform),
 * 6 "ifft_y", 7 "ifft_x" (IFT over k_x, k_y). */
int mmsar_stage_count(void);
const char *mmsar_stage_name(int stage);

/* Optional per-stage timing.  With n == mmsar_stage_count() + 1 events
 * (cudaEvent_t passed as void*, owned by the caller), every later
 * mmsar_image call on this plan records events[i] on its stream right before
 * stage i and events[n - 1] after the last stage.  n == 0 (events NULL)
 * turns it off. */
mmsar_status mmsar_plan_set_stage_events(mmsar_plan *plan, void *const *events, int n);

/* Form one image (Sec. II-C Eq. 11-12 followed by Eq. 16), stream-ordered.
 *   workspace   device, >= mmsar_plan_workspace_bytes, 256-byte aligned; its
 *               contents are scratch (overwritten by every call)
 *   echo        device [n_tx][n_rx][n_pos][n_k] in shape.dtype
 *   echo_scale  device float scalar multiplying a scaled FP16/BF16 echo;
 *               NULL for MMSAR_ECHO_C64
 *   pos         device double [n_pos][3]  radar reference point per position
 *   tx, rx      device double [n_tx][3], [n_rx][3]  element offsets from it
 *   vol         device complex64 [nx][ny][nz] output (fully overwritten)
 * Inputs are read only; the output may not alias any input or the
 * workspace. */
mmsar_status mmsar_image(mmsar_plan *plan, void *workspace, size_t workspace_bytes,
                         const void *echo, const float *echo_scale,
                         const double *pos, const double *tx, const double *rx,
                         void *vol, void *stream);

/* Direct back-projection, the paper's reference algorithm (Sec. III, used
 * for comparison in Sec. V):
 *   o_BP(r) = sum_{t,r,p,k} s(t,r,p,k) exp(+j k (|T - r| + |R - r|)),
 * k = 2 pi (f0 + k df) / c, unnormalised, at n_voxels voxel centres
 * `voxels` (device double [n][3]) or, with voxels == NULL, at every voxel of
 * the plan's grid (output in the mmsar_image layout).  out: device complex64
 * [n].  Complex64 echoes only.  Cost: voxels x samples x frequencies; meant
 * for cross-checks and small grids.  Stream-ordered. */
mmsar_status mmsar_backproject(const mmsar_plan *plan, const void *echo, const double *pos,
                               const double *tx, const double *rx, const double *voxels,
                               int64_t n_voxels, void *out, void *stream);

/* One image request of a batch: its plan, its own workspace, inputs, output. */
typedef struct {
    mmsar_plan *plan;
    void *workspace;
    size_t workspace_bytes;
    const void *echo;
    const float *echo_scale;
    const double *pos, *tx, *rx;
    void *vol;
} mmsar_request;

/* Form n images of possibly different shapes (Sec. III imaging of several
 * independent scans).  Request i runs on streams[i % n_streams] (cudaStream_t
 * as void*), so uneven scans overlap on the device; ordering between the
 * given streams is the caller's.  Each request needs its own workspace.
 * Returns the first validation or launch error (requests before it were
 * enqueued). */
mmsar_status mmsar_image_batch(const mmsar_request *reqs, int n, void *const *streams, int n_streams);

/* The same n images (Sec. III imaging of several independent scans) as
 * fused launches on one stream: every stage of mmsar_image runs as one
 * launch for all requests that use the same kernel instance (up to 32 scans
 * per launch; requests of other FFT lengths, gridding shapes, echo types or
 * Stolt grids form further launches), so an uneven batch fills the GPU with
 * a handful of launches instead of ten per scan.  Each request needs its own
 * workspace; the images are bit for bit those of mmsar_image.  `launches`
 * (may be NULL) receives the number of kernels enqueued.  Returns the first
 * validation or launch error (nothing is enqueued after a validation error
 * of any request). */
mmsar_status mmsar_image_batch_fused(const mmsar_request *reqs, int n, void *stream, int *launches);

/* Read (and clear) the device error word of the last call that used this
 * workspace: synchronises `stream`, returns MMSAR_OK or the first device-side
 * condition (MMSAR_ERR_NONFINITE, MMSAR_ERR_INVALID_ARG for Z_c <= 0).
 * workspace == NULL reads the built-in scratch area of mmsar_image_static on
 * the current device (the error word of the last static call there). */
mmsar_status mmsar_poll_error(const void *workspace, void *stream);

/* Peak voxel of a complex64 volume (utility; Sec. V compares images by
 * their peaks): writes to `result` (device) an int64 linear index -- the
 * lowest index whose |o| is within 1e-6 (relative) of the maximum -- followed
 * by the float maximum |o|.  `scratch` (device) must hold
 * mmsar_peak_scratch_bytes(n) bytes.  n >= 1. */
size_t mmsar_peak_scratch_bytes(int64_t n);
mmsar_status mmsar_peak(const void *vol, int64_t n, void *scratch, void *result, void *stream);

/* Imaging without a caller-provided workspace (the paper has no
 * counterpart; this is a deployment convenience).  For callers that cannot
 * allocate device memory while they run -- hard real-time acquisition loops
 * that forbid blocking or failing allocations after start-up, plug-ins that
 * only receive buffers from their host -- this call runs mmsar_image on a
 * scratch area built into the library: a fixed device array of
 * mmsar_static_workspace_bytes() bytes (32 MiB) that every GPU using the
 * library holds until the process exits.  Arguments as for mmsar_image; the
 * caller still passes inputs and the output.  Plans whose workspace exceeds
 * the area are rejected with MMSAR_ERR_UNSUPPORTED_SIZE.  A call made outside
 * stream capture looks up the area's device address on the current device
 * (so a device reset, which may move it, is followed correctly) and keeps
 * it; a call made while `stream` is being captured uses the address kept by
 * the last plain call on that device and fails with MMSAR_ERR_INVALID_ARG if
 * there was none, so make one plain call on each device before any stream
 * capture (and again after a device reset).  All calls on a device share the
 * area: calls that overlap on the GPU race on it, so serialise them.  The
 * device error word of the last call is read with
 * mmsar_poll_error(NULL, stream).  No device memory is allocated. */
size_t mmsar_static_workspace_bytes(void);
mmsar_status mmsar_image_static(mmsar_plan *plan, const void *echo, const float *echo_scale,
                                const double *pos, const double *tx, const double *rx,
                                void *vol, void *stream);

/* Reduced-precision echo storage (a storage choice of this library; the
 * paper keeps full precision).  Converts the complex64 echo echo_c64 (device,
 * n_complex values, 16-byte aligned) into interleaved FP16 or BF16 pairs in
 * `out` (device, 4 * n_complex bytes) and writes the per-scan scale to
 * `scale` (device float): scale = max(|Re|, |Im|) / 16384 (1 for an all-zero
 * echo), out = round(echo / scale).  Pass `out` and `scale` to mmsar_image on
 * a plan with the matching dtype; the arithmetic there is FP32.  `scratch` is
 * one device int (overwritten).  Stream-ordered. */
mmsar_status mmsar_quantize_echo(const void *echo_c64, int64_t n_complex, mmsar_echo_dtype dtype,
                                 void *out, float *scale, int *scratch, void *stream);

/* Thread-local text of the last error returned on this thread. */
const char *mmsar_last_error(void);

/* Release a plan (NULL is ignored). */
void mmsar_plan_destroy(mmsar_plan *plan);

/* Library version string. */
const char *mmsar_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MMSAR_H */

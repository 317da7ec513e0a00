/*
 * dos.h - C ABI of the GB300 (sm_103a) engine for the forward model and the
 * gradient of wavelength-multiplexed diffractive optical storage
 * (Shen, Li, Isil et al., arxiv 2604.02624).
 *
 * The engine evaluates, for N_w independent wavelength channels at once, the
 * cascade of Section 4 of the paper:
 *
 *   u_0      = 1 on the centred A x A input aperture, 0 elsewhere (N x N)
 *   v_1      = P_{z_0}(u_0)
 *   u_l      = t_l * v_l,   t_l = exp(-2 pi kappa h/lambda)
 *                                  * exp(-j 2 pi (n - n_medium) h / lambda)   (Eq. 1)
 *              with h = h_l + h_base                                            (Eq. 2)
 *   v_{l+1}  = P_{z_l}(u_l),  l = 1..K                                          (Eq. 5)
 *   o        = central F x F window of v_{K+1},   I = |o|^2                     (Section 2)
 *
 * where P_z is free-space propagation by the angular-spectrum transfer
 * function of the Rayleigh-Sommerfeld impulse response of Eq. 4,
 *   P_z(u) = crop_N( IDFT_M( H_z * DFT_M( zero_pad_M(u) ) ) ),
 *   H_z(fx, fy) = exp(j 2 pi z sqrt((n_medium/lambda)^2 - fx^2 - fy^2)),
 * fx, fy the DFT bin frequencies of an M-point grid of pitch Delta, and for
 * evanescent bins exp(-2 pi z sqrt(fx^2 + fy^2 - (n_medium/lambda)^2)) (or 0).
 * The objective is the MSE between I and per-channel targets (Section 2) and
 * the gradient with respect to every thickness pixel is the adjoint of the
 * cascade, summed over the channels that share the layers.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Lengths are in metres (pitch, gaps, wavelengths, thickness).
 *  - Arrays are C-contiguous, row-major; images are [row y][column x].
 *  - "d_" pointers are CUDA device pointers on the context's device; they are
 *    owned by the caller, must stay valid until the work queued on the
 *    context's stream has finished, and are never freed by the library.
 *  - "h_" pointers are host pointers, read during the call only.
 *  - Complex arrays are interleaved (re, im) float pairs.
 *  - All work is queued on the context's CUDA stream; calls return before the
 *    GPU finishes unless stated otherwise.
 *  - A context is not thread-safe; use one context per host thread / stream.
 *  - Every int-returning call returns DOS_OK (0) or one of DOS_ERR_*; no C++
 *    exception crosses the ABI. dos_last_error(ctx) describes the last failure
 *    of the calling thread.
 */
#ifndef DOS_H_
#define DOS_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define DOS_API __attribute__((visibility("default")))
#else
#define DOS_API
#endif

/* Status codes. */
enum {
  DOS_OK = 0,
  DOS_ERR_ARG = 1,         /* invalid argument or unsupported size           */
  DOS_ERR_OOM = 2,         /* device or host allocation failed               */
  DOS_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed    */
  DOS_ERR_STATE = 4,       /* call out of order (e.g. backward w/o forward)  */
  DOS_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up             */
  DOS_ERR_UNSUPPORTED = 6  /* valid request that this build cannot serve     */
};

/* Evanescent bins of the transfer function (q < 0). */
enum { DOS_EVAN_DECAY = 0, DOS_EVAN_ZERO = 1 };

/* Objective of dos_loss (Section 2: an MSE between I and the targets). */
enum {
  DOS_LOSS_MSE = 0,        /* mean over channels and FOV pixels of (I - T)^2            */
  DOS_LOSS_MSE_SCALED = 1  /* same with sigma_w I, sigma_w = sum I T / sum I^2 per channel */
};

/*
 * Implementation of the propagation passes.
 *  DOS_PATH_MULTIPASS: a row pass and a column pass kernel per gap over all
 *    channels, row spectra staged in HBM (any supported M).
 *  DOS_PATH_MULTIPASS_BULK: the same passes, but blocks fetch their next item
 *    (a column tile by a TMA tensor copy, or the next channel's rows by
 *    bulk-async copies) into shared memory while computing the current one;
 *    the adjoint row pass stages both the spectra rows and the checkpoint
 *    rows. A pass whose stage does not fit (column: 128 N bytes + exchange
 *    within 227 KB, N <= 256) or whose rows are not 16-byte multiples (odd N)
 *    runs the plain kernel.
 *  DOS_PATH_FUSED: one persistent launch per sweep (forward or adjoint) in
 *    which a thread-block cluster carries one channel at a time through every
 *    gap with the field held in distributed shared memory (needs N <= M/2 and
 *    a compiled cluster configuration for M; see dos_describe).
 *  DOS_PATH_DFT_GEMM: the 2D DFTs as dense complex GEMMs on the tcgen05
 *    tensor cores in split-BF16 (three terms hi*hi + hi*lo + lo*hi, FP32
 *    accumulation in tensor memory), channels processed in chunks; only on
 *    request (it trades accuracy, ~1e-5..1e-4, and speed for tensor cores).
 *  DOS_PATH_DFT_GEMM_X3: the same with every operand split into three bf16
 *    parts and six products kept (~1e-7 per GEMM, twice the tensor work).
 *  DOS_PATH_AUTO: dos_create times one forward+backward of every available
 *    multi-pass (plain and bulk) / cluster-resident configuration and keeps
 *    the fastest; from per-kernel event times of the plain and the bulk
 *    multi-pass runs it also times the mix that runs the faster kernel of
 *    each pass kind (column, forward row, adjoint row).
 * Environment: DOS_FORCE_CONFIG="multipass", "multipass:bulk",
 * "multipass:bulk[<kinds>]" (<kinds>: col, row_fwd, row_adj joined by '+',
 * the kinds on bulk kernels; under DOS_PATH_AUTO only) or
 * "fused:C<c>:L<lines>" (names as printed by dos_describe) selects a
 * configuration without timing, when it is among the requested path's;
 * DOS_TUNE_CACHE=<file> stores and reuses the autotuner's decision per
 * (device, N, M, K, N_w, F).
 * Fault injection (tests): DOS_INJECT_WAIT_TIMEOUT=1 at dos_create makes the
 * first bulk-prefetch pass that the context launches announce its bytes
 * without copying them, so that the bounded waits of its blocks expire (one
 * second) and the next dos_read_loss reports DOS_ERR_TIMEOUT; later calls
 * run normally.  DOS_INJECT_WAIT_TIMEOUT=2 lets the copies land but makes the
 * odd threads of every block give up their first wait; =3, for a first bulk
 * pass that is a column pass, lets the copies land but makes every thread
 * give up its wait for the transfer-table tile of its block's last item.
 * Both are reported the same way.
 */
enum {
  DOS_PATH_AUTO = 0,
  DOS_PATH_MULTIPASS = 1,
  DOS_PATH_FUSED = 2,
  DOS_PATH_DFT_GEMM = 3,
  DOS_PATH_MULTIPASS_BULK = 4,
  DOS_PATH_DFT_GEMM_X3 = 5
};

typedef struct dos_config {
  int n;              /* N: thickness pixels per side of every layer (Section 4)     */
  int m;              /* M: zero-padded DFT size, M >= N, see dos_supported_m()      */
  int n_layers;       /* K: 1 <= K <= 64 diffractive layers                          */
  int n_lambda;       /* N_w >= 1 wavelength channels handled by this context        */
  int n_lambda_total; /* channels of the whole design (loss normalisation); 0 = N_w  */
  int fov;            /* F: output field of view side, N - F even, 1 <= F <= N       */
  int aperture;       /* A: input aperture side, N - A even; 0 means A = F            */
  double pitch;       /* Delta: sampling period = feature size [m] (Section 4)       */
  const double *gaps; /* K+1 distances [m]: input->L1, L1->L2, ..., LK->output (>= 0) */
  const double *lambda;  /* N_w vacuum wavelengths [m] (> 0)                          */
  const double *n_index; /* N_w real parts n(lambda) of the layer index (Eq. 1)       */
  const double *kappa;   /* N_w extinction coefficients kappa(lambda); NULL = all 0   */
  double n_medium;    /* index of the medium between layers (Eq. 1 n_air, Eq. 4 n); > 0 */
  double h_base;      /* base thickness of Eq. 2 [m], added to every pixel            */
  int evanescent;     /* DOS_EVAN_DECAY or DOS_EVAN_ZERO                               */
  int loss;           /* DOS_LOSS_MSE or DOS_LOSS_MSE_SCALED                           */
  int path;           /* DOS_PATH_*                                                    */
  int detector_bin;   /* b: one detector pixel integrates b x b simulation pixels of the
                         F x F output (Section 4: the FOV is divided into output pixels);
                         0 or 1 = score simulation pixels; b > 1 must divide F        */
} dos_config;

typedef struct dos_ctx dos_ctx;

/*
 * Sizes M accepted by this build (the padded DFT length); writes up to `cap`
 * of them to `out` and returns how many there are.  Host-only, no GPU needed.
 */
DOS_API int dos_supported_m(int *out, int cap);

/*
 * Creates a context on the current CUDA device for the design of `cfg`
 * (Section 4 geometry), binding it to `cuda_stream` (a cudaStream_t, may be
 * NULL for the legacy default stream).  Copies every array of `cfg`.
 * Allocates the device workspace (spectra, per-layer field checkpoints, the
 * transfer-function tables H_z for every distinct gap and wavelength, computed
 * here with an FP64 phase, and the aperture spectrum) and synchronises the
 * stream once.  On failure *out is NULL and nothing stays allocated.
 * Errors: DOS_ERR_ARG (sizes / values), DOS_ERR_OOM, DOS_ERR_CUDA.
 */
DOS_API int dos_create(dos_ctx **out, const dos_config *cfg, void *cuda_stream);

/* Rebinds the context to another stream (the caller orders the two streams). */
DOS_API int dos_set_stream(dos_ctx *ctx, void *cuda_stream);

/*
 * Forward model, Section 4 Eq. 1-5: every channel through the K layers.
 *   d_h  [K][N][N] float32 thickness h_l (learnable part of Eq. 2) [m].
 *   d_I  [N_w][F][F] float32 output intensities |o|^2, or NULL to skip.
 *   save_for_backward: nonzero keeps the incoming field of every layer
 *        (K x N_w x N x N complex64 in the workspace) and a copy of d_h
 *        (K x N x N float32) for dos_backward.
 * The complex output fields o are always kept (dos_loss, dos_backward and
 * dos_output_field read them).  Errors: DOS_ERR_ARG (NULL d_h), DOS_ERR_CUDA.
 */
DOS_API int dos_forward(dos_ctx *ctx, const float *d_h, float *d_I, int save_for_backward);

/*
 * Objective of the last forward (Section 2: MSE between O_w = |o_w|^2 and its
 * target, over all channels), with the per-channel PSNR.  The detector reads
 * D_w = O_w summed over blocks of b x b simulation pixels (b = detector_bin,
 * D = O for b <= 1); F_d = F / b detector pixels per side.
 *   d_T     [N_w][F_d][F_d] float32 targets (required).
 *   h_loss  host double receiving L; when non-NULL the call waits for the
 *           stream.  When NULL, L stays on the device (dos_read_loss).
 *   d_psnr  [N_w] float32: 10 log10(1 / mean_p (sigma_w D - T)^2), sigma_w the
 *           least-squares scale sum D T / sum D^2; NULL to skip.
 *   d_dLdI  [N_w][F][F] float32 gradient dL/dI of the configured loss with
 *           respect to the simulation-pixel intensities; NULL to skip.
 * L is normalised by n_lambda_total * F_d^2 so that shards of one design add up.
 * Errors: DOS_ERR_STATE (no forward yet), DOS_ERR_ARG, DOS_ERR_CUDA.
 */
DOS_API int dos_loss(dos_ctx *ctx, const float *d_T, double *h_loss, float *d_psnr,
                     float *d_dLdI);

/*
 * Largest n_lambda that dos_loss_noalloc accepts: its scratch is a fixed
 * array of DOS_NOALLOC_MAX_LAMBDA per-channel records of 32 bytes (2 MiB)
 * plus one double, held by every GPU that loads this library until exit.
 */
#define DOS_NOALLOC_MAX_LAMBDA 65536

/*
 * Scoring without any memory allocation (the paper has no counterpart: this
 * serves callers that cannot allocate device memory, e.g. code inside a
 * framework that owns all device memory through its own pool or runs under a
 * fixed budget, or a path where a cudaMalloc would stall the device).
 * Computes what dos_loss computes with detector_bin = 1, from caller
 * intensities instead of a context, using only a fixed-size scratch array in
 * the library itself (a caller with detector pixels passes their sums).
 *   d_I, d_T  [n_lambda][fov][fov] float32 intensities and targets.
 *   n_lambda  1..DOS_NOALLOC_MAX_LAMBDA; larger values fail with DOS_ERR_ARG.
 *   n_lambda_total, loss: as in dos_config; h_loss, d_psnr, d_dLdI: as in
 *   dos_loss (h_loss may be NULL; then the loss is not read back).
 *   cuda_stream  stream of the caller's device (NULL: legacy default stream).
 * The first call on each device (with that device current) looks up the
 * scratch address, and so does the first call under another CUDA context of
 * that device (a primary context recreated after cudaDeviceReset, a driver
 * context the caller made current); make such a first call before any stream
 * capture.  Calls allocate nothing: no cudaMalloc, cudaFree or allocating
 * library routine.
 * Every call on a device shares the same scratch, which keeps the contents
 * of the last call (each call overwrites what it reads, nothing has to be
 * cleared): calls that overlap on the GPU (other streams, other threads)
 * race and must be serialised by the caller.
 * Errors: DOS_ERR_ARG, DOS_ERR_CUDA, DOS_ERR_UNSUPPORTED (device index > 63);
 * the message is in dos_last_error(NULL).
 */
DOS_API int dos_loss_noalloc(const float *d_I, const float *d_T, int n_lambda, int fov,
                             int n_lambda_total, int loss, double *h_loss, float *d_psnr,
                             float *d_dLdI, void *cuda_stream);

/*
 * Misaligned layers (Section 3, "vaccination" against lateral and axial
 * displacements during training).  h_disp [K][3] holds the displacement
 * (dx, dy, dz) [m] of layers 1..K, or NULL to restore the aligned design.
 * The input aperture and the output plane stay fixed.  A layer displaced by D
 * modulates with t(r - D); as free space is shift invariant this equals
 * giving gap g the transfer function
 *   H(z_g + dz_{g+1} - dz_g) * exp(-2 pi j (fx a_x + fy a_y)),  a = D_g - D_{g+1},
 * which is how the engine applies it (exact up to the layer window).
 * Applies to every later dos_forward / dos_backward / dos_step / dos_propagate
 * until changed; a backward must follow a forward with the same setting.
 * The first call builds a table of sqrt(|q|) (N_w (M/2+1)^2 floats, FP64 roots).
 * Errors: DOS_ERR_ARG, DOS_ERR_OOM, DOS_ERR_CUDA.
 */
DOS_API int dos_set_misalignment(dos_ctx *ctx, const double *h_disp);

/*
 * Output diffraction efficiency of every channel of the last forward (Section
 * 2, Figs. 5-6): eta_w = sum over the FOV of |o_w|^2 divided by the power of
 * the unit-amplitude input aperture (A^2).  d_eta [N_w] float32.
 * Errors: DOS_ERR_STATE (no forward yet), DOS_ERR_ARG, DOS_ERR_CUDA.
 */
DOS_API int dos_efficiency(dos_ctx *ctx, float *d_eta);

/*
 * Phase bit depth B of the diffractive features (Section 2, Fig. 7): every
 * thickness, limited to [0, h_max], is replaced by the nearest of the 2^B
 * levels k h_max / (2^B - 1).  The level index is decided in FP32:
 * k = rint(fp32(clamp(h)) * fp32((2^B - 1) / h_max)), value k * fp32(h_max / (2^B - 1)).
 *   d_h, d_hq  `count` float32 values (may alias); h_max > 0 [m]; 1 <= bits <= 24.
 *   cuda_stream  stream to queue on (NULL: legacy default stream).
 * Errors: DOS_ERR_ARG, DOS_ERR_CUDA.
 */
DOS_API int dos_quantize_thickness(const float *d_h, float *d_hq, size_t count, double h_max, int bits,
                                   void *cuda_stream);

/*
 * Copies the loss of the last dos_loss to *h_loss (waits for the stream).
 * Returns DOS_ERR_TIMEOUT when a kernel queued since the previous check gave
 * up a bounded wait (bulk-copy or tensor-core completion); the loss and every
 * result of that work are then invalid.  The flag is cleared by the report.
 */
DOS_API int dos_read_loss(dos_ctx *ctx, double *h_loss);

/*
 * Gradient of a real objective with respect to the thickness, by the adjoint
 * of Eq. 1-5 (error back-propagation, Section 2), summed over the channels.
 *   d_dLdI [N_w][F][F] float32 dL/dI for the last forward's intensities.
 *   d_dLdh [K][N][N] float32, overwritten with dL/dh_l [1/m].
 * Needs the last dos_forward (or dos_step) to have had save_for_backward != 0:
 * the adjoint reads that forward's layer fields and rebuilds the layers'
 * transmissions t(h) from the copy of its thickness the context kept, so the
 * caller may change its d_h buffer in between.
 * The sum over channels has a fixed order: results are bitwise reproducible.
 * Errors: DOS_ERR_STATE (no saved forward), DOS_ERR_ARG (NULL pointer), DOS_ERR_CUDA.
 */
DOS_API int dos_backward(dos_ctx *ctx, const float *d_dLdI, float *d_dLdh);

/*
 * One design step: dos_forward(save) + dos_loss + dos_backward, replayed as a
 * CUDA graph.  The first call for a given set of pointers captures the step
 * on a stream private to the context (ordered after the context's stream by
 * an event, and the context's stream after it); later calls with the same
 * pointers replay the graph.
 *   d_h [K][N][N], d_T [N_w][F_d][F_d] inputs; d_dLdh [K][N][N] output (all required).
 *   d_I [N_w][F][F] and d_psnr [N_w] optional outputs (NULL to skip).
 *   h_loss: when non-NULL receives L (waits for the stream).
 * Afterwards the context holds the same state as after the three calls.
 * Errors: DOS_ERR_ARG, DOS_ERR_CUDA.
 */
DOS_API int dos_step(dos_ctx *ctx, const float *d_h, const float *d_T, float *d_dLdh, float *d_I,
                     float *d_psnr, double *h_loss);

/*
 * Copies the complex output field o of the last forward, [N_w][F][F] complex64
 * (interleaved floats), to d_o.  Errors: DOS_ERR_STATE, DOS_ERR_ARG, DOS_ERR_CUDA.
 */
DOS_API int dos_output_field(dos_ctx *ctx, float *d_o);

/*
 * Copies the incoming field v_l of layer `layer` (1..K, before its
 * modulation) saved by the last dos_forward(save_for_backward != 0),
 * [N_w][N][N] complex64, to d_v.  Errors: DOS_ERR_STATE, DOS_ERR_ARG, DOS_ERR_CUDA.
 */
DOS_API int dos_layer_field(dos_ctx *ctx, int layer, float *d_v);

/*
 * One free-space propagation P_z (Eq. 4-5, angular spectrum) of caller
 * fields over gap `gap` (0..K) for every channel, or its adjoint (the same
 * chain with conj(H)) when `adjoint` is nonzero.
 *   d_in, d_out [N_w][N][N] complex64; may not alias.
 * Errors: DOS_ERR_ARG, DOS_ERR_CUDA.
 */
DOS_API int dos_propagate(dos_ctx *ctx, int gap, const float *d_in, float *d_out, int adjoint);

/* Kernel kinds reported by dos_kernel_time. */
enum {
  DOS_KERNEL_COLUMN_FORWARD = 0,  /* column pass: DFT, H, IDFT              */
  DOS_KERNEL_COLUMN_ADJOINT = 1,  /* column pass with conj(H)               */
  DOS_KERNEL_ROW_FORWARD = 2,     /* row pass: IDFT, Eq. 1 modulation, DFT  */
  DOS_KERNEL_ROW_ADJOINT = 3,     /* adjoint row pass with dL/dh partials   */
  DOS_KERNEL_ROW_OUTPUT = 4,      /* output plane: o, I                     */
  DOS_KERNEL_ROW_SEED = 5,        /* adjoint seed 2 dL/dI o                 */
  DOS_KERNEL_LOSS = 6,            /* objective, PSNR, dL/dI                 */
  DOS_KERNEL_GRAD_REDUCE = 7,     /* fixed-order sum of dL/dh partials      */
  DOS_KERNEL_FUSED_FORWARD = 8,   /* cluster-resident forward sweep         */
  DOS_KERNEL_FUSED_ADJOINT = 9,   /* cluster-resident adjoint sweep         */
  DOS_KERNEL_GEMM_PROPAGATION = 10, /* one split-BF16 DFT-GEMM propagation (4 GEMMs + 5 conversions) */
  DOS_KERNEL_GEMM_FIELD = 11,     /* field conversions / seed / adjoint layer of the GEMM path */
  DOS_KERNEL_KINDS = 12
};

/*
 * Per-kernel timing with CUDA events recorded on the context's stream around
 * every launch (enable != 0 starts it and clears the totals; 0 stops it).
 */
DOS_API int dos_set_timing(dos_ctx *ctx, int enable);

/*
 * Launch count and total device time [ms] of kernel kind `kind` since timing
 * was enabled.  Waits for the stream.  Errors: DOS_ERR_ARG, DOS_ERR_CUDA.
 */
DOS_API int dos_kernel_time(dos_ctx *ctx, int kind, int *launches, double *ms);

/* Bytes of device memory held by the context. */
DOS_API size_t dos_workspace_bytes(const dos_ctx *ctx);

/* Number of kernel launches queued by the last dos_forward / dos_loss / dos_backward. */
DOS_API int dos_last_launch_count(const dos_ctx *ctx);

/* Implementation chosen for the context (DOS_PATH_MULTIPASS, _MULTIPASS_BULK, _FUSED, _DFT_GEMM or _DFT_GEMM_X3). */
DOS_API int dos_path(const dos_ctx *ctx);

/*
 * Writes a NUL-terminated, human-readable description of the chosen
 * implementation (path, cluster size, threads, clusters in flight) and of the
 * autotuner's timings to buf (at most cap bytes).  Returns the full length.
 */
DOS_API int dos_describe(const dos_ctx *ctx, char *buf, int cap);

/* Frees every resource of the context (waits for its stream).  NULL is a no-op. */
DOS_API void dos_destroy(dos_ctx *ctx);

/*
 * Message for the last failing call of the calling thread ("" if none).  ctx
 * may be NULL (a failed dos_create has no context); the message is the
 * thread's, which for a context used from one thread is that context's.
 */
DOS_API const char *dos_last_error(const dos_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* DOS_H_ */

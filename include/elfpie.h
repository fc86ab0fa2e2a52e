/*
 * elfpie.h - C ABI of the GB300-native Elfpie gradient step.
 *
 * Elfpie (arXiv 2209.14671) reconstructs the high-resolution spectrum Psi of a
 * sample and the pupil P of the objective from K low-resolution intensity
 * images, one per LED, by minimising Eq. 8 (an L1 fidelity on spatial gradients,
 * Eq. 5 or Eq. 4, plus a Hessian total-variation penalty on amplitude and phase,
 * Eqs. 6-7) with the modified AdaBelief update of Eq. 19.  One call of
 * elf_step(h, 1) is one outer iteration of Algorithm 1 over all K LEDs.
 *
 * Conventions shared by every entry point
 *  - Return value: ELF_OK (0) or a negative ELF_E* code; elf_last_error() gives
 *    a message for the calling thread's last failure.
 *  - Complex arrays are interleaved float pairs (re, im), row-major [y][x].
 *    Spectra (Psi, pupil) are centred: zero frequency at index (N/2, N/2) of the
 *    N x N spectrum and (n/2, n/2) of the n x n pupil.  Objects are spatial
 *    fields with the usual (0, 0) origin.
 *  - Buffers passed in are caller-owned; the library copies from them before the
 *    call returns (or, for device buffers, in stream order) and keeps no pointer.
 *    Buffers passed out are filled by the call.  "is_device" says whether a
 *    pointer is device memory (1) or host memory (0); unified addressing makes
 *    either work, the flag only documents intent.
 *  - All device work of a handle is ordered on the CUDA stream given at
 *    elf_create (0 = the legacy default stream).  elf_step returns without
 *    synchronising; every elf_get_* call synchronises that stream.
 *  - A handle is not thread-safe; distinct handles are independent.
 *  - The LED order given at elf_create fixes every summation order, so results
 *    are bitwise reproducible run to run on the same GPU.
 *  - The library allocates its device memory in elf_create (cudaMalloc) and
 *    frees it in elf_destroy.
 */
#ifndef ELFPIE_H
#define ELFPIE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ELF_OK = 0,
  ELF_EINVAL = -1,    /* invalid argument or problem (crop outside the grid, unsupported size, K = 0, NaN input) */
  ELF_ENOMEM = -2,    /* device allocation failed */
  ELF_ECUDA = -3,     /* a CUDA runtime call failed; see elf_last_error() */
  ELF_ENUMERIC = -4,  /* a non-finite cost was produced */
  ELF_ETIMEOUT = -5,  /* a bounded device wait ran out (a DSMEM exchange of the tile kernel or the
                         tensor-core path); the results are invalid */
  ELF_ESTATE = -6     /* call out of order (e.g. elf_step before elf_set_measurements) */
};

typedef struct elf_handle_s* elf_handle;

/* Imaging geometry of Sec. 3.1 / Eq. 1 (sequential FPM, M = 1).
 * The spectral pixel is dk = 1 / (n_lowres * pixel_um) cycles/um on both grids.
 * LED n is placed at the centred offset c_n = round-half-away(k_n / dk) and its
 * crop window is rows/cols [N/2 + c - n/2, N/2 + c + n/2), which must lie in
 * [0, N).  The pupil support is {j : |j - n/2|^2 dk^2 <= (na / wavelength_um)^2}. */
typedef struct {
  int n_lowres;           /* n: low-res image side; 16, 32, 64, 128 or 256 */
  int upsample;           /* u >= 1; N = u * n must be 32..1024 and a power of two */
  int n_led;              /* K >= 1 */
  const float* k_xy;      /* [K][2] (kx, ky) illumination spatial frequency, cycles/um; host, copied */
  double na;              /* objective numerical aperture (> 0) */
  double wavelength_um;   /* illumination wavelength (> 0) */
  double pixel_um;        /* low-res pixel size at the sample plane (> 0) */
  int n_mux;              /* M, LEDs lit together per measured image (Eq. 1); 0 or 1 = sequential FPM.
                             Image j is lit by LEDs jM .. jM+M-1 (caller order); K must be a multiple
                             of M and the measurements hold K/M images.  M > 1 needs tile_dft = 0. */
} elf_problem;

/* Hyper-parameters (Sec. 6.2) and the smoothing constants of the readings. */
typedef struct {
  int fidelity;      /* 0 = intensity (Eqs. 5, 11; default), 1 = amplitude (Eqs. 4, 10); Sec. 6.3 scaling maps
                        of Eq. 3: 2 = power g(x) = x^g_exponent, 3 = log g(x) = ln(x + 1).  For 2 and 3 the
                        residual is g(|o|^2) - g(max(I, 0)), W = g'(|o|^2) o nabla^T omega with |o| floored
                        at eta_h in g' of the power map, and Eqs. 16-17 take g(max(I, 0)). */
  int omega_iso;     /* 1 = isotropic normaliser of Eq. 12 (default), 0 = anisotropic */
  int learn_pupil;   /* 1 = update P with Eq. 18 + Eq. 19 (default) */
  int pupil_filter;  /* 1 = 3x3 Gaussian (sigma 1 px) on P before its update (note under Algorithm 1) */
  double alpha;      /* Hessian amplitude weight of Eq. 8; < 0 = automatic (Eq. 16/17) */
  double beta;       /* Hessian phase weight of Eq. 8; < 0 = automatic (Eq. 16/17) */
  double gamma1;     /* Eq. 19 first-moment decay (0.9) */
  double gamma2;     /* Eq. 19 belief decay (0.999) */
  double s0_psi;     /* initial step of Psi: delta^0 = s0^2 (1) */
  double s0_pupil;   /* initial step of P (1e-2) */
  double eta_opt;    /* Eq. 19 eta (1e-8) */
  double eta_h;      /* Eq. 14 eta and the |O| floor of Eq. 13 (1e-12) */
  double tau_fid;    /* smoothing radius of the L1 fidelity (1e-6) */
  double tau_h;      /* smoothing radius of the Hessian L1 terms (1e-4) */
  int tile_dft;      /* tile transforms: 0 = FP32 FFT (default); 1 = tensor-core DFT, BF16 3-term split with
                        FP32 accumulation (not in the paper; n_lowres = 128 with the support band <= 64 only) */
  double g_exponent; /* gamma of the power map (fidelity 2), in (0, 8]; 1 by default (Sec. 6.3) */
  int tile_path;     /* kernels of the FP32 tile work (same arithmetic): 0 = automatic (default: 2 for n_lowres >= 128,
                        else 1), 1 = one thread-block
                        cluster per LED, the tile kept on chip; 2 = three kernels per iteration (inverse row
                        transforms, column transforms + the stencil of Eqs. 5, 12, 11, forward row transforms) that
                        pass each LED's support band through device memory (2 K nb n complex more, nb = support
                        rows).  2 needs n_mux = 1 and tile_dft = 0. */
} elf_options;

/* Full optimiser state of Eq. 19 for Psi and P (Algorithm 1 keeps nothing else).
 * Every pointer is caller-owned.  Sizes: psi, mu_psi [N][N][2] float;
 * v_psi, delta_psi [N][N] float; pupil, mu_pupil [n][n][2]; v_pupil, delta_pupil [n][n].
 * t is the number of completed iterations. */
typedef struct {
  float* psi; float* mu_psi; float* v_psi; float* delta_psi;
  float* pupil; float* mu_pupil; float* v_pupil; float* delta_pupil;
  int t;
  double alpha;
  double beta;
} elf_state;

/* Fills *o with the defaults listed above. */
int elf_default_options(elf_options* o);

/* Validates the problem, precomputes LED offsets, the pupil support and the
 * gather lists, and allocates all device memory (inputs, state, scratch).
 * opt may be NULL (defaults).  cuda_stream is a cudaStream_t (may be NULL). */
int elf_create(const elf_problem* prob, const elf_options* opt, void* cuda_stream, elf_handle* out);

/* Copies the K/M measured images I [K/M][n][n] float (host or device; M = n_mux,
 * one image per LED when M = 1) into the handle, estimates alpha = beta with
 * Eq. 16 (Eq. 17 for the amplitude fidelity) over those images when the options
 * ask for it, and initialises the state: Psi0 = u^2 * centred DFT of
 * sqrt(max(I_c, 0)) of the image holding the LED nearest the axis, Nyquist
 * row/column zeroed, placed at that LED's window; P0 = 1 on the support;
 * mu = v = 0; delta = s0^2; t = 0.  Non-finite input -> ELF_EINVAL. */
int elf_set_measurements(elf_handle h, const float* I, int is_device);

/* Runs n_iter outer iterations of Algorithm 1 (Eqs. 9-19) asynchronously. */
int elf_step(elf_handle h, int n_iter);

/* ---- LED sharding of one iteration --------------------------------------------------------
 * The fidelity gradient is a sum over LEDs (Eq. 9 for Psi, Eq. 18 for P) of terms that each need
 * only that LED's image and crop (Sec. 3.4), so handles of the same problem in several processes
 * (or on several GPUs), each holding all the measurements and the same state, can share the LED
 * work of an iteration.  elf_step(h, 1) is, in order:
 *   elf_shard_tiles(h, k0, k1)   the tile work (Eqs. 1, 5 or 4, 12, 11 or 10, F_B^H of Eq. 9) of
 *                                LEDs [k0, k1), plus the LED-free parts that precede the sums: the
 *                                Hessian branch (Eqs. 6-7, 13-14) and Eq. 19 for P off the support;
 *   elf_shard_import(h, ...)     for every other block of LEDs, its results from the handle that
 *                                computed it (elf_shard_export there);
 *   elf_shard_finish(h)          the sums over all K LEDs in LED order and the rest of the
 *                                iteration: Eq. 9 + Eq. 19 for Psi, Eq. 18 + the filter + Eq. 19
 *                                for P, the Eq. 8 costs, t += 1.
 * The per-LED results are exchanged unsummed and every sum over LEDs runs after the exchange in
 * LED order, so every handle ends the iteration in a state bitwise equal to elf_step(h, 1), for
 * any partition of [0, K) into blocks.  Exported block of LEDs [k0, k1) (caller-owned, host or
 * device, elf_shard_row_floats(h) floats per LED): (k1 - k0) * S complex tile gradients G_n on the
 * support (LED-major, in the support order of elf_get_support), then (k1 - k0) * C float pairs of
 * fidelity cost partials (C per LED, the tile kernel's cluster size).  All calls are ordered on
 * the handle's stream; export into host memory synchronises it.  Sequential FPM (n_mux = 1) with
 * tile_dft = 0 only (else ELF_EINVAL); elf_step, elf_cost_grad and elf_set_state return
 * ELF_ESTATE between elf_shard_tiles and elf_shard_finish. */
int elf_shard_row_floats(elf_handle h);
int elf_shard_tiles(elf_handle h, int led_begin, int led_end);
int elf_shard_export(elf_handle h, int led_begin, int led_end, float* dst, int is_device);
int elf_shard_import(elf_handle h, int led_begin, int led_end, const float* src, int is_device);
int elf_shard_finish(elf_handle h);

/* Object O = IDFT_N(ifftshift(Psi)) (Algorithm 1 output), [N][N][2] float. */
int elf_get_object(elf_handle h, float* obj, int is_device);
/* Current pupil P, [n][n][2] float (zero outside the support). */
int elf_get_pupil(elf_handle h, float* pupil, int is_device);
/* Current centred spectrum Psi, [N][N][2] float. */
int elf_get_spectrum(elf_handle h, float* psi, int is_device);
/* Per-iteration FP64 costs (L_fid, L_A, L_Phi) of Eq. 8 evaluated at the state
 * each iteration started from, oldest first, for the last min(t, max_iter, 4096)
 * iterations, into out [count][3] (host).  Returns count (>= 0) or an error. */
int elf_get_costs(elf_handle h, double* out, int max_iter);
/* Per-iteration FP64 norms (||g||, ||Delta Psi||) of the Psi update of Eq. 19: g = dL/dconj(Psi) of
 * Eq. 8 (Eq. 9 plus Eqs. 13-15) at the state the iteration started from, Delta Psi = Psi^(t+1) - Psi^t,
 * both summed over the N x N spectrum in a fixed order.  Oldest first, for the last min(t, max_iter,
 * 4096) iterations (t counts iterations since elf_set_measurements, or from the t of elf_set_state),
 * into out [count][2] (host).  Returns count (>= 0) or an error (ELF_ENUMERIC for a non-finite norm). */
int elf_get_norms(elf_handle h, double* out, int max_iter);
/* Self-test of the failure path of the library's bounded device waits (the tile kernels' cluster
 * exchanges wait on mbarriers with a poll limit; a wait that runs out sets the handle's error flag,
 * after which the getters return ELF_ETIMEOUT).  Runs one warp that waits on a barrier phase nothing
 * completes, with `limit` polls (1 .. 2^30), on the handle's stream: the wait runs out, sets the flag
 * and the kernel returns, leaving the device usable.  The handle then reports ELF_ETIMEOUT from its
 * getters for good (destroy it).  *ms (may be null) gets the kernel's duration. */
int elf_selftest_wait_timeout(elf_handle h, long long limit, double* ms);
/* Copies the optimiser state out / in (checkpoint and resume). */
int elf_get_state(elf_handle h, const elf_state* out, int is_device);
int elf_set_state(elf_handle h, const elf_state* in, int is_device);

/* Evaluates the cost of Eq. 8 and its Wirtinger gradients dL/d(conj Psi)
 * (Eq. 15 = Eq. 9 + alpha Eq. 13 + beta Eq. 14) and dL/d(conj P) (Eq. 18) at the
 * given (psi [N][N][2], pupil [n][n][2]) with the handle's measurements, alpha and
 * beta, without touching the optimiser state.  costs4 (host, 4 doubles) receives
 * (L_fid, L_A, L_Phi, L) in FP64, L = L_fid + alpha L_A + beta L_Phi of Eq. 8
 * summed on the device; g_psi / g_pupil (same layouts) may be NULL. */
int elf_cost_grad(elf_handle h, const float* psi, const float* pupil, double* costs4,
                  float* g_psi, float* g_pupil, int is_device);

/* Forward model of Eq. 1 for data synthesis: I_j = sum over the M LEDs of image j
 * of |o|^2 (|o_n|^2 per LED when M = 1) for the handle's geometry, from the spatial
 * object obj [N][N][2] and the unit pupil on the support.  Writes I_out [K/M][n][n]
 * float. */
int elf_simulate(elf_handle h, const float* obj, float* I_out, int is_device);

/* Inspection: the per-LED tile gradients G_n = u^-2 n^-2 fftshift(DFT_n(W_n))
 * (the F_B^H W_n factor of Eq. 9) of the last elf_step / elf_cost_grad, stored on
 * the pupil support only: G_out [K][S][2] float; the support pixels in that order
 * are given by elf_get_support (linear indices jy*n + jx, ascending). */
int elf_get_tile_grads(elf_handle h, float* G_out, int is_device);
/* Number of support pixels S, and (if idx != NULL) their linear indices [S] (host). */
int elf_get_support(elf_handle h, int* idx);
/* alpha and beta in use (after elf_set_measurements). */
int elf_get_weights(elf_handle h, double* alpha, double* beta);

/* Tracing.  Stages of one iteration, timed with CUDA events recorded on the
 * stream each stage runs on (inside the iteration graph when tracing is on). */
enum {
  ELF_STAGE_ITERATION = 0,     /* the whole iteration */
  ELF_STAGE_TILE = 1,          /* per-LED tile kernel (Eqs. 1, 5, 11, 12, F_B^H of Eq. 9) */
  ELF_STAGE_HESSIAN = 2,       /* O = F_A^-1 Psi, Eqs. 6-7, 13-14, F_A^H (second stream) */
  ELF_STAGE_PUPIL_GRAD = 3,    /* Eq. 18 partial sums; their last blocks apply Eq. 19 to P on the support */
  ELF_STAGE_GATHER = 4,        /* Eq. 9 gather fused with Eq. 19 for Psi */
  ELF_STAGE_PUPIL_UPDATE = 5,  /* Eq. 19 for P off the support (gradient 0), from the iteration start */
  ELF_STAGE_COST = 6,          /* FP64 reduction of Eq. 8's terms */
  ELF_NSTAGES = 7
};
/* enable != 0 records the stage events from the next elf_step on (the graph is
 * rebuilt); adds event nodes only, no extra kernels. */
int elf_set_tracing(elf_handle h, int enable);
/* Durations in ms of each stage of the most recent traced iteration, ms[ELF_NSTAGES]
 * (-1 for a stage that did not run).  Synchronises.  Returns the count written. */
int elf_get_stage_times(elf_handle h, float* ms, int max_stages);
/* Start and end of each stage of the most recent traced iteration in ms from the iteration's
 * start, spans[2 * stage] and spans[2 * stage + 1] (-1 for a stage that did not run): which
 * stream's chain ends the iteration.  Synchronises.  Returns the count of stages written. */
int elf_get_stage_spans(elf_handle h, float* spans, int max_stages);
/* Number of kernel launches in one iteration (kernel nodes of the iteration graph). */
int elf_graph_kernel_count(elf_handle h);

/* ---- evaluation of Sec. 4.1 (Eqs. 20-22); device pointers, the call synchronises ---- */

/* Degradation parameters of Eqs. 2 and 20. */
typedef struct {
  double illum_c;      /* c of Eq. 20, in [0, 1]: the illumination factor spans [1 - c, 1]; 0 = none */
  double waist_px;     /* 1/e^2 half-waist w of the Gaussian G of Eq. 20, low-res pixels (15 in Sec. 4.1) */
  double gauss_a;      /* a of Eq. 20, Gaussian form: I += a * xi; 0 = none */
  double snp_density;  /* a of Eq. 20, salt & pepper form, in [0, 1]: u < a/2 -> 0, a/2 <= u < a -> 1 */
} elf_degrade_params;

/* Eqs. 2 and 20 on the handle's image grid with caller-drawn random fields, per image j:
 *   I_out = ((1 - c) + c * N(G (x) zeta_j)) * I_clean + background[j] + a * xi, then salt & pepper,
 * where G (x) is the circular convolution with exp(-2 r^2 / w^2) normalised to unit sum and N the
 * min-max normalisation to [0, 1] of each image (N = 0 for a flat field).  I_clean, zeta, xi,
 * u_snp, I_out: [K/M][n][n] float on the device (I_out may not alias the inputs); background:
 * [K/M] float on the device or NULL; a field may be NULL when its parameter is 0.
 * Errors: ELF_EINVAL for missing fields or parameters out of range; n <= 1024. */
int elf_degrade(elf_handle h, const float* I_clean, const float* zeta, const float* background,
                const float* xi, const float* u_snp, const elf_degrade_params* prm, float* I_out);

/* NL of Eq. 21 in percent: the mean over the handle's dark-field images (every LED of the image
 * with |k| > NA / lambda) of ||I_sim - I_noised||_1 / ||I_sim||_1; 0 when there are none.
 * I_sim, I_noised: [K/M][n][n] float on the device.  Writes *nl on the host. */
int elf_noise_level(elf_handle h, const float* I_sim, const float* I_noised, double* nl);

/* LSNR of Eq. 22 in dB: max over b of 10 log10(||truth||^2 / ||truth - (rec + b)||^2), attained
 * at b = mean(truth - rec); sums in FP64.  rec, truth: count floats on the device; cuda_stream
 * may be NULL.  Writes *out on the host. */
int elf_lsnr(const float* rec, const float* truth, long long count, void* cuda_stream, double* out);

/* LSNR (Eq. 22) of the amplitude and of the phase (atan2) of the handle's current object against
 * the true object obj_true [N][N][2] float on the device, after multiplying the reconstruction
 * by the least-squares global phase e^{i phi0}, phi0 = arg sum conj(O) O_true (the global phase
 * is not observable from intensities).  Writes out2[0] (amplitude), out2[1] (phase) on the host. */
int elf_object_quality(elf_handle h, const float* obj_true, double* out2);

/* ---- Serving: continuous batching of independent reconstructions ----------
 * (Not in the paper.)  A server admits queued requests in arrival order while a
 * device-memory budget and a slot count allow, runs every admitted request's
 * whole job (measurements upload, initial state, n_iter iterations, object) on
 * its own stream so that jobs overlap on the device, and retires finished jobs
 * without blocking.  Handles are pooled per (problem, options) and reused; idle
 * pooled handles are freed, least recently used first, when a new shape needs
 * room.  A request's result is bitwise the same as a lone run of the same job. */
typedef struct elf_server_s* elf_server;

/* budget_bytes: device memory the server may hold; max_active: concurrent jobs. */
int elf_server_create(size_t budget_bytes, int max_active, elf_server* out);
/* Queues a request.  I [K][n][n] float (host; pinned memory makes the upload
 * asynchronous) is NOT copied: it must stay valid and unchanged until the
 * request's result has been collected.  tag identifies the request (unique among
 * unfinished and uncollected ones).  A problem that cannot fit the budget even
 * alone -> ELF_ENOMEM.  Non-finite inputs are not checked here. */
int elf_server_submit(elf_server s, const elf_problem* prob, const elf_options* opt, const float* I, int n_iter,
                      long long tag);
/* Non-blocking: retires finished jobs (their tags go to done_tags, at most
 * max_done of them, count in *n_done), then admits queued requests that fit. */
int elf_server_progress(elf_server s, long long* done_tags, int max_done, int* n_done);
/* Copies a finished request's object O [N][N][2] float to host memory and
 * forgets the request.  ELF_ESTATE if it has not finished. */
int elf_server_result(elf_server s, long long tag, float* obj);
/* Withdraws a request: a queued one is dropped; a running one (its whole job is already on the
 * device, which cannot be interrupted) is waited for, its handle kept for reuse and its result
 * discarded; a finished, uncollected one has its result discarded.  On return the request's input
 * buffer is no longer used and its tag is free.  ELF_EINVAL for an unknown tag. */
int elf_server_cancel(elf_server s, long long tag);
/* Device bytes held, jobs in flight, requests waiting, handles created so far. */
int elf_server_stats(elf_server s, size_t* used_bytes, int* n_active, int* n_queued, int* n_created);
/* Waits for jobs in flight, then frees everything. */
void elf_server_destroy(elf_server s);

/* ---- No-allocation entry point (the paper has no counterpart to this call) ----
 * Some callers cannot allocate device memory: a process whose device memory
 * belongs to another allocator or to a fixed budget, or code that runs while its
 * framework forbids new allocations.  For them this computes the alpha = beta
 * weight of Eq. 16 (fidelity 0) or Eq. 17 (fidelity 1) without a handle and
 * without allocating: no cudaMalloc, cudaFree or allocating library routine.
 * I: device [n_led][n_lowres][n_lowres] float (3 <= n_lowres <= 4096);
 * weights: device, 2 doubles (alpha, beta), written in stream order on
 * cuda_stream (a cudaStream_t, may be NULL); the call does not synchronise.
 * Scratch: a static device array of ELF_NOALLOC_WEIGHT_MAX_PARTIALS doubles
 * (128 KB) that every GPU loading this library holds until the process exits.
 * A problem needing more partials than that (n_led * ceil((n_lowres - 2) / 16))
 * is rejected with ELF_EINVAL before any GPU work.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current and keeps it, so make that first call before any stream capture; the
 * kept address dies with the device's primary context, so do not call this
 * again on a device after cudaDeviceReset.  All calls share the array; each call
 * overwrites every partial it reads, so nothing needs clearing, but calls that
 * overlap on the GPU race. */
#define ELF_NOALLOC_WEIGHT_MAX_PARTIALS 16384
int elf_estimate_weights_noalloc(const float* I, int n_led, int n_lowres, int fidelity, double* weights,
                                 void* cuda_stream);

/* ---- Measured FP32 peak (for the roofline of the FP32-bound tile kernel; not in the paper) ----
 * Runs an FMA-throughput kernel on the current device: 8 blocks of 256 threads per SM, each
 * thread iters x 8 independent FMAs; repeats timed launches (CUDA events on cuda_stream,
 * which may be NULL) after one warm-up launch.  Writes the best launch's throughput in
 * TFLOP/s (2 FLOP per FMA) to *tflops and its duration to *best_ms (may be NULL).
 * Synchronises the stream.  Allocates no device memory; changes no device setting. */
int elf_measure_fp32_peak(int iters, int repeats, void* cuda_stream, double* tflops, double* best_ms);

void elf_destroy(elf_handle h);
const char* elf_strerror(int code);
const char* elf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ELFPIE_H */

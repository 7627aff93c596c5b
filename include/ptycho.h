/* libptycho: batched mixed-state multislice ptychography forward model and
 * its adjoint on one NVIDIA B300 (sm_103a).
 *
 * The operations follow the problem statement of arXiv 2505.14372 ("phaser"):
 *   §3    multislice forward model: P_k shifted to each scan position X_j,
 *         multiplied by each object slice O_i, Fresnel-propagated over the gap
 *         dz_i under an anti-aliasing band limit, far field
 *         I = sum_k |F(exit wave_k)|^2 over incoherent probe modes;
 *   §3.1  amplitude / Anscombe and Poisson noise models (loss per pixel);
 *   §3.2  gradient of the loss with respect to every object slice and probe
 *         mode at once, and the Adam solver step;
 *   §2.2  per-iteration randomised grouping of scan positions;
 *   §2.3  client/server job model, reduced here to an in-process continuous-
 *         batching server (ptycho_submit / ptycho_poll).
 *
 * Conventions (the paper leaves them open; these are this library's):
 *   - complex64 is interleaved {re, im} float32 (ptycho_c64);
 *   - arrays are row-major and contiguous; window h = w = N with
 *     N in {64, 128, 192, 256}; the object is H x W per slice;
 *   - a scan position is (y, x) in object pixels of the window's top-left
 *     corner; the patch origin is floor(r + 1/2), the remainder is applied as
 *     a Fourier phase ramp (sub-pixel shift P(r - delta));
 *   - DFT kernel exp(-2 pi i k x / N); the far field is orthonormal; patterns
 *     have the zero frequency at [0][0] (no fftshift);
 *   - the Fresnel propagator is exp(-i pi lambda dz |q|^2) times a circular
 *     band limit at `bandlimit` x Nyquist (<= 0 disables it), applied in each
 *     of the S-1 propagations;
 *   - losses are summed over pixels and positions; amplitude/Anscombe:
 *     1/2 (sqrt(I+c+eps) - sqrt(I_exp+c+eps))^2; Poisson:
 *     I - I_exp - I_exp (log(I+eps) - log(I_exp+eps));
 *   - gradients are dL/dRe z + i dL/dIm z (twice the paper's conj(dL/dz)).
 *
 * Ownership: every array argument is a DEVICE pointer owned by the caller
 * unless marked "host".  Calls that take a stream only enqueue work on it
 * (no synchronisation, no allocation); they are safe to capture in a CUDA
 * graph.  Calls named *_host copy host buffers in and out and synchronise.
 *
 * Errors: every call returns PTYCHO_OK (0) or a negative code; nothing is
 * thrown across the ABI.  ptycho_last_error() gives a message for the
 * calling thread.  Arguments are validated on the host before any launch.
 * Scan positions in device memory are validated by the kernels: an item
 * whose window leaves the object is skipped and flagged in a device status
 * word that ptycho_check() reads (it synchronises the stream).
 */
#ifndef PTYCHO_H_
#define PTYCHO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PTYCHO_OK 0
#define PTYCHO_EINVAL (-1)       /* bad dimensions, null pointer, bad option */
#define PTYCHO_EOUTOFBOUNDS (-2) /* a scan window leaves the object */
#define PTYCHO_ENOMEM (-3)       /* scratch budget / HBM admission exceeded */
#define PTYCHO_ECUDA (-4)        /* a CUDA runtime call failed */
#define PTYCHO_ETIMEDOUT (-5)    /* a bounded wait ran out */
#define PTYCHO_EBUSY (-6)        /* request not finished / server busy */
#define PTYCHO_ENOTFOUND (-7)    /* unknown ticket */
#define PTYCHO_ECHECK (-8)       /* checked build only: an index check failed (a library bug) */
#define PTYCHO_ECANCELED (-9)    /* served request cancelled (ptycho_cancel) */
#define PTYCHO_ENONFINITE (-10)  /* served request's loss became non-finite (it diverged) */
/* bits of a device status word (ptycho_forward_static's status_out) */
#define PTYCHO_STATUS_BIT_OUT_OF_BOUNDS 1u /* a scan window left the object; its item was skipped */

typedef struct {
  float re, im;
} ptycho_c64;

/* cudaStream_t; NULL is the legacy default stream. */
typedef void* ptycho_stream;

/* Noise models (§3.1); GAUSSIAN: (I - I_exp)^2 / (2 c^2), c = sigma > 0. */
typedef enum { PTYCHO_LOSS_AMPLITUDE = 0, PTYCHO_LOSS_POISSON = 1, PTYCHO_LOSS_GAUSSIAN = 2 } ptycho_loss;

/* How the adjoint gets the entry wave of every slice: STORE keeps all of
 * them from the forward pass (B*K*S*N*N*8 bytes of scratch); RECOMPUTE runs
 * the forward pass inside the adjoint kernel, one cluster per scan position
 * at a time, so only min(B, resident clusters) positions' entry waves
 * (K*S*N*N*8 bytes each) exist at once; AUTO stores when it fits the
 * scratch budget.  (Halve the wave bytes for 16-bit storage.) */
typedef enum { PTYCHO_WAVES_AUTO = 0, PTYCHO_WAVES_STORE = 1, PTYCHO_WAVES_RECOMPUTE = 2 } ptycho_waves;

/* Evaluation of the small DFTs inside the shared-memory FFT tile: radix
 * butterflies on the FP32 CUDA cores (the default), or dense DFT-matrix
 * products on the tensor cores with the FP32 operands split into two tf32 or
 * bf16 terms (three products: 22 or 16 significand bits), a single tf32
 * product, or three bf16 terms (BF16X6: all 24 bits of an FP32 value, the
 * six largest products, FP32-level accuracy).  The tensor-core variants
 * exist for the 192 x 192 window. */
typedef enum {
  PTYCHO_DFT_FFT = 0,
  PTYCHO_DFT_TF32X3 = 1,
  PTYCHO_DFT_BF16X3 = 2,
  PTYCHO_DFT_TF32 = 3,
  PTYCHO_DFT_BF16X6 = 4
} ptycho_dft;

/* Storage format of the entry waves kept between the forward pass and the
 * object-gradient term of the adjoint (the stored array or the recompute
 * slot): FP32, IEEE binary16 or bfloat16, each part rounded to nearest even
 * from its FP32 value.  Only the object gradient reads these copies (the
 * wavefield itself stays FP32 in shared memory), so intensities, loss and
 * probe gradient are unchanged.  §2.2 names reduced-precision wavefields as
 * the way to cut memory traffic. */
typedef enum { PTYCHO_PREC_F32 = 0, PTYCHO_PREC_F16 = 1, PTYCHO_PREC_BF16 = 2 } ptycho_prec;

/* Geometry and noise model of one reconstruction problem (§3, §3.1). */
typedef struct {
  int32_t S, K;       /* slices, incoherent probe modes (K >= 1, S >= 1) */
  int32_t h, w;       /* window; h == w == N in {64, 128, 192, 256} */
  int32_t H, W;       /* object slice size, H >= h, W >= w */
  double dx;          /* pixel size [A] (> 0) */
  double lambda;      /* electron wavelength [A] (> 0) */
  const double* dz;   /* host, S-1 slice gaps [A]; copied by ptycho_create */
  double bandlimit;   /* band limit as a fraction of Nyquist; <= 0: off */
  int32_t loss;       /* ptycho_loss */
  double eps;         /* noise-model offset; Poisson needs eps > 0,
                         amplitude needs eps + c > 0 */
  double c;           /* amplitude-model offset (0 amplitude, 3/8 Anscombe) */
  int32_t waves;      /* ptycho_waves */
  int32_t dft;        /* ptycho_dft: how the 2-D DFTs are evaluated */
  int32_t wave_prec;  /* ptycho_prec: storage of the entry waves */
  int32_t deterministic; /* 0: object and probe gradients summed over the
                            group's positions with float atomics (the
                            order varies from run to run); 1: each
                            position's contribution is kept apart and the
                            sums run in position order, so gradients (and
                            a step's updates) are bit-identical across
                            runs; needs the recomputed-wave path with the
                            FFT tile and FP32 entry waves (EINVAL
                            otherwise) and B*(S+K)*N*N*8 more bytes of
                            scratch */
} ptycho_geom;

typedef struct ptycho_ctx ptycho_ctx;

/* Creates a context for one geometry on the current CUDA device: builds the
 * propagator tables and allocates `scratch_budget_bytes` of device scratch
 * once (0 picks the size that one call with B = max_batch needs).
 * max_batch bounds B in every later call.  Returns EINVAL / ENOMEM / ECUDA. */
int ptycho_create(const ptycho_geom* geom, int32_t max_batch, size_t scratch_budget_bytes,
                  ptycho_ctx** out);
int ptycho_destroy(ptycho_ctx* ctx);

/* Bytes of scratch one forward+adjoint call with B positions needs under
 * the given waves mode (STORE or RECOMPUTE; AUTO reports STORE). */
size_t ptycho_scratch_bytes(const ptycho_geom* geom, int32_t B, int32_t waves);

/* Forward model (§3): I_out[B][N][N] (float32, zero frequency at [0][0]) =
 * sum_k |F_o psi_exit(j, k)|^2 for the B positions pos[B][2].
 * O: [S][H][W], P: [K][N][N] complex64. */
int ptycho_forward(ptycho_ctx* ctx, const ptycho_c64* O, const ptycho_c64* P, const float* pos,
                   int32_t B, float* I_out, ptycho_stream stream);

/* Loss and gradient (§3.1, §3.2) for B positions with measured patterns
 * I_exp[B][N][N].  loss_out: device double (may be NULL).  gO [S][H][W] and
 * gP [K][N][N] are overwritten, or added to when accumulate != 0. */
int ptycho_adjoint(ptycho_ctx* ctx, const ptycho_c64* O, const ptycho_c64* P, const float* pos,
                   int32_t B, const float* I_exp, double* loss_out, ptycho_c64* gO, ptycho_c64* gP,
                   int32_t accumulate, ptycho_stream stream);

/* ptycho_adjoint plus the gradient with respect to the scan positions
 * (position correction, §1 and §3: positions X_j are reconstruction
 * variables): gpos_out[B][2] (device double, d L / d(y, x) in object pixels)
 * is overwritten, or added to when accumulate != 0.  The derivative goes
 * through the sub-pixel Fourier ramp; the integer patch origin is piecewise
 * constant. */
int ptycho_adjoint_positions(ptycho_ctx* ctx, const ptycho_c64* O, const ptycho_c64* P, const float* pos,
                             int32_t B, const float* I_exp, double* loss_out, ptycho_c64* gO, ptycho_c64* gP,
                             double* gpos_out, int32_t accumulate, ptycho_stream stream);

/* Vector-Jacobian product of the forward model (§3.2: the gradient engine
 * of the paper is the VJP of the forward simulation): for a cotangent
 * gI[B][N][N] = dL/dI of any real loss L(I), writes (or adds, accumulate
 * != 0) gO = dL/dRe O + i dL/dIm O and gP likewise.  The entry waves are
 * recomputed from O, P and pos (nothing is kept from ptycho_forward). */
int ptycho_vjp(ptycho_ctx* ctx, const ptycho_c64* O, const ptycho_c64* P, const float* pos, int32_t B,
               const float* gI, ptycho_c64* gO, ptycho_c64* gP, int32_t accumulate, ptycho_stream stream);

/* Allocation-free forward model, for callers that cannot allocate device
 * memory (a live-reconstruction loop that must not stall in cudaMalloc's
 * locks and device synchronisation, an application that gives all device
 * memory to its own pool, a plug-in whose host forbids allocating).  The
 * paper has no counterpart: it is a packaging of ptycho_forward.
 * Computes the same I_out[B][N][N] as ptycho_forward for the geometry *geom
 * (checked like ptycho_create's and read per call; no context), using the
 * kernels of ptycho_forward and a fixed 32 MiB scratch array that lives in
 * the library (every GPU that loads the library holds it until exit).  The
 * problem must fit it: K*N*N*8*(B+1) + (S-1)*N*8 plus a little alignment
 * <= 32 MiB, and S <= 65 (the slice gaps travel in the kernel's arguments),
 * else EINVAL with the sizes in the message.  Calls no cudaMalloc or
 * cudaFree and copies nothing from host memory; the array's device address
 * is resolved once per CUDA context (cudaGetSymbolAddress with that context
 * current) on the first call made in it, so make that first call before any
 * stream capture; the tensor-core DFT modes (geom->dft != 0) also fill their
 * constant tables on their first use on a device (a synchronous copy, no
 * allocation).  All calls share the array and it keeps the last call's
 * contents; each call clears what must start at zero.  Calls whose work
 * overlaps on the GPU (other streams, other host threads) race on the
 * shared scratch: order them.  Positions outside the object give zero
 * intensity for their pattern and set PTYCHO_STATUS_BIT_OUT_OF_BOUNDS in
 * the call's status word, which is copied (stream-ordered) to *status_out
 * when status_out (a device uint32) is not NULL.  A bounded exchange wait
 * of the 192 x 192 tile that runs out (a partner CTA that never answers;
 * not expected in practice) raises the library-wide time-out flag that the
 * next ptycho_check of any 192 x 192 context reports as ETIMEDOUT. */
int ptycho_forward_static(const ptycho_geom* geom, const ptycho_c64* O, const ptycho_c64* P, const float* pos,
                          int32_t B, float* I_out, uint32_t* status_out, ptycho_stream stream);

/* Adam hyper-parameters (§3.2; Optax-style defaults 0.9, 0.999, 1e-8) and
 * the weights of the cost regularisers added to the loss (§3.4; 0 = off):
 * object L2 lambda sum |O - 1|^2, in-plane Tikhonov lambda sum of squared
 * forward differences along y and x of every slice, Tikhonov across layers
 * lambda sum |O_{s+1} - O_s|^2, probe L2 lambda sum |P|^2, and total
 * variation in plane (reg_obj_tv) and across layers (reg_obj_layers_tv):
 * lambda sum (sqrt(|d|^2 + eta^2) - eta) over the same forward differences d,
 * eta = reg_tv_eps > 0 (EINVAL otherwise when a TV weight is set). */
typedef struct {
  float lr_O, lr_P;
  float beta1, beta2, eps;
  int32_t update_probe; /* 0: the probe is held fixed */
  float reg_obj_l2, reg_obj_tikhonov, reg_obj_layers, reg_probe_l2;
  float reg_obj_tv, reg_obj_layers_tv, reg_tv_eps;
} ptycho_opt;

/* Adam state: first moments m (complex64), second moments v (float32, |g|^2
 * based), device arrays shaped like O and P; t = steps taken (host, updated
 * by ptycho_step). */
typedef struct {
  ptycho_c64* mO;
  float* vO;
  ptycho_c64* mP;
  float* vP;
  int64_t t;
} ptycho_adam;

/* One gradient-descent iteration on one group of B scan positions:
 * idx[B] (device int32, each in [0, n_pos)) selects positions
 * pos_all[n_pos][2] and patterns I_exp_all[n_pos][N][N]; an index outside
 * that range is skipped and flagged like an out-of-bounds window; loss and gradient as ptycho_adjoint, then Adam on O
 * (and P unless update_probe == 0), in place.  stats_out (device double[2],
 * may be NULL) receives {loss, sqrt(sum |gO|^2 + sum |gP|^2)}. */
int ptycho_step(ptycho_ctx* ctx, ptycho_c64* O, ptycho_c64* P, ptycho_adam* state,
                const ptycho_opt* opt, const float* pos_all, const float* I_exp_all, int32_t n_pos,
                const int32_t* idx, int32_t B, double* stats_out, ptycho_stream stream);

/* ptycho_step with the group's positions and patterns in HOST memory
 * (pinned memory gives the fastest copies): copies them to the device,
 * steps, and returns loss and gradient norm to host doubles.  Synchronises
 * the stream.  Positions are validated on the host (EOUTOFBOUNDS). */
int ptycho_step_host(ptycho_ctx* ctx, ptycho_c64* O, ptycho_c64* P, ptycho_adam* state,
                     const ptycho_opt* opt, const float* pos_host, const float* I_exp_host,
                     int32_t B, double* loss_host, double* gnorm_host, ptycho_stream stream);

/* One ePIE / 3PIE update (§3.3.1) from one group of B scan positions (idx,
 * pos_all, I_exp_all and n_pos as in ptycho_step), in place: every position
 * of the group sees the same O and P; the detector-plane update of §3.1,
 * chi = (sqrt(I_exp + c) / (eps + sqrt(I + c)) - 1) A, is carried back
 * through the slices, where slice s receives conj(psi_s) chi_s /
 * max|psi_s|^2 (per position and mode) and the incident wave
 * conj(O_s) chi_s / max|O_s|^2 (maximum over the whole slice) is propagated
 * back with conj(H); then O += beta_O * (sum over positions and modes) and
 * P_k += beta_P * (mean over positions of the unshifted entry-plane
 * update).  beta_P = 0 holds the probe.  Needs the amplitude noise model
 * (c = 0 ePIE, c = 3/8 Anscombe), else EINVAL.  loss_out (device double,
 * may be NULL) receives the group's amplitude loss before the update. */
int ptycho_epie_step(ptycho_ctx* ctx, ptycho_c64* O, ptycho_c64* P, float beta_O, float beta_P,
                     const float* pos_all, const float* I_exp_all, int32_t n_pos, const int32_t* idx, int32_t B,
                     double* loss_out, ptycho_stream stream);

/* LSQML options (§3.3.2): step scales of the object and probe updates, the
 * absolute regularisers of the illumination and transmission normalisers,
 * and of the step-size denominators. */
typedef struct {
  float beta_O, beta_P;
  float delta_O, delta_P;
  float gamma;
} ptycho_lsqml_opt;

/* One LSQML update (§3.3.2) from one group of B scan positions (idx,
 * pos_all, I_exp_all and n_pos as in ptycho_step), in place.  Every position
 * of the group sees the same O and P.  From the detector update of §3.1 (as
 * ePIE) carried back through the slices come the object direction
 * sum conj(psi_s) chi_s and the probe direction (the entry-plane update
 * moved to the probe frame), summed over positions and modes and divided by
 * the illumination sum |psi_s|^2 + delta_O (object frame) and the
 * transmission sum prod_s |O_s|^2 + delta_P (probe frame); illum_prev
 * [S][H][W] and trans_prev [N][N] (device, may be NULL) replace those sums
 * (running sums of a previous iteration).  Per position j the least-squares
 * steps alpha_{s,j} = sum Re(chi_s conj(dO_s psi_s)) / (sum |dO_s psi_s|^2 + gamma)
 * and alpha_{P,j} (the same with O_0 S_j dP), then
 * O_s += beta_O dO_s sum_j alpha_{s,j} w_{s,j} / sum_j w_{s,j} (w = sum_k |psi_s|^2)
 * and P += beta_P dP sum_j alpha_{P,j} t_j / sum_j t_j (t = prod_s |O_s|^2).
 * The group's illumination and transmission are added to illum_acc and
 * trans_acc when given.  Needs the amplitude noise model, recomputed FP32
 * entry waves and the FFT tile (EINVAL otherwise); allocates its own
 * buffers (about 16 bytes per object pixel) on the first call.  loss_out
 * (device double, may be NULL) receives the group's amplitude loss before
 * the update. */
int ptycho_lsqml_step(ptycho_ctx* ctx, ptycho_c64* O, ptycho_c64* P, const ptycho_lsqml_opt* opt,
                      const float* illum_prev, const float* trans_prev, float* illum_acc, float* trans_acc,
                      const float* pos_all, const float* I_exp_all, int32_t n_pos, const int32_t* idx, int32_t B,
                      double* loss_out, ptycho_stream stream);

/* Synchronises `stream` and reports (then clears) the device status word:
 * PTYCHO_EOUTOFBOUNDS if any item was skipped since the last check.  In the
 * checked build (libptycho_checked.so, see ptycho_build_checked) it first
 * reports PTYCHO_ECHECK if an index check of this context's window size
 * failed since the last check (the access was skipped; the results are not
 * valid): a shared-memory slot outside the wavefield, a window coordinate
 * outside [0, N) or an item outside its problem. */
int ptycho_check(ptycho_ctx* ctx, ptycho_stream stream);

/* Grouping (§2.2): writes a permutation of 0..P-1 into out_idx[P] (host)
 * for `iteration` of a run seeded by `seed`; consecutive runs of B indices
 * are the groups.  mode 0 = sparse (random groups), 1 = compact (spatially
 * contiguous groups from a raster ordering of pos_host[P][2], group order
 * shuffled).  Deterministic across platforms. */
int ptycho_make_groups(int32_t P, int32_t B, uint64_t seed, int64_t iteration, int32_t mode,
                       const float* pos_host, int32_t* out_idx);

/* Per-kernel device time accumulated by this context's launches since the
 * last reset (CUDA events on the launching stream), enabled with
 * ptycho_set_timing(ctx, 1) for every kernel or ptycho_set_timing(ctx, 2)
 * for the tile kernels (forward / adjoint) only, which keeps the events out
 * of the short kernels of small problems.  Inside a stream capture the
 * events are captured as external nodes, so each replay records its times.
 * names/ms are host arrays of length cap; returns the number of entries, or
 * a negative code. */
int ptycho_set_timing(ptycho_ctx* ctx, int32_t enable);

/* Adam step count kept in device memory, so that a step captured in a CUDA
 * graph replays with the right bias corrections (§3.2 solver).  With t_dev
 * set (one int64 in device memory, owned by the caller), every ptycho_step /
 * ptycho_step_host of this context takes t = *t_dev + 1, stores it back and
 * computes the corrections 1 / (1 - beta^t) on the stream, before its Adam
 * update; the host count of ptycho_adam is then not used for them (it is
 * still incremented).  t_dev = NULL returns to the host count.  Not a
 * stream call: allocates 8 bytes of device memory on first use.  Errors:
 * EINVAL (NULL context), ENOMEM. */
int ptycho_set_step_counter(ptycho_ctx* ctx, int64_t* t_dev);
int ptycho_kernel_times(ptycho_ctx* ctx, const char** names, double* ms, int32_t* launches, int32_t cap);

/* Self-test of failure detection on the device (N = 192, the tile whose
 * layout switches wait on mbarriers): launches one cluster whose exchange
 * waits for data that nothing sends, with a short poll limit, so every wait
 * gives up, flags the time-out and returns (no hang, no fault).  Returns
 * PTYCHO_ETIMEDOUT when the flag was seen, as expected; PTYCHO_OK would
 * mean the wait did not give up.  Synchronises the device. */
int ptycho_exchange_selftest(int32_t N);

/* Stand-alone 2-D DFT of `count` natural-order N x N complex64 arrays
 * through the same shared-memory tile the model uses (dir < 0 forward,
 * dir > 0 inverse, both unnormalised).  For tests and diagnostics. */
int ptycho_fft2(int32_t N, int32_t dir, const ptycho_c64* in, ptycho_c64* out, int32_t count,
                ptycho_stream stream);
/* ptycho_fft2 through the tile of a given DFT evaluation (ptycho_dft: 0 the
 * FFT tile, 1-4 the warp-level tensor-core tiles, N = 192 only).  For tests
 * and for timing the DFT evaluations against each other. */
int ptycho_fft2_dft(int32_t N, int32_t dft, int32_t dir, const ptycho_c64* in, ptycho_c64* out, int32_t count,
                    ptycho_stream stream);

/* Batched 1-D DFTs of rows on Blackwell's tcgen05 tensor cores (the §2.2
 * precision option for the DFTs of §3): out[r][n] = sum_k in[r][k]
 * exp(dir 2 pi i k n / N) for r < rows, N in {64, 128, 192, 256}, dir -1
 * (forward) or +1 (inverse, unnormalised).  The complex rows are multiplied
 * by the real 2N x 2N form of the DFT matrix as one GEMM with FP32
 * accumulation in tensor memory; mode 1 splits both operands into two tf32
 * parts (three products, near-FP32 accuracy), 2 into two bf16 parts (three
 * products), 3 takes one tf32 product.  in, out: device arrays
 * [rows][N] complex64, 16-byte aligned, not overlapping.  The first call
 * in a CUDA context and (N, mode, dir) builds the split DFT matrix on the
 * host and uploads it (cudaMalloc + synchronous copy; kept until exit).
 * EINVAL for bad sizes or pointers or a non-Blackwell device, ECUDA if the
 * launch fails.  A bounded wait inside the kernel that runs out is reported
 * by ptycho_dft_rows_tc_check (synchronous) as ETIMEDOUT. */
int ptycho_dft_rows_tc(int32_t N, int32_t mode, int32_t dir, const ptycho_c64* in, ptycho_c64* out, int32_t rows,
                       ptycho_stream stream);
int ptycho_dft_rows_tc_check(void);

/* ---------------------------------------------------------------------------
 * Serving (§2.3 job model, in process): requests from datasets of different
 * shapes are admitted against an HBM budget, keep their object, probe and
 * Adam state resident on the device, and have their iterations batched into
 * shared launches with the other admitted requests.  All request data is
 * host memory; results point into library-owned host buffers that stay
 * valid until ptycho_release. */
typedef struct ptycho_server ptycho_server;

typedef struct {
  ptycho_geom geom;          /* geom.dz must stay valid until submit returns */
  int32_t n_pos;             /* scan positions P */
  const float* pos;          /* host [P][2] */
  const float* I_exp;        /* host [P][N][N] */
  const ptycho_c64* O_init;  /* host [S][H][W], or NULL for vacuum (O = 1) */
  const ptycho_c64* P_init;  /* host [K][N][N] */
  int32_t iterations;        /* full passes over the P positions */
  int32_t batch;             /* group size B */
  int32_t grouping;          /* 0 sparse, 1 compact */
  uint64_t seed;
  ptycho_opt opt;
} ptycho_request;

#define PTYCHO_REQ_QUEUED 0
#define PTYCHO_REQ_RUNNING 1
#define PTYCHO_REQ_DONE 2
#define PTYCHO_REQ_FAILED 3
#define PTYCHO_REQ_ADMITTING 4   /* device state being allocated and uploaded */

typedef struct {
  int32_t state;               /* PTYCHO_REQ_* */
  int32_t iterations_done;
  int32_t error;               /* error code when FAILED */
  double last_loss;
  double submit_ms, start_ms, finish_ms; /* wall clock relative to server start */
} ptycho_status;

typedef struct {
  const ptycho_c64* O;         /* host [S][H][W] (valid until release) */
  const ptycho_c64* P;         /* host [K][N][N] */
  const double* loss;          /* host [iterations * groups] per-step losses */
  int32_t n_loss;
  const double* step_ms;       /* host, device time of every shared launch this request rode in */
  int32_t n_step;
} ptycho_result;

typedef struct {
  int64_t submitted, admitted, finished, failed;
  int64_t queue_depth;
  size_t admitted_bytes, budget_bytes;
  int64_t launches;            /* shared tile-kernel launches issued (per tick and window size: one
                                  position-major launch, or a forward + adjoint pair when the
                                  budget has no room for its scratch) */
  double positions_per_s;      /* over the server's busy time */
  double p50_iter_ms, p99_iter_ms; /* per-iteration latency over finished steps */
} ptycho_server_stats;

/* hbm_budget_bytes: device memory the server may hold for admitted
 * requests (state + scratch).  max_active: requests resident at once. */
int ptycho_server_create(size_t hbm_budget_bytes, int32_t max_active, ptycho_server** out);
int ptycho_server_destroy(ptycho_server* srv); /* cancels unfinished work */
/* Non-blocking; copies the request's host arrays.  ENOMEM if the request
 * alone exceeds the budget; EINVAL for a geometry ptycho_create would
 * refuse, and for a non-finite value in the positions, patterns, probe or
 * object (the message names the first one); EOUTOFBOUNDS for a scan
 * position whose window leaves the object.  Served requests take 1 <= S <= 32 slices (the
 * per-window-size slot scratch is sized for 32; EINVAL beyond), the FFT
 * tile, FP32 entry waves and the atomic gradient sums; those with K <= 8
 * modes ride in the shared position-major launch of their window size,
 * more modes in a forward + recomputing adjoint launch pair. */
int ptycho_submit(ptycho_server* srv, const ptycho_request* req, uint64_t* ticket);
/* Non-blocking; fills st (and res once DONE).  ENOTFOUND for unknown tickets. */
int ptycho_poll(ptycho_server* srv, uint64_t ticket, ptycho_status* st, ptycho_result* res);
/* Blocks until the ticket is DONE/FAILED or timeout_ms passes (ETIMEDOUT). */
int ptycho_wait(ptycho_server* srv, uint64_t ticket, double timeout_ms);
int ptycho_release(ptycho_server* srv, uint64_t ticket);
/* Cancels a request: a queued one ends at once; an admitted one gets no
 * further step, and once the steps already enqueued for it are done its
 * device state is freed.  Either way it ends FAILED with error
 * PTYCHO_ECANCELED (ptycho_poll / ptycho_wait show it; release it as usual).
 * No effect on a request that has already ended.  The other requests are
 * not affected.  A served request whose loss turns non-finite (checked at
 * the end of every iteration) ends the same way with PTYCHO_ENONFINITE. */
int ptycho_cancel(ptycho_server* srv, uint64_t ticket);
/* Host-side fault injection for tests (the paper has no counterpart): the
 * server's worker thread sleeps `ms` milliseconds before its next tick, as
 * a stalled worker would, so that clients' time-outs (ptycho_wait) can be
 * exercised.  Nothing is done to the GPU. */
int ptycho_server_inject_stall(ptycho_server* srv, double ms);
int ptycho_server_stats_get(ptycho_server* srv, ptycho_server_stats* out);

/* FP32 CUDA-core throughput microbenchmark (measurement support: the
 * denominator of the roofline of the FFT tile kernels, whose arithmetic is
 * FP32 on the CUDA cores; the paper has no counterpart).  Enqueues ONE
 * kernel on `stream`: 8 blocks of 256 threads per SM, each thread running
 * 16 independent x <- x*a + b chains for iters x 16 rounds, as scalar FFMA
 * (packed = 0) or packed two-wide FFMA2 (packed != 0).  *flops_out (host)
 * receives the FP32 flops the launch performs (2 per FMA); the caller times
 * the launch on the stream (CUDA events) and divides.  sink: device float
 * array of ptycho_fp32_peak_sink_elems() elements (never written in
 * practice; keeps the chains live).  EINVAL for iters < 1 or NULL
 * pointers, ECUDA if the launch fails. */
int ptycho_fp32_peak_launch(int32_t packed, int32_t iters, float* sink, double* flops_out,
                            ptycho_stream stream);
int32_t ptycho_fp32_peak_sink_elems(void);

/* Number of CUDA kernels this library has launched in this process (all
 * contexts and servers); a diagnostic for counting device work. */
uint64_t ptycho_kernels_launched(void);

const char* ptycho_last_error(void);
const char* ptycho_version(void);
/* 1 in the checked build (libptycho_checked.so: the same entry points, with
 * index checks in the kernels that record a bit and skip the access instead
 * of trapping, reported by ptycho_check as PTYCHO_ECHECK), 0 in the normal
 * build.  The paper has no counterpart: a debugging aid. */
int32_t ptycho_build_checked(void);

#ifdef __cplusplus
}
#endif
#endif /* PTYCHO_H_ */

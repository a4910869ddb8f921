/*
 * pty.h -- C ABI of the GB300 (sm_103a) multislice ptychography hot path.
 *
 * The library evaluates, for a batch of scan positions, the mixed-state multislice forward model
 * of PtyRAD (arXiv 2505.07814, Sec. "Physical model", Eq. 1-4), the Gaussian or Poisson
 * negative-log-likelihood loss (Sec. "Optimizers and loss functions", Eq. 5-6) and the exact
 * gradient of that loss with respect to the six optimisable parameters of Sec. "AD-optimizable
 * parameters": object amplitude, object phase, probe modes, probe positions, local tilts and slice
 * spacing dz.  The gradient comes from a hand-written adjoint, not from automatic differentiation.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All array arguments are DEVICE pointers on the current CUDA device, row-major, axis 0 = rows,
 *    axis 1 = columns.  Complex arrays are interleaved (re, im) float32 pairs and must be 8-byte
 *    aligned; everything else 4-byte aligned.  The caller owns every buffer; the library allocates
 *    no device memory and keeps no pointer after a call returns.
 *  - Calls are asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream).  Results,
 *    including the device-side status word, are valid once the stream has reached them.
 *  - Return value: PTY_OK, or an error code with nothing launched (host-side validation).  The
 *    message of the last failure on the calling thread is available from pty_last_error().
 *    Conditions that only the device can see (a patch outside the object, a non-finite loss) set
 *    bits of the status word in the workspace; read them with pty_status().  The kernels clamp an
 *    out-of-range patch into the object instead of reading out of bounds.
 *  - Object amp/phase: float [Nz][H][W].  Probe: complex [M][N][N] (real-space modes).
 *    Positions: float [Ntot][2], (row, col) of the top-left corner of each N x N object patch, in
 *    pixels; the patch starts at round-half-to-even(pos) and the remainder pos - round(pos) is the
 *    sub-pixel shift applied to the probe (Sec. "Physical model").  Tilts: float [Ntot][2] radian
 *    (or [2] with global_tilt), (axis-0, axis-1) components of theta in Eq. 4.  dz: float[1]
 *    angstrom, the separation between slices (Eq. 3-4).  Measured and modelled patterns: float
 *    [.][N][N], DC-centred (fftshift of the DFT order), far field taken with the orthonormal DFT.
 *  - Batches: idx is an int32 [B] array of scan-position indices in [0, Ntot); the batch holds the
 *    patterns idx[0..B-1].  Repeated indices are allowed (their gradients add).
 *  - Complex gradients follow dL/dRe + i dL/dIm; amplitude/phase gradients are real.
 */
#ifndef PTY_H
#define PTY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return / status codes.  Device status bits are OR-ed into the workspace status word. */
enum {
  PTY_OK = 0,
  PTY_EINVAL = 1,      /* bad shape, unsupported N, null or misaligned pointer */
  PTY_EBOUNDS = 2,     /* device bit: a patch round(pos) .. round(pos)+N-1 left the object, or
                          a batch index was outside [0, Ntot) (then scan position 0 was used) */
  PTY_EWORKSPACE = 4,  /* workspace smaller than pty_workspace_size() */
  PTY_ECUDA = 8,       /* a CUDA launch failed; see pty_last_error() */
  PTY_ETIMEOUT = 16,   /* a bounded device wait gave up (tensor-core GEMM pipeline; the optional bulk-copy stages) */
  PTY_ENONFINITE = 32  /* device bit: the loss or its normaliser was not finite */
};

enum { PTY_LOSS_POISSON = 0, PTY_LOSS_GAUSSIAN = 1 };

/* Which gradients pty_loss_grad / pty_step compute (bit mask). */
enum {
  PTY_GRAD_AMP = 1,
  PTY_GRAD_PHASE = 2,
  PTY_GRAD_PROBE = 4,
  PTY_GRAD_POS = 8,
  PTY_GRAD_TILT = 16,
  PTY_GRAD_DZ = 32,
  PTY_GRAD_ALL = 63
};

/* Problem geometry.  N is the probe window, detector and FFT size: 64, 128 or 256 (N = 256 runs
 * each wave on a four-CTA thread-block cluster). */
typedef struct {
  int N;           /* probe / detector pixels per side */
  int M;           /* incoherent probe modes, >= 1 (Eq. 2) */
  int Nz;          /* object slices, >= 1 (Eq. 3) */
  int H, W;        /* object rows / columns, >= N */
  int Ntot;        /* scan positions: rows of pos, tilt and I_meas */
  float dx;        /* real-space pixel size, angstrom (sets the frequency grid of Eq. 4) */
  float lambda;    /* electron wavelength, angstrom (Eq. 4) */
  int loss;        /* PTY_LOSS_POISSON (Eq. 6) or PTY_LOSS_GAUSSIAN (Eq. 5) */
  float p;         /* exponent applied to the patterns in the loss; <= 0 selects the default
                      (1 for Poisson, 0.5 for Gaussian) */
  float eps;       /* Poisson stabiliser inside the log (Eq. 6), normally 1e-6 */
  int grad_mask;   /* PTY_GRAD_* bits */
  int global_tilt; /* 0: tilt is [Ntot][2] (local); 1: tilt is [2] shared by every position */
  int ckpt_stride; /* adjoint memory plan.  0 or 1: the forward keeps the wave entering every slice
                      (and every propagated spectrum) for the adjoint: B*M*(2 Nz - 1)*N^2*8 bytes.
                      K > 1: it keeps only the spectrum entering slices K, 2K, ... and the adjoint
                      re-runs each K-slice segment from there before differentiating it:
                      B*M*(ceil(Nz/K) - 1 + 2K + 1)*N^2*8 bytes and about one more forward pass of
                      work.  K >= Nz re-runs the whole forward. */
  int fft_impl;    /* PTY_FFT_*: how the per-slice 2D DFTs are computed.  PTY_FFT_FP32: FP32 FFTs in
                      shared memory (every N).  The split modes (N = 64, 128) run dense DFT matrix
                      products on the tensor cores with every FP32 operand cut into 16-bit pieces and
                      FP32 accumulation: PTY_FFT_SPLIT_BF16 and PTY_FFT_SPLIT_FP16 keep a high part
                      and a remainder (three products; 16 and 22 significant bits, fp16 after a
                      power-of-two rescaling of each batch), PTY_FFT_SPLIT3_BF16 three bf16 pieces
                      (six products, 24 bits).  The split modes keep every slice's checkpoint
                      (ckpt_stride is ignored) and add 4*B*M*N^2*8 bytes of workspace
                      (5*B*M*N^2*8 for three-piece bf16).  The first
                      split call on a device builds its DFT tables and waits for them (not
                      capturable into a CUDA graph). */
  float w_pacbed;  /* weight of the PACBED term (Eq. 7) added to the loss of pty_loss_grad / pty_step:
                      the batch-mean modelled pattern against the batch-mean measured one, compared
                      like Eq. 5 with exponent p_pacbed (<= 0: 0.5); 0 = off */
  float p_pacbed;
  float w_sparse;  /* weight of the phase-sparsity term (Eq. 8): <|phase|^p_sparse>^(1/p_sparse) over
                      every slice of every batch position's N x N patch (p_sparse <= 0: 1); 0 = off */
  float p_sparse;
  int obj_modes;   /* object modes K of the mixed-state object (Eq. 2), 0 or 1: a single object.  The
                      object arrays (amp, phase and their gradients and Adam moments) are
                      [K][Nz][H][W]; every pattern sums the intensities of all M x K (probe mode,
                      object mode) pairs; the sparsity term covers every mode's patches.  The
                      workspace's per-wave arrays grow by K. */
} pty_geom;

enum { PTY_FFT_FP32 = 0, PTY_FFT_SPLIT_BF16 = 1, PTY_FFT_SPLIT_FP16 = 2, PTY_FFT_SPLIT3_BF16 = 3 };

/* Adam state and hyper-parameters for pty_step / pty_adam (PyTorch's Adam: bias-corrected first and
 * second moments; complex tensors are treated as pairs of reals).  m_* and v_* are device float
 * arrays shaped like the parameter they belong to, zero-initialised by the caller before step 1.
 * A parameter is updated only if its PTY_GRAD_* bit is set in geom->grad_mask and its lr > 0; this
 * is the per-parameter learning rate and onset of Sec. "AD-optimizable parameters". */
typedef struct {
  float *m_amp, *v_amp, *m_phase, *v_phase, *m_probe, *v_probe;
  float *m_pos, *v_pos, *m_tilt, *v_tilt, *m_dz, *v_dz;
  float lr_amp, lr_phase, lr_probe, lr_pos, lr_tilt, lr_dz;
  float beta1, beta2, eps;
} pty_adam;

/* Bytes of workspace a call with batch size B needs (forward, loss and adjoint, for the gradients
 * named in geom->grad_mask).  0 on invalid geometry (see pty_last_error()). */
size_t pty_workspace_size(const pty_geom* geom, int B);

/* Memory plan of the adjoint: the per-slice choice between keeping the forward's entering waves
 * and recomputing them, for a batch of B positions whose workspace must fit budget_bytes.  Writes to
 * *stride the pty_geom.ckpt_stride to use, and to *ws_bytes (may be NULL) the workspace it needs:
 *  - 1 (keep every slice's entering wave and spectrum; no replay) when that fits;
 *  - otherwise the stride K in 2 .. Nz-1 of least work that fits.  Every K > 1 replays each slice
 *    once (about one more forward pass); fewer, longer segments ran faster on the large-window
 *    workload, so it is the largest K whose workspace fits and is below K = 1's.  The record is
 *    B*M*(ceil(Nz/K) - 1 + 2K + 1)*N^2*8 bytes: it shrinks with K up to K ~ sqrt(Nz / 2), then grows.
 * PTY_EWORKSPACE (message: the smallest workspace any plan needs) when no stride fits; the
 * split-precision modes keep every checkpoint, so for them only K = 1 is considered.  Host only. */
int pty_plan_ckpt(const pty_geom* geom, int B, size_t budget_bytes, int* stride, size_t* ws_bytes);

/* Forward model, Eq. 1-4: I_model[b] = fftshift( sum_m sum_n |F_ortho[psi_{idx[b]}^(m)(n)]|^2 ), [B][N][N]
 * (probe modes m, object modes n).
 * Reads amp, phase, probe, pos, tilt, dz; writes I_model.  ws must hold pty_workspace_size(). */
int pty_forward(const pty_geom* geom, int B, const int32_t* idx, const float* amp,
                const float* phase, const float* probe, const float* pos, const float* tilt,
                const float* dz, float* I_model, void* ws, size_t ws_bytes, void* stream);

/* Loss of the batch (Eq. 5 or 6, means over detector pixels and batch) and its gradients.
 *  I_meas  float [Ntot][N][N], DC-centred measured patterns (rows idx[b] are used).
 *  loss    double[1] device scalar (written).
 *  I_model float [B][N][N] or NULL.
 *  g_amp, g_phase float [Nz][H][W]; g_probe complex [M][N][N]; g_pos float [Ntot][2];
 *  g_tilt float [Ntot][2] (or [2] with global_tilt); g_dz float[1].  A gradient whose bit is not
 *  in geom->grad_mask may be NULL and is left untouched.
 *  accumulate = 0: every requested gradient array is overwritten in full (zeros where the batch
 *  does not reach); accumulate = 1: the batch's gradient is added (gradient accumulation over
 *  sub-batches). */
int pty_loss_grad(const pty_geom* geom, int B, const int32_t* idx, const float* amp,
                  const float* phase, const float* probe, const float* pos, const float* tilt,
                  const float* dz, const float* I_meas, double* loss, float* I_model,
                  float* g_amp, float* g_phase, float* g_probe, float* g_pos, float* g_tilt,
                  float* g_dz, int accumulate, void* ws, size_t ws_bytes, void* stream);

/* A batch split into parts: over data-parallel ranks (one part per GPU) or over sub-batches whose
 * gradients are accumulated.  The losses of Eq. 5 and 6 are means over the detector pixels D and the
 * whole batch B, divided by <I_meas^p> of that same batch (Sec. "Optimizers and loss functions"),
 * so a part's gradient depends on the rest of the batch through three sums: S = sum of I_meas^p,
 * Q = sum of (I_model^p - I_meas^p)^2 (Gaussian only) and D B.  pty_loss_stats writes this part's
 * three sums; adding them over the parts (an all-reduce) gives the whole batch's, which
 * pty_loss_grad_part then uses.  The parts' gradients (accumulate = 1 on one device, or an
 * all-reduce of each gradient across ranks) then add up to pty_loss_grad's gradient of the whole
 * batch, and the parts' losses to its loss.
 *
 * pty_loss_stats: stats = device double[3], overwritten with {S, Q, D B} of this call's B patterns.
 *   Poisson needs the measured patterns only (Q is written as 0, no forward pass runs); Gaussian
 *   runs the forward model to get Q.  ws: as pty_loss_grad (pty_workspace_size bytes).
 * pty_loss_grad_part: pty_loss_grad for the B patterns of one part, with the normaliser taken from
 *   whole_stats = device double[3], the sums {S, Q, D B} of the whole batch.  loss receives this
 *   part's share of the whole batch's loss (Poisson: -sum(I_meas^p log(I_model^p + eps) - I_model^p)
 *   / S over this part's pixels; Gaussian: sqrt(D B / Q) Q_part / S).  The PACBED and sparsity terms
 *   (w_pacbed, w_sparse) compare or average over the whole batch at once and must be 0 here
 *   (PTY_EINVAL).  Other arguments, layouts and error codes as pty_loss_grad. */
int pty_loss_stats(const pty_geom* geom, int B, const int32_t* idx, const float* amp,
                   const float* phase, const float* probe, const float* pos, const float* tilt,
                   const float* dz, const float* I_meas, double* stats, void* ws, size_t ws_bytes,
                   void* stream);
int pty_loss_grad_part(const pty_geom* geom, int B, const int32_t* idx, const float* amp,
                       const float* phase, const float* probe, const float* pos, const float* tilt,
                       const float* dz, const float* I_meas, const double* whole_stats, double* loss,
                       float* I_model, float* g_amp, float* g_phase, float* g_probe, float* g_pos,
                       float* g_tilt, float* g_dz, int accumulate, void* ws, size_t ws_bytes,
                       void* stream);

/* Forward model as pty_forward, keeping in ws what pty_backward needs (checkpoints per
 * geom->ckpt_stride, far-field waves, transmission, probe spectra).  The parameters and ws must not
 * change between this call and the matching pty_backward. */
int pty_forward_save(const pty_geom* geom, int B, const int32_t* idx, const float* amp,
                     const float* phase, const float* probe, const float* pos, const float* tilt,
                     const float* dz, float* I_model, void* ws, size_t ws_bytes, void* stream);

/* Adjoint of the forward model of the preceding pty_forward_save on the same ws and arguments: the
 * gradients of a caller-defined loss whose derivative with respect to the modelled patterns is
 * dL_dI (float [B][N][N], DC-centred).  Gradient arrays, mask and accumulate as pty_loss_grad.
 * This is the backward of an autograd function wrapping the forward model. */
int pty_backward(const pty_geom* geom, int B, const int32_t* idx, const float* amp,
                 const float* phase, const float* probe, const float* pos, const float* tilt,
                 const float* dz, const float* dL_dI, float* g_amp, float* g_phase, float* g_probe,
                 float* g_pos, float* g_tilt, float* g_dz, int accumulate, void* ws, size_t ws_bytes,
                 void* stream);

/* Constraints applied after an optimiser step (Sec. "Physical constraints").  Each object
 * constraint is relaxed: x <- x + r (C(x) - x) with r in [0, 1] (r = 1: the plain constraint,
 * r = 0: off).  Order: probe orthogonalisation; then, on the object, the k_z filter, the depth blur,
 * then clipping negative phase to zero (each object mode on its own).
 *   k_z filter (Eq. 10-12): amp and phase are each filtered through the periodic 3D DFT of the
 *     Nz x H x W object by W_a(k) = (1 - (2/pi) atan(beta^2 k_z^2 / (k_x^2 + k_y^2 + 1e-3)))
 *     exp(-alpha (k_x^2 + k_y^2)), k in cycles per angstrom (pixel size dx, slice spacing dz).
 *     On when kz_relax > 0 and beta or alpha > 0.  H, W <= 8192, Nz <= 128.
 *   depth blur (Eq. 13): a Gaussian of standard deviation rz_sigma slices along the slice axis,
 *     truncated at 4 sigma and renormalised at the top and bottom of the volume.  Nz <= 128.
 *   probe orthogonalisation (mixed-state probe): the M modes (rows of an M x N^2 matrix A) become
 *     the eigenmodes of their density matrix, Q = U^H A with A A^H = U diag(lambda) U^H, ordered by
 *     decreasing power lambda, each column of U turned so its largest-magnitude entry is real
 *     positive.  Not relaxed.  M <= 32. */
typedef struct {
  float phase_positivity; /* relaxation of the phase >= 0 clip, 0 = off */
  float rz_sigma;         /* depth-blur standard deviation in slices, 0 = off */
  float rz_relax;         /* relaxation of the depth blur */
  float kz_beta;          /* strength beta of the k_z filter (dimensionless) */
  float kz_alpha;         /* lateral Gaussian alpha of the k_z filter, square angstrom */
  float kz_relax;         /* relaxation of the k_z filter, 0 = off */
  int probe_orthogonalize; /* nonzero: orthogonalise the probe modes */
} pty_constraints;

/* Bytes of device workspace pty_constrain needs for `c` (0 when only the blur and the clip are
 * on, or on invalid arguments): the k_z filter's complex volume (8 Nz H W bytes) and the
 * orthogonalisation's Gram partials and eigenvectors. */
size_t pty_constrain_workspace_size(const pty_geom* geom, const pty_constraints* c);

/* Applies `c` in place on `stream`: amp, phase [Nz][H][W] float, probe [M][N][N] complex64 (real,
 * imaginary interleaved), dz the device scalar of the slice spacing (read by the k_z filter only).
 * Pointers that `c` does not use may be NULL.  ws: device workspace of at least
 * pty_constrain_workspace_size bytes, 256-byte aligned (NULL when that is 0).  Returns PTY_EINVAL
 * on bad arguments or sizes, PTY_ECUDA on a launch failure; no host synchronisation. */
int pty_constrain(const pty_geom* geom, float* amp, float* phase, float* probe, const float* dz,
                  const pty_constraints* c, void* ws, size_t ws_bytes, void* stream);

/* One Adam step on the parameters in place using the gradients already in g_* (pty_adam state).
 * step is the 1-based Adam step count used for bias correction. */
int pty_adam_update(const pty_geom* geom, float* amp, float* phase, float* probe, float* pos,
                    float* tilt, float* dz, const float* g_amp, const float* g_phase,
                    const float* g_probe, const float* g_pos, const float* g_tilt,
                    const float* g_dz, const pty_adam* adam, int step, void* stream);

/* pty_loss_grad (accumulate = 0) followed by pty_adam_update: one gradient-descent iteration on
 * one batch (Sec. "Optimizers and loss functions", Adam).  Parameters are updated in place. */
int pty_step(const pty_geom* geom, int B, const int32_t* idx, float* amp, float* phase,
             float* probe, float* pos, float* tilt, float* dz, const float* I_meas, double* loss,
             float* g_amp, float* g_phase, float* g_probe, float* g_pos, float* g_tilt,
             float* g_dz, const pty_adam* adam, int step, void* ws, size_t ws_bytes, void* stream);

/* Synchronises `stream` and returns the OR of the device status bits (PTY_EBOUNDS,
 * PTY_ENONFINITE, PTY_ETIMEOUT) set since the last call that used this workspace began; a negative value if the
 * status could not be read.  Each pty_forward / pty_loss_grad / pty_step clears the word first. */
int pty_status(const void* ws, void* stream);

/* Message of the last error returned on the calling thread ("" if none). */
const char* pty_last_error(void);

/* Bit mask of the FFT sizes N this build supports (bit k set: N = 2^k). */
int pty_supported_sizes(void);

/* pty_loss_grad without a caller-supplied workspace, for callers that cannot allocate device memory:
 * code running inside a host framework that owns every device allocation through its own pool, or
 * a real-time loop that cannot afford the device-wide synchronisation of cudaMalloc / cudaFree.
 * There is no counterpart in the paper; the computation is exactly pty_loss_grad's.
 *  - Scratch is a fixed array of PTY_NOALLOC_SCRATCH_BYTES (32 MiB) inside this library's device
 *    code.  Every GPU that loads the library holds it until the process exits.  A batch whose
 *    pty_workspace_size() exceeds it is rejected with PTY_EWORKSPACE before anything is launched.
 *    The workspace holds the transmission and its gradient (16 bytes per object voxel) besides the
 *    per-wave buffers, so the object alone must stay under 2 Mi voxels (for example 8 x 512 x 512
 *    does not fit, 1 x 1024 x 1024 fits with a few 64 x 64 waves).
 *  - The call allocates nothing.  Its first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call before any stream
 *    capture on the device.
 *  - All calls share the one array, which keeps the last call's contents (the pass clears what it
 *    accumulates into).  Calls whose work overlaps on the GPU (other streams, other host threads)
 *    race on it: serialise them.
 *  - status: optional device int that receives the call's device status bits (as pty_status would
 *    report them) once the stream reaches the end of the call; may be NULL.
 *  Other arguments, layouts and error codes as pty_loss_grad. */
#define PTY_NOALLOC_SCRATCH_BYTES (32u << 20)
int pty_loss_grad_noalloc(const pty_geom* geom, int B, const int32_t* idx, const float* amp,
                          const float* phase, const float* probe, const float* pos,
                          const float* tilt, const float* dz, const float* I_meas, double* loss,
                          float* I_model, float* g_amp, float* g_phase, float* g_probe,
                          float* g_pos, float* g_tilt, float* g_dz, int accumulate, int* status,
                          void* stream);

/* Diagnostics for throughput measurement (not needed to use the library).
 * pty_launch_count: number of kernels this library has launched in the process so far.
 * pty_profile_enable(1) resets and starts per-kernel timing: every later pipeline call records a CUDA
 *   event after each of its kernels on the call's stream (up to 256 calls are kept); (0) stops it.
 * pty_profile_read fills ms[k] with the summed device time of pipeline stage k over the recorded
 *   calls, for k < min(n, PTY_PROF_STAGES), synchronising on the recorded events; returns the number
 *   of calls recorded, or -1 on a CUDA error.  Stages: 0 prepare_object, 1 probe_spectrum, 2 forward,
 *   3 loss, 4 loss_finalize, 5 adjoint, 6 object_grad, 7 probe_grad, 8 scalar_grad. */
#define PTY_PROF_STAGES 9
long long pty_launch_count(void);
int pty_profile_enable(int on);
int pty_profile_read(double* ms, int n);

/* Diagnostics for failure detection (not needed to use the library).  Every spin-wait of the
 * tensor-core GEMM (split-precision DFTs, learned initialiser) is bounded: after a number of
 * non-blocking polls it gives up, sets PTY_ETIMEOUT in the status word, waits for the matrix
 * products it has already issued, releases its tensor memory and returns, so the context stays
 * usable.  pty_set_wait_limit sets the poll limit of the pipeline waits of later launches
 * (0 .. PTY_WAIT_POLLS_DEFAULT; negative restores the default), so a test can make a wait run out
 * without a fault.  The wait for the already-issued products before the tensor memory is released
 * always keeps the default limit.  Not thread-safe with concurrent launches; returns PTY_OK. */
#define PTY_WAIT_POLLS_DEFAULT (1LL << 24)
int pty_set_wait_limit(long long polls);

/* Diagnostics: FP32 fused-multiply-add throughput of this GPU, the measured denominator of the
 * ALU roofline.  Launches `blocks` CTAs of 512 threads on `stream`; each thread runs iters x 128
 * independent FMAs (eight chains), so a launch does blocks x 512 x iters x 256 flops.  sink: a
 * device float that is never written in practice.  Time it with events on the stream. */
int pty_fma_probe(float* sink, int blocks, int iters, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PTY_H */

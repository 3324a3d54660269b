/*
 * ss.h -- C ABI of libss: the simplified string method of Heistracher et al. (arXiv:1804.07135)
 * for atomistic skyrmion annihilation barriers, on one NVIDIA GB300 (sm_103a).
 *
 * Model (Sec. II, Eq. 1): classical unit spins s_i on an nx*ny*nz simple cubic lattice with free
 * (open) boundaries; Hamiltonian = exchange J over nearest-neighbour bonds + interfacial DMI D with
 * the (r_ij x z).(s_i x s_j) form + uniaxial anisotropy K along z + dipole-dipole coupling.
 * Reduced units throughout: energies in the unit of J, lengths in lattice constants, the field is
 * h_i = -dE/ds_i (Eq. 2 with mu0|S| absorbed) and the dipole strength is w = mu0|S|^2/(4 pi a^3).
 *
 * One iteration of the string (Sec. III) = for every image: effective field (Eqs. 2-7, the dipole
 * part as a zero-padded FFT convolution with the tensor of Eq. 7), per-image FP64 energy (Eq. 8),
 * one explicit projected-descent step s <- normalise(s + dt (h - (s.h) s)) (Eq. 10 with the force of
 * Eq. 13); then equal-arc-length reparametrisation of the images (Eqs. 11-12, piecewise-linear
 * interpolation followed by per-site renormalisation; the two end images are kept).
 *
 * Conventions shared by every entry point:
 *   - Return codes only; nothing is thrown across the ABI.  On failure ss_last_error() describes it.
 *   - Spin/field arrays crossing the ABI are [image][site][3] (x, y, z components), site index
 *     (z*ny + y)*nx + x, dtype SS_DTYPE_F32 or SS_DTYPE_F64, on the host (on_device = 0) or on the
 *     context's device (on_device = 1).  They are caller-owned and never retained.
 *   - All device memory is owned by the context (allocated in ss_create* or on first use of a variant,
 *     freed in ss_destroy), from cudaMalloc or from the allocator given to ss_set_allocator.
 *   - Work is issued on an internal stream that is ordered after, and before, opts.stream (or the
 *     legacy default stream when opts.stream is NULL).  ss_step is asynchronous; every other call
 *     that returns data synchronises.  A sticky device error word (non-finite values) is read at
 *     every synchronising call and reported as SS_ERR_NONFINITE.
 *   - A context is not thread-safe: calls on one context must not overlap.
 */
#ifndef SS_H
#define SS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ss_ctx ss_ctx; /* opaque; owned by the library */

typedef enum {
    SS_OK = 0,
    SS_ERR_INVALID_ARG = 1, /* bad dims, parameters, indices, dtype, or a zero-norm/non-finite spin */
    SS_ERR_CUDA = 2,        /* a CUDA runtime call failed (message in ss_last_error) */
    SS_ERR_OOM = 3,         /* device or host allocation failed */
    SS_ERR_NONFINITE = 4,   /* a NaN/Inf appeared in an energy or arc length on the device */
    SS_ERR_TIMEOUT = 5,     /* reserved for bounded device waits */
    SS_ERR_STATE = 6        /* call out of order (e.g. ss_step before any ss_set_path) */
} ss_status;

enum { SS_DTYPE_F32 = 0, SS_DTYPE_F64 = 1 };
enum { SS_PREC_FP32 = 0, /* FP32 spins, fields and FFTs; FP64 energies and arc lengths */
       SS_PREC_FP64 = 1  /* the plain FP64 GPU method: FP64 everywhere */ };
enum { SS_DIPOLE_OFF = 0, SS_DIPOLE_DIRECT = 1, SS_DIPOLE_FFT = 2 };

typedef struct {
    double dt;          /* step length of the projected-descent step (> 0); prefactors of Eq. 9 absorbed */
    int precision;      /* SS_PREC_FP32 or SS_PREC_FP64 */
    int dipole;         /* SS_DIPOLE_FFT (default: the zero-padded FFT convolution of Sec. II-A),
                           SS_DIPOLE_DIRECT (the O(N^2) sum of Eq. 6 over all pairs of an image, for
                           small lattices and as an FFT-free check), or SS_DIPOLE_OFF (dipole term
                           dropped whatever w) */
    int reparam_every;  /* 1 = reparametrise after every step (Sec. III); 0 = never (plain relaxation);
                           other values are SS_ERR_INVALID_ARG */
    void* stream;       /* cudaStream_t to order against, e.g. torch.cuda.current_stream(); NULL = legacy */
} ss_opts;

typedef struct {
    int nx, ny, nz;        /* lattice dimensions, each >= 1 */
    double J, D, K, w;     /* exchange, DMI, anisotropy, dipole strength (finite) */
    int n_images;          /* images of this string, >= 2 */
} ss_string_desc;

/* Fills *opts with dt = 0.1, SS_PREC_FP32, SS_DIPOLE_FFT, reparam_every = 1, stream = NULL. */
void ss_default_opts(ss_opts* opts);

/* Creates a context holding one string of n_images images on an nx*ny*nz lattice (Sec. II, III).
 * opts may be NULL (defaults).  Errors: SS_ERR_INVALID_ARG, SS_ERR_OOM, SS_ERR_CUDA; *out is NULL
 * on failure. */
ss_status ss_create(int nx, int ny, int nz, double J, double D, double K, double w_dip, int n_images,
                    const ss_opts* opts, ss_ctx** out);

/* Creates a context holding n_strings independent strings (a parameter study, Sec. IV), each with its
 * own lattice, constants and image count; strings of equal lattice size share one batched launch per
 * kernel and one dipole spectrum. */
ss_status ss_create_batch(int n_strings, const ss_string_desc* descs, const ss_opts* opts, ss_ctx** out);

/* Sets the path of string `string` from `spins` ([n_images][N][3], dtype, host or device).  Each spin
 * is normalised on copy.  Errors: SS_ERR_INVALID_ARG for a bad index/dtype or any zero-norm or
 * non-finite input spin (the stored path is then unspecified until the next successful call).
 * Synchronises. */
ss_status ss_set_path(ss_ctx* ctx, int string, const void* spins, int dtype, int on_device);

/* Copies the current (reparametrised) path of `string` into `out` ([n_images][N][3]).  Synchronises.
 * ss_get_path followed by ss_set_path resumes bit-exactly (checkpoint/resume). */
ss_status ss_get_path(ss_ctx* ctx, int string, void* out, int dtype, int on_device);

/* Runs n_iter >= 0 iterations of the string method (Sec. III) on every string of the context.
 * Asynchronous on the context's stream (replayed from a captured CUDA graph) under the Euler step;
 * under a Runge-Kutta integrator (ss_set_integrator) it synchronises once per round of attempts.
 * Errors raised on the device are reported by the next synchronising call.  SS_ERR_STATE if some
 * string has no path. */
ss_status ss_step(ss_ctx* ctx, int n_iter);

/* Energy (Eq. 1 / Eq. 8) of every image of the current path of `string`, into host out[n_images]: a
 * fresh FP64 evaluation of the current path -- the stored spins renormalised in FP64, every term
 * (the dipole convolution included) in FP64.  On an SS_PREC_FP32 context this is the FP64 pipeline
 * applied to the FP32 state widened to FP64, so the reported energies carry no FP32 round-off of
 * their own (only the FP32 trajectory's); its FP64 buffers (about twice the context's) are allocated
 * on the first call of this, ss_barrier, ss_energy_terms or ss_grad with dE_dJDKw.  Synchronises. */
ss_status ss_energies(ss_ctx* ctx, int string, double* out);

/* Per-image energies from the last ss_step iteration (the state before that iteration's step),
 * reduced in FP64 from per-site FP32 terms (FP64 terms on the FP64 path): the energy curve of each
 * iteration (Sec. III).  Host out[n_images].  Synchronises. */
ss_status ss_step_energies(ss_ctx* ctx, int string, double* out);

/* Barrier of `string` (Sec. III): *dE = max_k E_k - E_0 over the FP64 energies of ss_energies, *k_max =
 * the maximising image (lowest index on ties).  On an SS_PREC_FP32 context only the images that can
 * decide it are evaluated in FP64: the FP32 evaluation bounds every image's energy (its FFT round-off
 * bound), and image 0 and every image whose upper bound reaches the highest lower bound are evaluated by
 * the FP64 pipeline, so the result equals the one from all FP64 energies; the selection is made once
 * per size group and path state and shared by the group's strings.  Either pointer may be NULL.
 * Synchronises. */
ss_status ss_barrier(ss_ctx* ctx, int string, double* dE, int* k_max);

/* Effective field h = -dE/ds (Eqs. 2-7) of every image of the current path of `string` into `out`
 * ([n_images][N][3], dtype, host or device).  Synchronises. */
ss_status ss_field(ss_ctx* ctx, int string, void* out, int dtype, int on_device);

/* Derivatives of the energy of image `image` of `string` (Eq. 2 and the linearity of Eq. 1 in its
 * constants): dE_ds ([N][3], dtype, host or device; may be NULL) receives dE/ds = -h (the field in the
 * context's precision), and dE_dJDKw (host, 4 doubles; may be NULL) receives (dE/dJ, dE/dD, dE/dK,
 * dE/dw), each the energy term with its constant set to 1, from the FP64 evaluation of ss_energies.
 * Synchronises. */
ss_status ss_grad(ss_ctx* ctx, int string, int image, void* dE_ds, int dtype, int on_device, double* dE_dJDKw);

/* The four energy terms of every image of the current path of `string`, from one evaluation: host
 * out[n_images][4] = (dE/dJ, dE/dD, dE/dK, dE/dw) per image (Eq. 1 is linear in each constant, so each
 * entry is that term with its constant set to 1), from the FP64 evaluation of ss_energies.
 * Synchronises. */
ss_status ss_energy_terms(ss_ctx* ctx, int string, double* out);

/* Measures the kernels of one iteration in the current mode: each entry is launched on its own (not
 * from the graph) on the context's stream, bracketed by CUDA events, for `reps` >= 1 timed iterations
 * after one untimed iteration.  ms_out[i] (host, up to max_out entries) receives the mean duration in
 * milliseconds of entry i, in launch order.  Euler step, for each size group: xfwd, yz (with the FFT
 * dipole term), the direct dipole sums (with SS_DIPOLE_DIRECT), xinv (in its step, climbing-image or LLG
 * mode), the two climbing-image kernels as one entry (climbing image on), arc (which also
 * reparametrises), the spline apply kernel (spline on).  Runge-Kutta integrators, for each size group an
 * iteration with a single attempt round: the interval's opening (x-forward, copy into y0, control) as
 * one entry, per stage the assembly, xfwd, yz, direct sums and xinv (force mode) as above, then finish,
 * control, commit, arc and spline apply (an interval that needs more attempts is left unfinished; the
 * next ss_step opens a new one).  *n_out receives the number of entries.  The strings advance by
 * reps + 1 iterations.  Synchronises. */
ss_status ss_time_kernels(ss_ctx* ctx, int reps, double* ms_out, int max_out, int* n_out);

/* Effective field of a batch of images, for callers that cannot allocate device memory.  The paper
 * has no counterpart: this entry point exists for code that must not call cudaMalloc -- an application
 * that owns all device memory through its own pool, or a plugin whose host forbids allocation.  It
 * returns the same field as ss_field on an FP32 context (dipole term by the zero-padded FFT
 * convolution) without a context and without allocating: every intermediate lives in one device array
 * built into libss, of 32 MiB, which each GPU that loads the library keeps reserved until the process
 * exits.
 *   spins  device memory of the current device, [n_images][N][3] float32 (normalised on the fly; need
 *          not be unit length)
 *   field  device memory of the current device, [n_images][N][3] float32, written
 *   stream cudaStream_t (NULL = legacy default stream); the call synchronises it before returning
 * Limits: dims in [1,1024] x [1,1024] x [1,64], n_images in [1,1024], and the scratch the call needs
 * must fit the 32 MiB array -- roughly 96*nz*Px*Py bytes while the dipole spectrum is built (Px, Py
 * the padded lengths, about 2*nx and 2*ny) and 24*n_images*N + 48*ceil(n_images/2)*nz*ny*Px bytes
 * for the images; larger requests return SS_ERR_INVALID_ARG without touching the GPU.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress, with that
 * device current) and raises kernel shared-memory limits.  The call cannot be captured in a CUDA graph:
 * it synchronises its stream and reads an error word back, so a stream under capture is refused with
 * SS_ERR_STATE before any work is issued.  All calls share the one array and it keeps the last call's
 * contents (each call rewrites what it reads and clears its error word), so calls whose GPU work
 * overlaps -- on two streams, or from two threads -- race and must be serialised by the caller.
 * Errors: SS_ERR_INVALID_ARG (bad dims or constants, a pointer that is not device memory of the current
 * device, too large, or a zero-norm/non-finite input spin), SS_ERR_STATE (capturing stream),
 * SS_ERR_CUDA (no sm_103 device or a CUDA failure).  ss_last_error does not cover this call. */
ss_status ss_field_noalloc(int nx, int ny, int nz, double J, double D, double K, double w_dip, int n_images,
                           const float* spins, float* field, void* stream);

/* Launch configuration chosen for the size group of `string` (diagnostics): out[0..7] = padded
 * lengths Px, Py, rows per CTA of the x-forward and x-inverse kernels (autotuned at creation),
 * block sizes of the x-forward, y/z and x-inverse kernels, and the number of energy partials per
 * image. */
ss_status ss_launch_config(const ss_ctx* ctx, int string, int out[8]);

/* How ss_step evolves the images between reparametrisations (Sec. III). */
enum { SS_INT_EULER = 0, SS_INT_DOPRI5 = 1, SS_INT_DOPRI5_IMAGE = 2, SS_INT_RKF45 = 3, SS_INT_RKF45_IMAGE = 4 };

/* Chooses the evolution of the images.
 *   SS_INT_EULER (the default): one projected-Euler step of length opts.dt per iteration (Eqs. 10, 13).
 *   SS_INT_DOPRI5, SS_INT_DOPRI5_IMAGE: Sec. III's explicit Runge-Kutta evolution with adaptive step
 *   size -- the Dormand-Prince 5(4) pair integrates d phi/d tau = h - (phi.h) phi (Eq. 13) over the
 *   reduced interval opts.dt per iteration, either the whole string as one ODE system (DOPRI5: one
 *   error norm and one step per string) or every image as its own (DOPRI5_IMAGE: a norm and a step per
 *   image; the images do not interact between reparametrisations).
 *   SS_INT_RKF45, SS_INT_RKF45_IMAGE: the same with the Runge-Kutta-Fehlberg 4(5) pair (six stages, the
 *   fourth-order solution carried forward, the fifth-order one estimating the error), which Sec. III
 *   names beside Dormand-Prince.
 * An attempt is accepted when sqrt(mean_j (e_j / (atol + rtol max(|y_j|, |y5_j|)))^2) <= 1 over the
 * system's components (e = the 5th- minus the 4th-order increment).  The next step is
 * step * clamp(0.9 err^(-1/5), 0.2, 5), at most 1 after a rejection, and 0.2 after an attempt whose
 * stages overflowed to a non-finite norm (a rejection).  Attempts are cut to end at the interval's end.
 * Spins are renormalised after each accepted step, not at the stages.  Steps carry over from one
 * iteration to the next and restart at opts.dt when a path is set or an integrator is chosen.
 * Under the Runge-Kutta kinds ss_step synchronises once per round of attempts (the host decides whether
 * another round is needed) and replays no CUDA graph; every system of a size group takes part in each
 * round, a finished one with a zero step.  ss_step_energies reports the energies of the state each
 * interval started from.  rtol and atol (ignored for SS_INT_EULER) must be positive and finite.  A later
 * synchronising call returns SS_ERR_NONFINITE after more than 100000 attempts in one interval.
 * Allocates 9 copies of the string state per size group on first use. */
ss_status ss_set_integrator(ss_ctx* ctx, int kind, double rtol, double atol);

/* Adaptive-integrator state of `string`: for image = -1 the smallest carried step and the accepted and
 * rejected attempts summed over the string's systems; for image >= 0 those of the system holding that
 * image (the string's own under the whole-string kinds).  Counts run from the last ss_set_path or
 * ss_set_integrator; opts.dt and zeros under SS_INT_EULER.  Synchronises. */
ss_status ss_integrator_state(ss_ctx* ctx, int string, int image, double* step, long long* accepted,
                              long long* rejected);

/* Reparametrisation variants (Sec. III leaves the interpolation open, and names the climbing image as a
 * refinement of the saddle that the paper itself omits). */
enum { SS_INTERP_LINEAR = 0, SS_INTERP_SPLINE = 1 };

/* Chooses how the images are redistributed after each evolution.
 *   interp = SS_INTERP_LINEAR (the default): piecewise-linear interpolation in alpha (Eq. 12), then
 *   per-site renormalisation.  SS_INTERP_SPLINE: a natural cubic spline (second derivative zero at the
 *   ends) through (alpha*_j, phi*_j) per Cartesian component, evaluated at the targets and renormalised
 *   per site; a part of the string with a zero-length segment is interpolated linearly.  Strings of at
 *   most 256 images (longer: SS_ERR_INVALID_ARG).
 *   climb = 1: the climbing image.  The interior image of highest energy among the states an iteration
 *   started from climbs in the next iteration (none in a path's first iteration; lowest index on ties):
 *   its Euler step uses the projected force F = h - (s.h) s with its component along the unit tangent
 *   reversed, F - 2 (F.tau) tau / (tau.tau), tau = (phi_{kc+1} - phi_{kc-1}) projected per site onto
 *   the tangent plane at phi_kc (states before the step); the reparametrisation then treats [0, kc]
 *   and [kc, K-1] as two strings, each brought to equal arc length, kc keeping its place.  Climbing is
 *   defined for the Euler step only (SS_ERR_STATE under a Runge-Kutta integrator, and
 *   ss_set_integrator refuses a Runge-Kutta kind while it is on).
 * Adds 2 launches per size group and iteration for the climbing image and 1 for the spline; allocates
 * one string-state copy per size group for the climbing image and 2 K^2 doubles per string for the
 * spline on first use.  Takes effect at the next ss_step (a linear reparametrisation still pending
 * from the previous iteration is applied first); every string restarts without a climbing image. */
ss_status ss_set_reparam(ss_ctx* ctx, int interp, int climb);

/* The image of `string` that climbs in the next iteration, or -1 (none, or climbing off).  Synchronises. */
ss_status ss_climbing_image(ss_ctx* ctx, int string, int* k);

/* What ss_step integrates (Eq. 9). */
enum { SS_DYN_STRING = 0, SS_DYN_LLG = 1 };

/* Chooses the dynamics.  SS_DYN_STRING (the default): the string method of Sec. III (the damping force of
 * Eq. 13, then the reparametrisation).  SS_DYN_LLG: the full precessional Landau-Lifshitz-Gilbert
 * equation (Eq. 9) in reduced units (h in units of J, time in units of mu0 |S| / (gamma J)),
 *     ds/dtau = -1/(1 + alpha^2) s x h - alpha/(1 + alpha^2) s x (s x h),
 * for every image as an independent system with no reparametrisation: each ss_step iteration advances
 * time by opts.dt, by one explicit Euler step with renormalisation (SS_INT_EULER) or by the adaptive
 * Runge-Kutta evolution chosen with ss_set_integrator; ss_step_energies reports the energies of the
 * states each iteration started from.  alpha (the damping) must be finite and >= 0.  The climbing image
 * is refused under SS_DYN_LLG (SS_ERR_STATE) and the interpolation choice has no effect there.  Takes
 * effect at the next ss_step; no synchronisation. */
ss_status ss_set_dynamics(ss_ctx* ctx, int kind, double alpha);

/* Device allocator for contexts (optional).  By default a context's device memory comes from
 * cudaMalloc and goes back with cudaFree in ss_destroy.  A framework with its own caching allocator
 * (e.g. PyTorch's) can supply one instead: alloc(bytes, device, stream, user) returns device memory on
 * `device` aligned to 256 bytes (or NULL: the creating call fails with SS_ERR_OOM; a misaligned pointer
 * is handed back to free and the call fails with SS_ERR_INVALID_ARG), free(ptr, bytes, device, stream,
 * user) releases it; `stream` is the context's opts.stream.  The pair applies to contexts created after
 * the call (each context keeps the pair it was created with, and frees through it in ss_destroy after
 * synchronising its work), so the allocator must outlive them.  alloc and free both NULL restore
 * cudaMalloc; one NULL and not the other is SS_ERR_INVALID_ARG.  Process-wide and thread-safe.  Scratch
 * of ss_create's one-off tensor-spectrum build and ss_field_noalloc's array are not affected. */
typedef void* (*ss_alloc_fn)(size_t bytes, int device, void* stream, void* user);
typedef void (*ss_free_fn)(void* ptr, size_t bytes, int device, void* stream, void* user);
ss_status ss_set_allocator(ss_alloc_fn alloc, ss_free_fn free, void* user);

/* Shape queries. */
int ss_num_strings(const ss_ctx* ctx);
ss_status ss_string_info(const ss_ctx* ctx, int string, ss_string_desc* out);

/* Number of kernels ss_step launches per iteration (all strings), for launch accounting. */
int ss_kernels_per_iteration(const ss_ctx* ctx);

/* Last error message of this context (or of the last failed ss_create* when ctx is NULL). */
const char* ss_last_error(const ss_ctx* ctx);

/* Frees every resource of the context; NULL is allowed. */
void ss_destroy(ss_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SS_H */

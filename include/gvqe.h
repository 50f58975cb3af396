/*
 * gvqe.h -- C ABI of the GB300 (sm_103a) engine for the Graph-VQE hot path:
 * state-vector simulation of the RY+CX hardware-efficient ansatz, the
 * expectation of a Pauli-sum Hamiltonian, and its gradient (arxiv 2607.02749).
 *
 * Conventions used by every call:
 *   - Qubit q is bit q of the basis index x (little-endian).
 *   - A Pauli string has one character per qubit over {I, X, Y, Z};
 *     character i acts on qubit i.
 *   - The ansatz (Section IV-B, Eq. 7): an initial rotation layer, then
 *     `reps` repetitions of [entangler, rotation layer].  The linear entangler
 *     is CX(0,1), CX(1,2), ..., CX(n-2,n-1) in that order (others below).  A
 *     rotation layer is RY on every qubit (default) or the full EfficientSU2
 *     layer RY then RZ on every qubit (GVQE_OPT_GATES, below).
 *   - Parameters are flattened layer-major: theta[p] with p = r*n + q is the
 *     RY angle of layer r (0..reps) on qubit q; P = n*(reps+1) (Eq. 8 for the
 *     RY-only gate set; see GVQE_GATES_RY_RZ for the full one).
 *   - RY(t) = [[cos t/2, -sin t/2], [sin t/2, cos t/2]] (Eq. 7).
 *
 * Ownership: *_create copies every input; the caller owns the parameter,
 * mask, energy and gradient buffers it passes.  Handles own their device
 * workspaces, which grow on first use and are freed by gvqe_destroy.
 *
 * Errors: every call returns GVQE_OK (0) or a negative code below and sets a
 * thread-local message readable with gvqe_last_error().  Argument checks are
 * synchronous; GPU work is enqueued on `stream` (a cudaStream_t passed as a
 * void*, NULL = the legacy default stream) and is complete when the stream is.
 * A handle must not be used by two calls that overlap in time.
 */
#ifndef GVQE_H
#define GVQE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GVQE_OK 0
#define GVQE_EINVAL (-1)       /* bad argument: NULL, size out of range, bad letter, n mismatch */
#define GVQE_ENOMEM (-2)       /* the device workspace does not fit in free device memory */
#define GVQE_ECUDA (-3)        /* a CUDA runtime call failed (message has the CUDA error) */
#define GVQE_ETIMEOUT (-4)     /* a bounded device-side wait ran out (persistent batch kernel) */
#define GVQE_EUNSUPPORTED (-5) /* a valid request this build does not implement */
#define GVQE_ECORRUPT (-6)     /* debug build: a device write landed outside its workspace */

/* flags for gvqe_energy / gvqe_energy_grad / gvqe_batch_create */
#define GVQE_FP32 0x0             /* FP32 amplitudes, FP64 table and FP64 reductions (default) */
#define GVQE_FP64 0x1             /* FP64 amplitudes */
#define GVQE_GRAD_ADJOINT 0x0     /* reverse-mode (adjoint) gradient (default) */
#define GVQE_GRAD_PARAM_SHIFT 0x2 /* parameter-shift gradient, Eq. 13 (2 P_active + 1 energies) */

/* entanglers for gvqe_ansatz_create (Section IV-B names the first three; Table 2
 * runs the method with all six), each an ordered CNOT list; r = 1..reps is the
 * entangler layer:
 * LINEAR         CX(0,1), CX(1,2), ..., CX(n-2,n-1)
 * CIRCULAR       CX(n-1,0) (the wrap-around) first, then the LINEAR list
 * FULL           CX(i,j) for every i < j, i ascending, j ascending within i
 * REVERSE_LINEAR CX(n-2,n-1), CX(n-3,n-2), ..., CX(0,1) (the same unitary as FULL)
 * PAIRWISE       CX(i,i+1) for even i ascending, then for odd i ascending
 * SCA            the CIRCULAR list rotated right by (r-1) mod n (its last gates
 *                move to the front), every CX(c,t) turned into CX(t,c) when r-1
 *                is odd (shifted-circular-alternating) */
#define GVQE_ENT_LINEAR 0
#define GVQE_ENT_CIRCULAR 1
#define GVQE_ENT_FULL 2
#define GVQE_ENT_REVERSE_LINEAR 3
#define GVQE_ENT_PAIRWISE 4
#define GVQE_ENT_SCA 5

/* options for gvqe_ansatz_set_option */
#define GVQE_OPT_TILE_BITS 1 /* log2 amplitudes per on-chip tile, 10..13 (FP64: 10..12); 0 = auto (13 FP32, 12 FP64) */
#define GVQE_OPT_GATES 2     /* rotation layer: GVQE_GATES_RY (default) or GVQE_GATES_RY_RZ */
#define GVQE_OPT_SPLIT_PASSES 3 /* strided-pass bit layout: 0 auto, 1 never split, 2 always split (when a layer
                                   takes two strided passes), 2 + y: split with y top qubits.  A split pass
                                   covers two runs of qubits, the low and the top ones, so that no pass's tile
                                   spans more 2 MiB pages than needed; results are the same up to the order of
                                   FP32/FP64 additions. */

#define GVQE_OPT_XY_TILE_BITS 4 /* log2 amplitudes per tile of the X-mask pass (strings with X/Y letters, RY
                                   layers), 10..13 (FP64: at most 12), 0 = those of the first pass */
#define GVQE_OPT_MPS_LAYERS 5 /* leading layers written in closed form: 0 = auto (up to 4), -1 = none, 1..4 =
                                 at most that many.  After r entangler + RY layers on the analytic layer-0
                                 product state, the linear, full and reverse-linear entanglers leave a state
                                 that is a product of 2^r x 2^r matrices along the qubits; FP32 plans with
                                 n >= 14 and reps >= 2 write layers 1..min(4, reps - 1)
                                 from contracted tables of those matrices (a write-only pass per state)
                                 instead of running their tile passes.  Same results up to FP32 rounding;
                                 the last layer always runs as tile passes. */
#define GVQE_OPT_MPS_TENSOR 6 /* closed-form layers at bond dimension 16 (four closed-form layers): 0 = auto
                                 (the writer's product per 2^13-amplitude chunk, 128 x 16 x 64, and the
                                 gradient pass's two lambda contractions, 64 x 128 x 16 and 128 x 64 x 16, on
                                 the tensor cores as tcgen05 TF32 MMAs with every operand split into two TF32
                                 parts, FP32 accumulators), -1 = both on the FP32 pipe.  Same results up to
                                 FP32 rounding. */

/* gate sets of a rotation layer (Eq. 8).
 * RY:    RY on every qubit; P = n (reps+1), theta[r*n + q]; real amplitudes.
 * RY_RZ: the full EfficientSU2 layer, RY on every qubit, then RZ on every
 *        qubit, RZ(t) = diag(exp(-i t/2), exp(+i t/2)); P = 2 n (reps+1), layer
 *        r's RY angle of qubit q at theta[2 r n + q] and its RZ angle at
 *        theta[2 r n + n + q].  Complex amplitudes (twice the memory and
 *        bandwidth; strings with an odd number of Y letters now contribute);
 *        every call but gvqe_energy_static (GVQE_EUNSUPPORTED); batches of
 *        such instances run instance by instance. */
#define GVQE_GATES_RY 1
#define GVQE_GATES_RY_RZ 2

#define GVQE_MAX_QUBITS 30

typedef struct gvqe_hamiltonian_s *gvqe_hamiltonian;
typedef struct gvqe_ansatz_s *gvqe_ansatz;
typedef struct gvqe_batch_s *gvqe_batch;

/*
 * gvqe_hamiltonian_create -- H = sum_k c_k P_k with real c_k (Eq. 6).
 *   n_qubits: 1..30.
 *   n_terms:  >= 0.
 *   pauli:    host, n_terms * n_qubits characters, string k at offset
 *             k*n_qubits, no separators; letters I, X, Y, Z (upper case).
 *   coeffs:   host, n_terms doubles.
 *   out:      receives the handle.
 * Duplicate strings are summed.  Z-only strings (and the all-I string) are
 * folded into a diagonal table E(x) = sum_k c_k (-1)^popcount(x & z_k) built
 * on the device in FP64; strings with X/Y letters are grouped by X-mask.
 * Strings with an odd number of Y letters contribute exactly zero to the
 * energy and gradient of every state this ansatz prepares (its amplitudes are
 * real), so they are counted and dropped.
 * Errors: GVQE_EINVAL (NULL, n out of range, bad letter), GVQE_ENOMEM, GVQE_ECUDA.
 */
int gvqe_hamiltonian_create(int n_qubits, int n_terms, const char *pauli, const double *coeffs,
                            gvqe_hamiltonian *out);

/*
 * gvqe_ansatz_create -- the parameterised circuit U(theta) of Section IV-B
 * (RY layers with an entangler between them; Eq. 7, Eq. 8 with RY only).
 *   n_qubits: 1..30.  reps: 0..64 (the number D of [entangler, RY] repetitions).
 *   entangler: one of GVQE_ENT_LINEAR .. GVQE_ENT_SCA.
 * Errors: GVQE_EINVAL; GVQE_EUNSUPPORTED if the layer-1 gather of this
 * entangler cannot use split product-state tables (none of the six at 1..30).
 */
int gvqe_ansatz_create(int n_qubits, int reps, int entangler, gvqe_ansatz *out);

/* gvqe_ansatz_set_option -- tuning override (see GVQE_OPT_*); value 0 restores the default. */
int gvqe_ansatz_set_option(gvqe_ansatz a, int option, int value);

/*
 * gvqe_energy -- E_b = <psi(theta_b)|H|psi(theta_b)> for b in [0, batch) (Eq. 4).
 *   params:   device, batch x P doubles, row b = theta_b (layer-major, see above).
 *   batch:    >= 1.
 *   energies: device, batch doubles (written).
 *   flags:    GVQE_FP32 or GVQE_FP64.
 *   stream:   cudaStream_t as void*.
 * The energy reduction always accumulates in FP64.
 * Errors: GVQE_EINVAL (NULL, batch < 1, n of ansatz != n of H), GVQE_ENOMEM, GVQE_ECUDA.
 */
int gvqe_energy(gvqe_ansatz a, gvqe_hamiltonian h, const double *params, int batch,
                double *energies, int flags, void *stream);

/*
 * gvqe_energy_grad -- energies and dE/dtheta for b in [0, batch).
 *   params:   device, batch x P doubles.
 *   mask:     device, batch x P bytes, nonzero = active (Eq. 11: parameters
 *             outside the active block are held fixed), or NULL = all active.
 *             The mask changes the gradient only: inactive entries are written
 *             as 0.0, energies are unaffected.
 *   energies: device, batch doubles.  grad: device, batch x P doubles.
 *   flags:    GVQE_FP32 | GVQE_FP64, optionally | GVQE_GRAD_PARAM_SHIFT
 *             (Eq. 13; this path copies the mask to the host and synchronises
 *             `stream`).
 * Gradient reductions accumulate in FP64 (FP32 mode sums at most one warp's
 * products in FP32 first).
 * Errors: as gvqe_energy.
 */
int gvqe_energy_grad(gvqe_ansatz a, gvqe_hamiltonian h, const double *params, const uint8_t *mask,
                     int batch, double *energies, double *grad, int flags, void *stream);

/*
 * gvqe_batch_create -- a fixed set of independent restricted-update problems
 * (Section IV-D, Eq. 11): instance i pairs ansatze[i] with hams[i] (equal n)
 * and evaluates one parameter vector with its own active mask per run.  The
 * same pair of handles may appear in several slots (several parameter vectors
 * of one subproblem per run).  Instances with RY layers and a diagonal (I/Z-
 * only) Hamiltonian run together in the batch's CUDA graph under its schedule
 * (gvqe_batch_set_option: staged by default, or one persistent kernel
 * launch); the others (X/Y strings, RY+RZ layers) are evaluated by single
 * gvqe_energy_grad calls on the same stream in the same gvqe_batch_run, after
 * the graph.  Staged results equal single calls bit for bit; the persistent
 * kernel's 2^12-amplitude tiles fix another summation order, so its results
 * agree with single calls within the precision bounds.
 *   n_inst: >= 1.  ansatze, hams: host arrays of n_inst handles (borrowed: they
 *   must outlive the batch).  flags: GVQE_FP32 or GVQE_FP64.
 * Errors: GVQE_EINVAL, GVQE_ENOMEM, GVQE_ECUDA, GVQE_EUNSUPPORTED.
 */
int gvqe_batch_create(int n_inst, const gvqe_ansatz *ansatze, const gvqe_hamiltonian *hams,
                      int flags, gvqe_batch *out);

/*
 * gvqe_batch_run -- evaluate every instance once.
 *   params:   host array of n_inst device pointers, params[i] -> P_i doubles.
 *   masks:    host array of n_inst device pointers (P_i bytes each, entries may
 *             be NULL = all active), or NULL = all active everywhere.
 *   energies: device, n_inst doubles.
 *   grads:    host array of n_inst device pointers (P_i doubles each), or NULL
 *             for energies only.
 * Errors: GVQE_EINVAL, GVQE_ECUDA, GVQE_ETIMEOUT (a bounded device-side wait
 * ran out; detected when this call synchronises `stream` at its end).
 */
int gvqe_batch_run(gvqe_batch b, const double *const *params, const uint8_t *const *masks,
                   double *energies, double *const *grads, void *stream);

/*
 * gvqe_batch_set_option -- schedule option of a batch (Section IV-D, Eq. 11:
 * the paper runs its blocks concurrently; the schedule of the one persistent
 * launch is this library's own).
 *   GVQE_BATCH_OPT_WAVE_BYTES: waves whose live bytes (three states of each
 *     instance: a pass's input, output and stored state or table) add up to at
 *     most this many bytes (0: one wave), so a wave's states can stay in L2
 *     between their passes.  Persistent: the instances, larger first, each
 *     wave stage-major (every instance's pass s before any instance's pass
 *     s + 1).  Staged: the plan groups, larger first, the groups of a wave side
 *     by side and a wave after the previous one.  Default 0 (one wave).
 *   GVQE_BATCH_OPT_SCHEDULE: GVQE_BATCH_STAGED (default): the instances with
 *     the same plan (n, reps, entangler, strided layout) form a group whose
 *     states, partial sums and diagonal tables sit job after job, and each
 *     group runs its plan's passes as launches of the regular pass kernels over
 *     all its jobs (as gvqe_energy_grad runs a batch of vectors), on its own
 *     branch of the graph; the branches run side by side.  Results equal those
 *     of single gvqe_energy_grad calls bit for bit, and every instance with RY
 *     layers and a diagonal H takes part, whatever its n.
 *     GVQE_BATCH_PERSISTENT: one persistent launch whose CTAs claim items
 *     (one 2^tile-bits tile of one pass) in ticket order and wait, with a
 *     bounded spin, for the previous step of the item's instance.  Both are
 *     captured in the batch's CUDA graph.
 *   GVQE_BATCH_OPT_TILE_BITS: 10, 11 or 12 (default), the log2 amplitudes of
 *     one work item of the persistent launch (FP32; FP64 batches take 12 only,
 *     else GVQE_EUNSUPPORTED).  2^10 makes every CTA one warp.  Under the
 *     persistent schedule, instances with fewer qubits than this are evaluated
 *     by single calls in the same run.
 * The schedule is rebuilt on the next run.
 * Results do not depend on the option (each instance's passes and reductions
 * are the same).  Errors: GVQE_EINVAL.
 *
 * gvqe_batch_autotune -- run the batch under the persistent schedule with
 * tiles of 2^12, 2^11, 2^10 (FP64: 2^12) in one wave and 2^12 in 256 MiB
 * waves, and under the staged schedule in one wave and in 128 and 256 MiB
 * waves (one warm-up run and three
 * timed runs under CUDA
 * events on `stream` each, with the caller's params / masks / outputs as in
 * gvqe_batch_run) and keep the fastest.  report (host, report_len bytes, or
 * NULL) receives the choice and the sweep.  A batch that runs instance by
 * instance has nothing to tune.  Errors: those of gvqe_batch_run.
 */
#define GVQE_BATCH_OPT_WAVE_BYTES 1
#define GVQE_BATCH_OPT_TILE_BITS 2
#define GVQE_BATCH_OPT_SCHEDULE 3
#define GVQE_BATCH_PERSISTENT 0
#define GVQE_BATCH_STAGED 1
int gvqe_batch_set_option(gvqe_batch b, int option, long long value);
int gvqe_batch_autotune(gvqe_batch b, const double *const *params, const uint8_t *const *masks, double *energies,
                        double *const *grads, char *report, int report_len, void *stream);

/*
 * gvqe_energy_static -- the energies of gvqe_energy, computed without any
 * device allocation.  The paper has no counterpart: this is for callers that
 * cannot allocate device memory when they need an energy (under a runtime
 * that owns every device allocation of the process or enforces a fixed memory
 * budget this library may not draw on, or in a loop that cannot afford the
 * first-call workspace allocation of gvqe_energy).
 *   a, h:     handles as for gvqe_energy; h must be diagonal (I/Z letters only,
 *             else GVQE_EUNSUPPORTED).
 *   params:   device, batch x P doubles.  energies: device, batch doubles.
 *   flags:    GVQE_FP32 or GVQE_FP64.  stream: cudaStream_t as void*.
 * All scratch (diagonal table, trig table, state vectors, partial sums) comes
 * from one file-scope device array of GVQE_STATIC_SCRATCH_BYTES that every GPU
 * loading this library holds until the process exits; requests that need more
 * (about n <= 19 at batch 1) return GVQE_EINVAL with the required size.  The
 * first call on each device looks up the array's device address (make it
 * before any stream capture).  Every call reuses the same array and clears what
 * must start at zero; calls whose GPU work overlaps in time race on it.  Its
 * host-to-device copies read only memory owned by the handles (the merged
 * diagonal terms of h, the cached energy plan of a).  Its launches count in
 * gvqe_launch_count and the event profiler like those of gvqe_energy.
 * Errors: GVQE_EINVAL, GVQE_EUNSUPPORTED, GVQE_ECUDA.
 */
#define GVQE_STATIC_SCRATCH_BYTES (16 * 1024 * 1024)
int gvqe_energy_static(gvqe_ansatz a, gvqe_hamiltonian h, const double *params, int batch,
                       double *energies, int flags, void *stream);

/*
 * gvqe_autotune -- choose the ansatz's tile plan by measurement.  The paper has
 * no counterpart (it names no kernel layout); the plan decides how the RY
 * layers of Section IV-B are cut into tile passes for the evaluations of Eq. 4
 * and Eq. 13.  Every distinct plan among tile bits 10 .. 13 (FP64: 10 .. 12)
 * and the strided layouts (one run of qubits per pass, or a low and a top run
 * of y = 1 .. 8 top qubits) runs the requested evaluation once to warm up and
 * then once (three times when a call takes under 50 ms, averaged) under
 * CUDA events on `stream`; the fastest becomes the ansatz's plan in that
 * precision (the other precision keeps its own; setting GVQE_OPT_TILE_BITS or
 * GVQE_OPT_SPLIT_PASSES later replaces both).  With X/Y strings (RY layers),
 * the X-mask pass's own tile size (GVQE_OPT_XY_TILE_BITS) is swept first, on
 * the default plan, and the plans are then timed with the fastest.
 * Candidates that do not fit in device memory are skipped.  Results of the tuned plan equal those of any
 * other plan up to the order of FP32/FP64 additions.
 *   a, h:       handles with equal n.
 *   params:     device, batch x P doubles (the evaluation that is timed).
 *   flags:      GVQE_FP32 or GVQE_FP64, plus GVQE_TUNE_ENERGY to tune the
 *               energy-only path (default: energy and adjoint gradient).
 *   cache_path: host path of a JSON file of earlier winners, or NULL.  The
 *               entry for this call's key (gvqe_tune_key) is used without any
 *               timing when present; otherwise the sweep runs and its winner is
 *               stored.  A missing, unreadable or malformed file counts as
 *               empty and is rewritten whole; deleting it is always safe.
 *   report:     host buffer of report_len bytes (or NULL): the choice and the
 *               sweep, one "tb=<bits>/<layout>: <ms> ms" item per candidate.
 *               The same text is appended to gvqe_ansatz_describe.
 * Synchronises `stream`.  Errors: GVQE_EINVAL, GVQE_ENOMEM (no candidate fits),
 * GVQE_ECUDA.
 */
#define GVQE_TUNE_ENERGY 0x4
int gvqe_autotune(gvqe_ansatz a, gvqe_hamiltonian h, const double *params, int batch, int flags,
                  const char *cache_path, char *report, int report_len, void *stream);

/*
 * gvqe_tune_key -- the cache key gvqe_autotune uses for (a, h, batch, flags):
 * GPU name (or "no-gpu"), n, reps, entangler, gate set, precision, gradient or
 * energy only, diagonal H or not, batch.  Host only.  Errors: GVQE_EINVAL.
 *
 * gvqe_tune_cache_get -- look `key` up in the JSON cache at `path` (host only):
 * returns 1 and fills tile_bits, split (a GVQE_OPT_SPLIT_PASSES value) and ms (may
 * be NULL) when present, 0 when the file is missing, unreadable, malformed or
 * has no such key, GVQE_EINVAL on NULL arguments.
 *
 * gvqe_tune_cache_put -- store or replace the entry for `key` (host only); an
 * invalid existing file is replaced by one holding this entry.  The file is
 * written to <path>.tmp<pid> and renamed over <path>.  Errors: GVQE_EINVAL (bad
 * arguments, or the file cannot be written).  Several processes may tune into
 * one file: each writes its own temporary and renames it over the file, so the
 * file is always whole (the last writer's entries win).
 */
int gvqe_tune_key(gvqe_ansatz a, gvqe_hamiltonian h, int batch, int flags, char *buf, int buflen);
int gvqe_tune_cache_get(const char *path, const char *key, int *tile_bits, int *split, double *ms);
int gvqe_tune_cache_put(const char *path, const char *key, int tile_bits, int split, double ms, const char *sweep);

/*
 * gvqe_readout -- read out the prepared state |psi(theta)> (Section IV-F:
 * sample the final state, take the most probable bitstring; Section V-A:
 * 8192 shots, seed 0, and the CVaR-alpha objective of Section III).
 * p(x) = |psi(x)|^2 over the 2^n computational basis states, total = sum_x p(x)
 * (1 up to rounding; shots and CVaR use p / total).
 *   a, h:     handles with equal n; h is only read when alpha > 0 and may be
 *             NULL otherwise.
 *   params:   device, P doubles (one parameter vector).
 *   flags:    GVQE_FP32 or GVQE_FP64 (state precision; p, sums and the CVaR
 *             are FP64 either way).
 *   alpha:    CVaR level in (0, 1], or 0 to skip it.  CVaR_alpha =
 *             (1/alpha) * integral_0^alpha F^-1(u) du, F the distribution of
 *             the outcome energy E(x) = <x|H|x> (the I/Z terms of H) under p:
 *             the mean energy of the lowest-energy alpha fraction of outcomes,
 *             the boundary outcome counted fractionally.
 *   n_shots:  >= 0.  uniforms: device, n_shots doubles in [0, 1) (the caller's
 *             random numbers; NULL when n_shots is 0).  shots: device,
 *             n_shots int64 (or NULL when n_shots is 0): shot k is the
 *             smallest x whose cumulative probability (in increasing x)
 *             exceeds uniforms[k] * total.
 *   stats:    device, 4 doubles: p(argmax), CVaR_alpha (NaN when alpha is 0),
 *             total, and the number of histogram passes the CVaR search made
 *             over the state (0 when alpha is 0).  argmax: device, 1 int64: the
 *             most probable x (smallest x on ties).
 * Deterministic (fixed summation orders, integer histogram counts).  The
 * CVaR search reads small histograms back to the host, so the call
 * synchronises `stream`.
 * Errors: GVQE_EINVAL (bad handle or pointer, alpha outside [0, 1],
 * n_shots < 0), GVQE_ENOMEM, GVQE_ECUDA, GVQE_EUNSUPPORTED (CVaR search did
 * not converge).
 */
int gvqe_readout(gvqe_ansatz a, gvqe_hamiltonian h, const double *params, int flags, double alpha,
                 int n_shots, const double *uniforms, int64_t *shots, double *stats, int64_t *argmax,
                 void *stream);

/* gvqe_destroy -- free any handle above; NULL is accepted.  Synchronises the
 * device work the handle enqueued before freeing its memory. */
int gvqe_destroy(void *handle);

/*
 * gvqe_set_device_memory_limit -- a budget for the device memory this library
 * holds in its workspaces (all handles of the process together); 0 removes it.
 * A call that would exceed it fails with GVQE_ENOMEM and leaves every handle
 * usable (a call over several parameter vectors first runs fewer of them per
 * launch to fit).  Host only.
 * gvqe_device_memory_in_use -- bytes held now.
 * Errors: GVQE_EINVAL (bytes < 0).
 */
int gvqe_set_device_memory_limit(long long bytes);
long long gvqe_device_memory_in_use(void);

/*
 * gvqe_debug_check -- debug builds (compiled with GVQE_DEBUG, libgvqe_debug.so):
 * every device workspace is allocated with a 4 KiB guard zone on each side,
 * filled with a known byte.  This call synchronises the device and checks every
 * live workspace's guards; a kernel that wrote past either end of its buffer
 * makes it fail with GVQE_ECORRUPT, the message naming the buffer's size, the
 * side and the first overwritten byte.  The guards cost two memsets per
 * allocation and leave every result bit-identical to the regular build.
 * Regular builds return GVQE_EUNSUPPORTED.
 */
int gvqe_debug_check(void);

/*
 * gvqe_debug_poke_guard -- debug builds, for testing gvqe_debug_check: from the
 * host (cudaMemset, no kernel), set (restore = 0) or reset (restore = 1) the
 * first byte above the largest live workspace, as an overrun by one byte would.
 * Errors: GVQE_EINVAL (no live workspace); regular builds GVQE_EUNSUPPORTED.
 */
int gvqe_debug_poke_guard(int restore);

/* gvqe_last_error -- message of the last failing call on this thread ("" if none). */
const char *gvqe_last_error(void);

/*
 * Host-only introspection (no GPU needed).
 * gvqe_plan_describe -- write the tile-pass plan used for (n_qubits, reps,
 * flags, tile_bits; 0 = auto) as text into buf (NUL-terminated, truncated to
 * buflen).  Returns the number of passes per rotation layer, or a negative code.
 */
int gvqe_plan_describe(int n_qubits, int reps, int flags, int tile_bits, char *buf, int buflen);

/*
 * gvqe_ansatz_describe -- the same text for the energy+gradient plan of an
 * ansatz handle with its options (entangler, gate set, tile bits, split
 * layout) at precision flags (GVQE_FP32 / GVQE_FP64).  Host only: builds (and
 * caches) the plan, touches no device memory.  Returns the passes per rotation
 * layer, or a negative code (GVQE_EINVAL for a bad handle or flags).
 */
int gvqe_ansatz_describe(gvqe_ansatz a, int flags, char *buf, int buflen);

/*
 * gvqe_entangler_inverse -- basis-index map of one entangler layer (Section
 * IV-B, Table 2): the entangler of layer r (1..reps) sends |x> to |A x>, a
 * GF(2)-linear permutation of basis indices; this writes x[i] = A^-1 y[i] for
 * count indices, the map the gathering passes apply.  Host arrays (y, x may
 * alias); every y[i] must lie in [0, 2^n_qubits).
 * Errors: GVQE_EINVAL (bad entangler, n, layer, count < 0, NULL, y out of range).
 */
int gvqe_entangler_inverse(int entangler, int n_qubits, int layer, const long long *y, long long *x,
                           long long count);

/*
 * Host-only Hamiltonian partitioning (Section IV-C; no GPU needed).
 *
 * gvqe_interaction_graph -- the weighted qubit interaction graph of Eq. 9:
 * w[i*n + j] = sum of |c_k| over the terms whose letters on qubits i and j
 * (i != j) are both non-identity; w[i*n + i] = 0.
 *   n_qubits: 1..GVQE_GRAPH_MAX_NODES.  pauli / coeffs as for
 *   gvqe_hamiltonian_create (host; duplicates are simply added).
 *   w: host, n_qubits^2 doubles (written).
 * Errors: GVQE_EINVAL (sizes, NULL, a letter outside IXYZ, a non-finite c).
 *
 * gvqe_partition -- blocks of qubits by the Louvain method: local moving of
 * nodes to the neighbouring community of largest modularity gain, then
 * aggregation, until a level moves nothing; maximising Eq. 10 with a
 * resolution gamma (gamma = 1 is Eq. 10 as printed):
 *   Q = 1/(2m) sum_ij [w_ij - gamma k_i k_j / (2m)] delta(c_i, c_j).
 * Then blocks smaller than min_block are merged: the smallest block (lowest
 * label on ties) joins the block it shares the most weight with (lowest label
 * on ties), or, sharing none, the smallest other block, until every block has
 * min_block qubits or one block is left.  Deterministic: nodes are visited in
 * ascending order, a node moves only when the best gain beats staying by more
 * than a relative 1e-12, near-equal gains go to the lowest community label.
 *   w: host, n x n, symmetric, finite, >= 0, zero diagonal.
 *   resolution: gamma >= 0.  min_block: S_min >= 1.
 *   block_of: host, n ints (written): block of node i, blocks numbered in
 *   order of their lowest node.  n_blocks, modularity: written if not NULL
 *   (Q of the final blocks at this gamma).
 * Errors: GVQE_EINVAL.
 */
#define GVQE_GRAPH_MAX_NODES 1024
int gvqe_interaction_graph(int n_qubits, int n_terms, const char *pauli, const double *coeffs, double *w);
int gvqe_partition(int n, const double *w, double resolution, int min_block, int *block_of, int *n_blocks,
                   double *modularity);

/* gvqe_hamiltonian_stats -- counts after parsing: diagonal strings, X-mask
 * groups, grouped strings, dropped odd-Y strings (any pointer may be NULL). */
int gvqe_hamiltonian_stats(gvqe_hamiltonian h, int *n_diag, int *n_groups, int *n_grouped,
                           int *n_dropped);

/* gvqe_version -- library version as 10000*major + 100*minor + patch. */
int gvqe_version(void);

/*
 * Launch accounting and per-kernel timing (for benchmarks).
 * gvqe_launch_count -- number of kernels this library has enqueued in this
 *   process so far (all handles, all streams).
 * gvqe_profile_enable -- when `on` is nonzero, every tile-pass launch is
 *   bracketed by two CUDA events recorded on the launching stream, and its
 *   algorithmic bytes (each state, table and lambda element it must read or
 *   write, counted once) are recorded.  0 turns recording off.
 * gvqe_profile_read -- waits for the recorded events, then returns for one
 *   kernel kind (GVQE_PROF_*) the number of launches, their summed device time
 *   in ms and their summed algorithmic bytes; any pointer may be NULL.
 * gvqe_profile_reset -- drops all recorded launches.
 */
#define GVQE_PROF_FWD 0       /* forward rotation passes */
#define GVQE_PROF_BWD 1       /* adjoint passes (gradient + inverse rotation) */
#define GVQE_PROF_GRAD_L0 2   /* layer-0 gradient pass */
#define GVQE_PROF_LAMBDA_XY 3 /* H psi with X-mask groups */
#define GVQE_PROF_WHT 4       /* diagonal-table Walsh-Hadamard passes */
int64_t gvqe_launch_count(void);
int gvqe_profile_enable(int on);
int gvqe_profile_read(int kind, int64_t *launches, double *ms, double *bytes);
int gvqe_profile_reset(void);

#ifdef __cplusplus
}
#endif

#endif /* GVQE_H */

/*
 * lbw.h -- C ABI of the GB300 curvilinear wave lattice-Boltzmann library (liblbw.so).
 *
 * Method: Velasco, Munoz, Mendoza, "Lattice Boltzmann model for the simulation of the wave
 * equation in curvilinear coordinates" (arXiv:1705.01801).  The library advances D3Q7
 * populations on a Cartesian lattice of computational coordinates (q1, q2, q3) (Sec. III,
 * first paragraph) with BGK relaxation at tau = 1/2 (Sec. II, Eq. eq:evolution and
 * Eq. SecondOrder), the corrected equilibrium (Eq. EquilibriumCurvedSystemHermiteCorrected),
 * the shifted momentum with the geometric forcing term (Eq. JCorrectionForce, Appendix A
 * Eq. JShifted) and the lattice-weighted derivative (Eq. DerivativeFromTaylor, Appendix B).
 *
 * Conventions for every entry point:
 *  - Plain C types only.  Pointers named host_* are host memory owned by the caller; the
 *    library copies from / to them before returning.  Device memory of a grid is owned by
 *    the library (allocated in lbw_create_grid on the grid's stream, freed in lbw_destroy).
 *  - Every call returns an lbw_status and never aborts, traps or exits.  On failure the
 *    thread-local message of lbw_last_error() says why.  LBW_ECUDA means a CUDA runtime call
 *    failed (the message carries cudaGetErrorString).
 *  - Work is enqueued on the CUDA stream given at creation (a cudaStream_t passed as void*,
 *    0 = the legacy default stream).  Calls that return host data synchronise that stream.
 *  - Node (q1, q2, q3) sits at physical coordinates x^a = x0[a] + (q_a + 1/2) h[a].
 *    Memory layout of every per-node array: q2 fastest, then q1, then q3
 *    (index = (q3 * n1 + q1) * n2 + q2); populations are seven such planes, i = 0..6 for
 *    xi = 0, +e1, -e1, +e2, -e2, +e3, -e3.
 *  - Frequencies are in radians per time step; time steps are 1 (Sec. II, delta_t = 1).
 */
#ifndef LBW_H
#define LBW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBW_OK = 0,
  LBW_EINVAL = 1,    /* invalid argument or descriptor */
  LBW_ENOMEM = 2,    /* device or host allocation failed */
  LBW_ECUDA = 3,     /* a CUDA runtime call failed */
  LBW_EUNSTABLE = 4, /* a probe or field value is not finite */
  LBW_ETIMEOUT = 5,  /* a bounded device wait ran out */
  LBW_ESTATE = 6     /* call out of order (e.g. step before init) */
} lbw_status;

/* Coordinate systems of Sec. IV: Eq. cylindricalsystem (polar = cylindrical with n3 = 1),
 * Eq. coordinatesTrumpet (flare s(z), see horn_profile) and Eq. CoordinatesTorus. */
typedef enum {
  LBW_CARTESIAN = 0,   /* (x, y, z) */
  LBW_POLAR = 1,       /* (r, theta, z), n3 must be 1 */
  LBW_CYLINDRICAL = 2, /* (r, theta, z) */
  LBW_TRUMPET = 3,     /* (r, theta, z), x = r s(z) cos(theta), y = r s(z) sin(theta) */
  LBW_TOROIDAL = 4     /* (r, theta major, phi minor), geom[0] = R */
} lbw_metric;

/* Face rules of Sec. IV.A (periodic, bounce-back with damping D, free = copy of the normal
 * neighbour) and anti-bounce-back for a Dirichlet P = 0 wall. */
typedef enum {
  LBW_BC_PERIODIC = 0,
  LBW_BC_BOUNCE = 1,
  LBW_BC_ANTIBOUNCE = 2,
  LBW_BC_FREE = 3
} lbw_bc;

/* Storage of the populations.  *S = 16-bit storage of f_i / w_i (the deviation from the
 * rest state P = 0, scaled by the weight) with FP32 arithmetic. */
typedef enum { LBW_F64 = 0, LBW_F32 = 1, LBW_F16S = 2, LBW_BF16S = 3 } lbw_prec;

typedef struct {
  int32_t kind;         /* lbw_metric */
  int32_t n[3];         /* nodes along q1, q2, q3 (q2 is the fastest axis in memory) */
  double h[3];          /* physical spacing per cell; angles: 2 pi / n */
  double x0[3];         /* physical coordinate of the lower face of each axis (r_in for r) */
  double c;             /* wave speed, physical units per time step */
  double tau;           /* relaxation time; must be 0.5 (Sec. II) */
  double cs2;           /* lattice cs^2, 0 < cs2 < 1/3; weights w0 = 1 - 3 cs2, wi = cs2 / 2 */
  double damping;       /* D of the bounce-back rule, 0 < D <= 1 (1 = lossless) */
  double geom[4];       /* torus: R; Bessel horn: Zmax, lambda; exp horn: a0, b, alpha */
  int32_t horn_profile; /* 0 = Bessel horn s = (Zmax - z)^-lambda (Sec. IV.B),
                           1 = exponential s = (a0 + b e^{alpha z}) / (a0 + b) */
  int32_t bc[6];        /* lbw_bc of faces -q1, +q1, -q2, +q2, -q3, +q3 */
  int32_t prec;         /* lbw_prec */
  int32_t geom_mode;    /* lbw_geom_mode: where the step kernel takes the geometry from */
  int32_t equilibrium;  /* lbw_equilibrium */
  int32_t reserved;     /* must be 0 */
} lbw_grid_desc;

/* Equilibrium of the collision.  CURVILINEAR is the paper's method (Sec. III: the Hermite
 * equilibrium at c = cs plus the geometric forcing term, Eqs. JCorrectionForce and
 * EquilibriumCurvedSystemHermiteCorrected), valid for every kind.  The two Cartesian schemes
 * that Sec. II compares (LBW_CARTESIAN only, FP32 or FP64 storage, table geometry):
 * MOMENT_MATCHING is Chopard's equilibrium (Eq. feqMomentMatchingCartesian),
 * f_0 = P (1 - (c^2 / cs^2)(1 - w_0)), f_i = (w_i / cs^2)(c^2 P + xi_i . J), whose stress is
 * c^2 P delta for any c; HERMITE is the truncated Hermite equilibrium of Eq. EquilibriumHermite,
 * f_i = w_i [P + xi_i . J / cs^2 + P (c^2 - cs^2)(|xi_i|^2 - 3 cs^2) / (2 cs^4)], f_0 = P - sum
 * of the others, whose wave speed on D3Q7 is c only at cs^2 = 1/5 (in general c_eff^2 =
 * cs^2 + (c^2 - cs^2)(1 - 3 cs^2) / (2 cs^2)).  Neither uses a forcing term; both take c in
 * cells per step (h is not applied) and need the rest weight 1 - 3 E >= 0, E = c^2 or c_eff^2. */
typedef enum { LBW_EQ_CURVILINEAR = 0, LBW_EQ_MOMENT_MATCHING = 1, LBW_EQ_HERMITE = 2 } lbw_equilibrium;

/* Geometry source of the fused step (Sec. IV: sqrt g, g^{ab} and G^a enter every node's
 * forcing term through 16 coefficients per (q1, q3) row, the same along q2 for every kind).
 * TABLE: built once on the host in FP64, rounded to the arithmetic type, staged per plane by
 * TMA with the populations.  ANALYTIC: recomputed per row and plane inside the step kernel
 * from the closed-form metric in the arithmetic type (FP32 or FP64), by the producer warp's
 * lanes; only single lattices (not ensembles) with FP32 or FP64 storage on the tile kernel
 * (q2 extent a multiple of 64, non-periodic q1) accept it.  AUTO takes the table, the faster of
 * the two on the benchmark lattices (measured: 472 against 966 us per torus step). */
typedef enum { LBW_GEOM_AUTO = 0, LBW_GEOM_TABLE = 1, LBW_GEOM_ANALYTIC = 2 } lbw_geom_mode;

/* A Gaussian pulse P0 = amp exp(-|X - x|^2 / (2 sigma^2)) in the embedding distance. */
typedef struct {
  double x[3];
  double sigma;
  double amp;
} lbw_pulse;

typedef struct lbw_grid lbw_grid; /* opaque, library-owned */

/* Validate desc, build the geometry of the lattice (sqrt g, g^{ab} and the contracted
 * Christoffel symbols G^a = g^{bc} Gamma^a_{bc} of Sec. IV, written in lattice coordinates)
 * and allocate two population buffers on `stream`.  Rejects with LBW_EINVAL: tau != 1/2,
 * non-periodic angular axes, r <= 0 or a non-positive flare anywhere on the lattice or its
 * ghost layer, lattices whose largest c^2 (g^{11} + g^{22} + g^{33}) + 3 cs^2 exceeds
 * 3.0 (the step operator's spectral radius exceeds 1 at 4 in flat space), and geom_mode /
 * equilibrium settings outside the cases their enums list.  *out is set only on success;
 * release it with lbw_destroy. */
lbw_status lbw_create_grid(const lbw_grid_desc* desc, void* stream, lbw_grid** out);

/* Initial state at rest (J' = 0 in the sense of Eq. JShifted): rho0 = sqrt(g) P0 with P0 the
 * sum of the pulses, and post-collision populations f^eq(rho0, F(rho0) / 2).  n_pulses >= 0;
 * host_pulses may be NULL when n_pulses is 0 (zero field).  Resets the step counter and
 * the probe series. */
lbw_status lbw_init(lbw_grid* g, const lbw_pulse* host_pulses, int32_t n_pulses);

/* Advance n_steps >= 0 time steps (one fused stream + collide launch per step, captured in
 * CUDA graphs).  Asynchronous on the grid's stream; registered probes record P after each
 * step's streaming.  Every device wait inside a step is bounded: if one runs out, the kernel
 * raises a flag instead of hanging, and the next call that synchronises (lbw_probe_read,
 * lbw_spectrum, lbw_get_field, lbw_get_populations) returns LBW_ETIMEOUT until lbw_init. */
lbw_status lbw_step(lbw_grid* g, int64_t n_steps);

/* Harmonic sources (Sec. IV: the ring, plate and point sources that drive the pipe, horn
 * and torus): after every subsequent time step t (counted from lbw_init), each of the n
 * source nodes host_q = n x (q1, q2, q3) takes the equilibrium populations that carry
 * amp sin(omega t): kind 0 imposes P = amp sin(omega t) (f = f^eq(sqrt(g) P, 0)), kind 1
 * imposes J'_z (the q3 component of J') = amp sin(omega t) and keeps the node's rho.
 * omega in rad / step.  n = 0 removes the sources.  LBW_EINVAL for nodes outside the lattice
 * or kind not 0 / 1.  Without sources a step is a single kernel launch; with sources a small
 * second launch per step applies them. */
lbw_status lbw_source(lbw_grid* g, const int32_t* host_q, int32_t n, int32_t kind, double amp,
                      double omega);

/* Register n (0 <= n <= 64) probe nodes, host_q = n x (q1, q2, q3), with room for
 * `capacity` samples each (further samples are dropped).  Resets the series. */
lbw_status lbw_probe(lbw_grid* g, const int32_t* host_q, int32_t n, int64_t capacity);

/* Copy the series to host_out (n x cap_per_probe doubles, probe-major); *n_steps receives
 * the number of samples recorded (<= capacity).  LBW_EUNSTABLE if a sample is not finite. */
lbw_status lbw_probe_read(lbw_grid* g, double* host_out, int64_t cap_per_probe,
                          int64_t* n_steps);

/* Mode frequencies of a recorded series (probe >= 0) or of the sum of all series
 * (probe = -1), computed on the device: mean removed, Hann window, zero padding to the
 * smallest power of two >= 4 T, |DFT|^2, the k strongest local maxima above 1e-3 of the
 * largest (sorted by frequency), each refined by a parabola through log-power and 40
 * golden-section steps on the windowed DTFT over +-1 bin.  host_freq / host_amp receive up
 * to k values (rad/step, amplitude 2 |X| / sum w); *n_found how many.  LBW_EUNSTABLE (and no
 * peaks) when the series holds a non-finite value; the same holds for every spectrum call. */
lbw_status lbw_spectrum(lbw_grid* g, int32_t probe, int32_t k, double* host_freq,
                        double* host_amp, int32_t* n_found);

/* As lbw_spectrum, but the k LOWEST-frequency peaks whose power is at least rel_power
 * (0 < rel_power <= 1) of the strongest peak, sorted by frequency: the lowest normal modes
 * (the pipe-versus-horn comparison of Sec. IV.B), which the strongest peaks miss when many
 * modes share the band.  LBW_EINVAL for rel_power outside (0, 1]. */
lbw_status lbw_spectrum_lowest(lbw_grid* g, int32_t probe, int32_t k, double rel_power,
                               double* host_freq, double* host_amp, int32_t* n_found);

/* The same estimator on caller-provided series: host_x = n_series x T doubles. */
lbw_status lbw_spectrum_series(const double* host_x, int64_t T, int32_t n_series, int32_t k,
                               void* stream, double* host_freq, double* host_amp,
                               int32_t* host_n_found);

/* The same estimator for callers that must not allocate device memory -- for example a host
 * application whose own allocator has reserved the device memory, or a latency-critical loop
 * that cannot afford the synchronisation an allocation may cause.  The paper has no
 * counterpart: this is a deployment variant of lbw_spectrum_series.
 *  - dev_x: T doubles in device memory owned by the caller (one series, 4 <= T <= 16384;
 *    larger T is rejected with LBW_EINVAL).  host_freq / host_amp: room for k values;
 *    *host_n_found: how many.  k in [1, 64].
 *  - All workspace lives in one fixed device array of about 2.6 MB inside the library, which
 *    every GPU that loads the library holds until the process exits.  No call here allocates
 *    or frees device memory.
 *  - The array's device address is looked up (cudaGetSymbolAddress) by the first call in each
 *    device context, with that device current, and cached under the context's ID; a context
 *    created after a device reset gets a fresh look-up.
 *  - Every call on a device shares the array and leaves its contents behind; calls whose work
 *    overlaps on the GPU (different streams, no ordering between them) race, so callers must
 *    serialise them.  The call synchronises `stream` and copies its results to host memory
 *    before returning, so it cannot be made while `stream` is being captured into a graph. */
lbw_status lbw_spectrum_series_static(const double* dev_x, int64_t T, int32_t k, void* stream,
                                      double* host_freq, double* host_amp, int32_t* host_n_found);

/* P = rho / sqrt(g) of the current state (rho = sum of the stored post-collision
 * populations; the relaxation conserves it), N doubles in the layout above.  The field is
 * copied in every case; LBW_EUNSTABLE if any of its values is not finite. */
lbw_status lbw_get_field(lbw_grid* g, double* host_P);

/* Checkpoint / resume: the seven population planes as doubles (7 x N, same layout). */
lbw_status lbw_get_populations(lbw_grid* g, double* host_f);
lbw_status lbw_set_populations(lbw_grid* g, const double* host_f);

/* Number of time steps advanced since lbw_init. */
lbw_status lbw_step_count(lbw_grid* g, int64_t* out);

/* Failure injection for tests of the timeout path; the paper has no counterpart.  From the
 * next time step on, the step kernel's consumer warps wait on a barrier that no copy ever
 * completes.  The bounded wait runs out after a few hundred tries (under a millisecond), the
 * step raises its timeout flag, and every CTA leaves once the copies it issued have landed,
 * exactly as after a lost copy, with no device fault and no hang.  Calls that synchronise
 * then return LBW_ETIMEOUT; lbw_init clears the request and the flag.  LBW_ESTATE before
 * lbw_init; LBW_EINVAL on lattices that run the register-pipelined kernel (q2 extent not a
 * multiple of the tile width, or periodic q1), which has no device waits. */
lbw_status lbw_inject_wait_timeout(lbw_grid* g);

/* Frees the grid's device memory (stream-ordered) and graphs; NULL is allowed. */
void lbw_destroy(lbw_grid* g);

/* ------------------------------------------------------------------------------------------
 * Ensembles: many independent lattices of uneven sizes (each a full instance of the scheme
 * above with its own geometry and probes) advanced together.  One time step of the whole
 * ensemble is one launch of a persistent kernel over a (member, tile, q3 segment) work list;
 * steps are captured in CUDA graphs.  A member's results agree with the same lattice run
 * alone to the rounding of its storage (the kernels may sum in another order).
 * ---------------------------------------------------------------------------------------- */
typedef struct lbw_batch lbw_batch; /* opaque, library-owned */

/* n members (1..65536), all with the same prec; each descriptor is validated as in
 * lbw_create_grid.  Populations start at zero.  The initial launch shape is full-row tiles
 * with 16-plane segments where every member fits one (see lbw_batch_tune), else 7-row tiles
 * of 64 columns, else the register-pipelined kernel's default. */
lbw_status lbw_batch_create(const lbw_grid_desc* descs, int32_t n, void* stream, lbw_batch** out);

/* Initial state at rest for every member: host_counts[m] pulses for member m, taken in order
 * from host_pulses (the members' pulse lists concatenated). */
lbw_status lbw_batch_init(lbw_batch* b, const lbw_pulse* host_pulses, const int32_t* host_counts);

/* per_member probes for every member: host_q = n x per_member x (q1, q2, q3); capacity
 * samples each.  Resets the series. */
lbw_status lbw_batch_probe(lbw_batch* b, const int32_t* host_q, int32_t per_member, int64_t capacity);

/* Advance every member by n_steps (asynchronous on the ensemble's stream). */
lbw_status lbw_batch_step(lbw_batch* b, int64_t n_steps);

/* Harmonic sources for every member (see lbw_source): per_member nodes each, host_q =
 * n x per_member x (q1, q2, q3) in the members' own lattices, one angular frequency per member
 * (host_omega[n], rad / step), a common kind and amplitude.  A frequency sweep is one ensemble
 * of identical geometries with different omegas.  per_member = 0 removes the sources. */
lbw_status lbw_batch_source(lbw_batch* b, const int32_t* host_q, int32_t per_member, int32_t kind,
                            double amp, const double* host_omega);

/* All series: host_out = n x per_member x capacity doubles; *n_steps = samples recorded. */
lbw_status lbw_batch_probe_read(lbw_batch* b, double* host_out, int64_t* n_steps);

/* The steady-state response of the resonance sweeps (Sec. IV.A, Fig. Frequencies; Sec. IV.C,
 * Fig. FreqTorus: the pressure intensity at a probe after a transient): for every member and
 * probe the largest |P| over its last `tail` recorded samples, reduced on the device.
 * host_out = n x per_member doubles.  LBW_EINVAL if tail exceeds the recorded samples,
 * LBW_EUNSTABLE if a sample in the window is not finite. */
lbw_status lbw_batch_probe_peak(lbw_batch* b, int64_t tail, double* host_out);

/* Per member, the spectrum of the sum of its probes (the estimator of lbw_spectrum):
 * host_freq / host_amp = n x k, host_n_found = n. */
lbw_status lbw_batch_spectrum(lbw_batch* b, int32_t k, double* host_freq, double* host_amp,
                              int32_t* host_n_found);

/* As lbw_batch_spectrum, but the k LOWEST-frequency peaks of each member's summed series
 * whose power is at least rel_power (0 < rel_power <= 1) of that member's strongest peak,
 * sorted by frequency: the lowest modes of a large lattice, which its strongest peaks miss
 * when hundreds of modes share the band. */
lbw_status lbw_batch_spectrum_lowest(lbw_batch* b, int32_t k, double rel_power, double* host_freq,
                                     double* host_amp, int32_t* host_n_found);

/* Member's populations as doubles (7 x N of that member). */
lbw_status lbw_batch_get_populations(lbw_batch* b, int32_t member, double* host_f);

/* Autotuner: times candidate launch shapes for trial_steps steps each and keeps the fastest.
 * Ensembles whose members all wrap in q2 and have walls in q1 run the TMA-staged kernel
 * (tile rows 4 or 7 of 64 columns, or 0: full-row tiles, each member's whole rows with a
 * height that follows its row length, offered when every member fits one and the storage
 * is 32- or 64-bit; CTAs per SM 1/2); others the register-pipelined kernel (rows 4/8/16,
 * CTAs per SM 1/2/4); planes per q3 segment 16/32/64 for both.  With a cache_path (JSON
 * lines), a shape stored for the same ensemble signature is reused without timing and a new
 * choice is appended.  The trial steps run on the ensemble's buffers: call it before
 * lbw_batch_init.  A text report of the timings goes to report (may be NULL). */
lbw_status lbw_batch_tune(lbw_batch* b, int32_t trial_steps, const char* cache_path, char* report,
                          int32_t report_cap);

/* Sets the launch shape instead of the autotuner: tile_rows (one of the values the autotuner
 * offers this ensemble, see lbw_batch_tune), seg_planes >= 1, ctas_per_sm >= 1 and at most
 * what the kernel can keep resident.  LBW_EINVAL for a shape this ensemble cannot run.  The
 * populations are kept; the step kernels differ only in how they stage them (every shape
 * gives the same numbers). */
lbw_status lbw_batch_set_shape(lbw_batch* b, int32_t tile_rows, int32_t seg_planes, int32_t ctas_per_sm);

/* Total nodes and the launch shape in use (any pointer may be NULL). */
lbw_status lbw_batch_info(lbw_batch* b, int64_t* total_nodes, int32_t* tile_rows, int32_t* seg_planes,
                          int32_t* ctas_per_sm);

void lbw_batch_destroy(lbw_batch* b);

/* ------------------------------------------------------------------------------------------
 * Surrogate: a multilayer perceptron from ensemble geometry parameters to mode frequencies,
 * trained and evaluated on the device (the paper has no counterpart; the lattice-Boltzmann
 * runs stay the reference for its error).  depth weight layers in -> hidden -> ... -> out, tanh
 * after every layer but the last.  Loss: mean over samples and outputs of (y - t)^2.
 * Parameters: one FP32 vector, per layer W (out x in, row-major) then b (out).  Host arrays
 * are row-major float32 (n x in inputs, n x out targets).
 * ---------------------------------------------------------------------------------------- */
typedef struct lbw_mlp lbw_mlp; /* opaque, library-owned */

/* Glorot-uniform weights from a counter-based generator seeded by `seed`, zero biases. */
lbw_status lbw_mlp_create(int32_t in_dim, int32_t hidden, int32_t depth, int32_t out_dim, uint64_t seed,
                          void* stream, lbw_mlp** out);
lbw_status lbw_mlp_param_count(lbw_mlp* q, int64_t* n);
lbw_status lbw_mlp_get_params(lbw_mlp* q, float* host_params);
/* Also resets the Adam moments. */
lbw_status lbw_mlp_set_params(lbw_mlp* q, const float* host_params);
/* FP32 forward pass of n rows. */
lbw_status lbw_mlp_forward(lbw_mlp* q, const float* host_x, int32_t n, float* host_y);
/* Forward pass with the weights rounded to BF16 (biases and accumulation FP32). */
lbw_status lbw_mlp_predict_bf16(lbw_mlp* q, const float* host_x, int32_t n, float* host_y);
/* Loss and its gradient with respect to all parameters for one batch of n rows
 * (host_grad may be NULL). */
lbw_status lbw_mlp_grad(lbw_mlp* q, const float* host_x, const float* host_t, int32_t n, float* host_grad,
                        float* host_loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with a caller gradient. */
lbw_status lbw_mlp_adam_step(lbw_mlp* q, const float* host_grad, float lr);
/* n_steps Adam steps on minibatches of `batch` rows of the n samples: step s uses rows
 * host_order[s * batch .. s * batch + batch - 1] (the caller draws the order).  host_loss
 * (may be NULL) receives the minibatch loss before each step. */
lbw_status lbw_mlp_train(lbw_mlp* q, const float* host_x, const float* host_t, int32_t n,
                         const int32_t* host_order, int32_t n_steps, int32_t batch, float lr, float* host_loss);
void lbw_mlp_destroy(lbw_mlp* q);

/* Message of the last failure on the calling thread ("" if none). */
const char* lbw_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBW_H */

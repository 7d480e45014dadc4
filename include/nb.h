/*
 * nb.h -- C ABI of libnb: the GB300 (sm_103a) hot path of a Hermite
 * 6th-order direct N-body integrator with block time steps.
 *
 * The paper (Goz et al., "Astrophysical code migration into Exascale Era")
 * states the problem this library computes:
 *   - Sec. 2: a direct N-body code built on a 6th-order Hermite integrator
 *     and descended from HiGPUs; double precision is needed for the
 *     inter-particle distance and the acceleration; an extended-precision
 *     ("EX") number type built from pairs of single-precision numbers is the
 *     alternative on devices with weak double precision.
 *   - Sec. 4: the hot kernel is the O(N^2) evaluation over all particle pairs.
 * The paper prints no formulas; the steps follow the published 6th-order
 * Hermite scheme (Nitadori & Makino 2008) and power-of-two block time steps
 * (Makino 1991, Aarseth 2003).  Units: G = 1.
 *
 * Conventions for every call:
 *   - Every pointer named "device" is CUDA device memory of the GPU that was
 *     current at nb_init; "host" is ordinary (preferably pinned) host memory.
 *   - Vector fields are SoA, layout [3][n]: component d of particle i is at
 *     p[d * n + i].  Scalars are [n].  All floating point is IEEE double at
 *     the boundary, whatever the internal precision.
 *   - Calls never abort or exit; they return an nb_status.  NB_ECUDA carries
 *     the CUDA error text in nb_last_error().
 *   - Work is enqueued on the stream given to nb_init; calls that return
 *     host values synchronise that stream.  A context is not thread-safe;
 *     distinct contexts are independent.
 */
#ifndef NB_H
#define NB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nb_ctx nb_ctx; /* opaque, owned by libnb, freed by nb_free */

typedef enum {
    NB_OK = 0,
    NB_EINVAL = 1,       /* bad argument (sizes, pointers, parameters) */
    NB_ENOMEM = 2,       /* device or host allocation failed */
    NB_ECUDA = 3,        /* a CUDA call failed; see nb_last_error */
    NB_ENONFINITE = 4,   /* a non-finite value appeared in the state */
    NB_EDTUNDERFLOW = 5, /* reserved: the criterion asked for dt < dt_min
                            (counted, the step is clamped to dt_min) */
    NB_ETIMEOUT = 6,     /* a bounded device-side wait ran out */
    NB_ESTATE = 7        /* call not valid in the context's current state */
} nb_status;

/* Arithmetic of the pairwise evaluation (paper Sec. 2: DP, or EX pairs of
 * single-precision numbers).  Particle state, prediction, correction and
 * time steps are FP64 for every choice. */
typedef enum {
    NB_FP64 = 0, /* double precision throughout */
    NB_EX = 1,   /* float-float (hi + lo single-precision pair) arithmetic */
    NB_FP32 = 2, /* relative coordinates from split hi/lo singles, FP32 force
                    math, FP32 sums over j-chunks promoted to FP64 */
    NB_FP32X = 3 /* acceleration and potential in float-float (as NB_EX), jerk
                    and snap in FP32 (as NB_FP32): the 6th-order step
                    criterion needs the acceleration to about 1e-8, jerk and
                    snap only to about 1e-5 */
} nb_precision;

/* nb_params.flags */
#define NB_INIT_KEEP_STATE 1u /* nb_init: keep a, j, s, c, t, dt, pot as given
                                 (resume); skip the start-up evaluations */
#define NB_TIME_EVAL 2u       /* record CUDA events around every evaluation
                                 launch of nb_step / nb_run (nb_counters.eval_ms) */
#define NB_NO_STREAMK 4u      /* split one-cluster evaluations into j-range items
                                 as in a batch instead of equal stream-K ranges
                                 per CTA: a cluster's results are then
                                 bit-identical alone and in a batch that uses
                                 the same plan table */

typedef struct {
    double eps;      /* Plummer softening length; pairs use |r|^2 + eps^2 */
    double eta;      /* 6th-order time-step coefficient (e.g. 0.4) */
    double eta_init; /* start-up coefficient: dt0 = eta_init *
                        min(|a|/|j|, sqrt(|a|/|s|)) (e.g. 0.01) */
    double dt_min;   /* smallest block step, a power of two (e.g. 2^-20) */
    double dt_max;   /* largest block step, a power of two (e.g. 2^-3);
                        dt_min == dt_max gives shared steps */
    int32_t precision; /* nb_precision */
    uint32_t flags;    /* NB_INIT_* */
    int32_t order;     /* integration order: 6 (0 means 6) = the NM08 6th-order
                          scheme above; 4 = the 4th-order Hermite scheme of
                          Makino & Aarseth 1992 (predictor through jerk,
                          a and jerk evaluated, s = 0 in nb_evaluate's
                          output, Aarseth's criterion
                          dt = sqrt(eta (|a||a2| + |j|^2) / (|j||a3| + |a2|^2))
                          on the cubic-interpolated a2, a3 kept in s and c;
                          one start-up pass, dt0 = eta_init |a|/|j|);
                          any other value: NB_EINVAL */
    int32_t reserved;  /* must be 0 */
} nb_params;

/* Particle state: caller-owned DEVICE buffers that must stay alive for the
 * context's lifetime.  m, t, dt, pot: [n]; x, v, a, j, s, c: [3][n].
 * a = acceleration, j = jerk, s = snap, c = crackle (third derivative),
 * t = particle time, dt = its power-of-two step, pot = potential. */
typedef struct {
    double *m;
    double *x, *v, *a, *j, *s, *c;
    double *t, *dt, *pot;
} nb_state;

/* Counters accumulated since nb_init (read with nb_get_counters). */
typedef struct {
    int64_t block_steps;     /* block steps taken (per cluster, summed) */
    double interactions;     /* sum over steps of n_active * (n_cluster - 1) */
    int64_t dt_underflows;   /* criterion asked for dt < dt_min (clamped) */
    uint32_t device_errors;  /* device error word (0 when healthy) */
    int64_t kernel_launches; /* kernels launched by nb_step / nb_run */
    int64_t eval_launches;   /* evaluation launches timed (NB_TIME_EVAL) */
    double eval_ms;          /* their summed device time (CUDA events) */
} nb_counters;

/*
 * nb_init -- create a context over the caller's state and run the start-up
 * (Hermite-6 needs snap, which needs the other particles' accelerations:
 * pass 1 evaluates a and jerk with a = 0, pass 2 evaluates snap with that a;
 * crackle starts at 0; t = 0; dt from the start-up rule, a power of two in
 * [dt_min, dt_max]).  With order 4 only pass 1 runs (s = c = 0).  With
 * NB_INIT_KEEP_STATE the state is taken as is.
 *
 *   out             : receives the new context (NULL on failure)
 *   p               : parameters (copied)
 *   n               : number of particles (>= 1)
 *   st              : device state buffers (see nb_state); m, x, v are read,
 *                     the others written (unless NB_INIT_KEEP_STATE)
 *   n_clusters      : >= 1; clusters are independent systems (no cross
 *                     forces), each with its own block-step schedule
 *   cluster_offsets : HOST array of n_clusters + 1 increasing int64 with
 *                     offsets[0] = 0, offsets[n_clusters] = n; NULL means one
 *                     cluster
 *   stream          : cudaStream_t to enqueue on (NULL = legacy default)
 * Errors: NB_EINVAL (n < 1, bad offsets, eps < 0, eta <= 0, dt_min/dt_max
 * not powers of two or dt_min > dt_max, unknown precision or order,
 * reserved != 0), NB_ENOMEM,
 * NB_ECUDA.  Allocates the library's scratch (predicted j-arrays, active
 * lists, partial sums, graphs); nb_free releases it.
 */
nb_status nb_init(nb_ctx **out, const nb_params *p, int64_t n, const nb_state *st,
                  int32_t n_clusters, const int64_t *cluster_offsets, void *stream);

/*
 * nb_predict -- Taylor-extrapolate every particle from its own time t_i to
 * t_next through crackle (NM08 predictor; the paper's Sec. 2 integrator):
 *   x_p = x + v d + a d^2/2 + j d^3/6 + s d^4/24 + c d^5/120, d = t_next - t_i
 *   v_p = v + a d + j d^2/2 + s d^3/6 + c d^4/24
 *   a_p = a + j d + s d^2/2 + c d^3/6
 * into the context's packed j-array (in the context's precision), which the
 * next nb_evaluate reads.  out: optional DEVICE [10][n] double receiving
 * x_p[3], v_p[3], a_p[3], m (NULL to skip).  With order 4 the series stops
 * at the jerk term (s and c are then the criterion's interpolated
 * derivatives, not predictor terms).  Errors: NB_EINVAL, NB_ECUDA.
 */
nb_status nb_predict(nb_ctx *ctx, double t_next, double *out);

/*
 * nb_evaluate -- the paper's hot O(N_active x N) kernel (Sec. 4): for each
 * listed active particle i of cluster `cluster`, sum over every other j of
 * that cluster, on the state of the last nb_predict (r = x_j - x_i,
 * v = v_j - v_i, a = a_j - a_i, s2 = r.r + eps^2, alpha = r.v/s2,
 * beta = (v.v + r.a)/s2 + alpha^2):
 *   acc  += m_j r / s2^{3/2}                         (A0)
 *   jerk += m_j v / s2^{3/2} - 3 alpha A0            (A1)
 *   snap += m_j a / s2^{3/2} - 6 alpha A1 - 3 beta A0 (A2)
 *   pot  -= m_j / s2^{1/2}
 * With order 4 only A0, A1 and pot are summed (a is not read; snap = 0).
 * j == i is excluded by index.  The j range may be split across thread
 * blocks; partial sums are combined in a fixed order (deterministic).
 *   active  : DEVICE int32 [n_active], global particle indices inside the
 *             cluster's range (duplicates allowed)
 *   out_ajs : DEVICE double [10][n_active]: acc[3], jerk[3], snap[3], pot
 * Errors: NB_EINVAL (cluster out of range, n_active < 0 or > cluster size,
 * NULL pointers with n_active > 0), NB_ECUDA.  n_active == 0 is a no-op.
 */
nb_status nb_evaluate(nb_ctx *ctx, int32_t cluster, const int32_t *active, int32_t n_active,
                      double *out_ajs);

/*
 * nb_evaluate_range -- the sums of nb_evaluate restricted to the j-particles
 * [j_begin, j_end) of cluster `cluster` (indices relative to the cluster's
 * first particle): the contribution of one part of the j-set.  The paper's
 * code distributes the O(N^2) evaluation over processes (Sec. 2, MPI +
 * OpenMP; HiGPUs splits j across GPUs); summed over a partition of
 * [0, n_cluster) these partial sums give nb_evaluate's result up to the
 * order of the additions.  j == i is still excluded by index.
 *   active   : DEVICE int32 [n_active] as for nb_evaluate
 *   j_begin  : a multiple of 64 (the j-tile size), 0 <= j_begin <= j_end
 *   j_end    : a multiple of 64, or n_cluster; j_end <= n_cluster
 *   out_ajs  : DEVICE double [10][n_active]: partial acc, jerk, snap, pot
 *              (all 0 for an empty range)
 * Errors: NB_EINVAL (cluster, sizes, range not tile-aligned, NULL pointers
 * with n_active > 0), NB_ECUDA.  n_active == 0 is a no-op.
 */
nb_status nb_evaluate_range(nb_ctx *ctx, int32_t cluster, const int32_t *active, int32_t n_active,
                            int64_t j_begin, int64_t j_end, double *out_ajs);

/*
 * nb_correct_and_timestep -- NM08 6th-order corrector for the listed
 * particles from their times t_i to t_next (h = t_next - t_i):
 *   v1 = v0 + h/2 (a1 + a0) - h^2/10 (j1 - j0) + h^3/120 (s1 + s0)
 *   x1 = x0 + h/2 (v1 + v0) - h^2/10 (a1 - a0) + h^3/120 (j1 + j0)
 * then the 3rd-5th derivatives at t_next from the quintic matching (a, j, s)
 * at both ends, the new step dt = eta (A(1)/A(4))^{1/3},
 * A(k) = sqrt(|a^(k-1)| |a^(k+1)|) + |a^(k)|, quantised to a power of two
 * (shrink freely; double at most once and only when t_next is a multiple of
 * 2 dt; clamp to [dt_min, dt_max]), and t_i = t_next, c = a^(3)(t_next).
 *   active : DEVICE int32 [n_active] (no duplicates), in cluster `cluster`
 *   ajs    : DEVICE double [10][n_active] as written by nb_evaluate
 * With order 4: the Makino & Aarseth corrector
 *   v1 = v0 + h/2 (a0 + a1) + h^2/12 (j0 - j1)
 *   x1 = x0 + h/2 (v0 + v1) + h^2/12 (a0 - a1),
 * the 2nd and 3rd derivatives at t_next of the cubic matching (a, j) at
 * both ends (stored in s and c), and Aarseth's criterion (see nb_params),
 * with the same quantisation.
 * Errors: NB_EINVAL, NB_ECUDA.  Non-finite results set the device error word.
 */
nb_status nb_correct_and_timestep(nb_ctx *ctx, int32_t cluster, const int32_t *active,
                                  int32_t n_active, double t_next, const double *ajs);

/*
 * nb_step -- one block step of every cluster, on the device without host
 * round trips (replayed from a CUDA graph): t_next_c = min_i (t_i + dt_i),
 * active = {i : t_i + dt_i == t_next_c}, predict, evaluate, correct.
 *   t_next_out   : HOST, optional: smallest t_next over clusters
 *   n_active_out : HOST, optional: active particles summed over clusters
 * Passing either output synchronises the stream.  Errors: NB_ECUDA,
 * NB_ENONFINITE / NB_ETIMEOUT from the device error word (when synchronised).
 */
nb_status nb_step(nb_ctx *ctx, double *t_next_out, int32_t *n_active_out);

/*
 * nb_run -- block steps until no cluster has a block time <= t_end (each
 * cluster stops on its own), or until max_block_steps steps of the whole
 * batch (< 0: no limit).  Synchronises.  block_steps_out / interactions_out
 * (HOST, optional) receive this call's block steps (per cluster, summed) and
 * its sum of n_active * (n_cluster - 1).
 */
nb_status nb_run(nb_ctx *ctx, double t_end, int64_t max_block_steps, int64_t *block_steps_out,
                 double *interactions_out);

/*
 * nb_energy -- diagnostics at common time t for cluster `cluster` (-1: all,
 * summed): every particle predicted to t, the FP64 potential re-evaluated on
 * the predicted positions, E_kin = 1/2 sum m v^2, E_pot = 1/2 sum m pot,
 * P = sum m v, L = sum m x cross v.  Outputs are HOST.  Synchronises.
 */
nb_status nb_energy(nb_ctx *ctx, int32_t cluster, double t, double *ekin, double *epot,
                    double P[3], double L[3]);

/*
 * nb_energy_all -- the diagnostics of nb_energy for every cluster at once
 * (one potential evaluation of the whole batch at common time t).
 *   out : HOST double [n_clusters][8]: E_kin, E_pot, P[3], L[3] per cluster
 * Synchronises.  Errors: NB_EINVAL, NB_ECUDA.
 */
nb_status nb_energy_all(nb_ctx *ctx, double t, double *out);

/* nb_get_state / nb_set_state -- copy the whole particle state out of / into
 * the context's buffers.  dst / src pointers may be HOST or DEVICE (any mix).
 * Synchronises.  Used for checkpoint / resume and host-side I/O. */
nb_status nb_get_state(nb_ctx *ctx, const nb_state *dst);
nb_status nb_set_state(nb_ctx *ctx, const nb_state *src);

/* nb_get_counters -- counters since nb_init (HOST out).  Synchronises. */
nb_status nb_get_counters(nb_ctx *ctx, nb_counters *out);

/*
 * nb_autotune -- time the evaluation kernel for active-set sizes 1, 2, 4,
 * ... up to the largest cluster, over candidate (lanes per i, j-split)
 * choices, and install the fastest per size bucket.  cache_path: optional
 * file to read a previous table from / write the new one to (NULL: none).
 * The state is not modified.  Errors: NB_ECUDA, NB_EINVAL.
 */
nb_status nb_autotune(nb_ctx *ctx, const char *cache_path);

/*
 * nb_evaluate_noalloc -- the FP64 evaluation of nb_evaluate for callers that
 * cannot allocate device memory.  The paper has no counterpart.  Some callers
 * cannot call cudaMalloc: code embedded in a framework whose memory pool
 * already holds the device memory (a native allocation fails, or escapes the
 * framework's accounting), and latency-critical loops that must not allocate
 * (cudaMalloc can synchronise the whole device).  nb_init allocates scratch,
 * so those callers cannot use nb_evaluate.
 * This entry needs no context and allocates nothing: its working space (packed j
 * tiles, split partial sums, tile counters; about 5.8 MB) is a fixed array
 * compiled into the library, which every GPU that loads libnb keeps until the
 * process exits.
 *   jpred    : DEVICE double [10][n]: x[3], v[3], a[3], m of every particle
 *              (the layout nb_predict writes to its `out`)
 *   n        : 1 <= n <= 32768 (larger: NB_EINVAL)
 *   eps      : softening length (>= 0)
 *   active   : DEVICE int32 [n_active], indices in [0, n); 0 <= n_active <=
 *              32768; duplicates allowed
 *   out      : DEVICE double [10][n_active]: acc[3], jerk[3], snap[3], pot
 *              (the 6th-order pair terms; a 4th-order caller ignores snap)
 *   stream   : cudaStream_t (NULL = legacy default); the call synchronises it
 *              to read its error word
 * The first call on a device looks up the array's device address with that
 * device current.  Every call copies its error word to the host and synchronises `stream` before
 * it returns.  All calls share the array: calls that overlap on the GPU
 * (other streams, threads or processes sharing the library) race and must
 * be serialised by the caller.  Errors: NB_EINVAL (sizes, NULL pointers, an
 * index outside [0, n): that entry is skipped, its ten outputs are 0, the
 * other entries are evaluated and the call reports the bad index), NB_ECUDA
 * (also for a CUDA error already pending when the call starts), NB_ETIMEOUT;
 * messages through nb_last_error(NULL).
 */
nb_status nb_evaluate_noalloc(const double *jpred, int64_t n, double eps, const int32_t *active,
                              int32_t n_active, double *out, void *stream);

/* nb_sync -- wait for the context's stream and check the device error word. */
nb_status nb_sync(nb_ctx *ctx);

/* Message of the last failing call on this context (never NULL). */
const char *nb_last_error(const nb_ctx *ctx);

/* Name of a status code. */
const char *nb_status_string(nb_status s);

/* Release the context and its scratch (not the caller's state buffers). */
void nb_free(nb_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* NB_H */

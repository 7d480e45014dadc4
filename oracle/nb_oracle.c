/*
 * nb_oracle.c -- plain, slow, FP64 CPU oracle for the Hermite 6th-order direct
 * N-body method with block time steps.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * leg load it.  It shares no code, header, table or helper with the CUDA
 * library; the only thing both sides consume is the seeded initial-condition
 * generator (paper_1812_00367_gb300/ic.py), which holds none of the method.
 *
 * What the paper fixes and what comes from the method it builds on:
 *   - Sec. 2: the code integrates with a 6th-order Hermite scheme and descends
 *     from HiGPUs; distance and acceleration need double precision.
 *   - Sec. 4: the O(N^2) kernel (acceleration, jerk, snap of every active
 *     particle against all others) is where the run spends its time.
 *   - The paper prints no formulas.  The evaluation, predictor, corrector,
 *     quintic interpolation and time-step criterion below follow the published
 *     6th-order Hermite scheme of Nitadori & Makino 2008 (New Astron. 13, 498;
 *     "NM08" below); block (power-of-two) time steps follow Makino 1991 /
 *     Aarseth 2003.  Every reading where the paper is silent is listed in the
 *     repository's design notes and repeated at the function that takes it.
 *
 * Layout (deliberately the natural one, not the GPU one): vectors are [n][3]
 * row-major doubles, scalars [n].  Everything is IEEE double, compiled with
 * -ffp-contract=off so results do not depend on the host's FMA contraction.
 *
 * Pins (tests/test_oracle_*.py): degree-2 Taylor-jet arithmetic of the exact
 * force along polynomial trajectories, two-body closed form, Newton's third
 * law, permutation invariance, exactness of predictor / corrector /
 * interpolation on polynomials, a 6x6 Hermite solve, the Kepler problem in
 * closed form with measured convergence order ~6, the criterion on
 * exponential derivative ladders, scheduler brute force, energy conservation.
 * The 4th-order variant (Makino & Aarseth 1992; tests/test_oracle_hermite4.py):
 * exactness of its predictor / corrector / cubic interpolation on
 * polynomials, Aarseth's criterion on exponential ladders and under time
 * rescaling, Kepler convergence order ~4, energy and momentum.  Every function
 * here has a pin; none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Evaluation (NM08; the paper's Sec. 4 O(N^2) kernel)                        */
/* ------------------------------------------------------------------------- */

/*
 * For each listed active particle i, sum over all j != i (excluded by index,
 * so eps = 0 is valid) the softened Newtonian pair terms, in NM08's notation:
 *   r = x_j - x_i, v = v_j - v_i, a = a_j - a_i        (predicted values)
 *   s2 = r.r + eps^2
 *   A0 = m_j r / s2^{3/2}
 *   alpha = (r.v)/s2
 *   beta  = (v.v + r.a)/s2 + alpha^2
 *   A1 = m_j v / s2^{3/2} - 3 alpha A0
 *   A2 = m_j a / s2^{3/2} - 6 alpha A1 - 3 beta A0
 *   pot = - sum m_j / s2^{1/2}
 * acc += A0, jrk += A1, snp += A2.  j runs in increasing index order for every
 * i, so the result does not depend on the number of threads.
 */
void orc_force(int64_t n, const double *m, const double *xp, const double *vp,
               const double *ap, double eps2, int64_t n_act, const int64_t *act,
               double *acc, double *jrk, double *snp, double *pot)
{
    int64_t k;
#pragma omp parallel for schedule(dynamic, 4)
    for (k = 0; k < n_act; k++) {
        const int64_t i = act[k];
        double A[3] = {0, 0, 0}, J[3] = {0, 0, 0}, S[3] = {0, 0, 0}, P = 0.0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double r[3], v[3], a[3];
            for (int d = 0; d < 3; d++) {
                r[d] = xp[3 * j + d] - xp[3 * i + d];
                v[d] = vp[3 * j + d] - vp[3 * i + d];
                a[d] = ap[3 * j + d] - ap[3 * i + d];
            }
            double s2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + eps2;
            double rinv = 1.0 / sqrt(s2);
            double rinv2 = rinv * rinv;
            double mr3 = m[j] * rinv * rinv2;
            double alpha = (r[0] * v[0] + r[1] * v[1] + r[2] * v[2]) * rinv2;
            double beta = (v[0] * v[0] + v[1] * v[1] + v[2] * v[2] +
                           r[0] * a[0] + r[1] * a[1] + r[2] * a[2]) * rinv2 +
                          alpha * alpha;
            double A0[3], A1[3], A2[3];
            for (int d = 0; d < 3; d++) {
                A0[d] = mr3 * r[d];
                A1[d] = mr3 * v[d] - 3.0 * alpha * A0[d];
                A2[d] = mr3 * a[d] - 6.0 * alpha * A1[d] - 3.0 * beta * A0[d];
                A[d] += A0[d];
                J[d] += A1[d];
                S[d] += A2[d];
            }
            P -= m[j] * rinv;
        }
        for (int d = 0; d < 3; d++) {
            acc[3 * k + d] = A[d];
            jrk[3 * k + d] = J[d];
            snp[3 * k + d] = S[d];
        }
        pot[k] = P;
    }
}

/* ------------------------------------------------------------------------- */
/* Predictor (NM08): Taylor series through crackle                            */
/* ------------------------------------------------------------------------- */

/*
 * Each particle is extrapolated from its own time t[i] to t_next with
 * dt = t_next - t[i]:
 *   xp = x + v dt + a dt^2/2 + j dt^3/6 + s dt^4/24 + c dt^5/120
 *   vp = v + a dt + j dt^2/2 + s dt^3/6 + c dt^4/24
 *   ap = a + j dt + s dt^2/2 + c dt^3/6
 * (Reading: the paper gives no predictor; NM08's 6th-order scheme predicts
 * with the derivatives it stores, through crackle c.)
 */
void orc_predict(int64_t n, const double *x, const double *v, const double *a,
                 const double *j, const double *s, const double *c,
                 const double *t, double t_next, double *xp, double *vp,
                 double *ap)
{
    for (int64_t i = 0; i < n; i++) {
        double dt = t_next - t[i];
        double d2 = dt * dt / 2.0, d3 = dt * dt * dt / 6.0;
        double d4 = dt * dt * dt * dt / 24.0, d5 = dt * dt * dt * dt * dt / 120.0;
        for (int d = 0; d < 3; d++) {
            const int64_t o = 3 * i + d;
            xp[o] = x[o] + v[o] * dt + a[o] * d2 + j[o] * d3 + s[o] * d4 + c[o] * d5;
            vp[o] = v[o] + a[o] * dt + j[o] * d2 + s[o] * d3 + c[o] * d4;
            ap[o] = a[o] + j[o] * dt + s[o] * d2 + c[o] * d3;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Quintic Hermite interpolation and corrector (NM08)                        */
/* ------------------------------------------------------------------------- */

/*
 * a(t) on [t0, t1], h = t1 - t0, is taken as the unique quintic matching
 * (a, j, s) at both ends.  Written around the midpoint, tau in [-T, T],
 * T = h/2, p(tau) = sum_k c_k tau^k; with a+- = (a1 +- a0)/2 (likewise j, s)
 * the even and odd parts decouple:
 *   even:  c0 + c2 T^2 + c4 T^4 = a+,  2 c2 T + 4 c4 T^3 = j-,  2 c2 + 12 c4 T^2 = s+
 *   odd:   c1 T + c3 T^3 + c5 T^5 = a-,  c1 + 3 c3 T^2 + 5 c5 T^4 = j+,
 *          6 c3 T + 20 c5 T^3 = s-
 * and the 3rd, 4th and 5th derivatives at t1 (tau = T) follow.  A test checks
 * this against a direct 6x6 solve and exact recovery of a known quintic.
 */
void orc_interp_derivs(double h, const double a0[3], const double j0[3],
                       const double s0[3], const double a1[3], const double j1[3],
                       const double s1[3], double d3[3], double d4[3], double d5[3])
{
    const double T = 0.5 * h;
    for (int d = 0; d < 3; d++) {
        double am = 0.5 * (a1[d] - a0[d]);
        double jp = 0.5 * (j1[d] + j0[d]), jm = 0.5 * (j1[d] - j0[d]);
        double sp = 0.5 * (s1[d] + s0[d]), sm = 0.5 * (s1[d] - s0[d]);
        /* even part: c4 then c2 */
        double c4 = (sp * T - jm) / (8.0 * T * T * T);
        /* odd part: c5 then c3 */
        double c5 = (sm * T * T - 3.0 * jp * T + 3.0 * am) / (8.0 * T * T * T * T * T);
        double c3 = (sm - 20.0 * c5 * T * T * T) / (6.0 * T);
        d3[d] = 6.0 * c3 + 24.0 * c4 * T + 60.0 * c5 * T * T;
        d4[d] = 24.0 * c4 + 120.0 * c5 * T;
        d5[d] = 120.0 * c5;
    }
}

/*
 * NM08 6th-order corrector, h = t1 - t0:
 *   v1 = v0 + h/2 (a1 + a0) - h^2/10 (j1 - j0) + h^3/120 (s1 + s0)
 *   x1 = x0 + h/2 (v1 + v0) - h^2/10 (a1 - a0) + h^3/120 (j1 + j0)
 */
void orc_correct(double h, const double x0[3], const double v0[3],
                 const double a0[3], const double j0[3], const double s0[3],
                 const double a1[3], const double j1[3], const double s1[3],
                 double x1[3], double v1[3])
{
    for (int d = 0; d < 3; d++) {
        v1[d] = v0[d] + h / 2.0 * (a1[d] + a0[d]) - h * h / 10.0 * (j1[d] - j0[d]) +
                h * h * h / 120.0 * (s1[d] + s0[d]);
        x1[d] = x0[d] + h / 2.0 * (v1[d] + v0[d]) - h * h / 10.0 * (a1[d] - a0[d]) +
                h * h * h / 120.0 * (j1[d] + j0[d]);
    }
}

/* ------------------------------------------------------------------------- */
/* Time steps                                                                 */
/* ------------------------------------------------------------------------- */

static double norm3(const double *q) { return sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]); }

/*
 * NM08's generalised Aarseth criterion for a p-th order scheme,
 *   dt = eta (A(1) / A(p-2))^{1/(p-3)},
 *   A(k) = sqrt(|a^(k-1)| |a^(k+1)|) + |a^(k)|,
 * with p = 6: dt = eta (A(1)/A(4))^{1/3}, a^(0) = a, a^(1) = j, a^(2) = s.
 * A(4) == 0 imposes no limit (returns +inf).
 */
double orc_dt_criterion(const double a[3], const double j[3], const double s[3],
                        const double d3[3], const double d4[3], const double d5[3],
                        double eta)
{
    double A1 = sqrt(norm3(a) * norm3(s)) + norm3(j);
    double A4 = sqrt(norm3(d3) * norm3(d5)) + norm3(d4);
    if (!(A4 > 0.0)) return INFINITY;
    return eta * cbrt(A1 / A4);
}

/* Ratio with "no constraint" when the denominator vanishes. */
static double safe_ratio(double num, double den) { return den > 0.0 ? num / den : INFINITY; }

/*
 * Initial step (reading: the configuration gives no start-up rule; we take
 * dt0 = eta_init * min(|a|/|j|, sqrt(|a|/|s|)) from the start-up a, j, s).
 */
double orc_dt_initial(const double a[3], const double j[3], const double s[3],
                      double eta_init)
{
    double an = norm3(a);
    double r1 = safe_ratio(an, norm3(j));
    double r2 = safe_ratio(an, norm3(s));
    double r = r1 < sqrt(r2) ? r1 : sqrt(r2);
    return eta_init * r;
}

/* Largest power of two <= x (x > 0, finite). */
static double pow2_floor(double x)
{
    int e;
    double f = frexp(x, &e); /* x = f 2^e, f in [0.5, 1) */
    (void)f;
    return ldexp(1.0, e - 1);
}

/*
 * Power-of-two block step (Makino 1991; Aarseth 2003):
 *  - dt_crit < dt_old: shrink to the largest power of two <= dt_crit;
 *  - dt_crit >= 2 dt_old and t1 a multiple of 2 dt_old: double once;
 *  - otherwise keep dt_old;
 * then clamp to [dt_min, dt_max].  *underflow is set when dt_crit < dt_min.
 */
double orc_dt_quantize(double dt_crit, double dt_old, double t1, double dt_min,
                       double dt_max, int *underflow)
{
    double dt = dt_old;
    if (dt_crit < dt_min || dt_crit != dt_crit) {
        if (underflow) *underflow = 1;
        return dt_min;
    }
    if (dt_crit < dt_old) {
        dt = pow2_floor(dt_crit);
    } else if (dt_crit >= 2.0 * dt_old && fmod(t1, 2.0 * dt_old) == 0.0) {
        dt = 2.0 * dt_old;
    }
    if (dt > dt_max) dt = dt_max;
    if (dt < dt_min) dt = dt_min;
    return dt;
}

/* Start-up quantisation: largest power of two <= dt0, clamped. */
double orc_dt_quantize_initial(double dt0, double dt_min, double dt_max)
{
    if (dt0 != dt0 || dt0 <= 0.0) return dt_min;
    if (isinf(dt0)) return dt_max;
    double dt = pow2_floor(dt0);
    if (dt > dt_max) dt = dt_max;
    if (dt < dt_min) dt = dt_min;
    return dt;
}

/* ------------------------------------------------------------------------- */
/* 4th-order Hermite scheme (Makino & Aarseth 1992): the lower-order member   */
/* of the family the paper's code inherits from HiGPUs; uses a and jerk only  */
/* ------------------------------------------------------------------------- */

/* Predictor through jerk: xp = x + v d + a d^2/2 + j d^3/6, vp = v + a d + j d^2/2. */
void orc_predict4(int64_t n, const double *x, const double *v, const double *a,
                  const double *j, const double *t, double t_next, double *xp, double *vp)
{
    for (int64_t i = 0; i < n; i++) {
        double dt = t_next - t[i];
        double d2 = dt * dt / 2.0, d3 = dt * dt * dt / 6.0;
        for (int d = 0; d < 3; d++) {
            const int64_t o = 3 * i + d;
            xp[o] = x[o] + v[o] * dt + a[o] * d2 + j[o] * d3;
            vp[o] = v[o] + a[o] * dt + j[o] * d2;
        }
    }
}

/*
 * 4th-order Hermite corrector, h = t1 - t0:
 *   v1 = v0 + h/2 (a0 + a1) + h^2/12 (j0 - j1)
 *   x1 = x0 + h/2 (v0 + v1) + h^2/12 (a0 - a1)
 */
void orc_correct4(double h, const double x0[3], const double v0[3], const double a0[3],
                  const double j0[3], const double a1[3], const double j1[3],
                  double x1[3], double v1[3])
{
    for (int d = 0; d < 3; d++) {
        v1[d] = v0[d] + h / 2.0 * (a0[d] + a1[d]) + h * h / 12.0 * (j0[d] - j1[d]);
        x1[d] = x0[d] + h / 2.0 * (v0[d] + v1[d]) + h * h / 12.0 * (a0[d] - a1[d]);
    }
}

/*
 * The cubic through (a, j) at t0 and t1: its 2nd and 3rd derivatives at t1.
 * With p(u) = a0 + j0 u + c2 u^2 + c3 u^3, u = t - t0, p(h) = a1, p'(h) = j1:
 *   c2 = (3 (a1 - a0) - h (2 j0 + j1)) / h^2,  c3 = (2 (a0 - a1) + h (j0 + j1)) / h^3,
 *   a''(t1) = 2 c2 + 6 c3 h,  a'''(t1) = 6 c3.
 */
void orc_interp4(double h, const double a0[3], const double j0[3], const double a1[3],
                 const double j1[3], double s1[3], double c1[3])
{
    for (int d = 0; d < 3; d++) {
        double c2 = (3.0 * (a1[d] - a0[d]) - h * (2.0 * j0[d] + j1[d])) / (h * h);
        double c3 = (2.0 * (a0[d] - a1[d]) + h * (j0[d] + j1[d])) / (h * h * h);
        s1[d] = 2.0 * c2 + 6.0 * c3 * h;
        c1[d] = 6.0 * c3;
    }
}

/* Aarseth's criterion: dt = sqrt(eta (|a||a2| + |j|^2) / (|j||a3| + |a2|^2)). */
double orc_dt_aarseth(const double a[3], const double j[3], const double s[3],
                      const double c[3], double eta)
{
    double an = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    double jn = sqrt(j[0] * j[0] + j[1] * j[1] + j[2] * j[2]);
    double sn = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    double cn = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    double den = jn * cn + sn * sn;
    if (!(den > 0.0)) return INFINITY;
    return sqrt(eta * (an * sn + jn * jn) / den);
}

/* ------------------------------------------------------------------------- */
/* The integrator: start-up, block step, run, diagnostics                     */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t n;
    double eps2, eta, eta_init, dt_min, dt_max;
    double *m;                         /* [n] */
    double *x, *v, *a, *j, *s, *c;     /* [n][3] */
    double *t, *dt, *pot;              /* [n] */
    /* work */
    double *xp, *vp, *ap;              /* [n][3] predicted */
    int64_t *act;                      /* [n] */
    double *fa, *fj, *fs, *fp;         /* [n][3], [n] evaluation output */
    int64_t n_underflow;
    int order;                         /* 6 (default) or 4 */
    /* optional relative perturbation of every evaluation (orc_set_noise) */
    double noise_a, noise_j, noise_s;
    uint64_t noise_seed, noise_calls;
} orc_sim;

size_t orc_sim_sizeof(void) { return sizeof(orc_sim); }

/*
 * Bind a simulation to caller-owned state arrays (m, x, v: inputs; a, j, s, c,
 * t, dt, pot: outputs of orc_init).  Work arrays are allocated here and
 * released by orc_free.  Returns 0 on success.
 */
int orc_bind(orc_sim *S, int64_t n, double eps, double eta, double eta_init,
             double dt_min, double dt_max, double *m, double *x, double *v,
             double *a, double *j, double *s, double *c, double *t, double *dt,
             double *pot)
{
    memset(S, 0, sizeof *S);
    S->n = n;
    S->eps2 = eps * eps;
    S->eta = eta;
    S->eta_init = eta_init;
    S->dt_min = dt_min;
    S->dt_max = dt_max;
    S->m = m; S->x = x; S->v = v; S->a = a; S->j = j; S->s = s; S->c = c;
    S->t = t; S->dt = dt; S->pot = pot;
    size_t v3 = (size_t)(n > 0 ? n : 1) * 3 * sizeof(double);
    S->xp = malloc(v3); S->vp = malloc(v3); S->ap = malloc(v3);
    S->fa = malloc(v3); S->fj = malloc(v3); S->fs = malloc(v3);
    S->fp = malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    S->act = malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!S->xp || !S->vp || !S->ap || !S->fa || !S->fj || !S->fs || !S->fp || !S->act)
        return 1;
    return 0;
}

void orc_free(orc_sim *S)
{
    free(S->xp); free(S->vp); free(S->ap);
    free(S->fa); free(S->fj); free(S->fs); free(S->fp); free(S->act);
    S->xp = S->vp = S->ap = S->fa = S->fj = S->fs = S->fp = NULL;
    S->act = NULL;
}

/*
 * Perturbed evaluations, for experiments on how accurate the pair arithmetic
 * must be (the paper's Sec. 2: double precision is needed in the distances
 * and accelerations).  Off unless orc_set_noise gave a non-zero size; with
 * all sizes 0 nothing below changes any result.  Each component q of a, jerk
 * and snap of every evaluated particle is multiplied by (1 + e_q u), u
 * uniform in [-1, 1), so the relative error of each vector stays <= e_q.
 * u comes from the counter-based SplitMix64 generator (Steele, Lea & Flood
 * 2014) keyed by (seed, evaluation number, particle, component): the
 * perturbation does not depend on the number of threads.
 */
static uint64_t splitmix64(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static double noise_unit(uint64_t seed, uint64_t call, int64_t i, int q)
{
    uint64_t h = splitmix64(seed ^ splitmix64((call << 40) ^ ((uint64_t)i * 16u + (uint64_t)q)));
    return (double)(h >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

static void orc_perturb(orc_sim *S, int64_t na)
{
    if (S->noise_a == 0.0 && S->noise_j == 0.0 && S->noise_s == 0.0) return;
    const uint64_t call = S->noise_calls++;
    for (int64_t k = 0; k < na; k++) {
        const int64_t i = S->act[k];
        for (int d = 0; d < 3; d++) {
            S->fa[3 * k + d] *= 1.0 + S->noise_a * noise_unit(S->noise_seed, call, i, d);
            S->fj[3 * k + d] *= 1.0 + S->noise_j * noise_unit(S->noise_seed, call, i, 3 + d);
            S->fs[3 * k + d] *= 1.0 + S->noise_s * noise_unit(S->noise_seed, call, i, 6 + d);
        }
    }
}

/* Relative sizes of the evaluation perturbation (all 0: none, the default). */
int orc_set_noise(orc_sim *S, double ea, double ej, double es, uint64_t seed)
{
    if (!(ea >= 0.0) || !(ej >= 0.0) || !(es >= 0.0)) return 1;
    S->noise_a = ea;
    S->noise_j = ej;
    S->noise_s = es;
    S->noise_seed = seed;
    S->noise_calls = 0;
    return 0;
}

/*
 * Start-up at t = 0 (reading: snap needs the j-particles' accelerations, so
 * the first pass runs with a = 0 and yields a and jerk, the second pass uses
 * that a and yields snap; crackle starts at 0).
 */
void orc_init(orc_sim *S)
{
    const int64_t n = S->n;
    for (int64_t i = 0; i < n; i++) {
        S->t[i] = 0.0;
        S->act[i] = i;
        for (int d = 0; d < 3; d++) {
            S->a[3 * i + d] = S->j[3 * i + d] = S->s[3 * i + d] = S->c[3 * i + d] = 0.0;
        }
    }
    /* the 4th-order scheme needs no snap: one pass (a = 0 in the predictor) */
    const int passes = S->order == 4 ? 1 : 2;
    for (int pass = 0; pass < passes; pass++) {
        orc_predict(n, S->x, S->v, S->a, S->j, S->s, S->c, S->t, 0.0, S->xp, S->vp, S->ap);
        orc_force(n, S->m, S->xp, S->vp, S->ap, S->eps2, n, S->act, S->fa, S->fj, S->fs, S->fp);
        orc_perturb(S, n);
        for (int64_t i = 0; i < n; i++) {
            for (int d = 0; d < 3; d++) {
                S->a[3 * i + d] = S->fa[3 * i + d];
                S->j[3 * i + d] = S->fj[3 * i + d];
                S->s[3 * i + d] = pass == 1 ? S->fs[3 * i + d] : 0.0;
            }
            S->pot[i] = S->fp[i];
        }
    }
    for (int64_t i = 0; i < n; i++) {
        double dt0 = orc_dt_initial(&S->a[3 * i], &S->j[3 * i], &S->s[3 * i], S->eta_init);
        S->dt[i] = orc_dt_quantize_initial(dt0, S->dt_min, S->dt_max);
    }
}

/*
 * Block scheduler: t_next = min_i (t_i + dt_i); the active set is every i with
 * t_i + dt_i == t_next, exactly (dt are powers of two and t_i multiples of
 * dt_i), listed in increasing index order.  Returns the number of active
 * particles; writes t_next.
 */
int64_t orc_select(const orc_sim *S, double *t_next, int64_t *act)
{
    double tn = INFINITY;
    for (int64_t i = 0; i < S->n; i++) {
        double ti = S->t[i] + S->dt[i];
        if (ti < tn) tn = ti;
    }
    int64_t na = 0;
    for (int64_t i = 0; i < S->n; i++)
        if (S->t[i] + S->dt[i] == tn) act[na++] = i;
    *t_next = tn;
    return na;
}

/*
 * One block step: select, predict everybody to t_next, evaluate the active
 * set on the predicted state, correct, interpolate the higher derivatives,
 * set the new power-of-two step.  Returns the number of active particles.
 */
/* 4th-order block step: predictor through jerk, a and jerk evaluated (the
 * relative accelerations are set to zero, snap is not used), 4th-order
 * corrector, cubic-interpolated 2nd/3rd derivatives (kept in s and c),
 * Aarseth's criterion, the same power-of-two quantisation. */
static int64_t orc_block_step4(orc_sim *S, double tn, int64_t na)
{
    orc_predict4(S->n, S->x, S->v, S->a, S->j, S->t, tn, S->xp, S->vp);
    for (int64_t q = 0; q < 3 * S->n; q++) S->ap[q] = 0.0;
    orc_force(S->n, S->m, S->xp, S->vp, S->ap, S->eps2, na, S->act, S->fa, S->fj, S->fs, S->fp);
    orc_perturb(S, na);
    for (int64_t k = 0; k < na; k++) {
        const int64_t i = S->act[k];
        double *x = &S->x[3 * i], *v = &S->v[3 * i], *a = &S->a[3 * i];
        double *jj = &S->j[3 * i], *s = &S->s[3 * i], *c = &S->c[3 * i];
        const double *a1 = &S->fa[3 * k], *j1 = &S->fj[3 * k];
        double h = tn - S->t[i];
        double x1[3], v1[3], s1[3], c1[3];
        orc_correct4(h, x, v, a, jj, a1, j1, x1, v1);
        orc_interp4(h, a, jj, a1, j1, s1, c1);
        double dtc = orc_dt_aarseth(a1, j1, s1, c1, S->eta);
        int uf = 0;
        double dtn = orc_dt_quantize(dtc, S->dt[i], tn, S->dt_min, S->dt_max, &uf);
        if (uf) S->n_underflow++;
        for (int d = 0; d < 3; d++) {
            x[d] = x1[d];
            v[d] = v1[d];
            a[d] = a1[d];
            jj[d] = j1[d];
            s[d] = s1[d];
            c[d] = c1[d];
        }
        S->pot[i] = S->fp[k];
        S->t[i] = tn;
        S->dt[i] = dtn;
    }
    return na;
}

int64_t orc_block_step(orc_sim *S, double *t_next_out)
{
    double tn;
    int64_t na = orc_select(S, &tn, S->act);
    if (S->order == 4) {
        orc_block_step4(S, tn, na);
        if (t_next_out) *t_next_out = tn;
        return na;
    }
    orc_predict(S->n, S->x, S->v, S->a, S->j, S->s, S->c, S->t, tn, S->xp, S->vp, S->ap);
    orc_force(S->n, S->m, S->xp, S->vp, S->ap, S->eps2, na, S->act, S->fa, S->fj, S->fs, S->fp);
    orc_perturb(S, na);
    for (int64_t k = 0; k < na; k++) {
        const int64_t i = S->act[k];
        double *x = &S->x[3 * i], *v = &S->v[3 * i], *a = &S->a[3 * i];
        double *jj = &S->j[3 * i], *s = &S->s[3 * i], *c = &S->c[3 * i];
        const double *a1 = &S->fa[3 * k], *j1 = &S->fj[3 * k], *s1 = &S->fs[3 * k];
        double h = tn - S->t[i];
        double x1[3], v1[3], d3[3], d4[3], d5[3];
        orc_correct(h, x, v, a, jj, s, a1, j1, s1, x1, v1);
        orc_interp_derivs(h, a, jj, s, a1, j1, s1, d3, d4, d5);
        double dtc = orc_dt_criterion(a1, j1, s1, d3, d4, d5, S->eta);
        int uf = 0;
        double dtn = orc_dt_quantize(dtc, S->dt[i], tn, S->dt_min, S->dt_max, &uf);
        if (uf) S->n_underflow++;
        for (int d = 0; d < 3; d++) {
            x[d] = x1[d];
            v[d] = v1[d];
            a[d] = a1[d];
            jj[d] = j1[d];
            s[d] = s1[d];
            c[d] = d3[d];
        }
        S->pot[i] = S->fp[k];
        S->t[i] = tn;
        S->dt[i] = dtn;
    }
    if (t_next_out) *t_next_out = tn;
    return na;
}

/*
 * Block steps until every particle has reached t_end (the next block time
 * would exceed t_end).  Returns the number of block steps; *interactions
 * accumulates sum over steps of n_active * (n - 1).
 */
int64_t orc_run(orc_sim *S, double t_end, int64_t max_steps, double *interactions)
{
    int64_t steps = 0;
    double inter = 0.0;
    while (max_steps < 0 || steps < max_steps) {
        double tn = INFINITY;
        for (int64_t i = 0; i < S->n; i++) {
            double ti = S->t[i] + S->dt[i];
            if (ti < tn) tn = ti;
        }
        if (!(tn <= t_end)) break;
        int64_t na = orc_block_step(S, NULL);
        inter += (double)na * (double)(S->n - 1);
        steps++;
    }
    if (interactions) *interactions += inter;
    return steps;
}

/*
 * Diagnostics at a common time t: every particle is predicted to t (exact
 * for synchronised particles), the potential is re-evaluated on the predicted
 * positions, then E_kin = 1/2 sum m v^2, E_pot = 1/2 sum m_i pot_i, total
 * momentum P = sum m v and angular momentum L = sum m x cross v.
 */
void orc_energy(orc_sim *S, double t, double *ekin, double *epot, double P[3],
                double L[3])
{
    const int64_t n = S->n;
    if (S->order == 4)
        orc_predict4(n, S->x, S->v, S->a, S->j, S->t, t, S->xp, S->vp);
    else
        orc_predict(n, S->x, S->v, S->a, S->j, S->s, S->c, S->t, t, S->xp, S->vp, S->ap);
    for (int64_t i = 0; i < n; i++) S->act[i] = i;
    orc_force(n, S->m, S->xp, S->vp, S->ap, S->eps2, n, S->act, S->fa, S->fj, S->fs, S->fp);
    double ek = 0, ep = 0, p[3] = {0, 0, 0}, l[3] = {0, 0, 0};
    for (int64_t i = 0; i < n; i++) {
        const double *x = &S->xp[3 * i], *v = &S->vp[3 * i];
        double mi = S->m[i];
        ek += 0.5 * mi * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        ep += 0.5 * mi * S->fp[i];
        for (int d = 0; d < 3; d++) p[d] += mi * v[d];
        l[0] += mi * (x[1] * v[2] - x[2] * v[1]);
        l[1] += mi * (x[2] * v[0] - x[0] * v[2]);
        l[2] += mi * (x[0] * v[1] - x[1] * v[0]);
    }
    *ekin = ek;
    *epot = ep;
    for (int d = 0; d < 3; d++) {
        P[d] = p[d];
        L[d] = l[d];
    }
}

int64_t orc_underflows(const orc_sim *S) { return S->n_underflow; }

/* Integration order of the simulation: 6 (default) or 4.  Call before orc_init. */
int orc_set_order(orc_sim *S, int order)
{
    if (order != 4 && order != 6) return 1;
    S->order = order;
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel loops from now on (>= 1; ignored without OpenMP).
 * Results do not depend on it: each i sums its j in a fixed order. */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

// nb_step.cuh -- per-particle FP64 device functions of the integrator:
// predictor, corrector + quintic derivatives + time step, start-up step,
// and the 4th-order Hermite corrector + cubic derivatives + Aarseth step.
//
// Method: the paper's Sec. 2 integrator (Hermite 6th order, block time
// steps, inherited from HiGPUs); formulas after Nitadori & Makino 2008,
// power-of-two steps after Makino 1991 / Aarseth 2003.
#pragma once

#include "nb_internal.cuh"

namespace nb {

// Largest power of two <= x for normal positive x (exponent bits only).
__device__ __forceinline__ double pow2_floor_dev(double x) {
    return __hiloint2double(__double2hiint(x) & 0x7ff00000, 0);
}

__device__ __forceinline__ double norm3_dev(double a, double b, double c) {
    return sqrt(fma(a, a, fma(b, b, c * c)));
}

// Start-up step: eta_init * min(|a|/|j|, sqrt(|a|/|s|)), quantised down to a
// power of two and clamped; a vanishing denominator imposes no limit.
__device__ __forceinline__ double dt_start(const Dev &d, const double o[10]) {
    const double an = norm3_dev(o[0], o[1], o[2]);
    const double jn = norm3_dev(o[3], o[4], o[5]);
    const double sn = norm3_dev(o[6], o[7], o[8]);
    double r = INFINITY;
    if (jn > 0.0) r = an / jn;
    if (sn > 0.0) r = fmin(r, sqrt(an / sn));
    const double dt0 = d.eta_init * r;
    double dt;
    if (!(dt0 > 0.0)) dt = d.dt_min;          // zero or NaN
    else if (isinf(dt0)) dt = d.dt_max;
    else dt = fmin(fmax(pow2_floor_dev(dt0), d.dt_min), d.dt_max);
    return dt;
}

// Power-of-two block step from the criterion's dt: shrink to the largest
// power of two below it, double once when it allows twice the old step and
// t1 is a multiple of that, clamp to [dt_min, dt_max]; a criterion below
// dt_min (or NaN) is counted as an underflow.
__device__ __forceinline__ double block_step_quantize(const Dev &d, double dtc, double dt_old,
                                                      double tn) {
    double dtn = dt_old;
    if (!(dtc >= d.dt_min)) {               // below the floor, or NaN
        dtn = d.dt_min;
        atomicAdd(d.ctr_underflow, 1ull);
    } else if (dtc < dt_old) {
        dtn = pow2_floor_dev(dtc);
    } else if (dtc >= 2.0 * dt_old) {
        const double q = tn * (0.5 / dt_old);  // exact: power-of-two scaling
        if (q == trunc(q)) dtn = 2.0 * dt_old;
    }
    return fmin(fmax(dtn, d.dt_min), d.dt_max);
}

// Predict particle i (global index) to time tn; Horner-free power form,
// small terms summed first:  x_p = x + (v d + (a d^2/2 + (j d^3/6 + ...))).
// The 4th-order scheme predicts through jerk only (its s and c hold the
// interpolated derivatives used by the time-step criterion).
__device__ __forceinline__ void predict_particle(const Dev &d, int64_t i, double tn,
                                                 double xp[3], double vp[3], double ap[3]) {
    const int64_t n = d.n;
    const bool through_crackle = d.order != 4;
    const double h = tn - d.t[i];
    const double h2 = h * h * 0.5;
    const double h3 = h2 * h * (1.0 / 3.0);
    const double h4 = h3 * h * 0.25;
    const double h5 = h4 * h * 0.2;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double x = d.x[k * n + i], v = d.v[k * n + i], a = d.a[k * n + i];
        const double jj = d.j[k * n + i];
        const double s = through_crackle ? d.s[k * n + i] : 0.0;
        const double c = through_crackle ? d.c[k * n + i] : 0.0;
        xp[k] = x + fma(h, v, fma(h2, a, fma(h3, jj, fma(h4, s, h5 * c))));
        vp[k] = v + fma(h, a, fma(h2, jj, fma(h3, s, h4 * c)));
        ap[k] = a + fma(h, jj, fma(h2, s, h3 * c));
    }
}

// Corrector, interpolated derivatives, new power-of-two step; writes the
// state of particle i.  o = {a1[3], j1[3], s1[3], pot} evaluated at tn on the
// predicted state.
//
//   v1 = v0 + h/2 (a1 + a0) - h^2/10 (j1 - j0) + h^3/120 (s1 + s0)
//   x1 = x0 + h/2 (v1 + v0) - h^2/10 (a1 - a0) + h^3/120 (j1 + j0)
// The quintic through (a, j, s) at both ends has, at t1, with
// D = a1 - a0, Jp/Jm = j1 +/- j0, Sp/Sm = s1 +/- s0:
//   c5 = (6 D - 3 h Jp + h^2 Sm / 2) / h^5      (so a^(5) = 120 c5)
//   c4 = (h Sp / 4 - Jm / 2) / h^3
//   a^(5) = 120 c5,  a^(4) = 24 c4 + 60 h c5,  a^(3) = Sm/h + 12 h c4 + 10 h^2 c5
// New step: eta (A1/A4)^{1/3}, A1 = sqrt(|a||s|) + |j|, A4 = sqrt(|a3||a5|) + |a4|.
__device__ __forceinline__ void correct_particle(const Dev &d, int64_t i, double tn,
                                                 const double o[10]) {
    const int64_t n = d.n;
    const double t0 = d.t[i];
    const double h = tn - t0;
    const double hinv = 1.0 / h;
    const double hinv2 = hinv * hinv;
    const double hinv3 = hinv2 * hinv;
    const double hinv5 = hinv3 * hinv2;
    double x1[3], v1[3], d3[3], d4[3], d5[3];
    bool finite = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double x0 = d.x[k * n + i], v0 = d.v[k * n + i];
        const double a0 = d.a[k * n + i], j0 = d.j[k * n + i], s0 = d.s[k * n + i];
        const double a1 = o[k], j1 = o[3 + k], s1 = o[6 + k];
        const double hh = h * h, hhh = hh * h;
        v1[k] = v0 + (0.5 * h * (a1 + a0) - 0.1 * hh * (j1 - j0) + (hhh / 120.0) * (s1 + s0));
        x1[k] = x0 + (0.5 * h * (v1[k] + v0) - 0.1 * hh * (a1 - a0) + (hhh / 120.0) * (j1 + j0));
        const double D = a1 - a0, Jp = j1 + j0, Jm = j1 - j0, Sp = s1 + s0, Sm = s1 - s0;
        const double c5 = (6.0 * D - 3.0 * h * Jp + 0.5 * hh * Sm) * hinv5;
        const double c4 = (0.25 * h * Sp - 0.5 * Jm) * hinv3;
        d5[k] = 120.0 * c5;
        d4[k] = 24.0 * c4 + 60.0 * h * c5;
        d3[k] = Sm * hinv + 12.0 * h * c4 + 10.0 * hh * c5;
        finite = finite && isfinite(x1[k]) && isfinite(v1[k]) && isfinite(a1) && isfinite(j1) &&
                 isfinite(s1) && isfinite(d3[k]);
    }
    const double an = norm3_dev(o[0], o[1], o[2]);
    const double jn = norm3_dev(o[3], o[4], o[5]);
    const double sn = norm3_dev(o[6], o[7], o[8]);
    const double A1 = sqrt(an * sn) + jn;
    const double A4 = sqrt(norm3_dev(d3[0], d3[1], d3[2]) * norm3_dev(d5[0], d5[1], d5[2])) +
                      norm3_dev(d4[0], d4[1], d4[2]);
    const double dtc = (A4 > 0.0) ? d.eta * cbrt(A1 / A4) : INFINITY;
    const double dtn = block_step_quantize(d, dtc, d.dt[i], tn);
    if (!finite) atomicOr(d.err, kErrNonFinite);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        d.x[k * n + i] = x1[k];
        d.v[k * n + i] = v1[k];
        d.a[k * n + i] = o[k];
        d.j[k * n + i] = o[3 + k];
        d.s[k * n + i] = o[6 + k];
        d.c[k * n + i] = d3[k];
    }
    d.pot[i] = o[9];
    d.t[i] = tn;
    d.dt[i] = dtn;
}

// 4th-order Hermite corrector (Makino & Aarseth 1992), o = {a1, j1, -, pot}:
//   v1 = v0 + h/2 (a0 + a1) + h^2/12 (j0 - j1)
//   x1 = x0 + h/2 (v0 + v1) + h^2/12 (a0 - a1)
// The cubic through (a, j) at both ends gives at t1
//   a2 = (6 (a0 - a1) + 2 h (j0 + 2 j1)) / h^2,  a3 = (12 (a0 - a1) + 6 h (j0 + j1)) / h^3,
// kept in s and c; new step from Aarseth's criterion
//   dt = sqrt(eta (|a1||a2| + |j1|^2) / (|j1||a3| + |a2|^2)).
__device__ __forceinline__ void correct_particle4(const Dev &d, int64_t i, double tn,
                                                  const double o[10]) {
    const int64_t n = d.n;
    const double h = tn - d.t[i];
    const double hinv = 1.0 / h;
    const double hinv2 = hinv * hinv;
    const double hh12 = h * h * (1.0 / 12.0);
    double x1[3], v1[3], a2[3], a3[3];
    bool finite = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double x0 = d.x[k * n + i], v0 = d.v[k * n + i];
        const double a0 = d.a[k * n + i], j0 = d.j[k * n + i];
        const double a1 = o[k], j1 = o[3 + k];
        v1[k] = v0 + (0.5 * h * (a0 + a1) + hh12 * (j0 - j1));
        x1[k] = x0 + (0.5 * h * (v0 + v1[k]) + hh12 * (a0 - a1));
        const double D = a0 - a1;
        a2[k] = (6.0 * D + 2.0 * h * (j0 + 2.0 * j1)) * hinv2;
        a3[k] = (12.0 * D + 6.0 * h * (j0 + j1)) * (hinv2 * hinv);
        finite = finite && isfinite(x1[k]) && isfinite(v1[k]) && isfinite(a1) && isfinite(j1) &&
                 isfinite(a3[k]);
    }
    const double an = norm3_dev(o[0], o[1], o[2]);
    const double jn = norm3_dev(o[3], o[4], o[5]);
    const double sn = norm3_dev(a2[0], a2[1], a2[2]);
    const double cn = norm3_dev(a3[0], a3[1], a3[2]);
    const double den = fma(jn, cn, sn * sn);
    const double dtc = (den > 0.0) ? sqrt(d.eta * fma(an, sn, jn * jn) / den) : INFINITY;
    const double dtn = block_step_quantize(d, dtc, d.dt[i], tn);
    if (!finite) atomicOr(d.err, kErrNonFinite);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        d.x[k * n + i] = x1[k];
        d.v[k * n + i] = v1[k];
        d.a[k * n + i] = o[k];
        d.j[k * n + i] = o[3 + k];
        d.s[k * n + i] = a2[k];
        d.c[k * n + i] = a3[k];
    }
    d.pot[i] = o[9];
    d.t[i] = tn;
    d.dt[i] = dtn;
}

}  // namespace nb

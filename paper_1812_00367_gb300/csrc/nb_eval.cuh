// nb_eval.cuh -- the hot O(N_active x N) evaluation of acceleration, jerk,
// snap and potential (the paper's Sec. 4 kernel; 6th-order Hermite pair terms
// of Nitadori & Makino 2008) in three arithmetics, plus its j-split reduction.
//
// Per pair, with r = x_j - x_i, v = v_j - v_i, a = a_j - a_i (predicted),
// y = (r.r + eps^2)^{-1/2}, q = m_j y^3, alpha = (r.v) y^2, zeta = (v.v + r.a) y^2,
// beta = zeta + alpha^2:
//   w1 = v - 3 alpha r,            A1 = q w1         (jerk term)
//   w2 = a - 6 alpha w1 - 3 beta r, A2 = q w2         (snap term)
//   A0 = q r,  pot -= m_j y
// i.e. NM08's A1 = m v/s^3 - 3 alpha A0 and A2 = m a/s^3 - 6 alpha A1 - 3 beta A0
// with the large alpha terms cancelling inside each pair before it is summed
// (that keeps the FP32 path within its bound on strongly cancelling sums).
// Every per-pair operation is a multiply, an add or a fused multiply-add:
// 50 FP64 instructions per pair on the FP64 path (the reciprocal square
// root's seed is refined on the FP32 and integer pipes, NB_FP64_RSQRT3; one
// exact doubling is done on the integer pipe; the potential m y is summed in
// float-float on the FP32 pipe, NB_FP64_POT_FF).  The 4th-order scheme (Makino & Aarseth 1992) keeps
// A0, A1 and the potential only (interact4: 29 FP64 instructions per pair).
//
// Work decomposition: a piece of work is (cluster, i-tile, j-range).  An
// i-tile holds kTPB / gl active particles; gl lanes of a warp share one i and
// take every gl-th j of each tile (gl = 1: i-parallel, j broadcast from
// shared memory; gl = 32: j-parallel for tiny active sets, warp-shuffle
// reduction).  A batch of clusters is cut into split items (each cluster's j
// range split S ways, items fetched dynamically); a single cluster into
// stream-K ranges (CTA k takes units [U k / G, U (k+1) / G) of the U =
// i-tiles x j-tiles units).  j-tiles of kTJ particles are copied global ->
// shared by the TMA engine (cp.async.bulk) into a ring of stages guarded by
// mbarriers.  When an i-tile's j range is covered by several pieces, each
// writes FP64 partial sums; the CTA that finishes the i-tile last (atomic
// counter) adds them in piece order (deterministic) and finalises.  Thread 0
// describes each piece in a shared-memory record so that the pair loop keeps
// only its own state in registers.
#pragma once

#include "nb_internal.cuh"
#include "nb_step.cuh"

namespace nb {

template <int P>
struct Prec;

// ===================================================================== FP64
template <>
struct Prec<NB_FP64> {
    using J = J64;
    static constexpr int kPerRec = 1;  // particles per record
    struct I {
        double x[3], v[3], a[3];
        double m1, nz;  // -1.0, -0.0 from kernel parameters (see Dev)
    };
    struct Acc {
        double a[3], j[3], s[3], p;
#if NB_FP64_POT_FF
        ff pf;  // the current j-tile's potential as a float pair
#endif
    };
    static __device__ __forceinline__ void prepare(I &i, const Dev &d) {
        i.m1 = d.neg_one;
        i.nz = d.neg_zero;
    }
    // product and difference; as FMAs with run-time -0.0 / -1.0 when
    // NB_FP64_ALL_FMA (same IEEE results: a*b + (-0) == a*b, b*(-1) + a == a - b)
    static __device__ __forceinline__ double fma_rt(double a, double b, double c) {
        double r;
        asm("fma.rn.f64 %0, %1, %2, %3;" : "=d"(r) : "d"(a), "d"(b), "d"(c));
        return r;
    }
    static __device__ __forceinline__ double mul(const I &i, double a, double b) {
        if constexpr (NB_FP64_ALL_FMA) return fma_rt(a, b, i.nz);
        else return a * b;
    }
    static __device__ __forceinline__ double sub(const I &i, double a, double b) {
        if constexpr (NB_FP64_ALL_FMA) return fma_rt(b, i.m1, a);
        else return a - b;
    }
    static __device__ __forceinline__ I load_i(const J *jarr, int64_t k) {
        const J e = jarr[k];
        I r;
        r.x[0] = e.q[0].x; r.x[1] = e.q[0].y; r.x[2] = e.q[1].x;
        r.v[0] = e.q[2].x; r.v[1] = e.q[2].y; r.v[2] = e.q[3].x;
        r.a[0] = e.q[3].y; r.a[1] = e.q[4].x; r.a[2] = e.q[4].y;
        return r;
    }
    static __device__ __forceinline__ void zero(Acc &c) {
#pragma unroll
        for (int k = 0; k < 3; ++k) c.a[k] = c.j[k] = c.s[k] = 0.0;
        c.p = 0.0;
#if NB_FP64_POT_FF
        c.pf = ff{0.f, 0.f};
#endif
    }
    // potential term m y: FP64 DFMA, or float-float on the FP32 pipe
    static __device__ __forceinline__ void pot_term(const J &jj, bool self, double m, double y,
                                                    Acc &c) {
#if NB_FP64_POT_FF
        (void)m;
        const float2 mf = jj.mf;
        const ff yf = ff_from_pos_double(y);
        const ff mff = ff{self ? 0.f : mf.x, self ? 0.f : mf.y};
        // renormalised every term (|lo| stays below half an ulp of hi): a
        // 64-term tile sum is good to ~2^-45, and tiles add up in FP64
        c.pf = ff_add(c.pf, ff_mul_lazy(mff, yf));
#else
        (void)jj;
        (void)self;
        c.p = fma(m, y, c.p);
#endif
    }
#if NB_FP64_POT_FF
    // End of a j-tile: the tile's float-pair potential joins the FP64 total.
    static __device__ __forceinline__ void tile_done(Acc &c) {
        c.p += (double)c.pf.hi + (double)c.pf.lo;
        c.pf = ff{0.f, 0.f};
    }
#else
    static __device__ __forceinline__ void tile_done(Acc &) {}
#endif
    static __device__ __forceinline__ void interact(const I &i, const J &jj, bool self,
                                                    double eps2, float, Acc &c) {
        const double2 q0 = jj.q[0], q1 = jj.q[1], q2 = jj.q[2], q3 = jj.q[3], q4 = jj.q[4];
        const double rx = sub(i, q0.x, i.x[0]), ry = sub(i, q0.y, i.x[1]), rz = sub(i, q1.x, i.x[2]);
        const double vx = sub(i, q2.x, i.v[0]), vy = sub(i, q2.y, i.v[1]), vz = sub(i, q3.x, i.v[2]);
        const double ax = sub(i, q3.y, i.a[0]), ay = sub(i, q4.x, i.a[1]), az = sub(i, q4.y, i.a[2]);
        double r2 = fma(rx, rx, fma(ry, ry, fma(rz, rz, eps2)));
        double m = q1.y;
        r2 = self ? 1.0 : r2;  // selects, not FP64 arithmetic
        m = self ? 0.0 : m;
        const double y = NB_FP64_RSQRT3 ? rsqrt_f64_3(r2, i.nz)
                         : (NB_FP64_ALL_FMA ? rsqrt_f64_fma(r2, i.nz) : rsqrt_f64(r2));
        const double y2 = mul(i, y, y);
        pot_term(jj, self, m, y, c);               // potential: sum m y
        const double q = mul(i, mul(i, m, y2), y); // m y^3
        const double rv = fma(rx, vx, fma(ry, vy, mul(i, rz, vz)));
        const double w = fma(vx, vx, fma(vy, vy, fma(vz, vz, fma(rx, ax, fma(ry, ay, mul(i, rz, az))))));
        const double al = mul(i, rv, y2);
        const double ze = mul(i, w, y2);
        const double al3 = mul(i, 3.0, al);
        const double be3 = mul(i, 3.0, fma(al, al, ze));  // 3 beta
        const double al6 = twice_int(al3);          // exact doubling, integer pipe
        const double w1x = fma(-al3, rx, vx), w1y = fma(-al3, ry, vy), w1z = fma(-al3, rz, vz);
        const double w2x = fma(-be3, rx, fma(-al6, w1x, ax));
        const double w2y = fma(-be3, ry, fma(-al6, w1y, ay));
        const double w2z = fma(-be3, rz, fma(-al6, w1z, az));
        c.a[0] = fma(q, rx, c.a[0]); c.a[1] = fma(q, ry, c.a[1]); c.a[2] = fma(q, rz, c.a[2]);
        c.j[0] = fma(q, w1x, c.j[0]); c.j[1] = fma(q, w1y, c.j[1]); c.j[2] = fma(q, w1z, c.j[2]);
        c.s[0] = fma(q, w2x, c.s[0]); c.s[1] = fma(q, w2y, c.s[1]); c.s[2] = fma(q, w2z, c.s[2]);
    }
    // 4th-order pair term (Makino & Aarseth 1992): A0 = q r, A1 = q (v - 3 alpha r);
    // 29 FP64 instructions (31 with the 5-operation root, one more without
    // NB_FP64_POT_FF)
    static __device__ __forceinline__ void interact4(const I &i, const J &jj, bool self,
                                                     double eps2, float, Acc &c) {
        const double2 q0 = jj.q[0], q1 = jj.q[1], q2 = jj.q[2], q3 = jj.q[3];
        const double rx = sub(i, q0.x, i.x[0]), ry = sub(i, q0.y, i.x[1]), rz = sub(i, q1.x, i.x[2]);
        const double vx = sub(i, q2.x, i.v[0]), vy = sub(i, q2.y, i.v[1]), vz = sub(i, q3.x, i.v[2]);
        double r2 = fma(rx, rx, fma(ry, ry, fma(rz, rz, eps2)));
        double m = q1.y;
        r2 = self ? 1.0 : r2;
        m = self ? 0.0 : m;
        const double y = NB_FP64_RSQRT3 ? rsqrt_f64_3(r2, i.nz)
                         : (NB_FP64_ALL_FMA ? rsqrt_f64_fma(r2, i.nz) : rsqrt_f64(r2));
        const double y2 = mul(i, y, y);
        pot_term(jj, self, m, y, c);
        const double q = mul(i, mul(i, m, y2), y);
        const double rv = fma(rx, vx, fma(ry, vy, mul(i, rz, vz)));
        const double al3 = mul(i, 3.0, mul(i, rv, y2));
        const double w1x = fma(-al3, rx, vx), w1y = fma(-al3, ry, vy), w1z = fma(-al3, rz, vz);
        c.a[0] = fma(q, rx, c.a[0]); c.a[1] = fma(q, ry, c.a[1]); c.a[2] = fma(q, rz, c.a[2]);
        c.j[0] = fma(q, w1x, c.j[0]); c.j[1] = fma(q, w1y, c.j[1]); c.j[2] = fma(q, w1z, c.j[2]);
    }
    // pot-only pair term (energy diagnostics)
    static __device__ __forceinline__ void interact_pot(const I &i, const J &jj, bool self,
                                                        double eps2, Acc &c) {
        const double2 q0 = jj.q[0], q1 = jj.q[1];
        const double rx = q0.x - i.x[0], ry = q0.y - i.x[1], rz = q1.x - i.x[2];
        double r2 = fma(rx, rx, fma(ry, ry, fma(rz, rz, eps2)));
        double m = q1.y;
        r2 = self ? 1.0 : r2;
        m = self ? 0.0 : m;
        c.p = fma(m, rsqrt_f64(r2), c.p);
    }
    static __device__ __forceinline__ void finish(const Acc &c, const double *, int, double o[10]) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o[k] = c.a[k];
            o[3 + k] = c.j[k];
            o[6 + k] = c.s[k];
        }
#if NB_FP64_POT_FF
        o[9] = -(c.p + ((double)c.pf.hi + (double)c.pf.lo));
#else
        o[9] = -c.p;
#endif
    }
};

// ======================================================================= EX
// Float-float pair terms, two j per thread and step like the FP32 path: the
// record (JEXP) gives both particles' hi and lo parts as two-lane operands
// and every float-float primitive runs on float2 lanes (ff2).  Sums and
// products are kept unnormalised wherever the next operation only folds lo
// into first-order terms (the lazy forms); the accumulators are renormalised
// once per j-tile.
template <>
struct Prec<NB_EX> {
    using J = JEXP;
    static constexpr int kPerRec = 2;
    struct I {  // the i-particle, both lanes equal
        ff2 x[3], v[3], a[3];
    };
    struct Acc {  // lane l sums the j of parity l
        ff2 a[3], j[3], s[3], p;
    };
    static __device__ __forceinline__ ff2 dup(float hi, float lo) { return ff2{f2s(hi), f2s(lo)}; }
    static __device__ __forceinline__ I load_i(const J *jarr, int64_t k) {
        const float *f = reinterpret_cast<const float *>(jarr + (k >> 1)) + (k & 1);
        I r;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            r.x[q] = dup(f[2 * q], f[2 * (4 + q)]);
            r.v[q] = dup(f[2 * (8 + q)], f[2 * (12 + q)]);
        }
        r.a[0] = dup(f[2 * 11], f[2 * 15]);
        r.a[1] = dup(f[2 * 16], f[2 * 18]);
        r.a[2] = dup(f[2 * 17], f[2 * 19]);
        return r;
    }
    static __device__ __forceinline__ void zero(Acc &c) {
        const float2 z = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 3; ++k) c.a[k] = c.j[k] = c.s[k] = ff2{z, z};
        c.p = ff2{z, z};
    }
    // relative positions and velocities, normalised (after cancellation lo
    // can exceed hi)
    static __device__ __forceinline__ void rel(const I &i, const J &jj, ff2 r[3], ff2 v[3]) {
        const float4 q0 = jj.q[0], q1 = jj.q[1], q2 = jj.q[2], q3 = jj.q[3];
        const float4 q4 = jj.q[4], q5 = jj.q[5], q6 = jj.q[6], q7 = jj.q[7];
        r[0] = ff_sub(ff2{lo2(q0), lo2(q2)}, i.x[0]);
        r[1] = ff_sub(ff2{hi2(q0), hi2(q2)}, i.x[1]);
        r[2] = ff_sub(ff2{lo2(q1), lo2(q3)}, i.x[2]);
        v[0] = ff_sub(ff2{lo2(q4), lo2(q6)}, i.v[0]);
        v[1] = ff_sub(ff2{hi2(q4), hi2(q6)}, i.v[1]);
        v[2] = ff_sub(ff2{lo2(q5), lo2(q7)}, i.v[2]);
    }
    static __device__ __forceinline__ void exclude_self(bool self0, bool self1, ff2 &r2, ff2 &m) {
        r2.hi.x = self0 ? 1.f : r2.hi.x;  // selects, not arithmetic
        r2.lo.x = self0 ? 0.f : r2.lo.x;
        m.hi.x = self0 ? 0.f : m.hi.x;
        m.lo.x = self0 ? 0.f : m.lo.x;
        r2.hi.y = self1 ? 1.f : r2.hi.y;
        r2.lo.y = self1 ? 0.f : r2.lo.y;
        m.hi.y = self1 ? 0.f : m.hi.y;
        m.lo.y = self1 ? 0.f : m.lo.y;
    }
    static __device__ __forceinline__ void interact(const I &i, const J &jj, bool self0, bool self1,
                                                    ff2 eps2, Acc &c) {
        ff2 r[3], v[3], a[3];
        rel(i, jj, r, v);
        a[0] = ff_sub(ff2{hi2(jj.q[5]), hi2(jj.q[7])}, i.a[0]);
        a[1] = ff_sub(ff2{lo2(jj.q[8]), lo2(jj.q[9])}, i.a[1]);
        a[2] = ff_sub(ff2{hi2(jj.q[8]), hi2(jj.q[9])}, i.a[2]);
        ff2 r2 = ff_dot3_add_lazy(r, r, eps2);
        ff2 m{hi2(jj.q[1]), hi2(jj.q[3])};
        exclude_self(self0, self1, r2, m);
        const ff2 y = rsqrt_ff(r2);
        const ff2 rv = ff_dot3_lazy(r, v);
        const ff2 y2 = ff_sqr_lazy(y);
        const ff2 my = ff_mul_lazy(m, y);
        const ff2 q = ff_mul_lazy(my, y2);
        const ff2 w = ff_dot3x2_lazy(v, v, r, a);
        const ff2 al = ff_mul_lazy(rv, y2);
        const ff2 ze = ff_mul_lazy(w, y2);
        const ff2 al3 = ff_mul_f_lazy(al, f2s(3.0f));
        const ff2 be3 = ff_mul_f_lazy(ff_sum_lazy(ff_sqr_lazy(al), ze), f2s(3.0f));
        const ff2 al6 = ff2{add2(al3.hi, al3.hi), add2(al3.lo, al3.lo)};  // exact
        ff_add_lazy(c.p, my);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const ff2 w1 = ff_fnma_lazy(al3, r[k], v[k]);
            const ff2 w2 = ff_fnma_lazy(be3, r[k], ff_fnma_lazy(al6, w1, a[k]));
            ff_fma_acc_lazy(c.a[k], q, r[k]);
            ff_fma_acc_lazy(c.j[k], q, w1);
            ff_fma_acc_lazy(c.s[k], q, w2);
        }
    }
    static __device__ __forceinline__ void interact4(const I &i, const J &jj, bool self0, bool self1,
                                                     ff2 eps2, Acc &c) {
        ff2 r[3], v[3];
        rel(i, jj, r, v);
        ff2 r2 = ff_dot3_add(r, r, eps2);
        ff2 m{hi2(jj.q[1]), hi2(jj.q[3])};
        exclude_self(self0, self1, r2, m);
        const ff2 y = rsqrt_ff(r2);
        const ff2 y2 = ff_sqr_lazy(y);
        const ff2 my = ff_mul_lazy(m, y);
        const ff2 q = ff_mul_lazy(my, y2);
        const ff2 al3 = ff_mul_f_lazy(ff_mul_lazy(ff_dot3(r, v), y2), f2s(3.0f));
        ff_add_lazy(c.p, my);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const ff2 w1 = ff_fnma_lazy(al3, r[k], v[k]);
            ff_fma_acc_lazy(c.a[k], q, r[k]);
            ff_fma_acc_lazy(c.j[k], q, w1);
        }
    }
    // End of a j-tile: renormalise the lazily kept sums.
    static __device__ __forceinline__ void tile_done(Acc &c) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            c.a[k] = ff_renorm(c.a[k].hi, c.a[k].lo);
            c.j[k] = ff_renorm(c.j[k].hi, c.j[k].lo);
            c.s[k] = ff_renorm(c.s[k].hi, c.s[k].lo);
        }
        c.p = ff_renorm(c.p.hi, c.p.lo);
    }
    // both lanes' float-float sums as one double (each hi + lo is exact in
    // FP64; one rounding joins the lanes)
    static __device__ __forceinline__ double to_d(ff2 a) {
        return ((double)a.hi.x + (double)a.lo.x) + ((double)a.hi.y + (double)a.lo.y);
    }
    static __device__ __forceinline__ void finish(const Acc &c, const double *, int, double o[10]) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o[k] = to_d(c.a[k]);
            o[3 + k] = to_d(c.j[k]);
            o[6 + k] = to_d(c.s[k]);
        }
        o[9] = -to_d(c.p);
    }
};

// ===================================================================== FP32
// Two j per thread and step: the pair record (J32P) gives both particles'
// values as two-lane operands, and every add, multiply and FMA of the pair
// terms is one packed f32x2 instruction (per lane the same IEEE operations
// as the scalar form).  Lane l of every packed value belongs to particle
// 2 k + l of the tile.
template <>
struct Prec<NB_FP32> {
    using J = J32P;
    static constexpr int kPerRec = 2;  // particles per record
    struct I {  // the i-particle's values, both lanes equal
        float2 xh[3], xl[3], vh[3], vl[3], a[3];
    };
    // Two FP32 levels: per-tile sums (64 pairs, two lanes) are added into
    // chunk sums, which are promoted to FP64 every kFp32FlushTiles tiles.
    struct Acc {
        float2 a[3], j[3], s[3], p;
        float ca[3], cj[3], cs[3], cp;
    };
    static __device__ __forceinline__ I load_i(const J *jarr, int64_t k) {
        const float *f = reinterpret_cast<const float *>(jarr + (k >> 1)) + (k & 1);
        I r;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            r.xh[q] = f2s(f[2 * q]);
            r.xl[q] = f2s(f[2 * (4 + q)]);
            r.vh[q] = f2s(f[2 * (8 + q)]);
            r.vl[q] = f2s(f[2 * (12 + q)]);
            r.a[q] = f2s(f[2 * (7 + 4 * q)]);
        }
        return r;
    }
    static __device__ __forceinline__ void zero(Acc &c) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            c.a[k] = c.j[k] = c.s[k] = make_float2(0.f, 0.f);
            c.ca[k] = c.cj[k] = c.cs[k] = 0.f;
        }
        c.p = make_float2(0.f, 0.f);
        c.cp = 0.f;
    }
    // relative coordinates from the hi/lo split: (hi_j - hi_i) + (lo_j - lo_i)
    static __device__ __forceinline__ void rel(const I &i, const J &jj, float2 r[3], float2 v[3]) {
        const float4 q0 = jj.q[0], q1 = jj.q[1], q2 = jj.q[2], q3 = jj.q[3];
        const float4 q4 = jj.q[4], q5 = jj.q[5], q6 = jj.q[6], q7 = jj.q[7];
        r[0] = add2(sub2(lo2(q0), i.xh[0]), sub2(lo2(q2), i.xl[0]));
        r[1] = add2(sub2(hi2(q0), i.xh[1]), sub2(hi2(q2), i.xl[1]));
        r[2] = add2(sub2(lo2(q1), i.xh[2]), sub2(lo2(q3), i.xl[2]));
        v[0] = add2(sub2(lo2(q4), i.vh[0]), sub2(lo2(q6), i.vl[0]));
        v[1] = add2(sub2(hi2(q4), i.vh[1]), sub2(hi2(q6), i.vl[1]));
        v[2] = add2(sub2(lo2(q5), i.vh[2]), sub2(lo2(q7), i.vl[2]));
    }
    // 1/sqrt(r2) per lane: SFU value and one Newton step y (3/2 - r2 y^2 / 2)
    static __device__ __forceinline__ float2 rsqrt2(float2 r2) {
        float2 y;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y.x) : "f"(r2.x));
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y.y) : "f"(r2.y));
        const float2 t = mul2(mul2(f2s(-0.5f), r2), y);
        return mul2(y, fma2(t, y, f2s(1.5f)));
    }
    static __device__ __forceinline__ void interact(const I &i, const J &jj, bool self0, bool self1,
                                                    float2 eps2, Acc &c) {
        float2 r[3], v[3];
        rel(i, jj, r, v);
        const float2 ax = sub2(hi2(jj.q[3]), i.a[0]);
        const float2 ay = sub2(hi2(jj.q[5]), i.a[1]);
        const float2 az = sub2(hi2(jj.q[7]), i.a[2]);
        float2 r2 = fma2(r[0], r[0], fma2(r[1], r[1], fma2(r[2], r[2], eps2)));
        float2 m = hi2(jj.q[1]);
        r2.x = self0 ? 1.f : r2.x;  // selects, not arithmetic
        r2.y = self1 ? 1.f : r2.y;
        m.x = self0 ? 0.f : m.x;
        m.y = self1 ? 0.f : m.y;
        const float2 y = rsqrt2(r2);
        const float2 y2 = mul2(y, y);
        const float2 my = mul2(m, y);
        const float2 q = mul2(my, y2);
        c.p = add2(c.p, my);
        const float2 rv = fma2(r[0], v[0], fma2(r[1], v[1], mul2(r[2], v[2])));
        const float2 w = fma2(v[0], v[0], fma2(v[1], v[1], fma2(v[2], v[2],
                         fma2(r[0], ax, fma2(r[1], ay, mul2(r[2], az))))));
        const float2 al = mul2(rv, y2);
        const float2 ze = mul2(w, y2);
        const float2 nal3 = mul2(f2s(-3.f), al);              // -3 alpha
        const float2 nbe3 = mul2(f2s(-3.f), fma2(al, al, ze)); // -3 beta
        const float2 nal6 = add2(nal3, nal3);
        const float2 aa[3] = {ax, ay, az};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float2 w1 = fma2(nal3, r[k], v[k]);
            const float2 w2 = fma2(nbe3, r[k], fma2(nal6, w1, aa[k]));
            c.a[k] = fma2(q, r[k], c.a[k]);
            c.j[k] = fma2(q, w1, c.j[k]);
            c.s[k] = fma2(q, w2, c.s[k]);
        }
    }
    static __device__ __forceinline__ void interact4(const I &i, const J &jj, bool self0, bool self1,
                                                     float2 eps2, Acc &c) {
        float2 r[3], v[3];
        rel(i, jj, r, v);
        float2 r2 = fma2(r[0], r[0], fma2(r[1], r[1], fma2(r[2], r[2], eps2)));
        float2 m = hi2(jj.q[1]);
        r2.x = self0 ? 1.f : r2.x;
        r2.y = self1 ? 1.f : r2.y;
        m.x = self0 ? 0.f : m.x;
        m.y = self1 ? 0.f : m.y;
        const float2 y = rsqrt2(r2);
        const float2 y2 = mul2(y, y);
        const float2 my = mul2(m, y);
        const float2 q = mul2(my, y2);
        c.p = add2(c.p, my);
        const float2 nal3 =
            mul2(f2s(-3.f), mul2(fma2(r[0], v[0], fma2(r[1], v[1], mul2(r[2], v[2]))), y2));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float2 w1 = fma2(nal3, r[k], v[k]);
            c.a[k] = fma2(q, r[k], c.a[k]);
            c.j[k] = fma2(q, w1, c.j[k]);
        }
    }
    // End of a tile: add both lanes of the tile sums into the chunk sums.
    static __device__ __forceinline__ void tile_done(Acc &c) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            c.ca[k] += c.a[k].x + c.a[k].y;
            c.cj[k] += c.j[k].x + c.j[k].y;
            c.cs[k] += c.s[k].x + c.s[k].y;
            c.a[k] = c.j[k] = c.s[k] = make_float2(0.f, 0.f);
        }
        c.cp += c.p.x + c.p.y;
        c.p = make_float2(0.f, 0.f);
    }
    // Promote the FP32 chunk sums into the FP64 totals and restart them.
    // t64: the ten FP64 totals, element q at t64[q * st]
    static __device__ __forceinline__ void flush(Acc &c, double *t64, int st) {
        tile_done(c);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            t64[k * st] += (double)c.ca[k];
            t64[(3 + k) * st] += (double)c.cj[k];
            t64[(6 + k) * st] += (double)c.cs[k];
        }
        t64[9 * st] += (double)c.cp;
        zero(c);
    }
    static __device__ __forceinline__ void finish(Acc &c, double *t64, int st, double o[10]) {
        flush(c, t64, st);
#pragma unroll
        for (int k = 0; k < 9; ++k) o[k] = t64[k * st];
        o[9] = -t64[9 * st];
    }
};

// ==================================================================== FP32X
// The acceleration and the potential in float-float (the EX pair terms'
// arithmetic), jerk and snap in FP32 (the FP32 pair terms' arithmetic, on
// the float-float relative position and coefficients rounded to FP32): the
// 6th-order step criterion interpolates a^(3..5) from differences of the
// accelerations at both step ends over h^3..h^5 and needs the acceleration
// to about 1e-8, the jerk and snap only to about 1e-5.  Two j per thread and
// step on packed f32x2 lanes, from the EX records.
template <>
struct Prec<NB_FP32X> {
    using J = JEXP;
    static constexpr int kPerRec = 2;
    struct I {  // both lanes equal
        ff2 x[3];
        float2 vh[3], vl[3], a[3];
    };
    struct Acc {
        ff2 a[3], p;         // float-float sums, renormalised per j-tile
        float2 j[3], s[3];   // FP32 tile sums, lane l for the j of parity l
        float cj[3], cs[3];  // FP32 chunk sums, promoted to FP64 every kFp32FlushTiles tiles
    };
    static __device__ __forceinline__ I load_i(const J *jarr, int64_t k) {
        const float *f = reinterpret_cast<const float *>(jarr + (k >> 1)) + (k & 1);
        I r;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            r.x[q] = ff2{f2s(f[2 * q]), f2s(f[2 * (4 + q)])};
            r.vh[q] = f2s(f[2 * (8 + q)]);
            r.vl[q] = f2s(f[2 * (12 + q)]);
        }
        r.a[0] = f2s(f[2 * 11]);
        r.a[1] = f2s(f[2 * 16]);
        r.a[2] = f2s(f[2 * 17]);
        return r;
    }
    static __device__ __forceinline__ void zero(Acc &c) {
        const float2 z = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            c.a[k] = ff2{z, z};
            c.j[k] = c.s[k] = z;
            c.cj[k] = c.cs[k] = 0.f;
        }
        c.p = ff2{z, z};
    }
    // float-float relative positions (normalised), FP32 relative velocities
    // from the hi/lo split
    static __device__ __forceinline__ void rel(const I &i, const J &jj, ff2 r[3], float2 v[3]) {
        const float4 q0 = jj.q[0], q1 = jj.q[1], q2 = jj.q[2], q3 = jj.q[3];
        const float4 q4 = jj.q[4], q5 = jj.q[5], q6 = jj.q[6], q7 = jj.q[7];
        r[0] = ff_sub(ff2{lo2(q0), lo2(q2)}, i.x[0]);
        r[1] = ff_sub(ff2{hi2(q0), hi2(q2)}, i.x[1]);
        r[2] = ff_sub(ff2{lo2(q1), lo2(q3)}, i.x[2]);
        v[0] = add2(sub2(lo2(q4), i.vh[0]), sub2(lo2(q6), i.vl[0]));
        v[1] = add2(sub2(hi2(q4), i.vh[1]), sub2(hi2(q6), i.vl[1]));
        v[2] = add2(sub2(lo2(q5), i.vh[2]), sub2(lo2(q7), i.vl[2]));
    }
    // the float-float part: y, y^2 and q = m y^3; the sums of a and pot
    static __device__ __forceinline__ void acc_part(const ff2 r[3], ff2 r2, ff2 m, Acc &c, float2 &y2f,
                                                    float2 &qf) {
        const ff2 y = rsqrt_ff(r2);
        const ff2 y2 = ff_sqr_lazy(y);
        const ff2 my = ff_mul_lazy(m, y);
        const ff2 q = ff_mul_lazy(my, y2);
        ff_add_lazy(c.p, my);
#pragma unroll
        for (int k = 0; k < 3; ++k) ff_fma_acc_lazy(c.a[k], q, r[k]);
        y2f = y2.hi;  // the lazy pair's high part: the product rounded to FP32
        qf = q.hi;
    }
    static __device__ __forceinline__ void interact(const I &i, const J &jj, bool self0, bool self1,
                                                    ff2 eps2, Acc &c) {
        ff2 r[3];
        float2 v[3];
        rel(i, jj, r, v);
        const float2 aa[3] = {sub2(hi2(jj.q[5]), i.a[0]), sub2(lo2(jj.q[8]), i.a[1]),
                              sub2(hi2(jj.q[8]), i.a[2])};
        ff2 r2 = ff_dot3_add_lazy(r, r, eps2);
        ff2 m{hi2(jj.q[1]), hi2(jj.q[3])};
        Prec<NB_EX>::exclude_self(self0, self1, r2, m);
        float2 y2f, qf;
        acc_part(r, r2, m, c, y2f, qf);
        const float2 rf[3] = {r[0].hi, r[1].hi, r[2].hi};
        const float2 rv = fma2(rf[0], v[0], fma2(rf[1], v[1], mul2(rf[2], v[2])));
        const float2 w = fma2(v[0], v[0], fma2(v[1], v[1], fma2(v[2], v[2],
                         fma2(rf[0], aa[0], fma2(rf[1], aa[1], mul2(rf[2], aa[2]))))));
        const float2 al = mul2(rv, y2f);
        const float2 ze = mul2(w, y2f);
        const float2 nal3 = mul2(f2s(-3.f), al);
        const float2 nbe3 = mul2(f2s(-3.f), fma2(al, al, ze));
        const float2 nal6 = add2(nal3, nal3);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float2 w1 = fma2(nal3, rf[k], v[k]);
            const float2 w2 = fma2(nbe3, rf[k], fma2(nal6, w1, aa[k]));
            c.j[k] = fma2(qf, w1, c.j[k]);
            c.s[k] = fma2(qf, w2, c.s[k]);
        }
    }
    static __device__ __forceinline__ void interact4(const I &i, const J &jj, bool self0, bool self1,
                                                     ff2 eps2, Acc &c) {
        ff2 r[3];
        float2 v[3];
        rel(i, jj, r, v);
        ff2 r2 = ff_dot3_add_lazy(r, r, eps2);
        ff2 m{hi2(jj.q[1]), hi2(jj.q[3])};
        Prec<NB_EX>::exclude_self(self0, self1, r2, m);
        float2 y2f, qf;
        acc_part(r, r2, m, c, y2f, qf);
        const float2 rf[3] = {r[0].hi, r[1].hi, r[2].hi};
        const float2 nal3 =
            mul2(f2s(-3.f), mul2(fma2(rf[0], v[0], fma2(rf[1], v[1], mul2(rf[2], v[2]))), y2f));
#pragma unroll
        for (int k = 0; k < 3; ++k) c.j[k] = fma2(qf, fma2(nal3, rf[k], v[k]), c.j[k]);
    }
    // End of a j-tile: renormalise the float-float sums, add both lanes of
    // the FP32 tile sums into the chunk sums.
    static __device__ __forceinline__ void tile_done(Acc &c) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            c.a[k] = ff_renorm(c.a[k].hi, c.a[k].lo);
            c.cj[k] += c.j[k].x + c.j[k].y;
            c.cs[k] += c.s[k].x + c.s[k].y;
            c.j[k] = c.s[k] = make_float2(0.f, 0.f);
        }
        c.p = ff_renorm(c.p.hi, c.p.lo);
    }
    // Promote the FP32 chunk sums of jerk and snap into the FP64 totals
    // (t64[q * st], q = 3..8) and restart them.
    static __device__ __forceinline__ void flush(Acc &c, double *t64, int st) {
        tile_done(c);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            t64[(3 + k) * st] += (double)c.cj[k];
            t64[(6 + k) * st] += (double)c.cs[k];
            c.cj[k] = c.cs[k] = 0.f;
        }
    }
    static __device__ __forceinline__ void finish(Acc &c, double *t64, int st, double o[10]) {
        flush(c, t64, st);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o[k] = Prec<NB_EX>::to_d(c.a[k]);
            o[3 + k] = t64[(3 + k) * st];
            o[6 + k] = t64[(6 + k) * st];
        }
        o[9] = -Prec<NB_EX>::to_d(c.p);
    }
};

// ================================================================ kernel
// Per-arithmetic launch configuration of the evaluation kernel.
template <int P>
struct EvalCfg {
    static constexpr int stages = kStages;
    static constexpr int min_blocks = NB_EVAL_MIN_BLOCKS;
    static constexpr bool t64_smem = false;
};
template <>
struct EvalCfg<NB_EX> {
    static constexpr int stages = kStages;
    static constexpr int min_blocks = NB_EX_MIN_BLOCKS;
    static constexpr bool t64_smem = false;
};
// Resident CTAs per SM the compiler must allow for one kernel.  The packed EX
// pair terms of the 4th-order modes measured faster at 3 CTAs per SM (140
// registers: 1.16e11 against 1.10e11 pairs/s at 4 CTAs, N = 65536); the
// 6th-order ones are as fast at 4 (128 registers) as at 3 (166).
template <int P, int MODE>
constexpr int eval_min_blocks() {
    if constexpr (P == NB_EX && is_order4_mode(MODE)) return NB_EX4_MIN_BLOCKS;
    return EvalCfg<P>::min_blocks;
}
template <>
struct EvalCfg<NB_FP32> {
    static constexpr int stages = NB_FP32_STAGES;
    static constexpr int min_blocks = NB_FP32_MIN_BLOCKS;
    static constexpr bool t64_smem = NB_FP32_T64_SMEM != 0;
};
template <>
struct EvalCfg<NB_FP32X> {
    static constexpr int stages = kStages;
    static constexpr int min_blocks = NB_FP32X_MIN_BLOCKS;
    static constexpr bool t64_smem = true;
};

// One piece of work, described by thread 0 for the whole CTA.
struct PieceRec {
    long long item, item_end;  // current item / unit and the end of this CTA's work
    long long tb, te;          // j-tiles of the piece
    long long local, tile0, pslot0, off, nc, ntj;
    int c, gl, split, A, tile, sk;  // c < 0: no more work
};

template <int P>
struct SmemLayout {
    typename Prec<P>::J tile[EvalCfg<P>::stages][kTJ / Prec<P>::kPerRec];
    double red[10 * kTPB];  // cross-split reduction: group sums, then totals
    double t64[EvalCfg<P>::t64_smem ? 10 * kTPB : 1];  // FP32 totals, [q][thread]
    uint64_t bar[EvalCfg<P>::stages];
    PieceRec pc;
    int flag;
    int fail;
};

__device__ __forceinline__ int find_cluster(const ClusterPlan *plan, int nc, int64_t item) {
    int lo = 0, hi = nc - 1;  // largest c with plan[c].item0 <= item
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (plan[mid].item0 <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int P, int MODE>
__device__ __forceinline__ void finalize_one(const Dev &d, const EvalLaunch &L, int c, int64_t gi,
                                             int iloc, const double o[10]) {
    if constexpr (MODE == kModeOut || MODE == kModeOut4) {
        for (int q = 0; q < 10; ++q) L.out[(int64_t)q * L.n_active + iloc] = o[q];
    } else if constexpr (MODE == kModeStep) {
        correct_particle(d, gi, d.tnext[c], o);
    } else if constexpr (MODE == kModeStep4) {
        correct_particle4(d, gi, d.tnext[c], o);
    } else if constexpr (MODE == kModeInit1 || MODE == kModeInit2 || MODE == kModeInit4) {
        const int64_t n = d.n;
        for (int k = 0; k < 3; ++k) {
            d.a[k * n + gi] = o[k];
            d.j[k * n + gi] = o[3 + k];
            d.s[k * n + gi] = (MODE == kModeInit2) ? o[6 + k] : 0.0;
        }
        d.pot[gi] = o[9];
        // the 4th-order start-up has no snap: dt0 = eta_init |a| / |j|
        if constexpr (MODE != kModeInit1) d.dt[gi] = dt_start(d, o);
    } else {  // kModePot
        d.pot_tmp[gi] = o[9];
    }
}

// Units of a stream-K launch (one cluster): i-tiles x j-tiles (of the
// launch's j-range).
__device__ __forceinline__ int64_t sk_units(const Dev &d, const EvalLaunch &L) {
    const int c = L.direct ? L.cluster : 0;
    const int64_t tiles = L.direct ? L.tiles : d.plan[0].tiles;
    const int64_t ntj = cdiv(d.offsets[c + 1] - d.offsets[c], kTJ);
    return tiles * (L.direct ? (L.jt1 > 0 ? (int64_t)L.jt1 : ntj) - L.jt0 : ntj);
}

template <int P, int MODE>
__global__ void __launch_bounds__(kTPB, (eval_min_blocks<P, MODE>())) k_eval(const Dev d, const EvalLaunch L) {
    using T = Prec<P>;
    constexpr int kSt = EvalCfg<P>::stages;
    using J = typename T::J;
    constexpr int kRecs = kTJ / T::kPerRec;  // records per j-tile
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SmemLayout<P> &S = *reinterpret_cast<SmemLayout<P> *>(smem_raw);
    PieceRec &R = S.pc;
    const int tid = threadIdx.x;

    // Work: a stream-K launch (one cluster) gives CTA k the unit range
    // [U k / G, U (k+1) / G) and walks it piece by piece (one piece per i-tile
    // it touches).  Otherwise work items (cluster, i-tile, split index):
    // direct launches (equal-cost items of one cluster) take a static round
    // robin; planned launches fetch items dynamically, since clusters of a
    // batch give items of unequal cost.  Either way a piece's arithmetic and
    // the reduction order do not depend on the CTA that runs it.  Thread 0
    // keeps the piece's bookkeeping in shared memory, so that the pair loop
    // holds only what it uses in registers.
    if (tid == 0) {
        for (int s = 0; s < kSt; ++s) mbar_init(&S.bar[s], 1);
        S.fail = 0;
        fence_mbar_init();
        R.sk = L.direct ? L.streamk != 0 : (d.n_clusters == 1 && d.plan[0].streamk != 0);
        if (R.sk) {
            R.item = sk_begin(sk_units(d, L), gridDim.x, blockIdx.x);
            R.item_end = sk_begin(sk_units(d, L), gridDim.x, blockIdx.x + 1);
        } else {
            R.item_end = L.direct ? (int64_t)L.tiles * L.split : *d.n_items;
            R.item = L.direct ? (int64_t)blockIdx.x : (long long)atomicAdd(d.item_ctr, 1ull);
        }
    }
    uint32_t phase = 0;   // bit s: parity of stage s
    uint32_t pending = 0; // bit s: a copy into stage s is in flight

    for (;;) {
        // thread 0: describe the current piece (or the end of the work)
        if (tid == 0) {
            const int64_t item = R.item;
            if (item >= R.item_end) {
                R.c = -1;
            } else {
                int c, gl, split, A;
                int64_t item0, tile0, pslot0;
                if (L.direct) {
                    c = L.cluster; gl = L.gl; split = L.split; A = L.n_active; item0 = 0; tile0 = 0;
                    pslot0 = 0;
                } else {
                    c = R.sk ? 0 : find_cluster(d.plan, d.n_clusters, item);
                    const ClusterPlan pl = d.plan[c];
                    gl = pl.gl; split = pl.split; A = pl.active; item0 = pl.item0; tile0 = pl.tile0;
                    pslot0 = pl.pslot0;
                }
                const int64_t off = d.offsets[c];
                const int64_t nc = d.offsets[c + 1] - off;
                // the j-tiles this launch covers: all of the cluster's, or a
                // host-given range [jt0, jt0 + ntj) of them (direct launches)
                const int64_t jt0 = L.direct ? L.jt0 : 0;
                const int64_t ntj = (L.direct && L.jt1 > 0 ? (int64_t)L.jt1 : cdiv(nc, kTJ)) - jt0;
                int tile;
                int64_t tb, te, local = 0;
                if (R.sk) {
                    tile = (int)(item / ntj);
                    tb = item - (int64_t)tile * ntj;
                    te = min(ntj, tb + (int64_t)(R.item_end - item));
                } else {
                    local = item - item0;
                    tile = (int)(local / split);
                    const int sidx = (int)(local % split);
                    tb = ntj * sidx / split;
                    te = ntj * (sidx + 1) / split;
                }
                tb += jt0;
                te += jt0;
                R.c = c; R.gl = gl; R.split = split; R.A = A; R.tile = tile;
                R.tile0 = tile0; R.pslot0 = pslot0; R.local = local;
                R.off = off; R.nc = nc; R.ntj = ntj; R.tb = tb; R.te = te;
            }
        }
        __syncthreads();
        if (R.c < 0) break;

        const int c = R.c;
        const int gl = R.gl;
        const int64_t tb = R.tb, te = R.te;
        const int ilane = tid / gl;
        const int jsub = tid % gl;
        const bool valid = R.tile * (kTPB / gl) + ilane < R.A;
        const J *jc = reinterpret_cast<const J *>(d.jarr) + d.jofs[c] / T::kPerRec;
        // this thread's i: global index, bounds-checked against its cluster
        auto i_of = [&](int il, bool &bad) -> int64_t {
            const int64_t off = R.off;
            int64_t g;
            if (L.identity) g = off + il;
            else if (L.direct) g = L.active[il];
            else g = d.active[off + il];
            bad = g < off || g >= off + R.nc;
            return bad ? off : g;
        };
        int64_t ji = 0;
        if (valid) {
            bool bad;
            ji = i_of(R.tile * (kTPB / gl) + ilane, bad) - R.off;
            if (bad) atomicOr(d.err, kErrIndex);  // caller-given index outside the cluster
        }
        typename T::I me = T::load_i(jc, ji);
        if constexpr (P == NB_FP64) T::prepare(me, d);
        typename T::Acc acc;
        T::zero(acc);
        double t64r[EvalCfg<P>::t64_smem ? 1 : 10];
        double *t64 = EvalCfg<P>::t64_smem ? S.t64 + tid : t64r;
        constexpr int t64st = EvalCfg<P>::t64_smem ? kTPB : 1;
#pragma unroll
        for (int q = 0; q < 10; ++q) t64[q * t64st] = 0.0;
        const double eps2 = d.eps2;
        const float eps2f = (float)eps2;
        const float2 eps2f2 = d.eps2_hi2;
        const ff2 eps2ff2{d.eps2_hi2, d.eps2_lo2};

        const bool warp_active = __any_sync(0xffffffffu, valid);

        // prologue: fill the ring
        if (tid == 0) {
            for (int s = 0; s < kSt && tb + s < te; ++s) {
                mbar_expect_tx(&S.bar[s], kRecs * sizeof(J));
                tma_load_1d(&S.tile[s][0], jc + (tb + s) * kRecs, kRecs * sizeof(J), &S.bar[s]);
                pending |= 1u << s;
            }
        }
        bool ok = true;
        for (int64_t tt = tb; tt < te; ++tt) {
            const int s = (int)((tt - tb) % kSt);
            if (ok) ok = mbar_wait_bounded(&S.bar[s], (phase >> s) & 1u);
            phase ^= 1u << s;
            if (ok && warp_active) {
                const J *tl = &S.tile[s][0];
                const int64_t jbase = tt * kTJ;
                if constexpr (MODE == kModePot) {
                    for (int k = jsub; k < kTJ; k += gl)
                        T::interact_pot(me, tl[k], jbase + k == ji, eps2, acc);
                } else if constexpr (P == NB_FP32 && uses_order4_terms(MODE)) {
                    // record k holds particles 2k and 2k + 1 of the tile
#pragma unroll kEvalUnroll
                    for (int k = jsub; k < kRecs; k += gl)
                        T::interact4(me, tl[k], jbase + 2 * k == ji, jbase + 2 * k + 1 == ji,
                                     eps2f2, acc);
                } else if constexpr (P == NB_FP32) {
#pragma unroll kEvalUnroll
                    for (int k = jsub; k < kRecs; k += gl)
                        T::interact(me, tl[k], jbase + 2 * k == ji, jbase + 2 * k + 1 == ji,
                                    eps2f2, acc);
                } else if constexpr (P == NB_FP32X && uses_order4_terms(MODE)) {
#pragma unroll 1
                    for (int k = jsub; k < kRecs; k += gl)
                        T::interact4(me, tl[k], jbase + 2 * k == ji, jbase + 2 * k + 1 == ji,
                                     eps2ff2, acc);
                } else if constexpr (P == NB_FP32X) {
#pragma unroll 1
                    for (int k = jsub; k < kRecs; k += gl)
                        T::interact(me, tl[k], jbase + 2 * k == ji, jbase + 2 * k + 1 == ji,
                                    eps2ff2, acc);
                } else if constexpr (P == NB_EX && uses_order4_terms(MODE)) {
#pragma unroll 1
                    for (int k = jsub; k < kRecs; k += gl)
                        T::interact4(me, tl[k], jbase + 2 * k == ji, jbase + 2 * k + 1 == ji,
                                     eps2ff2, acc);
                } else if constexpr (P == NB_EX) {
#pragma unroll 1
                    for (int k = jsub; k < kRecs; k += gl)
                        T::interact(me, tl[k], jbase + 2 * k == ji, jbase + 2 * k + 1 == ji,
                                    eps2ff2, acc);
                } else if constexpr (uses_order4_terms(MODE)) {
#pragma unroll kEvalUnroll
                    for (int k = jsub; k < kTJ; k += gl)
                        T::interact4(me, tl[k], jbase + k == ji, eps2, eps2f, acc);
                } else {
#pragma unroll kEvalUnroll
                    for (int k = jsub; k < kTJ; k += gl)
                        T::interact(me, tl[k], jbase + k == ji, eps2, eps2f, acc);
                }
                if constexpr (P == NB_FP32 || P == NB_FP32X) {
                    if ((tt - tb + 1) % kFp32FlushTiles == 0) T::flush(acc, t64, t64st);
                    else T::tile_done(acc);
                } else if constexpr (P == NB_EX && MODE != kModePot) {
                    T::tile_done(acc);
                } else if constexpr (P == NB_FP64 && NB_FP64_POT_FF && MODE != kModePot) {
                    T::tile_done(acc);
                }
            }
            if (!ok) S.fail = 1;
            __syncthreads();
            if (S.fail) break;
            if (tid == 0) {
                pending &= ~(1u << s);
                if (tt + kSt < te) {
                    mbar_expect_tx(&S.bar[s], kRecs * sizeof(J));
                    tma_load_1d(&S.tile[s][0], jc + (tt + kSt) * kRecs, kRecs * sizeof(J), &S.bar[s]);
                    pending |= 1u << s;
                }
            }
        }
        if (S.fail) {
            // a copy did not land in time: record it, drain (bounded) what this
            // CTA still has in flight, and leave the kernel
            if (tid == 0) {
                atomicOr(d.err, kErrTimeout);
                for (int s = 0; s < kSt; ++s)
                    if (pending & (1u << s)) (void)mbar_wait_bounded(&S.bar[s], (phase >> s) & 1u);
            }
            return;
        }

        double o[10];
        T::finish(acc, t64, t64st, o);
        // lanes sharing an i: butterfly sum (fixed order)
        for (int w = gl >> 1; w >= 1; w >>= 1) {
#pragma unroll
            for (int q = 0; q < 10; ++q) o[q] += __shfl_xor_sync(0xffffffffu, o[q], w);
        }

        // ---- epilogue: the piece's bookkeeping comes back from shared memory
        const int tile = R.tile, A = R.A, split = R.split;
        const int Ti = kTPB / gl;
        const int64_t ntj = R.ntj;
        const bool sk = R.sk;
        // pieces of this i-tile: split items, or the CTAs whose ranges meet it
        int npieces = split;
        int64_t sk_first = 0, sk_maxp = 0, sk_loc0 = 0;
        if (sk) {
            const int64_t U = sk_units(d, L);
            sk_first = sk_owner(U, gridDim.x, (int64_t)tile * ntj);
            npieces = (int)(sk_owner(U, gridDim.x, (int64_t)(tile + 1) * ntj - 1) - sk_first + 1);
            sk_maxp = sk_max_pieces(U, gridDim.x, ntj);
            // the first piece's CTA may have started in an earlier i-tile; the
            // others start inside this one (their local tile index is 0)
            sk_loc0 = tile - sk_begin(U, gridDim.x, sk_first) / ntj;
        }
        const int64_t pslot0 = R.pslot0;
        // partial-sum slot (doubles) of piece s of this tile: CTA k keeps one
        // slot per i-tile its range touches
        auto piece_slot = [&](int64_t s) -> int64_t {
            if (sk) return ((sk_first + s) * sk_maxp + (s == 0 ? sk_loc0 : 0)) * (10 * Ti);
            return pslot0 + ((int64_t)tile * split + s) * (10 * Ti);
        };
        if (npieces == 1) {
            if (valid && jsub == 0) {
                bool bad;
                const int il = tile * Ti + ilane;
                const int64_t gi = i_of(il, bad);
                if (!bad) finalize_one<P, MODE>(d, L, c, gi, il, o);
            }
        } else {
            // this CTA's piece of the tile
            double *part = d.partial + (sk ? piece_slot((int64_t)blockIdx.x - sk_first)
                                           : pslot0 + R.local * (int64_t)(10 * Ti));
            if (jsub == 0) {
#pragma unroll
                for (int q = 0; q < 10; ++q) part[q * Ti + ilane] = o[q];
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) {
                const int prev = atomicAdd(&d.tile_cnt[R.tile0 + tile], 1);
                S.flag = (prev == npieces - 1);
            }
            __syncthreads();
            if (S.flag) {
                // Last CTA of this i-tile: add the partials of its pieces for
                // every (i, q) pair in two fixed-order levels.  Level 1: thread
                // (p, r) sums the r-th contiguous group of pieces of pair p in
                // piece order; level 2 adds the R group sums in group order.  The
                // order depends only on (pieces, valid i count), so results are
                // reproducible.
                __threadfence();
                const int nv = min(Ti, A - tile * Ti);     // valid i in this tile
                const int npair = nv * 10;
                const int Rg = max(1, kTPB / npair);
                for (int w = tid; w < npair * Rg; w += kTPB) {
                    const int p = w % npair, r = w / npair;
                    const int q = p / nv, il = p % nv;
                    const int s0 = (int)((int64_t)npieces * r / Rg), s1 = (int)((int64_t)npieces * (r + 1) / Rg);
                    double acc2 = 0.0;
                    if (sk) {
                        for (int sp = s0; sp < s1; ++sp) acc2 += __ldcg(d.partial + piece_slot(sp) + q * Ti + il);
                    } else {
                        const double *base = d.partial + piece_slot(0);
#pragma unroll 4
                        for (int sp = s0; sp < s1; ++sp) acc2 += __ldcg(base + (int64_t)sp * (10 * Ti) + q * Ti + il);
                    }
                    S.red[r * npair + p] = acc2;
                }
                __syncthreads();
                if (tid < nv) {
                    double sum[10];
#pragma unroll
                    for (int q = 0; q < 10; ++q) {
                        double a2 = 0.0;
                        for (int r = 0; r < Rg; ++r) a2 += S.red[r * npair + q * nv + tid];
                        sum[q] = a2;
                    }
                    const int il = tile * Ti + tid;
                    bool bad;
                    const int64_t g2 = i_of(il, bad);
                    if (!bad) finalize_one<P, MODE>(d, L, c, g2, il, sum);
                }
                if (tid == 0) d.tile_cnt[R.tile0 + tile] = 0;
            }
        }
        // next piece: every thread is done with this piece's record
        __syncthreads();
        if (tid == 0) {
            if (R.sk) R.item += R.te - R.tb;
            else if (L.direct) R.item += gridDim.x;
            else R.item = (long long)atomicAdd(d.item_ctr, 1ull);
        }
    }
}

template <int P, int MODE>
cudaError_t launch_eval_t(const Dev &d, const EvalLaunch &L, int grid, cudaStream_t st) {
    const size_t smem = sizeof(SmemLayout<P>);  // < 48 KB: no opt-in attribute needed
    static_assert(sizeof(SmemLayout<P>) <= 48 * 1024, "evaluation tile ring exceeds 48 KB");
    k_eval<P, MODE><<<grid, kTPB, smem, st>>>(d, L);
    return cudaGetLastError();
}

template <int P, int MODE>
int occupancy_t() {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_eval<P, MODE>, kTPB, sizeof(SmemLayout<P>));
    return b;
}

}  // namespace nb

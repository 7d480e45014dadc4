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
// 52 FP64 instructions per pair on the FP64 path (one exact doubling is done
// on the integer pipe; the potential m y is summed in float-float on the FP32
// pipe, NB_FP64_POT_FF).  The 4th-order scheme (Makino & Aarseth 1992) keeps
// A0, A1 and the potential only (interact4: 31 FP64 instructions per pair).
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
        const double y = NB_FP64_ALL_FMA ? rsqrt_f64_fma(r2, i.nz) : rsqrt_f64(r2);
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
    // 31 FP64 instructions (32 without NB_FP64_POT_FF)
    static __device__ __forceinline__ void interact4(const I &i, const J &jj, bool self,
                                                     double eps2, float, Acc &c) {
        const double2 q0 = jj.q[0], q1 = jj.q[1], q2 = jj.q[2], q3 = jj.q[3];
        const double rx = sub(i, q0.x, i.x[0]), ry = sub(i, q0.y, i.x[1]), rz = sub(i, q1.x, i.x[2]);
        const double vx = sub(i, q2.x, i.v[0]), vy = sub(i, q2.y, i.v[1]), vz = sub(i, q3.x, i.v[2]);
        double r2 = fma(rx, rx, fma(ry, ry, fma(rz, rz, eps2)));
        double m = q1.y;
        r2 = self ? 1.0 : r2;
        m = self ? 0.0 : m;
        const double y = NB_FP64_ALL_FMA ? rsqrt_f64_fma(r2, i.nz) : rsqrt_f64(r2);
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
template <>
struct Prec<NB_EX> {
    using J = JEX;
    struct I {
        ff x[3], v[3], a[3];
    };
    struct Acc {
        ff a[3], j[3], s[3], p;
    };
    static __device__ __forceinline__ I load_i(const J *jarr, int64_t k) {
        const J e = jarr[k];
        I r;
        r.x[0] = ff{e.q[0].x, e.q[1].x}; r.x[1] = ff{e.q[0].y, e.q[1].y}; r.x[2] = ff{e.q[0].z, e.q[1].z};
        r.v[0] = ff{e.q[2].x, e.q[3].x}; r.v[1] = ff{e.q[2].y, e.q[3].y}; r.v[2] = ff{e.q[2].z, e.q[3].z};
        r.a[0] = ff{e.q[2].w, e.q[3].w}; r.a[1] = ff{e.q[4].x, e.q[4].z}; r.a[2] = ff{e.q[4].y, e.q[4].w};
        return r;
    }
    static __device__ __forceinline__ void zero(Acc &c) {
#pragma unroll
        for (int k = 0; k < 3; ++k) c.a[k] = c.j[k] = c.s[k] = ff{0.f, 0.f};
        c.p = ff{0.f, 0.f};
    }
    static __device__ __forceinline__ void interact(const I &i, const J &jj, bool self, double,
                                                    float, Acc &c, ff eps2) {
        const float4 q0 = jj.q[0], q1 = jj.q[1], q2 = jj.q[2], q3 = jj.q[3], q4 = jj.q[4];
        ff r[3], v[3], a[3];
        r[0] = ff_sub(ff{q0.x, q1.x}, i.x[0]);
        r[1] = ff_sub(ff{q0.y, q1.y}, i.x[1]);
        r[2] = ff_sub(ff{q0.z, q1.z}, i.x[2]);
        v[0] = ff_sub(ff{q2.x, q3.x}, i.v[0]);
        v[1] = ff_sub(ff{q2.y, q3.y}, i.v[1]);
        v[2] = ff_sub(ff{q2.z, q3.z}, i.v[2]);
        a[0] = ff_sub(ff{q2.w, q3.w}, i.a[0]);
        a[1] = ff_sub(ff{q4.x, q4.z}, i.a[1]);
        a[2] = ff_sub(ff{q4.y, q4.w}, i.a[2]);
        ff r2 = NB_EX_LAZY ? ff_dot3_add_lazy(r, r, eps2) : ff_add(ff_dot3(r, r), eps2);
        ff m = ff{q0.w, q1.w};
        if (self) {
            r2 = ff{1.f, 0.f};
            m = ff{0.f, 0.f};
        }
        const ff y = rsqrt_ff(r2);
        const ff rv = NB_EX_LAZY ? ff_dot3_lazy(r, v) : ff_dot3(r, v);
        ff y2, my, q, w, al, ze, al3, be3;
        if constexpr (NB_EX_LAZY) {
            y2 = ff_sqr_lazy(y);
            my = ff_mul_lazy(m, y);
            q = ff_mul_lazy(my, y2);
            w = ff_dot3x2_lazy(v, v, r, a);
            al = ff_mul_lazy(rv, y2);
            ze = ff_mul_lazy(w, y2);
            al3 = ff_mul_f_lazy(al, 3.0f);
            be3 = ff_mul_f_lazy(ff_sum_lazy(ff_sqr_lazy(al), ze), 3.0f);
        } else {
            y2 = ff_sqr(y);
            my = ff_mul(m, y);
            q = ff_mul(my, y2);
            w = ff_add(ff_dot3(v, v), ff_dot3(r, a));
            al = ff_mul(rv, y2);
            ze = ff_mul(w, y2);
            al3 = ff_mul_f(al, 3.0f);
            be3 = ff_mul_f(ff_add(ff_sqr(al), ze), 3.0f);
        }
        const ff al6 = ff{2.0f * al3.hi, 2.0f * al3.lo};  // exact
        if constexpr (NB_EX_LAZY) {
            ff_add_lazy(c.p, my);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const ff w1 = ff_fnma_lazy(al3, r[k], v[k]);
                const ff w2 = ff_fnma_lazy(be3, r[k], ff_fnma_lazy(al6, w1, a[k]));
                ff_fma_acc_lazy(c.a[k], q, r[k]);
                ff_fma_acc_lazy(c.j[k], q, w1);
                ff_fma_acc_lazy(c.s[k], q, w2);
            }
        } else {
            c.p = ff_add(c.p, my);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const ff w1 = ff_fnma(al3, r[k], v[k]);
                const ff w2 = ff_fnma(be3, r[k], ff_fnma(al6, w1, a[k]));
                ff_fma_acc(c.a[k], q, r[k]);
                ff_fma_acc(c.j[k], q, w1);
                ff_fma_acc(c.s[k], q, w2);
            }
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
    static __device__ __forceinline__ void interact4(const I &i, const J &jj, bool self, double,
                                                     float, Acc &c, ff eps2) {
        const float4 q0 = jj.q[0], q1 = jj.q[1], q2 = jj.q[2], q3 = jj.q[3];
        ff r[3], v[3];
        r[0] = ff_sub(ff{q0.x, q1.x}, i.x[0]);
        r[1] = ff_sub(ff{q0.y, q1.y}, i.x[1]);
        r[2] = ff_sub(ff{q0.z, q1.z}, i.x[2]);
        v[0] = ff_sub(ff{q2.x, q3.x}, i.v[0]);
        v[1] = ff_sub(ff{q2.y, q3.y}, i.v[1]);
        v[2] = ff_sub(ff{q2.z, q3.z}, i.v[2]);
        ff r2 = NB_EX_LAZY ? ff_dot3_add(r, r, eps2) : ff_add(ff_dot3(r, r), eps2);
        ff m = ff{q0.w, q1.w};
        if (self) {
            r2 = ff{1.f, 0.f};
            m = ff{0.f, 0.f};
        }
        const ff y = rsqrt_ff(r2);
        const ff y2 = NB_EX_LAZY ? ff_sqr_lazy(y) : ff_sqr(y);
        const ff my = NB_EX_LAZY ? ff_mul_lazy(m, y) : ff_mul(m, y);
        const ff q = NB_EX_LAZY ? ff_mul_lazy(my, y2) : ff_mul(my, y2);
        const ff al3 = NB_EX_LAZY ? ff_mul_f_lazy(ff_mul_lazy(ff_dot3(r, v), y2), 3.0f)
                                  : ff_mul_f(ff_mul(ff_dot3(r, v), y2), 3.0f);
        if constexpr (NB_EX_LAZY) {
            ff_add_lazy(c.p, my);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const ff w1 = ff_fnma_lazy(al3, r[k], v[k]);
                ff_fma_acc_lazy(c.a[k], q, r[k]);
                ff_fma_acc_lazy(c.j[k], q, w1);
            }
        } else {
            c.p = ff_add(c.p, my);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const ff w1 = ff_fnma(al3, r[k], v[k]);
                ff_fma_acc(c.a[k], q, r[k]);
                ff_fma_acc(c.j[k], q, w1);
            }
        }
    }
    static __device__ __forceinline__ double to_d(ff a) { return (double)a.hi + (double)a.lo; }
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
template <>
struct Prec<NB_FP32> {
    using J = J32;
    struct I {
        float xh[3], xl[3], vh[3], vl[3], a[3];
    };
    // Two FP32 levels: per-tile sums (64 pairs) are added into chunk sums,
    // which are promoted to FP64 every kFp32FlushTiles tiles.
    struct Acc {
        float a[3], j[3], s[3], p;
        float ca[3], cj[3], cs[3], cp;
    };
    static __device__ __forceinline__ I load_i(const J *jarr, int64_t k) {
        const J e = jarr[k];
        I r;
        r.xh[0] = e.q[0].x; r.xh[1] = e.q[0].y; r.xh[2] = e.q[0].z;
        r.xl[0] = e.q[1].x; r.xl[1] = e.q[1].y; r.xl[2] = e.q[1].z;
        r.vh[0] = e.q[2].x; r.vh[1] = e.q[2].y; r.vh[2] = e.q[2].z;
        r.vl[0] = e.q[3].x; r.vl[1] = e.q[3].y; r.vl[2] = e.q[3].z;
        r.a[0] = e.q[1].w; r.a[1] = e.q[2].w; r.a[2] = e.q[3].w;
        return r;
    }
    static __device__ __forceinline__ void zero(Acc &c) {
#pragma unroll
        for (int k = 0; k < 3; ++k) c.a[k] = c.j[k] = c.s[k] = c.ca[k] = c.cj[k] = c.cs[k] = 0.f;
        c.p = c.cp = 0.f;
    }
    static __device__ __forceinline__ void interact(const I &i, const J &jj, bool self, double,
                                                    float eps2, Acc &c) {
        const float4 q0 = jj.q[0], q1 = jj.q[1], q2 = jj.q[2], q3 = jj.q[3];
        // relative coordinates from the hi/lo split: (hi_j - hi_i) + (lo_j - lo_i)
        const float rx = (q0.x - i.xh[0]) + (q1.x - i.xl[0]);
        const float ry = (q0.y - i.xh[1]) + (q1.y - i.xl[1]);
        const float rz = (q0.z - i.xh[2]) + (q1.z - i.xl[2]);
        const float vx = (q2.x - i.vh[0]) + (q3.x - i.vl[0]);
        const float vy = (q2.y - i.vh[1]) + (q3.y - i.vl[1]);
        const float vz = (q2.z - i.vh[2]) + (q3.z - i.vl[2]);
        const float ax = q1.w - i.a[0], ay = q2.w - i.a[1], az = q3.w - i.a[2];
        float r2 = fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, eps2)));
        float m = q0.w;
        r2 = self ? 1.f : r2;
        m = self ? 0.f : m;
        float y;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r2));
        const float hr2 = 0.5f * r2;             // one Newton step on the SFU value
        y = y * fmaf(-hr2 * y, y, 1.5f);
        const float y2 = y * y;
        const float my = m * y;
        const float q = my * y2;
        c.p += my;
        const float rv = fmaf(rx, vx, fmaf(ry, vy, rz * vz));
        const float w = fmaf(vx, vx, fmaf(vy, vy, fmaf(vz, vz, fmaf(rx, ax, fmaf(ry, ay, rz * az)))));
        const float al = rv * y2;
        const float ze = w * y2;
        const float al3 = 3.f * al;
        const float be3 = 3.f * fmaf(al, al, ze);
        const float al6 = al3 + al3;
        const float w1x = fmaf(-al3, rx, vx), w1y = fmaf(-al3, ry, vy), w1z = fmaf(-al3, rz, vz);
        const float w2x = fmaf(-be3, rx, fmaf(-al6, w1x, ax));
        const float w2y = fmaf(-be3, ry, fmaf(-al6, w1y, ay));
        const float w2z = fmaf(-be3, rz, fmaf(-al6, w1z, az));
        c.a[0] = fmaf(q, rx, c.a[0]); c.a[1] = fmaf(q, ry, c.a[1]); c.a[2] = fmaf(q, rz, c.a[2]);
        c.j[0] = fmaf(q, w1x, c.j[0]); c.j[1] = fmaf(q, w1y, c.j[1]); c.j[2] = fmaf(q, w1z, c.j[2]);
        c.s[0] = fmaf(q, w2x, c.s[0]); c.s[1] = fmaf(q, w2y, c.s[1]); c.s[2] = fmaf(q, w2z, c.s[2]);
    }
    static __device__ __forceinline__ void interact4(const I &i, const J &jj, bool self, double,
                                                     float eps2, Acc &c) {
        const float4 q0 = jj.q[0], q1 = jj.q[1], q2 = jj.q[2], q3 = jj.q[3];
        const float rx = (q0.x - i.xh[0]) + (q1.x - i.xl[0]);
        const float ry = (q0.y - i.xh[1]) + (q1.y - i.xl[1]);
        const float rz = (q0.z - i.xh[2]) + (q1.z - i.xl[2]);
        const float vx = (q2.x - i.vh[0]) + (q3.x - i.vl[0]);
        const float vy = (q2.y - i.vh[1]) + (q3.y - i.vl[1]);
        const float vz = (q2.z - i.vh[2]) + (q3.z - i.vl[2]);
        float r2 = fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, eps2)));
        float m = q0.w;
        r2 = self ? 1.f : r2;
        m = self ? 0.f : m;
        float y;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r2));
        const float hr2 = 0.5f * r2;
        y = y * fmaf(-hr2 * y, y, 1.5f);
        const float y2 = y * y;
        const float my = m * y;
        const float q = my * y2;
        c.p += my;
        const float al3 = 3.f * (fmaf(rx, vx, fmaf(ry, vy, rz * vz)) * y2);
        const float w1x = fmaf(-al3, rx, vx), w1y = fmaf(-al3, ry, vy), w1z = fmaf(-al3, rz, vz);
        c.a[0] = fmaf(q, rx, c.a[0]); c.a[1] = fmaf(q, ry, c.a[1]); c.a[2] = fmaf(q, rz, c.a[2]);
        c.j[0] = fmaf(q, w1x, c.j[0]); c.j[1] = fmaf(q, w1y, c.j[1]); c.j[2] = fmaf(q, w1z, c.j[2]);
    }
    // End of a tile: add the tile sums into the chunk sums.
    static __device__ __forceinline__ void tile_done(Acc &c) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            c.ca[k] += c.a[k]; c.cj[k] += c.j[k]; c.cs[k] += c.s[k];
            c.a[k] = c.j[k] = c.s[k] = 0.f;
        }
        c.cp += c.p;
        c.p = 0.f;
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
template <>
struct EvalCfg<NB_FP32> {
    static constexpr int stages = NB_FP32_STAGES;
    static constexpr int min_blocks = NB_FP32_MIN_BLOCKS;
    static constexpr bool t64_smem = NB_FP32_T64_SMEM != 0;
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
    typename Prec<P>::J tile[EvalCfg<P>::stages][kTJ];
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

// Units of a stream-K launch (one cluster): i-tiles x j-tiles.
__device__ __forceinline__ int64_t sk_units(const Dev &d, const EvalLaunch &L) {
    const int c = L.direct ? L.cluster : 0;
    const int64_t tiles = L.direct ? L.tiles : d.plan[0].tiles;
    return tiles * cdiv(d.offsets[c + 1] - d.offsets[c], kTJ);
}

template <int P, int MODE>
__global__ void __launch_bounds__(kTPB, EvalCfg<P>::min_blocks) k_eval(const Dev d, const EvalLaunch L) {
    using T = Prec<P>;
    constexpr int kSt = EvalCfg<P>::stages;
    using J = typename T::J;
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
                const int64_t ntj = cdiv(nc, kTJ);
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
        const J *jc = reinterpret_cast<const J *>(d.jarr) + d.jofs[c];
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
        ff eps2ff;
        eps2ff.hi = (float)eps2;
        eps2ff.lo = (float)(eps2 - (double)eps2ff.hi);

        const bool warp_active = __any_sync(0xffffffffu, valid);

        // prologue: fill the ring
        if (tid == 0) {
            for (int s = 0; s < kSt && tb + s < te; ++s) {
                mbar_expect_tx(&S.bar[s], kTJ * sizeof(J));
                tma_load_1d(&S.tile[s][0], jc + (tb + s) * kTJ, kTJ * sizeof(J), &S.bar[s]);
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
                } else if constexpr (P == NB_EX && uses_order4_terms(MODE)) {
#pragma unroll 1
                    for (int k = jsub; k < kTJ; k += gl)
                        T::interact4(me, tl[k], jbase + k == ji, eps2, eps2f, acc, eps2ff);
                } else if constexpr (P == NB_EX) {
#pragma unroll 1
                    for (int k = jsub; k < kTJ; k += gl)
                        T::interact(me, tl[k], jbase + k == ji, eps2, eps2f, acc, eps2ff);
                } else if constexpr (uses_order4_terms(MODE)) {
#pragma unroll kEvalUnroll
                    for (int k = jsub; k < kTJ; k += gl)
                        T::interact4(me, tl[k], jbase + k == ji, eps2, eps2f, acc);
                } else {
#pragma unroll kEvalUnroll
                    for (int k = jsub; k < kTJ; k += gl)
                        T::interact(me, tl[k], jbase + k == ji, eps2, eps2f, acc);
                }
                if constexpr (P == NB_FP32) {
                    if ((tt - tb + 1) % kFp32FlushTiles == 0) T::flush(acc, t64, t64st);
                    else T::tile_done(acc);
                } else if constexpr (P == NB_EX && NB_EX_LAZY && MODE != kModePot) {
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
                    mbar_expect_tx(&S.bar[s], kTJ * sizeof(J));
                    tma_load_1d(&S.tile[s][0], jc + (tt + kSt) * kTJ, kTJ * sizeof(J), &S.bar[s]);
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

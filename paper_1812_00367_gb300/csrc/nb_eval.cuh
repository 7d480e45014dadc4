// nb_eval.cuh -- the hot O(N_active x N) evaluation of acceleration, jerk,
// snap and potential (the paper's Sec. 4 kernel; 6th-order Hermite pair terms
// of Nitadori & Makino 2008) in three arithmetics, plus its j-split reduction.
//
// Per pair, with r = x_j - x_i, v = v_j - v_i, a = a_j - a_i (predicted),
// y = (r.r + eps^2)^{-1/2}, q = m_j y^3, alpha = (r.v) y^2, zeta = (v.v + r.a) y^2:
//   A0 = q r
//   A1 = q v - 3 alpha A0                = q v - 3 (q alpha) r
//   A2 = q a - 6 alpha A1 - 3 beta A0    = q a - 6 (q alpha) v + 3 q (5 alpha^2 - zeta) r
// (beta = zeta + alpha^2).  The six sums
//   sum q r, sum q v, sum q alpha r, sum q a, sum q alpha v, sum q (5 alpha^2 - zeta) r
// are accumulated separately and combined once per (i, j-range):
//   acc = S_qr, jerk = S_qv - 3 S_qar, snap = S_qa - 6 S_qav + 3 S_qcr, pot = -sum m_j y.
// That keeps every per-pair operation a multiply or a fused multiply-add
// (54 FP64 instructions per pair on the FP64 path).
//
// Work decomposition: a work item is (cluster, i-tile, j-range).  An i-tile
// holds kTPB / gl active particles; gl lanes of a warp share one i and take
// every gl-th j of each tile (gl = 1: i-parallel, j broadcast from shared
// memory; gl = 32: j-parallel for tiny active sets, warp-shuffle reduction).
// j-tiles of kTJ particles are copied global -> shared by the TMA engine
// (cp.async.bulk) into a kStages-deep ring guarded by mbarriers.  When the j
// range of a cluster is split over S items, each item writes FP64 partial
// sums; the CTA that finishes an i-tile last (atomic counter) adds the S
// partials in split order (deterministic) and finalises.
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
    };
    struct Acc {
        double qr[3], qv[3], qar[3], qa[3], qav[3], qcr[3], p;
    };
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
        for (int k = 0; k < 3; ++k) c.qr[k] = c.qv[k] = c.qar[k] = c.qa[k] = c.qav[k] = c.qcr[k] = 0.0;
        c.p = 0.0;
    }
    static __device__ __forceinline__ void interact(const I &i, const J &jj, bool self,
                                                    double eps2, float, Acc &c) {
        const double2 q0 = jj.q[0], q1 = jj.q[1], q2 = jj.q[2], q3 = jj.q[3], q4 = jj.q[4];
        const double rx = q0.x - i.x[0], ry = q0.y - i.x[1], rz = q1.x - i.x[2];
        const double vx = q2.x - i.v[0], vy = q2.y - i.v[1], vz = q3.x - i.v[2];
        const double ax = q3.y - i.a[0], ay = q4.x - i.a[1], az = q4.y - i.a[2];
        double r2 = fma(rx, rx, fma(ry, ry, fma(rz, rz, eps2)));
        double m = q1.y;
        r2 = self ? 1.0 : r2;  // selects, not FP64 arithmetic
        m = self ? 0.0 : m;
        const double y = rsqrt_f64(r2);
        const double y2 = y * y;
        const double my = m * y;
        const double q = my * y2;
        c.p += my;
        const double rv = fma(rx, vx, fma(ry, vy, rz * vz));
        const double w = fma(vx, vx, fma(vy, vy, fma(vz, vz, fma(rx, ax, fma(ry, ay, rz * az)))));
        const double al = rv * y2;
        const double ze = w * y2;
        const double qa = q * al;
        const double cc = fma(al * 5.0, al, -ze);
        const double qc = q * cc;
        c.qr[0] = fma(q, rx, c.qr[0]); c.qr[1] = fma(q, ry, c.qr[1]); c.qr[2] = fma(q, rz, c.qr[2]);
        c.qv[0] = fma(q, vx, c.qv[0]); c.qv[1] = fma(q, vy, c.qv[1]); c.qv[2] = fma(q, vz, c.qv[2]);
        c.qar[0] = fma(qa, rx, c.qar[0]); c.qar[1] = fma(qa, ry, c.qar[1]); c.qar[2] = fma(qa, rz, c.qar[2]);
        c.qa[0] = fma(q, ax, c.qa[0]); c.qa[1] = fma(q, ay, c.qa[1]); c.qa[2] = fma(q, az, c.qa[2]);
        c.qav[0] = fma(qa, vx, c.qav[0]); c.qav[1] = fma(qa, vy, c.qav[1]); c.qav[2] = fma(qa, vz, c.qav[2]);
        c.qcr[0] = fma(qc, rx, c.qcr[0]); c.qcr[1] = fma(qc, ry, c.qcr[1]); c.qcr[2] = fma(qc, rz, c.qcr[2]);
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
    static __device__ __forceinline__ void tile_done(Acc &, double *, int) {}
    static __device__ __forceinline__ void finish(const Acc &c, const double *, double o[10]) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o[k] = c.qr[k];
            o[3 + k] = fma(-3.0, c.qar[k], c.qv[k]);
            o[6 + k] = fma(3.0, c.qcr[k], fma(-6.0, c.qav[k], c.qa[k]));
        }
        o[9] = -c.p;
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
        ff qr[3], qv[3], qar[3], qa[3], qav[3], qcr[3], p;
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
        for (int k = 0; k < 3; ++k)
            c.qr[k] = c.qv[k] = c.qar[k] = c.qa[k] = c.qav[k] = c.qcr[k] = ff{0.f, 0.f};
        c.p = ff{0.f, 0.f};
    }
    // 1/sqrt(r2) in float-float: SFU seed y0, residual e = 1 - r2 y0^2 from the
    // exact square of y0 and FMA-exact products, then y0 (1 + e/2 + 3e^2/8).
    static __device__ __forceinline__ ff rsqrt_ff(ff r2) {
        float y0;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(r2.hi));
        const float p = __fmul_rn(y0, y0);
        const float pe = __fmaf_rn(y0, y0, -p);
        const float u = __fmul_rn(r2.hi, p);
        float ue = __fmaf_rn(r2.hi, p, -u);
        ue = __fmaf_rn(r2.hi, pe, ue);
        ue = __fmaf_rn(r2.lo, p, ue);
        const float e = __fsub_rn(__fsub_rn(1.0f, u), ue);
        const float corr = __fmul_rn(__fmul_rn(y0, e), __fmaf_rn(e, 0.375f, 0.5f));
        return ff_renorm(y0, corr);
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
        ff r2 = ff_add(ff_dot3(r, r), eps2);
        ff m = ff{q0.w, q1.w};
        if (self) {
            r2 = ff{1.f, 0.f};
            m = ff{0.f, 0.f};
        }
        const ff y = rsqrt_ff(r2);
        const ff y2 = ff_sqr(y);
        const ff my = ff_mul(m, y);
        const ff q = ff_mul(my, y2);
        c.p = ff_add(c.p, my);
        const ff rv = ff_dot3(r, v);
        const ff w = ff_add(ff_dot3(v, v), ff_dot3(r, a));
        const ff al = ff_mul(rv, y2);
        const ff ze = ff_mul(w, y2);
        const ff qa = ff_mul(q, al);
        const ff cc = ff_sub(ff_mul(ff_mul_f(al, 5.0f), al), ze);
        const ff qc = ff_mul(q, cc);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            ff_fma_acc(c.qr[k], q, r[k]);
            ff_fma_acc(c.qv[k], q, v[k]);
            ff_fma_acc(c.qar[k], qa, r[k]);
            ff_fma_acc(c.qa[k], q, a[k]);
            ff_fma_acc(c.qav[k], qa, v[k]);
            ff_fma_acc(c.qcr[k], qc, r[k]);
        }
    }
    static __device__ __forceinline__ void tile_done(Acc &, double *, int) {}
    static __device__ __forceinline__ double to_d(ff a) { return (double)a.hi + (double)a.lo; }
    static __device__ __forceinline__ void finish(const Acc &c, const double *, double o[10]) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o[k] = to_d(c.qr[k]);
            o[3 + k] = fma(-3.0, to_d(c.qar[k]), to_d(c.qv[k]));
            o[6 + k] = fma(3.0, to_d(c.qcr[k]), fma(-6.0, to_d(c.qav[k]), to_d(c.qa[k])));
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
    struct Acc {
        float qr[3], qv[3], qar[3], qa[3], qav[3], qcr[3], p;
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
        for (int k = 0; k < 3; ++k) c.qr[k] = c.qv[k] = c.qar[k] = c.qa[k] = c.qav[k] = c.qcr[k] = 0.f;
        c.p = 0.f;
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
        const float y2 = y * y;
        const float my = m * y;
        const float q = my * y2;
        c.p += my;
        const float rv = fmaf(rx, vx, fmaf(ry, vy, rz * vz));
        const float w = fmaf(vx, vx, fmaf(vy, vy, fmaf(vz, vz, fmaf(rx, ax, fmaf(ry, ay, rz * az)))));
        const float al = rv * y2;
        const float ze = w * y2;
        const float qa = q * al;
        const float cc = fmaf(al * 5.f, al, -ze);
        const float qc = q * cc;
        c.qr[0] = fmaf(q, rx, c.qr[0]); c.qr[1] = fmaf(q, ry, c.qr[1]); c.qr[2] = fmaf(q, rz, c.qr[2]);
        c.qv[0] = fmaf(q, vx, c.qv[0]); c.qv[1] = fmaf(q, vy, c.qv[1]); c.qv[2] = fmaf(q, vz, c.qv[2]);
        c.qar[0] = fmaf(qa, rx, c.qar[0]); c.qar[1] = fmaf(qa, ry, c.qar[1]); c.qar[2] = fmaf(qa, rz, c.qar[2]);
        c.qa[0] = fmaf(q, ax, c.qa[0]); c.qa[1] = fmaf(q, ay, c.qa[1]); c.qa[2] = fmaf(q, az, c.qa[2]);
        c.qav[0] = fmaf(qa, vx, c.qav[0]); c.qav[1] = fmaf(qa, vy, c.qav[1]); c.qav[2] = fmaf(qa, vz, c.qav[2]);
        c.qcr[0] = fmaf(qc, rx, c.qcr[0]); c.qcr[1] = fmaf(qc, ry, c.qcr[1]); c.qcr[2] = fmaf(qc, rz, c.qcr[2]);
    }
    // Promote the FP32 chunk sums (combined to acc/jerk/snap/pot) into the
    // FP64 totals and restart the FP32 sums.
    static __device__ __forceinline__ void flush(Acc &c, double *t64) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            t64[k] += (double)c.qr[k];
            t64[3 + k] += (double)fmaf(-3.f, c.qar[k], c.qv[k]);
            t64[6 + k] += (double)fmaf(3.f, c.qcr[k], fmaf(-6.f, c.qav[k], c.qa[k]));
        }
        t64[9] += (double)c.p;
        zero(c);
    }
    static __device__ __forceinline__ void finish(Acc &c, double *t64, double o[10]) {
        flush(c, t64);
#pragma unroll
        for (int k = 0; k < 9; ++k) o[k] = t64[k];
        o[9] = -t64[9];
    }
};

// ================================================================ kernel
template <int P>
struct SmemLayout {
    typename Prec<P>::J tile[kStages][kTJ];
    uint64_t bar[kStages];
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
    if constexpr (MODE == kModeOut) {
        for (int q = 0; q < 10; ++q) L.out[(int64_t)q * L.n_active + iloc] = o[q];
    } else if constexpr (MODE == kModeStep) {
        correct_particle(d, gi, d.tnext[c], o);
    } else if constexpr (MODE == kModeInit1 || MODE == kModeInit2) {
        const int64_t n = d.n;
        for (int k = 0; k < 3; ++k) {
            d.a[k * n + gi] = o[k];
            d.j[k * n + gi] = o[3 + k];
            d.s[k * n + gi] = (MODE == kModeInit2) ? o[6 + k] : 0.0;
        }
        d.pot[gi] = o[9];
        if constexpr (MODE == kModeInit2) d.dt[gi] = dt_start(d, o);
    } else {  // kModePot
        d.pot_tmp[gi] = o[9];
    }
}

template <int P, int MODE>
__global__ void __launch_bounds__(kTPB) k_eval(const Dev d, const EvalLaunch L) {
    using T = Prec<P>;
    using J = typename T::J;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SmemLayout<P> &S = *reinterpret_cast<SmemLayout<P> *>(smem_raw);
    const int tid = threadIdx.x;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&S.bar[s], 1);
        S.fail = 0;
        fence_mbar_init();
    }
    __syncthreads();

    const int64_t n_items = L.direct ? (int64_t)L.tiles * L.split : *d.n_items;
    const J *jall = reinterpret_cast<const J *>(d.jarr);
    const double eps2 = d.eps2;
    const float eps2f = (float)d.eps2;
    ff eps2ff;
    eps2ff.hi = (float)d.eps2;
    eps2ff.lo = (float)(d.eps2 - (double)eps2ff.hi);
    uint32_t phase = 0;   // bit s: parity of stage s
    uint32_t pending = 0; // bit s: a copy into stage s is in flight

    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        int c, gl, split, A;
        int64_t item0, tile0, pslot0;
        if (L.direct) {
            c = L.cluster; gl = L.gl; split = L.split; A = L.n_active; item0 = 0; tile0 = 0;
            pslot0 = 0;
        } else {
            c = find_cluster(d.plan, d.n_clusters, item);
            const ClusterPlan pl = d.plan[c];
            gl = pl.gl; split = pl.split; A = pl.active; item0 = pl.item0; tile0 = pl.tile0;
            pslot0 = pl.pslot0;
        }
        const int64_t local = item - item0;
        const int tile = (int)(local / split);
        const int sidx = (int)(local % split);
        const int Ti = kTPB / gl;
        const int ilane = tid / gl;
        const int jsub = tid % gl;
        const int iloc = tile * Ti + ilane;
        const bool valid = iloc < A;
        const int64_t off = d.offsets[c];
        const int64_t nc = d.offsets[c + 1] - off;
        const J *jc = jall + d.jofs[c];
        int64_t gi = off;
        bool bad_index = false;
        if (valid) {
            if (L.identity) gi = off + iloc;
            else if (L.direct) gi = L.active[iloc];
            else gi = d.active[off + iloc];
            if (gi < off || gi >= off + nc) {  // caller-given index outside the cluster
                atomicOr(d.err, kErrIndex);
                gi = off;
                bad_index = true;
            }
        }
        const int64_t ji = gi - off;
        const typename T::I me = T::load_i(jc, ji);
        typename T::Acc acc;
        T::zero(acc);
        double t64[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) t64[q] = 0.0;

        const int64_t ntj = cdiv(nc, kTJ);
        const int64_t tb = ntj * sidx / split;
        const int64_t te = ntj * (sidx + 1) / split;
        const bool warp_active = __any_sync(0xffffffffu, valid);

        // prologue: fill the ring
        if (tid == 0) {
            for (int s = 0; s < kStages && tb + s < te; ++s) {
                mbar_expect_tx(&S.bar[s], kTJ * sizeof(J));
                tma_load_1d(&S.tile[s][0], jc + (tb + s) * kTJ, kTJ * sizeof(J), &S.bar[s]);
                pending |= 1u << s;
            }
        }
        bool ok = true;
        for (int64_t tt = tb; tt < te; ++tt) {
            const int s = (int)((tt - tb) % kStages);
            if (ok) ok = mbar_wait_bounded(&S.bar[s], (phase >> s) & 1u);
            phase ^= 1u << s;
            if (ok && warp_active) {
                const J *tl = &S.tile[s][0];
                const int64_t jbase = tt * kTJ;
                if constexpr (MODE == kModePot) {
                    for (int k = jsub; k < kTJ; k += gl)
                        T::interact_pot(me, tl[k], jbase + k == ji, eps2, acc);
                } else if constexpr (P == NB_EX) {
#pragma unroll 1
                    for (int k = jsub; k < kTJ; k += gl)
                        T::interact(me, tl[k], jbase + k == ji, eps2, eps2f, acc, eps2ff);
                } else {
#pragma unroll 2
                    for (int k = jsub; k < kTJ; k += gl)
                        T::interact(me, tl[k], jbase + k == ji, eps2, eps2f, acc);
                }
                if constexpr (P == NB_FP32) {
                    if ((tt - tb + 1) % kFp32FlushTiles == 0) T::flush(acc, t64);
                }
            }
            if (!ok) S.fail = 1;
            __syncthreads();
            if (S.fail) break;
            if (tid == 0) {
                pending &= ~(1u << s);
                if (tt + kStages < te) {
                    mbar_expect_tx(&S.bar[s], kTJ * sizeof(J));
                    tma_load_1d(&S.tile[s][0], jc + (tt + kStages) * kTJ, kTJ * sizeof(J), &S.bar[s]);
                    pending |= 1u << s;
                }
            }
        }
        if (S.fail) {
            // a copy did not land in time: record it, drain (bounded) what this
            // CTA still has in flight, and leave the kernel
            if (tid == 0) {
                atomicOr(d.err, kErrTimeout);
                for (int s = 0; s < kStages; ++s)
                    if (pending & (1u << s)) (void)mbar_wait_bounded(&S.bar[s], (phase >> s) & 1u);
            }
            return;
        }

        double o[10];
        T::finish(acc, t64, o);
        // lanes sharing an i: butterfly sum (fixed order)
        for (int w = gl >> 1; w >= 1; w >>= 1) {
#pragma unroll
            for (int q = 0; q < 10; ++q) o[q] += __shfl_xor_sync(0xffffffffu, o[q], w);
        }

        if (split == 1) {
            if (valid && jsub == 0 && !bad_index) finalize_one<P, MODE>(d, L, c, gi, iloc, o);
            continue;
        }
        double *part = d.partial + (pslot0 + local) * (int64_t)(10 * kTPB);
        if (jsub == 0) {
#pragma unroll
            for (int q = 0; q < 10; ++q) part[q * kTPB + ilane] = o[q];
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const int prev = atomicAdd(&d.tile_cnt[tile0 + tile], 1);
            S.flag = (prev == split - 1);
        }
        __syncthreads();
        if (S.flag) {
            __threadfence();
            if (tid < Ti) {
                const int il = tile * Ti + tid;
                if (il < A) {
                    double sum[10];
#pragma unroll
                    for (int q = 0; q < 10; ++q) sum[q] = 0.0;
                    const double *base = d.partial + (pslot0 + (int64_t)tile * split) * (10 * kTPB);
                    for (int sp = 0; sp < split; ++sp) {
                        const double *pp = base + (int64_t)sp * (10 * kTPB);
#pragma unroll
                        for (int q = 0; q < 10; ++q) sum[q] += __ldcg(pp + q * kTPB + tid);
                    }
                    int64_t g2;
                    if (L.identity) g2 = off + il;
                    else if (L.direct) g2 = L.active[il];
                    else g2 = d.active[off + il];
                    if (g2 >= off && g2 < off + nc) finalize_one<P, MODE>(d, L, c, g2, il, sum);
                }
            }
            if (tid == 0) d.tile_cnt[tile0 + tile] = 0;
        }
        __syncthreads();
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

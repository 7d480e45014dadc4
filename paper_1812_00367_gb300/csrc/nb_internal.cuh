// nb_internal.cuh -- device-side data structures and primitives of libnb.
//
// Everything here is internal to the CUDA library; the public boundary is
// include/nb.h.  Sm_103a only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/nb.h"

namespace nb {

// ---------------------------------------------------------------- constants
#ifndef NB_EVAL_TPB
#define NB_EVAL_TPB 128       // threads per evaluation CTA (64, 128 or 256)
#endif
constexpr int kTPB = NB_EVAL_TPB;
static_assert(kTPB == 64 || kTPB == 128 || kTPB == 256, "evaluation CTA: 64, 128 or 256 threads");
constexpr int kTJ = 64;        // j-particles per shared-memory tile
#ifndef NB_EVAL_STAGES
#define NB_EVAL_STAGES 4
#endif
#ifndef NB_EVAL_MIN_BLOCKS
#define NB_EVAL_MIN_BLOCKS 4  // resident evaluation CTAs per SM the compiler must allow
#endif
#ifndef NB_EVAL_UNROLL
#define NB_EVAL_UNROLL 2      // j-loop unrolling of the FP64 / FP32 evaluation
#endif
#ifndef NB_EX_LAZY
// 1: the EX evaluation keeps its sums and intermediate products unnormalised
// (hi + lo with every error term kept; sums renormalised once per j-tile).
// Measured: 1.126x the pair rate at N = 65536, and the same maximum errors
// against FP64 at N = 2^20 (Kroupa masses, eps = 1e-5) to two digits.
#define NB_EX_LAZY 1
#endif
#ifndef NB_FP64_ALL_FMA
// 1: the FP64 evaluation issues its products and differences as FMAs with
// run-time -0.0 / -1.0 operands.  On GB300, DADD and DMUL run at 84 % of the
// DFMA instruction rate (nb_probe_fma_peak modes 5, 6 vs 0), and this form
// measured 5.9 % faster for the whole pair evaluation.
#define NB_FP64_ALL_FMA 1
#endif
// FP32 evaluation: its own ring depth, residency and place of the FP64
// chunk totals (registers, or shared memory when NB_FP32_T64_SMEM)
#ifndef NB_FP32_STAGES
#define NB_FP32_STAGES NB_EVAL_STAGES
#endif
#ifndef NB_FP32_MIN_BLOCKS
#define NB_FP32_MIN_BLOCKS NB_EVAL_MIN_BLOCKS
#endif
#ifndef NB_EX_MIN_BLOCKS
#define NB_EX_MIN_BLOCKS NB_EVAL_MIN_BLOCKS
#endif
#ifndef NB_FP32X_MIN_BLOCKS
#define NB_FP32X_MIN_BLOCKS NB_EVAL_MIN_BLOCKS
#endif
#ifndef NB_EX4_MIN_BLOCKS
#define NB_EX4_MIN_BLOCKS 3
#endif
#ifndef NB_FP32_T64_SMEM
#define NB_FP32_T64_SMEM 1
#endif
constexpr int kStages = NB_EVAL_STAGES;  // TMA pipeline depth
constexpr int kEvalUnroll = NB_EVAL_UNROLL;
constexpr int kChunk = 2048;   // particles per select / predict chunk
constexpr int kSelTPB = 256;   // threads per select / predict CTA
constexpr int kPlanTPB = 1024; // threads of the single planning CTA
constexpr int kBuckets = 32;   // active-set size buckets (floor log2 A)
constexpr int kFp32FlushTiles = 32;  // FP32 path: j-tiles summed in FP32 before
                                     // promotion to FP64 (32 x 64 = 2048 j)

// device error word bits
constexpr uint32_t kErrNonFinite = 1u;
constexpr uint32_t kErrTimeout = 2u;
constexpr uint32_t kErrIndex = 4u;   // a caller-given index outside its cluster

// wait budget of a bounded device-side wait, nanoseconds
constexpr unsigned long long kWaitBudgetNs = 2000000000ull;

// ------------------------------------------------------------ packed j-data
#ifndef NB_FP64_POT_FF
// 1: the FP64 pair terms sum the potential in float-float on the FP32 pipe
// (m y from the mass's float pair and y's bits; renormalised every term, a
// j-tile's sum added to an FP64 total), one DFMA fewer per pair: measured
// +1.5 % FP64 pair rate, potential within 1e-12 of the oracle at N = 2^20
// (the j record grows from 80 to 96 bytes)
#define NB_FP64_POT_FF 1
#endif
// FP64: x, y, z, m, vx, vy, vz, ax, ay, az as five 16-byte pairs (and, with
// NB_FP64_POT_FF, the mass as a float pair).
struct alignas(16) J64 {
    double2 q[5];  // (x,y) (z,m) (vx,vy) (vz,ax) (ay,az)
#if NB_FP64_POT_FF
    float2 mf;     // (m_hi, m_lo)
    float2 pad_;
#endif
};
// Fill the record's float-pair mass (no-op without NB_FP64_POT_FF).
__host__ __device__ inline void j64_set_mass_split(J64 &w, double m) {
#if NB_FP64_POT_FF
    const float hi = (float)m;
    w.mf = make_float2(hi, (float)(m - (double)hi));
    w.pad_ = make_float2(0.f, 0.f);
#else
    (void)w;
    (void)m;
#endif
}
// EX and FP32X: 80 bytes per particle (hi/lo single pairs), stored as records of two
// particles whose values interleave like the FP32 records below: value f of
// lane l of record r is float r * 40 + 2 f + l, f in the order
//   xh, yh, zh, mh, xl, yl, zl, ml, vxh, vyh, vzh, axh, vxl, vyl, vzl, axl,
//   ayh, azh, ayl, azl
// so q[k] of a record holds (value 2k of lanes 0, 1; value 2k + 1 of lanes 0, 1).
struct alignas(16) JEX {  // one particle's share of the array (sizing only)
    float4 q[5];
};
struct alignas(16) JEXP {  // a record of two particles
    float4 q[10];
};
constexpr int kJEXVals = 20;
// FP32: 64 bytes per particle, stored as records of two particles whose
// values interleave, so that one 16-byte shared-memory load gives two
// two-lane operands of the packed FP32 arithmetic.  Value f of lane l (the
// particle's index parity) of record r is float r * 32 + 2 f + l, f in the
// order xh, yh, zh, m, xl, yl, zl, ax, vxh, vyh, vzh, ay, vxl, vyl, vzl, az:
//   q[0] = (xh0, xh1, yh0, yh1)  q[1] = (zh0, zh1, m0, m1)
//   q[2] = (xl0, xl1, yl0, yl1)  q[3] = (zl0, zl1, ax0, ax1)
//   q[4] = (vxh0, vxh1, vyh0, vyh1)  q[5] = (vzh0, vzh1, ay0, ay1)
//   q[6] = (vxl0, vxl1, vyl0, vyl1)  q[7] = (vzl0, vzl1, az0, az1)
struct alignas(16) J32 {  // one particle's share of the array (sizing only)
    float4 q[4];
};
struct alignas(16) J32P {  // a record of two particles
    float4 q[8];
};
constexpr int kJ32Vals = 16;
// Write particle jx's NV values (the orders above) into a two-particle
// record array (FP32: NV = 16, EX: NV = 20).
template <int NV>
__device__ __forceinline__ void jpair_store(void *jarr, int64_t jx, const float v[NV]) {
    float *p = reinterpret_cast<float *>(jarr) + (jx >> 1) * (2 * NV) + (jx & 1);
#pragma unroll
    for (int f = 0; f < NV; ++f) p[2 * f] = v[f];
}

// ------------------------------------------------------------ planning data
struct ClusterPlan {
    int32_t gl;     // lanes cooperating on one i (1..32, power of two)
    int32_t split;  // number of j-ranges (S)
    int32_t tiles;  // i-tiles of kTPB / gl active particles
    int32_t active; // A for this step (0: idle)
    int64_t item0;  // first work item of the cluster
    int64_t tile0;  // first i-tile of the cluster (counter index)
    int64_t pslot0; // first partial-sum double (only clusters with split > 1 use them)
    int32_t streamk; // 1: single-cluster launch split stream-K style (split unused)
    int32_t pad_;
};

struct PlanEntry {  // per active-set bucket
    int32_t gl;
    int32_t target_items;  // desired work items per evaluation
};

// Everything a kernel needs, passed by value.
struct Dev {
    int64_t n;
    int32_t n_clusters;
    int32_t n_chunks;
    int32_t precision;
    int32_t grid_eval;  // persistent evaluation grid (CTAs)
    const int64_t *offsets;      // [nc+1] particle offsets
    const int64_t *jofs;         // [nc+1] padded j-array offsets
    const int32_t *chunk_cluster;// [n_chunks]
    const int64_t *chunk_begin;  // [n_chunks]
    const int64_t *chunk_end;    // [n_chunks]
    const int32_t *cluster_chunk0;  // [nc+1]
    // state (caller-owned), SoA [3][n]
    double *m, *x, *v, *a, *j, *s, *c, *t, *dt, *pot;
    // predicted j-arrays
    void *jarr;        // precision-specific (J64 / JEX (EX, FP32X) / J32)
    J64 *jarr64;       // FP64 copy (energy, nb_predict output); == jarr for FP64
    // select
    double *chunk_min;
    int32_t *chunk_cnt;
    double *tnext;     // [nc]
    int32_t *nact;     // [nc]
    int32_t *active;   // [n], cluster c's list at offsets[c]
    // plan
    ClusterPlan *plan; // [nc]
    int64_t *n_items;  // [1]
    unsigned long long *item_ctr;  // [1]: next work item (dynamic fetch), reset by k_plan
    const PlanEntry *table;  // [kBuckets]
    // reduction scratch
    double *partial;   // [max_items][10][kTPB]
    int64_t partial_cap;     // capacity in doubles (an item of Ti i's uses 10 Ti)
    int32_t *tile_cnt; // [max_tiles]
    // counters / flags
    unsigned long long *ctr_steps;
    double *ctr_inter;
    unsigned long long *ctr_underflow;
    uint32_t *err;
    int32_t *busy;     // [1]: clusters active in the last select
    double *t_end;     // [1]: clusters whose next block time exceeds it stay idle
    double *pot_tmp;   // [n] energy potential
    double *energy_part;  // [blocks][8]
    // parameters
    double eps2, eta, eta_init, dt_min, dt_max;
    // -1.0 and -0.0 as run-time values: FP64 products and differences issued
    // as FMAs (a*b - 0, a - b = b*(-1) + a) cannot be folded back by compilers
    double neg_one, neg_zero;
    // 6: NM08 6th order; 4: Makino & Aarseth 4th order.  Kept last: inserting
    // it among the fields above measured 2.8 % slower FP64 evaluation.
    int32_t order;
    int32_t streamk_off;  // NB_NO_STREAMK
    unsigned int *sel_ctr;  // [1]: chunks done in select pass 1 (the last one finishes the pass)
    // eps^2 as a float-float pair, both lanes equal: hi = fl(eps^2),
    // lo = fl(eps^2 - hi).  Formed on the host: the single-precision kernels
    // read them as parameters, where converting eps2 in the kernel costs
    // FP64-pipe conversions wherever the compiler re-forms the values.
    float2 eps2_hi2, eps2_lo2;
};

// eps^2 and its float-float pair (host side; every context and launch).
inline void set_eps2(Dev &d, double eps) {
    d.eps2 = eps * eps;
    const float hi = (float)d.eps2;
    const float lo = (float)(d.eps2 - (double)hi);
    d.eps2_hi2 = make_float2(hi, hi);
    d.eps2_lo2 = make_float2(lo, lo);
}

// How one evaluation launch obtains its work.
struct EvalLaunch {
    int32_t direct;     // 1: single cluster, host-given list / plan
    int32_t cluster;    // direct mode
    int32_t n_active;   // direct mode
    int32_t gl;         // direct mode
    int32_t split;      // direct mode
    int32_t tiles;      // direct mode
    int32_t identity;   // active list is 0..A-1 of the cluster (init, energy)
    const int32_t *active;  // direct mode list (global indices)
    double *out;        // direct mode output [10][n_active]
    int32_t streamk;    // direct mode: stream-K ranges instead of split items
    int32_t jt0, jt1;   // direct mode: j-tiles [jt0, jt1) of the cluster (jt1 = 0: all)
};

// Out/Step/Init1/Init2: 6th-order pair terms (a, jerk, snap); the *4 modes
// evaluate the 4th-order terms (a, jerk; snap slots stay 0); Pot: potential.
enum EvalMode {
    kModeOut = 0, kModeStep = 1, kModeInit1 = 2, kModeInit2 = 3, kModePot = 4,
    kModeOut4 = 5, kModeStep4 = 6, kModeInit4 = 7
};
constexpr bool is_order4_mode(int mode) { return mode >= kModeOut4; }
// Modes that sum only acceleration, jerk and potential (the 4th-order pair
// terms): the 4th-order modes, and the first start-up pass of the 6th-order
// scheme, whose only output that survives is the acceleration (pass 2 needs
// it for the relative accelerations; it recomputes a and jerk with snap).
constexpr bool uses_order4_terms(int mode) { return is_order4_mode(mode) || mode == kModeInit1; }

// ---------------------------------------------------------- small helpers
__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

constexpr int kMinTilesPerItem = 4;  // a j-range holds at least 4 x 64 j

// Stream-K decomposition of a single cluster's evaluation.  Its work is
// U = tiles x ntj units (one i-tile against one j-tile, all of equal cost);
// CTA k of G takes the contiguous unit range [U k / G, U (k+1) / G), so every
// CTA (and every SM) gets the same work to within one unit.  A range splits
// at i-tile boundaries into pieces; an i-tile covered by several CTAs gets one
// partial sum per CTA, added in CTA order by the last one to finish.
#ifndef NB_STREAMK
#define NB_STREAMK 1
#endif
#ifndef NB_STREAMK_MIN_UNITS
#define NB_STREAMK_MIN_UNITS 4
#endif
constexpr int kStreamKMinUnits = NB_STREAMK_MIN_UNITS;  // units per CTA below which splits are used
__host__ __device__ inline int64_t sk_begin(int64_t U, int64_t G, int64_t k) { return U * k / G; }
// CTA whose range holds unit p (the largest k with sk_begin(k) <= p; U >= G)
__host__ __device__ inline int64_t sk_owner(int64_t U, int64_t G, int64_t p) {
    return ((p + 1) * G + U - 1) / U - 1;
}
// most i-tiles one CTA's range can touch
__host__ __device__ inline int64_t sk_max_pieces(int64_t U, int64_t G, int64_t ntj) {
    return (cdiv(U, G) - 1) / ntj + 2;
}
// whether a launch of `tiles` i-tiles of Ti i's over ntj j-tiles on G CTAs
// runs stream-K: enough units per CTA, partial sums within the scratch
__host__ __device__ inline bool sk_use(int64_t tiles, int64_t Ti, int64_t ntj, int64_t G,
                                       int64_t partial_cap) {
    if (!NB_STREAMK || tiles <= 0) return false;
    const int64_t U = tiles * ntj;
    if (U < kStreamKMinUnits * G) return false;
    return G * sk_max_pieces(U, G, ntj) * 10 * Ti <= partial_cap;
}

// Number of j-ranges (split S) for `tiles` i-tiles over a cluster of `ntj`
// j-tiles.  Start from the bucket's target item count; keep at least
// kMinTilesPerItem j-tiles per item; for `grid` resident CTAs, take the
// smallest S in [S0/2, 2 S0] whose items fill the largest fraction of whole
// waves (equal-cost items: a last, partly filled wave leaves SMs idle).  The
// result depends on this cluster alone, so a cluster's plan (and therefore
// its rounding) is the same in a batch as on its own.
__host__ __device__ inline int64_t choose_split(int64_t tiles, int64_t ntj, int64_t target,
                                                int64_t grid) {
    const int64_t smax = ntj / kMinTilesPerItem > 1 ? ntj / kMinTilesPerItem : 1;
    int64_t s0 = cdiv(target, tiles > 0 ? tiles : 1);
    s0 = s0 < 1 ? 1 : (s0 > smax ? smax : s0);
    if (grid <= 0) return s0;
    // efficiency items / (waves * grid), compared by cross-multiplication in
    // integers.  Within one wave count w the efficiency grows with S, so only
    // the largest S of each w can win: visit the wave counts of the window
    // (a few) instead of every S (a few hundred 64-bit divisions in the
    // planner's single thread); stepping w upwards and keeping only strict
    // improvements returns the smallest S of the best efficiency.
    int64_t best = s0, best_items = 0, best_slots = 1;
    const int64_t lo = s0 / 2 > 1 ? s0 / 2 : 1;
    const int64_t hi = 2 * s0 < smax ? 2 * s0 : smax;
    const int64_t t = tiles > 0 ? tiles : 1;
    const int64_t w_lo = cdiv(t * lo, grid), w_hi = cdiv(t * hi, grid);
    for (int64_t w = w_lo; w <= w_hi; ++w) {
        int64_t s = (w * grid) / t;  // the largest S with t S <= w grid
        s = s > hi ? hi : s;
        if (s < lo || t * s <= (w - 1) * grid) continue;  // no S of the window fills w waves
        const int64_t items = t * s, slots = w * grid;
        if (items * best_slots > best_items * slots) {
            best_items = items;
            best_slots = slots;
            best = s;
        }
    }
    return best;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------- FP64 rsqrt
// 1/sqrt(r2) for r2 in [2^-126, 2^128).  Seed: the exponent and top 20
// mantissa bits of r2 are moved into an FP32 word with integer operations,
// the SFU gives rsqrt.approx, and the result is moved back the same way
// (relative seed error below 2^-19).  One third-order step
//   y = y0 (1 + e/2 + 3 e^2/8),  e = 1 - r2 y0^2
// (the binomial series of (1 - e)^{-1/2}) leaves a truncation error of about
// (5/16) e^3 < 2^-55; y0 has 21 significant bits, so y0^2 is exact.  Five FP64
// operations, none of them on the seed.
__device__ __forceinline__ double rsqrt_f64(double r2) {
    const int hi = __double2hiint(r2);
    const float f = __int_as_float((hi - 0x38000000) << 3);
    float yf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(f));
    const double y0 = __hiloint2double((__float_as_int(yf) >> 3) + 0x38000000, 0);
    const double y2 = y0 * y0;
    const double e = fma(-r2, y2, 1.0);
    const double p = fma(e, 0.375, 0.5);
    const double t = y0 * e;
    return fma(t, p, y0);
}

// The same with its two products issued as FMAs against a run-time -0.0
// (x*y + (-0) == x*y, signed zeros included): every instruction is a DFMA.
__device__ __forceinline__ double fma_rn_f64(double a, double b, double c) {
    double r;
    asm("fma.rn.f64 %0, %1, %2, %3;" : "=d"(r) : "d"(a), "d"(b), "d"(c));
    return r;
}
__device__ __forceinline__ double rsqrt_f64_fma(double r2, double neg_zero) {
    const int hi = __double2hiint(r2);
    const float f = __int_as_float((hi - 0x38000000) << 3);
    float yf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(f));
    const double y0 = __hiloint2double((__float_as_int(yf) >> 3) + 0x38000000, 0);
    const double y2 = fma_rn_f64(y0, y0, neg_zero);
    const double e = fma(-r2, y2, 1.0);
    const double p = fma(e, 0.375, 0.5);
    const double t = fma_rn_f64(y0, e, neg_zero);
    return fma(t, p, y0);
}

// SFU approximation of 1/sqrt (rsqrt.approx.ftz.f32), per lane for float2.
__device__ __forceinline__ float rsqrt_sfu(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float2 rsqrt_sfu(float2 x) {
    return make_float2(rsqrt_sfu(x.x), rsqrt_sfu(x.y));
}
#ifndef NB_FP64_RSQRT3
// 1: the FP64 pair terms take 1/sqrt from rsqrt_f64_3 (three FP64
// operations, the seed refined on the FP32 and integer pipes) instead of
// rsqrt_f64_fma (five)
#define NB_FP64_RSQRT3 1
#endif

// 1/sqrt(x) for a positive normal double x, with three FP64 operations.
//  - x = 2^(2m) x', x' in [1, 4): an exact exponent shift (integer pipe).
//  - x' as a float pair xh + xl (24 + 23 significant bits) from its bits:
//    xh truncated (integer pipe), xl an integer of 23 bits turned into a
//    float by the 2^23 bias trick (one FP32 subtraction) and scaled.
//  - y0 = SFU 1/sqrt(xh); residual e = 1 - x' y0^2 from exact FP32 products
//    (1 - u is exact by Sterbenz, u = xh y0^2 lying within 2^-21 of 1);
//    c = y0 e (1/2 + 3e/8), the third-order step of the binomial series of
//    (1 - e)^{-1/2}, so y0 + c is within about 2^-44 of 1/sqrt(x').
//  - Y = y0 + c rounded to 30 significant bits and assembled as a double on
//    the integer pipe (its exponent renormalised when the correction crosses
//    a power of two), Y/2 by an exponent decrement.
//  - One Newton step in FP64: y' = Y + (Y/2)(1 - x' Y^2); with
//    |1 - x' Y^2| < 2^-28 its truncation error (3/8)(1 - x' Y^2)^2 is below
//    2^-57, and the roundings of Y^2 and the last FMA stay near 1 ulp.
//  - y = 2^-m y' (integer pipe, exact).
__device__ __forceinline__ double rsqrt_f64_3(double x, double neg_zero) {
    const int hx = __double2hiint(x), lx = __double2loint(x);
    const int m = ((((unsigned)hx >> 20) & 0x7ff) - 1023) >> 1;  // floor(exponent / 2)
    const int hxp = hx - (m << 21);                              // x' = 2^-2m x
    const int exp_p = (hxp >> 20) - 1023;                        // 0 or 1
    const double xp = __hiloint2double(hxp, lx);
    const float xh =
        __int_as_float((int)__funnelshift_l((unsigned)lx, (unsigned)(hxp - 0x38000000), 3));
    const float l23 = __fsub_rn(__int_as_float(0x4B000000 | (((unsigned)lx >> 6) & 0x7FFFFFu)),
                                8388608.0f);                     // next 23 bits, exact
    const float xl = __fmul_rn(l23, __int_as_float((127 - 46 + exp_p) << 23));
    const float y0 = rsqrt_sfu(xh);
    const float p = __fmul_rn(y0, y0);
    const float pe = __fmaf_rn(y0, y0, -p);
    const float u = __fmul_rn(xh, p);
    float ue = __fmaf_rn(xh, p, -u);
    ue = __fmaf_rn(xh, pe, ue);
    ue = __fmaf_rn(xl, p, ue);
    const float e = __fsub_rn(__fsub_rn(1.0f, u), ue);
    const float c = __fmul_rn(__fmul_rn(y0, e), __fmaf_rn(e, 0.375f, 0.5f));
    // Y = y0 + c in units of 2^(ey - 29), ey the exponent of y0 (-1 or 0)
    const int yb = __float_as_int(y0);
    int ey = ((yb >> 23) & 0xff) - 127;
    const float cs = __fmaf_rn(c, __int_as_float((127 + 29 - ey) << 23), 12582912.0f);
    int M = (((yb & 0x7FFFFF) | 0x800000) << 6) + (__float_as_int(cs) - 0x4B400000);
    if (M >= (1 << 30)) {
        M >>= 1;
        ey += 1;
    } else if (M < (1 << 29)) {
        M <<= 1;
        ey -= 1;
    }
    const int frac = M - (1 << 29);
    const int hy = ((ey + 1023) << 20) | (frac >> 9);
    const int ly = (frac & 0x1FF) << 23;
    const double Y = __hiloint2double(hy, ly);
    const double Yh = __hiloint2double(hy - (1 << 20), ly);
    const double Y2 = fma_rn_f64(Y, Y, neg_zero);
    const double e2 = fma(-xp, Y2, 1.0);
    const double yp = fma(Yh, e2, Y);
    return __hiloint2double(__double2hiint(yp) - (m << 20), __double2loint(yp));
}

// 2x by adding one to the exponent field on the integer pipe (exact for
// normal x whose double does not overflow).  Zero, subnormal, infinite and NaN
// inputs are returned unchanged (a subnormal is then off by a factor two, at
// the 1e-308 level; a NaN stays NaN).
__device__ __forceinline__ double twice_int(double x) {
    const int hi = __double2hiint(x);
    const int ex = hi & 0x7ff00000;
    const bool ok = ex != 0 && ex < 0x7fe00000;
    return __hiloint2double(ok ? hi + 0x00100000 : hi, __double2loint(x));
}

// --------------------------------------------- packed two-lane FP32 (f32x2)
// sm_100 and later execute FP32 add / multiply / FMA on a pair of floats in
// one instruction (PTX add/sub/mul/fma.rn.f32x2): the same per-lane IEEE
// round-to-nearest results as the scalar instructions, half the issue slots.
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 ta, tb, tr;\n\tmov.b64 ta, {%2, %3};\n\tmov.b64 tb, {%4, %5};\n\t"
        "sub.rn.f32x2 tr, ta, tb;\n\tmov.b64 {%0, %1}, tr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 lo2(float4 q) { return make_float2(q.x, q.y); }
__device__ __forceinline__ float2 hi2(float4 q) { return make_float2(q.z, q.w); }

// ------------------------------------------------------- float-float (EX)
// A value is hi + lo with |lo| <= ulp(hi)/2 (Dekker 1971; Knuth TAOCP 2;
// Hida, Li & Bailey 2001 for the double-double algorithms, here on floats).
// Every primitive is written once for a lane type T: float (one value) or
// float2 (two independent values, one per lane, each with the IEEE results
// of the float form, evaluated by the packed f32x2 instructions).
template <class T>
struct ffT {
    T hi, lo;
};
using ff = ffT<float>;
using ff2 = ffT<float2>;

__device__ __forceinline__ float o_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float o_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float o_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float o_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float o_neg(float a) { return -a; }
__device__ __forceinline__ float o_cst(float, float c) { return c; }
__device__ __forceinline__ float2 o_add(float2 a, float2 b) { return add2(a, b); }
__device__ __forceinline__ float2 o_sub(float2 a, float2 b) { return sub2(a, b); }
__device__ __forceinline__ float2 o_mul(float2 a, float2 b) { return mul2(a, b); }
__device__ __forceinline__ float2 o_fma(float2 a, float2 b, float2 c) { return fma2(a, b, c); }
__device__ __forceinline__ float2 o_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 o_cst(float2, float c) { return f2s(c); }

// exact: s + e = a + b (Knuth TwoSum)
template <class T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e) {
    s = o_add(a, b);
    const T bb = o_sub(s, a);
    e = o_add(o_sub(a, o_sub(s, bb)), o_sub(b, bb));
}
// exact: s + e = a - b (TwoSum of a and -b, the negation folded in)
template <class T>
__device__ __forceinline__ void two_diff(T a, T b, T &s, T &e) {
    s = o_sub(a, b);
    const T bb = o_sub(s, a);
    e = o_sub(o_sub(a, o_sub(s, bb)), o_add(b, bb));
}
// exact when |a| >= |b| (Dekker FastTwoSum)
template <class T>
__device__ __forceinline__ void fast_two_sum(T a, T b, T &s, T &e) {
    s = o_add(a, b);
    e = o_sub(b, o_sub(s, a));
}
template <class T>
__device__ __forceinline__ ffT<T> ff_renorm(T s, T e) {
    ffT<T> r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}
template <class T>
__device__ __forceinline__ ffT<T> ff_add(ffT<T> a, ffT<T> b) {
    T s, e;
    two_sum(a.hi, b.hi, s, e);
    e = o_add(e, o_add(a.lo, b.lo));
    return ff_renorm(s, e);
}
template <class T>
__device__ __forceinline__ ffT<T> ff_neg(ffT<T> a) { return ffT<T>{o_neg(a.hi), o_neg(a.lo)}; }
// a - b, normalised
template <class T>
__device__ __forceinline__ ffT<T> ff_sub(ffT<T> a, ffT<T> b) {
    T s, e;
    two_diff(a.hi, b.hi, s, e);
    e = o_add(e, o_sub(a.lo, b.lo));
    return ff_renorm(s, e);
}
// product, error terms folded with FMA (Dekker TwoProduct via FMA)
template <class T>
__device__ __forceinline__ ffT<T> ff_mul(ffT<T> a, ffT<T> b) {
    const T p = o_mul(a.hi, b.hi);
    T e = o_fma(a.hi, b.hi, o_neg(p));
    e = o_fma(a.hi, b.lo, e);
    e = o_fma(a.lo, b.hi, e);
    return ff_renorm(p, e);
}
template <class T>
__device__ __forceinline__ ffT<T> ff_mul_f(ffT<T> a, T b) {
    const T p = o_mul(a.hi, b);
    T e = o_fma(a.hi, b, o_neg(p));
    e = o_fma(a.lo, b, e);
    return ff_renorm(p, e);
}
template <class T>
__device__ __forceinline__ ffT<T> ff_sqr(ffT<T> a) {
    const T p = o_mul(a.hi, a.hi);
    T e = o_fma(a.hi, a.hi, o_neg(p));
    e = o_fma(o_add(a.hi, a.hi), a.lo, e);
    return ff_renorm(p, e);
}
// acc += a * b, product and sum kept exact to float-float accuracy
template <class T>
__device__ __forceinline__ void ff_fma_acc(ffT<T> &acc, ffT<T> a, ffT<T> b) {
    const T p = o_mul(a.hi, b.hi);
    T pe = o_fma(a.hi, b.hi, o_neg(p));
    pe = o_fma(a.hi, b.lo, pe);
    pe = o_fma(a.lo, b.hi, pe);
    T s, e;
    two_sum(acc.hi, p, s, e);
    e = o_add(e, o_add(acc.lo, pe));
    acc = ff_renorm(s, e);
}
// a - b*c: the product's error terms folded by FMA, one renormalisation
template <class T>
__device__ __forceinline__ ffT<T> ff_fnma(ffT<T> b, ffT<T> c, ffT<T> a) {
    const T p = o_mul(b.hi, c.hi);
    T pe = o_fma(b.hi, c.hi, o_neg(p));
    pe = o_fma(b.hi, c.lo, pe);
    pe = o_fma(b.lo, c.hi, pe);
    T s, e;
    two_diff(a.hi, p, s, e);
    e = o_add(e, o_sub(a.lo, pe));
    return ff_renorm(s, e);
}
// dot products: high parts summed with exact TwoSum, all second-order terms
// gathered in one value, one renormalisation at the end.
template <class T>
__device__ __forceinline__ ffT<T> ff_dot3(const ffT<T> a[3], const ffT<T> b[3]) {
    T p0 = o_mul(a[0].hi, b[0].hi), p1 = o_mul(a[1].hi, b[1].hi), p2 = o_mul(a[2].hi, b[2].hi);
    T lo = o_fma(a[0].hi, b[0].hi, o_neg(p0));
    lo = o_add(o_fma(a[1].hi, b[1].hi, o_neg(p1)), lo);
    lo = o_add(o_fma(a[2].hi, b[2].hi, o_neg(p2)), lo);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo = o_fma(a[k].hi, b[k].lo, lo);
        lo = o_fma(a[k].lo, b[k].hi, lo);
    }
    T s, e;
    two_sum(p0, p1, s, e);
    lo = o_add(lo, e);
    two_sum(s, p2, s, e);
    lo = o_add(lo, e);
    return ff_renorm(s, lo);
}

// Lazy forms: the sum's high part takes the exact TwoSum, the low part
// gathers every error term, and renormalisation is left to the caller (once
// per j-tile for accumulators).  |lo| may reach a few ulps of |hi|; every
// consumer below folds lo into first-order terms only.
template <class T>
__device__ __forceinline__ void ff_fma_acc_lazy(ffT<T> &acc, ffT<T> a, ffT<T> b) {
    const T p = o_mul(a.hi, b.hi);
    T pe = o_fma(a.hi, b.hi, o_neg(p));
    pe = o_fma(a.hi, b.lo, pe);
    pe = o_fma(a.lo, b.hi, pe);
    T s, e;
    two_sum(acc.hi, p, s, e);
    acc.hi = s;
    acc.lo = o_add(acc.lo, o_add(e, pe));
}
template <class T>
__device__ __forceinline__ ffT<T> ff_mul_lazy(ffT<T> a, ffT<T> b) {
    const T p = o_mul(a.hi, b.hi);
    T e = o_fma(a.hi, b.hi, o_neg(p));
    e = o_fma(a.hi, b.lo, e);
    e = o_fma(a.lo, b.hi, e);
    return ffT<T>{p, e};
}
template <class T>
__device__ __forceinline__ ffT<T> ff_mul_f_lazy(ffT<T> a, T b) {
    const T p = o_mul(a.hi, b);
    T e = o_fma(a.hi, b, o_neg(p));
    e = o_fma(a.lo, b, e);
    return ffT<T>{p, e};
}
template <class T>
__device__ __forceinline__ ffT<T> ff_sqr_lazy(ffT<T> a) {
    const T p = o_mul(a.hi, a.hi);
    T e = o_fma(a.hi, a.hi, o_neg(p));
    e = o_fma(o_add(a.hi, a.hi), a.lo, e);
    return ffT<T>{p, e};
}
template <class T>
__device__ __forceinline__ ffT<T> ff_sum_lazy(ffT<T> a, ffT<T> b) {
    T s, e;
    two_sum(a.hi, b.hi, s, e);
    return ffT<T>{s, o_add(e, o_add(a.lo, b.lo))};
}
template <class T>
__device__ __forceinline__ void ff_add_lazy(ffT<T> &acc, ffT<T> b) {
    T s, e;
    two_sum(acc.hi, b.hi, s, e);
    acc.hi = s;
    acc.lo = o_add(acc.lo, o_add(e, b.lo));
}
template <class T>
__device__ __forceinline__ ffT<T> ff_fnma_lazy(ffT<T> b, ffT<T> c, ffT<T> a) {
    const T p = o_mul(b.hi, c.hi);
    T pe = o_fma(b.hi, c.hi, o_neg(p));
    pe = o_fma(b.hi, c.lo, pe);
    pe = o_fma(b.lo, c.hi, pe);
    T s, e;
    two_diff(a.hi, p, s, e);
    return ffT<T>{s, o_add(e, o_sub(a.lo, pe))};
}
// 1/sqrt(r2) in float-float: SFU seed y0, residual e = 1 - r2 y0^2 from the
// exact square of y0 and FMA-exact products, then y0 (1 + e/2 + 3e^2/8).
// Lazy form: y0 + corr as it is (|corr| ~ 2^-22 |y0|).  Domain: the normal
// FP32 range of r2.hi.
template <class T>
__device__ __forceinline__ ffT<T> rsqrt_ff(ffT<T> r2) {
    const T y0 = rsqrt_sfu(r2.hi);
    const T p = o_mul(y0, y0);
    const T pe = o_fma(y0, y0, o_neg(p));
    const T u = o_mul(r2.hi, p);
    T ue = o_fma(r2.hi, p, o_neg(u));
    ue = o_fma(r2.hi, pe, ue);
    ue = o_fma(r2.lo, p, ue);
    const T e = o_sub(o_sub(o_cst(y0, 1.0f), u), ue);
    const T corr = o_mul(o_mul(y0, e), o_fma(e, o_cst(y0, 0.375f), o_cst(y0, 0.5f)));
    if constexpr (NB_EX_LAZY) return ffT<T>{y0, corr};
    else return ff_renorm(y0, corr);
}

// A positive double y in [2^-74, 2^127] as a float pair, from its bits with
// no FP64 instruction and no int-to-float conversion: hi = the top 24
// significant bits (truncated), lo = the next 23 bits, an integer turned
// into a float by the 2^23 bias trick (exact) and scaled by 2^(E - 1069)
// (the remaining 6 bits dropped: the pair holds y to 2^-47).
__device__ __forceinline__ ff ff_from_pos_double(double y) {
    const int hi = __double2hiint(y);
    const int lo = __double2loint(y);
    const float yh = __int_as_float((int)__funnelshift_l((unsigned)lo, (unsigned)(hi - 0x38000000), 3));
    const float scale = __int_as_float(((hi & 0x7ff00000) - (942 << 20)) << 3);  // 2^(E - 1069)
    const float l23 = __fsub_rn(__int_as_float(0x4B000000 | (((unsigned)lo >> 6) & 0x7FFFFFu)),
                                8388608.0f);
    return ff{yh, __fmul_rn(l23, scale)};
}

// a.b, unnormalised (hi + lo with every error term in lo)
template <class T>
__device__ __forceinline__ ffT<T> ff_dot3_lazy(const ffT<T> a[3], const ffT<T> b[3]) {
    T p[3], lo;
#pragma unroll
    for (int k = 0; k < 3; ++k) p[k] = o_mul(a[k].hi, b[k].hi);
    lo = o_fma(a[0].hi, b[0].hi, o_neg(p[0]));
#pragma unroll
    for (int k = 1; k < 3; ++k) lo = o_add(o_fma(a[k].hi, b[k].hi, o_neg(p[k])), lo);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo = o_fma(a[k].hi, b[k].lo, lo);
        lo = o_fma(a[k].lo, b[k].hi, lo);
    }
    T s = p[0], e;
#pragma unroll
    for (int k = 1; k < 3; ++k) {
        two_sum(s, p[k], s, e);
        lo = o_add(lo, e);
    }
    return ffT<T>{s, lo};
}
// a0.b0 + a1.b1, unnormalised
template <class T>
__device__ __forceinline__ ffT<T> ff_dot3x2_lazy(const ffT<T> a0[3], const ffT<T> b0[3],
                                                 const ffT<T> a1[3], const ffT<T> b1[3]) {
    T p[6];
    T lo = o_cst(a0[0].hi, 0.f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        p[k] = o_mul(a0[k].hi, b0[k].hi);
        p[3 + k] = o_mul(a1[k].hi, b1[k].hi);
        lo = o_add(o_fma(a0[k].hi, b0[k].hi, o_neg(p[k])), lo);
        lo = o_add(o_fma(a1[k].hi, b1[k].hi, o_neg(p[3 + k])), lo);
        lo = o_fma(a0[k].hi, b0[k].lo, lo);
        lo = o_fma(a0[k].lo, b0[k].hi, lo);
        lo = o_fma(a1[k].hi, b1[k].lo, lo);
        lo = o_fma(a1[k].lo, b1[k].hi, lo);
    }
    T s = p[0], e;
#pragma unroll
    for (int k = 1; k < 6; ++k) {
        two_sum(s, p[k], s, e);
        lo = o_add(lo, e);
    }
    return ffT<T>{s, lo};
}
// a.b + c, unnormalised
template <class T>
__device__ __forceinline__ ffT<T> ff_dot3_add_lazy(const ffT<T> a[3], const ffT<T> b[3], ffT<T> c) {
    T p[3], lo = c.lo;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        p[k] = o_mul(a[k].hi, b[k].hi);
        lo = o_add(o_fma(a[k].hi, b[k].hi, o_neg(p[k])), lo);
        lo = o_fma(a[k].hi, b[k].lo, lo);
        lo = o_fma(a[k].lo, b[k].hi, lo);
    }
    T s = c.hi, e;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        two_sum(s, p[k], s, e);
        lo = o_add(lo, e);
    }
    return ffT<T>{s, lo};
}
// a.b + c, one renormalisation
template <class T>
__device__ __forceinline__ ffT<T> ff_dot3_add(const ffT<T> a[3], const ffT<T> b[3], ffT<T> c) {
    const ffT<T> r = ff_dot3_add_lazy(a, b, c);
    return ff_renorm(r.hi, r.lo);
}

// ------------------------------------------------------------ TMA / mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// 1-D bulk copy global -> shared (TMA engine), completion counted in bytes on bar.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false after kWaitBudgetNs without completion.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  unsigned long long budget_ns = kWaitBudgetNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > budget_ns) return false;
    }
}

// ------------------------------------------------------------ launchers
// (implemented in the kernel translation units)
cudaError_t launch_select_min(const Dev &d, cudaStream_t st);
cudaError_t launch_select_compact(const Dev &d, double unused, cudaStream_t st);
cudaError_t launch_predict(const Dev &d, int also64, int use_fixed_t, double t_fixed,
                           cudaStream_t st);
cudaError_t launch_pad(const Dev &d, cudaStream_t st);
cudaError_t launch_eval(const Dev &d, int mode, const EvalLaunch &L, int grid, cudaStream_t st);
cudaError_t launch_correct(const Dev &d, int64_t lo, int64_t hi, const int32_t *active,
                           int32_t n_active, double t_next, const double *ajs, cudaStream_t st);
cudaError_t launch_init_clear(const Dev &d, cudaStream_t st);
cudaError_t launch_energy(const Dev &d, int64_t begin, int64_t end, int blocks, cudaStream_t st);
int eval_occupancy(int precision, int mode);  // CTAs per SM

}  // namespace nb

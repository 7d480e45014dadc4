// nb_kernels.cu -- block-time selection, work planning, prediction, padding,
// stand-alone correction, start-up helpers and energy sums.
//
// Block scheduler (Makino 1991; the paper's Sec. 2 integrator lineage):
// t_next = min_i (t_i + dt_i) per cluster, active = {i : t_i + dt_i == t_next}
// in increasing index order.  Two passes over fixed chunks of kChunk
// particles (chunks never straddle clusters): pass 1 writes each chunk's
// minimum and how many of its particles reach it, and its last CTA (a
// counter) combines the chunk minima and counts of every cluster into the
// cluster's t_next and active count; pass 2 computes each chunk's offset from
// the counts of the cluster's earlier chunks and compacts its active
// particles in order.  The planner and the predictor need only t_next and the
// count, so they run beside pass 2.  The active list takes no atomics and is
// deterministic.
#include "nb_internal.cuh"
#include "nb_step.cuh"

namespace nb {

// ------------------------------------------------------------ block helpers
template <typename T, typename Op>
__device__ __forceinline__ T block_reduce(T v, Op op, T *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    for (int o = 16; o >= 1; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    T r = sm[0];
    for (int w = 1; w < nw; ++w) r = op(r, sm[w]);
    __syncthreads();
    return r;
}

struct MinOp {
    __device__ double operator()(double a, double b) const { return fmin(a, b); }
};
struct SumI {
    __device__ int operator()(int a, int b) const { return a + b; }
};

// -------------------------------------------------------------- select pass 1
__global__ void __launch_bounds__(kSelTPB) k_select_min(const Dev d) {
    __shared__ double smd[kSelTPB / 32];
    __shared__ int smi[kSelTPB / 32];
    const int k = blockIdx.x;
    const int64_t b = d.chunk_begin[k], e = d.chunk_end[k];
    double mn = INFINITY;
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) mn = fmin(mn, d.t[i] + d.dt[i]);
    mn = block_reduce(mn, MinOp(), smd);
    int cnt = 0;
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) cnt += (d.t[i] + d.dt[i] == mn);
    cnt = block_reduce(cnt, SumI(), smi);
    __shared__ int last;
    if (threadIdx.x == 0) {
        d.chunk_min[k] = mn;
        d.chunk_cnt[k] = cnt;
        __threadfence();
        last = atomicAdd(d.sel_ctr, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    // The last CTA: each cluster's t_next = the least chunk minimum, its
    // active count = the counts of the chunks that reach it.  A cluster of at
    // most kSelThread chunks is taken by one thread, one of at most kSelWarp
    // chunks by a warp (its lanes load the chunk values side by side), larger
    // ones by the whole CTA; clusters that find their list full fall back to
    // the tier below.
    __threadfence();
    constexpr int kSelThread = 8;
    constexpr int kSelWarp = 64;
    constexpr int kSelMid = 256;
    constexpr int kSelLarge = 64;
    __shared__ int mid[kSelMid];
    __shared__ int large[kSelLarge];
    __shared__ int n_mid, n_large;
    if (threadIdx.x == 0) n_mid = n_large = 0;
    __syncthreads();
    const double t_end = *d.t_end;
    for (int c = threadIdx.x; c < d.n_clusters; c += blockDim.x) {
        const int k0 = d.cluster_chunk0[c], k1 = d.cluster_chunk0[c + 1];
        if (k1 - k0 > kSelWarp) {
            const int slot = atomicAdd(&n_large, 1);
            if (slot < kSelLarge) {
                large[slot] = c;
                continue;
            }
        }
        if (k1 - k0 > kSelThread) {
            const int slot = atomicAdd(&n_mid, 1);
            if (slot < kSelMid) {
                mid[slot] = c;
                continue;
            }
        }
        double tn = INFINITY;
        for (int kk = k0; kk < k1; ++kk) tn = fmin(tn, __ldcg(&d.chunk_min[kk]));
        int total = 0;
        for (int kk = k0; kk < k1; ++kk)
            if (__ldcg(&d.chunk_min[kk]) == tn) total += __ldcg(&d.chunk_cnt[kk]);
        d.tnext[c] = tn;
        d.nact[c] = tn <= t_end ? total : 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int nm = n_mid < kSelMid ? n_mid : kSelMid;
    for (int q = threadIdx.x >> 5; q < nm; q += nwarps) {
        const int c = mid[q];
        const int k0 = d.cluster_chunk0[c], k1 = d.cluster_chunk0[c + 1];
        double tn = INFINITY;
        for (int kk = k0 + lane; kk < k1; kk += 32) tn = fmin(tn, __ldcg(&d.chunk_min[kk]));
        for (int o = 16; o >= 1; o >>= 1) tn = fmin(tn, __shfl_xor_sync(0xffffffffu, tn, o));
        int total = 0;
        for (int kk = k0 + lane; kk < k1; kk += 32)
            if (__ldcg(&d.chunk_min[kk]) == tn) total += __ldcg(&d.chunk_cnt[kk]);
        for (int o = 16; o >= 1; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
        if (lane == 0) {
            d.tnext[c] = tn;
            d.nact[c] = tn <= t_end ? total : 0;
        }
    }
    const int nl = n_large < kSelLarge ? n_large : kSelLarge;
    for (int q = 0; q < nl; ++q) {
        const int c = large[q];
        const int k0 = d.cluster_chunk0[c], k1 = d.cluster_chunk0[c + 1];
        double tn = INFINITY;
        for (int kk = k0 + threadIdx.x; kk < k1; kk += blockDim.x) tn = fmin(tn, __ldcg(&d.chunk_min[kk]));
        tn = block_reduce(tn, MinOp(), smd);
        int total = 0;
        for (int kk = k0 + threadIdx.x; kk < k1; kk += blockDim.x)
            if (__ldcg(&d.chunk_min[kk]) == tn) total += __ldcg(&d.chunk_cnt[kk]);
        total = block_reduce(total, SumI(), smi);
        if (threadIdx.x == 0) {
            d.tnext[c] = tn;
            d.nact[c] = tn <= t_end ? total : 0;
        }
    }
    if (threadIdx.x == 0) *d.sel_ctr = 0u;  // ready for the next pass
}

// -------------------------------------------------------------- select pass 2
__global__ void __launch_bounds__(kSelTPB) k_select_compact(const Dev d) {
    __shared__ int smi[kSelTPB / 32];
    __shared__ int warp_cnt[kSelTPB / 32];
    const int k = blockIdx.x;
    const int c = d.chunk_cluster[k];
    const int k0 = d.cluster_chunk0[c];
    // t_next and the count come from pass 1's last CTA
    const double tn = d.tnext[c];
    if (d.nact[c] == 0 || d.chunk_min[k] != tn) return;
    int before = 0;
    for (int kk = k0 + threadIdx.x; kk < k; kk += blockDim.x)
        if (d.chunk_min[kk] == tn) before += d.chunk_cnt[kk];
    before = block_reduce(before, SumI(), smi);
    const int64_t b = d.chunk_begin[k], e = d.chunk_end[k];
    int32_t *out = d.active + d.offsets[c] + before;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int base = 0;
    for (int64_t i0 = b; i0 < e; i0 += blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        const bool f = (i < e) && (d.t[i] + d.dt[i] == tn);
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) warp_cnt[warp] = __popc(bal);
        __syncthreads();
        int wbase = base;
        for (int w = 0; w < warp; ++w) wbase += warp_cnt[w];
        int round = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) round += warp_cnt[w];
        if (f) out[wbase + __popc(bal & ((1u << lane) - 1u))] = (int32_t)i;
        base += round;
        __syncthreads();
    }
}

// --------------------------------------------------------------------- plan
// Block-wide inclusive scan of one value per thread (Hillis-Steele).
__device__ __forceinline__ long long block_scan_incl(long long v, long long *sm) {
    const int tid = threadIdx.x;
    sm[tid] = v;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        const long long add = tid >= o ? sm[tid - o] : 0;
        __syncthreads();
        sm[tid] += add;
        __syncthreads();
    }
    const long long r = sm[tid];
    __syncthreads();
    return r;
}
__device__ __forceinline__ double block_sum_d(double v, double *sm) {
    const int tid = threadIdx.x;
    sm[tid] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o >= 1; o >>= 1) {
        if (tid < o) sm[tid] += sm[tid + o];
        __syncthreads();
    }
    const double r = sm[0];
    __syncthreads();
    return r;
}

// One CTA.  Per cluster: A -> bucket floor(log2 A) -> (gl, target items) ->
// i-tiles and split S (clamped to the cluster's j-tiles); exclusive scans
// give each cluster its first item and first tile.  If the items that need
// partial sums exceed the scratch capacity, every split falls back to 1.
// mode_init: every particle active (start-up and energy evaluations).
__global__ void __launch_bounds__(kPlanTPB) k_plan(const Dev d, int mode_init, int count) {
    __shared__ long long s_l[kPlanTPB];
    __shared__ double s_d[kPlanTPB];
    const int tid = threadIdx.x;
    for (int fallback = 0; fallback < 2; ++fallback) {
        long long carry_items = 0, carry_tiles = 0, carry_slots = 0;
        double inter = 0.0, busy = 0.0;
        for (int base = 0; base < d.n_clusters; base += (int)blockDim.x) {
            const int c = base + tid;
            ClusterPlan pl{1, 1, 0, 0, 0, 0, 0, 0, 0};
            long long items = 0, tiles = 0;
            double my_inter = 0.0;
            if (c < d.n_clusters) {
                const int64_t ncl = d.offsets[c + 1] - d.offsets[c];
                const int A = mode_init ? (int)ncl : d.nact[c];
                if (A > 0) {
                    const PlanEntry e = d.table[31 - __clz(A)];
                    tiles = cdiv(A, kTPB / e.gl);
                    const long long ntj = cdiv(ncl, kTJ);
                    if (d.n_clusters == 1 && !d.streamk_off &&
                        sk_use(tiles, kTPB / e.gl, ntj, d.grid_eval, d.partial_cap)) {
                        // one cluster, enough work: stream-K ranges (one "item")
                        items = 1;
                        pl = ClusterPlan{e.gl, 1, (int)tiles, A, 0, 0, 0, 1, 0};
                    } else {
                        const long long S =
                            fallback ? 1 : choose_split(tiles, ntj, e.target_items, d.grid_eval);
                        items = tiles * S;
                        pl = ClusterPlan{e.gl, (int)S, (int)tiles, A, 0, 0, 0, 0, 0};
                    }
                    my_inter = (double)A * (double)(ncl - 1);
                }
            }
            // partial sums: 10 doubles per i of every item of a split cluster
            const long long sitems = pl.split > 1 ? items * 10 * (kTPB / pl.gl) : 0;
            const long long ii = block_scan_incl(items, s_l);
            const long long it = block_scan_incl(tiles, s_l);
            const long long is = block_scan_incl(sitems, s_l);
            pl.item0 = carry_items + ii - items;
            pl.tile0 = carry_tiles + it - tiles;
            pl.pslot0 = carry_slots + is - sitems;
            if (c < d.n_clusters) d.plan[c] = pl;
            // the last thread holds the inclusive totals
            if (tid == (int)blockDim.x - 1) {
                s_l[0] = ii;
                s_l[1] = it;
                s_l[2] = is;
            }
            __syncthreads();
            carry_items += s_l[0];
            carry_tiles += s_l[1];
            carry_slots += s_l[2];
            __syncthreads();
            inter += block_sum_d(my_inter, s_d);
            busy += block_sum_d(pl.active > 0 ? 1.0 : 0.0, s_d);
        }
        // the split items' partial sums must fit the scratch (uniform decision)
        if (!fallback && carry_slots > d.partial_cap) continue;
        if (tid == 0) {
            *d.n_items = carry_items;
            *d.item_ctr = 0ull;
            *d.busy = (int)busy;
            if (count && !mode_init) {
                *d.ctr_steps += (unsigned long long)busy;
                *d.ctr_inter += inter;
            }
        }
        break;
    }
}

// ---------------------------------------------------------------- predictor
__device__ __forceinline__ void split_ff(double x, float &hi, float &lo) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
}

__global__ void __launch_bounds__(kSelTPB) k_predict(const Dev d, int also64, int use_fixed,
                                                     double t_fixed) {
    // kChunk / kSelTPB CTAs per chunk: one particle per thread, all SMs busy
    constexpr int kSub = kChunk / kSelTPB;
    const int k = blockIdx.x / kSub;
    const int c = d.chunk_cluster[k];
    if (!use_fixed && d.nact[c] == 0) return;  // idle cluster this step
    const double tn = use_fixed ? t_fixed : d.tnext[c];
    const int64_t off = d.offsets[c];
    const int64_t jo = d.jofs[c];
    const int64_t b = d.chunk_begin[k] + (int64_t)(blockIdx.x % kSub) * kSelTPB, e = d.chunk_end[k];
    for (int64_t i = b + threadIdx.x; i < e && i < b + kSelTPB; i += blockDim.x) {
        double xp[3], vp[3], ap[3];
        predict_particle(d, i, tn, xp, vp, ap);
        const double m = d.m[i];
        const int64_t jx = jo + (i - off);
        if (d.precision == NB_FP64 || also64) {
            J64 w;
            w.q[0] = make_double2(xp[0], xp[1]);
            w.q[1] = make_double2(xp[2], m);
            w.q[2] = make_double2(vp[0], vp[1]);
            w.q[3] = make_double2(vp[2], ap[0]);
            w.q[4] = make_double2(ap[1], ap[2]);
            j64_set_mass_split(w, m);
            d.jarr64[jx] = w;
        }
        if (d.precision == NB_EX || d.precision == NB_FP32X) {
            float xh[3], xl[3], vh[3], vl[3], ah[3], al[3], mh, ml;
            for (int q = 0; q < 3; ++q) {
                split_ff(xp[q], xh[q], xl[q]);
                split_ff(vp[q], vh[q], vl[q]);
                split_ff(ap[q], ah[q], al[q]);
            }
            split_ff(m, mh, ml);
            const float w[kJEXVals] = {xh[0], xh[1], xh[2], mh, xl[0], xl[1], xl[2], ml,
                                       vh[0], vh[1], vh[2], ah[0], vl[0], vl[1], vl[2], al[0],
                                       ah[1], ah[2], al[1], al[2]};
            jpair_store<kJEXVals>(d.jarr, jx, w);
        } else if (d.precision == NB_FP32) {
            float xh[3], xl[3], vh[3], vl[3];
            for (int q = 0; q < 3; ++q) {
                split_ff(xp[q], xh[q], xl[q]);
                split_ff(vp[q], vh[q], vl[q]);
            }
            const float w[kJ32Vals] = {xh[0], xh[1], xh[2], __double2float_rn(m),
                                       xl[0], xl[1], xl[2], __double2float_rn(ap[0]),
                                       vh[0], vh[1], vh[2], __double2float_rn(ap[1]),
                                       vl[0], vl[1], vl[2], __double2float_rn(ap[2])};
            jpair_store<kJ32Vals>(d.jarr, jx, w);
        }
    }
}

// Padding j-entries (beyond each cluster's size, up to a whole tile): zero
// mass at a far point, so their pair terms are exactly zero.
__global__ void k_pad(const Dev d) {
    const int c = blockIdx.x;
    const int64_t ncl = d.offsets[c + 1] - d.offsets[c];
    const int64_t jo = d.jofs[c];
    const int64_t jend = d.jofs[c + 1];
    const double far = 1.0e6;
    for (int64_t jx = jo + ncl + threadIdx.x; jx < jend; jx += blockDim.x) {
        J64 w;
        w.q[0] = make_double2(far, far);
        w.q[1] = make_double2(far, 0.0);
        w.q[2] = w.q[3] = w.q[4] = make_double2(0.0, 0.0);
        j64_set_mass_split(w, 0.0);
        d.jarr64[jx] = w;
        if (d.precision == NB_EX || d.precision == NB_FP32X) {
            float w[kJEXVals] = {};
            w[0] = w[1] = w[2] = (float)far;
            jpair_store<kJEXVals>(d.jarr, jx, w);
        } else if (d.precision == NB_FP32) {
            float w[kJ32Vals] = {};
            w[0] = w[1] = w[2] = (float)far;
            jpair_store<kJ32Vals>(d.jarr, jx, w);
        }
    }
}

// ------------------------------------------------------ stand-alone corrector
__global__ void k_correct(const Dev d, const int32_t *active, int32_t n_active, double t_next,
                          const double *ajs, int64_t lo, int64_t hi) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_active) return;
    const int64_t i = active[k];
    if (i < lo || i >= hi) {  // outside the cluster: reject, touch nothing
        atomicOr(d.err, kErrIndex);
        return;
    }
    double o[10];
    for (int q = 0; q < 10; ++q) o[q] = ajs[(int64_t)q * n_active + k];
    if (d.order == 4) correct_particle4(d, i, t_next, o);
    else correct_particle(d, i, t_next, o);
}

// ---------------------------------------------------------------- start-up
__global__ void k_init_clear(const Dev d) {
    const int64_t n = d.n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < 3; ++k) {
            d.a[k * n + i] = 0.0;
            d.j[k * n + i] = 0.0;
            d.s[k * n + i] = 0.0;
            d.c[k * n + i] = 0.0;
        }
        d.t[i] = 0.0;
    }
}

// ------------------------------------------------------------------ energy
// Per chunk: 1/2 m v^2, 1/2 m pot, m v, m x cross v of the particles in
// [begin, end) from the FP64 predicted array; the host adds the chunk sums
// in chunk order.
__global__ void __launch_bounds__(kSelTPB) k_energy(const Dev d, int64_t begin, int64_t end) {
    __shared__ double sm[kSelTPB / 32];
    const int k = blockIdx.x;
    const int c = d.chunk_cluster[k];
    const int64_t off = d.offsets[c], jo = d.jofs[c];
    const int64_t b = d.chunk_begin[k], e = d.chunk_end[k];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
        if (i < begin || i >= end) continue;
        const J64 w = d.jarr64[jo + (i - off)];
        const double x = w.q[0].x, y = w.q[0].y, z = w.q[1].x, m = w.q[1].y;
        const double vx = w.q[2].x, vy = w.q[2].y, vz = w.q[3].x;
        acc[0] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        acc[1] += 0.5 * m * d.pot_tmp[i];
        acc[2] += m * vx;
        acc[3] += m * vy;
        acc[4] += m * vz;
        acc[5] += m * (y * vz - z * vy);
        acc[6] += m * (z * vx - x * vz);
        acc[7] += m * (x * vy - y * vx);
    }
    struct Add {
        __device__ double operator()(double a, double b) const { return a + b; }
    };
    for (int q = 0; q < 8; ++q) {
        const double r = block_reduce(acc[q], Add(), sm);
        if (threadIdx.x == 0) d.energy_part[(int64_t)k * 8 + q] = r;
    }
}

// FP64 predicted values to the caller's [10][n] layout (nb_predict output).
__global__ void __launch_bounds__(kSelTPB) k_unpack64(const Dev d, double *out) {
    const int k = blockIdx.x;
    const int c = d.chunk_cluster[k];
    const int64_t off = d.offsets[c], jo = d.jofs[c], n = d.n;
    for (int64_t i = d.chunk_begin[k] + threadIdx.x; i < d.chunk_end[k]; i += blockDim.x) {
        const J64 w = d.jarr64[jo + (i - off)];
        const double v[10] = {w.q[0].x, w.q[0].y, w.q[1].x, w.q[2].x, w.q[2].y,
                              w.q[3].x, w.q[3].y, w.q[4].x, w.q[4].y, w.q[1].y};
        for (int q = 0; q < 10; ++q) out[q * n + i] = v[q];
    }
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_select_min(const Dev &d, cudaStream_t st) {
    k_select_min<<<d.n_chunks, kSelTPB, 0, st>>>(d);
    return cudaGetLastError();
}
cudaError_t launch_select_compact(const Dev &d, double, cudaStream_t st) {
    k_select_compact<<<d.n_chunks, kSelTPB, 0, st>>>(d);
    return cudaGetLastError();
}
cudaError_t launch_plan_ex(const Dev &d, int mode_init, int count, cudaStream_t st) {
    // a power of two >= the cluster count (the scans assume it), 32..1024
    int threads = 32;
    while (threads < d.n_clusters && threads < kPlanTPB) threads *= 2;
    k_plan<<<1, threads, 0, st>>>(d, mode_init, count);
    return cudaGetLastError();
}
cudaError_t launch_unpack64(const Dev &d, double *out, cudaStream_t st) {
    k_unpack64<<<d.n_chunks, kSelTPB, 0, st>>>(d, out);
    return cudaGetLastError();
}
cudaError_t launch_predict(const Dev &d, int also64, int use_fixed, double t_fixed,
                           cudaStream_t st) {
    k_predict<<<d.n_chunks * (kChunk / kSelTPB), kSelTPB, 0, st>>>(d, also64, use_fixed, t_fixed);
    return cudaGetLastError();
}
cudaError_t launch_pad(const Dev &d, cudaStream_t st) {
    k_pad<<<d.n_clusters, 64, 0, st>>>(d);
    return cudaGetLastError();
}
cudaError_t launch_correct(const Dev &d, int64_t lo, int64_t hi, const int32_t *active,
                           int32_t n_active, double t_next, const double *ajs, cudaStream_t st) {
    if (n_active <= 0) return cudaSuccess;
    k_correct<<<(unsigned)cdiv(n_active, 128), 128, 0, st>>>(d, active, n_active, t_next, ajs, lo, hi);
    return cudaGetLastError();
}
cudaError_t launch_init_clear(const Dev &d, cudaStream_t st) {
    const int blocks = (int)(cdiv(d.n, 256) < 4096 ? cdiv(d.n, 256) : 4096);
    k_init_clear<<<blocks, 256, 0, st>>>(d);
    return cudaGetLastError();
}
cudaError_t launch_energy(const Dev &d, int64_t begin, int64_t end, int, cudaStream_t st) {
    k_energy<<<d.n_chunks, kSelTPB, 0, st>>>(d, begin, end);
    return cudaGetLastError();
}

}  // namespace nb

// plan_check.cu -- host-only checks of the work-planning arithmetic shared by
// the evaluation kernel and its planners (stream-K ranges, split choice), and
// of the host-formed launch parameters (eps^2 as a float-float pair).
// Runs on the CPU: it makes no CUDA call.  Prints "ok <cases>" or the first
// violated property and exits non-zero.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_1812_00367_gb300/csrc/nb_internal.cuh"

using namespace nb;

static uint64_t rng_state = 0x9e3779b97f4a7c15ull;
static uint64_t next_u64() {  // splitmix64
    uint64_t z = (rng_state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
static int64_t uniform(int64_t lo, int64_t hi) { return lo + (int64_t)(next_u64() % (uint64_t)(hi - lo + 1)); }

#define CHECK(cond, ...)                                   \
    do {                                                   \
        if (!(cond)) {                                     \
            std::printf("FAIL %s: ", #cond);               \
            std::printf(__VA_ARGS__);                      \
            std::printf("\n");                             \
            std::exit(1);                                  \
        }                                                  \
    } while (0)

// Every unit in exactly one CTA range; every piece's slot unique and within
// G * max_pieces; the CTAs meeting an i-tile are consecutive, each holds one
// piece of it, and their number is what the kernel counts.
static void check_streamk(int64_t tiles, int64_t ntj, int64_t G) {
    const int64_t U = tiles * ntj;
    const int64_t maxp = sk_max_pieces(U, G, ntj);
    std::vector<int> cover(U, 0);
    std::vector<char> slot_used(G * maxp, 0);
    std::vector<int64_t> pieces(tiles, 0), first_k(tiles, -1), last_k(tiles, -1);
    for (int64_t k = 0; k < G; ++k) {
        int64_t p = sk_begin(U, G, k);
        const int64_t e = sk_begin(U, G, k + 1);
        CHECK(e > p, "empty range k=%lld U=%lld G=%lld", (long long)k, (long long)U, (long long)G);
        CHECK(sk_owner(U, G, p) == k && sk_owner(U, G, e - 1) == k, "owner k=%lld", (long long)k);
        while (p < e) {
            const int64_t t = p / ntj, tb = p - t * ntj;
            const int64_t te = std::min(ntj, tb + (e - p));
            for (int64_t u = t * ntj + tb; u < t * ntj + te; ++u) cover[u]++;
            const int64_t loc = t - sk_begin(U, G, k) / ntj;
            CHECK(loc >= 0 && loc < maxp, "local tile %lld of %lld", (long long)loc, (long long)maxp);
            CHECK(!slot_used[k * maxp + loc], "slot reused");
            slot_used[k * maxp + loc] = 1;
            if (first_k[t] < 0) first_k[t] = k;
            CHECK(last_k[t] < 0 || last_k[t] == k - 1, "CTAs of tile %lld not consecutive", (long long)t);
            last_k[t] = k;
            pieces[t]++;
            p += te - tb;
        }
    }
    for (int64_t u = 0; u < U; ++u) CHECK(cover[u] == 1, "unit %lld covered %d times", (long long)u, cover[u]);
    for (int64_t t = 0; t < tiles; ++t) {
        const int64_t f = sk_owner(U, G, t * ntj), l = sk_owner(U, G, (t + 1) * ntj - 1);
        CHECK(f == first_k[t] && l == last_k[t] && l - f + 1 == pieces[t], "pieces of tile %lld", (long long)t);
        // the first piece's local slot, the others at local slot 0
        for (int64_t k = f + 1; k <= l; ++k) CHECK(t - sk_begin(U, G, k) / ntj == 0, "later piece not local 0");
    }
}

// The split chooser's choice by exhaustive search: every S of the window,
// the smallest of the best wave efficiency.
static int64_t split_by_scan(int64_t tiles, int64_t ntj, int64_t target, int64_t grid) {
    const int64_t smax = std::max<int64_t>(1, ntj / kMinTilesPerItem);
    const int64_t s0 = std::min(std::max<int64_t>(1, cdiv(target, tiles)), smax);
    const int64_t lo = std::max<int64_t>(1, s0 / 2), hi = std::min(2 * s0, smax);
    int64_t best = s0, bi = 0, bs = 1;
    for (int64_t s = lo; s <= hi; ++s) {
        const int64_t items = tiles * s, slots = cdiv(items, grid) * grid;
        if (items * bs > bi * slots) {
            bi = items;
            bs = slots;
            best = s;
        }
    }
    return best;
}

// S in [1, ntj / kMinTilesPerItem] (or 1), within [S0/2, 2 S0] of the target's
// S0, and no S in that window fills whole waves better; the same S as an
// exhaustive scan of the window.
static void check_split(int64_t tiles, int64_t ntj, int64_t target, int64_t grid) {
    const int64_t S = choose_split(tiles, ntj, target, grid);
    CHECK(S == split_by_scan(tiles, ntj, target, grid), "S=%lld scan %lld (tiles %lld ntj %lld target %lld grid %lld)",
          (long long)S, (long long)split_by_scan(tiles, ntj, target, grid), (long long)tiles,
          (long long)ntj, (long long)target, (long long)grid);
    const int64_t smax = std::max<int64_t>(1, ntj / kMinTilesPerItem);
    CHECK(S >= 1 && S <= smax, "S=%lld smax=%lld", (long long)S, (long long)smax);
    int64_t s0 = std::min(std::max<int64_t>(1, cdiv(target, tiles)), smax);
    const int64_t lo = std::max<int64_t>(1, s0 / 2), hi = std::min(2 * s0, smax);
    CHECK(S >= lo && S <= hi, "S=%lld outside [%lld, %lld]", (long long)S, (long long)lo, (long long)hi);
    const double eff = (double)(tiles * S) / (double)(cdiv(tiles * S, grid) * grid);
    for (int64_t s = lo; s <= hi; ++s) {
        const double e = (double)(tiles * s) / (double)(cdiv(tiles * s, grid) * grid);
        CHECK(e <= eff + 1e-12, "S=%lld eff %.6f beaten by s=%lld eff %.6f", (long long)S, eff, (long long)s, e);
        if (e == eff) {
            CHECK(s >= S, "not the smallest best S");
            break;
        }
    }
}

// eps^2 as the single-precision kernels read it: hi = fl32(eps^2), lo the
// float nearest the remainder, both lanes equal; the pair holds eps^2 to
// within half an ulp of lo (about 2^-48 relative) and is normalised.
static void check_eps2(double eps) {
    Dev d{};
    set_eps2(d, eps);
    const double e2 = eps * eps;
    CHECK(d.eps2 == e2, "eps %.17g", eps);
    CHECK(d.eps2_hi2.x == (float)e2 && d.eps2_hi2.y == d.eps2_hi2.x, "hi of eps %.17g", eps);
    CHECK(d.eps2_lo2.y == d.eps2_lo2.x, "lo lanes of eps %.17g", eps);
    const double hi = d.eps2_hi2.x, lo = d.eps2_lo2.x;
    CHECK(std::fabs(lo) <= 0.5 * std::ldexp(1.0, std::ilogb(hi > 0 ? hi : 1.0) - 23) || hi == 0.0,
          "lo not below half an ulp of hi, eps %.17g", eps);
    CHECK(std::fabs(hi + lo - e2) <= std::ldexp(std::fabs(e2), -47), "pair error, eps %.17g: %.3g", eps,
          std::fabs(hi + lo - e2) / e2);
}

int main() {
    int cases = 0;
    for (double eps : {0.0, 1e-5, 1e-4, 1e-3, 1e-2, 0.1, 1.0}) {
        check_eps2(eps);
        ++cases;
    }
    // eps^2 in [2^-100, 2^100], where lo (about 2^-24 eps^2) is a normal float
    for (int r = 0; r < 2000; ++r) {
        check_eps2(std::exp2(-50.0 + 100.0 * (double)(next_u64() >> 11) * 0x1.0p-53));
        ++cases;
    }
    const int64_t grids[] = {152, 456, 608, 1216};
    // fixed shapes of the benchmark system, then random ones
    const int64_t fixed[][2] = {{512, 1024}, {299, 1024}, {67, 1024}, {3, 1024}, {16, 257}, {1000, 3}};
    for (auto &f : fixed)
        for (int64_t G : grids)
            if (f[0] * f[1] >= kStreamKMinUnits * G) {
                check_streamk(f[0], f[1], G);
                ++cases;
            }
    for (int r = 0; r < 400; ++r) {
        const int64_t tiles = uniform(1, 2000), ntj = uniform(1, 1500), G = grids[uniform(0, 3)];
        if (tiles * ntj >= kStreamKMinUnits * G) {
            check_streamk(tiles, ntj, G);
            ++cases;
        }
        check_split(tiles, ntj, uniform(1, 16 * G), G);
        ++cases;
    }
    // the shapes of tiny active sets against large clusters (the planner's
    // common case in block steps): one to a few i-tiles, many j-tiles
    for (int r = 0; r < 2000; ++r) {
        const int64_t G = grids[uniform(0, 3)];
        check_split(uniform(1, 64), uniform(1, 70000), uniform(1, 16 * G), G);
        ++cases;
    }
    std::printf("ok %d\n", cases);
    return 0;
}

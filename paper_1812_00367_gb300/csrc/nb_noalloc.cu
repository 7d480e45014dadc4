// nb_noalloc.cu -- nb_evaluate_noalloc: the FP64 evaluation for callers that
// cannot allocate device memory (see include/nb.h).
//
// All scratch lives in one file-scope static __device__ arena: the packed,
// padded j-array, the split partial sums, the i-tile counters and a small
// header (cluster offsets and an error word).  Host code never uses the
// arena's symbol as an address: on the first call on each device (with that
// device current) it asks the runtime for the device address once and keeps
// it.  Every call reuses the same arena, so calls that overlap on the GPU
// race; each call clears what must start at zero (tile counters, error word).
#include <mutex>
#include <string>

#include "nb_eval.cuh"

namespace nb {
cudaError_t launch_eval_fp64(const Dev &, int, const EvalLaunch &, int, cudaStream_t);
int occupancy_fp64(int);
void set_global_error(const char *msg);

namespace {
constexpr int64_t kNaMaxN = 32768;       // particles (and active entries) per call
constexpr int64_t kNaMaxItems = 256;     // work items that keep split partial sums
constexpr int64_t kNaMaxTiles = kNaMaxN / 4 + 64;  // i-tiles (at least 4 i per tile)

constexpr size_t kNaJarrBytes = (size_t)kNaMaxN * sizeof(J64);
constexpr size_t kNaPartBytes = (size_t)kNaMaxItems * 10 * kTPB * sizeof(double);
constexpr size_t kNaTileBytes = (size_t)kNaMaxTiles * sizeof(int32_t);
constexpr size_t kNaOffJarr = 0;
constexpr size_t kNaOffPart = kNaOffJarr + kNaJarrBytes;
constexpr size_t kNaOffTile = kNaOffPart + kNaPartBytes;
constexpr size_t kNaOffAux = kNaOffTile + ((kNaTileBytes + 255) / 256) * 256;
constexpr size_t kNaBytes = kNaOffAux + 256;  // about 5.8 MB in all

struct NaAux {
    int64_t offsets[2];
    int64_t jofs[2];
    uint32_t err;
};

static __device__ __align__(256) unsigned char g_na_scratch[kNaBytes];

struct DevSlot {
    unsigned char *base = nullptr;
    int grid = 0;
};
std::mutex g_na_mutex;
DevSlot g_na_slots[128];

// Pack the caller's [10][n] predicted values into J64 entries (96 bytes:
// position, mass, velocity, acceleration and the mass as a float pair), pad to
// whole 64-particle tiles with zero-mass particles far away, clear the tile
// counters and the error word, and write the one-cluster offsets.
__global__ void k_na_prepare(unsigned char *base, const double *jp, int64_t n, int64_t npad,
                             int64_t tiles) {
    J64 *jarr = reinterpret_cast<J64 *>(base + kNaOffJarr);
    int32_t *tc = reinterpret_cast<int32_t *>(base + kNaOffTile);
    NaAux *aux = reinterpret_cast<NaAux *>(base + kNaOffAux);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = i0; i < npad; i += stride) {
        J64 w;
        if (i < n) {
            w.q[0] = make_double2(jp[0 * n + i], jp[1 * n + i]);
            w.q[1] = make_double2(jp[2 * n + i], jp[9 * n + i]);
            w.q[2] = make_double2(jp[3 * n + i], jp[4 * n + i]);
            w.q[3] = make_double2(jp[5 * n + i], jp[6 * n + i]);
            w.q[4] = make_double2(jp[7 * n + i], jp[8 * n + i]);
            j64_set_mass_split(w, jp[9 * n + i]);
        } else {
            w.q[0] = make_double2(1.0e6, 1.0e6);
            w.q[1] = make_double2(1.0e6, 0.0);
            w.q[2] = w.q[3] = w.q[4] = make_double2(0.0, 0.0);
            j64_set_mass_split(w, 0.0);
        }
        jarr[i] = w;
    }
    for (int64_t k = i0; k < tiles; k += stride) tc[k] = 0;
    if (i0 == 0) {
        aux->offsets[0] = 0;
        aux->offsets[1] = n;
        aux->jofs[0] = 0;
        aux->jofs[1] = npad;
        aux->err = 0;
    }
}
}  // namespace
}  // namespace nb

using namespace nb;

extern "C" nb_status nb_evaluate_noalloc(const double *jpred, int64_t n, double eps,
                                         const int32_t *active, int32_t n_active, double *out,
                                         void *stream) {
    if (n < 1 || n > kNaMaxN) {
        set_global_error("nb_evaluate_noalloc: n must be in [1, 32768]");
        return NB_EINVAL;
    }
    if (n_active < 0 || n_active > kNaMaxN) {
        set_global_error("nb_evaluate_noalloc: n_active must be in [0, 32768]");
        return NB_EINVAL;
    }
    if (!(eps >= 0.0) || !(eps < INFINITY)) {
        set_global_error("nb_evaluate_noalloc: eps must be finite and >= 0");
        return NB_EINVAL;
    }
    if (n_active == 0) return NB_OK;
    if (!jpred || !active || !out) {
        set_global_error("nb_evaluate_noalloc: NULL pointer");
        return NB_EINVAL;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
        set_global_error("nb_evaluate_noalloc: no usable current device");
        return NB_ECUDA;
    }
    DevSlot slot;
    {
        std::lock_guard<std::mutex> lk(g_na_mutex);
        if (!g_na_slots[dev].base) {  // first call on this device: set-up
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
            if (e != cudaSuccess || !p) {
                set_global_error("nb_evaluate_noalloc: cudaGetSymbolAddress failed");
                return NB_ECUDA;
            }
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
                set_global_error("nb_evaluate_noalloc: device query failed");
                return NB_ECUDA;
            }
            g_na_slots[dev].base = static_cast<unsigned char *>(p);
            g_na_slots[dev].grid = (occupancy_fp64(kModeOut) > 0 ? occupancy_fp64(kModeOut) : 1) * sms;
        }
        slot = g_na_slots[dev];
    }
    // plan: lanes per i from the active-set size, splits within the arena
    const int gl = n_active < 64 ? 32 : (n_active < 1024 ? 8 : (n_active < 4096 ? 2 : 1));
    const int tiles = (int)cdiv(n_active, kTPB / gl);
    const int64_t ntj = cdiv(n, kTJ);
    int64_t split = choose_split(tiles, ntj, 8LL * slot.grid, slot.grid);
    const int64_t per_item = 10LL * (kTPB / gl);         // partial doubles per item
    const int64_t cap = kNaMaxItems * 10LL * kTPB;        // arena partial doubles
    if (split > 1 && (int64_t)tiles * split * per_item > cap)
        split = cap / (per_item * tiles) > 1 ? cap / (per_item * tiles) : 1;

    // an error left pending by earlier, unrelated work is reported as such,
    // not as a failure of this call's launches
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_global_error((std::string("nb_evaluate_noalloc: CUDA error pending before the call: ") +
                          cudaGetErrorString(e)).c_str());
        return NB_ECUDA;
    }
    // entries whose index is rejected are skipped by the kernel: they read 0
    e = cudaMemsetAsync(out, 0, sizeof(double) * 10 * (size_t)n_active, st);
    if (e == cudaSuccess) {
        k_na_prepare<<<(unsigned)cdiv(ntj * kTJ, 256), 256, 0, st>>>(slot.base, jpred, n,
                                                                      ntj * kTJ, tiles);
        e = cudaGetLastError();
    }
    NaAux *aux = reinterpret_cast<NaAux *>(slot.base + kNaOffAux);
    Dev d{};
    d.n = n;
    d.n_clusters = 1;
    d.n_chunks = 0;
    d.precision = NB_FP64;
    d.grid_eval = slot.grid;
    d.offsets = aux->offsets;
    d.jofs = aux->jofs;
    d.jarr = slot.base + kNaOffJarr;
    d.jarr64 = reinterpret_cast<J64 *>(slot.base + kNaOffJarr);
    d.partial = reinterpret_cast<double *>(slot.base + kNaOffPart);
    d.partial_cap = kNaMaxItems * 10 * kTPB;  // doubles
    d.tile_cnt = reinterpret_cast<int32_t *>(slot.base + kNaOffTile);
    d.err = &aux->err;
    set_eps2(d, eps);
    d.neg_one = -1.0;
    d.neg_zero = -0.0;
    EvalLaunch L{};
    L.direct = 1;
    L.cluster = 0;
    L.n_active = n_active;
    L.gl = gl;
    L.split = (int)split;
    L.tiles = tiles;
    L.active = active;
    L.out = out;
    const int grid = (int)((int64_t)tiles * split < slot.grid ? (int64_t)tiles * split : slot.grid);
    if (e == cudaSuccess) e = launch_eval_fp64(d, kModeOut, L, grid, st);
    uint32_t err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &aux->err, sizeof(err), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_global_error(cudaGetErrorString(e));
        return NB_ECUDA;
    }
    if (err & kErrTimeout) {
        set_global_error("nb_evaluate_noalloc: a bounded device-side wait timed out");
        return NB_ETIMEOUT;
    }
    if (err & kErrIndex) {
        set_global_error("nb_evaluate_noalloc: an active index lies outside [0, n)");
        return NB_EINVAL;
    }
    return NB_OK;
}

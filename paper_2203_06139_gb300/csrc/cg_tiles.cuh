// cg_tiles.cuh -- tile grid of the fused kernels: a tile is (parameter
// point, contiguous chunk of elements); a persistent grid of (#SMs x
// resident CTAs) blocks walks the tiles round-robin and writes one partial
// vector per tile, summed later in chunk order by a finalize kernel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <mutex>
#include <unordered_map>

#include "cg_internal.cuh"
#include "cg_models.cuh"

namespace cg {

static constexpr int kMaxTiles = 16384;

// Resident blocks per SM of a kernel on the current device, cached per
// (device, kernel, threads, dynamic shared memory): the figure depends on the
// device's limits, so a process driving several GPUs keeps one per device.
inline int resident_blocks(const void* fn, int threads, size_t smem) {
    struct Key {
        int dev;
        const void* fn;
        int threads;
        size_t smem;
        bool operator==(const Key& o) const {
            return dev == o.dev && fn == o.fn && threads == o.threads && smem == o.smem;
        }
    };
    struct Hash {
        size_t operator()(const Key& k) const {
            return std::hash<const void*>()(k.fn) ^ ((size_t)k.dev << 1) ^ ((size_t)k.threads << 8) ^ (k.smem << 20);
        }
    };
    static std::mutex mu;
    static std::unordered_map<Key, int, Hash> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
    const Key key{dev, fn, threads, smem};
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int r = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, fn, threads, smem) != cudaSuccess || r < 1) r = 1;
    cache[key] = r;
    return r;
}

inline int max_nbx(int64_t n_theta) {
    int64_t m = (kMaxTiles + n_theta - 1) / n_theta;
    return (int)(m < 1 ? 1 : m);
}

// Choose the tile grid: among chunk counts per point that keep at least 8
// elements per thread per tile (and the workspace bound), the one whose tile
// count best fills whole waves of the persistent grid (every CTA gets the
// same number of tiles), preferring about 4 waves; chunk a multiple of
// 2*NT (keeps 16-byte alignment).
inline TileGrid make_tiles(int64_t n_elem, int64_t n_theta, int NT, int grid_blocks) {
    TileGrid tg;
    tg.n_elem = n_elem;
    const int64_t per_tile_min = (int64_t)NT * 8;
    int64_t most = (n_elem + per_tile_min - 1) / per_tile_min;
    if (most > max_nbx(n_theta)) most = max_nbx(n_theta);
    if (most < 1) most = 1;
    const int64_t G = grid_blocks > 0 ? grid_blocks : 1;
    int64_t best = 1;
    double best_score = -1.0;
    for (int64_t nbx = 1; nbx <= most; ++nbx) {
        // the chunk that nbx implies (rounded to 2*NT) and the tile count it really gives
        int64_t chunk = (n_elem + nbx - 1) / nbx;
        chunk = (chunk + 2 * NT - 1) / (2 * NT) * (2 * NT);
        const int64_t real = (n_elem + chunk - 1) / chunk;
        if (real != nbx) continue;
        const int64_t nt = n_theta * nbx;
        const int64_t waves = (nt + G - 1) / G;
        const double eff = (double)nt / (double)(waves * G);
        const double score = eff - 0.002 * (double)(waves > 4 ? waves - 4 : 4 - waves);
        if (score > best_score + 1e-12) {
            best_score = score;
            best = nbx;
        }
    }
    int64_t chunk = (n_elem + best - 1) / best;
    chunk = (chunk + 2 * NT - 1) / (2 * NT) * (2 * NT);
    if (chunk < 2 * NT) chunk = 2 * NT;
    int64_t nbx = (n_elem + chunk - 1) / chunk;
    if (nbx < 1) nbx = 1;
    tg.chunk = chunk;
    tg.nbx = (int)nbx;
    tg.n_theta = (int)n_theta;
    tg.n_tiles = (int)(n_theta * nbx);
    return tg;
}

template <typename KernelT, typename DataT>
inline cg_status launch_tiles(KernelT kern, int NT, const DataT& d, const double* theta, int64_t n_elem,
                              int64_t n_theta, double* part, WsHeader* hdr, TileGrid* tg_out,
                              cudaStream_t st, const int* gate = nullptr) {
    const int R = resident_blocks((const void*)kern, NT, 0);
    const int G = device_sm_count() * R;
    TileGrid tg = make_tiles(n_elem, n_theta, NT, G);
    tg.gate = gate;
    int grid = tg.n_tiles < G ? tg.n_tiles : G;
    prof_begin(st);
    kern<<<grid, NT, 0, st>>>(d, theta, tg, part, hdr);
    prof_end(st);
    *tg_out = tg;
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

// Tile grid of the FP64 kernels, whose time is set by the FP64 unit of each
// SM: among chunk counts per point group nbx (chunks of at least 2 elements
// per thread, even, within the workspace bound), the one whose busiest CTA
// of the persistent grid (grid = n_sm x resident CTAs, tiles dealt out
// round-robin) gets the fewest element-points, i.e. the smallest
// ceil(n_groups * nbx / grid) * chunk, with a 5 % penalty per missing tile
// below two tiles per SM (one CTA per SM leaves too few warps to cover the
// FP64 latencies; measured on the 10,000-bin x 100-point workload); ties:
// fewer tiles.  n_groups = ceil(n_theta / pt) groups of pt points.
inline TileGrid make_tiles_balanced(int64_t n_elem, int64_t n_theta, int pt, int NT, int n_sm, int resident) {
    TileGrid tg;
    tg.n_elem = n_elem;
    const int64_t groups = (n_theta + pt - 1) / pt;
    int64_t most = (n_elem + 2 * NT - 1) / (2 * NT);
    const int64_t cap = (kMaxTiles + groups - 1) / groups;
    if (most > cap) most = cap;
    if (most > max_nbx(n_theta)) most = max_nbx(n_theta);
    if (most < 1) most = 1;
    const int64_t S = n_sm > 0 ? n_sm : 1;
    const int64_t G = S * (resident > 0 ? resident : 1);
    int64_t best = 1, best_cost = -1;
    for (int64_t nbx = 1; nbx <= most; ++nbx) {
        int64_t chunk = (n_elem + nbx - 1) / nbx;
        chunk += chunk & 1;
        if ((n_elem + chunk - 1) / chunk != nbx) continue;
        const double per_sm = (double)(groups * nbx) / (double)S;
        const double pen = per_sm < 2.0 ? 1.0 + 0.05 * (2.0 - per_sm) : 1.0;
        const int64_t cost = (int64_t)((double)((groups * nbx + G - 1) / G * chunk) * pen);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = nbx;
        }
    }
    int64_t chunk = (n_elem + best - 1) / best;
    chunk += chunk & 1;
    if (chunk < 2) chunk = 2;
    tg.chunk = chunk;
    tg.nbx = (int)((n_elem + chunk - 1) / chunk);
    tg.n_theta = (int)groups;
    tg.n_tiles = (int)(groups * tg.nbx);
    tg.pt = pt;
    tg.n_pts = (int)n_theta;
    return tg;
}

template <typename KernelT, typename DataT>
inline cg_status launch_tiles_balanced(KernelT kern, int NT, int pt, const DataT& d, const double* theta,
                                       int64_t n_elem, int64_t n_theta, double* part, WsHeader* hdr,
                                       TileGrid* tg_out, cudaStream_t st, const int* gate = nullptr) {
    const int nsm = device_sm_count();
    const int R = resident_blocks((const void*)kern, NT, 0);
    TileGrid tg = make_tiles_balanced(n_elem, n_theta, pt, NT, nsm, R);
    tg.gate = gate;
    const int G = nsm * R;
    const int grid = tg.n_tiles < G ? tg.n_tiles : G;
    prof_begin(st);
    kern<<<grid, NT, 0, st>>>(d, theta, tg, part, hdr);
    prof_end(st);
    *tg_out = tg;
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

// Write one tile's partial sums: part[(th * (NACC + 1) + a) * nbx + c].
template <int NACC>
__device__ __forceinline__ void write_partial(double* __restrict__ part, const TileGrid& tg, int th,
                                              int c, const double* tot, int bad) {
    // one value per thread: NACC sums and the domain flag
    if (threadIdx.x <= NACC) {
        double* p = part + (size_t)th * (NACC + 1) * tg.nbx + c;
        p[(size_t)threadIdx.x * tg.nbx] = (threadIdx.x < NACC) ? tot[threadIdx.x] : (bad ? 1.0 : 0.0);
    }
}

}  // namespace cg

// Ragged batches: many segments, each with its own kmax (e.g. the shell
// quartets of an ERI batch, kmax_s = la+lb+lc+ld), in ONE persistent launch.
//
// Work decomposition: the concatenated argument array x[0, total) is cut into
// flat tiles of blockDim*XPT arguments; resident CTAs take tiles from a
// global atomic counter (the only scratch memory) until none are left, which
// balances the very uneven per-argument cost of different kmax.  A thread
// finds the segment of each of its arguments by binary search over seg_off
// restricted to the tile's segment range, and evaluates it with exactly the
// code boys_eval uses for that segment's kmax (bitwise-identical results).
// A warp whose lanes straddle segments with different kmax loops over the
// distinct values (rare: only warps that cross a segment boundary).
//
// Output of segment s (length len_s = seg_off[s+1] - seg_off[s]) is its own
// order-major block: F_k(x[seg_off[s] + j]) at out[out_off[s] + k*len_s + j].
#include <algorithm>
#include <array>
#include <chrono>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include "boys_fp64.cuh"
#include "boys_internal.h"

namespace boys {
namespace ragged {

constexpr int kMaxBlock = 256;
// Resident blocks of kMaxBlock threads per SM the register allocation allows:
// 4 caps the kernel at 64 registers.  The register count follows the largest
// per-kmax body (kmax = 32, which then spills a little), and uncapped it held
// the small-kmax bodies that dominate typical batches to a quarter of the
// warps (2.40 ms vs 2.12 ms on 4096 segments at mean kmax 4.07).
#ifndef BOYS_RAGGED_MIN_BLOCKS
#define BOYS_RAGGED_MIN_BLOCKS 4
#endif

struct Workspace {
    unsigned long long next_tile;  // work counter, zeroed before every launch
    unsigned long long error;      // nonzero: a segment had kmax outside [0, 32]
};
static_assert(sizeof(Workspace) <= 256, "workspace fits its published size");

// One argument's orders 0..K to dst[k * row]: the stored mode's evaluation
// (same bits), which keeps only half of the orders live.
template <int K>
__device__ __noinline__ void eval_store(double xv, double* __restrict__ dst, int64_t row) {
    fp64::eval_store<K>(xv, dst, row);
}

__device__ __forceinline__ void dispatch(int k, double xv, double* dst, int64_t row) {
#define BOYS_RAGGED_CASE(K) \
    case K: eval_store<K>(xv, dst, row); break;
    switch (k) {
        BOYS_RAGGED_CASE(0) BOYS_RAGGED_CASE(1) BOYS_RAGGED_CASE(2) BOYS_RAGGED_CASE(3)
        BOYS_RAGGED_CASE(4) BOYS_RAGGED_CASE(5) BOYS_RAGGED_CASE(6) BOYS_RAGGED_CASE(7)
        BOYS_RAGGED_CASE(8) BOYS_RAGGED_CASE(9) BOYS_RAGGED_CASE(10) BOYS_RAGGED_CASE(11)
        BOYS_RAGGED_CASE(12) BOYS_RAGGED_CASE(13) BOYS_RAGGED_CASE(14) BOYS_RAGGED_CASE(15)
        BOYS_RAGGED_CASE(16) BOYS_RAGGED_CASE(17) BOYS_RAGGED_CASE(18) BOYS_RAGGED_CASE(19)
        BOYS_RAGGED_CASE(20) BOYS_RAGGED_CASE(21) BOYS_RAGGED_CASE(22) BOYS_RAGGED_CASE(23)
        BOYS_RAGGED_CASE(24) BOYS_RAGGED_CASE(25) BOYS_RAGGED_CASE(26) BOYS_RAGGED_CASE(27)
        BOYS_RAGGED_CASE(28) BOYS_RAGGED_CASE(29) BOYS_RAGGED_CASE(30) BOYS_RAGGED_CASE(31)
        BOYS_RAGGED_CASE(32)
        default: break;
    }
#undef BOYS_RAGGED_CASE
}

// Largest s in [lo, hi] with seg_off[s] <= i (seg_off non-decreasing; lo if
// there is none): a 32-way search by a whole warp.  Each round the lanes
// probe 32 evenly spaced offsets and a ballot keeps the interval between the
// last probe at or below i and the next one, so 4096 segments take three
// dependent loads instead of twelve.  All 32 lanes must call it together;
// every lane returns the result.
__device__ __forceinline__ int find_segment_warp(const int64_t* __restrict__ seg_off, int lo, int hi, int64_t i) {
    const int lane = threadIdx.x & 31;
    while (hi > lo) {
        const int span = hi - lo + 1;
        const int step = (span + 31) / 32;
        const int probe = lo + lane * step;
        const bool le = probe <= hi && __ldg(seg_off + probe) <= i;
        const unsigned m = __ballot_sync(0xffffffffu, le);
        const int last = m ? 31 - __clz((int)m) : 0;  // none at or below i: stay at lo, as the binary search does
        lo = lo + last * step;
        hi = min(hi, lo + step - 1);
        if (step == 1) break;
    }
    return lo;
}

// Largest s in [lo, hi] with seg_off[s] <= i (seg_off non-decreasing).
__device__ __forceinline__ int find_segment(const int64_t* __restrict__ seg_off, int lo, int hi, int64_t i) {
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(seg_off + mid) <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int XPT>
__global__ void __launch_bounds__(kMaxBlock, BOYS_RAGGED_MIN_BLOCKS) k_ragged(const double* __restrict__ x,
                                                      const int64_t* __restrict__ seg_off,
                                                      const int32_t* __restrict__ seg_kmax, int nseg,
                                                      double* __restrict__ out,
                                                      const int64_t* __restrict__ out_off,
                                                      Workspace* __restrict__ ws,
                                                      const unsigned* __restrict__ gate) {
    if (gate && *gate == 0) return;  // a fallback launch that is not needed
    __shared__ long long s_tile;
    __shared__ int s_seg_lo, s_seg_hi;
    const int64_t total = __ldg(seg_off + nseg);
    const int64_t per_tile = (int64_t)blockDim.x * XPT;
    const int64_t ntiles = (total + per_tile - 1) / per_tile;
    const unsigned lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x < 32) {  // warp 0 takes the next tile and finds its segments
            long long t = 0;
            if (threadIdx.x == 0) t = (long long)atomicAdd(&ws->next_tile, 1ULL);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (threadIdx.x == 0) s_tile = t;
            if (t < ntiles) {
                const int64_t first = t * per_tile;
                const int64_t last = min(first + per_tile, total) - 1;
                const int lo = find_segment_warp(seg_off, 0, nseg - 1, first);
                const int hi = find_segment_warp(seg_off, lo, nseg - 1, last);
                if (threadIdx.x == 0) {
                    s_seg_lo = lo;
                    s_seg_hi = hi;
                }
            }
        }
        __syncthreads();
        const long long t = s_tile;
        const int seg_lo = s_seg_lo, seg_hi = s_seg_hi;
        __syncthreads();
        if (t >= ntiles) break;
        const int64_t base = t * per_tile;
#pragma unroll 1
        for (int j = 0; j < XPT; ++j) {
            const int64_t i = base + (int64_t)j * blockDim.x + threadIdx.x;
            bool valid = i < total;
            int km = 0;
            double xv = 0.0;
            double* dst = nullptr;
            int64_t row = 0;
            if (valid) {
                const int s = find_segment(seg_off, seg_lo, seg_hi, i);
                const int64_t s0 = __ldg(seg_off + s);
                row = __ldg(seg_off + s + 1) - s0;
                km = __ldg(seg_kmax + s);
                if (km < 0 || km > 32) {
                    atomicOr(&ws->error, 1ULL);
                    valid = false;
                } else {
                    xv = __ldcs(x + i);
                    dst = out + __ldg(out_off + s) + (i - s0);
                }
            }
            unsigned pending = __ballot_sync(0xffffffffu, valid);
            while (pending) {
                const int leader = __ffs(pending) - 1;
                const int k = __shfl_sync(0xffffffffu, km, leader);
                const bool mine = valid && km == k && ((pending >> lane) & 1u);
                if (mine) dispatch(k, xv, dst, row);
                pending &= ~__ballot_sync(0xffffffffu, mine);
            }
        }
    }
}

// ---------------------------------------------- kmax-grouped launches (plans)
//
// A plan may instead launch one kernel per kmax present, each over a table of
// tiles (up to blockDim consecutive arguments of one segment) built on the
// host when the plan is created.  Every such kernel inlines one evaluation
// body -- the stored mode's, so the bits are those of boys_eval -- with its
// own register allocation, no segment search and no per-warp kmax dispatch;
// the launches are parallel branches of the plan's graph.

struct Tile {
    int32_t seg;    // segment index
    int32_t len;    // arguments in this tile (<= blockDim)
    int64_t start;  // first argument, relative to the segment
};
static_assert(sizeof(Tile) == 16, "tile table entries are 16 bytes");

// 48 / 64 registers at 256 threads; BOYS_GROUPED_MIN_BLOCKS forces one value
constexpr int grouped_min_blocks(int kmax) {
#ifdef BOYS_GROUPED_MIN_BLOCKS
    return BOYS_GROUPED_MIN_BLOCKS + 0 * kmax;
#else
    return kmax <= 16 ? 5 : 4;
#endif
}

// One tile of a kmax group: its arguments, one per thread.
template <int K>
__device__ __forceinline__ void group_tile(const double* __restrict__ x, const int64_t* __restrict__ seg_off,
                                           double* __restrict__ out, const int64_t* __restrict__ out_off,
                                           const Tile& tl) {
    if ((int)threadIdx.x < tl.len) {
        const int64_t s0 = __ldg(seg_off + tl.seg);
        const int64_t row = __ldg(seg_off + tl.seg + 1) - s0;
        const int64_t j = tl.start + threadIdx.x;
        fp64::eval_store<K>(__ldcs(x + s0 + j), out + __ldg(out_off + tl.seg) + j, row);
    }
}

template <int K>
__global__ void __launch_bounds__(kMaxBlock, grouped_min_blocks(K)) k_ragged_group(
        const double* __restrict__ x, const int64_t* __restrict__ seg_off, double* __restrict__ out,
        const int64_t* __restrict__ out_off, const Tile* __restrict__ tiles, int64_t ntiles) {
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) group_tile<K>(x, seg_off, out, out_off, tiles[t]);
}

using GroupFn = void (*)(const double*, const int64_t*, double*, const int64_t*, const Tile*, int64_t);

template <int... K>
constexpr auto group_table(std::integer_sequence<int, K...>) {
    return std::array<GroupFn, sizeof...(K)>{&k_ragged_group<K>...};
}

// ------------------------------------ kmax-grouped launches without a plan
//
// With a large enough workspace, boys_eval_ragged builds the kmax-grouped tile
// table itself, on the device, at every call: a count of tiles per kmax, an
// exclusive scan of the 33 counts, and a fill in which each segment takes a
// contiguous range of its group with one atomic (the order of tiles inside a
// group varies, the values do not).  Then one kernel per kmax reads its
// group's range from the workspace.  If the table would exceed the
// workspace's capacity, the group kernels return at once and a persistent
// launch, gated on that condition, evaluates the batch instead.

constexpr int kGroupTile = 128;  // arguments per tile = threads per block of the group kernels

struct GroupHeader {
    Workspace ws;             // error word (the persistent fallback also uses next_tile)
    unsigned count[33];       // tiles per kmax
    unsigned base[33];        // first tile of each group
    unsigned cursor[33];      // fill positions
    unsigned total;           // tiles in all
    unsigned overflow;        // 1: the table does not fit, the persistent fallback runs
};
constexpr size_t kGroupHeaderBytes = 512;
static_assert(sizeof(GroupHeader) <= kGroupHeaderBytes, "group header fits its reserved bytes");

__device__ __forceinline__ bool bad_kmax(int k) { return k < 0 || k > 32; }

__global__ void k_group_count(const int64_t* __restrict__ seg_off, const int32_t* __restrict__ seg_kmax, int nseg,
                              GroupHeader* __restrict__ h) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x) {
        const int64_t len = __ldg(seg_off + s + 1) - __ldg(seg_off + s);
        const int k = __ldg(seg_kmax + s);
        if (len <= 0) continue;
        if (bad_kmax(k)) {
            atomicOr(&h->ws.error, 1ULL);
            continue;
        }
        atomicAdd(&h->count[k], (unsigned)((len + kGroupTile - 1) / kGroupTile));
    }
}

__global__ void k_group_scan(GroupHeader* __restrict__ h, unsigned long long capacity) {
    if (threadIdx.x != 0) return;
    unsigned long long run = 0;
    for (int k = 0; k <= 32; ++k) {
        h->base[k] = (unsigned)run;
        h->cursor[k] = (unsigned)run;
        run += h->count[k];
    }
    h->total = (unsigned)run;
    h->overflow = run > capacity ? 1u : 0u;
}

__global__ void k_group_fill(const int64_t* __restrict__ seg_off, const int32_t* __restrict__ seg_kmax, int nseg,
                             GroupHeader* __restrict__ h, Tile* __restrict__ tiles) {
    if (h->overflow) return;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x) {
        const int64_t len = __ldg(seg_off + s + 1) - __ldg(seg_off + s);
        const int k = __ldg(seg_kmax + s);
        if (len <= 0 || bad_kmax(k)) continue;
        const unsigned n = (unsigned)((len + kGroupTile - 1) / kGroupTile);
        const unsigned p = atomicAdd(&h->cursor[k], n);
        for (unsigned t = 0; t < n; ++t) {
            const int64_t a = (int64_t)t * kGroupTile;
            tiles[p + t] = Tile{s, (int32_t)min((int64_t)kGroupTile, len - a), a};
        }
    }
}

template <int K>
__global__ void __launch_bounds__(kGroupTile, 2 * grouped_min_blocks(K)) k_ragged_group_dev(
        const double* __restrict__ x, const int64_t* __restrict__ seg_off, double* __restrict__ out,
        const int64_t* __restrict__ out_off, const Tile* __restrict__ tiles, const GroupHeader* __restrict__ h) {
    // The groups write disjoint outputs and read only the finished table, so
    // the next kmax's kernel may start at once (programmatic dependent launch):
    // its blocks take the SMs as this kernel's blocks retire, with no drain.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (h->overflow) return;
    const unsigned n = h->count[K];
    const Tile* __restrict__ g = tiles + h->base[K];
    for (unsigned t = blockIdx.x; t < n; t += gridDim.x) group_tile<K>(x, seg_off, out, out_off, g[t]);
}

using GroupDevFn = void (*)(const double*, const int64_t*, double*, const int64_t*, const Tile*, const GroupHeader*);

template <int... K>
constexpr auto group_dev_table(std::integer_sequence<int, K...>) {
    return std::array<GroupDevFn, sizeof...(K)>{&k_ragged_group_dev<K>...};
}

using KernelFn = void (*)(const double*, const int64_t*, const int32_t*, int, double*, const int64_t*, Workspace*,
                          const unsigned*);

inline KernelFn kernel_for(int xpt) { return xpt == 2 ? &k_ragged<2> : &k_ragged<1>; }

struct Config {
    int block = 128;
    int xpt = 1;
    int waves = 1;  // resident CTAs per SM multiplier for the persistent grid;
                    // 0: one launch per kmax group (plans only; tile = block)
};

inline int grid_size(const Config& c) {
    const int per_sm = blocks_per_sm((const void*)kernel_for(c.xpt), c.block);
    return std::max(1, sm_count() * per_sm * c.waves);
}

boys_status check_args(const double* x, const int64_t* seg_off, const int32_t* seg_kmax, int32_t nseg,
                       double* out, const int64_t* out_off, const char* fn) {
    if (nseg < 0) return fail(BOYS_ERR_INVALID_ARG, "%s: nseg=%d < 0", fn, nseg);
    if (nseg == 0) return BOYS_OK;
    if (!x || !seg_off || !seg_kmax || !out || !out_off) return fail(BOYS_ERR_INVALID_ARG, "%s: NULL pointer", fn);
    if (!aligned(x, 8) || !aligned(out, 8) || !aligned(seg_off, 8) || !aligned(out_off, 8) || !aligned(seg_kmax, 4))
        return fail(BOYS_ERR_ALIGNMENT, "%s: pointer not aligned to its element size", fn);
    return BOYS_OK;
}

boys_status launch(const Config& c, const double* x, const int64_t* seg_off, const int32_t* seg_kmax, int32_t nseg,
                   double* out, const int64_t* out_off, Workspace* ws, cudaStream_t stream) {
    boys_status st = check_cuda(cudaMemsetAsync(ws, 0, sizeof(Workspace), stream), "ragged workspace reset");
    if (st != BOYS_OK) return st;
    kernel_for(c.xpt)<<<grid_size(c), c.block, 0, stream>>>(x, seg_off, seg_kmax, nseg, out, out_off, ws, nullptr);
    return check_cuda(cudaGetLastError(), "ragged launch");
}

// The plan-less kmax-grouped batch on a workspace of `bytes` >= kGroupHeaderBytes
// + 16: reset the header, build the table on the device, one launch per kmax,
// then the persistent kernel gated on the table's overflow flag.
boys_status launch_grouped(const double* x, const int64_t* seg_off, const int32_t* seg_kmax, int32_t nseg, double* out,
                           const int64_t* out_off, void* workspace, size_t bytes, cudaStream_t stream) {
    GroupHeader* h = (GroupHeader*)workspace;
    Tile* tiles = (Tile*)((char*)workspace + kGroupHeaderBytes);
    const unsigned long long capacity = std::min<unsigned long long>((bytes - kGroupHeaderBytes) / sizeof(Tile),
                                                                     0xFFFFFFFFull);  // tile indices are 32-bit
    boys_status st = check_cuda(cudaMemsetAsync(h, 0, sizeof(GroupHeader), stream), "ragged group header reset");
    if (st != BOYS_OK) return st;
    const int sgrid = (int)std::min<int64_t>((nseg + 255) / 256, (int64_t)sm_count() * 4);
    k_group_count<<<sgrid, 256, 0, stream>>>(seg_off, seg_kmax, nseg, h);
    k_group_scan<<<1, 32, 0, stream>>>(h, capacity);
    k_group_fill<<<sgrid, 256, 0, stream>>>(seg_off, seg_kmax, nseg, h, tiles);
    st = check_cuda(cudaGetLastError(), "ragged group table");
    // One kernel per kmax, each launched as a programmatic dependent of the
    // previous launch: a group kernel signals its dependents as it starts, and
    // the fill kernel never does, so every group still starts after the table
    // is complete.
    static constexpr auto tg = group_dev_table(std::make_integer_sequence<int, 33>{});
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t lc = {};
    lc.blockDim = dim3(kGroupTile);
    lc.stream = stream;
    lc.attrs = &attr;
    lc.numAttrs = 1;
    for (int k = 0; k <= 32 && st == BOYS_OK; ++k) {
        lc.gridDim = dim3(sm_count() * blocks_per_sm((const void*)tg[k], kGroupTile));
        st = check_cuda(cudaLaunchKernelEx(&lc, tg[k], x, seg_off, out, out_off, (const Tile*)tiles,
                                           (const GroupHeader*)h), "ragged group launch");
    }
    if (st != BOYS_OK) return st;
    const Config c;
    lc.gridDim = dim3(grid_size(c));
    lc.blockDim = dim3(c.block);
    return check_cuda(cudaLaunchKernelEx(&lc, kernel_for(c.xpt), x, seg_off, seg_kmax, (int)nseg, out, out_off,
                                         &h->ws, (const unsigned*)&h->overflow),
                      "ragged fallback launch");
}

// ------------------------------------------------------------- autotuning

const std::vector<Config>& candidates() {
    static const std::vector<Config> c = [] {
        std::vector<Config> v;
        for (int block : {64, 128, 256})
            for (int xpt : {1, 2})
                for (int waves : {1, 2}) v.push_back(Config{block, xpt, waves});
        for (int block : {128, 256}) v.push_back(Config{block, 1, 0});
        return v;
    }();
    return c;
}

std::string device_key() {
    int dev = 0, drv = 0;
    cudaGetDevice(&dev);
    cudaDriverGetVersion(&drv);
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
    char buf[512];
    snprintf(buf, sizeof(buf), "%.200s|sm%d%d|%dSM|drv%d|lib%d", p.name, p.major, p.minor, p.multiProcessorCount, drv,
             boys_version());
    for (char* q = buf; *q; ++q)
        if (*q == ' ') *q = '_';
    return buf;
}

struct TuneCache {
    std::mutex mu;
    std::unordered_map<std::string, Config> mem;
    bool loaded = false;

    static const char* path() { return getenv("BOYS_AUTOTUNE_CACHE"); }

    void load() {
        if (loaded) return;
        loaded = true;
        const char* p = path();
        if (!p) return;
        FILE* f = fopen(p, "r");
        if (!f) return;
        char key[512];
        Config c;
        while (fscanf(f, "%511s %d %d %d", key, &c.block, &c.xpt, &c.waves) == 4) mem[key] = c;
        fclose(f);
    }

    bool get(const std::string& k, Config* c) {
        std::lock_guard<std::mutex> lk(mu);
        load();
        auto it = mem.find(k);
        if (it == mem.end()) return false;
        *c = it->second;
        return true;
    }

    void put(const std::string& k, const Config& c) {
        std::lock_guard<std::mutex> lk(mu);
        load();
        mem[k] = c;
        const char* p = path();
        if (!p) return;
        FILE* f = fopen(p, "a");
        if (!f) return;
        fprintf(f, "%s %d %d %d\n", k.c_str(), c.block, c.xpt, c.waves);
        fclose(f);
    }
};

TuneCache& cache() {
    static TuneCache c;
    return c;
}

}  // namespace ragged
}  // namespace boys

using namespace boys;

struct boys_ragged_plan {
    const double* x;
    const int64_t* seg_off;
    const int32_t* seg_kmax;
    int32_t nseg;
    double* out;
    const int64_t* out_off;
    ragged::Workspace* ws;
    ragged::Config cfg;
    int64_t total;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    float tuned_ms;
    // kmax-grouped launches: host copies of the descriptors and the tile table
    std::vector<int64_t> off_host;
    std::vector<int32_t> km_host;
    ragged::Tile* tiles;
    int tiles_block;
    int64_t group_begin[33], group_count[33];
};

BOYS_API size_t boys_ragged_workspace_size(void) { return 256; }

BOYS_API size_t boys_ragged_workspace_size_grouped(int32_t nseg, int64_t total) {
    if (nseg < 0 || total < 0) return 0;
    // every segment of len arguments takes ceil(len / 128) <= len / 128 + 1 tiles
    return ragged::kGroupHeaderBytes + sizeof(ragged::Tile) * ((size_t)total / ragged::kGroupTile + (size_t)nseg + 1);
}

BOYS_API boys_status boys_eval_ragged(const double* x, const int64_t* seg_off, const int32_t* seg_kmax,
                                      int32_t nseg, double* out, const int64_t* out_off, void* workspace,
                                      size_t workspace_bytes, void* stream) {
    boys_status st = ragged::check_args(x, seg_off, seg_kmax, nseg, out, out_off, "boys_eval_ragged");
    if (st != BOYS_OK || nseg == 0) return st;
    if (!workspace) return fail(BOYS_ERR_INVALID_ARG, "boys_eval_ragged: NULL workspace");
    if (workspace_bytes < boys_ragged_workspace_size())
        return fail(BOYS_ERR_INVALID_ARG, "boys_eval_ragged: workspace_bytes=%zu < %zu", workspace_bytes,
                    boys_ragged_workspace_size());
    if (!aligned(workspace, 16)) return fail(BOYS_ERR_ALIGNMENT, "boys_eval_ragged: workspace not 16-byte aligned");
    if (workspace_bytes >= ragged::kGroupHeaderBytes + sizeof(ragged::Tile))
        return ragged::launch_grouped(x, seg_off, seg_kmax, nseg, out, out_off, workspace, workspace_bytes,
                                      (cudaStream_t)stream);
    ragged::Config c;
    return ragged::launch(c, x, seg_off, seg_kmax, nseg, out, out_off, (ragged::Workspace*)workspace,
                          (cudaStream_t)stream);
}

BOYS_API boys_status boys_ragged_status(const void* workspace, int* bad_kmax, void* stream) {
    if (!workspace || !bad_kmax) return fail(BOYS_ERR_INVALID_ARG, "boys_ragged_status: NULL pointer");
    unsigned long long err = 0;
    const ragged::Workspace* ws = (const ragged::Workspace*)workspace;
    boys_status st = check_cuda(cudaMemcpyAsync(&err, &ws->error, sizeof(err), cudaMemcpyDeviceToHost,
                                                (cudaStream_t)stream), "boys_ragged_status copy");
    if (st != BOYS_OK) return st;
    st = check_cuda(cudaStreamSynchronize((cudaStream_t)stream), "boys_ragged_status sync");
    *bad_kmax = err ? 1 : 0;
    return st;
}

// Tile table for tiles of `block` arguments: the tiles of every segment, grouped
// by the segment's kmax (group k at [group_begin[k], + group_count[k])).
static boys_status build_tiles(boys_ragged_plan* p, int block) {
    if (p->tiles && p->tiles_block == block) return BOYS_OK;
    std::vector<ragged::Tile> tab;
    for (int k = 0; k <= 32; ++k) {
        p->group_begin[k] = (int64_t)tab.size();
        for (int32_t sg = 0; sg < p->nseg; ++sg) {
            if (p->km_host[sg] != k) continue;
            const int64_t len = p->off_host[sg + 1] - p->off_host[sg];
            for (int64_t a = 0; a < len; a += block)
                tab.push_back(ragged::Tile{sg, (int32_t)std::min<int64_t>(block, len - a), a});
        }
        p->group_count[k] = (int64_t)tab.size() - p->group_begin[k];
    }
    if (p->tiles) cudaFree(p->tiles);
    p->tiles = nullptr;
    p->tiles_block = 0;
    if (tab.empty()) return BOYS_OK;
    boys_status st = check_cuda(cudaMalloc((void**)&p->tiles, tab.size() * sizeof(ragged::Tile)), "plan tile table");
    if (st != BOYS_OK) return st;
    st = check_cuda(cudaMemcpy(p->tiles, tab.data(), tab.size() * sizeof(ragged::Tile), cudaMemcpyHostToDevice),
                    "plan tile table upload");
    if (st == BOYS_OK) p->tiles_block = block;
    return st;
}

// Streams and events that fork the kmax groups off the capturing stream and
// join them back; created before the capture begins (object creation is not
// a capturable operation) and destroyed after it ends.
struct GroupFork {
    cudaEvent_t fork = nullptr;
    std::vector<int> ks;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    ~GroupFork() {
        for (cudaEvent_t j : joins) cudaEventDestroy(j);
        for (cudaStream_t g : streams) cudaStreamDestroy(g);
        if (fork) cudaEventDestroy(fork);
    }
};

static boys_status prepare_groups(boys_ragged_plan* p, const ragged::Config& c, GroupFork* f) {
    boys_status st = build_tiles(p, c.block);  // allocates and copies: before any capture
    if (st != BOYS_OK) return st;
    st = check_cuda(cudaEventCreateWithFlags(&f->fork, cudaEventDisableTiming), "fork event");
    for (int k = 0; k <= 32 && st == BOYS_OK; ++k) {
        if (p->group_count[k] == 0) continue;
        cudaStream_t g;
        cudaEvent_t j;
        st = check_cuda(cudaStreamCreateWithFlags(&g, cudaStreamNonBlocking), "group stream");
        if (st != BOYS_OK) break;
        f->streams.push_back(g);
        st = check_cuda(cudaEventCreateWithFlags(&j, cudaEventDisableTiming), "join event");
        if (st != BOYS_OK) break;
        f->joins.push_back(j);
        f->ks.push_back(k);
    }
    return st;
}

// Records the batch for configuration c on the capturing stream s: the
// workspace reset, then either the persistent kernel or, for waves == 0, one
// kernel per kmax group, forked onto their own streams and joined back.
static boys_status record_launch(boys_ragged_plan* p, const ragged::Config& c, const GroupFork& f, cudaStream_t s) {
    if (c.waves != 0)
        return ragged::launch(c, p->x, p->seg_off, p->seg_kmax, p->nseg, p->out, p->out_off, p->ws, s);
    boys_status st = check_cuda(cudaMemsetAsync(p->ws, 0, sizeof(ragged::Workspace), s), "ragged workspace reset");
    if (st != BOYS_OK) return st;
    static constexpr auto tg = ragged::group_table(std::make_integer_sequence<int, 33>{});
    st = check_cuda(cudaEventRecord(f.fork, s), "fork record");
    for (size_t q = 0; q < f.ks.size() && st == BOYS_OK; ++q) {
        const int k = f.ks[q];
        const int64_t n = p->group_count[k];
        int per_sm = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tg[k], c.block, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        const int64_t grid = std::min<int64_t>(n, (int64_t)sm_count() * per_sm);
        cudaStreamWaitEvent(f.streams[q], f.fork, 0);
        tg[k]<<<(unsigned)grid, c.block, 0, f.streams[q]>>>(p->x, p->seg_off, p->out, p->out_off,
                                                             p->tiles + p->group_begin[k], n);
        st = check_cuda(cudaGetLastError(), "ragged group launch");
        cudaEventRecord(f.joins[q], f.streams[q]);
        cudaStreamWaitEvent(s, f.joins[q], 0);
    }
    return st;
}

static boys_status capture(boys_ragged_plan* p, const ragged::Config& c, cudaGraph_t* graph, cudaGraphExec_t* exec) {
    *graph = nullptr;
    *exec = nullptr;
    GroupFork f;
    boys_status st = c.waves == 0 ? prepare_groups(p, c, &f) : BOYS_OK;
    if (st != BOYS_OK) return st;
    cudaStream_t s;
    st = check_cuda(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "plan stream");
    if (st != BOYS_OK) return st;
    st = check_cuda(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (st == BOYS_OK) {
        boys_status lst = record_launch(p, c, f, s);
        cudaGraph_t g = nullptr;
        boys_status est = check_cuda(cudaStreamEndCapture(s, &g), "end capture");
        st = lst != BOYS_OK ? lst : est;
        if (st == BOYS_OK) {
            *graph = g;
            st = check_cuda(cudaGraphInstantiate(exec, g, 0), "graph instantiate");
            if (st != BOYS_OK) {
                cudaGraphDestroy(g);
                *graph = nullptr;
            }
        } else if (g) {
            cudaGraphDestroy(g);
        }
    }
    cudaStreamDestroy(s);
    return st;
}

static boys_status capture_graph(boys_ragged_plan* p) { return capture(p, p->cfg, &p->graph, &p->exec); }

// Mean time of one replay of configuration c's captured graph (-1 on failure).
static float time_config(boys_ragged_plan* p, const ragged::Config& c, cudaStream_t s, int reps) {
    cudaGraph_t g;
    cudaGraphExec_t e;
    if (capture(p, c, &g, &e) != BOYS_OK) return -1.0f;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaGraphLaunch(e, s);  // warm
    cudaEventRecord(a, s);
    for (int r = 0; r < reps; ++r) cudaGraphLaunch(e, s);
    cudaEventRecord(b, s);
    float ms = -1.0f;
    if (cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaGraphExecDestroy(e);
    cudaGraphDestroy(g);
    return ms > 0 ? ms / reps : -1.0f;
}

BOYS_API boys_status boys_ragged_plan_create(const double* x, const int64_t* seg_off, const int32_t* seg_kmax,
                                             int32_t nseg, double* out, const int64_t* out_off, int flags,
                                             boys_ragged_plan** plan) {
    if (!plan) return fail(BOYS_ERR_INVALID_ARG, "boys_ragged_plan_create: NULL plan");
    *plan = nullptr;
    boys_status st = ragged::check_args(x, seg_off, seg_kmax, nseg, out, out_off, "boys_ragged_plan_create");
    if (st != BOYS_OK) return st;
    if (nseg == 0) return fail(BOYS_ERR_INVALID_ARG, "boys_ragged_plan_create: nseg must be > 0");
    // Read the descriptors once (plan creation is a set-up step and may synchronise).
    std::vector<int64_t> off(nseg + 1);
    std::vector<int32_t> km(nseg);
    st = check_cuda(cudaMemcpy(off.data(), seg_off, sizeof(int64_t) * (nseg + 1), cudaMemcpyDeviceToHost), "read seg_off");
    if (st != BOYS_OK) return st;
    st = check_cuda(cudaMemcpy(km.data(), seg_kmax, sizeof(int32_t) * nseg, cudaMemcpyDeviceToHost), "read seg_kmax");
    if (st != BOYS_OK) return st;
    int64_t hist[33] = {0};
    for (int32_t s = 0; s < nseg; ++s) {
        if (off[s + 1] < off[s]) return fail(BOYS_ERR_INVALID_ARG, "boys_ragged_plan_create: seg_off decreases at %d", s);
        if (km[s] < 0 || km[s] > 32) return fail(BOYS_ERR_KMAX, "boys_ragged_plan_create: seg_kmax[%d]=%d", s, km[s]);
        hist[km[s]] += off[s + 1] - off[s];
    }
    if (off[0] != 0) return fail(BOYS_ERR_INVALID_ARG, "boys_ragged_plan_create: seg_off[0] must be 0");

    boys_ragged_plan* p = new boys_ragged_plan{};
    p->x = x; p->seg_off = seg_off; p->seg_kmax = seg_kmax; p->nseg = nseg; p->out = out; p->out_off = out_off;
    p->total = off[nseg];
    p->off_host = off;
    p->km_host = km;
    st = check_cuda(cudaMalloc((void**)&p->ws, 256), "plan workspace");
    if (st != BOYS_OK) { delete p; return st; }

    if (flags & BOYS_PLAN_AUTOTUNE) {
        // workload key: device + size bucket + argument-weighted kmax histogram (coarse)
        char wk[256];
        int64_t wsum = 0;
        for (int k = 0; k <= 32; ++k) wsum += hist[k] * (k + 1);
        snprintf(wk, sizeof(wk), "|n2^%d|seg%d|w%.2f", 64 - __builtin_clzll((unsigned long long)std::max<int64_t>(1, p->total)),
                 nseg, p->total ? (double)wsum / p->total : 0.0);
        const std::string key = ragged::device_key() + wk;
        ragged::Config best;
        if (!ragged::cache().get(key, &best)) {
            cudaStream_t s;
            cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            float best_ms = 1e30f;
            for (const auto& c : ragged::candidates()) {
                const float ms = time_config(p, c, s, 3);
                if (ms > 0 && ms < best_ms) { best_ms = ms; best = c; }
            }
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
            p->tuned_ms = best_ms;
            st = check_cuda(cudaGetLastError(), "autotune");
            if (st != BOYS_OK) { boys_ragged_plan_destroy(p); return st; }
            ragged::cache().put(key, best);
        }
        p->cfg = best;
    }
    if (flags & BOYS_PLAN_FORCE_CONFIG) {
        // BOYS_FORCE_CONFIG="block,xpt,waves" overrides tuning (tests use it)
        const char* f = getenv("BOYS_FORCE_CONFIG");
        ragged::Config c;
        if (f && sscanf(f, "%d,%d,%d", &c.block, &c.xpt, &c.waves) == 3 && (c.block == 64 || c.block == 128 || c.block == 256) &&
            (c.xpt == 1 || c.xpt == 2) && c.waves >= 0 && c.waves <= 8)
            p->cfg = c;
    }
    st = capture_graph(p);
    if (st != BOYS_OK) { boys_ragged_plan_destroy(p); return st; }
    *plan = p;
    return BOYS_OK;
}

BOYS_API boys_status boys_ragged_plan_launch(boys_ragged_plan* plan, void* stream) {
    if (!plan) return fail(BOYS_ERR_INVALID_ARG, "boys_ragged_plan_launch: NULL plan");
    return check_cuda(cudaGraphLaunch(plan->exec, (cudaStream_t)stream), "graph launch");
}

BOYS_API boys_status boys_ragged_plan_config(const boys_ragged_plan* plan, int* block, int* xpt, int* waves) {
    if (!plan || !block || !xpt || !waves) return fail(BOYS_ERR_INVALID_ARG, "boys_ragged_plan_config: NULL pointer");
    *block = plan->cfg.block;
    *xpt = plan->cfg.xpt;
    *waves = plan->cfg.waves;
    return BOYS_OK;
}

BOYS_API void boys_ragged_plan_destroy(boys_ragged_plan* plan) {
    if (!plan) return;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    if (plan->ws) cudaFree(plan->ws);
    if (plan->tiles) cudaFree(plan->tiles);
    delete plan;
}

// ------------------------------------------------ ragged batch without allocation
//
// boys_eval_ragged_noalloc serves callers that cannot hand the library any
// device memory of their own: the ragged kernel's scratch (tile counter and
// error word, 16 bytes) lives instead in the array below, which is part of
// this library's device image.  Every GPU that loads the library holds the
// array (kNoAllocScratchBytes) until the process exits.

namespace boys {
namespace ragged {

constexpr size_t kNoAllocScratchBytes = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
static_assert(sizeof(Workspace) <= kNoAllocScratchBytes, "ragged scratch must fit the static array");

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[kNoAllocMaxDevices];   // device address of the array, per device
static int g_noalloc_grid[kNoAllocMaxDevices];    // persistent grid of k_ragged<1> at 128 threads

// Per-device set-up on the first call with that device current: the array's
// name is only a host-side stand-in, so its device address comes from
// cudaGetSymbolAddress.  Nothing is allocated.
static boys_status noalloc_setup(int dev, void** ptr, int* grid) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return check_cuda(e, "boys_eval_ragged_noalloc: cudaGetSymbolAddress");
        int sms = 0, per_sm = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return check_cuda(e, "boys_eval_ragged_noalloc: SM count");
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ragged<1>, 128, 0);
        if (e != cudaSuccess) return check_cuda(e, "boys_eval_ragged_noalloc: occupancy");
        g_noalloc_grid[dev] = std::max(1, sms * std::max(1, per_sm));
        g_noalloc_ptr[dev] = p;
    }
    *ptr = g_noalloc_ptr[dev];
    *grid = g_noalloc_grid[dev];
    return BOYS_OK;
}

}  // namespace ragged
}  // namespace boys

BOYS_API boys_status boys_eval_ragged_noalloc(const double* x, const int64_t* seg_off, const int32_t* seg_kmax,
                                              int32_t nseg, double* out, const int64_t* out_off, void* stream) {
    boys_status st = ragged::check_args(x, seg_off, seg_kmax, nseg, out, out_off, "boys_eval_ragged_noalloc");
    if (st != BOYS_OK || nseg == 0) return st;
    // A call's scratch need does not grow with its sizes (one tile counter and
    // one error word); it is checked against the array all the same.
    if (sizeof(ragged::Workspace) > ragged::kNoAllocScratchBytes)
        return fail(BOYS_ERR_INVALID_ARG, "boys_eval_ragged_noalloc: needs %zu bytes of scratch, the static array holds %zu",
                    sizeof(ragged::Workspace), ragged::kNoAllocScratchBytes);
    int dev = 0;
    st = check_cuda(cudaGetDevice(&dev), "boys_eval_ragged_noalloc: cudaGetDevice");
    if (st != BOYS_OK) return st;
    if (dev < 0 || dev >= ragged::kNoAllocMaxDevices)
        return fail(BOYS_ERR_INVALID_ARG, "boys_eval_ragged_noalloc: device %d beyond the %d supported", dev,
                    ragged::kNoAllocMaxDevices);
    void* scratch = nullptr;
    int grid = 1;
    st = ragged::noalloc_setup(dev, &scratch, &grid);
    if (st != BOYS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's contents: the counter must restart at zero
    st = check_cuda(cudaMemsetAsync(scratch, 0, sizeof(ragged::Workspace), s), "boys_eval_ragged_noalloc: scratch reset");
    if (st != BOYS_OK) return st;
    ragged::k_ragged<1><<<grid, 128, 0, s>>>(x, seg_off, seg_kmax, nseg, out, out_off, (ragged::Workspace*)scratch,
                                             nullptr);
    return check_cuda(cudaGetLastError(), "boys_eval_ragged_noalloc launch");
}

// The error word of the static array on the current device, read after the
// stream's work so far; copying from the symbol needs no device address and
// no allocation.
BOYS_API boys_status boys_ragged_noalloc_status(int* bad_kmax, void* stream) {
    if (!bad_kmax) return fail(BOYS_ERR_INVALID_ARG, "boys_ragged_noalloc_status: NULL pointer");
    unsigned long long err = 0;
    cudaStream_t s = (cudaStream_t)stream;
    boys_status st = check_cuda(cudaMemcpyFromSymbolAsync(&err, ragged::g_noalloc_scratch, sizeof(err),
                                                          offsetof(ragged::Workspace, error), cudaMemcpyDeviceToHost, s),
                                "boys_ragged_noalloc_status copy");
    if (st != BOYS_OK) return st;
    st = check_cuda(cudaStreamSynchronize(s), "boys_ragged_noalloc_status sync");
    *bad_kmax = err ? 1 : 0;
    return st;
}

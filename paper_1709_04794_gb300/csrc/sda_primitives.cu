// Device primitives of the operator build (stable radix sort, prefix sum),
// the thread-local error state, and the host-side column-tile scheduler.
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <atomic>

#include "sda_common.cuh"

namespace sda {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local int g_code = 0;
static thread_local char g_msg[512] = {0};

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    g_code = code;
    return code;
}

void clear_error() {
    g_code = 0;
    g_msg[0] = 0;
}

int cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    int code = (e == cudaErrorMemoryAllocation) ? SDA_ERR_OOM : SDA_ERR_CUDA;
    (void)cudaGetLastError();
    return fail(code, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

int last_error(char *buf, int len) {
    if (buf && len > 0) {
        snprintf(buf, (size_t)len, "%s", g_msg);
    }
    return g_code;
}

static std::atomic<long long> g_launches{0};
static thread_local bool g_capturing = false;

void note_launch(int64_t n) {
    if (!g_capturing) g_launches.fetch_add((long long)n, std::memory_order_relaxed);
}
void set_capturing(bool on) { g_capturing = on; }
int64_t launch_count() { return (int64_t)g_launches.load(); }

// An operator's arrays live on the device that was current when it was built;
// a call that would launch on another device is refused before any launch.
int check_device(int op_device) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__);
    if (dev != op_device)
        return fail(SDA_ERR_INVALID_ARG, "the operator lives on device %d but device %d is current", op_device, dev);
    return SDA_OK;
}

int device_sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

// ---------------------------------------------------------------------------
// exclusive prefix sum (int64, in place): tiles of 2048, recursive on tile sums
// ---------------------------------------------------------------------------
constexpr int kScanItems = 8;
constexpr int kScanTile = kBlock * kScanItems;

__global__ void __launch_bounds__(kBlock) k_scan_tiles(int64_t *data, int64_t n, int64_t *sums) {
    __shared__ int64_t sh[kScanTile];
    __shared__ int64_t wsum[kBlock / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int i = threadIdx.x; i < kScanTile; i += kBlock) sh[i] = (base + i < n) ? data[base + i] : 0;
    __syncthreads();
    int64_t loc[kScanItems];
    int64_t t = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        loc[k] = t;
        t += sh[threadIdx.x * kScanItems + k];
    }
    // inclusive warp scan of the thread totals
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t inc = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    int64_t woff = 0, total = 0;
#pragma unroll
    for (int i = 0; i < kBlock / 32; ++i) {
        if (i < w) woff += wsum[i];
        total += wsum[i];
    }
    const int64_t excl = woff + inc - t;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) sh[threadIdx.x * kScanItems + k] = loc[k] + excl;
    __syncthreads();
    for (int i = threadIdx.x; i < kScanTile; i += kBlock)
        if (base + i < n) data[base + i] = sh[i];
    if (threadIdx.x == 0 && sums) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kBlock) k_scan_add(int64_t *data, int64_t n, const int64_t *sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    const int64_t add = sums[blockIdx.x];
    for (int i = threadIdx.x; i < kScanTile; i += kBlock)
        if (base + i < n) data[base + i] += add;
}

int scan_exclusive_i64(int64_t *data, int64_t n, cudaStream_t s) {
    if (n <= 0) return SDA_OK;
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles == 1) {
        k_scan_tiles<<<1, kBlock, 0, s>>>(data, n, nullptr);
        SDA_LAUNCHED();
        return SDA_OK;
    }
    DevBuf<int64_t> sums;
    SDA_TRY(sums.alloc((size_t)ntiles));
    k_scan_tiles<<<(unsigned)ntiles, kBlock, 0, s>>>(data, n, sums.p);
    SDA_LAUNCHED();
    SDA_TRY(scan_exclusive_i64(sums.p, ntiles, s));
    k_scan_add<<<(unsigned)ntiles, kBlock, 0, s>>>(data, n, sums.p);
    SDA_LAUNCHED();
    SDA_CUDA(cudaStreamSynchronize(s));   // `sums` is freed on return
    return SDA_OK;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (uint32 key, uint32 value), 8-bit digits
// ---------------------------------------------------------------------------
constexpr int kRadixBins = 256;
constexpr int kRadixRounds = 16;
constexpr int kRadixTile = kBlock * kRadixRounds;

__global__ void __launch_bounds__(kBlock) k_radix_hist(const uint32_t *keys, int64_t n, int shift,
                                                       int64_t *hist, int64_t ntiles) {
    __shared__ unsigned cnt[kRadixBins];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int r = 0; r < kRadixRounds; ++r) {
        const int64_t i = base + (int64_t)r * kBlock + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(kBlock) k_radix_scatter(const uint32_t *kin, const uint32_t *vin,
                                                          uint32_t *kout, uint32_t *vout, int64_t n,
                                                          int shift, const int64_t *offs,
                                                          int64_t ntiles) {
    __shared__ int64_t running[kRadixBins];
    __shared__ unsigned wcnt[kBlock / 32][kRadixBins];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    running[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
#pragma unroll
    for (int k = 0; k < kBlock / 32; ++k) wcnt[k][threadIdx.x] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int r = 0; r < kRadixRounds; ++r) {
        const int64_t i = base + (int64_t)r * kBlock + threadIdx.x;
        const bool valid = i < n;
        const uint32_t key = valid ? kin[i] : 0u;
        const uint32_t val = valid ? vin[i] : 0u;
        const unsigned digit = valid ? ((key >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, digit);
        const unsigned rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[w][digit] = __popc(peers);
        __syncthreads();
        if (valid) {
            int64_t pos = running[digit] + rank;
            for (int k = 0; k < w; ++k) pos += wcnt[k][digit];
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        {
            unsigned tot = 0;
#pragma unroll
            for (int k = 0; k < kBlock / 32; ++k) {
                tot += wcnt[k][threadIdx.x];
                wcnt[k][threadIdx.x] = 0;
            }
            running[threadIdx.x] += tot;
        }
        __syncthreads();
    }
}

int radix_sort_pairs(uint32_t *keys, uint32_t *vals, int64_t n, int key_bits, cudaStream_t s) {
    if (n <= 1 || key_bits <= 0) return SDA_OK;
    const int64_t ntiles = (n + kRadixTile - 1) / kRadixTile;
    DevBuf<uint32_t> k2, v2;
    DevBuf<int64_t> hist;
    SDA_TRY(k2.alloc((size_t)n));
    SDA_TRY(v2.alloc((size_t)n));
    SDA_TRY(hist.alloc((size_t)(ntiles * kRadixBins)));
    uint32_t *ka = keys, *va = vals, *kb = k2.p, *vb = v2.p;
    for (int shift = 0; shift < key_bits; shift += 8) {
        k_radix_hist<<<(unsigned)ntiles, kBlock, 0, s>>>(ka, n, shift, hist.p, ntiles);
        SDA_LAUNCHED();
        SDA_TRY(scan_exclusive_i64(hist.p, ntiles * kRadixBins, s));
        k_radix_scatter<<<(unsigned)ntiles, kBlock, 0, s>>>(ka, va, kb, vb, n, shift, hist.p, ntiles);
        SDA_LAUNCHED();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        SDA_CUDA(cudaMemcpyAsync(keys, ka, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        SDA_CUDA(cudaMemcpyAsync(vals, va, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
    SDA_CUDA(cudaStreamSynchronize(s));   // temporaries are freed on return
    return SDA_OK;
}

// ---------------------------------------------------------------------------
// tiles of consecutive segments
// ---------------------------------------------------------------------------
// lanes per segment of a multi-segment tile: at most eight nonzeros per lane
static int lanes_for(int64_t maxlen) {
    int g = 1;
    while (g < 32 && 8 * g < maxlen) g <<= 1;
    return g;
}

// Appends the tiles of the segments [0, d) of `colptr` (absolute nonzero
// offsets); split chunks take slots from `*slots` and split entries after the
// ones already in `splits`.
// Segments longer than big_seg become tiles of their own (split into chunks of
// at most tile_nnz); the others are grouped into multi-segment tiles of at most
// tile_nnz nonzeros and tile_segs segments.
// Chunk boundaries are multiples of `align` nonzeros from the segment start.
// returns false if a multi-column tile would exceed the limits (the blocked
// column pass keeps such a tile in a fixed per-warp scratch)
static bool append_seg_tiles(const int64_t *colptr, int64_t d, int64_t tile_nnz, int64_t tile_segs,
                             int64_t big_seg, int64_t align, std::vector<Tile> &tiles,
                             std::vector<SplitSeg> &splits, int64_t *slots, int64_t chunk_nnz = 0) {
    if (chunk_nnz <= 0) chunk_nnz = tile_nnz;
    int64_t j = 0;
    while (j < d) {
        const int64_t len = colptr[j + 1] - colptr[j];
        if (len > big_seg) {
            const int64_t nch0 = (len + chunk_nnz - 1) / chunk_nnz;
            const int64_t chunk0 = ((len + nch0 - 1) / nch0 + align - 1) / align * align;
            const int64_t nch = (len + chunk0 - 1) / chunk0;
            if (nch == 1) {
                tiles.push_back(Tile{colptr[j], colptr[j + 1], (int32_t)j, (int32_t)(j + 1), 0, -1, -1, 0});
            } else {
                const int64_t chunk = chunk0;
                const int32_t lseg = (int32_t)splits.size();
                splits.push_back(SplitSeg{(int32_t)*slots, (int32_t)nch});
                for (int64_t c = 0; c < nch; ++c) {
                    const int64_t a = colptr[j] + c * chunk;
                    const int64_t b = std::min(colptr[j + 1], a + chunk);
                    tiles.push_back(Tile{a, b, (int32_t)j, (int32_t)(j + 1), 0, (int32_t)(*slots + c), lseg, 0});
                }
                *slots += nch;
            }
            ++j;
            continue;
        }
        const int64_t start = j;
        int64_t nz = 0, maxlen = 0;
        while (j < d) {
            const int64_t l = colptr[j + 1] - colptr[j];
            if (l > big_seg || (j > start && (nz + l > tile_nnz || j - start >= tile_segs))) break;
            nz += l;
            maxlen = std::max(maxlen, l);
            ++j;
        }
        tiles.push_back(Tile{colptr[start], colptr[j], (int32_t)start, (int32_t)j, lanes_for(maxlen), -1, -1, 0});
        if (nz > std::max(tile_nnz, big_seg) || j - start > tile_segs) return false;
    }
    return true;
}

static int upload_schedule(const std::vector<Tile> &tiles, const std::vector<SplitSeg> &splits, int64_t slots,
                           ColSchedule &out) {
    if (slots > INT32_MAX || (int64_t)tiles.size() > INT32_MAX)
        return fail(SDA_ERR_UNSUPPORTED, "column schedule too large");
    out.ntiles = (int32_t)tiles.size();
    out.nsplits = (int32_t)splits.size();
    out.nslots = (int32_t)slots;
    SDA_TRY(out.tiles.alloc(tiles.size()));
    SDA_TRY(out.splits.alloc(splits.size()));
    if (!tiles.empty())
        SDA_CUDA(cudaMemcpy(out.tiles.p, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice));
    if (!splits.empty())
        SDA_CUDA(cudaMemcpy(out.splits.p, splits.data(), splits.size() * sizeof(SplitSeg),
                            cudaMemcpyHostToDevice));
    return SDA_OK;
}

int build_seg_schedule(const std::vector<int64_t> &colptr, ColSchedule &out) {
    std::vector<Tile> tiles;
    std::vector<SplitSeg> splits;
    int64_t slots = 0;
    if (!append_seg_tiles(colptr.data(), (int64_t)colptr.size() - 1, kTileNnz, kTileSegs, kBigSeg, 1, tiles, splits,
                          &slots))
        return fail(SDA_ERR_UNSUPPORTED, "segment tile over its limits");
    return upload_schedule(tiles, splits, slots, out);
}

int build_range_schedule(const std::vector<int64_t> &ptr, int nranges, int64_t d, ColSchedule &out,
                         std::vector<int32_t> &tile_off, int64_t chunk_nnz) {
    std::vector<Tile> tiles;
    std::vector<SplitSeg> splits;
    int64_t slots = 0;
    tile_off.assign((size_t)nranges + 1, 0);
    for (int r = 0; r < nranges; ++r) {
        if (!append_seg_tiles(ptr.data() + (size_t)r * (size_t)(d + 1), d, kWarpTileNnz, kWarpTileSegs,
                              kWarpBigSeg, 4, tiles, splits, &slots, chunk_nnz))
            return fail(SDA_ERR_UNSUPPORTED, "warp tile over its limits");
        if ((int64_t)tiles.size() > INT32_MAX) return fail(SDA_ERR_UNSUPPORTED, "column schedule too large");
        tile_off[(size_t)r + 1] = (int32_t)tiles.size();
    }
    return upload_schedule(tiles, splits, slots, out);
}

}  // namespace sda

// Internal definitions shared by the translation units of libsda.
#pragma once

#include <cuda/atomic>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sda.h"

namespace sda {

constexpr int kBlock = 256;          // threads per block of every pass kernel
constexpr int kMaxShifts = 64;       // shifts per solve
constexpr int kTileNnz = 4096;       // nonzeros per column tile / split chunk
constexpr int kTileSegs = 1024;      // columns per multi-column tile
constexpr int kBigSeg = 256;         // columns longer than this get whole-block tiles
constexpr int kMaxBlocksPerSm = 8;   // cap of resident blocks per SM used to size grids

// ---------------------------------------------------------------------------
// errors (thread-local last error, no exceptions across the ABI)
// ---------------------------------------------------------------------------
int fail(int code, const char *fmt, ...);
void clear_error();
int cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define SDA_CUDA(expr)                                                          \
    do {                                                                        \
        cudaError_t e_ = (expr);                                                \
        if (e_ != cudaSuccess) return ::sda::cuda_fail(e_, #expr, __FILE__, __LINE__); \
    } while (0)

// kernel launch accounting (instrumentation): every launch site calls
// SDA_LAUNCHED() right after the launch; launches recorded into a graph
// capture are not counted, graph replays count their kernels
void note_launch(int64_t n);
void set_capturing(bool on);
#define SDA_LAUNCHED()                                                          \
    do {                                                                        \
        ::sda::note_launch(1);                                                  \
        SDA_CUDA(cudaGetLastError());                                           \
    } while (0)

#define SDA_TRY(expr)                   \
    do {                                \
        int rc_ = (expr);               \
        if (rc_ < 0) return rc_;        \
    } while (0)

// device allocation helper: frees on destruction
template <class T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    int alloc(size_t count) {
        release();
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc(&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            (void)cudaGetLastError();
            return fail(SDA_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                        cudaGetErrorString(e));
        }
        n = count;
        return SDA_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    size_t bytes() const { return n * sizeof(T); }
};

// ---------------------------------------------------------------------------
// tiles of the sparse passes (built on the host from the segment pointers)
// ---------------------------------------------------------------------------
struct Tile {
    int64_t nz0, nz1;   // nonzero range (whole-block tiles)
    int32_t seg0, seg1; // column range
    int32_t lanes;      // > 0: multi-segment tile (nonzeros streamed, `lanes` lanes sum a
                        // segment); 0: whole-block tile
    int32_t slot;       // split chunk: slot of its partial sum; -1: the tile holds the whole column
    int32_t lseg;       // split chunk: index of its long column in the split tables
    int32_t pad;
};

struct SplitSeg {
    int32_t slot0;      // first slot of the column's chunks
    int32_t nchunks;
};

struct ColSchedule {
    DevBuf<Tile> tiles;
    DevBuf<SplitSeg> splits;
    int32_t ntiles = 0, nsplits = 0, nslots = 0;
};

// tiles of consecutive segments (rows or columns) of a CSR-like pointer array
int build_seg_schedule(const std::vector<int64_t> &ptr, ColSchedule &out);
// warp tiles (kWarpTileNnz, kWarpTileSegs, kWarpBigSeg, chunks aligned to quads)
// of `nranges` pointer arrays of d + 1 entries each, stored one after the other
// in `ptr`; the tiles of range r are [tile_off[r], tile_off[r + 1])
int build_range_schedule(const std::vector<int64_t> &ptr, int nranges, int64_t d, ColSchedule &out,
                         std::vector<int32_t> &tile_off, int64_t chunk_nnz);

// ---------------------------------------------------------------------------
// value storage types
// ---------------------------------------------------------------------------
struct Pattern {};  // no stored values: every entry is one

// get(): plain load; get_cs(): evict-first load for streams read once per pass
template <class VT>
struct Val;
template <>
struct Val<double> {
    static __device__ __forceinline__ double get(const double *v, int64_t e) { return v[e]; }
    static __device__ __forceinline__ double get_cs(const double *v, int64_t e) { return __ldcs(v + e); }
};
template <>
struct Val<float> {
    static __device__ __forceinline__ float get(const float *v, int64_t e) { return v[e]; }
    static __device__ __forceinline__ float get_cs(const float *v, int64_t e) { return __ldcs(v + e); }
};
template <>
struct Val<__half> {
    static __device__ __forceinline__ float get(const __half *v, int64_t e) { return __half2float(v[e]); }
    static __device__ __forceinline__ float get_cs(const __half *v, int64_t e) { return __half2float(__ldcs(v + e)); }
};
template <>
struct Val<__nv_fp8_e4m3> {
    static __device__ __forceinline__ float get(const __nv_fp8_e4m3 *v, int64_t e) { return float(v[e]); }
    static __device__ __forceinline__ float get_cs(const __nv_fp8_e4m3 *v, int64_t e) {
        __nv_fp8_e4m3 x;
        x.__x = (__nv_fp8_storage_t)__ldcs(reinterpret_cast<const unsigned char *>(v) + e);
        return float(x);
    }
};
template <>
struct Val<Pattern> {
    static __device__ __forceinline__ float get(const Pattern *, int64_t) { return 1.0f; }
    static __device__ __forceinline__ float get_cs(const Pattern *, int64_t) { return 1.0f; }
};

// Four consecutive stored values (a quad, 4-aligned) converted to the
// accumulation type, read with streaming loads.
template <class VT, class AccT>
struct Quad;
template <class AccT>
struct Quad<__half, AccT> {
    static __device__ __forceinline__ void load(const __half *v, int64_t q, AccT (&x)[4]) {
        const uint2 u = __ldcs(reinterpret_cast<const uint2 *>(v) + q);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
        x[0] = (AccT)a.x;
        x[1] = (AccT)a.y;
        x[2] = (AccT)b.x;
        x[3] = (AccT)b.y;
    }
};
template <class AccT>
struct Quad<__nv_fp8_e4m3, AccT> {
    static __device__ __forceinline__ void load(const __nv_fp8_e4m3 *v, int64_t q, AccT (&x)[4]) {
        const unsigned u = __ldcs(reinterpret_cast<const unsigned *>(v) + q);
        const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u & 0xffffu), __NV_E4M3);
        const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u >> 16), __NV_E4M3);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&lo));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&hi));
        x[0] = (AccT)a.x;
        x[1] = (AccT)a.y;
        x[2] = (AccT)b.x;
        x[3] = (AccT)b.y;
    }
};
template <class AccT>
struct Quad<float, AccT> {
    static __device__ __forceinline__ void load(const float *v, int64_t q, AccT (&x)[4]) {
        const float4 u = __ldcs(reinterpret_cast<const float4 *>(v) + q);
        x[0] = (AccT)u.x;
        x[1] = (AccT)u.y;
        x[2] = (AccT)u.z;
        x[3] = (AccT)u.w;
    }
};
template <class AccT>
struct Quad<double, AccT> {
    static __device__ __forceinline__ void load(const double *v, int64_t q, AccT (&x)[4]) {
        const double2 a = __ldcs(reinterpret_cast<const double2 *>(v) + 2 * q);
        const double2 b = __ldcs(reinterpret_cast<const double2 *>(v) + 2 * q + 1);
        x[0] = (AccT)a.x;
        x[1] = (AccT)a.y;
        x[2] = (AccT)b.x;
        x[3] = (AccT)b.y;
    }
};

// ---------------------------------------------------------------------------
// FP32 pair arithmetic (a value carried as an unevaluated sum hi + lo of two
// floats): Knuth's two-sum and the FMA form of Dekker's two-product, exact for
// finite operands without overflow.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float two_sum(float a, float b, float &e) {
    const float s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
    return s;
}
__device__ __forceinline__ float two_prod(float a, float b, float &e) {
    const float p = a * b;
    e = fmaf(a, b, -p);
    return p;
}
__device__ __forceinline__ void split_f32(double x, float &hi, float &lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// A running sum in the accumulation type of a sparse pass.  For FP32 it is a
// pair (hi + lo): every added term goes in through two-sum, so the sum of n
// terms carries O(eps) error instead of O(n eps); partial sums leave the pass
// as such pairs (float2) so that the consumer adds them without rounding.  For
// FP64 it is a plain double.
template <class AccT>
struct CompSum;
template <>
struct CompSum<float> {
    using Part = float2;
    float h = 0.f, l = 0.f;
    __device__ __forceinline__ void add(float x) {
        float e;
        h = two_sum(h, x, e);
        l += e;
    }
    __device__ __forceinline__ void add(const CompSum &o) {
        float e;
        h = two_sum(h, o.h, e);
        l += o.l + e;
    }
    __device__ __forceinline__ void xor_reduce(int o) {
        CompSum t;
        t.h = __shfl_xor_sync(0xffffffffu, h, o);
        t.l = __shfl_xor_sync(0xffffffffu, l, o);
        add(t);
    }
    __device__ __forceinline__ Part part() const {
        float e;
        const float s = two_sum(h, l, e);
        return make_float2(s, e);
    }
    __device__ __forceinline__ double to_double() const { return (double)h + (double)l; }
    static __device__ __forceinline__ Part from_double(double x) {
        float a, b;
        split_f32(x, a, b);
        return make_float2(a, b);
    }
    static __device__ __forceinline__ void add_part(CompSum &s, const Part &p) {
        CompSum t;
        t.h = p.x;
        t.l = p.y;
        s.add(t);
    }
    __device__ __forceinline__ float value() const { return h + l; }
};
template <>
struct CompSum<double> {
    using Part = double;
    double h = 0.0;
    __device__ __forceinline__ void add(double x) { h += x; }
    __device__ __forceinline__ void add(const CompSum &o) { h += o.h; }
    __device__ __forceinline__ void xor_reduce(int o) { h += __shfl_xor_sync(0xffffffffu, h, o); }
    __device__ __forceinline__ Part part() const { return h; }
    __device__ __forceinline__ double to_double() const { return h; }
    static __device__ __forceinline__ Part from_double(double x) { return x; }
    static __device__ __forceinline__ void add_part(CompSum &s, const Part &p) { s.h += p; }
    __device__ __forceinline__ double value() const { return h; }
};

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block in a fixed order; the result is returned to every thread.
// `red` holds kBlock/32 entries.  Contains __syncthreads().
template <class T>
__device__ __forceinline__ T block_sum(T v, T *red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    T s = 0;
#pragma unroll
    for (int i = 0; i < kBlock / 32; ++i) s += red[i];
    return s;
}

// Arrival on a device-scope counter with release/acquire ordering: the writes
// made before the arrival by the arriving thread are visible to the thread that
// observes the final count.  Returns the count before this arrival.
__device__ __forceinline__ unsigned arrive(unsigned *counter) {
    cuda::atomic_ref<unsigned, cuda::thread_scope_device> c(*counter);
    return c.fetch_add(1u, cuda::memory_order_acq_rel);
}

// Grid-wide "last block" protocol: every block stores its NDOT partials, the
// block that arrives last sees all of them (read them with __ldcg).  Returns true
// in that block only (for every thread of it).  The counter is reset by the caller.
template <int NDOT>
__device__ __forceinline__ bool arrive_last(const double *mine, double *partials, unsigned *counter) {
    __shared__ int last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k) partials[(int64_t)blockIdx.x * NDOT + k] = mine[k];
        last = (arrive(counter) == gridDim.x - 1);
    }
    __syncthreads();
    return last != 0;
}

// Threads of a block of the blocked column pass (kColBlkPerSm blocks per SM;
// a block's shared memory holds one range's slice of the gathered vector).  Its tiles are
// worked by single warps: at most kWarpTileNnz nonzeros and kWarpTileSegs
// columns; columns longer than kWarpBigSeg take whole-warp tiles.
constexpr int kColBlk = 1024;
constexpr int kColBlkPerSm = 1;   // blocks of the blocked column pass resident per SM
constexpr int kWarpTileNnz = 512;
// Row pass: leading features kept in shared memory (share of the nonzeros they
// should cover, and a cap measured on the 200k workload: 16k-32k features best)
constexpr double kRowHeadCover = 0.85;
constexpr int64_t kRowHeadMax = 32768;
constexpr int kWarpTileSegs = 128;
constexpr int kWarpBigSeg = 256;
// Chunk of a long column in one whole-warp tile (FP32 and FP64 vectors), and
// the quads a lane loads at once there (chunk / 128).
constexpr int kWarpChunkNnz = 1024;
constexpr int kWarpChunkNnz64 = 512;
constexpr int warp_chunk_nnz(int64_t fsz) { return fsz == 8 ? kWarpChunkNnz64 : kWarpChunkNnz; }
// Head of the batched column pass: the fewest most frequent columns covering
// kHeadCover of the nonzeros (at most kHeadMax), in ranges of kHeadRows rows
// (a range's slice of 16 FP64 vectors fills 192 KB of shared memory).
constexpr double kHeadCover = 0.7;
constexpr int64_t kHeadMax = 1024;
constexpr int64_t kHeadRows = 1536;
// Shared memory the blocked column pass keeps for itself besides the slice.
constexpr int kColBlkReserve = 2048;
// Per-warp scratch of the blocked column pass after the slice: the quad sums of
// one multi-column tile (kWarpTileNnz / 4 values of the iteration type) and its
// column starts (kWarpTileSegs + 1 16-bit quad offsets, padded to 16 bytes).
// The last kColBlkStreamWarps warps of a block stream the shift state instead,
// with a table of the shift scalars (kShiftTabBytes) at the end of the scratch.
constexpr int kColBlkStreamWarps = 4;
constexpr int kWarpTileQuads = kWarpTileNnz / 4;
constexpr int kWarpTilePosBytes = ((kWarpTileSegs + 1) * 2 + 15) / 16 * 16;
constexpr int kShiftTabBytes = 2048;
constexpr int64_t colblk_scratch(int64_t fsz) {
    return (int64_t)(kColBlk / 32 - kColBlkStreamWarps) * ((int64_t)kWarpTileQuads * fsz + kWarpTilePosBytes) +
           kShiftTabBytes;
}

// Shared-memory doubles a block reduction of up to four sums needs.
constexpr int kRedDoubles = 4 * (kBlock / 32);

// Block sums of NDOT per-thread values, in a fixed order.  Each warp adds its
// lanes in the values' own type (a shuffle tree, the NDOT sums interleaved); the
// kBlock/32 warp sums are then converted and added in FP64 by the first warp
// alone, so a block issues only a few FP64 instructions (GB300 runs FP64 at about
// 1/60 of its FP32 rate).  The result is valid in thread 0 only.  `red` holds
// NDOT * kBlock/32 doubles.  Contains __syncthreads().
template <int NDOT, class AT>
__device__ __forceinline__ void block_dots(AT (&v)[NDOT], double (&out)[NDOT], double *red) {
    constexpr int NW = kBlock / 32;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    AT *r = reinterpret_cast<AT *>(red);
    __syncthreads();   // `red` may still be read by an earlier reduction
    if (l == 0) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k) r[k * NW + w] = v[k];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k) {
            double x = l < NW ? (double)r[k * NW + l] : 0.0;
#pragma unroll
            for (int o = NW / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            out[k] = x;
        }
    }
}

// Block sums of NDOT compensated per-thread sums (CompSum): pair shuffle trees
// within each warp, then the first warp over the warp sums; no rounding to the
// plain type on the way.  The result (parts) is valid in thread 0 only.  `red`
// holds NDOT * kBlock/32 parts.  Contains __syncthreads().
template <int NDOT, class AT>
__device__ __forceinline__ void block_parts(CompSum<AT> (&v)[NDOT], typename CompSum<AT>::Part (&out)[NDOT],
                                            typename CompSum<AT>::Part *red) {
    constexpr int NW = kBlock / 32;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k) v[k].xor_reduce(o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();   // `red` may still be read by an earlier reduction
    if (l == 0) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k) red[k * NW + w] = v[k].part();
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k) {
            CompSum<AT> x;
            if (l < NW) CompSum<AT>::add_part(x, red[k * NW + l]);
#pragma unroll
            for (int o = NW / 2; o > 0; o >>= 1) x.xor_reduce(o);
            out[k] = x.part();
        }
    }
}

// Grid-wide "last block" protocol on compensated parts: every block stores its
// NDOT parts; returns true in the block that arrives last (for all its threads).
template <int NDOT, class Part>
__device__ __forceinline__ bool arrive_last_parts(const Part *mine, Part *partials, unsigned *counter) {
    __shared__ int last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k) partials[(int64_t)blockIdx.x * NDOT + k] = mine[k];
        last = (arrive(counter) == gridDim.x - 1);
    }
    __syncthreads();
    return last != 0;
}

// Fixed-order compensated sum of the grid's parts (called by every thread of
// the last block), converted to FP64 once; valid in thread 0 only.
template <int NDOT, class AT>
__device__ __forceinline__ void grid_parts(const typename CompSum<AT>::Part *partials, int nblocks,
                                           double (&out)[NDOT], typename CompSum<AT>::Part *red) {
    CompSum<AT> s[NDOT];
    for (int b = threadIdx.x; b < nblocks; b += kBlock) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k) CompSum<AT>::add_part(s[k], __ldcg(partials + (int64_t)b * NDOT + k));
    }
    typename CompSum<AT>::Part tot[NDOT];
    block_parts<NDOT, AT>(s, tot, red);
#pragma unroll
    for (int k = 0; k < NDOT; ++k) {
        CompSum<AT> t;
        CompSum<AT>::add_part(t, tot[k]);
        out[k] = t.to_double();
    }
}

// Fixed-order sum of the grid's NDOT-wide partials (called by every thread of
// the last block); the result is valid in thread 0 only.
template <int NDOT>
__device__ __forceinline__ void grid_dots(const double *partials, int nblocks, double (&out)[NDOT], double *red) {
    double s[NDOT];
#pragma unroll
    for (int k = 0; k < NDOT; ++k) s[k] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kBlock) {
#pragma unroll
        for (int k = 0; k < NDOT; ++k) s[k] += __ldcg(partials + (int64_t)b * NDOT + k);
    }
    block_dots<NDOT, double>(s, out, red);
}

// ---------------------------------------------------------------------------
// primitives (sda_primitives.cu)
// ---------------------------------------------------------------------------
// Stable LSD radix sort of (key, value) pairs on the low `key_bits` bits of
// the keys.  Sorted data ends in keys/vals.  Temporary buffers are allocated
// by the call.
int radix_sort_pairs(uint32_t *keys, uint32_t *vals, int64_t n, int key_bits, cudaStream_t s);
// Exclusive prefix sum in place (int64).
int scan_exclusive_i64(int64_t *data, int64_t n, cudaStream_t s);

int device_sm_count();
// SDA_OK if `op_device` is the current device, else SDA_ERR_INVALID_ARG naming both
int check_device(int op_device);

}  // namespace sda

// gp_rank.cu -- Spearman's rank correlation fitness (Sec. III-C3: ranks of
// the values, then Karl Pearson's coefficient of the ranks).
//
// Unlike the fused metrics this one needs every prediction of a program at
// once: a batch of programs is predicted into [B][N], each segment is sorted
// by value (a stable LSD radix sort, 8-bit digits in 4 passes, of
// order-preserving 32-bit keys with the row index as payload; the first
// pass reads the predictions themselves), ties get the mean of their
// positions, and the weighted moments of the rank pairs are summed in FP64
// with a fixed partition.  The target's ranks are computed the same way
// once per call.  Ranks are kept doubled (first + last position, 1-based),
// which is an integer; the correlation does not see the factor 2.
#include "gp_internal.cuh"

namespace gpk {
namespace {

// rank pass: 2048 sorted keys per block
constexpr int kTileItems = 8;                          // per thread
constexpr int kTileThreads = 256;
constexpr int kTile = kTileItems * kTileThreads;

// LSD radix sort: 8-bit digits, 4 passes over tiles of 4096 keys, which
// the histogram kernel reads as 256 threads x 16 keys (key r * 256 + t of
// the tile to thread t) and the scatter as 512 threads x 8
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadixBits = 8;
constexpr int kBins = 1 << kRadixBits;
constexpr int kPasses = 32 / kRadixBits;

// order-preserving key of a float (-0 and +0 become the same key)
__device__ __forceinline__ uint32_t float_key(float f) {
    if (f == 0.0f) f = 0.0f;
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// key of item m of a segment: pass 0 reads the float values, later passes
// the keys of the previous pass
template <bool FROM_FLOAT>
__device__ __forceinline__ uint32_t load_key(const void *src, int64_t m) {
    if (FROM_FLOAT) return float_key(static_cast<const float *>(src)[m]);
    return static_cast<const uint32_t *>(src)[m];
}

// digit counts of one tile: hist[seg][digit][tile].  Each thread loads its
// 16 keys first (independent loads), then counts them into its warp's own
// histogram; a warp whose 32 keys share one digit adds once.
template <bool FROM_FLOAT>
__global__ void __launch_bounds__(kSortThreads) hist_kernel(const void *__restrict__ src, int64_t n,
                                                            int n_tiles, int shift, int32_t *hist,
                                                            uint32_t *nan_flag) {
    __shared__ int32_t wh[kSortWarps][kBins];
    const int seg = blockIdx.y, tile = blockIdx.x, t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) wh[w][t] = 0;
    const int64_t t0 = (int64_t)tile * kSortTile;
    const int tl = (int)min((int64_t)kSortTile, n - t0);
    const int64_t so = (int64_t)seg * n + t0;
    uint32_t d[kSortItems];
    bool nan = false;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int i = r * kSortThreads + t;
        uint32_t k = 0;
        if (i < tl) {
            if (FROM_FLOAT) {
                const float f = static_cast<const float *>(src)[so + i];
                nan |= f != f;
                k = float_key(f);
            } else {
                k = static_cast<const uint32_t *>(src)[so + i];
            }
        }
        d[r] = i < tl ? (k >> shift) & (kBins - 1) : (uint32_t)kBins;  // kBins: not counted
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t d0 = __shfl_sync(0xffffffffu, d[r], 0);
        if (__all_sync(0xffffffffu, d[r] == d0)) {
            if (lane == 0 && d0 < kBins) atomicAdd(&wh[warp][d0], 32);
        } else if (d[r] < kBins) {
            atomicAdd(&wh[warp][d[r]], 1);
        }
    }
    if (FROM_FLOAT && __any_sync(0xffffffffu, nan) && lane == 0) atomicOr(nan_flag + seg, 1u);
    __syncthreads();
    int32_t c = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) c += wh[w][t];
    hist[((int64_t)seg * kBins + t) * n_tiles + tile] = c;
}

// per (segment, digit), one warp: exclusive scan of the tile counts in
// place, and the digit's total in tot[seg][digit]
__global__ void __launch_bounds__(256) tile_scan_kernel(int32_t *hist, int32_t *tot, int n_rows_hd,
                                                        int n_tiles) {
    const int lane = threadIdx.x & 31;
    const int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (row >= n_rows_hd) return;
    int32_t *h = hist + (int64_t)row * n_tiles;
    int32_t carry = 0;
    for (int base = 0; base < n_tiles; base += 32) {
        const int i = base + lane;
        const int32_t v = i < n_tiles ? h[i] : 0;
        int32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (i < n_tiles) h[i] = carry + x - v;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) tot[row] = carry;
}

// exclusive scan of one value per thread over the block (blockDim.x
// threads, wsum: one entry per warp)
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t *wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    int32_t before = 0;
    for (int q = 0; q < warp; ++q) before += wsum[q];
    __syncthreads();
    return before + x - v;
}

// the scatter's tile: 512 threads x 8 keys (warp w owns keys [256 w, 256 w + 256))
constexpr int kScatThreads = 512;
constexpr int kScatWarps = kScatThreads / 32;
constexpr int kScatItems = kSortTile / kScatThreads;

// lanes of the warp whose digit equals this lane's (8-bit digits): one
// ballot per bit, as CUB does it, or the match instruction
template <bool BALLOT>
__device__ __forceinline__ unsigned digit_peers(uint32_t d) {
    if constexpr (BALLOT) {
        unsigned peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < kRadixBits; ++b) {
            const bool bit = (d >> b) & 1u;
            const unsigned m = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? m : ~m;
        }
        return peers;
    } else {
        return __match_any_sync(0xffffffffu, d);
    }
}

constexpr bool kBallotPeers = true;

// Stable scatter of one tile by one digit.  The tile is ranked in shared
// memory first (warp-level digit groups in key order, then a scan over
// (digit, warp)), staged in sorted order, and written out run by run so
// that neighbouring threads store to neighbouring addresses.  Padding
// beyond a ragged tile's end takes digit 255 and, being last in key order,
// sorted positions >= the tile length, which are not written.  Pass 0
// reads float values and produces the payload: the row index, or, when
// vals is given, vals[row] (a per-row table shared by the segments).  Two
// blocks per SM (64 registers); three, at 40 registers with spills, ran
// the rank fitness 3% slower.
template <bool FROM_FLOAT>
__global__ void __launch_bounds__(kScatThreads, 2) scatter_kernel(
    const void *__restrict__ src, const uint32_t *__restrict__ vals, int64_t n, int n_tiles,
    int shift, const int32_t *__restrict__ offs, const int32_t *__restrict__ tot,
    uint32_t *keys_out, uint32_t *vals_out) {
    __shared__ uint32_t sk[kSortTile];
    __shared__ uint32_t sv[kSortTile];
    __shared__ int32_t wcnt[kScatWarps][kBins];
    __shared__ int32_t dstart[kBins];
    __shared__ int32_t gbase[kBins];
    __shared__ int32_t wsum[kScatWarps];
    const int seg = blockIdx.y, tile = blockIdx.x, t = threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    const int64_t t0 = (int64_t)tile * kSortTile;
    const int tl = (int)min((int64_t)kSortTile, n - t0);
    const int64_t so = (int64_t)seg * n;
    for (int i = t; i < kScatWarps * kBins; i += kScatThreads) (&wcnt[0][0])[i] = 0;
    // the digit totals and this tile's digit offsets, loaded ahead of the keys
    const int32_t my_tot = t < kBins ? tot[(int64_t)seg * kBins + t] : 0;
    const int32_t my_off = t < kBins ? offs[((int64_t)seg * kBins + t) * n_tiles + tile] : 0;
    uint32_t kk[kScatItems], vv[kScatItems];
#pragma unroll
    for (int r = 0; r < kScatItems; ++r) {
        const int i = warp * (kScatItems * 32) + r * 32 + lane;
        const bool in = i < tl;
        kk[r] = in ? load_key<FROM_FLOAT>(src, so + t0 + i) : 0xffffffffu;
        if (FROM_FLOAT) vv[r] = vals ? (in ? vals[t0 + i] : 0u) : (uint32_t)(t0 + i);
        else vv[r] = in ? vals[so + t0 + i] : 0u;
    }
    // global position of this tile's first item of digit t: the digit's
    // start in the segment plus the same digit in earlier tiles
    const int32_t dbase = block_exclusive_scan(my_tot, wsum);
    if (t < kBins) gbase[t] = dbase + my_off;
    // the lanes holding one digit in a round form a group; its lowest lane
    // reserves the group's places with one atomic (predicated, so that the
    // rounds' atomics issue back to back; shared-memory atomics of one warp
    // keep their order) and hands the old count to the others afterwards
    const unsigned lt = (1u << lane) - 1u;
    uint32_t old[kScatItems];
    int32_t off[kScatItems];
    unsigned char lead[kScatItems];
#pragma unroll
    for (int r = 0; r < kScatItems; ++r) {
        const uint32_t d = (kk[r] >> shift) & (kBins - 1);
        const unsigned peers = digit_peers<kBallotPeers>(d);
        const int leader = __ffs(peers) - 1;
        const uint32_t addr = (uint32_t)__cvta_generic_to_shared(&wcnt[warp][d]);
        old[r] = 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.eq.u32 p, %1, %2;\n\t"
            "@p atom.shared.add.u32 %0, [%3], %4;\n\t}"
            : "+r"(old[r])
            : "r"((uint32_t)lane), "r"((uint32_t)leader), "r"(addr), "r"((uint32_t)__popc(peers))
            : "memory");
        lead[r] = (unsigned char)leader;
        off[r] = __popc(peers & lt);
    }
#pragma unroll
    for (int r = 0; r < kScatItems; ++r)
        off[r] += (int32_t)__shfl_sync(0xffffffffu, old[r], lead[r]);
    __syncthreads();
    // digit t: warps' exclusive prefixes, then the digits' starts in the tile
    int32_t run = 0;
    if (t < kBins) {
#pragma unroll
        for (int w = 0; w < kScatWarps; ++w) {
            const int32_t c = wcnt[w][t];
            wcnt[w][t] = run;
            run += c;
        }
    }
    const int32_t ds = block_exclusive_scan(run, wsum);
    if (t < kBins) dstart[t] = ds;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kScatItems; ++r) {
        const uint32_t d = (kk[r] >> shift) & (kBins - 1);
        const int pos = dstart[d] + wcnt[warp][d] + off[r];
        sk[pos] = kk[r];
        sv[pos] = vv[r];
    }
    __syncthreads();
#pragma unroll 4
    for (int pos = t; pos < tl; pos += kScatThreads) {
        const uint32_t k = sk[pos];
        const uint32_t d = (k >> shift) & (kBins - 1);
        const int64_t g = so + gbase[d] + (pos - dstart[d]);
        keys_out[g] = k;
        vals_out[g] = sv[pos];
    }
}

// first index in [lo, hi) of k with k[i] >= v (k ascending)
__device__ int64_t lower_bound_u32(const uint32_t *k, int64_t lo, int64_t hi, uint32_t v) {
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (k[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ int64_t upper_bound_u32(const uint32_t *k, int64_t lo, int64_t hi, uint32_t v) {
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (k[mid] <= v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Tie-group ends at the tile edges: edge[seg][tile] = (first position of
// the group of the tile's first key, last position of the group of its last
// key).  One thread per tile; the binary search runs only when the group
// crosses the edge, which keeps the rank pass free of dependent global loads.
__global__ void __launch_bounds__(256) edges_kernel(const uint32_t *__restrict__ keys, int64_t n,
                                                    int n_tiles, int n_seg, int2 *edge) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (int64_t)n_tiles * n_seg) return;
    const int seg = (int)(g / n_tiles), tile = (int)(g - (int64_t)seg * n_tiles);
    const uint32_t *k = keys + (int64_t)seg * n;
    const int64_t t0 = (int64_t)tile * kTile;
    const int64_t t1 = min(n, t0 + kTile);  // one past the tile's last key
    const uint32_t first = k[t0], last = k[t1 - 1];
    const int64_t lo = (t0 > 0 && k[t0 - 1] == first) ? lower_bound_u32(k, 0, t0, first) : t0;
    const int64_t hi = (t1 < n && k[t1] == last) ? upper_bound_u32(k, t1, n, last) - 1 : t1 - 1;
    edge[g] = make_int2((int)lo, (int)hi);
}

// Doubled average rank of every sorted position (first + last + 2, 1-based
// positions of its tie group).  Groups inside a tile are found with
// ballots over the sorted keys in shared memory; a group that reaches the
// tile's edge takes its end from edge[] (edges_kernel).  Ranks enter the sums centred on
// n + 1 (their unweighted mean): exact integers, zero for every row of a
// constant program, and sums without the cancellation of uncentred squares.
// mode 0 (the target): r2[row] = rank, and part = (sum w, sum w b,
// sum w b^2) of the tile; mode 1 (programs): part = (sum w a, sum w a^2,
// sum w a b), b = the target's centred rank of the row, read from r2y by
// the row in vals or, with vals_are_ranks (unweighted rows), carried in
// vals itself by the sort.  Unweighted and
// with n <= 2^29 a thread's sums are exact 64-bit integers; otherwise FP64.
// One FP64 triple per (segment, tile), added in a fixed order.
__global__ void __launch_bounds__(kTileThreads) rank_kernel(
    const uint32_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n, int n_tiles,
    int mode, const int2 *__restrict__ edge, uint32_t *r2, const uint32_t *__restrict__ r2y,
    const float *__restrict__ w, double *part, int vals_are_ranks) {
    constexpr int kSegs = kTile / 32;  // 32-position segments of the tile
    __shared__ uint32_t sk[kTile];
    __shared__ int16_t sfirst[kTile], slast[kTile];
    __shared__ int seg_first[kSegs], seg_last[kSegs];
    __shared__ double red[3][kTileThreads / 32];
    const int seg = blockIdx.y, tile = blockIdx.x, t = threadIdx.x;
    const int lane = t & 31;
    const uint32_t *k = keys + (int64_t)seg * n;
    const uint32_t *vl = vals + (int64_t)seg * n;
    const int64_t t0 = (int64_t)tile * kTile;
    const int tl = (int)min((int64_t)kTile, n - t0);
    // the tile's keys: independent loads issued together
    uint32_t kv[kTileItems];
#pragma unroll
    for (int it = 0; it < kTileItems; ++it) {
        const int q = it * kTileThreads + t;
        kv[it] = q < tl ? k[t0 + q] : 0u;
    }
#pragma unroll
    for (int it = 0; it < kTileItems; ++it) {
        const int q = it * kTileThreads + t;
        if (q < tl) sk[q] = kv[it];
    }
    const int2 eg = edge[(int64_t)seg * n_tiles + tile];
    // the rows of this thread's items, then their target ranks: independent
    // loads issued together
    uint32_t rows[kTileItems], rb[kTileItems];
#pragma unroll
    for (int it = 0; it < kTileItems; ++it) {
        const int q = it * kTileThreads + t;
        rows[it] = q < tl ? vl[t0 + q] : 0u;
    }
#pragma unroll
    for (int it = 0; it < kTileItems; ++it) {
        const int q = it * kTileThreads + t;
        rb[it] = (mode == 1 && q < tl) ? (vals_are_ranks ? rows[it] : r2y[rows[it]]) : 0u;
    }
    __syncthreads();
    // tie groups inside the tile: the warp's 32 positions q = it * 256 + t
    // are consecutive, so ballots of the group-start and group-end flags
    // give each position the latest start at or before it and the earliest
    // end at or after it within its 32-position segment; a segment without
    // one takes it from the segments before (after) it, scanned by warp 0
    const unsigned le = (2u << lane) - 1u, ge = ~((1u << lane) - 1u);
#pragma unroll
    for (int it = 0; it < kTileItems; ++it) {
        const int q = it * kTileThreads + t;
        const int sgi = q >> 5;
        const bool in = q < tl;
        const uint32_t v = in ? sk[q] : 0u;
        const bool start = in && (q == 0 || sk[q - 1] != v);
        const bool end = in && (q == tl - 1 || sk[q + 1] != v);
        const unsigned bs = __ballot_sync(0xffffffffu, start);
        const unsigned be = __ballot_sync(0xffffffffu, end);
        if (in) {
            sfirst[q] = (int16_t)((bs & le) ? (sgi << 5) + 31 - __clz(bs & le) : -1);
            slast[q] = (int16_t)((be & ge) ? (sgi << 5) + __ffs(be & ge) - 1 : -1);
        }
        if (lane == 0) {
            seg_first[sgi] = bs ? (sgi << 5) + 31 - __clz(bs) : -1;
            seg_last[sgi] = be ? (sgi << 5) + __ffs(be) - 1 : INT_MAX;
        }
    }
    __syncthreads();
    if (t < 32) {
        // exclusive prefix max of the segments' latest starts, exclusive
        // suffix min of their earliest ends (two segments per lane)
        const int a0 = seg_first[2 * t], a1 = seg_first[2 * t + 1];
        const int b0 = seg_last[2 * t], b1 = seg_last[2 * t + 1];
        int x = max(a0, a1);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (t >= o) x = max(x, y);
        }
        int before = __shfl_up_sync(0xffffffffu, x, 1);
        if (t == 0) before = -1;
        int z = min(b0, b1);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_down_sync(0xffffffffu, z, o);
            if (t + o < 32) z = min(z, y);
        }
        int after = __shfl_down_sync(0xffffffffu, z, 1);
        if (t == 31) after = INT_MAX;
        __syncwarp();
        seg_first[2 * t] = before;
        seg_first[2 * t + 1] = max(before, a0);
        seg_last[2 * t + 1] = after;
        seg_last[2 * t] = min(after, b1);
    }
    __syncthreads();
    const bool exact = w == nullptr && n <= ((int64_t)1 << 29);
    long long is[3] = {0, 0, 0};
    double s[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int it = 0; it < kTileItems; ++it) {
        const int q = it * kTileThreads + t;
        if (q >= tl) break;
        int lq = sfirst[q], uq = slast[q];
        if (lq < 0) lq = seg_first[q >> 5];
        if (uq < 0) uq = seg_last[q >> 5];
        const int64_t first = lq == 0 ? (int64_t)eg.x : t0 + lq;
        const int64_t last = uq == tl - 1 ? (int64_t)eg.y : t0 + uq;
        const uint32_t rank2 = (uint32_t)(first + last + 2);
        const uint32_t row = rows[it];
        const int a = (int)((int64_t)rank2 - (n + 1));  // |a| <= n - 1
        if (mode == 0) r2[row] = rank2;
        const int b = mode == 0 ? 1 : (int)((int64_t)rb[it] - (n + 1));
        if (exact) {
            // mode 0: (count, sum a, sum a^2); mode 1: (sum a, sum a^2, sum a b)
            is[0] += mode == 0 ? 1 : a;
            is[1] += mode == 0 ? a : (long long)a * a;
            is[2] += (long long)a * (mode == 0 ? a : b);
        } else {
            const double wv = w ? (double)w[row] : 1.0;
            const double ad = (double)a;
            const double wa = wv * ad;
            if (mode == 0) {
                s[0] += wv;
                s[1] += wa;
                s[2] = fma(wa, ad, s[2]);
            } else {
                s[0] += wa;
                s[1] = fma(wa, ad, s[1]);
                s[2] = fma(wa, (double)b, s[2]);
            }
        }
    }
    if (exact) {
#pragma unroll
        for (int j = 0; j < 3; ++j) s[j] = (double)is[j];
    }
    // fixed butterfly inside each warp, then the warps in order
#pragma unroll
    for (int j = 0; j < 3; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[j] += __shfl_xor_sync(0xffffffffu, s[j], o);
    }
    if ((t & 31) == 0) {
#pragma unroll
        for (int j = 0; j < 3; ++j) red[j][t >> 5] = s[j];
    }
    __syncthreads();
    if (t < 3) {
        double v = 0.0;
        for (int q = 0; q < kTileThreads / 32; ++q) v += red[t][q];
        part[((int64_t)seg * n_tiles + tile) * 3 + t] = v;
    }
}

// sum of tile triples in a fixed order: lane-strided, then lanes in order
__device__ __forceinline__ void sum_tiles(const double *p, int n_tiles, double (&S)[3]) {
    const int lane = threadIdx.x & 31;
    double s[3] = {0.0, 0.0, 0.0};
    for (int i = lane; i < n_tiles; i += 32)
#pragma unroll
        for (int j = 0; j < 3; ++j) s[j] += p[(int64_t)i * 3 + j];
#pragma unroll
    for (int j = 0; j < 3; ++j) S[j] = 0.0;
    for (int l = 0; l < 32; ++l)
#pragma unroll
        for (int j = 0; j < 3; ++j) S[j] += __shfl_sync(0xffffffffu, s[j], l);
}

// one warp per segment: |r| of the ranks from the program's tile sums and
// the target's (sum w, sum w b, sum w b^2)
__global__ void __launch_bounds__(256) spearman_final_kernel(
    const double *part, const double *tpart, int n_seg, int n_tiles, const uint32_t *nan_flag,
    float *out, double *out64) {
    const int lane = threadIdx.x & 31;
    const int seg = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (seg >= n_seg) return;
    double P[3], T[3];
    sum_tiles(part + (int64_t)seg * n_tiles * 3, n_tiles, P);
    sum_tiles(tpart, n_tiles, T);
    if (lane != 0) return;
    const double sw = T[0];
    const double ma = P[0] / sw, mb = T[1] / sw;
    const double va = P[1] / sw - ma * ma, vb = T[2] / sw - mb * mb;
    const double cov = P[2] / sw - ma * mb;
    double f;
    if (nan_flag[seg] || !isfinite(va) || !isfinite(vb) || !isfinite(cov)) f = __longlong_as_double(0x7ff8000000000000LL);
    else if (!(va > 0.0) || !(vb > 0.0)) f = 0.0;
    else f = fabs(cov) / sqrt(va * vb);
    out[seg] = (float)f;
    if (out64) out64[seg] = f;
}

// Sorts each of n_seg segments of n float values into keys (order-preserving
// integers) with the row index as payload, or payload[row] when a per-row
// table is given; the result is in keys/vals.
// hist holds n_seg * 256 * n_tiles counts, tot n_seg * 256.
cudaError_t radix_sort_values(const float *v, uint32_t *keys, uint32_t *vals, uint32_t *keys2,
                              uint32_t *vals2, int n_seg, int64_t n, int32_t *hist, int32_t *tot,
                              uint32_t *nan_flag, const uint32_t *payload, cudaStream_t st) {
    const int n_tiles = (int)((n + kSortTile - 1) / kSortTile);
    const dim3 grid(n_tiles, n_seg);
    const int scan_rows = n_seg * kBins;
    const int scan_blocks = (scan_rows + 7) / 8;
    for (int pass = 0; pass < kPasses; ++pass) {
        const int shift = pass * kRadixBits;
        // pass 0: values -> keys2; then keys2 -> keys -> keys2 -> keys
        const uint32_t *ki = (pass & 1) ? keys2 : keys;
        const uint32_t *vi = (pass & 1) ? vals2 : vals;
        uint32_t *ko = (pass & 1) ? keys : keys2;
        uint32_t *vo = (pass & 1) ? vals : vals2;
        if (pass == 0) {
            hist_kernel<true><<<grid, kSortThreads, 0, st>>>(v, n, n_tiles, shift, hist, nan_flag);
        } else {
            hist_kernel<false><<<grid, kSortThreads, 0, st>>>(ki, n, n_tiles, shift, hist, nullptr);
        }
        tile_scan_kernel<<<scan_blocks, 256, 0, st>>>(hist, tot, scan_rows, n_tiles);
        if (pass == 0) {
            scatter_kernel<true><<<grid, kScatThreads, 0, st>>>(v, payload, n, n_tiles, shift, hist,
                                                                tot, ko, vo);
        } else {
            scatter_kernel<false><<<grid, kScatThreads, 0, st>>>(ki, vi, n, n_tiles, shift, hist,
                                                                 tot, ko, vo);
        }
    }
    return cudaGetLastError();  // 4 passes: the result is in keys/vals
}

}  // namespace

// scratch of one batch of n_seg segments: keys, vals and their second
// buffers, the tile digit counts, the digit totals, the rank partials and
// the NaN flags
struct RankScratch {
    uint32_t *keys, *vals, *keys2, *vals2;
    int32_t *hist, *tot;
    double *part;
    int2 *edge;
    uint32_t *nan_flag;
    size_t bytes;
};

RankScratch carve_rank(void *scratch, int n_seg, int64_t n) {
    const int64_t sort_tiles = (n + kSortTile - 1) / kSortTile;
    const int64_t rank_tiles = (n + kTile - 1) / kTile;
    auto al = [](int64_t x) { return (size_t)((x + 255) / 256 * 256); };
    char *b = static_cast<char *>(scratch);
    RankScratch r{};
    size_t o = 0;
    const size_t arr = al((int64_t)n_seg * n * 4);
    r.keys = reinterpret_cast<uint32_t *>(b + o); o += arr;
    r.vals = reinterpret_cast<uint32_t *>(b + o); o += arr;
    r.keys2 = reinterpret_cast<uint32_t *>(b + o); o += arr;
    r.vals2 = reinterpret_cast<uint32_t *>(b + o); o += arr;
    r.hist = reinterpret_cast<int32_t *>(b + o); o += al((int64_t)n_seg * kBins * sort_tiles * 4);
    r.tot = reinterpret_cast<int32_t *>(b + o); o += al((int64_t)n_seg * kBins * 4);
    r.part = reinterpret_cast<double *>(b + o); o += al((int64_t)n_seg * rank_tiles * 3 * 8);
    r.edge = reinterpret_cast<int2 *>(b + o); o += al((int64_t)n_seg * rank_tiles * 8);
    r.nan_flag = reinterpret_cast<uint32_t *>(b + o); o += al((int64_t)n_seg * 4);
    r.bytes = o;
    return r;
}

size_t rank_scratch_bytes(int n_seg, int64_t n) {
    return carve_rank(nullptr, n_seg, n).bytes;
}

size_t target_part_bytes(int64_t n) { return (size_t)((n + kTile - 1) / kTile) * 3 * 8; }

cudaError_t target_ranks(const float *y, const float *w, int64_t n, void *scratch, uint32_t *r2y,
                         double *tpart, cudaStream_t st) {
    const int64_t n_tiles = (n + kTile - 1) / kTile;
    const RankScratch r = carve_rank(scratch, 1, n);
    cudaError_t e = cudaMemsetAsync(r.nan_flag, 0, 4, st);
    if (e != cudaSuccess) return e;
    e = radix_sort_values(y, r.keys, r.vals, r.keys2, r.vals2, 1, n, r.hist, r.tot, r.nan_flag,
                          nullptr, st);
    if (e != cudaSuccess) return e;
    edges_kernel<<<(unsigned)((n_tiles + 255) / 256), 256, 0, st>>>(r.keys, n, (int)n_tiles, 1, r.edge);
    rank_kernel<<<dim3((unsigned)n_tiles, 1), kTileThreads, 0, st>>>(
        r.keys, r.vals, n, (int)n_tiles, 0, r.edge, r2y, nullptr, w, tpart, 0);
    return cudaGetLastError();
}

cudaError_t spearman_batch(const float *pred, int n_seg, int64_t n, const uint32_t *r2y,
                           const double *tpart, const float *w, void *scratch, float *out,
                           double *out64, cudaStream_t st) {
    const int64_t n_tiles = (n + kTile - 1) / kTile;
    const RankScratch r = carve_rank(scratch, n_seg, n);
    cudaError_t e = cudaMemsetAsync(r.nan_flag, 0, (size_t)n_seg * 4, st);
    if (e != cudaSuccess) return e;
    // unweighted rows need only the target's rank of each row: the sort
    // carries it as the payload, so the rank pass reads it in sorted order
    // instead of gathering it by row
    const bool carry_ranks = w == nullptr;
    e = radix_sort_values(pred, r.keys, r.vals, r.keys2, r.vals2, n_seg, n, r.hist, r.tot,
                          r.nan_flag, carry_ranks ? r2y : nullptr, st);
    if (e != cudaSuccess) return e;
    edges_kernel<<<(unsigned)((n_tiles * n_seg + 255) / 256), 256, 0, st>>>(r.keys, n, (int)n_tiles,
                                                                           n_seg, r.edge);
    rank_kernel<<<dim3((unsigned)n_tiles, n_seg), kTileThreads, 0, st>>>(
        r.keys, r.vals, n, (int)n_tiles, 1, r.edge, nullptr, r2y, w, r.part, carry_ranks ? 1 : 0);
    spearman_final_kernel<<<(n_seg + 7) / 8, 256, 0, st>>>(r.part, tpart, n_seg, (int)n_tiles,
                                                           r.nan_flag, out, out64);
    return cudaGetLastError();
}

}  // namespace gpk

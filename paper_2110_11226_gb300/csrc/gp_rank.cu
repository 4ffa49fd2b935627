// gp_rank.cu -- Spearman's rank correlation fitness (Sec. III-C3: ranks of
// the values, then Karl Pearson's coefficient of the ranks).
//
// Unlike the fused metrics this one needs every prediction of a program at
// once: a batch of programs is predicted into [B][N], each segment is sorted
// by value (a stable LSD radix sort, 4-bit digits, of order-preserving
// 32-bit keys with the row index as payload), ties get the mean of their
// positions, and the weighted moments of the rank pairs are summed in FP64
// with a fixed partition.  The target's ranks are computed the same way
// once per call.  Ranks are kept doubled (first + last position, 1-based),
// which is an integer; the correlation does not see the factor 2.
#include "gp_internal.cuh"

namespace gpk {
namespace {

constexpr int kTileItems = 8;                          // per thread
constexpr int kTileThreads = 256;
constexpr int kTile = kTileItems * kTileThreads;       // 2048 keys per tile
constexpr int kRadixBits = 4;
constexpr int kDigits = 1 << kRadixBits;

// order-preserving key of a float (-0 and +0 become the same key)
__device__ __forceinline__ uint32_t float_key(float f) {
    if (f == 0.0f) f = 0.0f;
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void __launch_bounds__(256) to_keys_kernel(const float *__restrict__ v, int n_seg,
                                                      int64_t n, uint32_t *keys, uint32_t *vals,
                                                      uint32_t *nan_flag) {
    const int64_t total = (int64_t)n_seg * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float f = v[i];
        if (f != f) atomicOr(nan_flag + i / n, 1u);
        keys[i] = float_key(f);
        vals[i] = (uint32_t)(i % n);
    }
}

// digit counts of one tile: hist[seg][digit][tile]
__global__ void __launch_bounds__(kTileThreads) hist_kernel(const uint32_t *__restrict__ keys,
                                                            int64_t n, int n_tiles, int shift,
                                                            int32_t *hist) {
    __shared__ int32_t cnt[kDigits];
    const int seg = blockIdx.y, tile = blockIdx.x;
    if (threadIdx.x < kDigits) cnt[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t *k = keys + (int64_t)seg * n;
    const int64_t base = (int64_t)tile * kTile + (int64_t)threadIdx.x * kTileItems;
#pragma unroll
    for (int it = 0; it < kTileItems; ++it) {
        const int64_t m = base + it;
        if (m < n) atomicAdd(&cnt[(k[m] >> shift) & (kDigits - 1)], 1);
    }
    __syncthreads();
    if (threadIdx.x < kDigits)
        hist[((int64_t)seg * kDigits + threadIdx.x) * n_tiles + tile] = cnt[threadIdx.x];
}

// exclusive scan of hist[seg][*][*] in digit-major order, one block per
// segment, 1024 entries at a time with a carry
__global__ void __launch_bounds__(1024) scan_kernel(int32_t *hist, int n_tiles) {
    __shared__ int32_t warp_sum[32];
    __shared__ int32_t carry;
    int32_t *h = hist + (int64_t)blockIdx.x * kDigits * n_tiles;
    const int64_t len = (int64_t)kDigits * n_tiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < len; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const int32_t v = i < len ? h[i] : 0;
        int32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int32_t s = warp_sum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            warp_sum[lane] = s;
        }
        __syncthreads();
        const int32_t before = carry + (warp > 0 ? warp_sum[warp - 1] : 0) + x - v;
        if (i < len) h[i] = before;
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + v;
        __syncthreads();
    }
}

// stable scatter of one tile by one digit: thread t owns items
// [t*8, t*8+8) of the tile in order; an item's place is the digit's
// segment offset for this tile, plus the same digit in earlier threads of
// the tile, plus the same digit in its own earlier items
__global__ void __launch_bounds__(kTileThreads) scatter_kernel(
    const uint32_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n, int n_tiles,
    int shift, const int32_t *__restrict__ offs, uint32_t *keys_out, uint32_t *vals_out) {
    __shared__ int32_t sc[kDigits * kTileThreads];
    __shared__ int32_t tsum[kTileThreads];
    const int seg = blockIdx.y, tile = blockIdx.x, t = threadIdx.x;
    const int64_t so = (int64_t)seg * n;
    const int64_t base = (int64_t)tile * kTile + (int64_t)t * kTileItems;
    uint32_t kk[kTileItems], vv[kTileItems];
    int32_t cnt[kDigits];
#pragma unroll
    for (int d = 0; d < kDigits; ++d) cnt[d] = 0;
#pragma unroll
    for (int it = 0; it < kTileItems; ++it) {
        const int64_t m = base + it;
        kk[it] = m < n ? keys[so + m] : 0u;
        vv[it] = m < n ? vals[so + m] : 0u;
        if (m < n) {
            const int d = (kk[it] >> shift) & (kDigits - 1);
#pragma unroll
            for (int e = 0; e < kDigits; ++e) cnt[e] += (d == e);
        }
    }
#pragma unroll
    for (int d = 0; d < kDigits; ++d) sc[d * kTileThreads + t] = cnt[d];
    __syncthreads();
    // exclusive scan over sc in digit-major order: thread t scans entries
    // [16t, 16t+16), then the 256 thread totals are scanned
    int32_t run = 0;
    int32_t loc[kDigits];
#pragma unroll
    for (int e = 0; e < kDigits; ++e) {
        loc[e] = run;
        run += sc[t * kDigits + e];
    }
    tsum[t] = run;
    __syncthreads();
    if (t < 32) {  // warp 0 scans the 256 totals, 8 per lane
        int32_t part = 0;
        int32_t v8[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            v8[q] = part;
            part += tsum[t * 8 + q];
        }
        int32_t x = part;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (t >= o) x += y;
        }
        const int32_t before = x - part;
#pragma unroll
        for (int q = 0; q < 8; ++q) tsum[t * 8 + q] = before + v8[q];
    }
    __syncthreads();
    const int32_t pre = tsum[t];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kDigits; ++e) sc[t * kDigits + e] = pre + loc[e];
    __syncthreads();
    // place of (digit d, thread t) within the tile's digit-d run
    int32_t start[kDigits];
#pragma unroll
    for (int d = 0; d < kDigits; ++d)
        start[d] = offs[((int64_t)seg * kDigits + d) * n_tiles + tile] +
                   (sc[d * kTileThreads + t] - sc[d * kTileThreads]);
#pragma unroll
    for (int it = 0; it < kTileItems; ++it) {
        const int64_t m = base + it;
        if (m >= n) continue;
        const int d = (kk[it] >> shift) & (kDigits - 1);
        int32_t pos = 0;
#pragma unroll
        for (int e = 0; e < kDigits; ++e)
            if (d == e) pos = start[e]++;
        keys_out[so + pos] = kk[it];
        vals_out[so + pos] = vv[it];
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

__device__ int smem_lower(const uint32_t *k, int lo, int hi, uint32_t v) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (k[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ int smem_upper(const uint32_t *k, int lo, int hi, uint32_t v) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (k[mid] <= v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Doubled average rank of every sorted position (first + last + 2, 1-based
// positions of its tie group).  Groups inside a tile are found in shared
// memory; a group that reaches the tile's edge is extended by one binary
// search over the segment per tile edge.  mode 0: r2[vals[m]] = rank (the
// target's ranks by row); mode 1: FP64 moment sums of (rank, r2y[row]),
// both centred on n + 1, with the row's weight, one partial per (segment,
// tile).
__global__ void __launch_bounds__(kTileThreads) rank_kernel(
    const uint32_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n, int n_tiles,
    int mode, uint32_t *r2, const uint32_t *__restrict__ r2y, const float *__restrict__ w,
    double *part) {
    __shared__ uint32_t sk[kTile];
    __shared__ int64_t edge[2];
    __shared__ double red[6][kTileThreads];
    const int seg = blockIdx.y, tile = blockIdx.x, t = threadIdx.x;
    const uint32_t *k = keys + (int64_t)seg * n;
    const uint32_t *vl = vals + (int64_t)seg * n;
    const int64_t t0 = (int64_t)tile * kTile;
    const int tl = (int)min((int64_t)kTile, n - t0);
    for (int q = t; q < tl; q += kTileThreads) sk[q] = k[t0 + q];
    if (t == 0) edge[0] = lower_bound_u32(k, 0, t0, k[t0]);
    if (t == 1) edge[1] = upper_bound_u32(k, t0 + tl, n, k[t0 + tl - 1]) - 1;
    __syncthreads();
    double s[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int it = 0; it < kTileItems; ++it) {
        const int q = t * kTileItems + it;
        if (q >= tl) break;
        const uint32_t v = sk[q];
        int lq = q, uq = q + 1;
        if ((q > 0 && sk[q - 1] == v) || q == 0) lq = smem_lower(sk, 0, q, v);
        if ((q + 1 < tl && sk[q + 1] == v) || q + 1 == tl) uq = smem_upper(sk, q + 1, tl, v);
        const int64_t first = lq == 0 ? edge[0] : t0 + lq;
        const int64_t last = uq == tl ? edge[1] : t0 + uq - 1;
        const uint32_t rank2 = (uint32_t)(first + last + 2);
        const uint32_t row = vl[t0 + q];
        if (mode == 0) {
            r2[row] = rank2;
        } else {
            // doubled ranks centred on n + 1 (their unweighted mean): exact
            // integers, zero for every row of a constant program, and sums
            // without the cancellation of uncentred squares
            const double wv = w ? (double)w[row] : 1.0;
            const double a = (double)((int64_t)rank2 - (n + 1));
            const double b = (double)((int64_t)r2y[row] - (n + 1));
            s[0] += wv;
            s[1] += wv * a;
            s[2] += wv * a * a;
            s[3] += wv * b;
            s[4] += wv * b * b;
            s[5] += wv * a * b;
        }
    }
    if (mode == 0) return;
#pragma unroll
    for (int j = 0; j < 6; ++j) red[j][t] = s[j];
    __syncthreads();
    for (int h = kTileThreads / 2; h > 0; h >>= 1) {
        if (t < h)
#pragma unroll
            for (int j = 0; j < 6; ++j) red[j][t] += red[j][t + h];
        __syncthreads();
    }
    if (t < 6) part[((int64_t)seg * n_tiles + tile) * 6 + t] = red[t][0];
}

// one warp per segment: tile partials in order, then |r| of the ranks
__global__ void __launch_bounds__(256) spearman_final_kernel(
    const double *part, int n_seg, int n_tiles, const uint32_t *nan_flag, float *out,
    double *out64) {
    const int lane = threadIdx.x & 31;
    const int seg = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (seg >= n_seg) return;
    double s[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = lane; i < n_tiles; i += 32)
        for (int j = 0; j < 6; ++j) s[j] += part[((int64_t)seg * n_tiles + i) * 6 + j];
    double S[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int l = 0; l < 32; ++l)
        for (int j = 0; j < 6; ++j) S[j] += __shfl_sync(0xffffffffu, s[j], l);
    if (lane != 0) return;
    const double sw = S[0];
    const double ma = S[1] / sw, mb = S[3] / sw;
    const double va = S[2] / sw - ma * ma, vb = S[4] / sw - mb * mb;
    const double cov = S[5] / sw - ma * mb;
    double f;
    if (nan_flag[seg] || !isfinite(va) || !isfinite(vb) || !isfinite(cov)) f = __longlong_as_double(0x7ff8000000000000LL);
    else if (!(va > 0.0) || !(vb > 0.0)) f = 0.0;
    else f = fabs(cov) / sqrt(va * vb);
    out[seg] = (float)f;
    if (out64) out64[seg] = f;
}

cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *keys2, uint32_t *vals2,
                             int n_seg, int64_t n, int32_t *hist, cudaStream_t st) {
    const int n_tiles = (int)((n + kTile - 1) / kTile);
    const dim3 grid(n_tiles, n_seg);
    for (int pass = 0; pass < 32 / kRadixBits; ++pass) {
        const int shift = pass * kRadixBits;
        const uint32_t *ki = (pass & 1) ? keys2 : keys;
        const uint32_t *vi = (pass & 1) ? vals2 : vals;
        uint32_t *ko = (pass & 1) ? keys : keys2;
        uint32_t *vo = (pass & 1) ? vals : vals2;
        hist_kernel<<<grid, kTileThreads, 0, st>>>(ki, n, n_tiles, shift, hist);
        scan_kernel<<<n_seg, 1024, 0, st>>>(hist, n_tiles);
        scatter_kernel<<<grid, kTileThreads, 0, st>>>(ki, vi, n, n_tiles, shift, hist, ko, vo);
    }
    return cudaGetLastError();  // 8 passes: the result is back in keys/vals
}

}  // namespace

size_t rank_scratch_bytes(int n_seg, int64_t n) {
    const int64_t n_tiles = (n + kTile - 1) / kTile;
    auto al = [](int64_t x) { return (size_t)((x + 255) / 256 * 256); };
    return 4 * al((int64_t)n_seg * n * 4) + al((int64_t)n_seg * kDigits * n_tiles * 4) +
           al((int64_t)n_seg * n_tiles * 6 * 8) + al((int64_t)n_seg * 4);
}

cudaError_t target_ranks(const float *y, int64_t n, void *scratch, uint32_t *r2y,
                         cudaStream_t st) {
    const int64_t n_tiles = (n + kTile - 1) / kTile;
    auto al = [](int64_t x) { return (int64_t)((x + 255) / 256 * 256); };
    char *b = static_cast<char *>(scratch);
    uint32_t *keys = reinterpret_cast<uint32_t *>(b);
    uint32_t *vals = reinterpret_cast<uint32_t *>(b + al(n * 4));
    uint32_t *keys2 = reinterpret_cast<uint32_t *>(b + 2 * al(n * 4));
    uint32_t *vals2 = reinterpret_cast<uint32_t *>(b + 3 * al(n * 4));
    int32_t *hist = reinterpret_cast<int32_t *>(b + 4 * al(n * 4));
    uint32_t *nan_flag = reinterpret_cast<uint32_t *>(b + 4 * al(n * 4) + al(kDigits * n_tiles * 4));
    cudaMemsetAsync(nan_flag, 0, 4, st);
    to_keys_kernel<<<1024, 256, 0, st>>>(y, 1, n, keys, vals, nan_flag);
    cudaError_t e = radix_sort_pairs(keys, vals, keys2, vals2, 1, n, hist, st);
    if (e != cudaSuccess) return e;
    rank_kernel<<<dim3((unsigned)n_tiles, 1), kTileThreads, 0, st>>>(keys, vals, n, (int)n_tiles, 0,
                                                                      r2y, nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t spearman_batch(const float *pred, int n_seg, int64_t n, const uint32_t *r2y,
                           const float *w, void *scratch, float *out, double *out64,
                           cudaStream_t st) {
    const int64_t n_tiles = (n + kTile - 1) / kTile;
    auto al = [](int64_t x) { return (int64_t)((x + 255) / 256 * 256); };
    const int64_t arr = al((int64_t)n_seg * n * 4);
    char *b = static_cast<char *>(scratch);
    uint32_t *keys = reinterpret_cast<uint32_t *>(b);
    uint32_t *vals = reinterpret_cast<uint32_t *>(b + arr);
    uint32_t *keys2 = reinterpret_cast<uint32_t *>(b + 2 * arr);
    uint32_t *vals2 = reinterpret_cast<uint32_t *>(b + 3 * arr);
    int32_t *hist = reinterpret_cast<int32_t *>(b + 4 * arr);
    double *part = reinterpret_cast<double *>(b + 4 * arr + al((int64_t)n_seg * kDigits * n_tiles * 4));
    uint32_t *nan_flag = reinterpret_cast<uint32_t *>(
        reinterpret_cast<char *>(part) + al((int64_t)n_seg * n_tiles * 6 * 8));
    cudaMemsetAsync(nan_flag, 0, (size_t)n_seg * 4, st);
    to_keys_kernel<<<2048, 256, 0, st>>>(pred, n_seg, n, keys, vals, nan_flag);
    cudaError_t e = radix_sort_pairs(keys, vals, keys2, vals2, n_seg, n, hist, st);
    if (e != cudaSuccess) return e;
    rank_kernel<<<dim3((unsigned)n_tiles, n_seg), kTileThreads, 0, st>>>(
        keys, vals, n, (int)n_tiles, 1, nullptr, r2y, w, part);
    spearman_final_kernel<<<(n_seg + 7) / 8, 256, 0, st>>>(part, n_seg, (int)n_tiles, nan_flag, out,
                                                           out64);
    return cudaGetLastError();
}

}  // namespace gpk
